// kernels.h — argument blocks and launchers of the LaueOT kernels.
#pragma once

#include <cuda_runtime.h>

namespace laue {

struct GeomDev {
    float e[3];
    float lam_min, lam_max, D;
    int n_det;
    float ctr[4][3], nrm[4][3], half[4];
    float Dd[4];                // cost length of each detector (D where none is set)
    float ax1[4][3], ax2[4][3];  // in-plane axes of each detector
};

// ----------------------------------------------------------------- forward
struct FwdArgs {
    GeomDev G;
    const float* R;
    const float* x;
    const float* omega;
    const float4* w_d0;
    const int* nharm;
    int N, M, T;
    long long n_rays;
    int n_blocks;
    int capacity;
    int* blocks;  // 2 * n_blocks: counts then exclusive offsets
    int* ctrl;
    int* J_off;
    int* grain;
    int* plane;
    int* angle;
    float4* ray;
    float4* center;
    float4* spot;
};

struct RefreshArgs {
    GeomDev G;
    const float* R;
    const float* x;
    const float* omega;
    const float4* w_d0;
    const int* nharm;
    int n;
    const int* grain;
    const int* plane;
    const int* angle;
    float4* ray;
    float4* center;
    float4* spot;
};

cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s);
cudaError_t launch_refresh(const RefreshArgs& a, cudaStream_t s);

// ---------------------------------------------------------------- Sinkhorn
// Potentials are kept internally in base-2 units scaled by the temperature:
// F_i = f_i log2(e) / eps, G_j = g_j log2(e) / eps.
struct SkArgs {
    int T;
    int n_obs, n_model;
    const int* I_off;
    const int* J_off;
    const float4* obs_p;   // caller's observed spots (p, unused)
    const float4* mod_c;   // caller's centres (c, unused)
    const float4* mod_r;   // caller's rays (r, lambda)
    const float4* mod_s;   // caller's model spots (s, detector index)
    // workspace, pair-interleaved (angle blocks padded to even counts):
    float4* obsX;          // {px_a, px_b, py_a, py_b}
    float4* obsY;          // {pz_a, pz_b, F_a, F_b}
    float4* modX;          // {-cx_a, -cx_b, -cy_a, -cy_b}
    float4* modY;          // {-cz_a, -cz_b, G_a, G_b}
    float4* modZ;          // {-rx_a, -rx_b, -ry_a, -ry_b}
    float4* modW;          // {-rz_a, -rz_b, -K_a, -K_b}: K_j = D_j^2 log2(e) / eps of the spot's detector
    int* I2_off;           // T+1 pair offsets of the observed blocks
    int* J2_off;           // T+1 pair offsets of the model blocks
    // spatial order: within each angle block the spots are packed sorted by the
    // direction of p (observed) or r (model); perm maps an ordered slot (global
    // index, block offset + rank) to the caller's index, pos a caller index to
    // its rank within the block
    int *obs_perm, *obs_pos, *mod_perm, *mod_pos;
    unsigned* sort_key;    // 2 (n_obs + n_model) keys (ping-pong)
    int* sort_idx;         // 2 (n_obs + n_model) indices
    // cones of the granules (kGran pairs of one block) for the exact skipping
    float4 *obs_cone, *mod_cone;
    float *obs_ext, *mod_ext;
    int *obs_gbase, *mod_gbase;  // T+1 first granule of each block
    int skip;              // skip (tile, chunk) pairs whose plan entries all underflow
    int4* row_tiles;
    int4* col_tiles;
    int4* ang_tiles;       // per angle: {first row tile, #row tiles, first col tile, #col tiles}
    float2* row_part;
    float2* col_part;
    float* dust;           // F0, F0n, G0, log2U, log2O (T each), errors
    int* ctrl;
    int max_row_tiles, max_col_tiles;
    int tile_rows, tile_cols;
    float negKD2;          // -D^2 log2(e) / eps
    float negK_det[4];     // -D_k^2 log2(e) / eps of each detector k
    int n_det;
    float skipK;           // smallest K_j of any spot (the cone bounds take it)
    float kc;              // c_out log2(e) / eps
    double frac;           // unmatched-model fraction
    float to_user;         // eps ln 2: internal -> mm^2
    int mode;              // 0 global dustbins, 1 per angle, 2 unbalanced (no dustbins)
    int warm;
    float tau_row, tau_col;  // unbalanced exponents kappa/(kappa+eps), lambda/(lambda+eps)
    // user buffers
    float* f;
    float* g;
    float* dust_out;
    int* assign;
    float* margin;
    float* marg_err;
    float* q;
};

// ------------------------------------------------------- sparse Sinkhorn
// E-step restricted to the rho nearest observed spots of each model spot
// (sparse.cu).  Potentials in base 2 as for SkArgs, indexed by the caller's
// spot order.
struct SpArgs {
    int T;
    int n_obs, n_model;
    int rho;
    const int* I_off;
    const int* J_off;
    const float4* p;       // observed spots (p, unused)
    const float4* c;       // model centres (c, unused)
    const float4* r;       // model rays (r, lambda)
    const float4* s;       // model spots (s, detector index)
    float kdet[4];         // (D_k / D)^2 of each detector k
    int n_det;
    // workspace
    int2* cent;            // n_model x rho: {observed index or -1, e2 (D_j / D)^2 bits}, by increasing e2
    int2* rent;            // CSR rows: {model index, e2 bits}, ascending model index
    int* rptr;             // n_obs + 1 row starts
    int* rfill;            // n_obs fill counters
    float* F;              // n_obs
    float* G;              // n_model
    float* dust;           // F0, F0n, G0, log2U, log2O (nd each), errors (4)
    float2* rpart;         // per row tile: LSE of F_i - kc
    float2* cpart;         // per column tile: LSE of G_j
    int4* rtile;           // {angle, first row, end row, 0}
    int4* ctile;           // {angle, first column, end column, 0}
    int* rt_base;          // T + 1 first row tile of each angle (entry T = row tile count)
    int* ct_base;          // T + 1
    float* gmax;           // T: largest G of each angle block (shift of the row pass)
    float* fmax;           // T: largest F of each angle block (shift of the column pass)
    int max_rt, max_ct;
    int* ctrl;
    float negK;            // -D^2 log2(e) / eps
    float kc;              // c_out log2(e) / eps
    double frac;
    float to_user;
    int mode;              // 0 global dustbins, 1 per angle
    int warm;
    // user buffers
    float* f;
    float* g;
    float* dust_out;
    int* assign;
    float* margin;
    float* marg_err;
    float* q;
    int* nbr_out;          // optional n_model x rho neighbour lists
};

constexpr int kSparseMaxRho = 64;  // neighbour lists live in shared memory while they are built
size_t sparse_workspace_bytes(int T, int n_obs, int n_model, int rho);
void sparse_carve(SpArgs& a, char* base, int T, int n_obs, int n_model, int rho);
cudaError_t sparse_sinkhorn_run(const SpArgs& a, int n_iter, bool rows, bool cols, cudaStream_t s);

constexpr int kSkVariants = 4;       // launch shapes of the pair passes (see sinkhorn.cu)
constexpr int kSkDefaultVariant = 3;  // 64-pair tiles: the autotuner's usual pick

struct SkLaunch {
    int row_grid, col_grid, hrv_grid, hcol_grid;
    int row_variant, col_variant;
};

cudaError_t sinkhorn_run(const SkArgs& a, const SkLaunch& l, int n_iter, bool want_rows, bool want_cols,
                         cudaStream_t s);
cudaError_t sinkhorn_prepare(const SkArgs& a, cudaStream_t s);
cudaError_t sinkhorn_iterate(const SkArgs& a, const SkLaunch& l, int n_iter, cudaStream_t s);
cudaError_t sinkhorn_finish(const SkArgs& a, const SkLaunch& l, bool want_rows, bool want_cols, cudaStream_t s);
int sinkhorn_occupancy(int* row_blocks_per_sm, int* col_blocks_per_sm);  // kSkVariants entries each
int sk_variant_threads(int v);
void sinkhorn_row_pass(const SkArgs& a, const SkLaunch& l, cudaStream_t s);
void sinkhorn_col_pass(const SkArgs& a, const SkLaunch& l, cudaStream_t s);

// ------------------------------------------------------------------ M-step
struct MsArgs {
    SkArgs sk;              // layout, tiles and pair-interleaved copies (F, G of the E-step)
    const float4* w_d0;     // plane directions (M)
    int M;
    const float* omega;
    int T, N, n_model;
    const int* J_off;
    const int* grain;
    const int* plane;
    const int* angle;
    float* R;               // N x 9, in/out
    float* x;               // N x 3, in/out
    float* jsum;            // 12 floats per model spot
    int* seg;               // T x (N + 1) segment starts
    float* gstate;          // 4 floats per grain
    float* step_norms;      // optional N x 2
    float tol_x, tol_R, hreg;
    int n_newton, n_mm;
    float e[3];
    float D2;               // D^2
    float D2det[4];         // D_k^2 of each detector (the cost length of its spots)
    float* grad;            // N x 6 (adjoint)
    float* value;           // N (adjoint, optional)
};

cudaError_t mstep_run(const MsArgs& m, const SkLaunch& l, cudaStream_t s);
cudaError_t mstep_adjoint_run(const MsArgs& m, const SkLaunch& l, int n_steps, cudaStream_t s);

// ------------------------------------------------------- single-grain fits
constexpr int kSfMaxT = 1024;       // angles a fit supports

struct SfArgs {
    GeomDev G;
    const float4* w_d0;
    const int* nharm;
    int M;
    const float* omega;
    int T;
    const int* I_off;
    const float4* p;
    const float* R0;
    const float* x0;
    int S;
    float* R_out;
    float* x_out;
    int* keep;
    float* unmatched;
    float eps_final, c_out, f_out, tol_x, tol_R, hreg;
    int k_max, n_newton, n_mm;
    float anneal;  // eps_init / eps_final
    int recut;     // re-list the visible spots at every step
    float* scratch;
    int cap, icap;
    int ncap;      // near-row list capacity per CTA (sf_near_cap of the workspace's n_obs)
    int* queue;  // 2 ints: start queue head, completion ticket
    int* ctrl;
};

// SPOT prototype selection
struct SpotArgs {
    float eps_s;
    int* count;          // Nc
    int* row_ptr;        // Nc + 1
    int* col;            // nnz observed indices
    float* val;          // nnz values
    long long* nnz_total;
    float* best;         // n_obs: max_{n in S} Lbar_in
    int* chosen;         // Nc
    float* part_g;       // per-block partial argmax
    int* part_i;
    int* tick;
    int* cur;
    int* order;          // k_max
    float* gains;        // k_max
    int* kstar;
};

cudaError_t spot_matrix_run(const SfArgs& a, const SpotArgs& sp, int ctas, bool count_only, cudaStream_t s);
cudaError_t spot_greedy_run(const SpotArgs& sp, int n_obs, int Nc, int k_max, int sm_count, cudaStream_t s);
cudaError_t single_fit_run(const SfArgs& a, int ctas, cudaStream_t s);
cudaError_t grad_run(const MsArgs& m, const SkLaunch& l, cudaStream_t s);
cudaError_t axis_angle_run(const float* w, const float* R0, float* R, float* JlT, int N, cudaStream_t s);
cudaError_t axis_angle_vjp_run(const float* w, const float* grad, const float* gout, float* gw, float* gx, int N,
                               cudaStream_t s);

}  // namespace laue
