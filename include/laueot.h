/*
 * laueot.h — C ABI of the GB300 (sm_103a) implementation of the LaueOT
 * Sinkhorn-EM indexing hot path (Laue indexing with Optimal Transport,
 * arXiv 2404.06478).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Return value: LAUE_OK (0) on success, a negative LAUE_ERR_* code on
 *    failure, LAUE_WARN_* (> 0) when results are valid but a warning applies.
 *    laue_last_error() gives a message for the last failure on the handle.
 *  - Ownership: the caller owns every buffer.  Array arguments are DEVICE
 *    pointers unless the name ends in _host.  The library never allocates
 *    device memory: scratch space comes from the caller's workspace
 *    (laue_workspace_size / laue_set_workspace).
 *  - Streams: `stream` is a cudaStream_t passed as void*.  Calls are
 *    asynchronous on it, except where a function is documented to return a
 *    host-side count (it then synchronises that stream).  No entry point
 *    synchronises the device.
 *  - Device-side failures (a bounded wait that ran out, a non-finite
 *    potential) are recorded in a status word inside the workspace; read and
 *    clear it with laue_device_status().
 *  - Spot lists are structure-of-arrays sorted by rotation angle t, with
 *    offsets *_off[T+1] (int32, device): the spots of angle t are
 *    [off[t], off[t+1]).  Vector data are packed as 4 floats per spot
 *    (16-byte aligned rows) so that kernels read them as float4.
 *  - Units: lengths in mm, wavelengths in Angstrom, angles in radians,
 *    costs, potentials and the temperature eps in mm^2.
 *  - One handle per host thread.
 *
 * Frame (paper Section "Laue analysis", read in a beam-along-z frame): beam
 * direction e; the sample rotation Gamma_t is a right-handed rotation about
 * +y by omega_t; detectors are planes with a centre gamma, a unit normal nu
 * and a half side l/2.
 */
#ifndef LAUEOT_H
#define LAUEOT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ----------------------------------------------------- */
#define LAUE_OK 0
#define LAUE_WARN_NOT_CONVERGED 1
#define LAUE_ERR_INVALID_ARG (-1)
#define LAUE_ERR_CAPACITY (-2)
#define LAUE_ERR_CUDA (-3)
#define LAUE_ERR_NUMERIC (-4)
#define LAUE_ERR_TIMEOUT (-5)
#define LAUE_ERR_UNIMPLEMENTED (-6)
#define LAUE_ERR_WORKSPACE (-7)

typedef struct laue_handle laue_handle;

/* ---- problem description ---------------------------------------------- */

/* Experiment geometry (host struct, copied at each call).  Paper Section
 * "Laue diffraction" (Eq. spot_position) and "Detected spots": beam e,
 * wavelength band [lam_min, lam_max], detectors (gamma, nu, l).  D is the
 * length that turns ray distances into the pair cost C = D^2 |rhat - r|^2
 * (the sample-detector distance).  Detector k is the plane through
 * det_centre[k] with normal det_normal[k] (any orientation); it holds the
 * plane points s with |(s - centre).a| < det_half[k] for both in-plane axes
 * a1 = (y x n)/|y x n| (x when n is along y) and a2 = n x a1, n the unit
 * normal (for a plane normal to z: the square with edges along x and y).
 * det_D[k] > 0 is the cost length of the spots on detector k (the paper's
 * two-detector setups, Appendix "Experimental details", place the detectors
 * at different distances): the pair cost of model spot j is then
 * D_j^2 |rhat - r_j|^2 with D_j = det_D of the detector its ray hits, and D
 * where det_D[k] <= 0. */
typedef struct {
    float beam[3];
    float lam_min, lam_max;
    float D;
    int n_det; /* 1..4 */
    float det_centre[4][3];
    float det_normal[4][3];
    float det_half[4];
    float det_D[4];
} LaueGeometry;

/* Plausible plane set (paper Section "Tomography experiments": the set
 * {(w_m, d_m)} is an input).  One entry per ray direction: w_d0[4m..4m+2] is
 * the unit crystal direction w_m, w_d0[4m+3] the spacing d0 of its base
 * reflection g0, nharm[m] the number of allowed harmonics n*g0 (n = 1..nharm),
 * which share the ray.  Device arrays. */
typedef struct {
    const float* w_d0; /* M x 4 */
    const int* nharm;  /* M */
    int M;
} LaueLattice;

/* Detected spots {p_i, t_i} (paper Section "Detected spots"), sorted by t. */
typedef struct {
    int T;
    int n;
    const int* I_off; /* T+1 */
    const float* p;   /* n x 4: x, y, z, (unused) */
} LaueObsSpots;

/* Model spots S (Eq. model_spot_cut) with labels t_j, n_j, m_j, sorted by t
 * then grain then plane.  Written by laue_forward, rays and centres
 * rewritten in place by laue_refresh. */
typedef struct {
    int T;
    int n;        /* number of spots in the list */
    int capacity; /* rows allocated in every array below */
    int* J_off;   /* T+1 */
    int* grain;   /* n_j */
    int* plane;   /* m_j */
    int* angle;   /* t_j */
    float* ray;    /* n x 4: r_j (unit), lambda_j */
    float* center; /* n x 4: c_j = Gamma_t x_n, (unused) */
    float* spot;   /* n x 4: s_j, detector index (as float) */
} LaueModelSpots;

/* E-step parameters (paper Section "E-step with Sinkhorn updates" and
 * Algorithm BalancedOT).  The extended plan has observed rows plus an
 * unmatched-model row of mass U = ceil(unmatched_frac |J|), model columns
 * plus an outlier column of mass O = U + |I| - |J| (when O < 0, U = |J| - |I|
 * and O = 0).  Costs: C_ij pair cost, C_i0 = c_out, C_0j = 0, C_00 = c_out.
 * dust_mode 0: one dustbin row/column for all angles; 1: one per angle
 * (masses computed per angle block); 2: unbalanced OT (Appendix "Optimal
 * transport variants", Problem (B), Algorithm UnbalancedOT): no dustbins, the
 * marginals relaxed by generalised KL terms of weights kappa (observed rows)
 * and lambda (model columns), i.e. each log-domain update of f (g) is the
 * balanced one scaled by kappa / (kappa + eps) (lambda / (lambda + eps)).  In
 * that mode c_out and unmatched_frac are unused, dust is not written, and the
 * hard assignment of a row whose plan mass is below 1/2 is -1. */
typedef struct {
    double unmatched_frac;
    float eps;
    float c_out;
    int n_iter;
    int dust_mode;
    int warm_start; /* nonzero: f, g, dust hold the starting potentials */
    float kappa;    /* dust_mode 2: weight of the observed-row marginal KL term (mm^2) */
    float lambda;   /* dust_mode 2: weight of the model-column marginal KL term (mm^2) */
    int pad_;
} LaueOTParams;

/* M-step parameters (paper Section "The M-step updates", Algorithms
 * LauePosNewton and LaueRotMM). */
typedef struct {
    float eps;      /* temperature of the E-step whose potentials are given */
    int n_newton;   /* Newton steps on x (4 in the paper's single-grain fits) */
    int n_mm;       /* MM steps on R */
    float tol_x;    /* stop Newton when |dx| < tol_x (mm) */
    float tol_R;    /* stop MM when |dR|_F < tol_R */
    float hreg;     /* Hessian shift: iota = max(0, lmax(H) + hreg |H|_F) */
} LaueMParams;

/* Annealed multi-grain EM (paper Algorithm LaueOT; Section "Deterministic
 * annealing") for laue_em: steps k = k_first .. k_last of an n_em-step
 * schedule eps_k = eps_final anneal^(1 - k/K), K = ceil(0.75 n_em), eps_k =
 * eps_final for k >= K. */
typedef struct {
    double unmatched_frac;
    float eps_final;
    float c_out;
    float anneal;      /* eps_0 / eps_final; <= 0 means 100 */
    int n_em;
    int n_sinkhorn;    /* Sinkhorn iterations of each E-step (from f = g = 0) */
    int dust_mode;     /* 0 global, 1 per-angle dustbins */
    int mstep_kind;    /* 0 Newton + MM (laue_mstep), 1 adjoint (laue_mstep_adjoint:
                          mstep.n_newton damped Gauss-Newton steps, mstep.hreg the damping) */
    int k_first, k_last;
    LaueMParams mstep; /* eps is set per step */
} LaueEMParams;

/* Sizes that bound a problem, for laue_workspace_size. */
typedef struct {
    int T;
    int n_obs;
    int n_model;
    int n_grains;
    int n_planes;
    int n_starts;     /* nonzero when laue_single_fit will run */
    int n_candidates; /* candidates of laue_prototype_select (its sparse matrix
                         uses the workspace beyond laue_workspace_size) */
} LaueProblemDims;

/* Single-grain fit parameters (paper Appendix "Single-grain fitting",
 * Algorithm SingleLaueOT; filter f_out of Section "Selection of Prototypes
 * with Optimal Transport"). */
typedef struct {
    float eps_final; /* final temperature */
    float c_out;
    float f_out;     /* keep a fit when #unmatched rays < f_out |J| */
    int k_max;       /* annealed EM steps per start */
    LaueMParams mstep;
    float anneal;    /* eps starts at anneal * eps_final (laue_anneal_eps); <= 0 means 100 */
    int recut;       /* nonzero: list the visible spots again at the pose of every step */
} LaueSingleParams;

/* ---- handle and workspace --------------------------------------------- */

/* Creates a handle bound to CUDA device `device`.  Allocates host memory
 * only.  Errors: LAUE_ERR_INVALID_ARG (null pointer), LAUE_ERR_CUDA (bad
 * device). */
int laue_create(laue_handle** h, int device);
int laue_destroy(laue_handle* h);
const char* laue_last_error(const laue_handle* h);

/* Workspace bytes needed for problems bounded by *dims. */
int laue_workspace_size(laue_handle* h, const LaueProblemDims* dims, size_t* bytes);

/* Hands the library a device buffer of `bytes` bytes (256-byte aligned) to
 * use as scratch; it must stay valid while calls that use it are in flight.
 * The first 256 bytes hold the device status word and must be zeroed by
 * this call's stream order before first use: laue_set_workspace enqueues that
 * clear on `stream`. */
int laue_set_workspace(laue_handle* h, void* dev_ptr, size_t bytes, void* stream);

/* Synchronises `stream`, returns the device status word (LAUE_OK or a
 * LAUE_ERR_* code recorded by a kernel) in *status_host and clears it. */
int laue_device_status(laue_handle* h, void* stream, int* status_host);

/* Measurement helper (no counterpart in the paper): throughput of the
 * arithmetic pipes the pair passes use, measured on this device by
 * microbenchmark kernels.  out_host[0..5] = FP32 FMA ops/s, packed f32x2 FMA
 * ops/s (2 per instruction), MUFU ex2/s, MUFU rsqrt/s, MUFU lg2/s, SM count.
 * Synchronises `stream`.  Needs the workspace. */
int laue_alu_peaks(laue_handle* h, double* out_host, void* stream);

/* ---- host helper ------------------------------------------------------- */

/* Plausible plane set of a cubic lattice (paper Section "Crystallographic
 * planes": d = a / |hkl|): every hkl with max(|h|,|k|,|l|) <= hmax allowed by
 * the centering (0 = P, 1 = I: h+k+l even, 2 = F: h,k,l unmixed), one entry per
 * ray direction (Friedel pairs and harmonics merged), ordered by |g0|^2
 * ascending then g0 descending.  Host arrays: w_d0_host (cap x 4),
 * nharm_host (cap), hkl0_host (cap x 3, may be NULL).  *M = number of entries;
 * LAUE_ERR_CAPACITY if *M > cap (nothing beyond cap written). */
int laue_reflections(double a, int hmax, int centering, int cap, float* w_d0_host,
                     int* nharm_host, int* hkl0_host, int* M);

/* Outlier cost c_out of the extended cost matrix (paper Eq. update_L: the
 * likelihood of a pair at 3 sigma, Section "Simulations and experiments"):
 * the pair cost of two unit rays 3 sigma_mm / D apart,
 * D^2 |a - b|^2 = 4 D^2 sin^2(1.5 sigma_mm / D), in mm^2.  Host function;
 * returns -1 when sigma_mm <= 0 or D <= 0. */
double laue_c_out(double sigma_mm, double D);

/* Temperature of annealed step k (paper Section "Deterministic annealing"):
 * eps_k = eps_final factor^(1 - k/K) for 0 <= k < K = ceil(0.75 n_em), then
 * eps_final (also when K < 1).  The one schedule of the library: laue_index,
 * laue_single_fit (factor 100, n_em = k_max) and the binding's EM driver all
 * use it.  Host function; returns -1 for eps_final <= 0, n_em < 0, k < 0 or
 * factor <= 0. */
double laue_anneal_eps(double eps_final, int n_em, int k, double factor);

/* Reciprocal basis of a lattice with cell edges a, b, c (Angstrom) and angles
 * alpha, beta, gamma (degrees; paper Section "Crystallographic planes": the
 * reciprocal vectors g = B hkl, d = 1 / |g|).  Convention: the direct basis has
 * a1 along x, a2 in the xy plane at gamma from a1, a3 completing the cell;
 * B_host (3 x 3, row-major) holds b1, b2, b3 as columns with a_i . b_j =
 * delta_ij (no 2 pi).  A grain's R maps this crystal frame to the sample
 * frame.  Host function.  LAUE_ERR_INVALID_ARG for a non-positive edge or
 * angles that do not close a cell. */
int laue_reciprocal_basis(double a, double b, double c, double alpha_deg, double beta_deg, double gamma_deg,
                          double* B_host);

/* Plausible plane set of any lattice (the paper takes the set {(w_m, d_m)} as
 * an input, Section "Tomography experiments"): from the reciprocal basis
 * B_host (3 x 3 row-major, laue_reciprocal_basis) and a host list of the n
 * allowed reflections hkl_host (n x 3, e.g. every hkl within a bound that the
 * space group's reflection conditions allow; order and Friedel mates free).
 * Reflections on one line through the origin share a ray, so there is one
 * entry per line: its multiples in the list must be m0, 2 m0, ..., nh m0 of
 * the line's primitive vector p (first nonzero index positive); the entry's
 * base reflection is g0 = m0 p, w = B g0 / |B g0|, d0 = 1 / |B g0|, nharm = nh.
 * Order: |B g0|^2 ascending (equal within 1e-9 relative), then g0
 * descending.  Outputs as laue_reflections (w_d0_host cap x 4, nharm_host cap,
 * hkl0_host cap x 3, may be NULL); LAUE_ERR_CAPACITY if *M > cap,
 * LAUE_ERR_INVALID_ARG when a line's multiples are not of that form. */
int laue_reflections_hkl(const double* B_host, const int* hkl_host, int n, int cap, float* w_d0_host,
                         int* nharm_host, int* hkl0_host, int* M);

/* ---- hot path ---------------------------------------------------------- */

/* Forward Laue model and cut (paper Eqs. ray_mnt, s_mnt, wavelength,
 * model_spot_cut): for every (t, n, m), u = Gamma_t R_n w_m,
 * r = e - 2 (u.e) u, lambda = 2 d0 |u.e| / n for the smallest harmonic n with
 * lambda in band, spot s = c + tau r on the detector with the smallest
 * tau > 0 whose square contains it, c = Gamma_t x_n.  Visible spots are
 * written to *out sorted by (t, n, m) (deterministic).
 * R: N x 9 row-major (crystal -> sample), x: N x 3, omega: T (device).
 * *total_host receives the number of visible spots; this call synchronises
 * `stream` to read it.  LAUE_ERR_CAPACITY if it exceeds out->capacity (then
 * only J_off and the first capacity rows are valid).  Needs the workspace. */
int laue_forward(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                 const float* R, const float* x, int N, const float* omega, int T,
                 LaueModelSpots* out, int* total_host, void* stream);

/* Rays, centres, wavelengths and spot positions of a frozen model-spot list
 * at new poses (the list stays the one of the prototypes, paper Section
 * "Assignments with outlier and missing spots").  Asynchronous. */
int laue_refresh(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                 const float* R, const float* x, const float* omega,
                 LaueModelSpots* model, void* stream);

/* Fused pair cost + log-domain balanced Sinkhorn (paper Eqs. update_L,
 * estep_obj, Algorithm BalancedOT), blocked by angle, never materialising the
 * cost matrix: C_ij = D^2 |rhat_ij - r_j|^2, rhat_ij = (p_i - c_j)/|p_i - c_j|.
 * Starts at f = g = 0 unless warm_start, runs the row update first, n_iter
 * iterations.  Outputs (device):
 *   f (obs->n) and g (model->n) potentials, dust: [f_0 | g_0] (2 floats in
 *   global mode, 2T in per-angle mode: T row values then T column values),
 *   assign (obs->n, optional): argmax of plan row i over the block's model
 *   spots and the outlier column (-1); ties to the lowest index,
 *   margin (optional): top1 - top2 of the row's plan entries,
 *   marg_err (optional, 2 floats): largest row and column marginal error,
 *   q (optional, model->n): column mass sum_i Q_ij over observed rows.
 * Asynchronous.  Non-finite potentials set LAUE_ERR_NUMERIC in the device
 * status word. */
int laue_cost_sinkhorn(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs,
                       const LaueModelSpots* model, const LaueOTParams* prm, float* f, float* g,
                       float* dust, int* assign, float* margin, float* marg_err, float* q,
                       void* stream);

/* The same E-step as laue_cost_sinkhorn (same arguments and outputs, no
 * handle) for callers that cannot allocate device memory: code that runs
 * while a stream is being captured into a CUDA graph, where an allocation
 * would break or synchronise the capture; hard real-time loops, where the
 * implicit device synchronisation of cudaMalloc stalls the pipeline; plugins
 * hosted by a framework that owns every device allocation.  This entry point
 * has no counterpart in the paper.
 *
 * Scratch: a fixed 64 MiB array in device memory owned by this library
 * module, reserved on every GPU where the module is loaded and held there
 * until the process exits; the call allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  It fits problems whose E-step
 * layout (laue_workspace_size with only T, n_obs, n_model set, up to the
 * E-step regions) is at most 64 MiB, about 1.5 million observed plus 1 million
 * model spots; larger problems return LAUE_ERR_CAPACITY before any launch.
 * The first call on a device looks the array's device address up (with that
 * device current) and caches it: make that first call before any stream
 * capture begins.  Every call on a device shares the one array, which keeps
 * the previous call's contents (the call clears its counters and status word
 * itself): calls whose work overlaps on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  Runs on the current
 * device; `stream` must belong to it.  status (optional, one device int)
 * receives the device status word (LAUE_OK or a LAUE_ERR_* code) in stream
 * order.  Asynchronous. */
int laue_cost_sinkhorn_noalloc(const LaueGeometry* geom, const LaueObsSpots* obs,
                               const LaueModelSpots* model, const LaueOTParams* prm, float* f,
                               float* g, float* dust, int* assign, float* margin, float* marg_err,
                               float* q, int* status, void* stream);

/* Autotuner of the pair passes (no counterpart in the paper): times each
 * launch shape of the row and column passes of laue_cost_sinkhorn on this
 * problem (shape v: {256, 128, 128 with a 128-register cap, 64 with a
 * 128-register cap} threads per CTA, one row/column pair per thread; the tile
 * size follows the CTA width), n_iter passes each after one warm-up
 * iteration, and keeps the fastest row and column shapes in the handle for
 * later calls.  choice_host (optional, 2 ints): the chosen row and column
 * shapes; ms_host (optional, 2 x 4 floats): mean milliseconds per row and
 * column pass of each shape.  Needs the workspace of laue_cost_sinkhorn plus
 * 4 (n_obs + n_model + 2T + 8) bytes.  Synchronises `stream`. */
int laue_autotune(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs,
                  const LaueModelSpots* model, const LaueOTParams* prm, int n_iter, int* choice_host,
                  float* ms_host, void* stream);

/* Device counters (no counterpart in the paper), accumulated since the last
 * call on the handle's workspace, then cleared; the first n (<= 5) go to
 * counts_host: [0] row and [1] column log-sum-exps of laue_cost_sinkhorn's pair
 * passes recomputed on the exact (running-maximum) path because their fast
 * sum, shifted by the angle block's largest potential, fell below 1e-30
 * (modulo 2^32); [2] pair evaluations (one cost and one exponential each) of
 * laue_single_fit; [3] pair evaluations of the row and column passes of
 * laue_cost_sinkhorn (after the exact skipping); [4] pairs the M-step pair
 * passes of laue_mstep, laue_mstep_adjoint and laue_objective_grad visit
 * (after the exact skipping).  Synchronises `stream`. */
int laue_read_counters(laue_handle* h, void* stream, long long* counts_host, int n);

/* Exact underflow skipping in the Sinkhorn pair passes (no counterpart in the
 * paper; on by default): within each angle block the spots are ordered by
 * direction, each run of 32 pairs (a quarter of a staged chunk of 128)
 * carries a cone bounding its directions, and a pass skips a (tile, granule)
 * combination when the cones prove that every shifted exponent is below
 * -130, i.e. every plan entry flushes to exactly 0; the potentials are
 * bit-identical either way.  The M-step pair passes skip, by the same cone
 * bounds, the granules whose every plan entry is below 2^-40 (entries their
 * sums leave out), so their results are bit-identical too.  enable = 0 turns
 * the skipping off (the ordering stays).  Read the evaluated pairs with
 * laue_read_counters. */
int laue_set_pair_skipping(laue_handle* h, int enable);

/* Sparse E-step (paper Section "Working with sparse assignment matrices":
 * only the rho nearest neighbours of each spot carry assignment weight).
 * Support: each model spot j keeps N(j), the rho observed spots of its angle
 * block with the smallest pair cost C_ij (fewer when the block has fewer;
 * ties to the lower observed index, costs compared in float); every other
 * observed-model entry of the plan is 0, the outlier column and the
 * unmatched-model row stay dense.  Then Algorithm BalancedOT as in
 * laue_cost_sinkhorn restricted to that support:
 *   f_i = -eps LSE({(g_j - C_ij)/eps : i in N(j)} u {(g_0 - c_out)/eps})
 *   g_j = -eps LSE({(f_i - C_ij)/eps : i in N(j)} u {f_0/eps})
 * with the dustbin updates of laue_cost_sinkhorn, row update first, n_iter
 * iterations.  Arguments and outputs as for laue_cost_sinkhorn (assign and
 * margin over the row's support and the outlier column; q over the column's
 * support); dust_mode 0 or 1 (the unbalanced mode is not offered here);
 * rho 1..64.  nbr (optional, device, model->n x rho ints): N(j) in order of
 * increasing cost, -1 past its end.  Needs a workspace of
 * laue_sparse_workspace_size bytes (16 rho |J| + 16 (|I| + |J|) bytes plus
 * small tables).  Asynchronous. */
int laue_sparse_workspace_size(int T, int n_obs, int n_model, int rho, size_t* bytes);
int laue_cost_sinkhorn_sparse(laue_handle* h, const LaueGeometry* geom, const LaueObsSpots* obs,
                              const LaueModelSpots* model, const LaueOTParams* prm, int rho, float* f,
                              float* g, float* dust, int* assign, float* margin, float* marg_err, float* q,
                              int* nbr, void* stream);

/* Sets the launch shapes (0..3, as for laue_autotune) of the row and column
 * passes used by later calls on the handle; shape 3 is the default. */
int laue_set_launch_shape(laue_handle* h, int row_shape, int col_shape);

/* M-step (paper Section "The M-step updates", Appendix "M-steps"): with the
 * plan Q_ij = exp((f_i + g_j - C_ij)/eps) of the E-step (costs from the
 * model list's current rays and centres, which must be those of the E-step),
 * per grain n_newton Newton steps on x_n (exact gradient and Hessian of
 * sum Q rhat.r), then n_mm MM steps on R_n (Eqs. M0, Mm, majmin_step; Wahba by
 * the 4x4 quaternion eigenproblem).  R (N x 9) and x (N x 3) are updated in
 * place.  step_norms (optional, N x 2): last |dx| and |dR|_F.  Asynchronous. */
int laue_mstep(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
               const LaueObsSpots* obs, const LaueModelSpots* model, const float* f,
               const float* g, const LaueMParams* prm, const float* omega, float* R, float* x,
               int N, float* step_norms, void* stream);

/* Adjoint M-step (an addition beside Section "The M-step updates"; the paper's
 * M-step is laue_mstep): per grain, prm->n_newton Levenberg-Marquardt steps on
 * the OT-weighted spot cost E_n = sum_{j in J_n} sum_i Q_ij C_ij(R_n, x_n),
 * the plan Q held at the E-step (potentials f, g and the model list's rays and
 * centres, which must be those of the E-step), over theta = (phi, x) with
 * R <- exp([phi]x) R.  Each step runs the adjoint pair pass at the current
 * pose (the gradient of laue_objective_grad, costs recomputed, never stored)
 * together with the sums q_j = sum_i Q_ij, s1_j = sum_i Q_ij / tau_ij and
 * s2_j = sum_i Q_ij / tau_ij^2; the Gauss-Newton matrix takes each spot's
 * model-ray projector P_j = I - r_j r_j^T:
 *   H = 2 D^2 sum_j [[q A^T A, s1 A^T P Gamma], [s1 Gamma^T P A, s2 Gamma^T P Gamma]],
 *   A_j = dr_j/dphi = 2 (u e^T + (u.e) I) Gamma [R w_m]x,  u = Gamma R w_m;
 * delta = -(H + hreg diag(H))^-1 grad (Cholesky; a grain whose damped matrix
 * is not positive definite keeps its pose), R <- exp([delta_phi]x) R,
 * x <- x + delta_x.  prm->n_mm, tol_x and tol_R are not used.  R (N x 9),
 * x (N x 3) are updated in place; step_norms (optional, N x 2): last
 * |delta_x| and |delta_phi|.  Asynchronous. */
int laue_mstep_adjoint(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                       const LaueObsSpots* obs, const LaueModelSpots* model, const float* f,
                       const float* g, const LaueMParams* prm, const float* omega, float* R, float* x,
                       int N, float* step_norms, void* stream);

/* Gradient of the OT-weighted spot cost E_n = sum_{j in J_n} sum_i Q_ij C_ij
 * with Q held at the plan of potentials (f, g) and the current costs
 * (Danskin), with respect to a left-multiplicative axis-angle perturbation
 * R_n <- exp([w]x) R_n and to x_n: grad (N x 6) = [dE/dw, dE/dx]; value (N,
 * optional) = E_n.  Costs are recomputed, not stored.  Asynchronous. */
int laue_objective_grad(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                        const LaueObsSpots* obs, const LaueModelSpots* model, const float* f,
                        const float* g, float eps, const float* omega, const float* R,
                        const float* x, int N, float* grad, float* value, void* stream);

/* Rotation parameterisation used with laue_objective_grad (no counterpart in
 * the paper): R = exp([w]x) R0 for axis-angle w (N x 3) and base rotations R0
 * (N x 9); JlT (optional, N x 9) receives the transpose of the left Jacobian
 * of SO(3) at w, which turns the left-perturbation gradient returned by
 * laue_objective_grad at R into the gradient with respect to w.
 * Asynchronous. */
int laue_axis_angle(laue_handle* h, const float* w, const float* R0, float* R, float* JlT, int N,
                    void* stream);

/* Vector-Jacobian product for laue_objective_grad under the parameterisation
 * of laue_axis_angle (no counterpart in the paper): with grad (N x 6) =
 * [dE/dphi, dE/dx] at R = exp([w]x) R0 (phi the left perturbation),
 * gw (N x 3) = gout_n J_l(w_n)^T dE/dphi_n and gx (N x 3, optional) =
 * gout_n dE/dx_n; gout (N, optional) defaults to 1.  w: N x 3.
 * Asynchronous. */
int laue_axis_angle_vjp(laue_handle* h, const float* w, const float* grad, const float* gout, float* gw,
                        float* gx, int N, void* stream);

/* Start grid of the single-grain fits (paper Section "Single-grain fitting":
 * quasi-uniform starts over orientations and positions, the orientations
 * restricted by the crystal symmetry).  The paper's Sobol sequence over
 * modified Rodrigues parameters is read as the super-Fibonacci spiral of
 * Alexa (CVPR 2022): n_full unit quaternions q_i (s = i + 1/2,
 * q = (sqrt(s/n) sin(2 pi s/sqrt 2), sqrt(s/n) cos(2 pi s/sqrt 2),
 *      sqrt(1 - s/n) sin(2 pi s/psi), sqrt(1 - s/n) cos(2 pi s/psi)),
 * psi^4 = psi + 4).  sym = 24 keeps, in spiral order, the points of the
 * fundamental zone of the cubic group 432 (scalar part the largest |<q, g>|
 * over the group), sym = 6 of the trigonal group 32 and sym = 12 of the
 * hexagonal group 622 (n-fold axis along z, a 2-fold axis along x: the
 * frame of laue_reciprocal_basis for hexagonal cells); sym = 1 keeps every
 * point.  Each kept orientation is paired with the k^3
 * cell centres of the cube of side cube_mm centred at the origin (first
 * coordinate slowest): start s = o k^3 + p.  Writes min(S, cap) starts
 * (R_out cap x 9 row-major, x_out cap x 3; device) and *S_host = S (cap = 0
 * only counts).  Synchronises `stream`.  Needs a workspace of at least
 * 4.5 KiB + 4 (n_full / 1024 + 1) bytes.  Errors: LAUE_ERR_INVALID_ARG (sym
 * not 1, 6, 12 or 24, k outside 1..64, n_full < 0), LAUE_ERR_WORKSPACE. */
int laue_start_grid(laue_handle* h, long long n_full, int sym, int k, float cube_mm, long long cap, float* R_out,
                    float* x_out, long long* S_host, void* stream);

/* Batched single-grain fitting (paper Section "Single-grain fitting",
 * Appendix "Single-grain fitting", Eq. elbo_single, Algorithm SingleLaueOT)
 * from S starts (startR S x 9, startX S x 3): per start, the model spots
 * visible at the start pose are listed and frozen; k_max annealed EM steps
 * with the row-normalised E-step Q_ij = exp(-C_ij/eps) / (sum_j' exp(-C_ij'/eps)
 * + exp(-c_out/eps)) over the grain's spots at t_i, each followed by
 * mstep.n_newton Newton and mstep.n_mm MM steps.  Filter at the final pose: a
 * ray is unmatched when its column mass sum_i Q_ij at eps_final is < 0.5;
 * keep[s] = 1 when #unmatched < f_out |J| and |J| > 0.  Outputs (device):
 * R_out (S x 9), x_out (S x 3), keep (S, int), unmatched (S, fraction,
 * optional).  A start with more than 2048 visible spots is fitted on the first
 * 2048 only, not kept, and sets LAUE_ERR_CAPACITY in the status word.
 * Needs the workspace sized with n_starts > 0.  Asynchronous. */
int laue_single_fit(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                    const LaueObsSpots* obs, const float* omega, const float* startR,
                    const float* startX, int S, const LaueSingleParams* prm, float* R_out,
                    float* x_out, int* keep, float* unmatched, void* stream);

/* SPOT prototype selection (paper Section "Selection of Prototypes with
 * Optimal Transport", Appendix "Selection of prototypes", Eqs.
 * prototype_function, prototype_loss, spot_ngrains, Algorithm LaueSpotGreedy):
 * candidate grains (candR Nc x 9, candX Nc x 3) make their spots (same cut as
 * laue_forward); the grain-to-spot matrix, read as the gain over the outlier
 * baseline, Lbar_in = max(0, LSE_{j of n at t_i}(-C_ij/eps_s) + c_out/eps_s), is
 * built sparse by candidate; greedy facility-location selection of k_max
 * prototypes maximising f(S) = sum_i max_{n in S} Lbar_in (ties to the lowest
 * index); order (k_max, device, -1 once no candidate is left), gains (k_max,
 * device: the increments Delta_k), *k_star_host = argmax over 2 <= k <= K of
 * Delta_k - Delta_{k+1} with Delta_{K+1} = 0 (K = k_max; k* = K when K < 2).
 * The sparse matrix (8 bytes per nonzero) lives in the workspace beyond
 * laue_workspace_size (with n_candidates = Nc); *nnz_host (optional) receives
 * its nonzero count, and LAUE_ERR_CAPACITY is returned when it does not fit.
 * Synchronises `stream`. */
int laue_prototype_select(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
                          const LaueObsSpots* obs, const float* omega, const float* candR,
                          const float* candX, int Nc, float eps_s, float c_out, int k_max,
                          int* order, float* gains, int* k_star_host, long long* nnz_host,
                          void* stream);

/* End-to-end indexing (paper Algorithm LaueOT preceded by the pre-processing
 * of Section "Pre-processing"): batched single-grain fits from the S starts
 * (startR S x 9, startX S x 3), or, with startR = startX = NULL, from the
 * library's start grid (laue_start_grid with grid_n, grid_sym, grid_k,
 * grid_cube; S must then be at least the grid's start count), with k_single
 * annealed steps (from anneal_single eps_final, re-listing the visible spots
 * every step when recut_single is set) and the f_out filter
 * (laue_single_fit); SPOT selection over the kept fits at eps_final
 * with k_max = min(#kept, n_max) (laue_prototype_select); the model list of
 * the k* prototypes (laue_forward); n_em annealed EM steps (eps from
 * 100 eps_final down to eps_final at step ceil(0.75 n_em), n_sinkhorn
 * iterations each, then laue_mstep, or laue_mstep_adjoint with mstep_kind = 1)
 * and a final E-step at eps_final.
 * Outputs: R_out / x_out (capacity n_max grains), *n_grains_host = k*, and
 * assign (obs->n): the grain of each observed spot's argmax model spot, -1
 * for the outlier column.  Needs laue_index_workspace_size bytes.
 * Synchronises `stream`. */
typedef struct {
    double unmatched_frac;
    float eps_final;
    float c_out;
    float f_out;
    int n_em;
    int n_sinkhorn;
    int k_single; /* annealed steps of each single-grain fit */
    int dust_mode;
    LaueMParams mstep;
    float anneal_single; /* eps_init / eps_final of the single-grain fits (<= 0: 100) */
    int recut_single;    /* nonzero: the fits re-list visible spots every step */
    long long grid_n;    /* start grid (used when startR is NULL): spiral points */
    int grid_sym;        /* 1, 6, 12 or 24: the rotation group whose fundamental zone the grid covers */
    int grid_k;          /* k^3 positions per orientation */
    float grid_cube;     /* side of the sample cube (mm) */
    int mstep_kind;      /* 0: laue_mstep (Newton on x, MM on R); 1: laue_mstep_adjoint */
} LaueIndexParams;

int laue_index_workspace_size(laue_handle* h, int T, int n_obs, int S, int n_max, int n_planes,
                              size_t* bytes);

int laue_index(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat,
               const LaueObsSpots* obs, const float* omega, const float* startR,
               const float* startX, int S, const LaueIndexParams* prm, float* R_out,
               float* x_out, int n_max, int* n_grains_host, int* assign, void* stream);

/* Multi-grain EM on a frozen model-spot list (paper Algorithm LaueOT): for
 * each step k = k_first .. k_last (0 <= k_first <= k_last <= n_em):
 * laue_refresh at the current poses, laue_cost_sinkhorn at eps_k
 * (n_sinkhorn iterations), then for k < n_em the M-step at eps_k (Newton +
 * MM, or the adjoint Gauss-Newton step) updating R (N x 9) and x (N x 3) in
 * place; step k = n_em is the final E-step alone.  f, g, dust receive the
 * last E-step's potentials; assign and margin (optional) the read-out of
 * the E-step of step k_last (as for laue_cost_sinkhorn).  The
 * whole solve is k_first = 0, k_last = n_em.  Asynchronous and free of host
 * synchronisation and allocation, so it can be captured in a CUDA graph.
 * Needs the workspace of laue_workspace_size with T, n_obs, n_model and
 * n_grains = N set. */
int laue_em(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const LaueObsSpots* obs,
            const float* omega, LaueModelSpots* model, float* R, float* x, int N, const LaueEMParams* prm,
            float* f, float* g, float* dust, int* assign, float* margin, void* stream);

/* ---- learned proposal (an addition beside the paper's method) ---------- */

/* The paper proposes candidate grains by single-grain fits from a grid of
 * starts (Section "Pre-processing").  The calls below add a learned
 * proposal: a set encoder (per-spot MLP of three 256-wide ReLU layers, masked
 * mean and max pooling, a two-layer head emitting 8 hypotheses of 6-D
 * rotation + 3-D position) that reads a seed-conditioned set of observed
 * spots and proposes poses for those fits.  Its per-spot layers and head run
 * in BF16 on the tensor cores with FP32 accumulation.  The paper has no counterpart
 * for any of these calls. */

/* BF16 GEMM on the tcgen05 tensor cores: D[m][n] = sum_k A[m][k] B[n][k].
 * A: M x K BF16, row-major with leading dimension lda (elements); B: N x K
 * BF16 with ldb.  flags bit 1: A is stored MN-major instead, as the K x M
 * array A^T (element (m, k) at A[k lda + m], lda >= M); flags bit 2: B is
 * stored as the K x N array B^T (ldb >= N).  M % 128 == 0, N % bn == 0 with
 * bn in {64, 128, 256}, K % 64 == 0, (K / 64) % splits == 0, lda, ldb % 8 ==
 * 0, all pointers 16-byte aligned.  mode 0: D_f32 receives `splits` FP32 partial products
 * (split s covers K range [s K/splits, (s+1) K/splits)) at D_f32 + s M N,
 * row-major M x N.  mode 1: relu(acc + bias[n]) rounded to BF16 (nearest
 * even) into D_bf16 (M x N row-major) and/or DT_bf16 (N rows of leading
 * dimension ldt >= M: DT[n][m]); splits must be 1.  mode 2: acc where the
 * BF16 mask[m][n] (M x N row-major) is > 0, else 0, same outputs.
 * Modes 1 and 2 with N = 256, K in {64, 256} and both operands K-major run
 * a persistent, warp-specialised kernel (weights resident in shared memory,
 * two tensor-memory accumulators); flags bit 0 forces the one-tile-per-CTA
 * kernel.
 * Asynchronous on `stream`; device memory is the caller's.  Needs the
 * workspace (status word).  Errors: LAUE_ERR_INVALID_ARG for shapes,
 * alignment or a missing output. */
int laue_gemm_bf16(laue_handle* h, const void* A, long long lda, const void* B, long long ldb, int M,
                   int N, int K, int bn, int splits, int mode, const float* bias, const void* mask,
                   float* D_f32, void* D_bf16, void* DT_bf16, long long ldt, int flags, void* stream);

/* Sizes of the set encoder's buffers (host helpers, no device work).
 * Parameter vector (FP32, laue_lp_param_count() values): W1 (256 x 64), b1,
 * W2 (256 x 256), b2, W3 (256 x 256), b3, W4 (256 x 512), b4, W5 (72 x 256),
 * b5; weights row-major [out][in].  Network buffer: laue_lp_net_bytes()
 * bytes of device memory holding the parameters, Adam moments, gradients,
 * BF16 weight copies and split-K partials.  Batch buffer for n_sets sets:
 * laue_lp_batch_bytes(n_sets) bytes (features, activations, errors, head
 * arrays); both 256-byte aligned and owned by the caller.
 * laue_lp_batch_offset(n_sets, region) is the byte offset of a region of
 * the batch buffer (-1 if unknown): 0 X (n_sets*set_size x 64 BF16 features),
 * 1 unused (-1), 2 seed frames F (n_sets x 9 FP32, row-major, columns n0 a1 a2),
 * 3 valid elements per set (int), 4 R_loc targets (n_sets x 9), 5 position
 * targets (n_sets x 3, x / 2.5 mm), 6 set valid flags (FP32), 7 network
 * outputs O (n_sets x 72: 8 hypotheses of 6-D rotation + 3-D position),
 * 8 per-set losses, 9 per-set best rotation error, 10 best hypothesis
 * (int), 11 H1, 12 H3 (n_sets*set_size x 256 BF16), 13 pooled features
 * (n_sets x 512 FP32), 14 dL/dO, 15 dL/dZ3 (BF16). */
size_t laue_lp_param_count(void);
size_t laue_lp_set_size(void); /* spots per set (the seed + its nearest neighbours) */
size_t laue_lp_net_bytes(void);
size_t laue_lp_batch_bytes(int n_sets);
long long laue_lp_batch_offset(int n_sets, int region);

/* Loads parameters (host FP32 vector) into a network buffer, clears the
 * Adam state and step counter and writes the BF16 weight copies.
 * Synchronises `stream` (the host copy is pageable). */
int laue_lp_net_init(laue_handle* h, void* net, const float* params_host, void* stream);

/* Copies the parameters and/or the last gradients (laue_lp_param_count()
 * FP32 each; either pointer may be NULL) to the host.  Synchronises. */
int laue_lp_net_params(laue_handle* h, const void* net, float* params_host, float* grads_host,
                       void* stream);

/* Training scenes simulated by the forward model (Eqs. ray_mnt, s_mnt,
 * wavelength, model_spot_cut).  Counter-based Philox4x32-10 draws, keyed by
 * `seed`: per scene s < S a window start t0 in [0, T - W] and a grain count
 * in [gmin, gmax]; per grain g < Gmax a uniform rotation (Shoemake) into
 * grainR[(s Gmax + g) 9] and a position uniform in the cube of side cube_mm
 * into grainX.  Virtual angle v = s W + k has rotation omega[t0 + k]
 * (written to omega_v[v]); its spots are the grains' visible spots with
 * N(0, sigma_mm^2) noise on x and y (dropped if pushed off the detector),
 * followed by floor(outlier_ratio n_true + u) uniform outliers.  Outputs:
 * I_off (S W + 1), p (float4 x, y, z, 0 per spot, 16-byte aligned) and
 * label (s Gmax + g, or -1 for an outlier), at most `capacity` spots
 * (beyond it the status word records LAUE_ERR_CAPACITY and the list is
 * cut).  scene_i32 is scratch of 4 S W + 2 S ints (grain counts, window
 * starts, per-angle counts).  Planes must number at most 65535, and every
 * detector's normal must lie along z (the noise and the outliers are drawn in
 * the detectors' x and y; LAUE_ERR_INVALID_ARG otherwise).
 * Asynchronous; nothing is read back. */
int laue_lp_scene(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const float* omega,
                  int T, int W, int S, int Gmax, int gmin, int gmax, float cube_mm, float sigma_mm,
                  double outlier_ratio, unsigned long long seed, float* grainR, float* grainX,
                  int* scene_i32, int* I_off, float* omega_v, float* p, int* label, int capacity,
                  void* stream);

/* Seeds of a training batch: per scene s and set j < per_scene, the first
 * inlier among up to 64 spots of the scene drawn uniformly by Philox (or
 * -1); the window of set (s, j) is [s W, (s+1) W).  Outputs seeds, wlo,
 * whi (S per_scene ints each).  Asynchronous. */
int laue_lp_scene_seeds(laue_handle* h, const int* I_off, const int* label, int W, int S, int per_scene,
                        unsigned long long seed, int* seeds, int* wlo, int* whi, void* stream);

/* Seed-conditioned sets.  Spots p (float4, 16-byte aligned) sorted by angle
 * with offsets I_off (n_angles + 1), rotation angles omega (n_angles), at
 * most n_cap spots.  For set b: seed spot seeds[b] (-1: an empty set) and
 * window of angles [wlo[b], whi[b]).  Each spot's sample-frame axis is
 * n = Gamma_t^T u with u parallel to p/|p| - e (the plane normal of a
 * reflection off a grain at the origin, Eq. ray_mnt); the set holds the
 * seed and the laue_lp_set_size() - 1 spots of the window whose axes are nearest the seed's
 * (distance 1 - |n.n0|, ties by index), as 64 BF16 features in the seed
 * frame [n0, a1, n0 x a1] (a1: unit part of +y orthogonal to n0), written
 * to the batch buffer (regions 0-3).  With label (spot -> grain, -1 for an
 * outlier) and grainR / grainX (9 and 3 FP32 per grain), the targets
 * R_loc = F0^T R and x / 2.5 mm and the valid flags are written too.
 * axes_scratch: 16 n_cap bytes.  ids (n_sets x set_size ints, -1 for padding)
 * may be NULL.  Asynchronous. */
int laue_lp_sets(laue_handle* h, const LaueGeometry* geom, const float* p, const int* I_off,
                 const float* omega, int n_angles, int n_cap, const int* seeds, const int* wlo,
                 const int* whi, int n_sets, const int* label, const float* grainR,
                 const float* grainX, void* axes_scratch, void* batch, int* ids, void* stream);

/* Network forward over the sets in the batch buffer: per-spot layers as
 * BF16 tcgen05 GEMMs with FP32 accumulation and fused bias + ReLU, masked
 * mean and max pooling, the head as two more such GEMMs (the pooled
 * features and hidden units rounded to BF16); outputs O (FP32) in batch
 * region 7.
 * Asynchronous. */
int laue_lp_forward(laue_handle* h, const void* net, void* batch, int n_sets, void* stream);

/* One training step on the sets and targets in the batch buffer: forward;
 * per set the loss min_h L_h + 0.05 mean_h L_h with L_h = min over the 24
 * cube rotations S of ||GS(o_h) - R_loc S||_F^2 + 0.1 ||xhat_h - x||^2,
 * averaged over the valid sets; backward (every GEMM on the tensor cores,
 * the errors they read rounded to BF16; weight gradients read the row-major
 * activations MN-major); Adam (beta 0.9, 0.999,
 * eps 1e-8, learning rate lr; lr = 0 leaves the parameters unchanged).
 * Losses, best errors and hypotheses land in batch regions 8-10, gradients
 * in the network buffer.  Asynchronous. */
int laue_lp_train_step(laue_handle* h, void* net, void* batch, int n_sets, float lr, void* stream);

/* Proposals from the outputs O: per set and hypothesis h, R = F0 GS(o_h)
 * (row-major 3x3, R_out n_sets x 8 x 9) and x = 2.5 mm o_h[6:9] (x_out
 * n_sets x 8 x 3); empty sets give the identity and 0.  Asynchronous. */
int laue_lp_decode(laue_handle* h, const void* batch, int n_sets, float* R_out, float* x_out,
                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* LAUEOT_H */
