// index.cu — end-to-end indexing (paper Algorithm LaueOT preceded by the
// pre-processing of Section "Pre-processing"): batched single-grain fits from
// a start grid, the f_out filter, SPOT prototype selection with k*, the cut at
// the prototypes, and the annealed multi-grain EM.  The host only sequences
// launches and reads back three counts (kept candidates, k*, visible spots).
#include <cmath>
#include <cstring>

#include "api_internal.h"

namespace laue {

// keep flags -> ordered indices of the kept starts, and their count
__global__ void compact_kept_kernel(const int* keep, int S, int* idx, int* count) {
    __shared__ int wc[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    for (int s0 = 0; s0 < S; s0 += blockDim.x) {
        int s = s0 + threadIdx.x;
        bool k = s < S && keep[s];
        unsigned b = __ballot_sync(0xffffffffu, k);
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) wc[w] = __popc(b);
        __syncthreads();
        int before = 0, tot = 0;
        for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
            if (q < w) before += wc[q];
            tot += wc[q];
        }
        if (k) idx[base + before + __popc(b & ((1u << lane) - 1u))] = s;
        __syncthreads();
        if (threadIdx.x == 0) base += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

__global__ void gather_poses_kernel(const int* idx, int n, const float* R, const float* x, float* Ro, float* xo) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    int s = idx[k];
    for (int q = 0; q < 9; ++q) Ro[9 * k + q] = R[9 * s + q];
    for (int q = 0; q < 3; ++q) xo[3 * k + q] = x[3 * s + q];
}

__global__ void spot_to_grain_kernel(const int* assign_j, const int* grain, int n, int* assign) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int j = assign_j[i];
    assign[i] = j >= 0 ? grain[j] : -1;
}

}  // namespace laue

using namespace laue;

namespace {
struct Carve {
    char* p;
    size_t used;
    template <class T>
    T* take(size_t n) {
        size_t a = align_up(used, 256);
        used = a + sizeof(T) * (n > 0 ? n : 1);
        return (T*)(p + a);
    }
};

size_t index_carve_bytes(int T, int n_obs, int S, int n_max) {
    size_t cap = (size_t)n_max * kSfCap;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += align_up(bytes > 0 ? bytes : 1, 256) + 256; };
    add(sizeof(float) * 12 * (size_t)S * 3);  // grid starts, fitted and kept poses
    add(sizeof(int) * (size_t)S * 2 + 64);    // keep, indices, count
    add(sizeof(int) * (size_t)n_max + sizeof(float) * (size_t)n_max);
    add(sizeof(int) * (T + 1));
    add(sizeof(int) * 3 * cap);
    add(sizeof(float) * 12 * cap);
    add(sizeof(float) * ((size_t)n_obs + cap + 2 * T + 16));
    add(sizeof(int) * (size_t)n_obs);
    return b;
}
}  // namespace

extern "C" int laue_index_workspace_size(laue_handle* h, int T, int n_obs, int S, int n_max, int n_planes,
                                         size_t* bytes) {
    if (!h || !bytes || T < 1 || n_obs < 0 || S < 0 || n_max < 0 || n_planes < 1)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "index_workspace_size: bad arguments");
    size_t cap = (size_t)n_max * kSfCap;
    LaueProblemDims a{T, n_obs, (int)cap, n_max, n_planes, 1, S > n_max ? S : n_max};
    size_t sub = make_layout(a, h->sm_count).total;
    // the SPOT matrix (8 bytes per nonzero) needs room beyond the sub-call layout
    size_t spot_tail = (size_t)S * 1024 + (1 << 20);
    *bytes = sub + spot_tail + index_carve_bytes(T, n_obs, S, n_max);
    return LAUE_OK;
}

extern "C" int laue_index(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const LaueObsSpots* obs,
                          const float* omega, const float* startR, const float* startX, int S,
                          const LaueIndexParams* prm, float* R_out, float* x_out, int n_max, int* n_grains_host,
                          int* assign, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    int rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if ((rc = laue_check_obs(h, obs))) return rc;
    const bool grid = !startR && !startX;
    if (!lat || lat->M < 1 || !prm || S < 0 || n_max < 1 || !R_out || !x_out || !n_grains_host || !omega ||
        (!grid && S > 0 && (!startR || !startX)) || (obs->n > 0 && !assign) ||
        (grid && (prm->grid_n < 0 || (prm->grid_sym != 1 && prm->grid_sym != 6 && prm->grid_sym != 12 &&
                                      prm->grid_sym != 24) || prm->grid_k < 1 ||
                  !(prm->grid_cube >= 0.0f))) ||
        (prm && prm->mstep_kind != 0 && prm->mstep_kind != 1))
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "index: bad arguments");
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    const int T = obs->T;
    size_t carve = index_carve_bytes(T, obs->n, S, n_max);
    if (carve + (1 << 20) > h->ws_bytes) return laue_fail(h, LAUE_ERR_WORKSPACE, "index: workspace too small");
    cudaStream_t s = (cudaStream_t)stream;
    // the carve sits at the end of the workspace; sub-calls see the rest
    size_t full = h->ws_bytes;
    Carve C{(char*)h->ws + align_up(full - carve, 256) - 256, 0};
    float* gridR = C.take<float>(9 * (size_t)S);
    float* gridX = C.take<float>(3 * (size_t)S);
    float* fitR = C.take<float>(9 * (size_t)S);
    float* fitX = C.take<float>(3 * (size_t)S);
    float* kR = C.take<float>(9 * (size_t)S);
    float* kX = C.take<float>(3 * (size_t)S);
    int* keep = C.take<int>(S);
    int* kidx = C.take<int>(S);
    int* kcount = C.take<int>(16);
    int* order = C.take<int>(n_max);
    float* gains = C.take<float>(n_max);
    size_t cap = (size_t)n_max * kSfCap;
    int* J_off = C.take<int>(T + 1);
    int* mgrain = C.take<int>(cap);
    int* mplane = C.take<int>(cap);
    int* mangle = C.take<int>(cap);
    float* mray = C.take<float>(4 * cap);
    float* mcen = C.take<float>(4 * cap);
    float* mspot = C.take<float>(4 * cap);
    float* f = C.take<float>((size_t)obs->n + 1);
    float* g = C.take<float>(cap + 1);
    float* dust = C.take<float>(2 * (size_t)T + 2);
    int* assign_j = C.take<int>((size_t)obs->n + 1);
    h->ws_bytes = (size_t)((char*)C.p - (char*)h->ws);
    auto restore = [&](int code) {
        h->ws_bytes = full;
        return code;
    };
    *n_grains_host = 0;
    // 0. the start grid (Section "Single-grain fitting"), unless starts are given
    if (grid) {
        long long Sg = 0;
        if ((rc = laue_start_grid(h, prm->grid_n, prm->grid_sym, prm->grid_k, prm->grid_cube, S, gridR, gridX, &Sg,
                                  stream)))
            return restore(rc);
        if (Sg > S)
            return restore(laue_fail(h, LAUE_ERR_CAPACITY, "index: the start grid has %lld starts, S = %d", Sg, S));
        S = (int)Sg;
        startR = gridR;
        startX = gridX;
    }
    // 1. batched single-grain fits
    LaueSingleParams sp{prm->eps_final, prm->c_out, prm->f_out, prm->k_single, prm->mstep,
                        prm->anneal_single > 0.0f ? prm->anneal_single : 100.0f, prm->recut_single};
    if ((rc = laue_single_fit(h, geom, lat, obs, omega, startR, startX, S, &sp, fitR, fitX, keep, nullptr, stream)))
        return restore(rc);
    // 2. kept candidates (in start order)
    compact_kept_kernel<<<1, 1024, 0, s>>>(keep, S, kidx, kcount);
    int Nc = 0;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(&Nc, kcount, sizeof(int), cudaMemcpyDeviceToHost, s), "count")))
        return restore(rc);
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "index synchronise"))) return restore(rc);
    if (Nc > 0) gather_poses_kernel<<<(Nc + 127) / 128, 128, 0, s>>>(kidx, Nc, fitR, fitX, kR, kX);
    // 3. SPOT selection
    int k_max = Nc < n_max ? Nc : n_max, kstar = 0;
    long long nnz = 0;
    if ((rc = laue_prototype_select(h, geom, lat, obs, omega, kR, kX, Nc, prm->eps_final, prm->c_out, k_max, order,
                                    gains, &kstar, &nnz, stream)))
        return restore(rc);
    if (kstar == 0) {
        if (obs->n > 0) cudaMemsetAsync(assign, 0xff, sizeof(int) * obs->n, s);
        return restore(laue_cuda_check(h, cudaGetLastError(), "index"));
    }
    gather_poses_kernel<<<(kstar + 127) / 128, 128, 0, s>>>(order, kstar, kR, kX, R_out, x_out);
    // 4. frozen model list at the prototypes
    LaueModelSpots ms{T, 0, (int)cap, J_off, mgrain, mplane, mangle, mray, mcen, mspot};
    int total = 0;
    if ((rc = laue_forward(h, geom, lat, R_out, x_out, kstar, omega, T, &ms, &total, stream))) return restore(rc);
    // 5. annealed EM (Algorithm LaueOT) with a final E-step for the assignment
    LaueEMParams ep{prm->unmatched_frac, prm->eps_final, prm->c_out, 100.0f, prm->n_em, prm->n_sinkhorn,
                    prm->dust_mode, prm->mstep_kind, 0, prm->n_em, prm->mstep};
    if ((rc = laue_em(h, geom, lat, obs, omega, &ms, R_out, x_out, kstar, &ep, f, g, dust, assign_j, nullptr,
                      stream)))
        return restore(rc);
    if (obs->n > 0) spot_to_grain_kernel<<<(obs->n + 255) / 256, 256, 0, s>>>(assign_j, mgrain, obs->n, assign);
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "index synchronise"))) return restore(rc);
    *n_grains_host = kstar;
    return restore(LAUE_OK);
}

extern "C" int laue_em(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const LaueObsSpots* obs,
                       const float* omega, LaueModelSpots* model, float* R, float* x, int N, const LaueEMParams* prm,
                       float* f, float* g, float* dust, int* assign, float* margin, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (!prm || !geom || !lat || !obs || !model || !omega || (N > 0 && (!R || !x)) || !f || !g || !dust)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "em: null argument");
    if (prm->n_em < 0 || prm->k_first < 0 || prm->k_first > prm->k_last || prm->k_last > prm->n_em ||
        prm->n_sinkhorn < 0 || !(prm->eps_final > 0.0f) || prm->dust_mode < 0 || prm->dust_mode > 1 ||
        prm->mstep_kind < 0 || prm->mstep_kind > 1 || N < 0)
        return laue_fail(h, LAUE_ERR_INVALID_ARG,
                         "em: 0 <= k_first <= k_last <= n_em, eps_final > 0, dust_mode 0 or 1, mstep_kind 0 or 1");
    const double anneal = prm->anneal > 0.0f ? prm->anneal : 100.0;
    LaueOTParams op{prm->unmatched_frac, 0.0f, prm->c_out, prm->n_sinkhorn, prm->dust_mode, 0, 0.0f, 0.0f, 0};
    int rc;
    for (int k = prm->k_first; k <= prm->k_last; ++k) {
        const double eps = anneal_eps(prm->eps_final, prm->n_em, k, anneal);
        op.eps = (float)eps;
        if ((rc = laue_refresh(h, geom, lat, R, x, omega, model, stream))) return rc;
        const bool last = k == prm->k_last;  // the read-out of the call's last E-step
        if ((rc = laue_cost_sinkhorn(h, geom, obs, model, &op, f, g, dust, last ? assign : nullptr,
                                     last ? margin : nullptr, nullptr, nullptr, stream)))
            return rc;
        if (k == prm->n_em) break;  // the final E-step
        LaueMParams mp = prm->mstep;
        mp.eps = (float)eps;
        rc = prm->mstep_kind == 1
                 ? laue_mstep_adjoint(h, geom, lat, obs, model, f, g, &mp, omega, R, x, N, nullptr, stream)
                 : laue_mstep(h, geom, lat, obs, model, f, g, &mp, omega, R, x, N, nullptr, stream);
        if (rc) return rc;
    }
    return LAUE_OK;
}
