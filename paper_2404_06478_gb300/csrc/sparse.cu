// sparse.cu — the E-step on a sparse plan (paper Section "Working with
// sparse assignment matrices": only the rho nearest neighbours of each spot
// carry assignment weight, so a Sinkhorn update costs rho |J| instead of
// |I| |J|).
//
// Support: each model spot j keeps the rho observed spots of its angle block
// with the smallest pair cost C_ij = D_j^2 |rhat_ij - r_j|^2 (D_j the cost
// length of the spot's detector; ties to the lower observed index); every
// other observed-model entry of the plan is 0, the outlier column and the
// unmatched-model row stay dense.  The records hold
// e2_ij = (D_j / D)^2 |rhat_ij - r_j|^2.  The neighbour lists
// are built once per call from the model list's rays and centres, then
// transposed into rows (CSR by observed spot, ascending model index).  The
// updates are those of the dense passes restricted to the support, in base 2
// with K = D^2 log2(e)/eps and kc = c_out log2(e)/eps:
//   F_i = -LSE2({G_j - K e2_ij : i in N(j)} u {G_0 - kc})
//   G_j = -LSE2({F_i - K e2_ij : i in N(j)} u {F_0})
// and the dustbin updates in the same order as the dense passes.
//
// Work split: the spots of each angle block are cut into tiles of kSpTile;
// one CTA per tile, one warp per spot, the lanes over the spot's entries
// (8-byte {index, e2} records read coalesced), a warp log-sum-exp with the
// running maximum (no shifted fast sum, so no underflow fallback is needed).
// The last CTA of a pass (completion ticket) merges the per-tile partial
// log-sum-exps into the dustbin potentials, one warp per dustbin.
#include <algorithm>

#include "api_internal.h"

namespace laue {

constexpr int kSpThreads = 256;
constexpr int kSpWarps = kSpThreads / 32;
constexpr int kSpTile = 512;  // spots per tile
constexpr int kKnnThreads = 256;

struct SpDust {
    float *F0, *F0n, *G0, *log2U, *log2O, *err;
};

__device__ __forceinline__ SpDust sp_dust(float* base, int nd) {
    SpDust d;
    d.F0 = base;
    d.F0n = base + nd;
    d.G0 = base + 2 * nd;
    d.log2U = base + 3 * nd;
    d.log2O = base + 4 * nd;
    d.err = base + 5 * nd;
    return d;
}

// running-maximum log-sum-exp accumulation of one term
__device__ __forceinline__ void acc_lse(float& m, float& s, float v) {
    if (v > m) {
        s = s * ex2(m - v) + 1.0f;
        m = v;
    } else {
        s += ex2(v - m);
    }
}

// |rhat - r|^2 for one pair (the scalar form of the dense passes' cost)
__device__ __forceinline__ float sp_e2(float4 p, float4 c, float4 r) {
    float dx = p.x - c.x, dy = p.y - c.y, dz = p.z - c.z;
    float s = rsq(fmaf(dx, dx, fmaf(dy, dy, dz * dz)));
    float ex = fmaf(dx, s, -r.x), ey = fmaf(dy, s, -r.y), ez = fmaf(dz, s, -r.z);
    return fmaf(ex, ex, fmaf(ey, ey, ez * ez));
}

// ---------------------------------------------------------------- schedule
__global__ void sp_schedule_kernel(SpArgs a) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    int nr = 0, nc = 0;
    for (int t = 0; t < a.T; ++t) {
        a.rt_base[t] = nr;
        for (int s = a.I_off[t]; s < a.I_off[t + 1]; s += kSpTile)
            a.rtile[nr++] = make_int4(t, s, min(s + kSpTile, a.I_off[t + 1]), 0);
        a.ct_base[t] = nc;
        for (int s = a.J_off[t]; s < a.J_off[t + 1]; s += kSpTile)
            a.ctile[nc++] = make_int4(t, s, min(s + kSpTile, a.J_off[t + 1]), 0);
    }
    a.rt_base[a.T] = nr;
    a.ct_base[a.T] = nc;
}

// ------------------------------------------------------------- neighbours
// Inserts (i, v) into the sorted list L of n <= rho entries (an equal e2 goes
// after: its index is larger); worst becomes the largest kept e2 once the list
// is full.
__device__ __forceinline__ void knn_insert(int2* L, int rho, int& n, float& worst, int i, float v) {
    int q = n < rho ? n++ : rho - 1;
    while (q > 0 && __int_as_float(L[q - 1].y) > v) {
        L[q] = L[q - 1];
        --q;
    }
    L[q] = make_int2(i, __float_as_int(v));
    if (n == rho) worst = __int_as_float(L[rho - 1].y);
}

// One thread per model spot (column tiles): the rho smallest e2 over its
// block's observed spots in shared memory, kept sorted by (e2, index).
__global__ void __launch_bounds__(kKnnThreads) sp_knn_kernel(SpArgs a) {
    extern __shared__ int2 sp_heap[];
    if ((int)blockIdx.x >= a.ct_base[a.T]) return;
    const int4 td = a.ctile[blockIdx.x];
    const int i0 = a.I_off[td.x], i1 = a.I_off[td.x + 1];
    int2* L = sp_heap + (size_t)threadIdx.x * a.rho;
    for (int j = td.y + threadIdx.x; j < td.z; j += kKnnThreads) {
        const float4 c = a.c[j], r = a.r[j];
        int n = 0;
        float worst = 3.0e38f;  // the list's largest e2 once it holds rho entries
        int i = i0;
        for (; i + 4 <= i1; i += 4) {  // four independent costs, then the rare insertions in index order
            float v0 = sp_e2(a.p[i], c, r), v1 = sp_e2(a.p[i + 1], c, r);
            float v2 = sp_e2(a.p[i + 2], c, r), v3 = sp_e2(a.p[i + 3], c, r);
            if (v0 < worst) knn_insert(L, a.rho, n, worst, i, v0);
            if (v1 < worst) knn_insert(L, a.rho, n, worst, i + 1, v1);
            if (v2 < worst) knn_insert(L, a.rho, n, worst, i + 2, v2);
            if (v3 < worst) knn_insert(L, a.rho, n, worst, i + 3, v3);
        }
        for (; i < i1; ++i) {
            float v = sp_e2(a.p[i], c, r);
            if (v < worst) knn_insert(L, a.rho, n, worst, i, v);
        }
        const int det = a.s ? (int)a.s[j].w : -1;
        const float kd = (det >= 0 && det < a.n_det) ? a.kdet[det] : 1.0f;
        int2* out = a.cent + (size_t)j * a.rho;
        for (int k = 0; k < a.rho; ++k)
            out[k] = k < n ? make_int2(L[k].x, __float_as_int(__int_as_float(L[k].y) * kd)) : make_int2(-1, 0);
        if (a.nbr_out)
            for (int k = 0; k < a.rho; ++k) a.nbr_out[(size_t)j * a.rho + k] = k < n ? L[k].x : -1;
    }
}

__global__ void sp_count_kernel(SpArgs a) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)a.n_model * a.rho) return;
    int i = a.cent[e].x;
    if (i >= 0) atomicAdd(&a.rptr[i + 1], 1);
}

// inclusive prefix sum of rptr[1..n_obs] by one CTA (rptr[0] = 0)
__global__ void __launch_bounds__(1024) sp_scan_kernel(SpArgs a) {
    __shared__ int part[1024];
    const int n = a.n_obs;
    const int per = (n + 1023) / 1024;
    const int b0 = 1 + (int)threadIdx.x * per, b1 = min(n + 1, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += a.rptr[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < 1024; ++k) {
            int v = part[k];
            part[k] = acc;
            acc += v;
        }
    }
    __syncthreads();
    int acc = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        acc += a.rptr[b];
        a.rptr[b] = acc;
    }
}

__global__ void sp_fill_kernel(SpArgs a) {
    size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= (size_t)a.n_model * a.rho) return;
    int2 v = a.cent[e];
    if (v.x < 0) return;
    int slot = a.rptr[v.x] + atomicAdd(&a.rfill[v.x], 1);
    a.rent[slot] = make_int2((int)(e / a.rho), v.y);
}

// each row in ascending model index (a fixed summation order)
__global__ void sp_sort_rows_kernel(SpArgs a) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n_obs) return;
    const int s0 = a.rptr[i], s1 = a.rptr[i + 1];
    for (int k = s0 + 1; k < s1; ++k) {
        int2 v = a.rent[k];
        int q = k - 1;
        while (q >= s0 && a.rent[q].x > v.x) {
            a.rent[q + 1] = a.rent[q];
            --q;
        }
        a.rent[q + 1] = v;
    }
}

// ------------------------------------------------------------------ init
__global__ void sp_init_pot_kernel(SpArgs a) {
    const float s = 1.0f / a.to_user;
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.n_obs) a.F[k] = a.warm ? a.f[k] * s : 0.0f;
    if (k < a.n_model) a.G[k] = a.warm ? a.g[k] * s : 0.0f;
}

// Masses, starting dustbin potentials and F_0 of the first row pass (from the
// starting G and G_0).  One CTA per dustbin.
__global__ void __launch_bounds__(1024) sp_init_dust_kernel(SpArgs a) {
    __shared__ float sm[32], ss[32];
    const int nd = a.mode ? a.T : 1;
    const int d = blockIdx.x;
    SpDust D = sp_dust(a.dust, nd);
    const float s = 1.0f / a.to_user;
    const long long nI = a.mode ? (a.I_off[d + 1] - a.I_off[d]) : a.I_off[a.T];
    const long long nJ = a.mode ? (a.J_off[d + 1] - a.J_off[d]) : a.J_off[a.T];
    const float g0 = (a.warm && a.dust_out) ? a.dust_out[nd + d] * s : 0.0f;
    float log2U = kNegHuge;
    if (threadIdx.x == 0) {
        double u = ceil(a.frac * (double)nJ - 1e-9);
        double o = u + (double)nI - (double)nJ;
        if (o < 0) {
            u = (double)(nJ - nI);
            o = 0;
        }
        log2U = u > 0 ? (float)log2(u) : kNegHuge;
        D.log2U[d] = log2U;
        D.log2O[d] = o > 0 ? (float)log2(o) : kNegHuge;
        D.F0[d] = (a.warm && a.dust_out) ? a.dust_out[d] * s : 0.0f;
        D.G0[d] = g0;
    }
    const int j0 = a.mode ? a.J_off[d] : 0, j1 = a.mode ? a.J_off[d + 1] : a.n_model;
    float m = kNegHuge, sum = 0.0f;
    for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) acc_lse(m, sum, a.warm ? a.g[j] * s : 0.0f);
    warp_lse_reduce(m, sum);
    if ((threadIdx.x & 31) == 0) {
        sm[threadIdx.x >> 5] = m;
        ss[threadIdx.x >> 5] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Lse2 L;
        L.init(g0 - a.kc);
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) L.merge(sm[w], ss[w]);
        D.F0n[d] = log2U - L.value();
    }
}

// Block log-sum-exp of the lanes' (m, s); the result is valid in thread 0.
__device__ __forceinline__ void sp_block_lse(float& m, float& s, float* red_m, float* red_s) {
    warp_lse_reduce(m, s);
    if ((threadIdx.x & 31) == 0) {
        red_m[threadIdx.x >> 5] = m;
        red_s[threadIdx.x >> 5] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Lse2 L;
        L.m = kNegHuge;
        L.s = 0.0f;
        for (int k = 0; k < kSpWarps; ++k) L.merge(red_m[k], red_s[k]);
        m = L.m;
        s = L.s;
    }
}

// True in the last CTA of the grid to arrive; that CTA resets the ticket.
__device__ __forceinline__ bool sp_last(int* ticket, int* flag) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
        if (last) *ticket = 0;
        *flag = last;
    }
    __syncthreads();
    bool last = *flag != 0;
    if (last) __threadfence();
    return last;
}

// Warp-level LSE of the partials of tiles [k0, k1) (valid in every lane).
__device__ __forceinline__ void sp_merge_parts(const float2* part, int k0, int k1, float& m, float& s) {
    m = kNegHuge;
    s = 0.0f;
    for (int k = k0 + (int)(threadIdx.x & 31); k < k1; k += 32) {
        float2 v = part[k];
        Lse2 L{m, s};
        L.merge(v.x, v.y);
        m = L.m;
        s = L.s;
    }
    warp_lse_reduce(m, s);
}

// --------------------------------------------------------------- row pass
// Each row is the sum of its support terms 2^(G_j - K e2 - shift) and the
// outlier term, shifted by shift = max(largest G of the angle block, the
// outlier exponent): every term is <= 1, so no running maximum is kept.  A row
// whose shifted sum falls below kSpTiny is recomputed with the running maximum.
// Eight lanes per row, four rows per warp; the lanes stride over the row's
// records.
constexpr float kSpTiny = 1.0e-30f;
constexpr int kSpLanes = 8;  // lanes per spot

__device__ float sp_row_exact(const SpArgs& a, int i, float dustv, bool ub) {
    float m = kNegHuge, s = 0.0f;
    if (!ub) acc_lse(m, s, dustv);
    for (int e = a.rptr[i]; e < a.rptr[i + 1]; ++e) {
        int2 v = a.rent[e];
        acc_lse(m, s, a.G[v.x] + a.negK * __int_as_float(v.y));
    }
    return s > 0.0f ? m + lg2(s) : kNegHuge;
}

__device__ float sp_col_exact(const SpArgs& a, int j, float F0, bool ub) {
    float m = kNegHuge, s = 0.0f;
    if (!ub) acc_lse(m, s, F0);
    const int2* ce = a.cent + (size_t)j * a.rho;
    for (int k = 0; k < a.rho; ++k) {
        int2 v = ce[k];
        if (v.x >= 0) acc_lse(m, s, a.F[v.x] + a.negK * __int_as_float(v.y));
    }
    return s > 0.0f ? m + lg2(s) : kNegHuge;
}

// per-angle largest G of the starting potentials (one CTA per angle)
__global__ void __launch_bounds__(256) sp_gmax_kernel(SpArgs a) {
    __shared__ float red[8];
    const int t = blockIdx.x;
    float m = kNegHuge;
    for (int j = a.J_off[t] + threadIdx.x; j < a.J_off[t + 1]; j += blockDim.x) m = fmaxf(m, a.G[j]);
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) m = fmaxf(m, red[k]);
        a.gmax[t] = fmaxf(m, red[0]);
    }
}

__global__ void __launch_bounds__(kSpThreads) sp_row_kernel(SpArgs a) {
    __shared__ float red_m[kSpWarps], red_s[kSpWarps];
    __shared__ int flag;
    const int nd = a.mode ? a.T : 1;
    SpDust D = sp_dust(a.dust, nd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = lane / kSpLanes, gl = lane % kSpLanes;
    const int n_tiles = a.rt_base[a.T];
    float pm = kNegHuge, ps = 0.0f;  // LSE of F_i - kc over this lane's rows
    if ((int)blockIdx.x < n_tiles) {
        const int4 td = a.rtile[blockIdx.x];
        const float dustv = D.G0[a.mode ? td.x : 0] - a.kc;
        const float shift = fmaxf(a.gmax[td.x], dustv);
        const float dterm = ex2(dustv - shift);
        for (int ib = td.y + w * (32 / kSpLanes); ib < td.z; ib += kSpWarps * (32 / kSpLanes)) {
            const int i = ib + grp;
            const bool vr = i < td.z;
            float sum = 0.0f;
            if (vr)
                for (int e = a.rptr[i] + gl; e < a.rptr[i + 1]; e += kSpLanes) {
                    int2 v = a.rent[e];
                    sum += ex2(a.G[v.x] + a.negK * __int_as_float(v.y) - shift);
                }
#pragma unroll
            for (int o = kSpLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (vr && gl == 0) {
                sum += dterm;
                float F = -(sum > kSpTiny ? shift + lg2(sum) : sp_row_exact(a, i, dustv, false));
                a.F[i] = F;
                acc_lse(pm, ps, F - a.kc);
            }
        }
    }
    sp_block_lse(pm, ps, red_m, red_s);
    if (threadIdx.x == 0 && (int)blockIdx.x < n_tiles) a.rpart[blockIdx.x] = make_float2(pm, ps);
    if (!sp_last(a.ctrl + CTRL_SP_DONE, &flag)) return;
    // promote F_0 and compute G_0 from the new F (as after a dense row pass)
    for (int d = w; d < nd; d += kSpWarps) {
        float m, s;
        sp_merge_parts(a.rpart, a.mode ? a.rt_base[d] : 0, a.mode ? a.rt_base[d + 1] : n_tiles, m, s);
        if (lane == 0) {
            float F0 = D.F0n[d];
            D.F0[d] = F0;
            Lse2 L{m, s};
            L.merge(F0 - a.kc, 1.0f);
            D.G0[d] = D.log2O[d] - L.value();
        }
    }
    // per-angle largest F for the column pass's shift (the tile partials keep max(F - kc))
    for (int t = w; t < a.T; t += kSpWarps) {
        float m = kNegHuge;
        for (int k = a.rt_base[t] + lane; k < a.rt_base[t + 1]; k += 32) m = fmaxf(m, a.rpart[k].x);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) a.fmax[t] = m > kNegHuge ? m + a.kc : kNegHuge;
    }
}

// ------------------------------------------------------------ column pass
__global__ void __launch_bounds__(kSpThreads) sp_col_kernel(SpArgs a) {
    __shared__ float red_m[kSpWarps], red_s[kSpWarps];
    __shared__ int flag;
    const int nd = a.mode ? a.T : 1;
    SpDust D = sp_dust(a.dust, nd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int grp = lane / kSpLanes, gl = lane % kSpLanes;
    const int n_tiles = a.ct_base[a.T];
    float pm = kNegHuge, ps = 0.0f;  // LSE of G_j over this lane's columns
    if ((int)blockIdx.x < n_tiles) {
        const int4 td = a.ctile[blockIdx.x];
        const float F0 = D.F0[a.mode ? td.x : 0];
        const float shift = fmaxf(a.fmax[td.x], F0);
        const float dterm = ex2(F0 - shift);
        for (int jb = td.y + w * (32 / kSpLanes); jb < td.z; jb += kSpWarps * (32 / kSpLanes)) {
            const int j = jb + grp;
            const bool vc = j < td.z;
            float sum = 0.0f;
            if (vc) {
                const int2* ce = a.cent + (size_t)j * a.rho;
                for (int k = gl; k < a.rho; k += kSpLanes) {
                    int2 v = ce[k];
                    if (v.x >= 0) sum += ex2(a.F[v.x] + a.negK * __int_as_float(v.y) - shift);
                }
            }
#pragma unroll
            for (int o = kSpLanes / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
            if (vc && gl == 0) {
                sum += dterm;
                float G = -(sum > kSpTiny ? shift + lg2(sum) : sp_col_exact(a, j, F0, false));
                a.G[j] = G;
                acc_lse(pm, ps, G);
            }
        }
    }
    sp_block_lse(pm, ps, red_m, red_s);
    if (threadIdx.x == 0 && (int)blockIdx.x < n_tiles) a.cpart[blockIdx.x] = make_float2(pm, ps);
    if (!sp_last(a.ctrl + CTRL_SP_DONE, &flag)) return;
    // F_0 of the next row pass from the new G and the current G_0
    for (int d = w; d < nd; d += kSpWarps) {
        float m, s;
        sp_merge_parts(a.cpart, a.mode ? a.ct_base[d] : 0, a.mode ? a.ct_base[d + 1] : n_tiles, m, s);
        if (lane == 0) {
            Lse2 L{m, s};
            L.merge(D.G0[d] - a.kc, 1.0f);
            D.F0n[d] = D.log2U[d] - L.value();
        }
    }
    // per-angle largest G for the next row pass's shift (the tile partials keep max G)
    for (int t = w; t < a.T; t += kSpWarps) {
        float m = kNegHuge;
        for (int k = a.ct_base[t] + lane; k < a.ct_base[t + 1]; k += 32) m = fmaxf(m, a.cpart[k].x);
        for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) a.gmax[t] = m;
    }
}

// ------------------------------------------------------------- read-out
struct SpTop2 {
    float b1, b2;
    int arg;
};

// the larger first value wins, equal values go to the lower model index
__device__ __forceinline__ SpTop2 sp_top2_merge(SpTop2 x, SpTop2 y) {
    bool xw = x.b1 > y.b1 || (x.b1 == y.b1 && (unsigned)x.arg < (unsigned)y.arg);
    SpTop2 w = xw ? x : y, l = xw ? y : x;
    w.b2 = fmaxf(w.b2, l.b1);
    return w;
}

__global__ void __launch_bounds__(kSpThreads) sp_harvest_row_kernel(SpArgs a) {
    __shared__ float red[kSpWarps];
    const int nd = a.mode ? a.T : 1;
    SpDust D = sp_dust(a.dust, nd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float my_err = 0.0f;
    if ((int)blockIdx.x < a.rt_base[a.T]) {
        const int4 td = a.rtile[blockIdx.x];
        const float dustv = D.G0[a.mode ? td.x : 0] - a.kc;
        for (int i = td.y + w; i < td.z; i += kSpWarps) {
            float m = kNegHuge, s = 0.0f;
            SpTop2 T2{kNegHuge, kNegHuge, -1};
            for (int e = a.rptr[i] + lane; e < a.rptr[i + 1]; e += 32) {
                int2 v = a.rent[e];
                float x = a.G[v.x] + a.negK * __int_as_float(v.y);
                acc_lse(m, s, x);
                if (x > T2.b1) {  // ascending model index per lane: ties keep the earlier
                    T2.b2 = T2.b1;
                    T2.b1 = x;
                    T2.arg = v.x;
                } else if (x > T2.b2) {
                    T2.b2 = x;
                }
            }
            warp_lse_reduce(m, s);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                SpTop2 y{__shfl_xor_sync(0xffffffffu, T2.b1, o), __shfl_xor_sync(0xffffffffu, T2.b2, o),
                         __shfl_xor_sync(0xffffffffu, T2.arg, o)};
                T2 = sp_top2_merge(T2, y);
            }
            if (lane == 0) {
                const float F = a.F[i];
                if (dustv > T2.b1) {  // the outlier column only when strictly larger
                    T2.b2 = T2.b1;
                    T2.b1 = dustv;
                    T2.arg = -1;
                } else if (dustv > T2.b2) {
                    T2.b2 = dustv;
                }
                Lse2 L{m, s};
                L.merge(dustv, 1.0f);
                my_err = fmaxf(my_err, fabsf(ex2(F + L.value()) - 1.0f));
                if (a.assign) a.assign[i] = T2.arg;
                if (a.margin) a.margin[i] = ex2(F + T2.b1) - (T2.b2 > kNegHuge ? ex2(F + T2.b2) : 0.0f);
            }
        }
    }
    if (lane == 0) red[w] = my_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        float e = 0.0f;
        for (int k = 0; k < kSpWarps; ++k) e = fmaxf(e, red[k]);
        atomicMax((int*)(D.err + 0), __float_as_int(e));  // non-negative floats order as ints
    }
}

__global__ void __launch_bounds__(kSpThreads) sp_harvest_col_kernel(SpArgs a) {
    __shared__ float red[kSpWarps];
    const int nd = a.mode ? a.T : 1;
    SpDust D = sp_dust(a.dust, nd);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float my_err = 0.0f;
    if ((int)blockIdx.x < a.ct_base[a.T]) {
        const int4 td = a.ctile[blockIdx.x];
        const float F0 = D.F0[a.mode ? td.x : 0];
        for (int j = td.y + w; j < td.z; j += kSpWarps) {
            const int2* ce = a.cent + (size_t)j * a.rho;
            const float G = a.G[j];
            float qj = 0.0f;
            for (int k = lane; k < a.rho; k += 32) {
                int2 v = ce[k];
                if (v.x >= 0) qj += ex2(a.F[v.x] + G + a.negK * __int_as_float(v.y));
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) qj += __shfl_xor_sync(0xffffffffu, qj, o);
            if (lane == 0) {
                if (a.q) a.q[j] = qj;
                my_err = fmaxf(my_err, fabsf(qj + ex2(G + F0) - 1.0f));
            }
        }
    }
    if (lane == 0) red[w] = my_err;
    __syncthreads();
    if (threadIdx.x == 0) {
        float e = 0.0f;
        for (int k = 0; k < kSpWarps; ++k) e = fmaxf(e, red[k]);
        atomicMax((int*)(D.err + 1), __float_as_int(e));
    }
}

__global__ void sp_finish_kernel(SpArgs a, int have_rows, int have_cols) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (k < a.n_obs) {
        float v = a.F[k];
        bad |= !isfinite(v);
        a.f[k] = v * a.to_user;
    }
    if (k < a.n_model) {
        float v = a.G[k];
        bad |= !isfinite(v);
        a.g[k] = v * a.to_user;
    }
    if (k == 0) {
        const int nd = a.mode ? a.T : 1;
        SpDust D = sp_dust(a.dust, nd);
        if (a.dust_out)
            for (int d = 0; d < nd; ++d) {
                a.dust_out[d] = D.F0[d] * a.to_user;
                a.dust_out[nd + d] = D.G0[d] * a.to_user;
            }
        if (a.marg_err) {
            float er = D.err[0];
            for (int d = 0; d < nd; ++d)  // the unmatched-model row
                if (D.log2U[d] > kNegHuge) er = fmaxf(er, fabsf(ex2(D.F0[d] - D.F0n[d]) - 1.0f));
            a.marg_err[0] = have_rows ? er : -1.0f;
            a.marg_err[1] = have_cols ? D.err[1] : -1.0f;
        }
    }
    if (bad) set_status(a.ctrl, LAUE_ERR_NUMERIC);
}

__global__ void sp_clear_err_kernel(SpArgs a) {
    SpDust D = sp_dust(a.dust, a.mode ? a.T : 1);
    D.err[0] = D.err[1] = 0.0f;
}

// ------------------------------------------------------------- host side
static size_t sp_max_tiles(int n, int T) { return (size_t)(n + kSpTile - 1) / kSpTile + (size_t)T; }

size_t sparse_workspace_bytes(int T, int n_obs, int n_model, int rho) {
    const size_t nnz = (size_t)n_model * rho;
    size_t b = 0;
    auto add = [&](size_t bytes) { b += align_up(bytes > 0 ? bytes : 1, 256); };
    add(sizeof(int2) * nnz);                         // cent
    add(sizeof(int2) * nnz);                         // rent
    add(sizeof(int) * ((size_t)n_obs + 2));          // rptr
    add(sizeof(int) * ((size_t)n_obs + 1));          // rfill
    add(sizeof(float) * ((size_t)n_obs + 1));        // F
    add(sizeof(float) * ((size_t)n_model + 1));      // G
    add(sizeof(float) * ((size_t)5 * T + 8));        // dust
    add(sizeof(float2) * sp_max_tiles(n_obs, T));    // rpart
    add(sizeof(float2) * sp_max_tiles(n_model, T));  // cpart
    add(sizeof(int4) * sp_max_tiles(n_obs, T));      // rtile
    add(sizeof(int4) * sp_max_tiles(n_model, T));    // ctile
    add(sizeof(int) * 2 * ((size_t)T + 1));          // rt_base, ct_base
    add(sizeof(float) * 2 * ((size_t)T + 1));        // gmax, fmax
    return b;
}

void sparse_carve(SpArgs& a, char* base, int T, int n_obs, int n_model, int rho) {
    const size_t nnz = (size_t)n_model * rho;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        char* p = base + off;
        off += align_up(bytes > 0 ? bytes : 1, 256);
        return p;
    };
    a.cent = (int2*)take(sizeof(int2) * nnz);
    a.rent = (int2*)take(sizeof(int2) * nnz);
    a.rptr = (int*)take(sizeof(int) * ((size_t)n_obs + 2));
    a.rfill = (int*)take(sizeof(int) * ((size_t)n_obs + 1));
    a.F = (float*)take(sizeof(float) * ((size_t)n_obs + 1));
    a.G = (float*)take(sizeof(float) * ((size_t)n_model + 1));
    a.dust = (float*)take(sizeof(float) * ((size_t)5 * T + 8));
    a.rpart = (float2*)take(sizeof(float2) * sp_max_tiles(n_obs, T));
    a.cpart = (float2*)take(sizeof(float2) * sp_max_tiles(n_model, T));
    a.rtile = (int4*)take(sizeof(int4) * sp_max_tiles(n_obs, T));
    a.ctile = (int4*)take(sizeof(int4) * sp_max_tiles(n_model, T));
    a.rt_base = (int*)take(sizeof(int) * 2 * ((size_t)T + 1));
    a.ct_base = a.rt_base + T + 1;
    a.gmax = (float*)take(sizeof(float) * 2 * ((size_t)T + 1));
    a.fmax = a.gmax + T + 1;
    a.max_rt = (int)sp_max_tiles(n_obs, T);
    a.max_ct = (int)sp_max_tiles(n_model, T);
}

size_t sparse_knn_smem(int rho) { return (size_t)kKnnThreads * rho * sizeof(int2); }

cudaError_t sparse_sinkhorn_run(const SpArgs& a, int n_iter, bool rows, bool cols, cudaStream_t s) {
    cudaError_t e;
    const size_t nnz = (size_t)a.n_model * a.rho;
    const int nd = a.mode ? a.T : 1;
    sp_schedule_kernel<<<1, 32, 0, s>>>(a);
    // neighbour lists and their transpose
    const size_t shm = sparse_knn_smem(a.rho);
    if ((e = cudaFuncSetAttribute(sp_knn_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm)) !=
        cudaSuccess)
        return e;
    sp_knn_kernel<<<a.max_ct, kKnnThreads, shm, s>>>(a);
    if ((e = cudaMemsetAsync(a.rptr, 0, sizeof(int) * ((size_t)a.n_obs + 2), s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(a.rfill, 0, sizeof(int) * ((size_t)a.n_obs + 1), s)) != cudaSuccess) return e;
    const unsigned nb = (unsigned)((nnz + 255) / 256);
    if (nnz > 0) sp_count_kernel<<<nb, 256, 0, s>>>(a);
    sp_scan_kernel<<<1, 1024, 0, s>>>(a);
    if (nnz > 0) sp_fill_kernel<<<nb, 256, 0, s>>>(a);
    if (a.n_obs > 0) sp_sort_rows_kernel<<<(a.n_obs + 255) / 256, 256, 0, s>>>(a);
    const int blocks = std::max(1, (std::max(a.n_obs, a.n_model) + 255) / 256);
    sp_init_pot_kernel<<<blocks, 256, 0, s>>>(a);
    sp_init_dust_kernel<<<nd, 1024, 0, s>>>(a);
    if (a.T > 0) sp_gmax_kernel<<<a.T, 256, 0, s>>>(a);
    for (int it = 0; it < n_iter; ++it) {
        sp_row_kernel<<<a.max_rt, kSpThreads, 0, s>>>(a);
        sp_col_kernel<<<a.max_ct, kSpThreads, 0, s>>>(a);
    }
    if (rows || cols) sp_clear_err_kernel<<<1, 1, 0, s>>>(a);
    if (rows) sp_harvest_row_kernel<<<a.max_rt, kSpThreads, 0, s>>>(a);
    if (cols) sp_harvest_col_kernel<<<a.max_ct, kSpThreads, 0, s>>>(a);
    sp_finish_kernel<<<blocks, 256, 0, s>>>(a, rows ? 1 : 0, cols ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace laue
