// sinkhorn.cu — fused pair cost + log-domain balanced Sinkhorn with dustbins
// (paper Eqs. update_L, elbo, estep_obj; Algorithm BalancedOT), blocked by
// rotation angle.
//
// Extended plan: observed rows i plus the unmatched-model row 0 (mass U),
// model columns j plus the outlier column 0 (mass O); costs C_ij (same angle
// only), C_i0 = c_out, C_0j = 0, C_00 = c_out.  In base-2 units with
// F = f log2(e)/eps, G = g log2(e)/eps and K = D^2 log2(e)/eps:
//   row    F_i = -LSE2({G_j - K e2_ij}_{j in J_t} u {G_0 - kc})
//   dust   F_0 = log2 U - LSE2({G_j}_j u {G_0 - kc})
//   column G_j = -LSE2({F_i - K e2_ij}_{i in I_t} u {F_0})
//   dust   G_0 = log2 O - LSE2({F_i - kc}_i u {F_0 - kc})
// with e2_ij = |rhat_ij - r_j|^2 and kc = c_out log2(e)/eps.  The cost matrix
// is never stored: every pass recomputes e2 from the spot coordinates.
//
// Each pass is one persistent launch over all angle blocks: CTAs pull tiles
// (angle t, first row, count) from a queue the scheduler kernel built on the
// device in longest-block-first order.  A tile keeps one row (column) per
// thread in registers and streams the other side of its angle block through
// shared memory in chunks loaded by the bulk-copy engine (cp.async.bulk) into
// a two-stage mbarrier pipeline.  The last CTA to finish a pass combines the
// per-tile partial log-sum-exps into the dustbin potentials:
//   end of a row pass:    F_0 <- F_0(next), then G_0 from the new F and F_0
//   end of a column pass: F_0(next) from the new G and G_0
// which reproduces the sequential order of the algorithm exactly.
#include "common.cuh"
#include "kernels.h"

namespace laue {

constexpr int kTPB = 256;    // threads per CTA = rows (columns) per tile
constexpr int kChunk = 256;  // spots staged per chunk
constexpr int kGroup = 8;    // pairs per max-then-sum group of the online LSE

struct DustPtrs {
    float *F0, *F0n, *G0, *log2U, *log2O, *err;
};

__device__ __forceinline__ DustPtrs dust_ptrs(float* base, int T) {
    DustPtrs d;
    d.F0 = base;
    d.F0n = base + T;
    d.G0 = base + 2 * T;
    d.log2U = base + 3 * T;
    d.log2O = base + 4 * T;
    d.err = base + 5 * T;
    return d;
}

// |rhat - r|^2 with rhat = (p - c)/|p - c|: no cancellation for close rays.
__device__ __forceinline__ float ray_e2(float px, float py, float pz, float cx, float cy, float cz,
                                        float rx, float ry, float rz) {
    float dx = px - cx, dy = py - cy, dz = pz - cz;
    float q = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
    float s = rsq(q);
    float ex = fmaf(dx, s, -rx), ey = fmaf(dy, s, -ry), ez = fmaf(dz, s, -rz);
    return fmaf(ex, ex, fmaf(ey, ey, ez * ez));
}

// ---------------------------------------------------------------- scheduler
// One CTA.  Builds the row and column tile queues (angles by descending work,
// tiles of one angle contiguous), per-angle tile ranges, the log2 masses of
// the dustbins, and clears the queue counters.
__global__ void __launch_bounds__(1024) sk_schedule_kernel(SkArgs a) {
    const int T = a.T;
    int* order_r = (int*)a.row_part;  // scratch until the passes run
    int* order_c = (int*)a.col_part;
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int wr = a.J_off[t + 1] - a.J_off[t];
        int wc = a.I_off[t + 1] - a.I_off[t];
        int rr = 0, rc = 0;
        for (int u = 0; u < T; ++u) {
            int ur = a.J_off[u + 1] - a.J_off[u];
            int uc = a.I_off[u + 1] - a.I_off[u];
            rr += (ur > wr) || (ur == wr && u < t);
            rc += (uc > wc) || (uc == wc && u < t);
        }
        order_r[rr] = t;
        order_c[rc] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nr = 0, nc = 0;
        for (int k = 0; k < T; ++k) {
            int t = order_r[k];
            int ni = a.I_off[t + 1] - a.I_off[t];
            int cnt = (ni + a.tile_rows - 1) / a.tile_rows;
            a.ang_tiles[t].x = nr;
            a.ang_tiles[t].y = cnt;
            nr += cnt;
        }
        for (int k = 0; k < T; ++k) {
            int t = order_c[k];
            int nj = a.J_off[t + 1] - a.J_off[t];
            int cnt = (nj + a.tile_cols - 1) / a.tile_cols;
            a.ang_tiles[t].z = nc;
            a.ang_tiles[t].w = cnt;
            nc += cnt;
        }
        if (nr > a.max_row_tiles || nc > a.max_col_tiles) {
            set_status(a.ctrl, LAUE_ERR_CAPACITY);
            nr = min(nr, a.max_row_tiles);
            nc = min(nc, a.max_col_tiles);
        }
        a.ctrl[CTRL_N_ROW_TILES] = nr;
        a.ctrl[CTRL_N_COL_TILES] = nc;
        for (int k = CTRL_ROW_NEXT; k <= CTRL_HCOL_DONE; ++k)
            if (k != CTRL_N_ROW_TILES && k != CTRL_N_COL_TILES && k != CTRL_FWD_TOTAL) a.ctrl[k] = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int4 at = a.ang_tiles[t];
        int i0 = a.I_off[t], ni = a.I_off[t + 1] - i0;
        for (int k = 0; k < at.y; ++k) {
            int idx = at.x + k;
            if (idx < a.max_row_tiles)
                a.row_tiles[idx] = make_int4(t, i0 + k * a.tile_rows, min(a.tile_rows, ni - k * a.tile_rows), 0);
        }
        int j0 = a.J_off[t], nj = a.J_off[t + 1] - j0;
        for (int k = 0; k < at.w; ++k) {
            int idx = at.z + k;
            if (idx < a.max_col_tiles)
                a.col_tiles[idx] = make_int4(t, j0 + k * a.tile_cols, min(a.tile_cols, nj - k * a.tile_cols), 0);
        }
    }
    // dustbin masses (paper: T_a = T_b - b^T 1 + a^T 1), in double precision
    DustPtrs D = dust_ptrs(a.dust, T);
    int nd = a.mode ? T : 1;
    for (int d = threadIdx.x; d < nd; d += blockDim.x) {
        long long nI = a.mode ? (a.I_off[d + 1] - a.I_off[d]) : a.I_off[T];
        long long nJ = a.mode ? (a.J_off[d + 1] - a.J_off[d]) : a.J_off[T];
        double u = ceil(a.frac * (double)nJ - 1e-9);
        double o = u + (double)nI - (double)nJ;
        if (o < 0) {
            u = (double)(nJ - nI);
            o = 0;
        }
        D.log2U[d] = u > 0 ? (float)log2(u) : kNegHuge;
        D.log2O[d] = o > 0 ? (float)log2(o) : kNegHuge;
    }
}

// ------------------------------------------------------------------- pack
// Workspace copies (p, F) and (c, G); F, G from the caller's potentials on a
// warm start, else 0.
__global__ void sk_pack_kernel(SkArgs a) {
    const float s = 1.0f / a.to_user;  // mm^2 -> base-2 internal units
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.n_obs) {
        float4 p = a.obs_p[k];
        a.obsP[k] = make_float4(p.x, p.y, p.z, a.warm ? a.f[k] * s : 0.0f);
    }
    if (k < a.n_model) {
        float4 c = a.mod_c[k];
        a.modC[k] = make_float4(c.x, c.y, c.z, a.warm ? a.g[k] * s : 0.0f);
    }
    if (k == 0) {
        DustPtrs D = dust_ptrs(a.dust, a.T);
        int nd = a.mode ? a.T : 1;
        for (int d = 0; d < nd; ++d) {
            D.F0[d] = a.warm ? a.dust_out[d] * s : 0.0f;
            D.G0[d] = a.warm ? a.dust_out[nd + d] * s : 0.0f;
        }
    }
}

// One CTA: F_0(next) = log2 U - LSE2({G_j} u {G_0 - kc}) for the starting G.
__global__ void __launch_bounds__(1024) sk_init_dust_kernel(SkArgs a) {
    __shared__ float sm[32], ss[32];
    DustPtrs D = dust_ptrs(a.dust, a.T);
    int nd = a.mode ? a.T : 1;
    for (int d = 0; d < nd; ++d) {
        int j0 = a.mode ? a.J_off[d] : 0, j1 = a.mode ? a.J_off[d + 1] : a.n_model;
        float m = kNegHuge, s = 0.0f;
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
            float v = a.modC[j].w;
            if (v > m) {
                s = s * ex2(m - v) + 1.0f;
                m = v;
            } else {
                s += ex2(v - m);
            }
        }
        warp_lse_reduce(m, s);
        if ((threadIdx.x & 31) == 0) {
            sm[threadIdx.x >> 5] = m;
            ss[threadIdx.x >> 5] = s;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            Lse2 L;
            L.init(D.G0[d] - a.kc);
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) L.merge(sm[w], ss[w]);
            D.F0n[d] = D.log2U[d] - L.value();
        }
        __syncthreads();
    }
}

// ------------------------------------------------------ staged chunk pipeline
struct Stage2 {
    float4 a[2][kChunk];
    float4 b[2][kChunk];
    uint64_t bar[2];
    int tile;
    int last;
    float red_m[kTPB / 32], red_s[kTPB / 32];
};

// Thread 0 issues the bulk copies of chunk `ch` (one or two arrays) into the
// stage ch & 1.
__device__ __forceinline__ void issue_chunk(Stage2& S, int ch, const float4* srcA, const float4* srcB,
                                            int base, int n_total) {
    int st = ch & 1;
    int n = min(kChunk, n_total - ch * kChunk);
    uint32_t bytes = (uint32_t)n * 16u;
    mbar_expect_tx(&S.bar[st], srcB ? 2u * bytes : bytes);
    bulk_g2s(S.a[st], srcA + base + ch * kChunk, bytes, &S.bar[st]);
    if (srcB) bulk_g2s(S.b[st], srcB + base + ch * kChunk, bytes, &S.bar[st]);
}

__device__ __forceinline__ void block_lse(Stage2& S, float& m, float& s) {
    warp_lse_reduce(m, s);
    int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        S.red_m[w] = m;
        S.red_s[w] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        Lse2 L;
        L.m = kNegHuge;
        L.s = 0.0f;
        for (int k = 0; k < kTPB / 32; ++k) L.merge(S.red_m[k], S.red_s[k]);
        m = L.m;
        s = L.s;
    }
    __syncthreads();
}

__device__ __forceinline__ float block_max(Stage2& S, float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if ((threadIdx.x & 31) == 0) S.red_m[threadIdx.x >> 5] = v;
    __syncthreads();
    float r = S.red_m[0];
    for (int k = 1; k < kTPB / 32; ++k) r = fmaxf(r, S.red_m[k]);
    __syncthreads();
    return r;
}

// Pipeline of one tile: streams n_total spots of (srcA[, srcB]) starting at
// `base` through shared memory and calls body(stage, count, offset) for each
// chunk.
// Returns false (uniformly) when a bounded wait ran out.
template <class Body>
__device__ __forceinline__ bool stream_tile(Stage2& S, uint32_t (&parity)[2], const float4* srcA,
                                            const float4* srcB, int base, int n_total, Body body) {
    int nch = (n_total + kChunk - 1) / kChunk;
    if (threadIdx.x == 0) {
        for (int c = 0; c < nch && c < 2; ++c) issue_chunk(S, c, srcA, srcB, base, n_total);
    }
    bool ok_all = true;
    for (int ch = 0; ch < nch; ++ch) {
        int st = ch & 1;
        bool ok = mbar_wait_bounded(&S.bar[st], parity[st]);
        parity[st] ^= 1u;
        if (ok) body(st, min(kChunk, n_total - ch * kChunk), ch * kChunk);
        if (__syncthreads_or(!ok)) {
            ok_all = false;
            // let copies already in flight land before the CTA leaves
            if (threadIdx.x == 0) {
                for (int c = ch + 1; c < nch && c < ch + 2; ++c) {
                    mbar_wait_bounded(&S.bar[c & 1], parity[c & 1]);
                }
            }
            break;
        }
        if (threadIdx.x == 0 && ch + 2 < nch) issue_chunk(S, ch + 2, srcA, srcB, base, n_total);
    }
    return ok_all;
}

__device__ __forceinline__ void init_stage(Stage2& S) {
    if (threadIdx.x == 0) {
        mbar_init(&S.bar[0], 1);
        mbar_init(&S.bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
}

// Tile queue: thread 0 takes the next tile index; -1 when the queue is empty.
__device__ __forceinline__ int next_tile(Stage2& S, int* counter, int n_tiles) {
    if (threadIdx.x == 0) {
        int t = atomicAdd(counter, 1);
        S.tile = t < n_tiles ? t : -1;
    }
    __syncthreads();
    int t = S.tile;
    __syncthreads();
    return t;
}

// Completion ticket: true in exactly one CTA, the last one to finish.
__device__ __forceinline__ bool last_cta(Stage2& S, int* done) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        int k = atomicAdd(done, 1);
        S.last = (k == (int)gridDim.x - 1);
    }
    __syncthreads();
    bool last = S.last != 0;
    if (last) __threadfence();
    return last;
}

// Online base-2 log-sum-exp over one staged chunk for a row held in registers
// (px, py, pz); A = (c, G), B = (r, lambda).
__device__ __forceinline__ void row_chunk(const float4* __restrict__ A, const float4* __restrict__ B, int n,
                                          float px, float py, float pz, float negK, float& m, float& s) {
    int k = 0;
    for (; k + kGroup <= n; k += kGroup) {
        float v[kGroup];
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
            float4 c = A[k + u];
            float4 r = B[k + u];
            v[u] = fmaf(ray_e2(px, py, pz, c.x, c.y, c.z, r.x, r.y, r.z), negK, c.w);
        }
        float cm = v[0];
#pragma unroll
        for (int u = 1; u < kGroup; ++u) cm = fmaxf(cm, v[u]);
        if (cm > m) {
            s *= ex2(m - cm);
            m = cm;
        }
#pragma unroll
        for (int u = 0; u < kGroup; ++u) s += ex2(v[u] - m);
    }
    for (; k < n; ++k) {
        float4 c = A[k];
        float4 r = B[k];
        float v = fmaf(ray_e2(px, py, pz, c.x, c.y, c.z, r.x, r.y, r.z), negK, c.w);
        if (v > m) {
            s *= ex2(m - v);
            m = v;
        }
        s += ex2(v - m);
    }
}

// Same for a column held in registers (c, r); A = (p, F).
__device__ __forceinline__ void col_chunk(const float4* __restrict__ A, int n, float cx, float cy, float cz,
                                          float rx, float ry, float rz, float negK, float& m, float& s) {
    int k = 0;
    for (; k + kGroup <= n; k += kGroup) {
        float v[kGroup];
#pragma unroll
        for (int u = 0; u < kGroup; ++u) {
            float4 p = A[k + u];
            v[u] = fmaf(ray_e2(p.x, p.y, p.z, cx, cy, cz, rx, ry, rz), negK, p.w);
        }
        float cm = v[0];
#pragma unroll
        for (int u = 1; u < kGroup; ++u) cm = fmaxf(cm, v[u]);
        if (cm > m) {
            s *= ex2(m - cm);
            m = cm;
        }
#pragma unroll
        for (int u = 0; u < kGroup; ++u) s += ex2(v[u] - m);
    }
    for (; k < n; ++k) {
        float4 p = A[k];
        float v = fmaf(ray_e2(p.x, p.y, p.z, cx, cy, cz, rx, ry, rz), negK, p.w);
        if (v > m) {
            s *= ex2(m - v);
            m = v;
        }
        s += ex2(v - m);
    }
}

// --------------------------------------------------------------- row pass
__global__ void __launch_bounds__(kTPB) sk_row_kernel(SkArgs a) {
    __shared__ __align__(128) Stage2 S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_ROW_TILES];
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_ROW_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.row_tiles[tile];
        int t = td.x;
        int i = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int j0 = a.J_off[t], nj = a.J_off[t + 1] - j0;
        float dustv = D.G0[a.mode ? t : 0] - a.kc;
        float4 p = valid ? a.obsP[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float m = dustv, s = 1.0f;
        const float negK = a.negKD2;
        bool ok = stream_tile(S, parity, a.modC, a.modR, j0, nj, [&](int st, int n, int) {
            if (valid) row_chunk(S.a[st], S.b[st], n, p.x, p.y, p.z, negK, m, s);
        });
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        float F = -(m + lg2(s));
        if (valid) a.obsP[i] = make_float4(p.x, p.y, p.z, F);
        // tile partial of LSE2(F_i - kc) for the outlier column update
        float pm = valid ? F - a.kc : kNegHuge, ps = valid ? 1.0f : 0.0f;
        block_lse(S, pm, ps);
        if (threadIdx.x == 0) a.row_part[tile] = make_float2(pm, ps);
    }
    if (!last_cta(S, a.ctrl + CTRL_ROW_DONE)) return;
    // finalise: promote F_0 and compute G_0 from the new F
    if (a.mode) {
        for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
            D.F0[t] = D.F0n[t];
            int4 at = a.ang_tiles[t];
            Lse2 L;
            L.init(D.F0[t] - a.kc);
            for (int k = 0; k < at.y; ++k) {
                float2 pp = a.row_part[at.x + k];
                L.merge(pp.x, pp.y);
            }
            D.G0[t] = D.log2O[t] - L.value();
        }
    } else {
        float m = kNegHuge, s = 0.0f;
        for (int k = threadIdx.x; k < n_tiles; k += blockDim.x) {
            float2 pp = a.row_part[k];
            Lse2 L;
            L.m = m;
            L.s = s;
            L.merge(pp.x, pp.y);
            m = L.m;
            s = L.s;
        }
        block_lse(S, m, s);
        if (threadIdx.x == 0) {
            D.F0[0] = D.F0n[0];
            Lse2 L;
            L.init(D.F0[0] - a.kc);
            L.merge(m, s);
            D.G0[0] = D.log2O[0] - L.value();
        }
    }
    if (threadIdx.x == 0) {
        a.ctrl[CTRL_ROW_NEXT] = 0;
        a.ctrl[CTRL_ROW_DONE] = 0;
    }
}

// ------------------------------------------------------------ column pass
__global__ void __launch_bounds__(kTPB) sk_col_kernel(SkArgs a) {
    __shared__ __align__(128) Stage2 S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_COL_TILES];
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_COL_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.col_tiles[tile];
        int t = td.x;
        int j = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int i0 = a.I_off[t], ni = a.I_off[t + 1] - i0;
        float4 c = valid ? a.modC[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 r = valid ? a.modR[j] : make_float4(0.f, 0.f, 1.f, 0.f);
        float m = D.F0[a.mode ? t : 0], s = 1.0f;  // unmatched-model row, C_0j = 0
        const float negK = a.negKD2;
        bool ok = stream_tile(S, parity, a.obsP, nullptr, i0, ni, [&](int st, int n, int) {
            if (valid) col_chunk(S.a[st], n, c.x, c.y, c.z, r.x, r.y, r.z, negK, m, s);
        });
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        float G = -(m + lg2(s));
        if (valid) a.modC[j] = make_float4(c.x, c.y, c.z, G);
        float pm = valid ? G : kNegHuge, ps = valid ? 1.0f : 0.0f;
        block_lse(S, pm, ps);
        if (threadIdx.x == 0) a.col_part[tile] = make_float2(pm, ps);
    }
    if (!last_cta(S, a.ctrl + CTRL_COL_DONE)) return;
    // finalise: next F_0 from the new G and the current G_0
    if (a.mode) {
        for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
            int4 at = a.ang_tiles[t];
            Lse2 L;
            L.init(D.G0[t] - a.kc);
            for (int k = 0; k < at.w; ++k) {
                float2 pp = a.col_part[at.z + k];
                L.merge(pp.x, pp.y);
            }
            D.F0n[t] = D.log2U[t] - L.value();
        }
    } else {
        float m = kNegHuge, s = 0.0f;
        for (int k = threadIdx.x; k < n_tiles; k += blockDim.x) {
            float2 pp = a.col_part[k];
            Lse2 L;
            L.m = m;
            L.s = s;
            L.merge(pp.x, pp.y);
            m = L.m;
            s = L.s;
        }
        block_lse(S, m, s);
        if (threadIdx.x == 0) {
            Lse2 L;
            L.init(D.G0[0] - a.kc);
            L.merge(m, s);
            D.F0n[0] = D.log2U[0] - L.value();
        }
    }
    if (threadIdx.x == 0) {
        a.ctrl[CTRL_COL_NEXT] = 0;
        a.ctrl[CTRL_COL_DONE] = 0;
    }
}

// ------------------------------------------------------------ row harvest
// Plan read-out per observed spot with the final potentials: argmax over the
// block's model spots and the outlier column (ties to the lowest index, the
// outlier column only when strictly larger), top1 - top2 margin in plan
// units, and the row-marginal error.
__global__ void __launch_bounds__(kTPB) sk_harvest_row_kernel(SkArgs a) {
    __shared__ __align__(128) Stage2 S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_ROW_TILES];
    float my_err = 0.0f;
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_HRV_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.row_tiles[tile];
        int t = td.x;
        int i = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int j0 = a.J_off[t], nj = a.J_off[t + 1] - j0;
        float dustv = D.G0[a.mode ? t : 0] - a.kc;
        float4 p = valid ? a.obsP[i] : make_float4(0.f, 0.f, 0.f, 0.f);
        float m = kNegHuge, s = 0.0f, b1 = kNegHuge, b2 = kNegHuge;
        int arg = -1;
        const float negK = a.negKD2;
        bool ok = stream_tile(S, parity, a.modC, a.modR, j0, nj, [&](int st, int n, int off) {
            if (!valid) return;
            const float4* A = S.a[st];
            const float4* B = S.b[st];
            for (int k = 0; k < n; ++k) {
                float4 c = A[k];
                float4 r = B[k];
                float v = fmaf(ray_e2(p.x, p.y, p.z, c.x, c.y, c.z, r.x, r.y, r.z), negK, c.w);
                if (v > m) {
                    s = s * ex2(m - v) + 1.0f;
                    m = v;
                } else {
                    s += ex2(v - m);
                }
                if (v > b1) {  // strict: ties keep the lowest index
                    b2 = b1;
                    b1 = v;
                    arg = j0 + off + k;
                } else if (v > b2) {
                    b2 = v;
                }
            }
        });
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        if (valid) {
            if (dustv > b1) {  // outlier column last, only when strictly larger
                b2 = b1;
                b1 = dustv;
                arg = -1;
            } else if (dustv > b2) {
                b2 = dustv;
            }
            // row sum including the outlier column
            Lse2 L;
            L.m = m;
            L.s = s;
            L.merge(dustv, 1.0f);
            float F = p.w;
            float rs = ex2(F + L.value());
            my_err = fmaxf(my_err, fabsf(rs - 1.0f));
            if (a.assign) a.assign[i] = arg;
            if (a.margin) a.margin[i] = ex2(F + b1) - (b2 > kNegHuge ? ex2(F + b2) : 0.0f);
        }
    }
    float e = block_max(S, my_err);
    if (threadIdx.x == 0) atomicMax((int*)(D.err + 2), __float_as_int(e));  // non-negative floats
    if (!last_cta(S, a.ctrl + CTRL_HRV_DONE)) return;
    if (threadIdx.x == 0) {
        float err = __int_as_float(*(int*)(D.err + 2));
        int nd = a.mode ? a.T : 1;
        for (int d = 0; d < nd; ++d) {
            if (D.log2U[d] > kNegHuge) err = fmaxf(err, fabsf(ex2(D.F0[d] - D.F0n[d]) - 1.0f));
        }
        D.err[0] = err;
        a.ctrl[CTRL_HRV_NEXT] = 0;
        a.ctrl[CTRL_HRV_DONE] = 0;
    }
}

// --------------------------------------------------------- column harvest
// Column mass q_j = sum_i Q_ij over observed rows and the column-marginal
// error with the final potentials.
__global__ void __launch_bounds__(kTPB) sk_harvest_col_kernel(SkArgs a) {
    __shared__ __align__(128) Stage2 S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_COL_TILES];
    float my_err = 0.0f;
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_HCOL_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.col_tiles[tile];
        int t = td.x;
        int j = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int i0 = a.I_off[t], ni = a.I_off[t + 1] - i0;
        float4 c = valid ? a.modC[j] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 r = valid ? a.modR[j] : make_float4(0.f, 0.f, 1.f, 0.f);
        float m = kNegHuge, s = 0.0f;
        const float negK = a.negKD2;
        bool ok = stream_tile(S, parity, a.obsP, nullptr, i0, ni, [&](int st, int n, int) {
            if (valid) col_chunk(S.a[st], n, c.x, c.y, c.z, r.x, r.y, r.z, negK, m, s);
        });
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        if (valid) {
            float qj = s > 0.0f ? ex2(c.w + m + lg2(s)) : 0.0f;
            if (a.q) a.q[j] = qj;
            float q0 = ex2(c.w + D.F0[a.mode ? t : 0]);
            my_err = fmaxf(my_err, fabsf(qj + q0 - 1.0f));
        }
    }
    float e = block_max(S, my_err);
    if (threadIdx.x == 0) atomicMax((int*)(D.err + 3), __float_as_int(e));
    if (!last_cta(S, a.ctrl + CTRL_HCOL_DONE)) return;
    if (threadIdx.x == 0) {
        D.err[1] = __int_as_float(*(int*)(D.err + 3));
        a.ctrl[CTRL_HCOL_NEXT] = 0;
        a.ctrl[CTRL_HCOL_DONE] = 0;
    }
}

// ---------------------------------------------------------------- finish
__global__ void sk_finish_kernel(SkArgs a, int have_rows, int have_cols) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    bool bad = false;
    if (k < a.n_obs) {
        float v = a.obsP[k].w;
        bad |= !isfinite(v);
        a.f[k] = v * a.to_user;
    }
    if (k < a.n_model) {
        float v = a.modC[k].w;
        bad |= !isfinite(v);
        a.g[k] = v * a.to_user;
    }
    if (k == 0) {
        DustPtrs D = dust_ptrs(a.dust, a.T);
        int nd = a.mode ? a.T : 1;
        if (a.dust_out) {
            for (int d = 0; d < nd; ++d) {
                a.dust_out[d] = D.F0[d] * a.to_user;
                a.dust_out[nd + d] = D.G0[d] * a.to_user;
            }
        }
        if (a.marg_err) {
            a.marg_err[0] = have_rows ? D.err[0] : -1.0f;
            a.marg_err[1] = have_cols ? D.err[1] : -1.0f;
        }
    }
    if (bad) set_status(a.ctrl, LAUE_ERR_NUMERIC);
}

__global__ void sk_clear_err_kernel(SkArgs a) {
    DustPtrs D = dust_ptrs(a.dust, a.T);
    D.err[0] = D.err[1] = D.err[2] = D.err[3] = 0.0f;
}

cudaError_t sinkhorn_run(const SkArgs& a, const SkLaunch& l, int n_iter, bool want_rows, bool want_cols,
                         cudaStream_t s) {
    int nmax = a.n_obs > a.n_model ? a.n_obs : a.n_model;
    int pack_blocks = (nmax + 255) / 256;
    if (pack_blocks < 1) pack_blocks = 1;
    sk_schedule_kernel<<<1, 1024, 0, s>>>(a);
    sk_pack_kernel<<<pack_blocks, 256, 0, s>>>(a);
    sk_init_dust_kernel<<<1, 1024, 0, s>>>(a);
    for (int it = 0; it < n_iter; ++it) {
        sk_row_kernel<<<l.row_grid, kTPB, 0, s>>>(a);
        sk_col_kernel<<<l.col_grid, kTPB, 0, s>>>(a);
    }
    if (want_rows || want_cols) sk_clear_err_kernel<<<1, 1, 0, s>>>(a);
    if (want_rows) sk_harvest_row_kernel<<<l.hrv_grid, kTPB, 0, s>>>(a);
    if (want_cols) sk_harvest_col_kernel<<<l.hcol_grid, kTPB, 0, s>>>(a);
    sk_finish_kernel<<<pack_blocks, 256, 0, s>>>(a, want_rows ? 1 : 0, want_cols ? 1 : 0);
    return cudaGetLastError();
}

int sinkhorn_occupancy(int* row_blocks_per_sm, int* col_blocks_per_sm) {
    int r = 0, c = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, sk_row_kernel, kTPB, 0) != cudaSuccess) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, sk_col_kernel, kTPB, 0) != cudaSuccess) return -1;
    *row_blocks_per_sm = r;
    *col_blocks_per_sm = c;
    return 0;
}

}  // namespace laue
