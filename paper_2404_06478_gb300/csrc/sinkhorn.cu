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
// Unbalanced mode (Appendix "Optimal transport variants", Algorithm
// UnbalancedOT): no dustbins, and each balanced update is scaled by
// tau_row = kappa / (kappa + eps) (rows) or tau_col = lambda / (lambda + eps)
// (columns), the log-domain form of the exponents of the scaling updates.
//
// Layout.  The workspace holds the spots as pairs: each angle block is padded
// to an even count and element pairs (a, b) are interleaved into float4 rows
// such as {x_a, x_b, y_a, y_b}, so one 16-byte shared-memory load yields two
// packed operands for the f32x2 FMA/ADD/MUL instructions.  Model centres and
// rays are stored negated (d = p + (-c), e = d/|d| + (-r)).  Padding entries
// carry a potential of -3e38, which makes their plan entries exactly 0.
//
// Passes.  Each pass is one persistent launch over all angle blocks: CTAs pull
// tiles (angle t, first pair, count) from a queue the scheduler kernel built
// on the device in longest-block-first order.  A thread keeps one PAIR of rows
// (row pass) or columns (column pass) in registers and streams the other side
// of its angle block, as pairs, through shared memory in chunks loaded by the
// bulk-copy engine (cp.async.bulk) into a two-stage mbarrier pipeline: every
// staged pair feeds 4 pair evaluations.  The log-sum-exps are online, in
// groups of 4 staged pairs (8 values) per max/rescale step.  The last CTA to
// finish a pass combines the per-tile partial log-sum-exps into the dustbin
// potentials:
//   end of a row pass:    F_0 <- F_0(next), then G_0 from the new F and F_0
//   end of a column pass: F_0(next) from the new G and G_0
// which reproduces the sequential order of the algorithm exactly.
#include "pairs.cuh"

namespace laue {

// ---------------------------------------------------------------- scheduler
// One CTA.  Pair offsets of the padded blocks, row and column tile queues
// (angles by descending work, tiles of one angle contiguous), per-angle tile
// ranges, log2 masses of the dustbins; clears the queue counters.
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
        int ip = 0, jp = 0;
        for (int t = 0; t < T; ++t) {
            a.I2_off[t] = ip;
            a.J2_off[t] = jp;
            ip += (a.I_off[t + 1] - a.I_off[t] + 1) / 2;
            jp += (a.J_off[t + 1] - a.J_off[t] + 1) / 2;
        }
        a.I2_off[T] = ip;
        a.J2_off[T] = jp;
        int go = 0, gm = 0;
        for (int t = 0; t < T; ++t) {
            a.obs_gbase[t] = go;
            a.mod_gbase[t] = gm;
            go += (a.I2_off[t + 1] - a.I2_off[t] + kGran - 1) / kGran;
            gm += (a.J2_off[t + 1] - a.J2_off[t] + kGran - 1) / kGran;
        }
        a.obs_gbase[T] = go;
        a.mod_gbase[T] = gm;
        int nr = 0, nc = 0;
        for (int k = 0; k < T; ++k) {
            int t = order_r[k];
            int np = (a.I_off[t + 1] - a.I_off[t] + 1) / 2;
            int cnt = (np + a.tile_rows - 1) / a.tile_rows;
            a.ang_tiles[t].x = nr;
            a.ang_tiles[t].y = cnt;
            nr += cnt;
        }
        for (int k = 0; k < T; ++k) {
            int t = order_c[k];
            int np = (a.J_off[t + 1] - a.J_off[t] + 1) / 2;
            int cnt = (np + a.tile_cols - 1) / a.tile_cols;
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
        for (int k = CTRL_ROW_NEXT; k <= CTRL_GEN_DONE; ++k)
            if (k != CTRL_N_ROW_TILES && k != CTRL_N_COL_TILES && k != CTRL_FWD_TOTAL) a.ctrl[k] = 0;
    }
    __syncthreads();
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int4 at = a.ang_tiles[t];
        int i0 = a.I2_off[t], ni = a.I2_off[t + 1] - i0;
        for (int k = 0; k < at.y; ++k) {
            int idx = at.x + k;
            if (idx < a.max_row_tiles)
                a.row_tiles[idx] = make_int4(t, i0 + k * a.tile_rows, min(a.tile_rows, ni - k * a.tile_rows), 0);
        }
        int j0 = a.J2_off[t], nj = a.J2_off[t + 1] - j0;
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

// ------------------------------------------------------- spatial order
// Within each angle block the spots are ranked by a 23-bit key of their
// direction (observed: p / |p|, model: the ray r): the cube-map face of the
// direction and the Morton interleave of its two in-face coordinates at 10
// bits each.  Spots close on a detector get close ranks, so runs of kGran
// pairs are spatially compact and their cones are narrow.  One CTA sorts one
// block (LSD radix sort, 4-bit digits, stable: ties keep the caller's order).
__device__ __forceinline__ unsigned spread10(unsigned v) {
    v &= 1023u;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

__device__ __forceinline__ unsigned direction_key(float x, float y, float z) {
    float ax = fabsf(x), ay = fabsf(y), az = fabsf(z);
    int face;
    float m, u, v;
    if (ax >= ay && ax >= az) {
        face = x < 0.0f;
        m = ax;
        u = y;
        v = z;
    } else if (ay >= az) {
        face = 2 + (y < 0.0f);
        m = ay;
        u = x;
        v = z;
    } else {
        face = 4 + (z < 0.0f);
        m = az;
        u = x;
        v = y;
    }
    if (!(m > 0.0f)) return 0u;
    unsigned qu = (unsigned)fminf(1023.0f, fmaxf(0.0f, (u / m + 1.0f) * 512.0f));
    unsigned qv = (unsigned)fminf(1023.0f, fmaxf(0.0f, (v / m + 1.0f) * 512.0f));
    return ((unsigned)face << 20) | spread10(qu) | (spread10(qv) << 1);
}

constexpr int kSortThreads = 1024;

// Blocks 0..T-1 sort the observed blocks, T..2T-1 the model blocks.
__global__ void __launch_bounds__(kSortThreads) sk_sort_kernel(SkArgs a) {
    __shared__ int cnt[kSortThreads / 32][16];
    __shared__ int dbase[16];
    const bool mod = (int)blockIdx.x >= a.T;
    const int t = mod ? blockIdx.x - a.T : blockIdx.x;
    const int* off = mod ? a.J_off : a.I_off;
    const int b0 = off[t], n = off[t + 1] - b0;
    const size_t nsp = (size_t)a.n_obs + a.n_model + 2;
    const size_t side0 = mod ? (size_t)a.n_obs + 1 : 0;
    unsigned* kbuf[2] = {a.sort_key + side0 + b0, a.sort_key + nsp + side0 + b0};
    int* ibuf[2] = {a.sort_idx + side0 + b0, a.sort_idx + nsp + side0 + b0};
    int* perm = (mod ? a.mod_perm : a.obs_perm) + b0;
    int* pos = (mod ? a.mod_pos : a.obs_pos) + b0;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int l = threadIdx.x; l < n; l += kSortThreads) {
        float4 v = mod ? a.mod_r[b0 + l] : a.obs_p[b0 + l];
        kbuf[0][l] = direction_key(v.x, v.y, v.z);
        ibuf[0][l] = l;
    }
    __syncthreads();
    for (int pass = 0; pass < 6; ++pass) {
        const unsigned* sk = kbuf[pass & 1];
        const int* si = ibuf[pass & 1];
        unsigned* dk = kbuf[(pass + 1) & 1];
        int* di = ibuf[(pass + 1) & 1];
        const int shift = 4 * pass;
        if (threadIdx.x < 16) dbase[threadIdx.x] = 0;
        __syncthreads();
        for (int l = threadIdx.x; l < n; l += kSortThreads) atomicAdd(&dbase[(sk[l] >> shift) & 15u], 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = 0;
            for (int d = 0; d < 16; ++d) {
                int c = dbase[d];
                dbase[d] = acc;
                acc += c;
            }
        }
        __syncthreads();
        for (int c0 = 0; c0 < n; c0 += kSortThreads) {
            int l = c0 + threadIdx.x;
            bool valid = l < n;
            unsigned key = valid ? sk[l] : 0u;
            int idx = valid ? si[l] : 0;
            int d = valid ? (int)((key >> shift) & 15u) : 16;
            unsigned mine = 0u;
            for (int v = 0; v < 16; ++v) {
                unsigned b = __ballot_sync(0xffffffffu, d == v);
                if (d == v) mine = b;
                if (lane == 0) cnt[w][v] = __popc(b);
            }
            __syncthreads();
            if (threadIdx.x < 16) {
                int acc = dbase[threadIdx.x];
                for (int ww = 0; ww < kSortThreads / 32; ++ww) {
                    int c = cnt[ww][threadIdx.x];
                    cnt[ww][threadIdx.x] = acc;
                    acc += c;
                }
                dbase[threadIdx.x] = acc;
            }
            __syncthreads();
            if (valid) {
                int p = cnt[w][d] + __popc(mine & ((1u << lane) - 1u));
                dk[p] = key;
                di[p] = idx;
            }
            __syncthreads();
        }
    }
    // six passes: the sorted order is back in buffer 0
    for (int l = threadIdx.x; l < n; l += kSortThreads) {
        int idx = ibuf[0][l];
        perm[l] = b0 + idx;
        pos[idx] = l;
    }
}

// Cone of each granule (kGran pairs of one block), one warp per granule:
// axis = normalised mean direction, half-angle = largest angle from it, and
// the smallest |p| (observed) or largest |c| (model).
__global__ void __launch_bounds__(256) sk_cone_kernel(SkArgs a) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    int n_go = a.obs_gbase[a.T], n_gm = a.mod_gbase[a.T];
    if (warp >= n_go + n_gm) return;
    const bool mod = warp >= n_go;
    const int g = mod ? warp - n_go : warp;
    const int* gb = mod ? a.mod_gbase : a.obs_gbase;
    const int t = block_of(gb, a.T, g);
    const int* off = mod ? a.J_off : a.I_off;
    const int* poff = mod ? a.J2_off : a.I2_off;
    const int nspots = off[t + 1] - off[t];
    const int l0 = 2 * kGran * (g - gb[t]);            // first spot rank of the granule
    const int l1 = min(nspots, l0 + 2 * kGran);
    float d[2 * kGran / 32][3];
    float sx = 0.f, sy = 0.f, sz = 0.f, ext = mod ? 0.0f : 3.0e38f;
    int cntv = 0;
    for (int k = 0; k < 2 * kGran / 32; ++k) {
        int l = l0 + lane + 32 * k;
        d[k][0] = d[k][1] = d[k][2] = 0.0f;
        if (l >= l1) continue;
        int q = poff[t] + (l >> 1), ln = l & 1;
        float x, y, z;
        if (mod) {
            float4 Z = a.modZ[q], W = a.modW[q], X = a.modX[q], Y = a.modY[q];
            x = -(ln ? Z.y : Z.x);
            y = -(ln ? Z.w : Z.z);
            z = -(ln ? W.y : W.x);
            float cx = ln ? X.y : X.x, cy = ln ? X.w : X.z, cz = ln ? Y.y : Y.x;
            ext = fmaxf(ext, sqrtf(cx * cx + cy * cy + cz * cz));
        } else {
            float4 X = a.obsX[q], Y = a.obsY[q];
            x = ln ? X.y : X.x;
            y = ln ? X.w : X.z;
            z = ln ? Y.y : Y.x;
            float r = sqrtf(x * x + y * y + z * z);
            ext = fminf(ext, r);
        }
        float r = rsqrtf(fmaxf(x * x + y * y + z * z, 1e-30f));
        d[k][0] = x * r;
        d[k][1] = y * r;
        d[k][2] = z * r;
        sx += d[k][0];
        sy += d[k][1];
        sz += d[k][2];
        ++cntv;
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_xor_sync(0xffffffffu, sx, o);
        sy += __shfl_xor_sync(0xffffffffu, sy, o);
        sz += __shfl_xor_sync(0xffffffffu, sz, o);
        ext = mod ? fmaxf(ext, __shfl_xor_sync(0xffffffffu, ext, o)) : fminf(ext, __shfl_xor_sync(0xffffffffu, ext, o));
    }
    float n2 = sx * sx + sy * sy + sz * sz;
    float ax = 0.f, ay = 0.f, az = 1.f;
    bool degenerate = !(n2 > 1e-12f);
    if (!degenerate) {
        float r = rsqrtf(n2);
        ax = sx * r;
        ay = sy * r;
        az = sz * r;
    }
    float beta = 0.0f;
    for (int k = 0; k < 2 * kGran / 32; ++k) {
        int l = l0 + lane + 32 * k;
        if (l >= l1) continue;
        beta = fmaxf(beta, angle_between(ax, ay, az, d[k][0], d[k][1], d[k][2]));
    }
    for (int o = 16; o > 0; o >>= 1) beta = fmaxf(beta, __shfl_xor_sync(0xffffffffu, beta, o));
    if (lane == 0) {
        if (degenerate) beta = 3.2f;  // no bound
        float4* cone = mod ? a.mod_cone : a.obs_cone;
        float* ex = mod ? a.mod_ext : a.obs_ext;
        cone[g] = make_float4(ax, ay, az, beta + 1e-5f);
        ex[g] = ext;
    }
}

// ------------------------------------------------------------------- pack
// Pair-interleaved workspace copies; F, G from the caller's potentials on a
// warm start, else 0.  The thread of the last element of an odd block also
// writes the padding slot.
__global__ void sk_pack_kernel(SkArgs a) {
    const float s = 1.0f / a.to_user;  // mm^2 -> base-2 internal units
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < a.n_obs) {
        int t = block_of(a.I_off, a.T, k);
        int l = a.obs_pos[k];  // rank of the spot in its block's spatial order
        int q = a.I2_off[t] + (l >> 1), lane = l & 1;
        float4 p = a.obs_p[k];
        float* X = (float*)&a.obsX[q];
        float* Y = (float*)&a.obsY[q];
        X[lane] = p.x;
        X[2 + lane] = p.y;
        Y[lane] = p.z;
        Y[2 + lane] = a.warm ? a.f[k] * s : 0.0f;
        if (lane == 0 && l + 1 == a.I_off[t + 1] - a.I_off[t]) {
            X[1] = 0.0f;
            X[3] = 0.0f;
            Y[1] = kPadFar;
            Y[3] = kNegHuge;
        }
    }
    if (k < a.n_model) {
        int t = block_of(a.J_off, a.T, k);
        int l = a.mod_pos[k];
        int q = a.J2_off[t] + (l >> 1), lane = l & 1;
        float4 c = a.mod_c[k];
        float4 r = a.mod_r[k];
        float* X = (float*)&a.modX[q];
        float* Y = (float*)&a.modY[q];
        float* Z = (float*)&a.modZ[q];
        float* W = (float*)&a.modW[q];
        X[lane] = -c.x;
        X[2 + lane] = -c.y;
        Y[lane] = -c.z;
        Y[2 + lane] = a.warm ? a.g[k] * s : 0.0f;
        Z[lane] = -r.x;
        Z[2 + lane] = -r.y;
        W[lane] = -r.z;
        int det = a.mod_s ? (int)a.mod_s[k].w : -1;
        W[2 + lane] = (det >= 0 && det < a.n_det) ? a.negK_det[det] : a.negKD2;
        if (lane == 0 && l + 1 == a.J_off[t + 1] - a.J_off[t]) {
            X[1] = 0.0f;
            X[3] = 0.0f;
            Y[1] = 0.0f;
            Y[3] = kNegHuge;
            Z[1] = 0.0f;
            Z[3] = 0.0f;
            W[1] = -1.0f;
            W[3] = 0.0f;
        }
    }
    if (k == 0) {
        DustPtrs D = dust_ptrs(a.dust, a.T);
        int nd = a.mode ? a.T : 1;
        for (int d = 0; d < nd; ++d) {
            D.F0[d] = (a.warm && a.dust_out) ? a.dust_out[d] * s : 0.0f;
            D.G0[d] = (a.warm && a.dust_out) ? a.dust_out[nd + d] * s : 0.0f;
        }
    }
}

// One CTA: F_0(next) = log2 U - LSE2({G_j} u {G_0 - kc}) for the starting G.
__global__ void __launch_bounds__(1024) sk_init_dust_kernel(SkArgs a) {
    __shared__ float sm[32], ss[32];
    DustPtrs D = dust_ptrs(a.dust, a.T);
    int nd = a.mode ? a.T : 1;
    for (int d = 0; d < nd; ++d) {
        int q0 = a.mode ? a.J2_off[d] : 0, q1 = a.mode ? a.J2_off[d + 1] : a.J2_off[a.T];
        float m = kNegHuge, s = 0.0f;
        for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {
            float4 y = a.modY[q];
            for (int lane = 0; lane < 2; ++lane) {
                float v = lane ? y.w : y.z;
                if (v <= kNegHuge) continue;  // padding
                if (v > m) {
                    s = s * ex2(m - v) + 1.0f;
                    m = v;
                } else {
                    s += ex2(v - m);
                }
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

// Row pair (two observed spots) against the staged model pairs of one chunk.
struct RowPair {
    f2 pxa, pya, pza, pxb, pyb, pzb;
    RowLse A, B;
};

__device__ __forceinline__ void col_chunk(ColPair& C, const float4* __restrict__ sX, const float4* __restrict__ sY,
                                          int n) {
    int k = 0;
    for (; k + kGroup <= n; k += kGroup) {
        f2 va[kGroup], vb[kGroup];
#pragma unroll
        for (int g = 0; g < kGroup; ++g) {
            ulonglong2 X = *(const ulonglong2*)&sX[k + g];
            ulonglong2 Y = *(const ulonglong2*)&sY[k + g];
            va[g] = pair_v2(X.x, X.y, Y.x, C.ncxa, C.ncya, C.ncza, C.nrxa, C.nrya, C.nrza, C.ka, Y.y);
            vb[g] = pair_v2(X.x, X.y, Y.x, C.ncxb, C.ncyb, C.nczb, C.nrxb, C.nryb, C.nrzb, C.kb, Y.y);
        }
        C.A.add4(va);
        C.B.add4(vb);
    }
    for (; k < n; ++k) {
        ulonglong2 X = *(const ulonglong2*)&sX[k];
        ulonglong2 Y = *(const ulonglong2*)&sY[k];
        C.A.add1(pair_v2(X.x, X.y, Y.x, C.ncxa, C.ncya, C.ncza, C.nrxa, C.nrya, C.nrza, C.ka, Y.y));
        C.B.add1(pair_v2(X.x, X.y, Y.x, C.ncxb, C.ncyb, C.nczb, C.nrxb, C.nryb, C.nrzb, C.kb, Y.y));
    }
}

// Fast path of the passes: the staged potentials are shifted by the block's
// maximum (prep step), so every exponent is <= 0 and the sums need no running
// maximum: per staged pair, 2 x 13 packed instructions, 4 MUFU ex2 and 2
// packed adds for 4 pair evaluations.
__device__ __forceinline__ void row_chunk_sum(const RowPair& R, const float4* __restrict__ sX,
                                              const float4* __restrict__ sY, const float4* __restrict__ sZ,
                                              const float4* __restrict__ sW, int n, f2& Sa, f2& Sb) {
#pragma unroll 4
    for (int k = 0; k < n; ++k) {
        ulonglong2 X = *(const ulonglong2*)&sX[k];
        ulonglong2 Y = *(const ulonglong2*)&sY[k];
        ulonglong2 Z = *(const ulonglong2*)&sZ[k];
        ulonglong2 W = *(const ulonglong2*)&sW[k];
        f2 va = pair_v2(R.pxa, R.pya, R.pza, X.x, X.y, Y.x, Z.x, Z.y, W.x, W.y, Y.y);
        f2 vb = pair_v2(R.pxb, R.pyb, R.pzb, X.x, X.y, Y.x, Z.x, Z.y, W.x, W.y, Y.y);
        Sa = add2(Sa, pk(ex2(lo(va)), ex2(hi(va))));
        Sb = add2(Sb, pk(ex2(lo(vb)), ex2(hi(vb))));
    }
}

__device__ __forceinline__ void col_chunk_sum(const ColPair& C, const float4* __restrict__ sX,
                                              const float4* __restrict__ sY, int n, f2& Sa, f2& Sb) {
#pragma unroll 4
    for (int k = 0; k < n; ++k) {
        ulonglong2 X = *(const ulonglong2*)&sX[k];
        ulonglong2 Y = *(const ulonglong2*)&sY[k];
        f2 va = pair_v2(X.x, X.y, Y.x, C.ncxa, C.ncya, C.ncza, C.nrxa, C.nrya, C.nrza, C.ka, Y.y);
        f2 vb = pair_v2(X.x, X.y, Y.x, C.ncxb, C.ncyb, C.nczb, C.nrxb, C.nryb, C.nrzb, C.kb, Y.y);
        Sa = add2(Sa, pk(ex2(lo(va)), ex2(hi(va))));
        Sb = add2(Sb, pk(ex2(lo(vb)), ex2(hi(vb))));
    }
}

constexpr float kTinySum = 1.0e-30f;  // below ~2^-100 the fast sum is recomputed exactly

// Exact row log-sum-exp from global memory (running maximum), for rows whose
// shifted sum underflowed.
__device__ float row_exact(const SkArgs& a, int t, f2 px, f2 py, f2 pz, float dustv) {
    atomicAdd((unsigned*)a.ctrl + CTRL_EXACT_ROWS, 1u);
    RowLse L;
    L.init(dustv);
    for (int q = a.J2_off[t]; q < a.J2_off[t + 1]; ++q) {
        float4 x = a.modX[q], y = a.modY[q], z = a.modZ[q], w = a.modW[q];
        L.add1(pair_v2(px, py, pz, pk(x.x, x.y), pk(x.z, x.w), pk(y.x, y.y), pk(z.x, z.y), pk(z.z, z.w),
                       pk(w.x, w.y), pk(w.z, w.w), pk(y.z, y.w)));
    }
    return L.value();
}

__device__ float col_exact(const SkArgs& a, int t, f2 ncx, f2 ncy, f2 ncz, f2 nrx, f2 nry, f2 nrz, float dz, f2 K2) {
    atomicAdd((unsigned*)a.ctrl + CTRL_EXACT_COLS, 1u);
    RowLse L;
    L.init(dz);
    for (int q = a.I2_off[t]; q < a.I2_off[t + 1]; ++q) {
        float4 x = a.obsX[q], y = a.obsY[q];
        L.add1(pair_v2(pk(x.x, x.y), pk(x.z, x.w), pk(y.x, y.y), ncx, ncy, ncz, nrx, nry, nrz, K2, pk(y.z, y.w)));
    }
    return L.value();
}

// Per-angle maximum of the potentials written by a pass, from the per-tile
// partial log-sum-exps (their running maxima).
__device__ void block_maxima(const float2* part, const int4* ang, int T, bool rows, float add, float* out) {
    for (int t = threadIdx.x; t < T; t += blockDim.x) {
        int4 at = ang[t];
        int first = rows ? at.x : at.z, cnt = rows ? at.y : at.w;
        float m = kNegHuge;
        for (int k = 0; k < cnt; ++k) m = fmaxf(m, part[first + k].x);
        out[t] = m > kNegHuge ? m + add : kNegHuge;
    }
}

// --------------------------------------------------------------- row pass
template <int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) sk_row_kernel(SkArgs a) {
    __shared__ __align__(128) Stage S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_ROW_TILES];
    const Srcs src{{a.modX, a.modY, a.modZ, a.modW}, 4};
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_ROW_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.row_tiles[tile];
        int t = td.x;
        int q = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int ni = a.I_off[t + 1] - a.I_off[t];
        bool vb = valid && 2 * (q - a.I2_off[t]) + 1 < ni;
        int j0 = a.J2_off[t], nj = a.J2_off[t + 1] - j0;
        const bool ub = a.mode == 2;  // unbalanced OT: no dustbins, scaled update
        float dustv = ub ? kNegHuge : D.G0[a.mode ? t : 0] - a.kc;
        float4 X = valid ? a.obsX[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 Y = valid ? a.obsY[q] : make_float4(0.f, 0.f, kPadFar, kPadFar);
        RowPair R;
        R.pxa = dup(X.x);
        R.pya = dup(X.z);
        R.pza = dup(Y.x);
        R.pxb = dup(X.y);
        R.pyb = dup(X.w);
        R.pzb = dup(Y.y);
        const float shift = ub ? D.Gmax[t] : fmaxf(D.Gmax[t], dustv);
        f2 Sa = pk(ub ? 0.0f : ex2(dustv - shift), 0.0f), Sb = Sa;
        auto prep = [&](int st, int n) {
            for (int k = threadIdx.x; k < n; k += TPB) {
                float4& y = S.s[1][st][k];
                y.z -= shift;
                y.w -= shift;
            }
        };
        // the granules of a staged chunk selected by mask
        auto body = [&](int st, int n, int, int mask = (1 << kParts) - 1) {
            if (!valid) return;
            for_each_run(mask, n, [&](int h, int m) {
                row_chunk_sum(R, S.s[0][st] + h, S.s[1][st] + h, S.s[2][st] + h, S.s[3][st] + h, m, Sa, Sb);
            });
        };
        // the model granules this tile of observed spots can see (exact underflow skipping)
        const int nch = (nj + kChunk - 1) / kChunk;
        const bool use_list = a.skip && nch > 0 && nch <= kMaxList;
        int n_list = nch;
        if (use_list) {
            const Cone O = tile_cone(a.obs_cone, a.obs_ext, a.obs_gbase[t], a.I2_off[t], td.y, td.z, true);
            const float K = a.skipK;  // the smallest cost factor of any spot
            const int mg = a.mod_gbase[t], ng = (nj + kGran - 1) / kGran;
            n_list = build_chunk_list(S, nch, [&](int c) {
                int m = 0;
                for (int hh = 0; hh < kParts; ++hh)
                    if (kParts * c + hh < ng &&
                        min_scaled_cost(O, load_cone(a.mod_cone, a.mod_ext, mg + kParts * c + hh), K) <= kSkipLog2)
                        m |= 1 << hh;
                return m;
            });
        }
        bool ok = use_list ? stream_list_prep(S, parity, src, j0, nj, n_list, prep, body)
                           : stream_tile_prep(S, parity, src, j0, nj, prep, body);
        if (threadIdx.x == 0) {
            long long np = 0;
            if (use_list)
                for (int c = 0; c < n_list; ++c) np += list_pairs(S.list[c] & 0xffffff, (int)((unsigned)S.list[c] >> 24), nj);
            else
                np = nj;
            atomicAdd((unsigned long long*)(a.ctrl + CTRL_SK_PAIRS), (unsigned long long)(4LL * td.z * np));
        }
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        float sa = lo(Sa) + hi(Sa), sb = lo(Sb) + hi(Sb);
        float Fa = valid ? (sa > kTinySum ? -(shift + lg2(sa)) : -row_exact(a, t, R.pxa, R.pya, R.pza, dustv)) : 0.0f;
        float Fb = vb ? (sb > kTinySum ? -(shift + lg2(sb)) : -row_exact(a, t, R.pxb, R.pyb, R.pzb, dustv)) : 0.0f;
        if (ub) {  // Algorithm UnbalancedOT: the balanced update raised to kappa / (kappa + eps)
            Fa = nj > 0 ? a.tau_row * Fa : 0.0f;
            Fb = nj > 0 ? a.tau_row * Fb : 0.0f;
        }
        if (valid) *(float2*)&a.obsY[q].z = make_float2(Fa, vb ? Fb : kNegHuge);
        // tile partial of LSE2(F_i - kc) for the outlier column update
        float pm = kNegHuge, ps = 0.0f;
        if (valid) {
            pm = Fa - a.kc;
            ps = 1.0f;
            if (vb) lse_merge_into(pm, ps, Fb - a.kc, 1.0f);
        }
        block_lse(S, pm, ps);
        if (threadIdx.x == 0) a.row_part[tile] = make_float2(pm, ps);
    }
    if (!last_cta(S, a.ctrl + CTRL_ROW_DONE)) return;
    // finalise: promote F_0 and compute G_0 from the new F
    if (a.mode == 2) {
        // no dustbins
    } else if (a.mode) {
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
            lse_merge_into(m, s, pp.x, pp.y);
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
    block_maxima(a.row_part, a.ang_tiles, a.T, true, a.kc, D.Fmax);
    if (threadIdx.x == 0) {
        a.ctrl[CTRL_ROW_NEXT] = 0;
        a.ctrl[CTRL_ROW_DONE] = 0;
    }
}

// ------------------------------------------------------------ column pass
template <int TPB, int MINB>
__global__ void __launch_bounds__(TPB, MINB) sk_col_kernel(SkArgs a) {
    __shared__ __align__(128) Stage S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_COL_TILES];
    const Srcs src{{a.obsX, a.obsY, nullptr, nullptr}, 2};
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_COL_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.col_tiles[tile];
        int t = td.x;
        int q = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int nj = a.J_off[t + 1] - a.J_off[t];
        bool vb = valid && 2 * (q - a.J2_off[t]) + 1 < nj;
        int i0 = a.I2_off[t], ni = a.I2_off[t + 1] - i0;
        ColPair C;
        if (valid) load_col_pair(a, q, C);
        const bool ub = a.mode == 2;
        float dz = ub ? kNegHuge : D.F0[a.mode ? t : 0];  // unmatched-model row, C_0j = 0
        const float shift = ub ? D.Fmax[t] : fmaxf(D.Fmax[t], dz);
        f2 Sa = pk(ub ? 0.0f : ex2(dz - shift), 0.0f), Sb = Sa;
        auto prep = [&](int st, int n) {
            for (int k = threadIdx.x; k < n; k += TPB) {
                float4& y = S.s[1][st][k];
                y.z -= shift;
                y.w -= shift;
            }
        };
        auto body = [&](int st, int n, int, int mask = (1 << kParts) - 1) {
            if (!valid) return;
            for_each_run(mask, n, [&](int h, int m) { col_chunk_sum(C, S.s[0][st] + h, S.s[1][st] + h, m, Sa, Sb); });
        };
        // the observed granules this tile of model spots can see (exact underflow skipping)
        const int nch = (ni + kChunk - 1) / kChunk;
        const bool use_list = a.skip && nch > 0 && nch <= kMaxList;
        int n_list = nch;
        if (use_list) {
            const Cone M = tile_cone(a.mod_cone, a.mod_ext, a.mod_gbase[t], a.J2_off[t], td.y, td.z, false);
            const float K = a.skipK;  // the smallest cost factor of any spot
            const int og = a.obs_gbase[t], ng = (ni + kGran - 1) / kGran;
            n_list = build_chunk_list(S, nch, [&](int c) {
                int m = 0;
                for (int hh = 0; hh < kParts; ++hh)
                    if (kParts * c + hh < ng &&
                        min_scaled_cost(load_cone(a.obs_cone, a.obs_ext, og + kParts * c + hh), M, K) <= kSkipLog2)
                        m |= 1 << hh;
                return m;
            });
        }
        bool ok = use_list ? stream_list_prep(S, parity, src, i0, ni, n_list, prep, body)
                           : stream_tile_prep(S, parity, src, i0, ni, prep, body);
        if (threadIdx.x == 0) {
            long long np = 0;
            if (use_list)
                for (int c = 0; c < n_list; ++c) np += list_pairs(S.list[c] & 0xffffff, (int)((unsigned)S.list[c] >> 24), ni);
            else
                np = ni;
            atomicAdd((unsigned long long*)(a.ctrl + CTRL_SK_PAIRS), (unsigned long long)(4LL * td.z * np));
        }
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        float sa = lo(Sa) + hi(Sa), sb = lo(Sb) + hi(Sb);
        float Ga = valid ? (sa > kTinySum ? -(shift + lg2(sa))
                                          : -col_exact(a, t, C.ncxa, C.ncya, C.ncza, C.nrxa, C.nrya, C.nrza, dz, C.ka))
                         : 0.0f;
        float Gb = vb ? (sb > kTinySum ? -(shift + lg2(sb))
                                       : -col_exact(a, t, C.ncxb, C.ncyb, C.nczb, C.nrxb, C.nryb, C.nrzb, dz, C.kb))
                      : 0.0f;
        if (ub) {  // raised to lambda / (lambda + eps)
            Ga = ni > 0 ? a.tau_col * Ga : 0.0f;
            Gb = ni > 0 ? a.tau_col * Gb : 0.0f;
        }
        if (valid) *(float2*)&a.modY[q].z = make_float2(Ga, vb ? Gb : kNegHuge);
        float pm = kNegHuge, ps = 0.0f;
        if (valid) {
            pm = Ga;
            ps = 1.0f;
            if (vb) lse_merge_into(pm, ps, Gb, 1.0f);
        }
        block_lse(S, pm, ps);
        if (threadIdx.x == 0) a.col_part[tile] = make_float2(pm, ps);
    }
    if (!last_cta(S, a.ctrl + CTRL_COL_DONE)) return;
    // finalise: next F_0 from the new G and the current G_0
    if (a.mode == 2) {
        // no dustbins
    } else if (a.mode) {
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
            lse_merge_into(m, s, pp.x, pp.y);
        }
        block_lse(S, m, s);
        if (threadIdx.x == 0) {
            Lse2 L;
            L.init(D.G0[0] - a.kc);
            L.merge(m, s);
            D.F0n[0] = D.log2U[0] - L.value();
        }
    }
    block_maxima(a.col_part, a.ang_tiles, a.T, false, 0.0f, D.Gmax);
    if (threadIdx.x == 0) {
        a.ctrl[CTRL_COL_NEXT] = 0;
        a.ctrl[CTRL_COL_DONE] = 0;
    }
}

// ------------------------------------------------------------ row harvest
// Plan read-out per observed spot with the final potentials: argmax over the
// block's model spots and the outlier column (ties to the lowest index, the
// outlier column only when strictly larger), top1 - top2 margin in plan
// units, and the row-marginal error.  Scalar bookkeeping; once per E-step.
struct Top2 {
    float m, s, b1, b2;
    int arg;
    __device__ __forceinline__ void init() {
        m = kNegHuge;
        s = 0.0f;
        b1 = kNegHuge;
        b2 = kNegHuge;
        arg = -1;
    }
    // j: the spot's slot in the spatial order; perm maps slots to the caller's
    // indices, and ties go to the lowest caller index
    __device__ __forceinline__ void add(float v, int j, const int* perm) {
        if (v > m) {
            s = s * ex2(m - v) + 1.0f;
            m = v;
        } else {
            s += ex2(v - m);
        }
        if (v > b1 || (v == b1 && v > kNegHuge && perm[j] < perm[arg])) {
            b2 = b1;
            b1 = v;
            arg = j;
        } else if (v > b2) {
            b2 = v;
        }
    }
};

__global__ void __launch_bounds__(kTPB) sk_harvest_row_kernel(SkArgs a) {
    __shared__ __align__(128) Stage S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_ROW_TILES];
    const Srcs src{{a.modX, a.modY, a.modZ, a.modW}, 4};
    float my_err = 0.0f;
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_HRV_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.row_tiles[tile];
        int t = td.x;
        int q = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int ni = a.I_off[t + 1] - a.I_off[t];
        int lrow = 2 * (q - a.I2_off[t]);
        bool vb = valid && lrow + 1 < ni;
        int jbase = a.J_off[t], j0 = a.J2_off[t], nj = a.J2_off[t + 1] - j0;
        float dustv = a.mode == 2 ? kNegHuge : D.G0[a.mode ? t : 0] - a.kc;
        float4 X = valid ? a.obsX[q] : make_float4(0.f, 0.f, 0.f, 0.f);
        float4 Y = valid ? a.obsY[q] : make_float4(0.f, 0.f, kPadFar, kPadFar);
        f2 pxa = dup(X.x), pya = dup(X.z), pza = dup(Y.x), pxb = dup(X.y), pyb = dup(X.w), pzb = dup(Y.y);
        Top2 A, B;
        A.init();
        B.init();
        bool ok = stream_tile(S, parity, src, j0, nj, [&](int st, int n, int off) {
            if (!valid) return;
            for (int k = 0; k < n; ++k) {
                ulonglong2 Xm = *(const ulonglong2*)&S.s[0][st][k];
                ulonglong2 Ym = *(const ulonglong2*)&S.s[1][st][k];
                ulonglong2 Zm = *(const ulonglong2*)&S.s[2][st][k];
                ulonglong2 Wm = *(const ulonglong2*)&S.s[3][st][k];
                f2 va = pair_v2(pxa, pya, pza, Xm.x, Xm.y, Ym.x, Zm.x, Zm.y, Wm.x, Wm.y, Ym.y);
                f2 vv = pair_v2(pxb, pyb, pzb, Xm.x, Xm.y, Ym.x, Zm.x, Zm.y, Wm.x, Wm.y, Ym.y);
                int j = jbase + 2 * (off + k);
                A.add(lo(va), j, a.mod_perm);
                A.add(hi(va), j + 1, a.mod_perm);  // padding slots have -3e38 and never win
                B.add(lo(vv), j, a.mod_perm);
                B.add(hi(vv), j + 1, a.mod_perm);
            }
        });
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        if (valid) {
            int i = a.I_off[t] + lrow;
            for (int lane = 0; lane < 2; ++lane) {
                if (lane == 1 && !vb) break;
                Top2& P = lane ? B : A;
                float F = lane ? Y.w : Y.z;
                if (dustv > P.b1) {  // outlier column last, only when strictly larger
                    P.b2 = P.b1;
                    P.b1 = dustv;
                    P.arg = -1;
                } else if (dustv > P.b2) {
                    P.b2 = dustv;
                }
                Lse2 L;
                L.m = P.m;
                L.s = P.s;
                L.merge(dustv, 1.0f);
                float rs = ex2(F + L.value());
                my_err = fmaxf(my_err, fabsf(rs - 1.0f));
                // unbalanced plan: a spot that keeps most of its mass is an outlier
                if (a.mode == 2 && !(rs >= 0.5f)) P.arg = -1;
                int ic = a.obs_perm[i + lane];  // the caller's index of this observed spot
                if (a.assign) a.assign[ic] = P.arg >= 0 ? a.mod_perm[P.arg] : -1;
                if (a.margin) a.margin[ic] = ex2(F + P.b1) - (P.b2 > kNegHuge ? ex2(F + P.b2) : 0.0f);
            }
        }
    }
    float e = block_max(S, my_err);
    if (threadIdx.x == 0) atomicMax((int*)(D.err + 2), __float_as_int(e));  // non-negative floats
    if (!last_cta(S, a.ctrl + CTRL_HRV_DONE)) return;
    if (threadIdx.x == 0) {
        float err = __int_as_float(*(int*)(D.err + 2));
        int nd = a.mode == 2 ? 0 : (a.mode ? a.T : 1);
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
    __shared__ __align__(128) Stage S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    DustPtrs D = dust_ptrs(a.dust, a.T);
    const int n_tiles = a.ctrl[CTRL_N_COL_TILES];
    const Srcs src{{a.obsX, a.obsY, nullptr, nullptr}, 2};
    float my_err = 0.0f;
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_HCOL_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.col_tiles[tile];
        int t = td.x;
        int q = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int nj = a.J_off[t + 1] - a.J_off[t];
        int lcol = 2 * (q - a.J2_off[t]);
        bool vb = valid && lcol + 1 < nj;
        int i0 = a.I2_off[t], ni = a.I2_off[t + 1] - i0;
        ColPair C;
        if (valid) load_col_pair(a, q, C);
        C.A.init(kNegHuge);
        C.B.init(kNegHuge);
        C.A.S = pk(0.0f, 0.0f);
        C.B.S = pk(0.0f, 0.0f);
        bool ok = stream_tile(S, parity, src, i0, ni, [&](int st, int n, int) {
            if (valid) col_chunk(C, S.s[0][st], S.s[1][st], n);
        });
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        if (valid) {
            float4 Ym = a.modY[q];
            float F0 = a.mode == 2 ? kNegHuge : D.F0[a.mode ? t : 0];
            for (int lane = 0; lane < 2; ++lane) {
                if (lane == 1 && !vb) break;
                RowLse& L = lane ? C.B : C.A;
                float G = lane ? Ym.w : Ym.z;
                float ssum = lo(L.S) + hi(L.S);
                float qj = ssum > 0.0f ? ex2(G + L.m + lg2(ssum)) : 0.0f;
                if (a.q) a.q[a.mod_perm[a.J_off[t] + lcol + lane]] = qj;
                my_err = fmaxf(my_err, fabsf(qj + ex2(G + F0) - 1.0f));
            }
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
        int t = block_of(a.I_off, a.T, k);
        int l = a.obs_pos[k];
        float v = ((const float*)&a.obsY[a.I2_off[t] + (l >> 1)])[2 + (l & 1)];
        bad |= !isfinite(v);
        a.f[k] = v * a.to_user;
    }
    if (k < a.n_model) {
        int t = block_of(a.J_off, a.T, k);
        int l = a.mod_pos[k];
        float v = ((const float*)&a.modY[a.J2_off[t] + (l >> 1)])[2 + (l & 1)];
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

// Per-angle maxima of the starting G (for the first row pass) and F (for the
// M-step's skipping bound), padding excluded.
__global__ void __launch_bounds__(256) sk_init_gmax_kernel(SkArgs a) {
    __shared__ float red[8], redf[8];
    int t = blockIdx.x;
    float m = kNegHuge, f = kNegHuge;
    for (int q = a.J2_off[t] + threadIdx.x; q < a.J2_off[t + 1]; q += blockDim.x) {
        float4 y = a.modY[q];
        m = fmaxf(m, fmaxf(y.z, y.w));
    }
    for (int q = a.I2_off[t] + threadIdx.x; q < a.I2_off[t + 1]; q += blockDim.x) {
        float4 y = a.obsY[q];
        f = fmaxf(f, fmaxf(y.z, y.w));
    }
    for (int o = 16; o > 0; o >>= 1) {
        m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
        f = fmaxf(f, __shfl_xor_sync(0xffffffffu, f, o));
    }
    if ((threadIdx.x & 31) == 0) {
        red[threadIdx.x >> 5] = m;
        redf[threadIdx.x >> 5] = f;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < 8; ++k) {
            m = fmaxf(m, red[k]);
            f = fmaxf(f, redf[k]);
        }
        DustPtrs D = dust_ptrs(a.dust, a.T);
        D.Gmax[t] = m;
        D.Fmax[t] = f;  // the M-step's skipping bound; a row pass rewrites it
    }
}

cudaError_t sinkhorn_prepare(const SkArgs& a, cudaStream_t s) {
    int nmax = a.n_obs > a.n_model ? a.n_obs : a.n_model;
    int blocks = (nmax + 255) / 256;
    if (blocks < 1) blocks = 1;
    sk_schedule_kernel<<<1, 1024, 0, s>>>(a);
    if (a.T > 0) sk_sort_kernel<<<2 * a.T, kSortThreads, 0, s>>>(a);
    sk_pack_kernel<<<blocks, 256, 0, s>>>(a);
    {
        int max_gran = (a.n_obs + a.n_model) / (2 * kGran) + 2 * a.T + 2;  // bound on the granule count
        sk_cone_kernel<<<(max_gran * 32 + 255) / 256, 256, 0, s>>>(a);
    }
    if (a.mode != 2) sk_init_dust_kernel<<<1, 1024, 0, s>>>(a);
    if (a.T > 0) sk_init_gmax_kernel<<<a.T, 256, 0, s>>>(a);
    return cudaGetLastError();
}

// Launch shapes of the pair passes the autotuner chooses from:
// {threads per CTA (= pairs per tile), minimum resident CTAs per SM}.
typedef void (*SkKernel)(SkArgs);
static const SkKernel kRowKernels[kSkVariants] = {sk_row_kernel<256, 1>, sk_row_kernel<128, 1>, sk_row_kernel<128, 4>,
                                                  sk_row_kernel<64, 8>};
static const SkKernel kColKernels[kSkVariants] = {sk_col_kernel<256, 1>, sk_col_kernel<128, 1>, sk_col_kernel<128, 4>,
                                                  sk_col_kernel<64, 8>};

int sk_variant_threads(int v) { return v == 0 ? 256 : (v == 3 ? 64 : 128); }

void sinkhorn_row_pass(const SkArgs& a, const SkLaunch& l, cudaStream_t s) {
    kRowKernels[l.row_variant]<<<l.row_grid, sk_variant_threads(l.row_variant), 0, s>>>(a);
}

void sinkhorn_col_pass(const SkArgs& a, const SkLaunch& l, cudaStream_t s) {
    kColKernels[l.col_variant]<<<l.col_grid, sk_variant_threads(l.col_variant), 0, s>>>(a);
}

cudaError_t sinkhorn_iterate(const SkArgs& a, const SkLaunch& l, int n_iter, cudaStream_t s) {
    for (int it = 0; it < n_iter; ++it) {
        sinkhorn_row_pass(a, l, s);
        sinkhorn_col_pass(a, l, s);
    }
    return cudaGetLastError();
}

cudaError_t sinkhorn_finish(const SkArgs& a, const SkLaunch& l, bool want_rows, bool want_cols, cudaStream_t s) {
    int nmax = a.n_obs > a.n_model ? a.n_obs : a.n_model;
    int blocks = (nmax + 255) / 256;
    if (blocks < 1) blocks = 1;
    if (want_rows || want_cols) sk_clear_err_kernel<<<1, 1, 0, s>>>(a);
    // one thread per row (column) pair of the pass's tiles
    if (want_rows) sk_harvest_row_kernel<<<l.hrv_grid, sk_variant_threads(l.row_variant), 0, s>>>(a);
    if (want_cols) sk_harvest_col_kernel<<<l.hcol_grid, sk_variant_threads(l.col_variant), 0, s>>>(a);
    sk_finish_kernel<<<blocks, 256, 0, s>>>(a, want_rows ? 1 : 0, want_cols ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t sinkhorn_run(const SkArgs& a, const SkLaunch& l, int n_iter, bool want_rows, bool want_cols,
                         cudaStream_t s) {
    cudaError_t e = sinkhorn_prepare(a, s);
    if (e != cudaSuccess) return e;
    e = sinkhorn_iterate(a, l, n_iter, s);
    if (e != cudaSuccess) return e;
    return sinkhorn_finish(a, l, want_rows, want_cols, s);
}

int sinkhorn_occupancy(int* row_blocks_per_sm, int* col_blocks_per_sm) {
    for (int v = 0; v < kSkVariants; ++v) {
        int r = 0, c = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r, kRowKernels[v], sk_variant_threads(v), 0) != cudaSuccess)
            return -1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, kColKernels[v], sk_variant_threads(v), 0) != cudaSuccess)
            return -1;
        row_blocks_per_sm[v] = r > 0 ? r : 1;
        col_blocks_per_sm[v] = c > 0 ? c : 1;
    }
    return 0;
}

}  // namespace laue
