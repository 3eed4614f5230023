// mstep.cu — M-step of Sinkhorn-EM (paper Section "The M-step updates",
// Appendix "M-steps for grain position and rotation", Algorithms
// LauePosNewton, LaueRotMM and Wahba).
//
// The plan is never stored: Q_ij = 2^(F_i + G_j - K e2_ij) is recomputed from
// the E-step potentials and the E-step rays/centres of the model list (the
// pair-interleaved workspace copies made by the Sinkhorn pack kernel), pairs
// with Q_ij < 2^-40 are skipped, and the geometric terms use the current
// positions.  Per model spot a pass over its angle block accumulates, in
// registers:
//   Newton  g_c = sum_i Q (-(r - (rhat.r) rhat) / tau)
//           H_c = sum_i Q (3 (rhat.r) rhat rhat^T - rhat r^T - r rhat^T - (rhat.r) I) / tau^2
//           (exact gradient / Hessian of sum Q rhat.r w.r.t. c = Gamma_t x)
//   MM      v_j = sum_i Q rhat_ij
// Per-grain kernels then reduce the spots of a grain in a fixed order (angle
// by angle through a (t, n) segment table), solve the regularised Newton step
// x <- x - (H - iota I)^-1 g, iota = max(0, lmax(H) + hreg |H|_F), and run the
// majorisation-minimisation on R with M0_m = -sum Gamma^T (v e^T + e v^T) Gamma,
// M_m = M0_m + max(0, -lmin(M0_m)) I and R <- Wahba(M_m R w_m, w_m): the Wahba
// step maximises tr(R^T B), B = sum a b^T, through the top eigenvector of
// Horn's 4x4 symmetric matrix (a unit quaternion).
#include "pairs.cuh"
#include "mstep_common.cuh"

namespace laue {

constexpr float kQSkip = -40.0f;  // log2 of the smallest plan entry kept

// ------------------------------------------------------- segment table
// seg[t (N+1) + n] = first model spot of grain n at angle t (the list is sorted
// by (t, n, m)); seg[t (N+1) + N] = J_off[t+1].
__global__ void ms_seg_count_kernel(MsArgs m) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= m.n_model) return;
    atomicAdd(&m.seg[m.angle[j] * (m.N + 1) + m.grain[j]], 1);
}

__global__ void ms_seg_scan_kernel(MsArgs m) {
    int t = blockIdx.x;
    if (threadIdx.x != 0) return;
    int* s = m.seg + t * (m.N + 1);
    int acc = m.J_off[t];
    for (int n = 0; n < m.N; ++n) {
        int c = s[n];
        s[n] = acc;
        acc += c;
    }
    s[m.N] = acc;
}

__global__ void ms_init_kernel(MsArgs m) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= m.N) return;
    m.gstate[4 * n + 0] = 1.0f;  // Newton still active
    m.gstate[4 * n + 1] = 0.0f;  // last |dx|
    m.gstate[4 * n + 2] = 0.0f;  // last |dR|_F
}

// ------------------------------------------------------------ pair pass
// mode 0: Newton sums (9 floats in the x frame), mode 1: v_j (3 floats, lab),
// mode 2: adjoint of the OT-weighted cost (gradient w.r.t. axis-angle and x,
// and the spot's share of the objective; 7 floats), mode 3: the same adjoint at
// the current pose (the ray r_j of the current R, the plan of the E-step) plus
// the sums q_j = sum Q, s1_j = sum Q / tau, s2_j = sum Q / tau^2 of the
// Gauss-Newton matrix (10 floats).
struct MsCol {
    int j, n, t;
    bool ok;
    float cg, sg;
    float c[3];   // current centre Gamma_t x_n
    float r[3];   // E-step ray (mode 3: the ray at the current pose)
    float acc[10];
};

__device__ __forceinline__ void ms_pair(MsCol& C, int mode, float px, float py, float pz, float v) {
    if (!C.ok || v < kQSkip) return;
    float Q = ex2(v);
    float d0 = px - C.c[0], d1 = py - C.c[1], d2 = pz - C.c[2];
    float is = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    float h0 = d0 * is, h1 = d1 * is, h2 = d2 * is;
    if (mode >= 2) {
        // adjoint: sum Q (r - (rhat.r) rhat)/tau, sum Q (r - rhat), sum Q |rhat - r|^2
        float rr = h0 * C.r[0] + h1 * C.r[1] + h2 * C.r[2];
        float qs = Q * is;
        if (mode == 3) {
            C.acc[7] += Q;
            C.acc[8] += qs;
            C.acc[9] += qs * is;
        }
        C.acc[0] += qs * (C.r[0] - rr * h0);
        C.acc[1] += qs * (C.r[1] - rr * h1);
        C.acc[2] += qs * (C.r[2] - rr * h2);
        float e0 = C.r[0] - h0, e1 = C.r[1] - h1, e2 = C.r[2] - h2;
        C.acc[3] += Q * e0;
        C.acc[4] += Q * e1;
        C.acc[5] += Q * e2;
        C.acc[6] += Q * (e0 * e0 + e1 * e1 + e2 * e2);
        return;
    }
    if (mode == 1) {
        C.acc[0] += Q * h0;
        C.acc[1] += Q * h1;
        C.acc[2] += Q * h2;
        return;
    }
    float rr = h0 * C.r[0] + h1 * C.r[1] + h2 * C.r[2];
    float qs = Q * is;
    C.acc[0] -= qs * (C.r[0] - rr * h0);
    C.acc[1] -= qs * (C.r[1] - rr * h1);
    C.acc[2] -= qs * (C.r[2] - rr * h2);
    float q2 = qs * is;
    float h[3] = {h0, h1, h2};
    int k = 3;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) {
            float e = 3.0f * rr * h[a] * h[b] - h[a] * C.r[b] - C.r[a] * h[b] - (a == b ? rr : 0.0f);
            C.acc[k++] += q2 * e;
        }
}

template <int MODE>
__global__ void __launch_bounds__(kTPB) ms_pair_kernel(MsArgs m) {
    const SkArgs& a = m.sk;
    __shared__ __align__(128) Stage S;
    init_stage(S);
    uint32_t parity[2] = {0u, 0u};
    const int n_tiles = a.ctrl[CTRL_N_COL_TILES];
    const Srcs src{{a.obsX, a.obsY, nullptr, nullptr}, 2};
    while (true) {
        int tile = next_tile(S, a.ctrl + CTRL_GEN_NEXT, n_tiles);
        if (tile < 0) break;
        int4 td = a.col_tiles[tile];
        int t = td.x;
        int q = td.y + threadIdx.x;
        bool valid = (int)threadIdx.x < td.z;
        int nj = a.J_off[t + 1] - a.J_off[t];
        int lcol = 2 * (q - a.J2_off[t]);
        int i0 = a.I2_off[t], ni = a.I2_off[t + 1] - i0;
        float cg, sg;
        gamma_t(m.omega[t], cg, sg);
        ColPair P;
        MsCol A, B;
        float Ga = kNegHuge, Gb = kNegHuge;
        A.ok = B.ok = false;
        if (valid) {
            load_col_pair(a, q, P);
            float4 Y = a.modY[q];
            float4 Z = a.modZ[q];
            float4 W = a.modW[q];
            Ga = Y.z;
            Gb = Y.w;
            for (int lane = 0; lane < 2; ++lane) {
                MsCol& C = lane ? B : A;
                C.ok = lcol + lane < nj;
                if (!C.ok) continue;
                C.j = a.mod_perm[a.J_off[t] + lcol + lane];  // the caller's index
                C.n = m.grain[C.j];
                C.t = t;
                if (MODE == 0 && m.gstate[4 * C.n] == 0.0f) C.ok = false;  // converged grain
                gam_apply(cg, sg, m.x + 3 * C.n, C.c);
                C.r[0] = -(lane ? Z.y : Z.x);
                C.r[1] = -(lane ? Z.w : Z.z);
                C.r[2] = -(lane ? W.y : W.x);
                if (MODE == 3) {  // the ray of the current orientation
                    const float* Rn = m.R + 9 * C.n;
                    float4 wd = m.w_d0[m.plane[C.j]];
                    float v[3], u[3];
                    for (int r = 0; r < 3; ++r) v[r] = Rn[3 * r] * wd.x + Rn[3 * r + 1] * wd.y + Rn[3 * r + 2] * wd.z;
                    gam_apply(cg, sg, v, u);
                    float ue = u[0] * m.e[0] + u[1] * m.e[1] + u[2] * m.e[2];
                    for (int r = 0; r < 3; ++r) C.r[r] = m.e[r] - 2.0f * ue * u[r];
                }
                for (int k = 0; k < 10; ++k) C.acc[k] = 0.0f;
            }
        }
        const f2 Gpa = dup(Ga), Gpb = dup(Gb);
        // staged observed pairs [h, h + m) of stage st
        auto run = [&](int st, int h, int m) {
            const float4* sX = S.s[0][st];
            const float4* sY = S.s[1][st];
            for (int k = h; k < h + m; ++k) {
                ulonglong2 X = *(const ulonglong2*)&sX[k];
                ulonglong2 Y = *(const ulonglong2*)&sY[k];
                // E-step plan exponents of the 2 x 2 pairs: F_i + G_j - K e2
                f2 va = add2(pair_v2(X.x, X.y, Y.x, P.ncxa, P.ncya, P.ncza, P.nrxa, P.nrya, P.nrza, P.ka, Y.y), Gpa);
                f2 vb = add2(pair_v2(X.x, X.y, Y.x, P.ncxb, P.ncyb, P.nczb, P.nrxb, P.nryb, P.nrzb, P.kb, Y.y), Gpb);
                float m4 = fmaxf(fmaxf(lo(va), hi(va)), fmaxf(lo(vb), hi(vb)));
                if (m4 < kQSkip) continue;
                float4 x4 = sX[k], y4 = sY[k];
                ms_pair(A, MODE, x4.x, x4.z, y4.x, lo(va));
                ms_pair(A, MODE, x4.y, x4.w, y4.y, hi(va));
                ms_pair(B, MODE, x4.x, x4.z, y4.x, lo(vb));
                ms_pair(B, MODE, x4.y, x4.w, y4.y, hi(vb));
            }
        };
        auto body = [&](int st, int n, int, int mask = (1 << kParts) - 1) {
            if (!valid) return;
            for_each_run(mask, n, [&](int h, int m) { run(st, h, m); });
        };
        // the observed granules that can hold a plan entry >= 2^kQSkip for this
        // tile: log2 Q_ij = F_i + G_j - |K_j| e2 <= max_t F + max_tile G - the
        // cones' cost bound, so a granule whose bound exceeds
        // max F + max G - kQSkip holds only pairs the sums skip (exact)
        const float gtile = block_max(S, fmaxf(Ga, Gb));
        const int nch = (ni + kChunk - 1) / kChunk;
        const bool use_list = a.skip && nch > 0 && nch <= kMaxList;
        int n_list = nch;
        if (use_list) {
            const DustPtrs D = dust_ptrs(a.dust, a.T);
            const Cone M = tile_cone(a.mod_cone, a.mod_ext, a.mod_gbase[t], a.J2_off[t], td.y, td.z, false);
            const float K = a.skipK;  // the smallest cost factor of any spot
            const float lim = D.Fmax[t] + gtile - kQSkip + 1.0f;
            const int og = a.obs_gbase[t], ng = (ni + kGran - 1) / kGran;
            n_list = build_chunk_list(S, nch, [&](int c) {
                int msk = 0;
                for (int hh = 0; hh < kParts; ++hh)
                    if (kParts * c + hh < ng &&
                        min_scaled_cost(load_cone(a.obs_cone, a.obs_ext, og + kParts * c + hh), M, K) <= lim)
                        msk |= 1 << hh;
                return msk;
            });
        }
        auto no_prep = [](int, int) {};
        bool ok = use_list ? stream_list_prep(S, parity, src, i0, ni, n_list, no_prep, body)
                           : stream_tile(S, parity, src, i0, ni, [&](int st, int n, int) { body(st, n, 0); });
        if (threadIdx.x == 0) {
            long long np = 0;
            if (use_list)
                for (int c = 0; c < n_list; ++c)
                    np += list_pairs(S.list[c] & 0xffffff, (int)((unsigned)S.list[c] >> 24), ni);
            else
                np = ni;
            atomicAdd((unsigned long long*)(a.ctrl + CTRL_MS_PAIRS), (unsigned long long)(4LL * td.z * np));
        }
        if (!ok) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
            break;
        }
        if (valid) {
            for (int lane = 0; lane < 2; ++lane) {
                MsCol& C = lane ? B : A;
                if (lcol + lane >= nj) continue;
                const int jc = a.mod_perm[a.J_off[t] + lcol + lane];
                float* o = m.jsum + 12 * (size_t)jc;
                // cost length of the spot's detector: C_ij = D_j^2 |rhat - r|^2, so the
                // Newton and MM sums carry the weight (D_j / D)^2
                const int det = a.mod_s ? (int)a.mod_s[jc].w : -1;
                const float D2j = (det >= 0 && det < a.n_det) ? m.D2det[det] : m.D2;
                const float kd = D2j / m.D2;
                if (MODE >= 2) {
                    // per-spot gradient: x part Gamma^T dC/dc, rotation part
                    // v x (Gamma^T y), y = -2 ((gr.u) e + (u.e) gr), u = Gamma R w_m
                    float D2x2 = 2.0f * D2j;
                    float gc[3] = {D2x2 * C.acc[0], D2x2 * C.acc[1], D2x2 * C.acc[2]};
                    float gr[3] = {D2x2 * C.acc[3], D2x2 * C.acc[4], D2x2 * C.acc[5]};
                    float gx[3];
                    gamT_apply(cg, sg, gc, gx);
                    const float* Rn = m.R + 9 * C.n;
                    float4 wd = m.w_d0[m.plane[C.j]];
                    float v[3], u[3];
                    for (int r = 0; r < 3; ++r) v[r] = Rn[3 * r] * wd.x + Rn[3 * r + 1] * wd.y + Rn[3 * r + 2] * wd.z;
                    gam_apply(cg, sg, v, u);
                    float gu = gr[0] * u[0] + gr[1] * u[1] + gr[2] * u[2];
                    float ue = u[0] * m.e[0] + u[1] * m.e[1] + u[2] * m.e[2];
                    float y[3], Gy[3];
                    for (int r = 0; r < 3; ++r) y[r] = -2.0f * (gu * m.e[r] + ue * gr[r]);
                    gamT_apply(cg, sg, y, Gy);
                    o[0] = v[1] * Gy[2] - v[2] * Gy[1];
                    o[1] = v[2] * Gy[0] - v[0] * Gy[2];
                    o[2] = v[0] * Gy[1] - v[1] * Gy[0];
                    o[3] = gx[0];
                    o[4] = gx[1];
                    o[5] = gx[2];
                    o[6] = D2j * C.acc[6];
                    if (MODE == 3) {  // the Gauss-Newton sums, weighted (the grain kernel applies 2 D^2)
                        o[7] = kd * C.acc[7];
                        o[8] = kd * C.acc[8];
                        o[9] = kd * C.acc[9];
                    }
                    if (!C.ok)
                        for (int k = 0; k < (MODE == 3 ? 10 : 7); ++k) o[k] = 0.0f;
                } else if (MODE == 1) {
                    o[9] = C.ok ? kd * C.acc[0] : 0.0f;
                    o[10] = C.ok ? kd * C.acc[1] : 0.0f;
                    o[11] = C.ok ? kd * C.acc[2] : 0.0f;
                } else if (C.ok) {
                    float gx[3];
                    gamT_apply(cg, sg, C.acc, gx);
                    float hx[6];
                    sym_gamT_gam(cg, sg, C.acc + 3, hx);
                    for (int k = 0; k < 3; ++k) o[k] = kd * gx[k];
                    for (int k = 0; k < 6; ++k) o[3 + k] = kd * hx[k];
                } else {
                    for (int k = 0; k < 9; ++k) o[k] = 0.0f;
                }
            }
        }
    }
    if (!last_cta(S, a.ctrl + CTRL_GEN_DONE)) return;
    if (threadIdx.x == 0) {
        a.ctrl[CTRL_GEN_NEXT] = 0;
        a.ctrl[CTRL_GEN_DONE] = 0;
    }
}

// ------------------------------------------------------- Newton per grain
// One warp per grain: fixed-order reduction of the grain's spot sums, then the
// regularised Newton step on x.
__global__ void ms_newton_grain_kernel(MsArgs m) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m.N) return;
    int n = warp;
    if (m.gstate[4 * n] == 0.0f) return;
    float s[9];
    for (int k = 0; k < 9; ++k) s[k] = 0.0f;
    for (int t = lane; t < m.T; t += 32) {
        int j0 = m.seg[t * (m.N + 1) + n], j1 = m.seg[t * (m.N + 1) + n + 1];
        for (int j = j0; j < j1; ++j)
            for (int k = 0; k < 9; ++k) s[k] += m.jsum[12 * (size_t)j + k];
    }
    for (int k = 0; k < 9; ++k)
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if (lane != 0) return;
    float dx[3];
    if (!newton_step(s, s + 3, m.hreg, dx)) {
        m.gstate[4 * n] = 0.0f;
        return;
    }
    float nrm = sqrtf(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
    for (int a = 0; a < 3; ++a) m.x[3 * n + a] -= dx[a];
    m.gstate[4 * n + 1] = nrm;
    if (nrm < m.tol_x) m.gstate[4 * n] = 0.0f;
}

// ----------------------------------------------------------- MM per grain
constexpr int kMmThreads = 128;

__global__ void __launch_bounds__(kMmThreads) ms_mm_grain_kernel(MsArgs m) {
    extern __shared__ float sh[];
    float* M6 = sh;                        // M planes x 6 (M0, then M_m)
    float* red = sh + 6 * m.M;             // kMmThreads x 9
    __shared__ float Rs[9];
    __shared__ int stop;
    int n = blockIdx.x;
    for (int k = threadIdx.x; k < 6 * m.M; k += blockDim.x) M6[k] = 0.0f;
    if (threadIdx.x < 9) Rs[threadIdx.x] = m.R[9 * n + threadIdx.x];
    __syncthreads();
    const float e[3] = {m.e[0], m.e[1], m.e[2]};
    for (int t = 0; t < m.T; ++t) {
        int j0 = m.seg[t * (m.N + 1) + n], j1 = m.seg[t * (m.N + 1) + n + 1];
        float cg, sg;
        gamma_t(m.omega[t], cg, sg);
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {  // distinct planes within (t, n)
            const float* v = m.jsum + 12 * (size_t)j + 9;
            float A[6] = {2 * v[0] * e[0], v[0] * e[1] + e[0] * v[1], v[0] * e[2] + e[0] * v[2],
                          2 * v[1] * e[1], v[1] * e[2] + e[1] * v[2], 2 * v[2] * e[2]};
            float G[6];
            sym_gamT_gam(cg, sg, A, G);
            float* dst = M6 + 6 * m.plane[j];
            for (int k = 0; k < 6; ++k) dst[k] -= G[k];
        }
        __syncthreads();
    }
    // shift each plane's matrix to positive semi-definite
    for (int p = threadIdx.x; p < m.M; p += blockDim.x) psd_shift(M6 + 6 * p);
    if (threadIdx.x == 0) stop = 0;
    __syncthreads();
    float last = 0.0f;
    for (int it = 0; it < m.n_mm; ++it) {
        float B[9];
        for (int k = 0; k < 9; ++k) B[k] = 0.0f;
        for (int p = threadIdx.x; p < m.M; p += blockDim.x) mm_accumulate(M6 + 6 * p, m.w_d0[p], Rs, B);
        for (int k = 0; k < 9; ++k) red[9 * threadIdx.x + k] = B[k];
        __syncthreads();
        for (int w = kMmThreads / 2; w > 0; w >>= 1) {
            if ((int)threadIdx.x < w)
                for (int k = 0; k < 9; ++k) red[9 * threadIdx.x + k] += red[9 * (threadIdx.x + w) + k];
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            float Rn[9];
            if (!wahba_horn(red, Rn)) {
                stop = 1;
            } else {
                float d = 0.0f;
                for (int k = 0; k < 9; ++k) d += (Rn[k] - Rs[k]) * (Rn[k] - Rs[k]);
                last = sqrtf(d);
                for (int k = 0; k < 9; ++k) Rs[k] = Rn[k];
                if (last < m.tol_R) stop = 1;
            }
        }
        __syncthreads();
        if (stop) break;
    }
    if (threadIdx.x < 9) m.R[9 * n + threadIdx.x] = Rs[threadIdx.x];
    if (threadIdx.x == 0) m.gstate[4 * n + 2] = last;
}

__global__ void ms_norms_kernel(MsArgs m) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= m.N || !m.step_norms) return;
    m.step_norms[2 * n] = m.gstate[4 * n + 1];
    m.step_norms[2 * n + 1] = m.gstate[4 * n + 2];
}

// One warp per grain: fixed-order sum of the per-spot gradients and values.
__global__ void ms_grad_grain_kernel(MsArgs m) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m.N) return;
    int n = warp;
    float s[7];
    for (int k = 0; k < 7; ++k) s[k] = 0.0f;
    for (int t = lane; t < m.T; t += 32) {
        int j0 = m.seg[t * (m.N + 1) + n], j1 = m.seg[t * (m.N + 1) + n + 1];
        for (int j = j0; j < j1; ++j)
            for (int k = 0; k < 7; ++k) s[k] += m.jsum[12 * (size_t)j + k];
    }
    for (int k = 0; k < 7; ++k)
        for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_xor_sync(0xffffffffu, s[k], o);
    if (lane != 0) return;
    for (int k = 0; k < 6; ++k) m.grad[6 * n + k] = s[k];
    if (m.value) m.value[n] = s[6];
}

// ---------------------------------------------- adjoint M-step per grain
// One warp per grain: fixed-order sums of the per-spot gradients (mode 3) and
// of the Gauss-Newton blocks of each spot, built from its ray at the current
// pose with the model-ray projector P_j = I - r r^T:
//   H_phiphi += 2 D^2 q A^T A,  H_phix += 2 D^2 s1 A^T P Gamma,
//   H_xx += 2 D^2 s2 Gamma^T P Gamma,  A = 2 (u e^T + (u.e) I) Gamma [v]x;
// then a Levenberg-Marquardt step delta = -(H + lambda diag H)^-1 grad
// (Cholesky), R <- exp([delta_phi]x) R, x <- x + delta_x.
__device__ __forceinline__ int tri6(int a, int b) {
    int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo * 6 - lo * (lo - 1) / 2 + (hi - lo);
}

__global__ void ms_adj_grain_kernel(MsArgs m) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= m.N) return;
    int n = warp;
    float Rn[9];
    for (int k = 0; k < 9; ++k) Rn[k] = m.R[9 * n + k];
    const float D2x2 = 2.0f * m.D2;
    float g[6], H[21];
    for (int k = 0; k < 6; ++k) g[k] = 0.0f;
    for (int k = 0; k < 21; ++k) H[k] = 0.0f;
    for (int t = lane; t < m.T; t += 32) {
        int j0 = m.seg[t * (m.N + 1) + n], j1 = m.seg[t * (m.N + 1) + n + 1];
        if (j0 == j1) continue;
        float cg, sg;
        gamma_t(m.omega[t], cg, sg);
        for (int j = j0; j < j1; ++j) {
            const float* o = m.jsum + 12 * (size_t)j;
            for (int k = 0; k < 6; ++k) g[k] += o[k];
            float q = o[7], s1 = o[8], s2 = o[9];
            if (q == 0.0f) continue;
            float4 wd = m.w_d0[m.plane[j]];
            float v[3], u[3], r[3];
            for (int a = 0; a < 3; ++a) v[a] = Rn[3 * a] * wd.x + Rn[3 * a + 1] * wd.y + Rn[3 * a + 2] * wd.z;
            gam_apply(cg, sg, v, u);
            float ue = u[0] * m.e[0] + u[1] * m.e[1] + u[2] * m.e[2];
            for (int a = 0; a < 3; ++a) r[a] = m.e[a] - 2.0f * ue * u[a];
            // A = B Gamma [v]x with B = 2 (u e^T + ue I): column b of Gamma [v]x is Gamma (e_b x v)
            float A[9], PG[9], G[9];
            for (int b = 0; b < 3; ++b) {
                float eb[3] = {b == 0 ? 1.0f : 0.0f, b == 1 ? 1.0f : 0.0f, b == 2 ? 1.0f : 0.0f};
                float cr[3] = {eb[1] * v[2] - eb[2] * v[1], eb[2] * v[0] - eb[0] * v[2], eb[0] * v[1] - eb[1] * v[0]};
                float gc[3], ge[3];
                gam_apply(cg, sg, cr, gc);  // Gamma (e_b x v)
                gam_apply(cg, sg, eb, ge);  // column b of Gamma
                // [v]x e_b = v x e_b = -(e_b x v)
                gc[0] = -gc[0];
                gc[1] = -gc[1];
                gc[2] = -gc[2];
                float eg = m.e[0] * gc[0] + m.e[1] * gc[1] + m.e[2] * gc[2];
                for (int a = 0; a < 3; ++a) {
                    A[3 * a + b] = 2.0f * (u[a] * eg + ue * gc[a]);
                    G[3 * a + b] = ge[a];
                }
                float rg = r[0] * ge[0] + r[1] * ge[1] + r[2] * ge[2];
                for (int a = 0; a < 3; ++a) PG[3 * a + b] = ge[a] - r[a] * rg;
            }
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    float aa = 0.0f, ap = 0.0f, gp = 0.0f;
                    for (int k = 0; k < 3; ++k) {
                        aa += A[3 * k + a] * A[3 * k + b];
                        ap += A[3 * k + a] * PG[3 * k + b];
                        gp += G[3 * k + a] * PG[3 * k + b];
                    }
                    if (a <= b) {
                        H[tri6(a, b)] += D2x2 * q * aa;
                        H[tri6(3 + a, 3 + b)] += D2x2 * s2 * gp;
                    }
                    H[tri6(a, 3 + b)] += D2x2 * s1 * ap;
                }
        }
    }
    for (int k = 0; k < 6; ++k)
        for (int o = 16; o > 0; o >>= 1) g[k] += __shfl_xor_sync(0xffffffffu, g[k], o);
    for (int k = 0; k < 21; ++k)
        for (int o = 16; o > 0; o >>= 1) H[k] += __shfl_xor_sync(0xffffffffu, H[k], o);
    if (lane != 0) return;
    // Cholesky of H + lambda diag(H)
    float L[6][6], d[6], y[6];
    bool ok = true;
    for (int a = 0; a < 6 && ok; ++a) {
        if (!(H[tri6(a, a)] > 0.0f)) ok = false;
        for (int b = 0; b <= a && ok; ++b) {
            float sum = H[tri6(a, b)] + (a == b ? m.hreg * H[tri6(a, a)] : 0.0f);
            for (int k = 0; k < b; ++k) sum -= L[a][k] * L[b][k];
            if (a == b) {
                if (!(sum > 0.0f)) ok = false;
                else L[a][a] = sqrtf(sum);
            } else {
                L[a][b] = sum / L[b][b];
            }
        }
    }
    if (!ok) return;  // the grain keeps its pose
    for (int a = 0; a < 6; ++a) {
        float sum = -g[a];
        for (int k = 0; k < a; ++k) sum -= L[a][k] * y[k];
        y[a] = sum / L[a][a];
    }
    for (int a = 5; a >= 0; --a) {
        float sum = y[a];
        for (int k = a + 1; k < 6; ++k) sum -= L[k][a] * d[k];
        d[a] = sum / L[a][a];
    }
    // R <- exp([d_phi]x) R (Rodrigues), rows re-orthonormalised
    float th2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2], th = sqrtf(th2);
    float sa = th > 1e-6f ? sinf(th) / th : 1.0f - th2 / 6.0f;
    float cb = th > 1e-6f ? (1.0f - cosf(th)) / th2 : 0.5f - th2 / 24.0f;
    float K[9] = {0.0f, -d[2], d[1], d[2], 0.0f, -d[0], -d[1], d[0], 0.0f}, E[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            float k2 = K[3 * a] * K[b] + K[3 * a + 1] * K[3 + b] + K[3 * a + 2] * K[6 + b];
            E[3 * a + b] = (a == b ? 1.0f : 0.0f) + sa * K[3 * a + b] + cb * k2;
        }
    float Rs[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Rs[3 * a + b] = E[3 * a] * Rn[b] + E[3 * a + 1] * Rn[3 + b] + E[3 * a + 2] * Rn[6 + b];
    orthonormalise_rows(Rs);
    for (int k = 0; k < 9; ++k) m.R[9 * n + k] = Rs[k];
    for (int a = 0; a < 3; ++a) m.x[3 * n + a] += d[3 + a];
    m.gstate[4 * n + 1] = sqrtf(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
    m.gstate[4 * n + 2] = th;
}

static cudaError_t seg_table(const MsArgs& m, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(m.seg, 0, sizeof(int) * (size_t)m.T * (m.N + 1), s);
    if (e != cudaSuccess) return e;
    if (m.n_model > 0) ms_seg_count_kernel<<<(m.n_model + 255) / 256, 256, 0, s>>>(m);
    ms_seg_scan_kernel<<<m.T, 32, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t grad_run(const MsArgs& m, const SkLaunch& l, cudaStream_t s) {
    cudaError_t e = sinkhorn_prepare(m.sk, s);
    if (e != cudaSuccess) return e;
    if ((e = seg_table(m, s)) != cudaSuccess) return e;
    if (m.N > 0) ms_init_kernel<<<(m.N + 255) / 256, 256, 0, s>>>(m);
    ms_pair_kernel<2><<<l.col_grid, m.sk.tile_cols, 0, s>>>(m);
    if (m.N > 0) ms_grad_grain_kernel<<<(m.N * 32 + 127) / 128, 128, 0, s>>>(m);
    return cudaGetLastError();
}

// R = exp([w]x) R0 (Rodrigues) and, optionally, the transpose of the left
// Jacobian of SO(3) at w, J_l(w)^T, which maps a left-perturbation gradient
// to the gradient with respect to w:
//   J_l(w) = I + (1 - cos th)/th^2 [w]x + (th - sin th)/th^3 [w]x^2.
__global__ void axis_angle_kernel(const float* w, const float* R0, float* R, float* JlT, int N) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float a = w[3 * n], b = w[3 * n + 1], c = w[3 * n + 2];
    float th2 = a * a + b * b + c * c, th = sqrtf(th2);
    float A, B, C2;  // sin th / th, (1 - cos th)/th^2, (th - sin th)/th^3
    if (th < 1e-4f) {
        A = 1.0f - th2 / 6.0f;
        B = 0.5f - th2 / 24.0f;
        C2 = 1.0f / 6.0f - th2 / 120.0f;
    } else {
        float sn, cs;
        sincosf(th, &sn, &cs);
        A = sn / th;
        B = (1.0f - cs) / th2;
        C2 = (th - sn) / (th2 * th);
    }
    float K[9] = {0.0f, -c, b, c, 0.0f, -a, -b, a, 0.0f}, K2[9];
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) K2[3 * r + q] = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
    float E[9];
    for (int k = 0; k < 9; ++k) E[k] = (k % 4 == 0 ? 1.0f : 0.0f) + A * K[k] + B * K2[k];
    const float* P = R0 + 9 * n;
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q)
            R[9 * n + 3 * r + q] = E[3 * r] * P[q] + E[3 * r + 1] * P[3 + q] + E[3 * r + 2] * P[6 + q];
    if (JlT) {
        for (int r = 0; r < 3; ++r)
            for (int q = 0; q < 3; ++q) {
                float jl = (r == q ? 1.0f : 0.0f) + B * K[3 * r + q] + C2 * K2[3 * r + q];
                JlT[9 * n + 3 * q + r] = jl;  // transpose
            }
    }
}

// Vector-Jacobian product of E(exp([w]x) R0, x) for a gradient taken with
// respect to a left perturbation of R (laue_objective_grad):
//   dE/dw = J_l(w)^T dE/dphi,  dE/dx passed through, both scaled by gout_n.
__global__ void axis_angle_vjp_kernel(const float* w, const float* grad, const float* gout, float* gw, float* gx,
                                      int N) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    float a = w[3 * n], b = w[3 * n + 1], c = w[3 * n + 2];
    float th2 = a * a + b * b + c * c, th = sqrtf(th2);
    float B, C2;  // (1 - cos th)/th^2, (th - sin th)/th^3
    if (th < 1e-4f) {
        B = 0.5f - th2 / 24.0f;
        C2 = 1.0f / 6.0f - th2 / 120.0f;
    } else {
        float sn, cs;
        sincosf(th, &sn, &cs);
        B = (1.0f - cs) / th2;
        C2 = (th - sn) / (th2 * th);
    }
    float K[9] = {0.0f, -c, b, c, 0.0f, -a, -b, a, 0.0f};
    float s = gout ? gout[n] : 1.0f;
    const float* g = grad + 6 * n;
    for (int q = 0; q < 3; ++q) {  // (J_l^T g)_q = sum_r J_l[r][q] g_r
        float acc = 0.0f;
        for (int r = 0; r < 3; ++r) {
            float k2 = K[3 * r] * K[q] + K[3 * r + 1] * K[3 + q] + K[3 * r + 2] * K[6 + q];
            float jl = (r == q ? 1.0f : 0.0f) + B * K[3 * r + q] + C2 * k2;
            acc += jl * g[r];
        }
        gw[3 * n + q] = s * acc;
    }
    if (gx)
        for (int q = 0; q < 3; ++q) gx[3 * n + q] = s * g[3 + q];
}

cudaError_t axis_angle_vjp_run(const float* w, const float* grad, const float* gout, float* gw, float* gx, int N,
                               cudaStream_t s) {
    if (N > 0) axis_angle_vjp_kernel<<<(N + 127) / 128, 128, 0, s>>>(w, grad, gout, gw, gx, N);
    return cudaGetLastError();
}

cudaError_t mstep_adjoint_run(const MsArgs& m, const SkLaunch& l, int n_steps, cudaStream_t s) {
    cudaError_t e = sinkhorn_prepare(m.sk, s);  // the E-step plan: pair copies with F, G
    if (e != cudaSuccess) return e;
    if ((e = seg_table(m, s)) != cudaSuccess) return e;
    if (m.N > 0) ms_init_kernel<<<(m.N + 255) / 256, 256, 0, s>>>(m);
    for (int k = 0; k < n_steps; ++k) {
        ms_pair_kernel<3><<<l.col_grid, m.sk.tile_cols, 0, s>>>(m);
        if (m.N > 0) ms_adj_grain_kernel<<<(m.N * 32 + 127) / 128, 128, 0, s>>>(m);
    }
    if (m.N > 0) ms_norms_kernel<<<(m.N + 255) / 256, 256, 0, s>>>(m);
    return cudaGetLastError();
}

cudaError_t axis_angle_run(const float* w, const float* R0, float* R, float* JlT, int N, cudaStream_t s) {
    if (N > 0) axis_angle_kernel<<<(N + 127) / 128, 128, 0, s>>>(w, R0, R, JlT, N);
    return cudaGetLastError();
}

cudaError_t mstep_run(const MsArgs& m, const SkLaunch& l, cudaStream_t s) {
    cudaError_t e = sinkhorn_prepare(m.sk, s);  // schedule + pair-interleaved copies with F, G
    if (e != cudaSuccess) return e;
    if ((e = seg_table(m, s)) != cudaSuccess) return e;
    if (m.N > 0) ms_init_kernel<<<(m.N + 255) / 256, 256, 0, s>>>(m);
    for (int k = 0; k < m.n_newton; ++k) {
        ms_pair_kernel<0><<<l.col_grid, m.sk.tile_cols, 0, s>>>(m);
        if (m.N > 0) ms_newton_grain_kernel<<<(m.N * 32 + 127) / 128, 128, 0, s>>>(m);
    }
    if (m.n_mm > 0 && m.N > 0) {
        ms_pair_kernel<1><<<l.col_grid, m.sk.tile_cols, 0, s>>>(m);
        size_t shm = sizeof(float) * (6 * (size_t)m.M + 9 * kMmThreads);
        if (shm > 48 * 1024) {
            e = cudaFuncSetAttribute(ms_mm_grain_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
            if (e != cudaSuccess) return e;
        }
        ms_mm_grain_kernel<<<m.N, kMmThreads, shm, s>>>(m);
    }
    if (m.N > 0) ms_norms_kernel<<<(m.N + 255) / 256, 256, 0, s>>>(m);
    return cudaGetLastError();
}

}  // namespace laue
