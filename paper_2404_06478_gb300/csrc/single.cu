// single.cu — batched single-grain fitting (paper Section "Single-grain
// fitting", Appendix "Single-grain fitting", Eq. elbo_single, Algorithm
// SingleLaueOT) and the candidate filter of Section "Selection of Prototypes
// with Optimal Transport" (f_out).
//
// One CTA fits one start at a time (persistent CTAs pull starts from a
// queue).  Per start:
//   1. cut: the spots the start grain makes (Eq. model_spot_cut) are listed,
//      sorted by (t, m), in the CTA's scratch slice; the list stays frozen
//      unless recut is set, when it is listed again at the pose of every step
//      (Algorithm SingleLaueOT recomputes the grain's rays at every iteration);
//   2. k_max annealed EM steps: the E-step plan is row-normalised over the
//      grain's model spots at t_i plus the outlier column,
//        Q_ij = exp(-C_ij/eps) / (sum_j' exp(-C_ij'/eps) + exp(-c_out/eps)),
//      with the costs of the pose at the start of the step; n_newton Newton
//      steps on x (block-wide sums of the exact gradient / Hessian), then n_mm
//      MM steps on R (per-plane M0 from v_j = sum_i Q_ij rhat_ij, Wahba by
//      Horn's quaternion eigenproblem);
//   3. filter: the spots visible at the final pose, the plan at eps_final,
//      column masses q_j; a ray is unmatched when q_j < 0.5; the start is
//      kept when #unmatched < f_out |J| and |J| > 0.
// Plan entries below 2^-40 are skipped.  Every reduction runs in a fixed order.
#include "pairs.cuh"
#include "mstep_common.cuh"
#include "ray.cuh"

namespace laue {

constexpr int kSfThreads = 128;
constexpr float kSfSkip = -40.0f;

struct SfScratch {
    int* tm;     // cap: (t << 16) | m of the listed spots
    float* rE;   // cap x 3 E-step rays
    float* cE;   // cap x 3 E-step centres
    float* v;    // cap x 3 MM sums / filter column masses
    float* kd;   // cap: (D_j / D)^2, the cost length of the spot's detector relative to D
    float* lse;  // icap row normalisers of one angle block (log2)
};

__device__ __forceinline__ SfScratch sf_slice(const SfArgs& a, int cta) {
    SfScratch s;
    size_t per = (size_t)a.cap * kSfSpotFloats + a.icap;
    float* base = a.scratch + per * cta;
    s.tm = (int*)base;
    s.rE = base + a.cap;
    s.cE = base + 4 * a.cap;
    s.v = base + 7 * a.cap;
    s.kd = base + 10 * a.cap;
    s.lse = base + 11 * a.cap;
    return s;
}

// ray / centre of plane m at angle t for pose (R, x)
__device__ __forceinline__ void sf_ray(const SfArgs& a, const float* R, const float* x, int t, int m, float* r,
                                       float* c, float* lam0, int* nh) {
    float sg, cg;
    sincosf(a.omega[t], &sg, &cg);
    float4 wd = a.w_d0[m];
    float v0 = R[0] * wd.x + R[1] * wd.y + R[2] * wd.z;
    float v1 = R[3] * wd.x + R[4] * wd.y + R[5] * wd.z;
    float v2 = R[6] * wd.x + R[7] * wd.y + R[8] * wd.z;
    float u0 = cg * v0 + sg * v2, u1 = v1, u2 = -sg * v0 + cg * v2;
    c[0] = cg * x[0] + sg * x[2];
    c[1] = x[1];
    c[2] = -sg * x[0] + cg * x[2];
    float ue = u0 * a.G.e[0] + u1 * a.G.e[1] + u2 * a.G.e[2];
    r[0] = a.G.e[0] - 2.0f * ue * u0;
    r[1] = a.G.e[1] - 2.0f * ue * u1;
    r[2] = a.G.e[2] - 2.0f * ue * u2;
    if (lam0) *lam0 = 2.0f * wd.w * fabsf(ue);
    if (nh) *nh = a.nharm[m];
}

// Detector of a visible ray, -1 when the ray is not visible (same decisions
// as the forward kernel).
__device__ __forceinline__ int sf_visible(const GeomDev& G, const float* r, const float* c, float lam0, int nh) {
    bool in_band = false;
    for (int n = 1; n <= nh; ++n) {
        float ln = lam0 / (float)n;
        if (ln >= G.lam_min && ln <= G.lam_max) {
            in_band = true;
            break;
        }
    }
    if (!in_band) return -1;
    float s[3];
    return hit_detector(G, r, c, s);
}

struct SfShared {
    float R[9], x[3];
    int n_spots, overflow, stop, t_off[kSfMaxT + 1];
    float red[kSfThreads * 9];
    int start;
    int last;
};

// Lists the spots visible at pose (R, x) sorted by (t, m); t_off per angle.
__device__ void sf_cut(const SfArgs& a, SfShared& S, const SfScratch& Z) {
    if (threadIdx.x == 0) {
        S.n_spots = 0;
        S.overflow = 0;
    }
    __syncthreads();
    long long nr = (long long)a.T * a.M;
    __shared__ int warp_cnt[kSfThreads / 32];
    for (long long base = 0; base < nr; base += kSfThreads) {
        long long id = base + threadIdx.x;
        bool vis = false;
        int t = 0, m = 0, det = -1;
        if (id < nr) {
            t = (int)(id / a.M);
            m = (int)(id % a.M);
            float r[3], c[3], lam0;
            int nh;
            sf_ray(a, S.R, S.x, t, m, r, c, &lam0, &nh);
            det = sf_visible(a.G, r, c, lam0, nh);
            vis = det >= 0;
        }
        unsigned ball = __ballot_sync(0xffffffffu, vis);
        int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) warp_cnt[w] = __popc(ball);
        __syncthreads();
        int before = 0, total = 0;
        for (int k = 0; k < kSfThreads / 32; ++k) {
            if (k < w) before += warp_cnt[k];
            total += warp_cnt[k];
        }
        int pos = S.n_spots + before + __popc(ball & ((1u << lane) - 1u));
        if (vis) {
            if (pos < a.cap) {
                Z.tm[pos] = (t << 16) | m;
                float dr = a.G.Dd[det] / a.G.D;
                Z.kd[pos] = dr * dr;
            } else {
                S.overflow = 1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) S.n_spots += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (S.n_spots > a.cap) S.n_spots = a.cap;
        int j = 0;
        for (int t = 0; t <= a.T; ++t) {
            while (j < S.n_spots && (Z.tm[j] >> 16) < t) ++j;
            S.t_off[t] = j;
        }
    }
    __syncthreads();
}

// E-step rays/centres of the listed spots at the current pose.
__device__ void sf_refresh(const SfArgs& a, SfShared& S, const SfScratch& Z) {
    for (int j = threadIdx.x; j < S.n_spots; j += blockDim.x) {
        int t = Z.tm[j] >> 16, m = Z.tm[j] & 0xffff;
        sf_ray(a, S.R, S.x, t, m, Z.rE + 3 * j, Z.cE + 3 * j, nullptr, nullptr);
    }
    __syncthreads();
}

__device__ __forceinline__ float sf_e2(const float4& p, const float* c, const float* r) {
    float d0 = p.x - c[0], d1 = p.y - c[1], d2 = p.z - c[2];
    float s = rsq(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    float e0 = fmaf(d0, s, -r[0]), e1 = fmaf(d1, s, -r[1]), e2 = fmaf(d2, s, -r[2]);
    return fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
}

// Row normaliser (log2) of observed spot p at angle t over the listed spots;
// npair counts the pair evaluations of the calling thread.
__device__ __forceinline__ float sf_row_lse(const SfArgs& a, const SfShared& S, const SfScratch& Z, int t,
                                            const float4& p, float negK, float dust, unsigned long long& npair) {
    Lse2 L;
    L.init(dust);
    npair += (unsigned)(S.t_off[t + 1] - S.t_off[t]);
    for (int j = S.t_off[t]; j < S.t_off[t + 1]; ++j) {
        float v = negK * Z.kd[j] * sf_e2(p, Z.cE + 3 * j, Z.rE + 3 * j);
        L.merge(v, 1.0f);
    }
    return L.value();
}

__device__ float sf_block_sum9(SfShared& S, float* v) {
    for (int k = 0; k < 9; ++k) S.red[9 * threadIdx.x + k] = v[k];
    __syncthreads();
    for (int w = kSfThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int k = 0; k < 9; ++k) S.red[9 * threadIdx.x + k] += S.red[9 * (threadIdx.x + w) + k];
        __syncthreads();
    }
    return 0.0f;
}

// One Newton step on x with the plan of the E-step costs.
__device__ void sf_newton(const SfArgs& a, SfShared& S, const SfScratch& Z, float negK, float dust,
                          unsigned long long& npair) {
    float acc[9];
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    for (int t = 0; t < a.T; ++t) {
        int j0 = S.t_off[t], j1 = S.t_off[t + 1];
        if (j0 == j1) continue;
        float sg, cg;
        sincosf(a.omega[t], &sg, &cg);
        float c[3] = {cg * S.x[0] + sg * S.x[2], S.x[1], -sg * S.x[0] + cg * S.x[2]};
        float gc[3] = {0, 0, 0}, hc[6] = {0, 0, 0, 0, 0, 0};
        for (int i = a.I_off[t] + threadIdx.x; i < a.I_off[t + 1]; i += blockDim.x) {
            float4 p = a.p[i];
            float l = sf_row_lse(a, S, Z, t, p, negK, dust, npair);
            npair += (unsigned)(j1 - j0);
            for (int j = j0; j < j1; ++j) {
                float v = negK * Z.kd[j] * sf_e2(p, Z.cE + 3 * j, Z.rE + 3 * j) - l;
                if (v < kSfSkip) continue;
                float Q = ex2(v) * Z.kd[j];  // M-step weight Q_ij (D_j / D)^2
                const float* r = Z.rE + 3 * j;
                float d0 = p.x - c[0], d1 = p.y - c[1], d2 = p.z - c[2];
                float is = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
                float h[3] = {d0 * is, d1 * is, d2 * is};
                float rr = h[0] * r[0] + h[1] * r[1] + h[2] * r[2];
                float qs = Q * is, q2 = qs * is;
                for (int k = 0; k < 3; ++k) gc[k] -= qs * (r[k] - rr * h[k]);
                int kk = 0;
                for (int u = 0; u < 3; ++u)
                    for (int w = u; w < 3; ++w)
                        hc[kk++] += q2 * (3.0f * rr * h[u] * h[w] - h[u] * r[w] - r[u] * h[w] - (u == w ? rr : 0.0f));
            }
        }
        float gx[3], hx[6];
        gamT_apply(cg, sg, gc, gx);
        sym_gamT_gam(cg, sg, hc, hx);
        for (int k = 0; k < 3; ++k) acc[k] += gx[k];
        for (int k = 0; k < 6; ++k) acc[3 + k] += hx[k];
    }
    sf_block_sum9(S, acc);
    if (threadIdx.x == 0) {
        float dx[3];
        bool ok = newton_step(S.red, S.red + 3, a.hreg, dx);
        if (!ok) {
            S.stop = 1;
        } else {
            float nrm = sqrtf(dx[0] * dx[0] + dx[1] * dx[1] + dx[2] * dx[2]);
            for (int k = 0; k < 3; ++k) S.x[k] -= dx[k];
            if (nrm < a.tol_x) S.stop = 1;
        }
    }
    __syncthreads();
}

// v_j = sum_i Q_ij rhat_ij (rhat at the current x), or with massonly the
// column mass q_j, for every listed spot; one warp per spot, fixed order.
__device__ void sf_columns(const SfArgs& a, SfShared& S, const SfScratch& Z, float negK, float dust, bool massonly,
                           unsigned long long& npair) {
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = 0; t < a.T; ++t) {
        int j0 = S.t_off[t], j1 = S.t_off[t + 1];
        if (j0 == j1) continue;
        int i0 = a.I_off[t], ni = a.I_off[t + 1] - i0;
        int nl = min(ni, a.icap);
        for (int k = threadIdx.x; k < nl; k += blockDim.x)
            Z.lse[k] = sf_row_lse(a, S, Z, t, a.p[i0 + k], negK, dust, npair);
        __syncthreads();
        float sg, cg;
        sincosf(a.omega[t], &sg, &cg);
        float c[3] = {cg * S.x[0] + sg * S.x[2], S.x[1], -sg * S.x[0] + cg * S.x[2]};
        for (int j = j0 + warp; j < j1; j += blockDim.x / 32) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            for (int k = lane; k < ni; k += 32) {
                float4 p = a.p[i0 + k];
                float l = k < nl ? Z.lse[k] : sf_row_lse(a, S, Z, t, p, negK, dust, npair);
                ++npair;
                float v = negK * Z.kd[j] * sf_e2(p, Z.cE + 3 * j, Z.rE + 3 * j) - l;
                if (v < kSfSkip) continue;
                float Q = ex2(v);
                if (massonly) {
                    s0 += Q;
                    continue;
                }
                float d0 = p.x - c[0], d1 = p.y - c[1], d2 = p.z - c[2];
                float is = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
                s0 += Q * d0 * is;
                s1 += Q * d1 * is;
                s2 += Q * d2 * is;
            }
            for (int o = 16; o > 0; o >>= 1) {
                s0 += __shfl_xor_sync(0xffffffffu, s0, o);
                s1 += __shfl_xor_sync(0xffffffffu, s1, o);
                s2 += __shfl_xor_sync(0xffffffffu, s2, o);
            }
            if (lane == 0) {
                const float w = massonly ? 1.0f : Z.kd[j];  // MM weight (D_j / D)^2
                Z.v[3 * j] = s0 * w;
                Z.v[3 * j + 1] = s1 * w;
                Z.v[3 * j + 2] = s2 * w;
            }
        }
        __syncthreads();
    }
}

// MM on R (majorisation-minimisation with Wahba steps); planes in smem.
__device__ void sf_mm(const SfArgs& a, SfShared& S, const SfScratch& Z, float* M6) {
    for (int k = threadIdx.x; k < 6 * a.M; k += blockDim.x) M6[k] = 0.0f;
    __syncthreads();
    for (int t = 0; t < a.T; ++t) {
        int j0 = S.t_off[t], j1 = S.t_off[t + 1];
        if (j0 == j1) continue;
        float sg, cg;
        sincosf(a.omega[t], &sg, &cg);
        for (int j = j0 + threadIdx.x; j < j1; j += blockDim.x) {  // distinct planes within one angle
            const float* v = Z.v + 3 * j;
            const float* e = a.G.e;
            float A[6] = {2 * v[0] * e[0], v[0] * e[1] + e[0] * v[1], v[0] * e[2] + e[0] * v[2],
                          2 * v[1] * e[1], v[1] * e[2] + e[1] * v[2], 2 * v[2] * e[2]};
            float Gm[6];
            sym_gamT_gam(cg, sg, A, Gm);
            float* dst = M6 + 6 * (Z.tm[j] & 0xffff);
            for (int k = 0; k < 6; ++k) dst[k] -= Gm[k];
        }
        __syncthreads();
    }
    for (int p = threadIdx.x; p < a.M; p += blockDim.x) psd_shift(M6 + 6 * p);
    if (threadIdx.x == 0) S.stop = 0;
    __syncthreads();
    for (int it = 0; it < a.n_mm; ++it) {
        float B[9];
        for (int k = 0; k < 9; ++k) B[k] = 0.0f;
        for (int p = threadIdx.x; p < a.M; p += blockDim.x) mm_accumulate(M6 + 6 * p, a.w_d0[p], S.R, B);
        sf_block_sum9(S, B);
        if (threadIdx.x == 0) {
            float Rn[9];
            if (!wahba_horn(S.red, Rn)) {
                S.stop = 1;
            } else {
                float d = 0.0f;
                for (int k = 0; k < 9; ++k) d += (Rn[k] - S.R[k]) * (Rn[k] - S.R[k]);
                for (int k = 0; k < 9; ++k) S.R[k] = Rn[k];
                if (sqrtf(d) < a.tol_R) S.stop = 1;
            }
        }
        __syncthreads();
        if (S.stop) break;
    }
    __syncthreads();
}

__device__ __forceinline__ float sf_eps(const SfArgs& a, int k) {
    return (float)anneal_eps(a.eps_final, a.k_max, k, a.anneal);
}

__global__ void __launch_bounds__(kSfThreads) single_fit_kernel(SfArgs a) {
    extern __shared__ float M6[];
    __shared__ SfShared S;
    SfScratch Z = sf_slice(a, blockIdx.x);
    const float log2e = 1.4426950408889634f;
    while (true) {
        if (threadIdx.x == 0) S.start = atomicAdd(a.queue, 1);
        __syncthreads();
        int s = S.start;
        if (s >= a.S) break;
        if (threadIdx.x < 9) S.R[threadIdx.x] = a.R0[9 * s + threadIdx.x];
        if (threadIdx.x < 3) S.x[threadIdx.x] = a.x0[3 * s + threadIdx.x];
        __syncthreads();
        sf_cut(a, S, Z);
        bool overflow = S.overflow != 0;
        unsigned long long npair = 0;
        for (int k = 0; k < a.k_max; ++k) {
            if (k > 0 && a.recut) {  // the visible set at the pose of this step
                sf_cut(a, S, Z);
                overflow |= S.overflow != 0;
            }
            float eps = sf_eps(a, k);
            float negK = -a.G.D * a.G.D * log2e / eps, dust = -a.c_out * log2e / eps;
            sf_refresh(a, S, Z);  // E-step pose
            if (threadIdx.x == 0) S.stop = 0;
            __syncthreads();
            for (int q = 0; q < a.n_newton; ++q) {
                sf_newton(a, S, Z, negK, dust, npair);
                if (S.stop) break;
            }
            __syncthreads();
            if (a.n_mm > 0) {
                sf_columns(a, S, Z, negK, dust, false, npair);
                sf_mm(a, S, Z, M6);
            }
        }
        // candidate filter at the final pose
        sf_cut(a, S, Z);
        overflow |= S.overflow != 0;
        sf_refresh(a, S, Z);
        float negK = -a.G.D * a.G.D * log2e / a.eps_final, dust = -a.c_out * log2e / a.eps_final;
        sf_columns(a, S, Z, negK, dust, true, npair);
        atomicAdd((unsigned long long*)(a.ctrl + CTRL_SF_PAIRS), npair);
        if (threadIdx.x == 0) {
            int nun = 0;
            for (int j = 0; j < S.n_spots; ++j) nun += Z.v[3 * j] < 0.5f;
            int nf = S.n_spots;
            if (a.unmatched) a.unmatched[s] = nf > 0 ? (float)nun / (float)nf : 1.0f;
            if (a.keep) a.keep[s] = (nf > 0 && (float)nun < a.f_out * (float)nf && !overflow) ? 1 : 0;
            for (int k = 0; k < 9; ++k) a.R_out[9 * s + k] = S.R[k];
            for (int k = 0; k < 3; ++k) a.x_out[3 * s + k] = S.x[k];
            if (overflow) set_status(a.ctrl, LAUE_ERR_CAPACITY);
        }
        __syncthreads();
    }
    // completion ticket: the last CTA resets the queue for the next launch
    if (threadIdx.x == 0) {
        __threadfence();
        S.last = atomicAdd(a.queue + 1, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (S.last && threadIdx.x == 0) {
        a.queue[0] = 0;
        a.queue[1] = 0;
    }
}

// ---------------------------------------------------------------- SPOT
// Appendix "Selection of prototypes" (Algorithm LaueSpotGreedy): grain-to-spot
// matrix read as the gain over the outlier baseline,
//   Lbar_in = max(0, LSE_{j of n at t_i}(-C_ij / eps_s) + c_out / eps_s),
// stored sparse by candidate (CSR, rows in (t, i) order), then the greedy
// facility-location selection f(S) = sum_i max_{n in S} Lbar_in.

// One candidate per CTA.  count_only: nnz per candidate; else fill the CSR.
__global__ void __launch_bounds__(kSfThreads) spot_matrix_kernel(SfArgs a, SpotArgs sp, int count_only) {
    __shared__ SfShared S;
    __shared__ int wcnt[kSfThreads / 32];
    __shared__ int nnz;
    SfScratch Z = sf_slice(a, blockIdx.x);
    const float log2e = 1.4426950408889634f;
    const float negK = -a.G.D * a.G.D * log2e / sp.eps_s, kc = a.c_out * log2e / sp.eps_s;
    for (int n = blockIdx.x; n < a.S; n += gridDim.x) {
        if (threadIdx.x < 9) S.R[threadIdx.x] = a.R0[9 * n + threadIdx.x];
        if (threadIdx.x < 3) S.x[threadIdx.x] = a.x0[3 * n + threadIdx.x];
        if (threadIdx.x == 0) nnz = 0;
        __syncthreads();
        sf_cut(a, S, Z);
        if (S.overflow && threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_CAPACITY);
        sf_refresh(a, S, Z);
        int base = count_only ? 0 : sp.row_ptr[n];
        for (int t = 0; t < a.T; ++t) {
            int j0 = S.t_off[t], j1 = S.t_off[t + 1];
            if (j0 == j1) continue;
            for (int i0 = a.I_off[t]; i0 < a.I_off[t + 1]; i0 += blockDim.x) {
                int i = i0 + threadIdx.x;
                float val = 0.0f;
                if (i < a.I_off[t + 1]) {
                    float4 p = a.p[i];
                    Lse2 L;
                    L.m = kNegHuge;
                    L.s = 0.0f;
                    for (int j = j0; j < j1; ++j)
                        L.merge(negK * Z.kd[j] * sf_e2(p, Z.cE + 3 * j, Z.rE + 3 * j), 1.0f);
                    val = (L.value() + kc) * 0.6931471805599453f;
                }
                bool nz = val > 0.0f;
                unsigned ball = __ballot_sync(0xffffffffu, nz);
                int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
                if (lane == 0) wcnt[w] = __popc(ball);
                __syncthreads();
                int before = 0, total = 0;
                for (int k = 0; k < kSfThreads / 32; ++k) {
                    if (k < w) before += wcnt[k];
                    total += wcnt[k];
                }
                if (nz && !count_only) {
                    int pos = base + nnz + before + __popc(ball & ((1u << lane) - 1u));
                    sp.col[pos] = i;
                    sp.val[pos] = val;
                }
                __syncthreads();
                if (threadIdx.x == 0) nnz += total;
                __syncthreads();
            }
        }
        if (count_only && threadIdx.x == 0) sp.count[n] = nnz;
        __syncthreads();
    }
}

// Exclusive scan of the per-candidate counts by one CTA; row_ptr[Nc] = nnz.
__global__ void __launch_bounds__(1024) spot_scan_kernel(SpotArgs sp, int Nc) {
    __shared__ long long part[1024];
    int per = (Nc + 1023) / 1024;
    int b0 = threadIdx.x * per, b1 = min(Nc, b0 + per);
    long long s = 0;
    for (int b = b0; b < b1; ++b) s += sp.count[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int k = 0; k < 1024; ++k) {
            long long v = part[k];
            part[k] = acc;
            acc += v;
        }
        sp.row_ptr[Nc] = (int)(acc > 0x7fffffff ? 0x7fffffff : acc);
        sp.nnz_total[0] = acc;
    }
    __syncthreads();
    long long acc = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        sp.row_ptr[b] = (int)acc;
        acc += sp.count[b];
    }
}

__global__ void spot_init_kernel(SpotArgs sp, int n_obs, int Nc) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < n_obs) sp.best[k] = 0.0f;
    if (k < Nc) sp.chosen[k] = 0;
    if (k == 0) {
        sp.tick[0] = 0;
    }
}

// gain_n = sum over the candidate's entries of max(0, Lbar_in - best_i);
// one warp per candidate, then a grid argmax (largest gain, lowest index).
__global__ void __launch_bounds__(256) spot_gain_kernel(SpotArgs sp, int Nc, int step) {
    __shared__ float bg[8];
    __shared__ int bi[8];
    __shared__ int last;
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    float g = -1.0f;
    int gi = 0x7fffffff;
    for (int n = warp; n < Nc; n += (gridDim.x * blockDim.x) >> 5) {
        float s = 0.0f;
        if (!sp.chosen[n]) {
            for (int e = sp.row_ptr[n] + lane; e < sp.row_ptr[n + 1]; e += 32)
                s += fmaxf(0.0f, sp.val[e] - sp.best[sp.col[e]]);
        }
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (sp.chosen[n]) s = -1.0f;
        if (s > g || (s == g && n < gi)) {
            g = s;
            gi = n;
        }
    }
    // warp lanes hold identical (g, gi); reduce warps of the block
    int w = threadIdx.x >> 5;
    if (lane == 0) {
        bg[w] = g;
        bi[w] = gi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k)
            if (bg[k] > g || (bg[k] == g && bi[k] < gi)) {
                g = bg[k];
                gi = bi[k];
            }
        sp.part_g[blockIdx.x] = g;
        sp.part_i[blockIdx.x] = gi;
        __threadfence();
        last = atomicAdd(sp.tick, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    float G = -1.0f;
    int I = 0x7fffffff;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        float pg = sp.part_g[b];
        int pi = sp.part_i[b];
        if (pg > G || (pg == G && pi < I)) {
            G = pg;
            I = pi;
        }
    }
    if (I < Nc) {
        sp.order[step] = I;
        sp.gains[step] = G < 0.0f ? 0.0f : G;
        sp.chosen[I] = 1;
    } else {
        sp.order[step] = -1;
        sp.gains[step] = 0.0f;
    }
    sp.cur[0] = I < Nc ? I : -1;
    sp.tick[0] = 0;
}

__global__ void spot_update_kernel(SpotArgs sp) {
    int n = sp.cur[0];
    if (n < 0) return;
    for (int e = sp.row_ptr[n] + blockIdx.x * blockDim.x + threadIdx.x; e < sp.row_ptr[n + 1];
         e += gridDim.x * blockDim.x)
        sp.best[sp.col[e]] = fmaxf(sp.best[sp.col[e]], sp.val[e]);
}

// Eq. spot_ngrains read on the increments: k* = argmax_{2 <= k <= K}
// Delta_k - Delta_{k+1} (Delta_{K+1} = 0), K < 2 gives K.
__global__ void spot_kstar_kernel(SpotArgs sp, int K) {
    int best = K < 2 ? K : 2;
    float bv = -3.0e38f;
    for (int k = 2; k <= K; ++k) {
        float d = sp.gains[k - 1] - (k < K ? sp.gains[k] : 0.0f);
        if (d > bv) {
            bv = d;
            best = k;
        }
    }
    sp.kstar[0] = best;
}

cudaError_t spot_matrix_run(const SfArgs& a, const SpotArgs& sp, int ctas, bool count_only, cudaStream_t s) {
    if (a.S > 0) spot_matrix_kernel<<<ctas, kSfThreads, 0, s>>>(a, sp, count_only ? 1 : 0);
    if (count_only) spot_scan_kernel<<<1, 1024, 0, s>>>(sp, a.S);
    return cudaGetLastError();
}

cudaError_t spot_greedy_run(const SpotArgs& sp, int n_obs, int Nc, int k_max, int sm_count, cudaStream_t s) {
    int nmax = n_obs > Nc ? n_obs : Nc;
    spot_init_kernel<<<(nmax + 255) / 256 + 1, 256, 0, s>>>(sp, n_obs, Nc);
    int blocks = sm_count * 4;
    for (int k = 0; k < k_max; ++k) {
        spot_gain_kernel<<<blocks, 256, 0, s>>>(sp, Nc, k);
        spot_update_kernel<<<64, 256, 0, s>>>(sp);
    }
    spot_kstar_kernel<<<1, 1, 0, s>>>(sp, k_max);
    return cudaGetLastError();
}

static_assert(kSfCap == 2048 && kSfIcap == 4096, "the workspace layout reserves the single-fit scratch for these");

cudaError_t single_fit_run(const SfArgs& a, int ctas, cudaStream_t s) {
    size_t shm = sizeof(float) * 6 * (size_t)a.M;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(single_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    if (a.S > 0) single_fit_kernel<<<ctas, kSfThreads, shm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace laue
