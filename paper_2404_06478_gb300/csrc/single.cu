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
    float4* rk;  // cap: {-r_j, K_j} E-step ray and cost factor K_j = -D_j^2 log2(e) / eps
    int* tm;     // cap: (t << 16) | m of the listed spots
    float* cE;   // cap x 3 E-step centres (one per angle: every listed spot is the grain's)
    float* v;    // cap x 3 MM sums / filter column masses
    float* kd;   // cap: (D_j / D)^2, the cost length of the spot's detector relative to D
    float* lse;  // icap row normalisers of one angle block (log2)
    float4* near;  // near rows of the current E-step (ncap): {p, row normaliser (log2)}
    float4* nearu; // ncap: {u, t}, u = sum_j Q_ij (D_j / D)^2 r_j of the near row (lab frame), t its angle
};

__device__ __forceinline__ SfScratch sf_slice(const SfArgs& a, int cta) {
    SfScratch s;
    size_t per = (size_t)a.cap * kSfSpotFloats + a.icap + kSfNearFloats * (size_t)a.ncap;
    float* base = a.scratch + per * cta;  // 16-byte aligned: per is a multiple of 4 floats
    s.rk = (float4*)base;
    s.cE = base + 4 * a.cap;
    s.v = base + 7 * a.cap;
    s.tm = (int*)(base + 10 * a.cap);
    s.kd = base + 11 * a.cap;
    s.lse = base + 12 * a.cap;
    s.near = (float4*)(s.lse + a.icap);  // 16-byte aligned: cap, icap are multiples of 4
    s.nearu = s.near + a.ncap;           // ncap is a multiple of 4
    return s;
}

// ray / centre of plane m at angle t for pose (R, x); cs[t] = {cos, sin} of omega_t
__device__ __forceinline__ void sf_ray(const SfArgs& a, const float2* cs, const float* R, const float* x, int t, int m,
                                       float* r,
                                       float* c, float* lam0, int* nh) {
    const float cg = cs[t].x, sg = cs[t].y;
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
    // near rows of the E-step per angle: list entries [near_off[t], near_end[t]),
    // near_off[t] = -1 when angle t did not fit in the list
    int n_near, near_off[kSfMaxT], near_end[kSfMaxT];
    float red[kSfThreads * 9];
    int start;
    int last;
    int seg_total;  // visible rays of the current cut segment
    const float2* cs;  // {cos, sin} of each rotation angle (dynamic shared memory)
};

// Fills the angle table cs (T entries of dynamic shared memory) and points S.cs at it.
__device__ __forceinline__ void sf_angles(const SfArgs& a, SfShared& S, float2* cs) {
    for (int t = threadIdx.x; t < a.T; t += blockDim.x) {
        float sg, cg;
        sincosf(a.omega[t], &sg, &cg);
        cs[t] = make_float2(cg, sg);
    }
    if (threadIdx.x == 0) S.cs = cs;
    __syncthreads();
}

// Lists the spots visible at pose (R, x) sorted by (t, m); t_off per angle.
// The rays (t, m) of the whole scan in (t, m) order are taken kSfCutSeg at a
// time: every warp marks the visibility of 32 consecutive rays in one ballot
// word, warp 0 scans the words' counts, and each visible ray is written at its
// rank (its detector recomputed): four barriers per segment.
constexpr int kSfCutSeg = 4096;
__device__ void sf_cut(const SfArgs& a, SfShared& S, const SfScratch& Z) {
    __shared__ unsigned vis_w[kSfCutSeg / 32];
    __shared__ int w_off[kSfCutSeg / 32];
    if (threadIdx.x == 0) {
        S.n_spots = 0;
        S.overflow = 0;
    }
    __syncthreads();
    const int nr = a.T * a.M;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto detector_of = [&](int id, int& t, int& m) {
        t = id / a.M;
        m = id - t * a.M;
        float r[3], c[3], lam0;
        int nh;
        sf_ray(a, S.cs, S.R, S.x, t, m, r, c, &lam0, &nh);
        return sf_visible(a.G, r, c, lam0, nh);
    };
    for (int base = 0; base < nr; base += kSfCutSeg) {
        const int nseg = min(kSfCutSeg, nr - base), nw = (nseg + 31) / 32;
        for (int w0 = 32 * warp; w0 < nseg; w0 += kSfThreads) {  // warp-uniform bounds
            bool vis = false;
            if (w0 + lane < nseg) {
                int t, m;
                vis = detector_of(base + w0 + lane, t, m) >= 0;
            }
            const unsigned ball = __ballot_sync(0xffffffffu, vis);
            if (lane == 0) vis_w[w0 / 32] = ball;
        }
        __syncthreads();
        if (warp == 0) {  // exclusive prefix of the words' counts, in word order
            int run = 0;
            for (int w0 = 0; w0 < nw; w0 += 32) {
                const int c = w0 + lane < nw ? __popc(vis_w[w0 + lane]) : 0;
                int incl = c;
                for (int o = 1; o < 32; o <<= 1) {
                    const int y = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += y;
                }
                if (w0 + lane < nw) w_off[w0 + lane] = run + incl - c;
                run += __shfl_sync(0xffffffffu, incl, 31);
            }
            if (lane == 0) S.seg_total = run;
        }
        __syncthreads();
        for (int k = threadIdx.x; k < nseg; k += kSfThreads) {
            const unsigned word = vis_w[k >> 5], bit = 1u << (k & 31);
            if (!(word & bit)) continue;
            const int pos = S.n_spots + w_off[k >> 5] + __popc(word & (bit - 1u));
            if (pos < a.cap) {
                int t, m;
                const int det = detector_of(base + k, t, m);
                Z.tm[pos] = (t << 16) | m;
                const float dr = det >= 0 ? a.G.Dd[det] / a.G.D : 1.0f;  // same decision as above
                Z.kd[pos] = dr * dr;
            } else {
                S.overflow = 1;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) S.n_spots += S.seg_total;
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

// E-step rays/centres of the listed spots at the current pose, with the cost
// factors K_j = negK (D_j / D)^2 of the E-step temperature.
__device__ void sf_refresh(const SfArgs& a, SfShared& S, const SfScratch& Z, float negK) {
    for (int j = threadIdx.x; j < S.n_spots; j += blockDim.x) {
        int t = Z.tm[j] >> 16, m = Z.tm[j] & 0xffff;
        float r[3];
        sf_ray(a, S.cs, S.R, S.x, t, m, r, Z.cE + 3 * j, nullptr, nullptr);
        Z.rk[j] = make_float4(-r[0], -r[1], -r[2], negK * Z.kd[j]);
    }
    __syncthreads();
}

// Direction of an observed spot seen from the grain centre c of its angle:
// d = p - c and s = 1/|d|, computed once per row (every listed spot of the
// angle shares c).
struct SfRowG {
    float d0, d1, d2, s;
};

__device__ __forceinline__ SfRowG sf_rowg(const float4& p, const float* c) {
    SfRowG g;
    g.d0 = p.x - c[0];
    g.d1 = p.y - c[1];
    g.d2 = p.z - c[2];
    g.s = rsq(fmaf(g.d0, g.d0, fmaf(g.d1, g.d1, g.d2 * g.d2)));
    return g;
}

// Pair exponent K_j |rhat - r_j|^2 (<= 0) from the row's direction and the
// spot's {-r_j, K_j}.
__device__ __forceinline__ float sf_pair_v(const SfRowG& g, const float4& rk) {
    float e0 = fmaf(g.d0, g.s, rk.x), e1 = fmaf(g.d1, g.s, rk.y), e2 = fmaf(g.d2, g.s, rk.z);
    return rk.w * fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
}

// Row normaliser l (log2) of observed spot p at angle t over the listed spots
// and the outlier column, and the largest pair exponent vmax; npair counts the
// pair evaluations of the calling thread.  Every pair exponent
// v = negK kd e2 is <= 0, so while the outlier exponent dust is >= -100 the
// sum is taken relative to it with no running maximum (no term exceeds 2^100,
// the outlier term 1 never underflows); below that, with the running maximum.
__device__ __forceinline__ float sf_row_lse(const SfArgs& a, const SfShared& S, const SfScratch& Z, int t,
                                            const float4& p, float dust, unsigned long long& npair, float& vmax) {
    const int j0 = S.t_off[t], j1 = S.t_off[t + 1];
    npair += (unsigned)(j1 - j0);
    vmax = kNegHuge;
    if (j1 == j0) return dust;
    const SfRowG g = sf_rowg(p, Z.cE + 3 * j0);
    if (dust >= -100.0f) {
        // s >= 1 (the outlier term), so a term below 2^-25 (under half an ulp
        // of s) leaves s unchanged: such terms are not evaluated
        float s = 1.0f;
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
            float v = sf_pair_v(g, Z.rk[j]);
            vmax = fmaxf(vmax, v);
            const float dv = v - dust;
            if (dv >= -25.0f) s += ex2(dv);
        }
        return dust + lg2(s);
    }
    Lse2 L;
    L.init(dust);
    for (int j = j0; j < j1; ++j) {
        float v = sf_pair_v(g, Z.rk[j]);
        vmax = fmaxf(vmax, v);
        L.merge(v, 1.0f);
    }
    return L.value();
}

// Row normaliser l of observed spot p (as sf_row_lse) together with the row's
// plan-weighted ray sum u = sum_j Q_ij (D_j / D)^2 r_j (lab frame), Q_ij =
// 2^(v_ij - l) over every listed spot of angle t: with the row's direction
// fixed during the M-step, the Newton sums of the row are linear in u, so u
// is formed once per E-step.  The weight (D_j / D)^2 = K_j / negK.
__device__ __forceinline__ float sf_row_lse_u(const SfArgs& a, const SfShared& S, const SfScratch& Z, int t,
                                              const float4& p, float dust, float inv_negK,
                                              unsigned long long& npair, float& vmax, float* u) {
    const int j0 = S.t_off[t], j1 = S.t_off[t + 1];
    npair += (unsigned)(j1 - j0);
    vmax = kNegHuge;
    u[0] = u[1] = u[2] = 0.0f;
    if (j1 == j0) return dust;
    const SfRowG g = sf_rowg(p, Z.cE + 3 * j0);
    float m = dust, s = 1.0f, u0 = 0.0f, u1 = 0.0f, u2 = 0.0f;
    if (dust >= -100.0f) {  // relative to the outlier term, no running maximum
        // terms below 2^-25 leave s (>= 1) unchanged and are skipped; their
        // share of u is below 2^-25 of the row's plan mass
#pragma unroll 4
        for (int j = j0; j < j1; ++j) {
            const float4 rk = Z.rk[j];
            const float v = sf_pair_v(g, rk);
            vmax = fmaxf(vmax, v);
            const float dv = v - dust;
            if (dv < -25.0f) continue;
            const float w = ex2(dv), wk = w * rk.w;
            s += w;
            u0 = fmaf(-wk, rk.x, u0);  // r_j = -rk.xyz
            u1 = fmaf(-wk, rk.y, u1);
            u2 = fmaf(-wk, rk.z, u2);
        }
    } else {
        for (int j = j0; j < j1; ++j) {
            const float4 rk = Z.rk[j];
            const float v = sf_pair_v(g, rk);
            vmax = fmaxf(vmax, v);
            if (v > m) {
                const float f = ex2(m - v);
                s = fmaf(s, f, 1.0f);
                u0 = fmaf(u0, f, -rk.w * rk.x);
                u1 = fmaf(u1, f, -rk.w * rk.y);
                u2 = fmaf(u2, f, -rk.w * rk.z);
                m = v;
            } else {
                const float w = ex2(v - m), wk = w * rk.w;
                s += w;
                u0 = fmaf(-wk, rk.x, u0);
                u1 = fmaf(-wk, rk.y, u1);
                u2 = fmaf(-wk, rk.z, u2);
            }
        }
    }
    const float sc = inv_negK / s;  // 2^(m - l) = 1 / s
    u[0] = u0 * sc;
    u[1] = u1 * sc;
    u[2] = u2 * sc;
    return m + lg2(s);
}

// Two rows a and b of angle t at once (one pass over the listed spots, each
// spot's record loaded once for both), each with the arithmetic of
// sf_row_lse_u in the same order, so both results are bit-identical to it.
// Rows whose outlier exponent is below -100 take sf_row_lse_u one by one.
__device__ __forceinline__ void sf_row2_lse_u(const SfArgs& a, const SfShared& S, const SfScratch& Z, int t,
                                              const float4& pa, const float4& pb, bool hb, float dust,
                                              float inv_negK, unsigned long long& npair, float& la, float& lb,
                                              float& vma, float& vmb, float* ua, float* ub) {
    if (dust < -100.0f) {
        la = sf_row_lse_u(a, S, Z, t, pa, dust, inv_negK, npair, vma, ua);
        if (hb) lb = sf_row_lse_u(a, S, Z, t, pb, dust, inv_negK, npair, vmb, ub);
        return;
    }
    const int j0 = S.t_off[t], j1 = S.t_off[t + 1];
    npair += (unsigned)(j1 - j0) * (hb ? 2u : 1u);
    vma = vmb = kNegHuge;
    ua[0] = ua[1] = ua[2] = ub[0] = ub[1] = ub[2] = 0.0f;
    la = lb = dust;
    if (j1 == j0) return;
    const SfRowG ga = sf_rowg(pa, Z.cE + 3 * j0), gb = sf_rowg(pb, Z.cE + 3 * j0);
    float sa = 1.0f, sb = 1.0f, a0 = 0.0f, a1 = 0.0f, a2 = 0.0f, b0 = 0.0f, b1 = 0.0f, b2 = 0.0f;
#pragma unroll 2
    for (int j = j0; j < j1; ++j) {
        const float4 rk = Z.rk[j];
        const float va = sf_pair_v(ga, rk), vb = sf_pair_v(gb, rk);
        vma = fmaxf(vma, va);
        vmb = fmaxf(vmb, vb);
        const float dva = va - dust, dvb = vb - dust;
        if (dva >= -25.0f) {
            const float w = ex2(dva), wk = w * rk.w;
            sa += w;
            a0 = fmaf(-wk, rk.x, a0);
            a1 = fmaf(-wk, rk.y, a1);
            a2 = fmaf(-wk, rk.z, a2);
        }
        if (dvb >= -25.0f) {
            const float w = ex2(dvb), wk = w * rk.w;
            sb += w;
            b0 = fmaf(-wk, rk.x, b0);
            b1 = fmaf(-wk, rk.y, b1);
            b2 = fmaf(-wk, rk.z, b2);
        }
    }
    const float sca = inv_negK / sa, scb = inv_negK / sb;
    ua[0] = a0 * sca;
    ua[1] = a1 * sca;
    ua[2] = a2 * sca;
    ub[0] = b0 * scb;
    ub[1] = b1 * scb;
    ub[2] = b2 * scb;
    la = dust + lg2(sa);
    lb = dust + lg2(sb);
}

// Row normalisers of this EM step's E-step and the rows that carry plan mass.
// A row is near when some pair keeps Q_ij >= 2^kSfSkip (v_ij - l_i >=
// kSfSkip); every other row has all its plan entries below the cut-off that
// the Newton and MM sums skip, so only near rows enter them.  The near rows of
// each angle are listed with l (ascending row index) while the list has room;
// an angle that does not fit is marked near_off = -1 and its rows are scanned
// in full by the passes.  The plan stays the E-step's for the whole M-step,
// so the list serves every Newton and MM pass of the step.
__device__ void sf_near(const SfArgs& a, SfShared& S, const SfScratch& Z, float negK, float dust,
                        unsigned long long& npair, bool with_u) {
    const float inv_negK = 1.0f / negK;
    __shared__ int wcnt[kSfThreads / 32], wcnt2[kSfThreads / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) S.n_near = 0;
    __syncthreads();
    for (int t = 0; t < a.T; ++t) {
        const int base = S.n_near;
        int cnt = 0;
        if (S.t_off[t + 1] > S.t_off[t]) {
            const int i_beg = a.I_off[t], i_end = a.I_off[t + 1];
            const float4 zero4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            // chunks of 2 kSfThreads rows, two rows per thread (i and i + kSfThreads,
            // listed in row order); the next chunk's rows are loaded while this
            // chunk's are summed
            const int ia0 = i_beg + threadIdx.x, ib0 = ia0 + kSfThreads;
            float4 pa_next = ia0 < i_end ? a.p[ia0] : zero4, pb_next = ib0 < i_end ? a.p[ib0] : zero4;
            for (int i0 = i_beg; i0 < i_end; i0 += 2 * kSfThreads) {
                const int ia = i0 + threadIdx.x, ib = ia + kSfThreads;
                const bool ha = ia < i_end, hb = ib < i_end;
                const float4 pa = pa_next, pb = pb_next;
                if (ia + 2 * kSfThreads < i_end) pa_next = a.p[ia + 2 * kSfThreads];
                if (ib + 2 * kSfThreads < i_end) pb_next = a.p[ib + 2 * kSfThreads];
                bool near_a = false, near_b = false;
                float la = 0.0f, lb = 0.0f;
                float ua[3] = {0.0f, 0.0f, 0.0f}, ub[3] = {0.0f, 0.0f, 0.0f};
                if (ha) {
                    float vma, vmb = kNegHuge;
                    if (with_u) {
                        sf_row2_lse_u(a, S, Z, t, pa, pb, hb, dust, inv_negK, npair, la, lb, vma, vmb, ua, ub);
                    } else {
                        la = sf_row_lse(a, S, Z, t, pa, dust, npair, vma);
                        if (hb) lb = sf_row_lse(a, S, Z, t, pb, dust, npair, vmb);
                    }
                    near_a = vma - la >= kSfSkip;
                    near_b = hb && vmb - lb >= kSfSkip;
                }
                const unsigned balla = __ballot_sync(0xffffffffu, near_a), ballb = __ballot_sync(0xffffffffu, near_b);
                if (lane == 0) {
                    wcnt[w] = __popc(balla);
                    wcnt2[w] = __popc(ballb);
                }
                __syncthreads();
                int before_a = 0, total_a = 0, before_b = 0, total_b = 0;
                for (int k = 0; k < kSfThreads / 32; ++k) {
                    if (k < w) {
                        before_a += wcnt[k];
                        before_b += wcnt2[k];
                    }
                    total_a += wcnt[k];
                    total_b += wcnt2[k];
                }
                const unsigned below = (1u << lane) - 1u;
                const int pos_a = base + cnt + before_a + __popc(balla & below);
                const int pos_b = base + cnt + total_a + before_b + __popc(ballb & below);
                if (near_a && pos_a < a.ncap) {
                    Z.near[pos_a] = make_float4(pa.x, pa.y, pa.z, la);
                    if (with_u) Z.nearu[pos_a] = make_float4(ua[0], ua[1], ua[2], __int_as_float(t));
                }
                if (near_b && pos_b < a.ncap) {
                    Z.near[pos_b] = make_float4(pb.x, pb.y, pb.z, lb);
                    if (with_u) Z.nearu[pos_b] = make_float4(ub[0], ub[1], ub[2], __int_as_float(t));
                }
                cnt += total_a + total_b;
                __syncthreads();
            }
        }
        if (threadIdx.x == 0) {
            if (base + cnt <= a.ncap) {
                S.near_off[t] = base;
                S.near_end[t] = base + cnt;
                S.n_near = base + cnt;
            } else {
                S.near_off[t] = -1;
            }
        }
        __syncthreads();
    }
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

// Newton sums of observed spot p against the listed spots of its angle,
// accumulated in the sample frame of x (centre c of the current position,
// Gamma_t of cos/sin cg, sg): with the directions rotated back, h = Gamma^T
// rhat and r_j = Gamma^T r_j(lab), the gradient and Hessian of
// sum_j Q_ij rhat.r_j w.r.t. x are
//   g = -s sum_j Q_ij (r_j - (h.r_j) h),
//   H = s^2 sum_j Q_ij (3 (h.r_j) h h^T - h r_j^T - r_j h^T - (h.r_j) I),
// s = 1 / |p - c|.  h and s belong to the row, so both are linear in the
// row's u = sum_j Q_ij (D_j / D)^2 r_j (lab frame, from sf_row_lse_u; the
// weight is the M-step's), which the E-step plan fixes for the whole M-step.
__device__ __forceinline__ void sf_newton_row(const float4& p, const float* ul, const float* c, float cg, float sg,
                                              float* acc) {
    if (ul[0] == 0.0f && ul[1] == 0.0f && ul[2] == 0.0f) return;
    // direction at the current position
    const float d0 = p.x - c[0], d1 = p.y - c[1], d2 = p.z - c[2];
    const float is = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    const float hl[3] = {d0 * is, d1 * is, d2 * is};
    float h[3], u[3];
    gamT_apply(cg, sg, hl, h);
    gamT_apply(cg, sg, ul, u);
    const float hu = h[0] * u[0] + h[1] * u[1] + h[2] * u[2];
    const float is2 = is * is;
    for (int k = 0; k < 3; ++k) acc[k] -= is * (u[k] - hu * h[k]);
    int kk = 3;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b)
            acc[kk++] += is2 * (3.0f * hu * h[a] * h[b] - h[a] * u[b] - u[a] * h[b] - (a == b ? hu : 0.0f));
}

// One Newton step on x with the plan of the E-step costs (near rows of sf_near).
__device__ void sf_newton(const SfArgs& a, SfShared& S, const SfScratch& Z, float negK, float dust,
                          unsigned long long& npair) {
    float acc[9];
    for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
    const float inv_negK = 1.0f / negK;
    // the listed near rows of every angle, [0, n_near): one flat loop, four
    // rows per thread and step with their loads issued together (the rows sit
    // in global memory and the pass is bound by their latency)
    auto row = [&](const float4& q, const float4& uq) {
        const int t = __float_as_int(uq.w);
        const float cg = S.cs[t].x, sg = S.cs[t].y;
        const float c[3] = {cg * S.x[0] + sg * S.x[2], S.x[1], -sg * S.x[0] + cg * S.x[2]};
        const float ul[3] = {uq.x, uq.y, uq.z};
        sf_newton_row(q, ul, c, cg, sg, acc);
    };
    const int nn = S.n_near;
    int k = threadIdx.x;
    for (; k + 3 * kSfThreads < nn; k += 4 * kSfThreads) {
        float4 q[4], uq[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            q[r] = Z.near[k + r * kSfThreads];
            uq[r] = Z.nearu[k + r * kSfThreads];
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) row(q[r], uq[r]);
    }
    for (; k < nn; k += kSfThreads) row(Z.near[k], Z.nearu[k]);
    // angles whose near rows did not fit the list: every row, u recomputed
    for (int t = 0; t < a.T; ++t) {
        if (S.t_off[t + 1] == S.t_off[t] || S.near_off[t] >= 0) continue;
        const float cg = S.cs[t].x, sg = S.cs[t].y;
        const float c[3] = {cg * S.x[0] + sg * S.x[2], S.x[1], -sg * S.x[0] + cg * S.x[2]};
        for (int i = a.I_off[t] + threadIdx.x; i < a.I_off[t + 1]; i += blockDim.x) {
            const float4 p = a.p[i];
            float vmax, ul[3];
            sf_row_lse_u(a, S, Z, t, p, dust, inv_negK, npair, vmax, ul);
            sf_newton_row(p, ul, c, cg, sg, acc);
        }
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

// Column sums of listed spot j over the rows given by row(k), k = lane, lane +
// 32, ... < n: Q_ij rhat_ij, or with massonly the column mass.
template <class Row>
__device__ __forceinline__ void sf_column_sums(const SfScratch& Z, int j, int n, bool massonly, const float* c,
                                               Row row, float& s0, float& s1, float& s2,
                                               unsigned long long& npair) {
    const int lane = threadIdx.x & 31;
    const float4 rk = Z.rk[j];
    auto pair = [&](const float4& p, float l) {
        float v = sf_pair_v(sf_rowg(p, Z.cE + 3 * j), rk) - l;
        if (v < kSfSkip) return;
        float Q = ex2(v);
        if (massonly) {
            s0 += Q;
            return;
        }
        float d0 = p.x - c[0], d1 = p.y - c[1], d2 = p.z - c[2];
        float is = rsqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
        s0 += Q * d0 * is;
        s1 += Q * d1 * is;
        s2 += Q * d2 * is;
    };
    for (int k = lane; k < n; k += 32) {
        float4 p;
        float l;
        row(k, p, l);
        ++npair;
        pair(p, l);
    }
}

// v_j = sum_i Q_ij rhat_ij (rhat at the current x), or with massonly the
// column mass q_j, for every listed spot; one warp per spot, fixed order
// (the near rows of sf_near, or every row of an angle not in that list).
__device__ void sf_columns(const SfArgs& a, SfShared& S, const SfScratch& Z, float negK, float dust, bool massonly,
                           unsigned long long& npair) {
    int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int t = 0; t < a.T; ++t) {
        int j0 = S.t_off[t], j1 = S.t_off[t + 1];
        if (j0 == j1) continue;
        const int off = S.near_off[t];
        int i0 = a.I_off[t], ni = a.I_off[t + 1] - i0;
        int nl = min(ni, a.icap);
        if (off < 0) {
            for (int k = threadIdx.x; k < nl; k += blockDim.x) {
                float vmax;
                Z.lse[k] = sf_row_lse(a, S, Z, t, a.p[i0 + k], dust, npair, vmax);
            }
            __syncthreads();
        }
        const float cg = S.cs[t].x, sg = S.cs[t].y;
        float c[3] = {cg * S.x[0] + sg * S.x[2], S.x[1], -sg * S.x[0] + cg * S.x[2]};
        for (int j = j0 + warp; j < j1; j += blockDim.x / 32) {
            float s0 = 0.f, s1 = 0.f, s2 = 0.f;
            if (off >= 0) {
                sf_column_sums(Z, j, S.near_end[t] - off, massonly, c,
                               [&](int k, float4& p, float& l) {
                                   p = Z.near[off + k];
                                   l = p.w;
                               },
                               s0, s1, s2, npair);
            } else {
                sf_column_sums(Z, j, ni, massonly, c,
                               [&](int k, float4& p, float& l) {
                                   p = a.p[i0 + k];
                                   float vmax;
                                   l = k < nl ? Z.lse[k] : sf_row_lse(a, S, Z, t, p, dust, npair, vmax);
                               },
                               s0, s1, s2, npair);
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
        const float cg = S.cs[t].x, sg = S.cs[t].y;
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

__global__ void __launch_bounds__(kSfThreads, kSfCtasPerSm) single_fit_kernel(SfArgs a) {
    extern __shared__ float M6[];  // 6 M floats of MM matrices, then T float2 of the angle table
    __shared__ SfShared S;
    SfScratch Z = sf_slice(a, blockIdx.x);
    sf_angles(a, S, (float2*)(M6 + 6 * a.M));
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
            sf_refresh(a, S, Z, negK);  // E-step pose
            sf_near(a, S, Z, negK, dust, npair, a.n_newton > 0);
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
        float negK = -a.G.D * a.G.D * log2e / a.eps_final, dust = -a.c_out * log2e / a.eps_final;
        sf_refresh(a, S, Z, negK);
        sf_near(a, S, Z, negK, dust, npair, false);
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
    extern __shared__ float2 sp_cs[];  // T float2: the angle table
    __shared__ SfShared S;
    __shared__ int wcnt[kSfThreads / 32];
    __shared__ int nnz;
    SfScratch Z = sf_slice(a, blockIdx.x);
    sf_angles(a, S, sp_cs);
    const float log2e = 1.4426950408889634f;
    const float negK = -a.G.D * a.G.D * log2e / sp.eps_s, kc = a.c_out * log2e / sp.eps_s;
    for (int n = blockIdx.x; n < a.S; n += gridDim.x) {
        if (threadIdx.x < 9) S.R[threadIdx.x] = a.R0[9 * n + threadIdx.x];
        if (threadIdx.x < 3) S.x[threadIdx.x] = a.x0[3 * n + threadIdx.x];
        if (threadIdx.x == 0) nnz = 0;
        __syncthreads();
        sf_cut(a, S, Z);
        if (S.overflow && threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_CAPACITY);
        sf_refresh(a, S, Z, negK);
        int base = count_only ? 0 : sp.row_ptr[n];
        for (int t = 0; t < a.T; ++t) {
            int j0 = S.t_off[t], j1 = S.t_off[t + 1];
            if (j0 == j1) continue;
            for (int i0 = a.I_off[t]; i0 < a.I_off[t + 1]; i0 += blockDim.x) {
                int i = i0 + threadIdx.x;
                float val = 0.0f;
                if (i < a.I_off[t + 1]) {
                    const SfRowG g = sf_rowg(a.p[i], Z.cE + 3 * j0);
                    Lse2 L;
                    L.m = kNegHuge;
                    L.s = 0.0f;
                    for (int j = j0; j < j1; ++j) L.merge(sf_pair_v(g, Z.rk[j]), 1.0f);
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
    if (a.S > 0) spot_matrix_kernel<<<ctas, kSfThreads, sizeof(float2) * (size_t)a.T, s>>>(a, sp, count_only ? 1 : 0);
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

cudaError_t single_fit_run(const SfArgs& a, int ctas, cudaStream_t s) {
    size_t shm = sizeof(float) * 6 * (size_t)a.M + sizeof(float2) * (size_t)a.T;
    if (shm > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(single_fit_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
        if (e != cudaSuccess) return e;
    }
    if (a.S > 0) single_fit_kernel<<<ctas, kSfThreads, shm, s>>>(a);
    return cudaGetLastError();
}

}  // namespace laue
