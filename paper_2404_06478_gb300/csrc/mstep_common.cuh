// mstep_common.cuh — small linear algebra shared by the multi-grain M-step,
// the single-grain fits and the adjoint: rotations about +y, symmetric 3x3
// helpers, cyclic Jacobi, Horn's quaternion solution of Wahba's problem, the
// regularised Newton step and the MM accumulation (paper Appendix "M-steps for
// grain position and rotation", Appendix "Wahba's problem").
#pragma once

#include "common.cuh"

namespace laue {

__device__ __forceinline__ void gamma_t(float om, float& c, float& s) { sincosf(om, &s, &c); }

// Gamma = [[c, 0, s], [0, 1, 0], [-s, 0, c]]: v_lab = Gamma v, Gamma^T v_lab.
__device__ __forceinline__ void gam_apply(float c, float s, const float* v, float* o) {
    o[0] = c * v[0] + s * v[2];
    o[1] = v[1];
    o[2] = -s * v[0] + c * v[2];
}
__device__ __forceinline__ void gamT_apply(float c, float s, const float* v, float* o) {
    o[0] = c * v[0] - s * v[2];
    o[1] = v[1];
    o[2] = s * v[0] + c * v[2];
}

// Symmetric 3x3 stored as (xx, xy, xz, yy, yz, zz).
__device__ __forceinline__ void sym_full(const float* h, float* A) {
    A[0] = h[0]; A[1] = h[1]; A[2] = h[2];
    A[3] = h[1]; A[4] = h[3]; A[5] = h[4];
    A[6] = h[2]; A[7] = h[4]; A[8] = h[5];
}

// Gamma^T A Gamma for symmetric A given as 6 values.
__device__ __forceinline__ void sym_gamT_gam(float c, float s, const float* h, float* out) {
    float A[9], T1[9];
    sym_full(h, A);
    // T1 = A Gamma
    for (int r = 0; r < 3; ++r) {
        T1[3 * r + 0] = A[3 * r + 0] * c - A[3 * r + 2] * s;
        T1[3 * r + 1] = A[3 * r + 1];
        T1[3 * r + 2] = A[3 * r + 0] * s + A[3 * r + 2] * c;
    }
    // out = Gamma^T T1
    float O[9];
    for (int col = 0; col < 3; ++col) {
        O[0 + col] = c * T1[0 + col] - s * T1[6 + col];
        O[3 + col] = T1[3 + col];
        O[6 + col] = s * T1[0 + col] + c * T1[6 + col];
    }
    out[0] = O[0]; out[1] = O[1]; out[2] = O[2]; out[3] = O[4]; out[4] = O[5]; out[5] = O[8];
}

// Cyclic Jacobi eigen-decomposition of an n x n symmetric matrix (n = 3, 4),
// in place; V receives the eigenvectors as columns.
template <int n>
__device__ __forceinline__ void jacobi(float* A, float* V) {
    for (int a = 0; a < n * n; ++a) V[a] = (a % (n + 1) == 0) ? 1.0f : 0.0f;
    for (int sweep = 0; sweep < 12; ++sweep) {
        float off = 0.0f, tot = 0.0f;
        for (int p = 0; p < n; ++p)
            for (int q = 0; q < n; ++q) {
                float v = A[n * p + q] * A[n * p + q];
                tot += v;
                if (p != q) off += v;
            }
        if (off <= 1e-14f * tot || off == 0.0f) break;
        for (int p = 0; p < n - 1; ++p)
            for (int q = p + 1; q < n; ++q) {
                float apq = A[n * p + q];
                if (apq == 0.0f) continue;
                float theta = (A[n * q + q] - A[n * p + p]) / (2.0f * apq);
                float t = (theta >= 0.0f ? 1.0f : -1.0f) / (fabsf(theta) + sqrtf(theta * theta + 1.0f));
                float c = rsqrtf(t * t + 1.0f), s = t * c;
                for (int k = 0; k < n; ++k) {
                    float akp = A[n * k + p], akq = A[n * k + q];
                    A[n * k + p] = c * akp - s * akq;
                    A[n * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < n; ++k) {
                    float apk = A[n * p + k], aqk = A[n * q + k];
                    A[n * p + k] = c * apk - s * aqk;
                    A[n * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < n; ++k) {
                    float vkp = V[n * k + p], vkq = V[n * k + q];
                    V[n * k + p] = c * vkp - s * vkq;
                    V[n * k + q] = s * vkp + c * vkq;
                }
            }
    }
}

// Rotation maximising tr(R^T B) (Wahba, B = sum a b^T) from the top
// eigenvector of Horn's matrix with S = B^T.  Returns false when the top
// eigenvalue is (nearly) degenerate, i.e. rank(B) < 2.
__device__ __forceinline__ bool wahba_horn(const float* B, float* R) {
    float S[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) S[3 * a + b] = B[3 * b + a];
    float Sxx = S[0], Sxy = S[1], Sxz = S[2], Syx = S[3], Syy = S[4], Syz = S[5], Szx = S[6], Szy = S[7],
          Szz = S[8];
    float Nm[16] = {Sxx + Syy + Szz, Syz - Szy,        Szx - Sxz,        Sxy - Syx,
                    Syz - Szy,       Sxx - Syy - Szz,  Sxy + Syx,        Szx + Sxz,
                    Szx - Sxz,       Sxy + Syx,        -Sxx + Syy - Szz, Syz + Szy,
                    Sxy - Syx,       Szx + Sxz,        Syz + Szy,        -Sxx - Syy + Szz};
    float V[16];
    jacobi<4>(Nm, V);
    int top = 0;
    for (int k = 1; k < 4; ++k)
        if (Nm[5 * k] > Nm[5 * top]) top = k;
    float l1 = Nm[5 * top], l2 = -3.0e38f, scale = 0.0f;
    for (int k = 0; k < 4; ++k) {
        scale = fmaxf(scale, fabsf(Nm[5 * k]));
        if (k != top) l2 = fmaxf(l2, Nm[5 * k]);
    }
    if (!(scale > 0.0f) || l1 - l2 <= 1e-6f * scale) return false;
    float w = V[0 * 4 + top], x = V[1 * 4 + top], y = V[2 * 4 + top], z = V[3 * 4 + top];
    float nq = rsqrtf(w * w + x * x + y * y + z * z);
    w *= nq; x *= nq; y *= nq; z *= nq;
    R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z);     R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);     R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);     R[7] = 2 * (y * z + w * x);     R[8] = 1 - 2 * (x * x + y * y);
    return true;
}

// Regularised Newton ascent step: dx = (H - iota I)^-1 g with
// iota = max(0, lmax(H) + hreg |H|_F); H given as 6 symmetric entries.
// Returns false (no step) for a zero or singular matrix.
__device__ __forceinline__ bool newton_step(const float* g, const float* h6, float hreg, float* dx) {
    float H[9], Hc[9], V[9];
    sym_full(h6, H);
    float fro = 0.0f;
    for (int k = 0; k < 9; ++k) fro += H[k] * H[k];
    fro = sqrtf(fro);
    if (!(fro > 0.0f)) return false;
    for (int k = 0; k < 9; ++k) Hc[k] = H[k];
    jacobi<3>(Hc, V);
    float lmax = fmaxf(Hc[0], fmaxf(Hc[4], Hc[8]));
    float iota = fmaxf(0.0f, lmax + hreg * fro);
    H[0] -= iota;
    H[4] -= iota;
    H[8] -= iota;
    float det = H[0] * (H[4] * H[8] - H[5] * H[7]) - H[1] * (H[3] * H[8] - H[5] * H[6]) +
                H[2] * (H[3] * H[7] - H[4] * H[6]);
    if (det == 0.0f || !isfinite(det)) return false;
    float inv[9];
    inv[0] = (H[4] * H[8] - H[5] * H[7]) / det;
    inv[1] = (H[2] * H[7] - H[1] * H[8]) / det;
    inv[2] = (H[1] * H[5] - H[2] * H[4]) / det;
    inv[3] = (H[5] * H[6] - H[3] * H[8]) / det;
    inv[4] = (H[0] * H[8] - H[2] * H[6]) / det;
    inv[5] = (H[2] * H[3] - H[0] * H[5]) / det;
    inv[6] = (H[3] * H[7] - H[4] * H[6]) / det;
    inv[7] = (H[1] * H[6] - H[0] * H[7]) / det;
    inv[8] = (H[0] * H[4] - H[1] * H[3]) / det;
    for (int a = 0; a < 3; ++a) dx[a] = inv[3 * a] * g[0] + inv[3 * a + 1] * g[1] + inv[3 * a + 2] * g[2];
    return true;
}

// M_m = M0_m + max(0, -lmin(M0_m)) I, in place (6 symmetric entries).
__device__ __forceinline__ void psd_shift(float* m6) {
    float A[9], V[9];
    sym_full(m6, A);
    jacobi<3>(A, V);
    float lmin = fminf(A[0], fminf(A[4], A[8]));
    float iota = lmin < 0.0f ? -lmin : 0.0f;
    m6[0] += iota;
    m6[3] += iota;
    m6[5] += iota;
}

// B += (M R w) w^T for one plane (the linearised MM objective).
__device__ __forceinline__ void mm_accumulate(const float* m6, float4 wd, const float* R, float* B) {
    float w[3] = {wd.x, wd.y, wd.z};
    float Rw[3], a[3], Mf[9];
    for (int r = 0; r < 3; ++r) Rw[r] = R[3 * r] * w[0] + R[3 * r + 1] * w[1] + R[3 * r + 2] * w[2];
    sym_full(m6, Mf);
    for (int r = 0; r < 3; ++r) a[r] = Mf[3 * r] * Rw[0] + Mf[3 * r + 1] * Rw[1] + Mf[3 * r + 2] * Rw[2];
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) B[3 * r + c] += a[r] * w[c];
}

// Gram-Schmidt on the rows of a nearly orthogonal 3x3 matrix (the third row
// is the cross product of the first two, so the result is a rotation).
__device__ __forceinline__ void orthonormalise_rows(float* R) {
    float n0 = rsqrtf(R[0] * R[0] + R[1] * R[1] + R[2] * R[2]);
    for (int k = 0; k < 3; ++k) R[k] *= n0;
    float d = R[0] * R[3] + R[1] * R[4] + R[2] * R[5];
    for (int k = 0; k < 3; ++k) R[3 + k] -= d * R[k];
    float n1 = rsqrtf(R[3] * R[3] + R[4] * R[4] + R[5] * R[5]);
    for (int k = 0; k < 3; ++k) R[3 + k] *= n1;
    R[6] = R[1] * R[5] - R[2] * R[4];
    R[7] = R[2] * R[3] - R[0] * R[5];
    R[8] = R[0] * R[4] - R[1] * R[3];
}

}  // namespace laue
