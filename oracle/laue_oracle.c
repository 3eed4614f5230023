/*
 * laue_oracle.c — plain, slow, FP64 CPU oracle for the LaueOT Sinkhorn-EM
 * hot path (arXiv 2404.06478).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the tests, the smoke check and
 * the benchmark's CPU-baseline leg load this library.  It shares no source,
 * header, table or helper with the CUDA path, and it is deliberately written
 * as loops over the definitions, with no blocking, fusion or reordering.
 *
 * Every function names the passage of the paper it restates.  Readings of
 * passages that the paper leaves silent, ambiguous or garbled:
 *   frame       beam e=(0,0,1); detectors are planes given by (centre, normal,
 *               half size); sample rotation Gamma_t about +y by omega_t.
 *   ray / lam   r = e - 2(u.e)u for every plane; lambda = 2 d |u.e|, i.e. the
 *               member of the Friedel pair +-hkl with positive wavelength
 *               (Eqs. ray_mnt and wavelength_lambda).
 *   harmonics   reflections n*g0 share one ray; a direction is visible when some
 *               harmonic has lambda0/n inside the band and reports the largest
 *               such wavelength.
 *   cost        C_ij = D^2 |rhat_ij - r_j|^2 = 2 D^2 (1 - rhat.r), so that
 *               L_ij = kappa - kappa C_ij / (2 D^2) (Eq. update_L up to a
 *               constant); outlier column C_i0 = c_out, unmatched-model row
 *               C_0j = 0, corner C_00 = c_out.  Gibbs kernel exp(-C/eps),
 *               eps in mm^2.
 *   masses      observed and model spots carry 1; the unmatched-model row
 *               carries U = ceil(frac |J|), the outlier column O = U + |I| - |J|
 *               (balance of Section "E-step with Sinkhorn updates"); when O < 0,
 *               U = |J| - |I| and O = 0.  Per-angle mode applies the same rule
 *               inside each angle block.
 *   Sinkhorn    log-domain, start f = g = 0 (x = y = 1), row update first
 *               (Algorithm BalancedOT).
 *   Newton      exact gradient/Hessian of sum Q rhat.r in the lab frame (the
 *               appendix formulas without Gamma and sign); ascent step
 *               x <- x - (H - iota I)^-1 g, iota = max(0, lmax(H) + hreg |H|_F).
 *   MM          iota_m = max(0, -lmin(M0_m)); Wahba by SVD with the
 *               determinant correction; rank(B) < 2 keeps R.
 */
#include "laue_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------- */
/* small linear algebra (row-major 3x3)                                        */
/* ------------------------------------------------------------------------- */

static void mat_vec(const double A[9], const double v[3], double out[3]) {
    for (int a = 0; a < 3; ++a)
        out[a] = A[3 * a + 0] * v[0] + A[3 * a + 1] * v[1] + A[3 * a + 2] * v[2];
}

static void matT_vec(const double A[9], const double v[3], double out[3]) {
    for (int a = 0; a < 3; ++a)
        out[a] = A[0 + a] * v[0] + A[3 + a] * v[1] + A[6 + a] * v[2];
}

static void mat_mul(const double A[9], const double B[9], double C[9]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double s = 0.0;
            for (int k = 0; k < 3; ++k) s += A[3 * a + k] * B[3 * k + b];
            C[3 * a + b] = s;
        }
}

static double dot3(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

static double det3(const double A[9]) {
    return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
           A[2] * (A[3] * A[7] - A[4] * A[6]);
}

static void cross3(const double a[3], const double b[3], double c[3]) {
    c[0] = a[1] * b[2] - a[2] * b[1];
    c[1] = a[2] * b[0] - a[0] * b[2];
    c[2] = a[0] * b[1] - a[1] * b[0];
}

/* Solve A y = b by the adjugate (Cramer); returns 0 if A is singular. */
static int solve3(const double A[9], const double b[3], double y[3]) {
    double det = det3(A);
    if (det == 0.0 || !isfinite(det)) return 0;
    double inv[9];
    inv[0] = (A[4] * A[8] - A[5] * A[7]) / det;
    inv[1] = (A[2] * A[7] - A[1] * A[8]) / det;
    inv[2] = (A[1] * A[5] - A[2] * A[4]) / det;
    inv[3] = (A[5] * A[6] - A[3] * A[8]) / det;
    inv[4] = (A[0] * A[8] - A[2] * A[6]) / det;
    inv[5] = (A[2] * A[3] - A[0] * A[5]) / det;
    inv[6] = (A[3] * A[7] - A[4] * A[6]) / det;
    inv[7] = (A[1] * A[6] - A[0] * A[7]) / det;
    inv[8] = (A[0] * A[4] - A[1] * A[3]) / det;
    mat_vec(inv, b, y);
    return 1;
}

/* Cyclic Jacobi eigen-decomposition of a symmetric 3x3 matrix (textbook).
 * evals ascending; evecs columns (row-major storage, column k = vector k). */
void orc_sym3_eig(const double Ain[9], double evals[3], double evecs[9]) {
    double A[9], V[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(A, Ain, sizeof(A));
    for (int sweep = 0; sweep < 100; ++sweep) {
        double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
        double tot = off + A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
        if (off <= 1e-300 || off <= 1e-32 * tot) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double apq = A[3 * p + q];
                if (apq == 0.0) continue;
                double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
                double t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
                double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
                /* A <- J^T A J with J the rotation in the (p,q) plane */
                for (int k = 0; k < 3; ++k) {
                    double akp = A[3 * k + p], akq = A[3 * k + q];
                    A[3 * k + p] = c * akp - s * akq;
                    A[3 * k + q] = s * akp + c * akq;
                }
                for (int k = 0; k < 3; ++k) {
                    double apk = A[3 * p + k], aqk = A[3 * q + k];
                    A[3 * p + k] = c * apk - s * aqk;
                    A[3 * q + k] = s * apk + c * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    double vkp = V[3 * k + p], vkq = V[3 * k + q];
                    V[3 * k + p] = c * vkp - s * vkq;
                    V[3 * k + q] = s * vkp + c * vkq;
                }
            }
    }
    /* sort ascending */
    int idx[3] = {0, 1, 2};
    double d[3] = {A[0], A[4], A[8]};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (d[idx[b]] < d[idx[a]]) { int tmp = idx[a]; idx[a] = idx[b]; idx[b] = tmp; }
    for (int k = 0; k < 3; ++k) {
        evals[k] = d[idx[k]];
        for (int a = 0; a < 3; ++a) evecs[3 * a + k] = V[3 * a + idx[k]];
    }
}

/* One-sided (Hestenes) Jacobi SVD of a 3x3 matrix: B = U diag(S) V^T,
 * S descending.  Columns of U for zero singular values are completed to an
 * orthonormal basis. */
void orc_svd3(const double B[9], double U[9], double S[3], double V[9]) {
    double A[9], W[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
    memcpy(A, B, sizeof(A));
    for (int sweep = 0; sweep < 100; ++sweep) {
        int rotated = 0;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double alpha = 0, beta = 0, gamma = 0;
                for (int k = 0; k < 3; ++k) {
                    alpha += A[3 * k + p] * A[3 * k + p];
                    beta += A[3 * k + q] * A[3 * k + q];
                    gamma += A[3 * k + p] * A[3 * k + q];
                }
                if (gamma == 0.0 || fabs(gamma) <= 1e-15 * sqrt(alpha * beta)) continue;
                rotated = 1;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
                for (int k = 0; k < 3; ++k) {
                    double ap = A[3 * k + p], aq = A[3 * k + q];
                    A[3 * k + p] = c * ap - s * aq;
                    A[3 * k + q] = s * ap + c * aq;
                    double wp = W[3 * k + p], wq = W[3 * k + q];
                    W[3 * k + p] = c * wp - s * wq;
                    W[3 * k + q] = s * wp + c * wq;
                }
            }
        if (!rotated) break;
    }
    double sv[3];
    for (int k = 0; k < 3; ++k)
        sv[k] = sqrt(A[k] * A[k] + A[3 + k] * A[3 + k] + A[6 + k] * A[6 + k]);
    int idx[3] = {0, 1, 2};
    for (int a = 0; a < 3; ++a)
        for (int b = a + 1; b < 3; ++b)
            if (sv[idx[b]] > sv[idx[a]]) { int tmp = idx[a]; idx[a] = idx[b]; idx[b] = tmp; }
    double smax = sv[idx[0]];
    int nz = 0;
    for (int k = 0; k < 3; ++k) {
        int src = idx[k];
        S[k] = sv[src];
        for (int a = 0; a < 3; ++a) V[3 * a + k] = W[3 * a + src];
        if (S[k] > 1e-300 && S[k] > 1e-15 * smax) {
            for (int a = 0; a < 3; ++a) U[3 * a + k] = A[3 * a + src] / S[k];
            ++nz;
        } else {
            for (int a = 0; a < 3; ++a) U[3 * a + k] = 0.0;
        }
    }
    /* complete U where singular values vanish */
    if (nz == 2) {
        double u0[3] = {U[0], U[3], U[6]}, u1[3] = {U[1], U[4], U[7]}, u2[3];
        cross3(u0, u1, u2);
        for (int a = 0; a < 3; ++a) U[3 * a + 2] = u2[a];
    } else if (nz < 2) {
        double u0[3];
        if (nz == 1) {
            u0[0] = U[0]; u0[1] = U[3]; u0[2] = U[6];
        } else {
            u0[0] = 1; u0[1] = 0; u0[2] = 0;
        }
        double tmp[3] = {1, 0, 0};
        if (fabs(u0[0]) > 0.9) { tmp[0] = 0; tmp[1] = 1; }
        double u1[3], u2[3];
        cross3(u0, tmp, u1);
        double n1 = sqrt(dot3(u1, u1));
        for (int a = 0; a < 3; ++a) u1[a] /= n1;
        cross3(u0, u1, u2);
        for (int a = 0; a < 3; ++a) {
            U[3 * a + 0] = u0[a];
            U[3 * a + 1] = u1[a];
            U[3 * a + 2] = u2[a];
        }
    }
}

/* Appendix "Wahba's problem", Algorithm Wahba: B = sum w a b^T, B = U S V^T,
 * R = U diag(1, 1, det U det V) V^T.  Returns 0 (R untouched) when rank B < 2. */
int orc_wahba(const double B[9], double R[9]) {
    double U[9], S[3], V[9];
    orc_svd3(B, U, S, V);
    if (!(S[0] > 0.0) || S[1] <= 1e-12 * S[0]) return 0;
    double s = det3(U) * det3(V);
    double M[9] = {1, 0, 0, 0, 1, 0, 0, 0, s};
    double UM[9], Vt[9];
    mat_mul(U, M, UM);
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Vt[3 * a + b] = V[3 * b + a];
    mat_mul(UM, Vt, R);
    return 1;
}

/* ------------------------------------------------------------------------- */
/* geometry                                                                    */
/* ------------------------------------------------------------------------- */

typedef struct {
    double e[3];
    double lam_min, lam_max, D;
    int n_det;
    double ctr[4][3], nrm[4][3], half[4];
    double Dd[4];            /* cost length of each detector */
    double a1[4][3], a2[4][3];  /* in-plane axes of each detector */
} geom_t;

/* Packed geometry: beam (3), lam_min, lam_max, D, n_det, then per detector
 * centre (3), normal (3), half size, cost length (<= 0: D).  A detector's
 * square is the set of plane points s with |(s - centre).a| < half for both
 * in-plane axes a1 = (y x n)/|y x n| (x when n is along y) and a2 = n x a1
 * (n the unit normal): for a detector normal to the beam the axes are x and
 * y and the square has edges along them. */
static void geom_unpack(const double* g, geom_t* G) {
    for (int a = 0; a < 3; ++a) G->e[a] = g[a];
    G->lam_min = g[3];
    G->lam_max = g[4];
    G->D = g[5];
    G->n_det = (int)g[6];
    if (G->n_det > 4) G->n_det = 4;
    for (int k = 0; k < G->n_det; ++k) {
        const double* q = g + 7 + 8 * k;
        for (int a = 0; a < 3; ++a) {
            G->ctr[k][a] = q[a];
            G->nrm[k][a] = q[3 + a];
        }
        G->half[k] = q[6];
        G->Dd[k] = q[7] > 0.0 ? q[7] : G->D;
        double nn = sqrt(dot3(G->nrm[k], G->nrm[k]));
        double n[3] = {G->nrm[k][0] / nn, G->nrm[k][1] / nn, G->nrm[k][2] / nn};
        double a1[3] = {n[2], 0.0, -n[0]};  /* y x n */
        double l1 = sqrt(dot3(a1, a1));
        if (l1 < 1e-12) {
            a1[0] = 1.0; a1[1] = 0.0; a1[2] = 0.0;
        } else {
            for (int a = 0; a < 3; ++a) a1[a] /= l1;
        }
        double a2[3] = {n[1] * a1[2] - n[2] * a1[1], n[2] * a1[0] - n[0] * a1[2], n[0] * a1[1] - n[1] * a1[0]};
        for (int a = 0; a < 3; ++a) {
            G->a1[k][a] = a1[a];
            G->a2[k][a] = a2[a];
        }
    }
}

/* Cost length of model spot j: the distance of the detector its ray hits
 * (det[j]), D when the detector is unknown. */
static double det_D(const geom_t* G, const int* det, long j) {
    if (det) {
        int k = det[j];
        if (k >= 0 && k < G->n_det) return G->Dd[k];
    }
    return G->D;
}

/* Cost lengths of n model spots from their detectors (det_D). */
void orc_cost_lengths(const double* geom, int n, const int* det, double* out) {
    geom_t G;
    geom_unpack(geom, &G);
    for (int j = 0; j < n; ++j) out[j] = det_D(&G, det, j);
}

/* Section "Tomography experiments": Gamma_t, rotation about +y by omega. */
void orc_gamma(double omega, double G[9]) {
    double c = cos(omega), s = sin(omega);
    G[0] = c;  G[1] = 0; G[2] = s;
    G[3] = 0;  G[4] = 1; G[5] = 0;
    G[6] = -s; G[7] = 0; G[8] = c;
}

static int gcd_int(int a, int b) {
    a = abs(a); b = abs(b);
    while (b) { int t = a % b; a = b; b = t; }
    return a;
}

static int allowed_hkl(int h, int k, int l, int centering) {
    if (h == 0 && k == 0 && l == 0) return 0;
    if (centering == 1) return ((h + k + l) % 2 + 2) % 2 == 0;           /* I: h+k+l even */
    if (centering == 2) {                                                 /* F: unmixed */
        int ph = (h % 2 + 2) % 2, pk = (k % 2 + 2) % 2, pl = (l % 2 + 2) % 2;
        return ph == pk && pk == pl;
    }
    return 1;                                                             /* P */
}

typedef struct { int g0[3]; int n2; int nh; double w[3]; double d0; } refl_t;

static int refl_cmp(const void* A, const void* B) {
    const refl_t* a = (const refl_t*)A;
    const refl_t* b = (const refl_t*)B;
    if (a->n2 != b->n2) return a->n2 < b->n2 ? -1 : 1;
    for (int k = 0; k < 3; ++k)
        if (a->g0[k] != b->g0[k]) return a->g0[k] > b->g0[k] ? -1 : 1;
    return 0;
}

/* Section "Crystallographic planes" (d = a / sqrt(h^2+k^2+l^2)) and the
 * plausible plane set of Section "Tomography experiments": one entry per ray
 * direction.  The Friedel pair +-hkl shares the ray; harmonics n*g0 share it
 * too.  Order: |g0|^2 ascending, then g0 (h, k, l) descending. */
int orc_reflections(double a, int hmax, int centering, int cap,
                    double* w, double* d0, int* nharm, int* hkl0) {
    int maxn = (2 * hmax + 1) * (2 * hmax + 1) * (2 * hmax + 1);
    refl_t* list = (refl_t*)malloc(sizeof(refl_t) * (size_t)maxn);
    int n = 0;
    for (int h = -hmax; h <= hmax; ++h)
        for (int k = -hmax; k <= hmax; ++k)
            for (int l = -hmax; l <= hmax; ++l) {
                if (h == 0 && k == 0 && l == 0) continue;
                if (gcd_int(gcd_int(h, k), l) != 1) continue;
                int first = h != 0 ? h : (k != 0 ? k : l);
                if (first < 0) continue;      /* one of each Friedel pair */
                int pmax = abs(h);
                if (abs(k) > pmax) pmax = abs(k);
                if (abs(l) > pmax) pmax = abs(l);
                int mult[64], nm = 0;
                for (int m = 1; m * pmax <= hmax && nm < 64; ++m)
                    if (allowed_hkl(m * h, m * k, m * l, centering)) mult[nm++] = m;
                if (nm == 0) continue;
                /* allowed multipliers must be m0, 2 m0, ..., nm m0 */
                for (int q = 0; q < nm; ++q)
                    if (mult[q] != (q + 1) * mult[0]) { free(list); return -1; }
                refl_t* R = &list[n++];
                R->g0[0] = mult[0] * h;
                R->g0[1] = mult[0] * k;
                R->g0[2] = mult[0] * l;
                R->n2 = R->g0[0] * R->g0[0] + R->g0[1] * R->g0[1] + R->g0[2] * R->g0[2];
                R->nh = nm;
                double pn = sqrt((double)(h * h + k * k + l * l));
                R->w[0] = h / pn; R->w[1] = k / pn; R->w[2] = l / pn;
                R->d0 = a / sqrt((double)R->n2);
            }
    qsort(list, (size_t)n, sizeof(refl_t), refl_cmp);
    for (int m = 0; m < n && m < cap; ++m) {
        for (int q = 0; q < 3; ++q) {
            w[3 * m + q] = list[m].w[q];
            if (hkl0) hkl0[3 * m + q] = list[m].g0[q];
        }
        d0[m] = list[m].d0;
        nharm[m] = list[m].nh;
    }
    free(list);
    return n;
}

/* Eqs. ray_mnt, s_mnt, wavelength and the cut model_spot_cut for one
 * (angle, grain, plane).  Returns 1 if visible.  *margin is the smallest
 * relative distance of any in/out decision from its threshold. */
static int ray_one(const geom_t* G, const double Gam[9], const double R[9], const double x[3],
                   const double w[3], double d0, int nh,
                   double r[3], double* lam, double s[3], int* det, double c[3], double* margin) {
    double v[3], u[3];
    mat_vec(R, w, v);
    mat_vec(Gam, v, u);
    mat_vec(Gam, x, c);
    double ue = dot3(u, G->e);
    for (int a = 0; a < 3; ++a) r[a] = G->e[a] - 2.0 * ue * u[a];
    double lam0 = 2.0 * d0 * fabs(ue);
    double mrg = INFINITY;
    int in_band = 0;
    *lam = lam0;
    for (int n = 1; n <= nh; ++n) {
        double ln = lam0 / n;
        double m1 = fabs(ln - G->lam_min) / G->lam_min;
        double m2 = fabs(ln - G->lam_max) / G->lam_max;
        if (m1 < mrg) mrg = m1;
        if (m2 < mrg) mrg = m2;
        if (!in_band && ln >= G->lam_min && ln <= G->lam_max) {
            in_band = 1;
            *lam = ln;
        }
    }
    int best = -1;
    double best_tau = INFINITY;
    for (int k = 0; k < G->n_det; ++k) {
        double den = dot3(G->nrm[k], r);
        if (den == 0.0) continue;
        double gc[3] = {G->ctr[k][0] - c[0], G->ctr[k][1] - c[1], G->ctr[k][2] - c[2]};
        double tau = dot3(G->nrm[k], gc) / den;
        if (!(tau > 0.0)) continue;
        double sk[3], ds[3];
        for (int a = 0; a < 3; ++a) {
            sk[a] = c[a] + tau * r[a];
            ds[a] = sk[a] - G->ctr[k][a];
        }
        double d1 = fabs(dot3(ds, G->a1[k])), d2 = fabs(dot3(ds, G->a2[k]));
        double dist = d1 > d2 ? d1 : d2;
        double m3 = fabs(G->half[k] - dist) / G->half[k];
        if (m3 < mrg) mrg = m3;
        if (dist < G->half[k] && tau < best_tau) {
            best_tau = tau;
            best = k;
            for (int a = 0; a < 3; ++a) s[a] = sk[a];
        }
    }
    *det = best;
    *margin = mrg;
    return in_band && best >= 0;
}

/* Forward Laue model + cut (Eqs. ray_mnt, s_mnt, model_spot_cut): every
 * (t, n, m); visible spots are listed sorted by (t, n, m).  Writes at most cap
 * spots; returns the number of visible spots. */
long orc_forward(const double* geom, const double* w, const double* d0, const int* nharm, int M,
                 const double* R, const double* x, int N, const double* omega, int T,
                 long cap, int* J_off, int* grain, int* plane, double* ray4, double* spot3,
                 int* det, double* center3, signed char* vis_all, double* margin_all) {
    geom_t G;
    geom_unpack(geom, &G);
    long J = 0;
    for (int t = 0; t < T; ++t) {
        double Gam[9];
        orc_gamma(omega[t], Gam);
        if (J_off) J_off[t] = (int)J;
        for (int n = 0; n < N; ++n)
            for (int m = 0; m < M; ++m) {
                double r[3], lam, s[3], c[3], mrg;
                int dk;
                int vis = ray_one(&G, Gam, R + 9 * n, x + 3 * n, w + 3 * m, d0[m], nharm[m],
                                  r, &lam, s, &dk, c, &mrg);
                long flat = ((long)t * N + n) * M + m;
                if (vis_all) vis_all[flat] = (signed char)vis;
                if (margin_all) margin_all[flat] = mrg;
                if (!vis) continue;
                if (J < cap) {
                    grain[J] = n;
                    plane[J] = m;
                    for (int a = 0; a < 3; ++a) {
                        ray4[4 * J + a] = r[a];
                        spot3[3 * J + a] = s[a];
                        center3[3 * J + a] = c[a];
                    }
                    ray4[4 * J + 3] = lam;
                    det[J] = dk;
                }
                ++J;
            }
    }
    if (J_off) J_off[T] = (int)J;
    return J;
}

/* Rays and grain centres of a frozen model-spot list at new poses (the list
 * stays fixed during multi-grain fitting, Section "Assignments with outlier
 * and missing spots"). */
void orc_refresh(const double* geom, const double* w, const double* d0, const int* nharm,
                 const double* R, const double* x, const double* omega, int T,
                 const int* J_off, const int* grain, const int* plane,
                 double* ray4, double* center3) {
    geom_t G;
    geom_unpack(geom, &G);
    for (int t = 0; t < T; ++t) {
        double Gam[9];
        orc_gamma(omega[t], Gam);
        for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
            int n = grain[j], m = plane[j];
            double v[3], u[3], c[3];
            mat_vec(R + 9 * n, w + 3 * m, v);
            mat_vec(Gam, v, u);
            mat_vec(Gam, x + 3 * n, c);
            double ue = dot3(u, G.e);
            for (int a = 0; a < 3; ++a) {
                ray4[4 * j + a] = G.e[a] - 2.0 * ue * u[a];
                center3[3 * j + a] = c[a];
            }
            double lam0 = 2.0 * d0[m] * fabs(ue), lam = lam0;
            for (int k = 1; k <= nharm[m]; ++k)
                if (lam0 / k >= G.lam_min && lam0 / k <= G.lam_max) { lam = lam0 / k; break; }
            ray4[4 * j + 3] = lam;
        }
    }
}

/* Section "The likelihood": ray estimate rhat_ij = (s_i - c_j)/|s_i - c_j| and
 * the pair cost C_ij = D^2 |rhat_ij - r_j|^2. */
double orc_pair_cost(const double* p, const double* c, const double* r, double D) {
    double d[3] = {p[0] - c[0], p[1] - c[1], p[2] - c[2]};
    double tau = sqrt(dot3(d, d));
    double e2 = 0.0;
    for (int a = 0; a < 3; ++a) {
        double q = d[a] / tau - r[a];
        e2 += q * q;
    }
    return D * D * e2;
}

/* orc_pair_cost for n pairs (p_k, c_k, r_k), k < n. */
void orc_pair_costs(int n, const double* p, const double* c, const double* r, double D, double* out) {
    for (int k = 0; k < n; ++k) out[k] = orc_pair_cost(p + 3 * k, c + 3 * k, r + 3 * k, D);
}

/* ------------------------------------------------------------------------- */
/* E-step: balanced entropic OT with dustbins                                  */
/* ------------------------------------------------------------------------- */

/* log-sum-exp of n values, two passes (max, then sum); -inf for an empty or
 * all -inf list. */
static double lse(const double* v, int n) {
    double m = -INFINITY;
    for (int k = 0; k < n; ++k)
        if (v[k] > m) m = v[k];
    if (m == -INFINITY) return -INFINITY;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += exp(v[k] - m);
    return m + log(s);
}

static double ceil_frac(double frac, long n) { return ceil(frac * (double)n - 1e-9); }

/* Section "E-step with Sinkhorn updates": T_b (unmatched model spots) is the
 * user variable, T_a = T_b - b^T 1 + a^T 1 balances the problem. */
void orc_masses(int mode, double frac, int T, const int* I_off, const int* J_off,
                double* U, double* O) {
    int nd = mode ? T : 1;
    for (int d = 0; d < nd; ++d) {
        long nI = mode ? I_off[d + 1] - I_off[d] : I_off[T];
        long nJ = mode ? J_off[d + 1] - J_off[d] : J_off[T];
        double u = ceil_frac(frac, nJ);
        double o = u + (double)nI - (double)nJ;
        if (o < 0) {
            u = (double)(nJ - nI);
            o = 0;
        }
        U[d] = u;
        O[d] = o;
    }
}

static double logm(double m) { return m > 0 ? log(m) : -INFINITY; }

/* Threads of the Sinkhorn updates (OpenMP builds only; 1 = sequential). */
static int orc_nthreads = 1;

int orc_set_threads(int n) {
    orc_nthreads = n > 0 ? n : 1;
#ifdef _OPENMP
    return orc_nthreads;
#else
    return 1;
#endif
}

/* Algorithm BalancedOT in the log domain on the extended matrix (observed
 * rows + unmatched-model row 0, model columns + outlier column 0), blocked by
 * angle (Q_ij = 0 unless t_i = t_j).  Runs exactly n_iter iterations, or
 * fewer when tol > 0 and the largest row-marginal violation drops below tol.
 * warm != 0 starts from the given potentials.  Returns iterations done. */
int orc_sinkhorn(const double* Dj, int T, const int* I_off, const double* p,
                 const int* J_off, const double* c, const double* r,
                 double eps, double c_out, int mode, double frac, int n_iter, double tol,
                 int warm, double* f, double* g, double* fd, double* gd) {
    int nI = I_off[T], nJ = J_off[T];
    int nd = mode ? T : 1;
    double* U = (double*)malloc(sizeof(double) * nd);
    double* O = (double*)malloc(sizeof(double) * nd);
    orc_masses(mode, frac, T, I_off, J_off, U, O);
    if (!warm) {
        for (int i = 0; i < nI; ++i) f[i] = 0.0;
        for (int j = 0; j < nJ; ++j) g[j] = 0.0;
        for (int d = 0; d < nd; ++d) fd[d] = gd[d] = 0.0;
    }
    int big = (nI > nJ ? nI : nJ) + 2;
    double* buf = (double*)malloc(sizeof(double) * big);
    int it;
    for (it = 0; it < n_iter; ++it) {
        /* row update: observed rows, then the unmatched-model rows (both from g);
         * the angle blocks are independent, so with threads they are shared out
         * (every f_i is still computed by one thread in the same order) */
#pragma omp parallel num_threads(orc_nthreads) if (orc_nthreads > 1)
        {
            double* b = (double*)malloc(sizeof(double) * big);
#pragma omp for schedule(dynamic)
            for (int t = 0; t < T; ++t) {
                int dd = mode ? t : 0;
                for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                    int n = 0;
                    for (int j = J_off[t]; j < J_off[t + 1]; ++j)
                        b[n++] = (g[j] - orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j])) / eps;
                    b[n++] = (gd[dd] - c_out) / eps;
                    f[i] = -eps * lse(b, n);
                }
            }
            free(b);
        }
        for (int d = 0; d < nd; ++d) {
            int j0 = mode ? J_off[d] : 0, j1 = mode ? J_off[d + 1] : nJ;
            int n = 0;
            for (int j = j0; j < j1; ++j) buf[n++] = g[j] / eps;
            buf[n++] = (gd[d] - c_out) / eps;
            fd[d] = eps * logm(U[d]) - eps * lse(buf, n);
        }
        /* column update: model columns, then the outlier columns (both from f) */
#pragma omp parallel num_threads(orc_nthreads) if (orc_nthreads > 1)
        {
            double* b = (double*)malloc(sizeof(double) * big);
#pragma omp for schedule(dynamic)
            for (int t = 0; t < T; ++t) {
                int dd = mode ? t : 0;
                for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
                    int n = 0;
                    for (int i = I_off[t]; i < I_off[t + 1]; ++i)
                        b[n++] = (f[i] - orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j])) / eps;
                    b[n++] = fd[dd] / eps;
                    g[j] = -eps * lse(b, n);
                }
            }
            free(b);
        }
        for (int d = 0; d < nd; ++d) {
            int i0 = mode ? I_off[d] : 0, i1 = mode ? I_off[d + 1] : nI;
            int n = 0;
            for (int i = i0; i < i1; ++i) buf[n++] = (f[i] - c_out) / eps;
            buf[n++] = (fd[d] - c_out) / eps;
            gd[d] = eps * logm(O[d]) - eps * lse(buf, n);
        }
        if (tol > 0.0) {
            double err[2];
            orc_harvest(Dj, T, I_off, p, J_off, c, r, eps, c_out, mode, frac, f, g, fd, gd,
                        NULL, NULL, err, NULL, NULL);
            if (err[0] < tol) { ++it; break; }
        }
    }
    free(buf);
    free(U);
    free(O);
    return it;
}

/* Plan read-out: Q = exp((f + g - C)/eps) on the extended matrix.  assign[i]
 * is the argmax of row i over its block's model spots and the outlier column
 * (-1); ties go to the lowest index, the outlier column only wins when it is
 * strictly larger.  margin[i] = (top1 - top2)/a_i.  err[0] = largest row
 * violation, err[1] = largest column violation (dust rows/columns relative to
 * their mass).  q[j] = sum_i Q_ij and v[j] = sum_i Q_ij rhat_ij over observed
 * rows.  Any output pointer may be NULL. */
void orc_harvest(const double* Dj, int T, const int* I_off, const double* p,
                 const int* J_off, const double* c, const double* r,
                 double eps, double c_out, int mode, double frac,
                 const double* f, const double* g, const double* fd, const double* gd,
                 int* assign, double* margin, double* err, double* q, double* v) {
    int nJ = J_off[T];
    int nd = mode ? T : 1;
    double* U = (double*)malloc(sizeof(double) * nd);
    double* O = (double*)malloc(sizeof(double) * nd);
    orc_masses(mode, frac, T, I_off, J_off, U, O);
    double* colsum = (double*)calloc((size_t)nJ + 1, sizeof(double));
    double* drow = (double*)calloc((size_t)nd, sizeof(double));
    double* dcol = (double*)calloc((size_t)nd, sizeof(double));
    double row_err = 0.0;
    if (q) for (int j = 0; j < nJ; ++j) q[j] = 0.0;
    if (v) for (int j = 0; j < 3 * nJ; ++j) v[j] = 0.0;
    for (int t = 0; t < T; ++t) {
        int dd = mode ? t : 0;
        for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
            double rs = 0.0, top1 = -1.0, top2 = -1.0;
            int arg = -1;
            for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
                double Cij = orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j]);
                double Qij = exp((f[i] + g[j] - Cij) / eps);
                rs += Qij;
                colsum[j] += Qij;
                if (q) q[j] += Qij;
                if (v) {
                    double d[3] = {p[3 * i] - c[3 * j], p[3 * i + 1] - c[3 * j + 1],
                                   p[3 * i + 2] - c[3 * j + 2]};
                    double tau = sqrt(dot3(d, d));
                    for (int a = 0; a < 3; ++a) v[3 * j + a] += Qij * d[a] / tau;
                }
                if (Qij > top1) { top2 = top1; top1 = Qij; arg = j; }
                else if (Qij > top2) top2 = Qij;
            }
            double Qi0 = exp((f[i] + gd[dd] - c_out) / eps);
            rs += Qi0;
            dcol[dd] += Qi0;
            if (Qi0 > top1) { top2 = top1; top1 = Qi0; arg = -1; }
            else if (Qi0 > top2) top2 = Qi0;
            if (top2 < 0) top2 = 0.0;
            if (assign) assign[i] = arg;
            if (margin) margin[i] = top1 - top2;
            double e = fabs(rs - 1.0);
            if (e > row_err) row_err = e;
        }
        for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
            double Q0j = exp((fd[dd] + g[j]) / eps);
            colsum[j] += Q0j;
            drow[dd] += Q0j;
        }
    }
    for (int d = 0; d < nd; ++d) {
        double Q00 = exp((fd[d] + gd[d] - c_out) / eps);
        drow[d] += Q00;
        dcol[d] += Q00;
    }
    double col_err = 0.0;
    for (int j = 0; j < nJ; ++j) {
        double e = fabs(colsum[j] - 1.0);
        if (e > col_err) col_err = e;
    }
    for (int d = 0; d < nd; ++d) {
        if (U[d] > 0) {
            double e = fabs(drow[d] - U[d]) / U[d];
            if (e > row_err) row_err = e;
        }
        if (O[d] > 0) {
            double e = fabs(dcol[d] - O[d]) / O[d];
            if (e > col_err) col_err = e;
        }
    }
    if (err) { err[0] = row_err; err[1] = col_err; }
    free(colsum); free(drow); free(dcol); free(U); free(O);
}

/* ------------------------------------------------------------------------- */
/* M-step: Newton on positions, MM (Wahba) on orientations                     */
/* ------------------------------------------------------------------------- */

typedef double (*qfun_t)(void* ctx, int i, int j);

typedef struct {
    const double *p, *cE, *rE, *f, *g;
    double eps;
    const geom_t* G;
    const int* det;
} qpot_ctx;

/* M-step weight of pair (i, j): Q_ij of a converged E-step from its
 * potentials and the E-step costs, times (D_j / D)^2 (the cost of the pair is
 * D_j^2 |rhat - r|^2 with D_j the distance of model spot j's detector, so the
 * maximised sum_ij Q_ij D_j^2 rhat.r carries that factor; 1 when every
 * detector has the cost length D). */
static double q_from_potentials(void* vctx, int i, int j) {
    qpot_ctx* ctx = (qpot_ctx*)vctx;
    double Dj = det_D(ctx->G, ctx->det, j);
    double C = orc_pair_cost(ctx->p + 3 * i, ctx->cE + 3 * j, ctx->rE + 3 * j, Dj);
    return exp((ctx->f[i] + ctx->g[j] - C) / ctx->eps) * (Dj / ctx->G->D) * (Dj / ctx->G->D);
}

/* Phi(x) = sum_{j in J_n} sum_{i in I_tj} Q_ij rhat_ij(x).r_j */
static double newton_objective(const geom_t* G, const double* omega, const int* I_off,
                               const double* p, const int* js, int nj, const int* jt,
                               const double* rE, qfun_t qf, void* qc, const double x[3]) {
    (void)G;
    double phi = 0.0;
    for (int k = 0; k < nj; ++k) {
        int j = js[k], t = jt[k];
        double Gam[9], c[3];
        orc_gamma(omega[t], Gam);
        mat_vec(Gam, x, c);
        for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
            double Q = qf(qc, i, j);
            if (Q == 0.0) continue;
            double d[3] = {p[3 * i] - c[0], p[3 * i + 1] - c[1], p[3 * i + 2] - c[2]};
            double tau = sqrt(dot3(d, d));
            phi += Q * dot3(d, rE + 3 * j) / tau;
        }
    }
    return phi;
}

/* Appendix "M-steps", grain position: Newton iterations (Algorithm
 * LauePosNewton) with the exact gradient and Hessian of Phi in the lab frame:
 *   dPhi/dc   = -(r - (rhat.r) rhat) / tau
 *   d2Phi/dc2 = (3 (rhat.r) rhat rhat^T - rhat r^T - r rhat^T - (rhat.r) I) / tau^2
 * with c = Gamma_t x. */
static void newton_grain(const geom_t* G, const double* omega, const int* I_off, const double* p,
                         const int* js, int nj, const int* jt, const double* rE,
                         qfun_t qf, void* qc, int n_newton, double tol_x, double hreg,
                         double x[3], double* stats) {
    int k;
    double last = 0.0;
    stats[6] = newton_objective(G, omega, I_off, p, js, nj, jt, rE, qf, qc, x);
    for (k = 0; k < n_newton; ++k) {
        double gx[3] = {0, 0, 0}, Hx[9] = {0};
        for (int q = 0; q < nj; ++q) {
            int j = js[q], t = jt[q];
            double Gam[9], c[3];
            orc_gamma(omega[t], Gam);
            mat_vec(Gam, x, c);
            const double* r = rE + 3 * j;
            double gc[3] = {0, 0, 0}, Hc[9] = {0};
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                double Q = qf(qc, i, j);
                if (Q == 0.0) continue;
                double d[3] = {p[3 * i] - c[0], p[3 * i + 1] - c[1], p[3 * i + 2] - c[2]};
                double tau = sqrt(dot3(d, d));
                double rh[3] = {d[0] / tau, d[1] / tau, d[2] / tau};
                double rr = dot3(rh, r);
                for (int a = 0; a < 3; ++a) gc[a] += -Q * (r[a] - rr * rh[a]) / tau;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) {
                        double h = 3.0 * rr * rh[a] * rh[b] - rh[a] * r[b] - r[a] * rh[b] -
                                   (a == b ? rr : 0.0);
                        Hc[3 * a + b] += Q * h / (tau * tau);
                    }
            }
            /* back to x: g_x = Gamma^T g_c, H_x = Gamma^T H_c Gamma */
            double tmp[3], HG[9], GtHG[9], GamT[9];
            matT_vec(Gam, gc, tmp);
            for (int a = 0; a < 3; ++a) gx[a] += tmp[a];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) GamT[3 * a + b] = Gam[3 * b + a];
            mat_mul(Hc, Gam, HG);
            mat_mul(GamT, HG, GtHG);
            for (int a = 0; a < 9; ++a) Hx[a] += GtHG[a];
        }
        double fro = 0.0;
        for (int a = 0; a < 9; ++a) fro += Hx[a] * Hx[a];
        fro = sqrt(fro);
        if (!(fro > 0.0)) break;
        double ev[3], evec[9];
        orc_sym3_eig(Hx, ev, evec);
        double iota = ev[2] + hreg * fro;
        if (iota < 0.0) iota = 0.0;
        double A[9];
        memcpy(A, Hx, sizeof(A));
        A[0] -= iota; A[4] -= iota; A[8] -= iota;
        double dx[3];
        if (!solve3(A, gx, dx)) break;
        for (int a = 0; a < 3; ++a) x[a] -= dx[a];
        last = sqrt(dot3(dx, dx));
        if (last < tol_x) { ++k; break; }
    }
    stats[0] = k;
    stats[2] = last;
    stats[7] = newton_objective(G, omega, I_off, p, js, nj, jt, rE, qf, qc, x);
}

/* sum_m w_m^T R^T M0_m R w_m over the planes touched by the grain */
static double mm_objective(const double* M0, const int* planes, int np, const double* w,
                           const double R[9]) {
    double s = 0.0;
    for (int k = 0; k < np; ++k) {
        double Rw[3], MRw[3];
        mat_vec(R, w + 3 * planes[k], Rw);
        mat_vec(M0 + 9 * k, Rw, MRw);
        s += dot3(Rw, MRw);
    }
    return s;
}

/* Appendix "M-steps", grain rotation (Eqs. M0, Mm, majmin_step; Algorithm
 * LaueRotMM):  M0_m = -sum_{j in J_n & J_m} Gamma^T (v_j e^T + e v_j^T) Gamma
 * with v_j = sum_i Q_ij rhat_ij at the current position, M_m = M0_m + iota_m I,
 * then R^{k+1} = Wahba(M_m R^k w_m, w_m, 1). */
static void mm_grain(const geom_t* G, const double* omega, const int* I_off, const double* p,
                     const double* w, const int* js, int nj, const int* jt, const int* jm,
                     qfun_t qf, void* qc, int n_mm, double tol_R, const double x[3],
                     double R[9], double* stats) {
    int* planes = (int*)malloc(sizeof(int) * (nj + 1));
    double* M0 = (double*)calloc((size_t)9 * (nj + 1), sizeof(double));
    int np = 0;
    for (int q = 0; q < nj; ++q) {
        int j = js[q], t = jt[q], m = jm[q];
        double Gam[9], c[3];
        orc_gamma(omega[t], Gam);
        mat_vec(Gam, x, c);
        double vj[3] = {0, 0, 0};
        for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
            double Q = qf(qc, i, j);
            if (Q == 0.0) continue;
            double d[3] = {p[3 * i] - c[0], p[3 * i + 1] - c[1], p[3 * i + 2] - c[2]};
            double tau = sqrt(dot3(d, d));
            for (int a = 0; a < 3; ++a) vj[a] += Q * d[a] / tau;
        }
        int slot = -1;
        for (int k = 0; k < np; ++k)
            if (planes[k] == m) { slot = k; break; }
        if (slot < 0) { slot = np; planes[np++] = m; }
        double A[9], GamT[9], AG[9], GtAG[9];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                A[3 * a + b] = vj[a] * G->e[b] + G->e[a] * vj[b];
                GamT[3 * a + b] = Gam[3 * b + a];
            }
        mat_mul(A, Gam, AG);
        mat_mul(GamT, AG, GtAG);
        for (int a = 0; a < 9; ++a) M0[9 * slot + a] -= GtAG[a];
    }
    double* Mm = (double*)malloc(sizeof(double) * 9 * (np + 1));
    for (int k = 0; k < np; ++k) {
        double ev[3], evec[9];
        orc_sym3_eig(M0 + 9 * k, ev, evec);
        double iota = ev[0] < 0.0 ? -ev[0] : 0.0;
        for (int a = 0; a < 9; ++a) Mm[9 * k + a] = M0[9 * k + a];
        Mm[9 * k + 0] += iota; Mm[9 * k + 4] += iota; Mm[9 * k + 8] += iota;
    }
    stats[4] = mm_objective(M0, planes, np, w, R);
    int it;
    double last = 0.0;
    for (it = 0; it < n_mm; ++it) {
        double B[9] = {0};
        for (int k = 0; k < np; ++k) {
            const double* wm = w + 3 * planes[k];
            double Rw[3], a[3];
            mat_vec(R, wm, Rw);
            mat_vec(Mm + 9 * k, Rw, a);
            for (int u = 0; u < 3; ++u)
                for (int b = 0; b < 3; ++b) B[3 * u + b] += a[u] * wm[b];
        }
        double Rn[9];
        if (!orc_wahba(B, Rn)) break;
        double dr = 0.0;
        for (int a = 0; a < 9; ++a) dr += (Rn[a] - R[a]) * (Rn[a] - R[a]);
        last = sqrt(dr);
        memcpy(R, Rn, sizeof(Rn));
        if (last < tol_R) { ++it; break; }
    }
    stats[1] = it;
    stats[3] = last;
    stats[5] = mm_objective(M0, planes, np, w, R);
    free(planes); free(M0); free(Mm);
}

typedef struct { int* js; int* jt; int* jm; int n; } grain_list;

static void build_grain_lists(int T, const int* J_off, const int* grain, const int* plane, int N,
                              grain_list* L) {
    for (int n = 0; n < N; ++n) L[n].n = 0;
    int nJ = J_off[T];
    for (int j = 0; j < nJ; ++j) L[grain[j]].n++;
    for (int n = 0; n < N; ++n) {
        L[n].js = (int*)malloc(sizeof(int) * (L[n].n + 1));
        L[n].jt = (int*)malloc(sizeof(int) * (L[n].n + 1));
        L[n].jm = (int*)malloc(sizeof(int) * (L[n].n + 1));
        L[n].n = 0;
    }
    for (int t = 0; t < T; ++t)
        for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
            grain_list* g = &L[grain[j]];
            g->js[g->n] = j;
            g->jt[g->n] = t;
            g->jm[g->n] = plane[j];
            g->n++;
        }
}

static void free_grain_lists(grain_list* L, int N) {
    for (int n = 0; n < N; ++n) { free(L[n].js); free(L[n].jt); free(L[n].jm); }
}

/* Section "The M-step updates": per grain, Newton on x_n (with R^k), then MM
 * on R_n (with x^{k+1}); Q stays the E-step plan.  stats[8 n + .] =
 * {newton steps, mm steps, last |dx|, last |dR|_F, MM objective before,
 *  MM objective after, Phi before Newton, Phi after Newton}. */
int orc_mstep(const double* geom, const double* w, const double* omega, int T,
              const int* I_off, const double* p, const int* J_off,
              const int* grain, const int* plane, const int* det, int N,
              const double* cE, const double* rE,
              const double* f, const double* g, double eps,
              int n_newton, int n_mm, double tol_x, double tol_R, double hreg,
              double* R, double* x, double* stats) {
    geom_t G;
    geom_unpack(geom, &G);
    qpot_ctx qc = {p, cE, rE, f, g, eps, &G, det};
    grain_list* L = (grain_list*)malloc(sizeof(grain_list) * (N + 1));
    build_grain_lists(T, J_off, grain, plane, N, L);
    double st[8];
    for (int n = 0; n < N; ++n) {
        memset(st, 0, sizeof(st));
        newton_grain(&G, omega, I_off, p, L[n].js, L[n].n, L[n].jt, rE, q_from_potentials, &qc,
                     n_newton, tol_x, hreg, x + 3 * n, st);
        mm_grain(&G, omega, I_off, p, w, L[n].js, L[n].n, L[n].jt, L[n].jm, q_from_potentials,
                 &qc, n_mm, tol_R, x + 3 * n, R + 9 * n, st);
        if (stats) memcpy(stats + 8 * n, st, sizeof(st));
    }
    free_grain_lists(L, N);
    free(L);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* EM driver with deterministic annealing                                      */
/* ------------------------------------------------------------------------- */

/* Section "Deterministic annealing": eps_init = 100 eps_final, geometric
 * cooling that reaches eps_final at step ceil(0.75 n_em), then held. */
double orc_eps_schedule_f(double eps_final, int n_em, int k, double factor) {
    int K = (int)ceil(0.75 * n_em);
    if (K < 1 || k >= K) return eps_final;
    return eps_final * pow(factor, 1.0 - (double)k / (double)K);
}

double orc_eps_schedule(double eps_final, int n_em, int k) {
    return orc_eps_schedule_f(eps_final, n_em, k, 100.0);
}

/* Algorithm LaueOT (multi-grain fitting) with a fixed number of EM steps:
 * refresh rays -> BalancedOT -> LauePosNewton -> LaueRotMM -> cool.  A final
 * E-step at the last poses gives the plan read-out. */
int orc_em(const double* geom, const double* w, const double* d0, const int* nharm,
           const double* omega, int T, const int* I_off, const double* p,
           const int* J_off, const int* grain, const int* plane, const int* det, int N,
           double* R, double* x, double eps_final, int n_em, int n_sinkhorn,
           double c_out, int mode, double frac, int n_newton, int n_mm,
           double tol_x, double tol_R, double hreg, int mstep_kind,
           double* f, double* g, double* fd, double* gd, int* assign, double* margin) {
    geom_t G;
    geom_unpack(geom, &G);
    int nJ = J_off[T];
    double* ray4 = (double*)malloc(sizeof(double) * 4 * (nJ + 1));
    double* c3 = (double*)malloc(sizeof(double) * 3 * (nJ + 1));
    double* r3 = (double*)malloc(sizeof(double) * 3 * (nJ + 1));
    double* Dj = (double*)malloc(sizeof(double) * (nJ + 1));
    for (int j = 0; j < nJ; ++j) Dj[j] = det_D(&G, det, j);
    for (int k = 0; k <= n_em; ++k) {
        double eps = orc_eps_schedule(eps_final, n_em, k < n_em ? k : n_em);
        orc_refresh(geom, w, d0, nharm, R, x, omega, T, J_off, grain, plane, ray4, c3);
        for (int j = 0; j < nJ; ++j)
            for (int a = 0; a < 3; ++a) r3[3 * j + a] = ray4[4 * j + a];
        orc_sinkhorn(Dj, T, I_off, p, J_off, c3, r3, eps, c_out, mode, frac, n_sinkhorn, 0.0, 0,
                     f, g, fd, gd);
        if (k == n_em) {
            orc_harvest(Dj, T, I_off, p, J_off, c3, r3, eps, c_out, mode, frac, f, g, fd, gd,
                        assign, margin, NULL, NULL, NULL);
            break;
        }
        if (mstep_kind == 1)  /* the adjoint M-step; hreg is its damping */
            orc_mstep_adjoint(geom, w, omega, T, I_off, p, J_off, grain, plane, det, N, c3, r3, f, g, eps,
                              n_newton, hreg, R, x, NULL);
        else
            orc_mstep(geom, w, omega, T, I_off, p, J_off, grain, plane, det, N, c3, r3, f, g, eps,
                      n_newton, n_mm, tol_x, tol_R, hreg, R, x, NULL);
    }
    free(ray4); free(c3); free(r3); free(Dj);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Single-grain fitting (Algorithm SingleLaueOT)                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    const double* Q;      /* dense rows: Q[k * nIt_max + (i - I_off[t])] */
    const int* jpos;      /* global model index -> row k */
    const int* I_off;
    const int* jt;
    int stride;
    const double* wk;     /* (D_k / D)^2 of each ray */
} qdense_ctx;

/* M-step weight of pair (i, j) in a single-grain fit: Q_ij (D_j / D)^2, as
 * in q_from_potentials. */
static double q_dense(void* vctx, int i, int j) {
    qdense_ctx* c = (qdense_ctx*)vctx;
    int k = c->jpos[j];
    int t = c->jt[k];
    return c->Q[(long)k * c->stride + (i - c->I_off[t])] * c->wk[k];
}

/* Appendix "Single-grain fitting" (Eq. elbo_single): row-normalised E-step
 * Q_ij = K_ij / (sum_{j'} K_ij' + K_i0), K = exp(-C/eps), over the model spots
 * of the grain at angle t_i. */
static void single_estep(const double* Dk, const int* I_off, const double* p, int nj, const int* jt,
                         const double* c3, const double* r3, double eps, double c_out,
                         int stride, double* Q, int T) {
    double* buf = (double*)malloc(sizeof(double) * (nj + 2));
    for (int t = 0; t < T; ++t) {
        for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
            int n = 0;
            for (int k = 0; k < nj; ++k)
                if (jt[k] == t) buf[n++] = -orc_pair_cost(p + 3 * i, c3 + 3 * k, r3 + 3 * k, Dk[k]) / eps;
            buf[n++] = -c_out / eps;
            double l = lse(buf, n);
            for (int k = 0; k < nj; ++k)
                if (jt[k] == t)
                    Q[(long)k * stride + (i - I_off[t])] =
                        exp(-orc_pair_cost(p + 3 * i, c3 + 3 * k, r3 + 3 * k, Dk[k]) / eps - l);
        }
    }
    free(buf);
}

/* Algorithm SingleLaueOT for S starts.  The model-spot list of a start is
 * frozen at its starting pose (as for prototypes); k_max annealed EM steps
 * with the row-normalised E-step, n_newton Newton and n_mm MM steps each.
 * The candidate filter (Section "Selection of Prototypes", f_out) uses the
 * spots visible at the final pose: a model ray is unmatched when its column
 * mass q_j < 0.5 at eps_final; keep[s] = (#unmatched < f_out |J|). */
int orc_single_fit(const double* geom, const double* w, const double* d0, const int* nharm, int M,
                   const double* omega, int T, const int* I_off, const double* p,
                   int S, const double* R0, const double* x0,
                   double eps_final, int k_max, double c_out,
                   int n_newton, int n_mm, double tol_x, double tol_R, double hreg,
                   double f_out, double anneal, int recut,
                   double* R_out, double* x_out, int* keep, double* unmatched) {
    geom_t G;
    geom_unpack(geom, &G);
    int stride = 1;
    for (int t = 0; t < T; ++t)
        if (I_off[t + 1] - I_off[t] > stride) stride = I_off[t + 1] - I_off[t];
    long cap = (long)M * T;
    int* Joff = (int*)malloc(sizeof(int) * (T + 1));
    int* gr = (int*)malloc(sizeof(int) * cap);
    int* pl = (int*)malloc(sizeof(int) * cap);
    int* dk = (int*)malloc(sizeof(int) * cap);
    double* ray4 = (double*)malloc(sizeof(double) * 4 * cap);
    double* s3 = (double*)malloc(sizeof(double) * 3 * cap);
    double* c3 = (double*)malloc(sizeof(double) * 3 * cap);
    double* r3 = (double*)malloc(sizeof(double) * 3 * cap);
    int* jt = (int*)malloc(sizeof(int) * cap);
    int* jpos = (int*)malloc(sizeof(int) * cap);
    int* js = (int*)malloc(sizeof(int) * cap);
    double* Q = (double*)malloc(sizeof(double) * cap * stride);
    double* Dk = (double*)malloc(sizeof(double) * cap);
    double* wk = (double*)malloc(sizeof(double) * cap);
    for (int s = 0; s < S; ++s) {
        double R[9], x[3];
        memcpy(R, R0 + 9 * s, sizeof(R));
        memcpy(x, x0 + 3 * s, sizeof(x));
        long nj = 0;
        qdense_ctx qc = {Q, jpos, I_off, jt, stride, wk};
        for (int k = 0; k < k_max; ++k) {
            double eps = orc_eps_schedule_f(eps_final, k_max, k, anneal);
            /* Algorithm SingleLaueOT computes the model rays of the grain at
             * every iteration: with recut the visible set is listed again at
             * the pose of step k, otherwise it stays the one of the start */
            if (k == 0 || recut) {
                nj = orc_forward(geom, w, d0, nharm, M, R, x, 1, omega, T, cap, Joff, gr, pl, ray4,
                                 s3, dk, c3, NULL, NULL);
                for (int t = 0; t < T; ++t)
                    for (int j = Joff[t]; j < Joff[t + 1]; ++j) { jt[j] = t; jpos[j] = j; js[j] = j; }
                for (long j = 0; j < nj; ++j) {
                    Dk[j] = det_D(&G, dk, j);
                    wk[j] = (Dk[j] / G.D) * (Dk[j] / G.D);
                }
            }
            orc_refresh(geom, w, d0, nharm, R, x, omega, T, Joff, gr, pl, ray4, c3);
            for (long j = 0; j < nj; ++j)
                for (int a = 0; a < 3; ++a) r3[3 * j + a] = ray4[4 * j + a];
            single_estep(Dk, I_off, p, (int)nj, jt, c3, r3, eps, c_out, stride, Q, T);
            double st[8];
            newton_grain(&G, omega, I_off, p, js, (int)nj, jt, r3, q_dense, &qc, n_newton, tol_x,
                         hreg, x, st);
            mm_grain(&G, omega, I_off, p, w, js, (int)nj, jt, pl, q_dense, &qc, n_mm, tol_R, x, R,
                     st);
        }
        memcpy(R_out + 9 * s, R, sizeof(R));
        memcpy(x_out + 3 * s, x, sizeof(x));
        /* candidate filter at the final pose */
        long nf = orc_forward(geom, w, d0, nharm, M, R, x, 1, omega, T, cap, Joff, gr, pl, ray4,
                              s3, dk, c3, NULL, NULL);
        for (int t = 0; t < T; ++t)
            for (int j = Joff[t]; j < Joff[t + 1]; ++j) jt[j] = t;
        for (long j = 0; j < nf; ++j) {
            for (int a = 0; a < 3; ++a) r3[3 * j + a] = ray4[4 * j + a];
            Dk[j] = det_D(&G, dk, j);
        }
        single_estep(Dk, I_off, p, (int)nf, jt, c3, r3, eps_final, c_out, stride, Q, T);
        int nun = 0;
        for (long j = 0; j < nf; ++j) {
            int t = jt[j];
            double qj = 0.0;
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) qj += Q[j * stride + (i - I_off[t])];
            if (qj < 0.5) ++nun;
        }
        if (unmatched) unmatched[s] = nf > 0 ? (double)nun / (double)nf : 1.0;
        if (keep) keep[s] = nf > 0 && (double)nun < f_out * (double)nf;
    }
    free(Joff); free(gr); free(pl); free(dk); free(ray4); free(s3); free(c3); free(r3);
    free(jt); free(jpos); free(js); free(Q); free(Dk); free(wk);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* SPOT prototype selection                                                    */
/* ------------------------------------------------------------------------- */

/* Appendix "Selection of prototypes": grain-to-spot matrix, read as the gain
 * over the outlier baseline
 *   Lbar_in = max(0, LSE_{j in J_n, t_j = t_i}(-C_ij/eps_s) + c_out/eps_s),
 * dense I x Nc (row-major), from the spots each candidate makes at its pose. */
int orc_spot_matrix(const double* geom, const double* w, const double* d0, const int* nharm, int M,
                    const double* omega, int T, const int* I_off, const double* p,
                    int Nc, const double* R, const double* x, double eps_s, double c_out,
                    double* Lbar) {
    geom_t G;
    geom_unpack(geom, &G);
    int nI = I_off[T];
    long cap = (long)M * T;
    int* Joff = (int*)malloc(sizeof(int) * (T + 1));
    int* gr = (int*)malloc(sizeof(int) * cap);
    int* pl = (int*)malloc(sizeof(int) * cap);
    int* dk = (int*)malloc(sizeof(int) * cap);
    double* ray4 = (double*)malloc(sizeof(double) * 4 * cap);
    double* s3 = (double*)malloc(sizeof(double) * 3 * cap);
    double* c3 = (double*)malloc(sizeof(double) * 3 * cap);
    double* buf = (double*)malloc(sizeof(double) * (cap + 1));
    for (int n = 0; n < Nc; ++n) {
        orc_forward(geom, w, d0, nharm, M, R + 9 * n, x + 3 * n, 1, omega, T, cap, Joff, gr, pl,
                    ray4, s3, dk, c3, NULL, NULL);
        for (int t = 0; t < T; ++t)
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                int k = 0;
                for (int j = Joff[t]; j < Joff[t + 1]; ++j) {
                    double r[3] = {ray4[4 * j], ray4[4 * j + 1], ray4[4 * j + 2]};
                    buf[k++] = -orc_pair_cost(p + 3 * i, c3 + 3 * j, r, det_D(&G, dk, j)) / eps_s;
                }
                double val = k ? lse(buf, k) + c_out / eps_s : 0.0;
                Lbar[(long)i * Nc + n] = val > 0.0 ? val : 0.0;
            }
    }
    (void)nI;
    free(Joff); free(gr); free(pl); free(dk); free(ray4); free(s3); free(c3); free(buf);
    return 0;
}

/* f(S) = sum_i max_{n in S} Lbar_in  (closed form of Eq. prototype_function
 * when the source weights are free on S), f(empty) = 0. */
static double spot_value(int I, int Nc, const double* Lbar, const int* S, int k) {
    double tot = 0.0;
    for (int i = 0; i < I; ++i) {
        double best = 0.0;
        for (int q = 0; q < k; ++q) {
            double v = Lbar[(long)i * Nc + S[q]];
            if (v > best) best = v;
        }
        tot += best;
    }
    return tot;
}

/* Algorithm LaueSpotGreedy by the naive definition: at every step recompute
 * f(S u {n}) - f(S) for every candidate not yet chosen; ties go to the lowest
 * index.  gain[k] = increment of step k+1, F[k] = cumulative value. */
int orc_spot_greedy(int I, int Nc, const double* Lbar, int kmax,
                    int* order, double* gain, double* F) {
    int* S = (int*)malloc(sizeof(int) * (kmax + 1));
    char* used = (char*)calloc((size_t)Nc + 1, 1);
    double fS = 0.0;
    int k;
    for (k = 0; k < kmax && k < Nc; ++k) {
        int best = -1;
        double bestg = -1.0;
        for (int n = 0; n < Nc; ++n) {
            if (used[n]) continue;
            S[k] = n;
            double gn = spot_value(I, Nc, Lbar, S, k + 1) - fS;
            if (gn > bestg) { bestg = gn; best = n; }
        }
        S[k] = best;
        used[best] = 1;
        fS += bestg;
        order[k] = best;
        gain[k] = bestg;
        F[k] = fS;
    }
    free(S);
    free(used);
    return k;
}

/* Eq. spot_ngrains read on the increments Delta_k (gain[k-1]): the largest
 * drop, k* = argmax_{2 <= k <= K} Delta_k - Delta_{k+1} with Delta_{K+1} = 0;
 * k* = K when K < 2.  Ties go to the smallest k. */
int orc_kstar(int K, const double* gain) {
    if (K < 2) return K;
    int best = 2;
    double bv = -INFINITY;
    for (int k = 2; k <= K; ++k) {
        double dk = gain[k - 1];
        double dk1 = k < K ? gain[k] : 0.0;
        if (dk - dk1 > bv) { bv = dk - dk1; best = k; }
    }
    return best;
}

/* ------------------------------------------------------------------------- */
/* Adjoint: gradient of the OT-weighted spot cost                              */
/* ------------------------------------------------------------------------- */

/* E_n(R, x) = sum_{j in J_n} sum_{i in I_tj} Q_ij C_ij(R, x) with Q_ij fixed by
 * the potentials and the costs at the E-step (cE, rE). */
void orc_grain_objective(const double* geom, const double* w, const double* omega, int T,
                         const int* I_off, const double* p, const int* J_off,
                         const int* grain, const int* plane, const int* det, int N,
                         const double* cE, const double* rE,
                         const double* f, const double* g, double eps,
                         const double* R, const double* x, double* En) {
    geom_t G;
    geom_unpack(geom, &G);
    for (int n = 0; n < N; ++n) En[n] = 0.0;
    for (int t = 0; t < T; ++t) {
        double Gam[9];
        orc_gamma(omega[t], Gam);
        for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
            int n = grain[j], m = plane[j];
            double v[3], u[3], c[3], r[3];
            mat_vec(R + 9 * n, w + 3 * m, v);
            mat_vec(Gam, v, u);
            mat_vec(Gam, x + 3 * n, c);
            double ue = dot3(u, G.e);
            for (int a = 0; a < 3; ++a) r[a] = G.e[a] - 2.0 * ue * u[a];
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                double Dj = det_D(&G, det, j);
                double CE = orc_pair_cost(p + 3 * i, cE + 3 * j, rE + 3 * j, Dj);
                double Q = exp((f[i] + g[j] - CE) / eps);
                En[n] += Q * orc_pair_cost(p + 3 * i, c, r, Dj);
            }
        }
    }
}

/* Analytic gradient of E_n at the E-step poses (Danskin: Q held fixed) with
 * respect to a left-multiplicative axis-angle perturbation R <- exp([w]x) R
 * and to x:
 *   dC/dc     = (2 D^2 / tau) (r - (rhat.r) rhat),   c = Gamma x
 *   dC/dr     = 2 D^2 (r - rhat)
 *   dr/du     = -2 (u e^T + (u.e) I),  du/dw = -Gamma [R w_m]x
 * grad[6 n + 0..2] = dE_n/dw, grad[6 n + 3..5] = dE_n/dx. */
void orc_grain_grad(const double* geom, const double* w, const double* omega, int T,
                    const int* I_off, const double* p, const int* J_off,
                    const int* grain, const int* plane, const int* det, int N,
                    const double* f, const double* g, double eps,
                    const double* R, const double* x, double* grad) {
    geom_t G;
    geom_unpack(geom, &G);
    for (int k = 0; k < 6 * N; ++k) grad[k] = 0.0;
    for (int t = 0; t < T; ++t) {
        double Gam[9];
        orc_gamma(omega[t], Gam);
        for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
            int n = grain[j], m = plane[j];
            double Dj = det_D(&G, det, j), D2 = Dj * Dj;
            double v[3], u[3], c[3], r[3];
            mat_vec(R + 9 * n, w + 3 * m, v);
            mat_vec(Gam, v, u);
            mat_vec(Gam, x + 3 * n, c);
            double ue = dot3(u, G.e);
            for (int a = 0; a < 3; ++a) r[a] = G.e[a] - 2.0 * ue * u[a];
            double gr[3] = {0, 0, 0}, gc[3] = {0, 0, 0};
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                double C = orc_pair_cost(p + 3 * i, c, r, Dj);
                double Q = exp((f[i] + g[j] - C) / eps);
                if (Q == 0.0) continue;
                double d[3] = {p[3 * i] - c[0], p[3 * i + 1] - c[1], p[3 * i + 2] - c[2]};
                double tau = sqrt(dot3(d, d));
                double rh[3] = {d[0] / tau, d[1] / tau, d[2] / tau};
                double rr = dot3(rh, r);
                for (int a = 0; a < 3; ++a) {
                    gc[a] += Q * 2.0 * D2 / tau * (r[a] - rr * rh[a]);
                    gr[a] += Q * 2.0 * D2 * (r[a] - rh[a]);
                }
            }
            /* x part: Gamma^T dC/dc */
            double gx[3];
            matT_vec(Gam, gc, gx);
            /* rotation part: y^T = (dC/dr)^T dr/du = -2 ((gr.u) e + (u.e) gr)^T and
             * dE/dw = y^T (-Gamma [v]x) = v x (Gamma^T y) */
            double y[3];
            double gu = dot3(gr, u);
            for (int a = 0; a < 3; ++a) y[a] = -2.0 * (gu * G.e[a] + ue * gr[a]);
            double Gty[3], gw[3];
            matT_vec(Gam, y, Gty);
            cross3(v, Gty, gw);
            for (int a = 0; a < 3; ++a) {
                grad[6 * n + a] += gw[a];
                grad[6 * n + 3 + a] += gx[a];
            }
        }
    }
}

/* ------------------------------------------------------------------------- */
/* Start grid of the single-grain fits                                         */
/* ------------------------------------------------------------------------- */

/* The 24 rotations of the cubic point group as unit quaternions (w, x, y, z):
 * the identity, 90-degree turns about the cube axes (6), 180-degree turns
 * about the cube axes (3) and the face diagonals (6), 120-degree turns about
 * the body diagonals (8). */
static void cubic_group(double g[24][4]) {
    int k = 0;
    const double s = sqrt(0.5);
    g[k][0] = 1.0; g[k][1] = g[k][2] = g[k][3] = 0.0; ++k;
    for (int a = 1; a <= 3; ++a) {
        for (int sg = -1; sg <= 1; sg += 2) {
            g[k][0] = s; g[k][1] = g[k][2] = g[k][3] = 0.0; g[k][a] = sg * s; ++k;
        }
        g[k][0] = g[k][1] = g[k][2] = g[k][3] = 0.0; g[k][a] = 1.0; ++k;
    }
    for (int a = 1; a <= 3; ++a)
        for (int b = a + 1; b <= 3; ++b)
            for (int sg = -1; sg <= 1; sg += 2) {
                g[k][0] = g[k][1] = g[k][2] = g[k][3] = 0.0; g[k][a] = s; g[k][b] = sg * s; ++k;
            }
    for (int m = 0; m < 8; ++m) {
        g[k][0] = 0.5;
        g[k][1] = (m & 1) ? -0.5 : 0.5;
        g[k][2] = (m & 2) ? -0.5 : 0.5;
        g[k][3] = (m & 4) ? -0.5 : 0.5;
        ++k;
    }
}

/* Section "Single-grain fitting" starts the fits from a quasi-uniform grid over
 * orientations and positions, restricted by the lattice symmetry (sym: 1 none,
 * 24 cubic group 432, 6 trigonal 32, 12 hexagonal 622).  Reading
 * (the paper uses a Sobol sequence over modified Rodrigues parameters): the
 * super-Fibonacci spiral of Alexa (CVPR 2022) gives n_full quasi-uniform unit
 * quaternions q_i, i = 0..n_full-1, with s = i + 1/2,
 *   q = (sqrt(s/n) sin(2 pi s/phi), sqrt(s/n) cos(2 pi s/phi),
 *        sqrt(1-s/n) sin(2 pi s/psi), sqrt(1-s/n) cos(2 pi s/psi)),
 * phi = sqrt 2 and psi the real root of psi^4 = psi + 4.  With sym = 24 only
 * the q whose scalar part is the largest |<q, g>| over the cubic group (q
 * itself is the member of its symmetry class nearest the identity: the
 * fundamental zone) are kept, in order.  Each kept orientation is paired with
 * the k^3 cell centres of the cube of side `cube` centred at the origin
 * ((a + 1/2) cube/k - cube/2 per axis, x slowest).  Writes at most cap starts
 * (R row-major 3x3, x) and returns the number of starts. */
/* The rotations of the trigonal group 32 (D3: order 6) and the hexagonal group
 * 622 (D6: order 12) with the c axis along z and a 2-fold axis along x (the
 * hexagonal a1 axis): turns about z by multiples of 360/n degrees, and
 * 180-degree turns about the axes in the xy plane at multiples of 180/n
 * degrees (n = 3 or 6), as unit quaternions. */
static int dihedral_group(int n, double g[24][4]) {
    int k = 0;
    const double pi = 3.14159265358979323846;
    for (int q = 0; q < n; ++q) {
        double h = pi * q / n;  /* half of the turn 2 pi q / n */
        g[k][0] = cos(h); g[k][1] = 0.0; g[k][2] = 0.0; g[k][3] = sin(h); ++k;
    }
    for (int q = 0; q < n; ++q) {
        double phi = pi * q / n;
        g[k][0] = 0.0; g[k][1] = cos(phi); g[k][2] = sin(phi); g[k][3] = 0.0; ++k;
    }
    return k;
}

long orc_start_grid(long n_full, int sym, int k, double cube, long cap, double* R_out, double* x_out) {
    double G[24][4];
    int ng = 24;
    if (sym == 6) ng = dihedral_group(3, G);
    else if (sym == 12) ng = dihedral_group(6, G);
    else cubic_group(G);
    const double phi = sqrt(2.0), psi = 1.533751168755204288118041;
    const double two_pi = 6.283185307179586476925287;
    long n_kept = 0, S = 0;
    long kk = (long)k * k * k;
    for (long i = 0; i < n_full; ++i) {
        double s = (double)i + 0.5;
        double r = sqrt(s / (double)n_full), rr = sqrt(1.0 - s / (double)n_full);
        double q[4] = {r * sin(two_pi * s / phi), r * cos(two_pi * s / phi), rr * sin(two_pi * s / psi),
                       rr * cos(two_pi * s / psi)};
        if (sym == 24 || sym == 6 || sym == 12) {
            double id = fabs(q[0]);
            int inside = 1;
            for (int g = 1; g < ng; ++g) {
                double d = fabs(q[0] * G[g][0] + q[1] * G[g][1] + q[2] * G[g][2] + q[3] * G[g][3]);
                if (d > id) { inside = 0; break; }
            }
            if (!inside) continue;
        }
        ++n_kept;
        double w = q[0], x = q[1], y = q[2], z = q[3];
        double R[9] = {1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y),
                       2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x),
                       2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)};
        for (long p = 0; p < kk; ++p, ++S) {
            if (S >= cap) continue;
            long a = p / ((long)k * k), b = (p / k) % k, c = p % k;
            for (int e = 0; e < 9; ++e) R_out[9 * S + e] = R[e];
            x_out[3 * S + 0] = (a + 0.5) * cube / k - cube / 2;
            x_out[3 * S + 1] = (b + 0.5) * cube / k - cube / 2;
            x_out[3 * S + 2] = (c + 0.5) * cube / k - cube / 2;
        }
    }
    (void)n_kept;
    return S;
}

/* ------------------------------------------------------------------------- */
/* Adjoint M-step: damped Gauss-Newton on the OT-weighted spot cost            */
/* ------------------------------------------------------------------------- */

/* Exact gradient and Gauss-Newton matrix of E_n = sum_{j in J_n} sum_i Q_ij
 * C_ij(R, x) at the current pose, Q held at the E-step plan (potentials f, g,
 * costs of the E-step geometry cE, rE), for the perturbation theta = (phi, x),
 * R <- exp([phi]x) R.  With e_ij = rhat_ij - r_j and C = D^2 |e|^2:
 *   dE/dtheta = sum Q 2 D^2 e^T J_ij,  J_ij = [-A_j, -P_ij Gamma / tau_ij],
 *   A_j = dr_j/dphi = 2 (u e^T + (u.e) I) Gamma [v]x,  v = R w_m, u = Gamma v,
 *   P_ij = I - rhat rhat^T,  tau_ij = |p_i - c_j|.
 * The Gauss-Newton matrix 2 D^2 sum Q J^T J is taken with P_ij replaced by
 * the model ray's projector I - r_j r_j^T (exact where rhat = r):
 *   H_phiphi = 2 D^2 q_j A^T A,  H_phix = 2 D^2 s1_j A^T P_j Gamma,
 *   H_xx = 2 D^2 s2_j Gamma^T P_j Gamma,
 * q_j = sum_i Q_ij, s1_j = sum_i Q_ij / tau_ij, s2_j = sum_i Q_ij / tau_ij^2.
 * grad: N x 6, H: N x 36 (row-major), value: N (optional). */
void orc_grain_gn(const double* geom, const double* w, const double* omega, int T,
                  const int* I_off, const double* p, const int* J_off,
                  const int* grain, const int* plane, const int* det, int N,
                  const double* cE, const double* rE, const double* f, const double* g, double eps,
                  const double* R, const double* x, double* grad, double* H, double* value) {
    geom_t G;
    geom_unpack(geom, &G);
    for (int k = 0; k < 6 * N; ++k) grad[k] = 0.0;
    for (int k = 0; k < 36 * N; ++k) H[k] = 0.0;
    if (value) for (int n = 0; n < N; ++n) value[n] = 0.0;
    for (int t = 0; t < T; ++t) {
        double Gam[9];
        orc_gamma(omega[t], Gam);
        for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
            int n = grain[j], m = plane[j];
            double Dj = det_D(&G, det, j), D2 = Dj * Dj;
            double v[3], u[3], c[3], r[3];
            mat_vec(R + 9 * n, w + 3 * m, v);
            mat_vec(Gam, v, u);
            mat_vec(Gam, x + 3 * n, c);
            double ue = dot3(u, G.e);
            for (int a = 0; a < 3; ++a) r[a] = G.e[a] - 2.0 * ue * u[a];
            /* A = 2 (u e^T + (u.e) I) Gamma [v]x */
            double B[9], Vx[9] = {0, -v[2], v[1], v[2], 0, -v[0], -v[1], v[0], 0}, GV[9], A[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) B[3 * a + b] = 2.0 * (u[a] * G.e[b] + (a == b ? ue : 0.0));
            mat_mul(Gam, Vx, GV);
            mat_mul(B, GV, A);
            double gc[3] = {0, 0, 0}, ge[3] = {0, 0, 0}, q = 0.0, s1 = 0.0, s2 = 0.0, val = 0.0;
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                double CE = orc_pair_cost(p + 3 * i, cE + 3 * j, rE + 3 * j, Dj);
                double Q = exp((f[i] + g[j] - CE) / eps);
                if (Q == 0.0) continue;
                double d[3] = {p[3 * i] - c[0], p[3 * i + 1] - c[1], p[3 * i + 2] - c[2]};
                double tau = sqrt(dot3(d, d));
                double rh[3] = {d[0] / tau, d[1] / tau, d[2] / tau};
                double e[3] = {rh[0] - r[0], rh[1] - r[1], rh[2] - r[2]};
                double ee = dot3(e, rh);
                /* dC/dx = 2 D^2 e^T (-P Gamma / tau): accumulate -P e / tau in the lab frame */
                for (int a = 0; a < 3; ++a) {
                    gc[a] += Q * (-(e[a] - ee * rh[a]) / tau);
                    ge[a] += Q * e[a];
                }
                q += Q;
                s1 += Q / tau;
                s2 += Q / (tau * tau);
                val += Q * D2 * dot3(e, e);
            }
            double gx[3], gphi[3], tmp[3];
            matT_vec(Gam, gc, gx);
            /* dC/dphi = 2 D^2 e^T (-A) */
            for (int b = 0; b < 3; ++b) {
                tmp[b] = 0.0;
                for (int a = 0; a < 3; ++a) tmp[b] -= A[3 * a + b] * ge[a];
            }
            for (int a = 0; a < 3; ++a) {
                gphi[a] = 2.0 * D2 * tmp[a];
                grad[6 * n + a] += gphi[a];
                grad[6 * n + 3 + a] += 2.0 * D2 * gx[a];
            }
            if (value) value[n] += val;
            /* Gauss-Newton blocks with P_j = I - r r^T */
            double P[9], PG[9], GtPG[9], AtPG[9], AtA[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) P[3 * a + b] = (a == b ? 1.0 : 0.0) - r[a] * r[b];
            mat_mul(P, Gam, PG);
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    double s_gpg = 0.0, s_apg = 0.0, s_aa = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        s_gpg += Gam[3 * k + a] * PG[3 * k + b];
                        s_apg += A[3 * k + a] * PG[3 * k + b];
                        s_aa += A[3 * k + a] * A[3 * k + b];
                    }
                    GtPG[3 * a + b] = s_gpg;
                    AtPG[3 * a + b] = s_apg;
                    AtA[3 * a + b] = s_aa;
                }
            double* Hn = H + 36 * n;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    Hn[6 * a + b] += 2.0 * D2 * q * AtA[3 * a + b];
                    Hn[6 * a + 3 + b] += 2.0 * D2 * s1 * AtPG[3 * a + b];
                    Hn[6 * (3 + b) + a] += 2.0 * D2 * s1 * AtPG[3 * a + b];
                    Hn[6 * (3 + a) + 3 + b] += 2.0 * D2 * s2 * GtPG[3 * a + b];
                }
        }
    }
}

/* Solves the n x n system A y = b by Gaussian elimination with partial
 * pivoting (A and b are overwritten); returns 0 when a pivot vanishes. */
static int solve_gauss(double* A, double* b, int n, double* y) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[n * r + c]) > fabs(A[n * piv + c])) piv = r;
        if (A[n * piv + c] == 0.0) return 0;
        if (piv != c) {
            for (int k = 0; k < n; ++k) {
                double tmp = A[n * c + k];
                A[n * c + k] = A[n * piv + k];
                A[n * piv + k] = tmp;
            }
            double tb = b[c];
            b[c] = b[piv];
            b[piv] = tb;
        }
        for (int r = c + 1; r < n; ++r) {
            double fct = A[n * r + c] / A[n * c + c];
            for (int k = c; k < n; ++k) A[n * r + k] -= fct * A[n * c + k];
            b[r] -= fct * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double acc = b[r];
        for (int k = r + 1; k < n; ++k) acc -= A[n * r + k] * y[k];
        y[r] = acc / A[n * r + r];
    }
    return 1;
}

/* exp([phi]x) by Rodrigues' formula */
static void rotvec_mat(const double phi[3], double E[9]) {
    double th = sqrt(dot3(phi, phi));
    double K[9] = {0, -phi[2], phi[1], phi[2], 0, -phi[0], -phi[1], phi[0], 0}, K2[9];
    mat_mul(K, K, K2);
    double a = th > 0 ? sin(th) / th : 1.0, b = th > 0 ? (1.0 - cos(th)) / (th * th) : 0.5;
    for (int k = 0; k < 9; ++k) E[k] = (k % 4 == 0 ? 1.0 : 0.0) + a * K[k] + b * K2[k];
}

/* Adjoint M-step (an addition beside Section "The M-step updates"): n_steps
 * Levenberg-Marquardt steps per grain on E_n with Q held at the E-step plan,
 *   delta = -(H + lambda diag(H))^-1 grad,  R <- exp([delta_phi]x) R,
 *   x <- x + delta_x,
 * from orc_grain_gn at the pose of each step.  A grain whose system is
 * singular keeps its pose.  step_norms (optional, N x 2): last |delta_x| and
 * |delta_phi|. */
void orc_mstep_adjoint(const double* geom, const double* w, const double* omega, int T,
                       const int* I_off, const double* p, const int* J_off,
                       const int* grain, const int* plane, const int* det, int N,
                       const double* cE, const double* rE, const double* f, const double* g, double eps,
                       int n_steps, double lambda, double* R, double* x, double* step_norms) {
    double* grad = (double*)malloc(sizeof(double) * 6 * (N > 0 ? N : 1));
    double* H = (double*)malloc(sizeof(double) * 36 * (N > 0 ? N : 1));
    for (int it = 0; it < n_steps; ++it) {
        orc_grain_gn(geom, w, omega, T, I_off, p, J_off, grain, plane, det, N, cE, rE, f, g, eps, R, x, grad, H,
                     NULL);
        for (int n = 0; n < N; ++n) {
            double A[36], b[6], d[6];
            for (int k = 0; k < 36; ++k) A[k] = H[36 * n + k];
            for (int k = 0; k < 6; ++k) {
                A[7 * k] += lambda * H[36 * n + 7 * k];
                b[k] = -grad[6 * n + k];
            }
            int ok = 1;
            for (int k = 0; k < 6; ++k) ok &= A[7 * k] > 0.0;
            if (!ok || !solve_gauss(A, b, 6, d)) continue;
            double E[9], Rn[9];
            rotvec_mat(d, E);
            mat_mul(E, R + 9 * n, Rn);
            for (int k = 0; k < 9; ++k) R[9 * n + k] = Rn[k];
            for (int k = 0; k < 3; ++k) x[3 * n + k] += d[3 + k];
            if (step_norms) {
                step_norms[2 * n] = sqrt(d[3] * d[3] + d[4] * d[4] + d[5] * d[5]);
                step_norms[2 * n + 1] = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            }
        }
    }
    free(grad);
    free(H);
}

/* ------------------------------------------------------------------------- */
/* Unbalanced optimal transport (Appendix "Optimal transport variants")        */
/* ------------------------------------------------------------------------- */

/* Algorithm UnbalancedOT in the log domain on the plain cost matrix (no
 * dustbins), blocked by angle, from f = g = 0, row update first:
 *   f_i = tau_a (-eps LSE_j ((g_j - C_ij)/eps)),  tau_a = kappa / (kappa + eps)
 *   g_j = tau_b (-eps LSE_i ((f_i - C_ij)/eps)),  tau_b = lambda / (lambda + eps)
 * (log a = log b = 0).  Reading: Problem (B) puts kappa on the row marginal
 * (Q 1 against a, the observed spots) and lambda on the column marginal (Q^T 1
 * against b, the model spots); the printed algorithm attaches the exponents the
 * other way round, and the scaling that solves Problem (B) is used here.  A row
 * (column) of an angle block with no columns (rows) keeps potential 0. */
int orc_sinkhorn_unbalanced(const double* Dj, int T, const int* I_off, const double* p,
                            const int* J_off, const double* c, const double* r,
                            double eps, double kappa, double lambda, int n_iter,
                            double* f, double* g) {
    int nI = I_off[T], nJ = J_off[T];
    double ta = kappa / (kappa + eps), tb = lambda / (lambda + eps);
    for (int i = 0; i < nI; ++i) f[i] = 0.0;
    for (int j = 0; j < nJ; ++j) g[j] = 0.0;
    int big = (nI > nJ ? nI : nJ) + 1;
    double* buf = (double*)malloc(sizeof(double) * big);
    for (int it = 0; it < n_iter; ++it) {
        for (int t = 0; t < T; ++t)
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                int n = 0;
                for (int j = J_off[t]; j < J_off[t + 1]; ++j)
                    buf[n++] = (g[j] - orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j])) / eps;
                f[i] = n ? -ta * eps * lse(buf, n) : 0.0;
            }
        for (int t = 0; t < T; ++t)
            for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
                int n = 0;
                for (int i = I_off[t]; i < I_off[t + 1]; ++i)
                    buf[n++] = (f[i] - orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j])) / eps;
                g[j] = n ? -tb * eps * lse(buf, n) : 0.0;
            }
    }
    free(buf);
    return n_iter;
}

/* Plan read-out of the unbalanced plan Q_ij = exp((f_i + g_j - C_ij)/eps):
 * row mass r_i and column mass q_j (optional); assign_i = argmax_j Q_ij (ties
 * to the lowest index), or -1 when r_i < 1/2 (reading: a spot that keeps less
 * than half its mass untransported is an outlier); margin = top1 - top2 of
 * the row's plan entries. */
void orc_harvest_unbalanced(const double* Dj, int T, const int* I_off, const double* p,
                            const int* J_off, const double* c, const double* r, double eps,
                            const double* f, const double* g, int* assign, double* margin,
                            double* rowmass, double* q) {
    int nJ = J_off[T];
    if (q) for (int j = 0; j < nJ; ++j) q[j] = 0.0;
    for (int t = 0; t < T; ++t)
        for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
            double rs = 0.0, top1 = -1.0, top2 = -1.0;
            int arg = -1;
            for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
                double Qij = exp((f[i] + g[j] - orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j])) / eps);
                rs += Qij;
                if (q) q[j] += Qij;
                if (Qij > top1) { top2 = top1; top1 = Qij; arg = j; }
                else if (Qij > top2) top2 = Qij;
            }
            if (top1 < 0) top1 = 0.0;
            if (top2 < 0) top2 = 0.0;
            if (assign) assign[i] = rs < 0.5 ? -1 : arg;
            if (margin) margin[i] = top1 - top2;
            if (rowmass) rowmass[i] = rs;
        }
}

/* ------------------------------------------------------------------------- */
/* General lattices (reciprocal basis B, a list of allowed reflections)        */
/* ------------------------------------------------------------------------- */

/* Reciprocal basis of the lattice (a, b, c, alpha, beta, gamma), Angstrom and
 * degrees: the direct basis a1 = a x, a2 in the xy plane at gamma from a1,
 * a3 completing it; B holds the reciprocal vectors b1, b2, b3 as columns
 * (a_i . b_j = delta_ij, no 2 pi), so that g = B (h, k, l) and d = 1 / |g|
 * (Section "Crystallographic planes"). */
void orc_reciprocal_basis(double a, double b, double c, double alpha, double beta, double gamma, double B[9]) {
    const double deg = 3.14159265358979323846 / 180.0;
    double ca = cos(alpha * deg), cb = cos(beta * deg), cg = cos(gamma * deg);
    double sg = sin(gamma * deg);
    double A[3][3];  /* rows: a1, a2, a3 */
    A[0][0] = a;      A[0][1] = 0.0;    A[0][2] = 0.0;
    A[1][0] = b * cg; A[1][1] = b * sg; A[1][2] = 0.0;
    double c1 = c * cb, c2 = c * (ca - cb * cg) / sg;
    A[2][0] = c1;     A[2][1] = c2;     A[2][2] = sqrt(c * c - c1 * c1 - c2 * c2);
    double V = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1]) - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0]) +
               A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    /* b1 = a2 x a3 / V, b2 = a3 x a1 / V, b3 = a1 x a2 / V */
    double bv[3][3];
    cross3(A[1], A[2], bv[0]);
    cross3(A[2], A[0], bv[1]);
    cross3(A[0], A[1], bv[2]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) B[3 * i + j] = bv[j][i] / V;
}

typedef struct { int p[3]; int m; double len2; } hkl_item_t;

static int hkl_item_cmp(const void* A, const void* B) {
    const hkl_item_t* x = (const hkl_item_t*)A;
    const hkl_item_t* y = (const hkl_item_t*)B;
    for (int k = 0; k < 3; ++k)
        if (x->p[k] != y->p[k]) return x->p[k] < y->p[k] ? -1 : 1;
    return x->m < y->m ? -1 : (x->m > y->m ? 1 : 0);
}

typedef struct { int g0[3]; double len2; int nh; double w[3]; double d0; } grefl_t;

static int grefl_cmp(const void* A, const void* B) {
    const grefl_t* a = (const grefl_t*)A;
    const grefl_t* b = (const grefl_t*)B;
    double tol = 1e-9 * (a->len2 > b->len2 ? a->len2 : b->len2);
    if (fabs(a->len2 - b->len2) > tol) return a->len2 < b->len2 ? -1 : 1;
    for (int k = 0; k < 3; ++k)
        if (a->g0[k] != b->g0[k]) return a->g0[k] > b->g0[k] ? -1 : 1;
    return 0;
}

/* The plausible plane set from a list of allowed reflections (the paper takes
 * it as an input, Section "Tomography experiments"): reflections on one line
 * through the origin share a ray (Friedel mates +-hkl and harmonics n hkl);
 * for each line the multiples present must be m0, 2 m0, ..., nh m0 of its
 * primitive vector; the entry is g0 = m0 p with p's first nonzero index
 * positive, w = B g0 / |B g0|, d0 = 1 / |B g0|, nh.  Order: |B g0|^2
 * ascending (equal within 1e-9 relative), then g0 descending.  Returns the
 * number of entries, or -1 when a line's multiples are not of that form. */
int orc_reflections_hkl(const double B[9], const int* hkl, int n, int cap,
                        double* w, double* d0, int* nharm, int* hkl0) {
    hkl_item_t* it = (hkl_item_t*)malloc(sizeof(hkl_item_t) * (size_t)(n > 0 ? n : 1));
    int ni = 0;
    for (int q = 0; q < n; ++q) {
        int h = hkl[3 * q], k = hkl[3 * q + 1], l = hkl[3 * q + 2];
        if (h == 0 && k == 0 && l == 0) continue;
        int g = gcd_int(gcd_int(h, k), l);
        int p[3] = {h / g, k / g, l / g};
        int first = p[0] != 0 ? p[0] : (p[1] != 0 ? p[1] : p[2]);
        if (first < 0) { p[0] = -p[0]; p[1] = -p[1]; p[2] = -p[2]; }
        it[ni].p[0] = p[0]; it[ni].p[1] = p[1]; it[ni].p[2] = p[2];
        it[ni].m = g;
        ++ni;
    }
    qsort(it, (size_t)ni, sizeof(hkl_item_t), hkl_item_cmp);
    grefl_t* out = (grefl_t*)malloc(sizeof(grefl_t) * (size_t)(ni > 0 ? ni : 1));
    int no = 0;
    for (int s = 0; s < ni;) {
        int e = s;
        while (e < ni && it[e].p[0] == it[s].p[0] && it[e].p[1] == it[s].p[1] && it[e].p[2] == it[s].p[2]) ++e;
        /* distinct multiples of this line */
        int mult[256], nm = 0;
        for (int q = s; q < e; ++q)
            if (nm == 0 || it[q].m != mult[nm - 1]) {
                if (nm >= 256) { free(it); free(out); return -1; }
                mult[nm++] = it[q].m;
            }
        for (int q = 0; q < nm; ++q)
            if (mult[q] != (q + 1) * mult[0]) { free(it); free(out); return -1; }
        grefl_t* R = &out[no++];
        for (int a = 0; a < 3; ++a) R->g0[a] = mult[0] * it[s].p[a];
        double g[3];
        for (int a = 0; a < 3; ++a) g[a] = B[3 * a] * R->g0[0] + B[3 * a + 1] * R->g0[1] + B[3 * a + 2] * R->g0[2];
        R->len2 = dot3(g, g);
        double len = sqrt(R->len2);
        for (int a = 0; a < 3; ++a) R->w[a] = g[a] / len;
        R->d0 = 1.0 / len;
        R->nh = nm;
        s = e;
    }
    qsort(out, (size_t)no, sizeof(grefl_t), grefl_cmp);
    for (int m = 0; m < no && m < cap; ++m) {
        for (int q = 0; q < 3; ++q) {
            w[3 * m + q] = out[m].w[q];
            if (hkl0) hkl0[3 * m + q] = out[m].g0[q];
        }
        d0[m] = out[m].d0;
        nharm[m] = out[m].nh;
    }
    free(it);
    free(out);
    return no;
}

/* ------------------------------------------------------------------------- */
/* Sparse assignment (Section "Working with sparse assignment matrices")       */
/* ------------------------------------------------------------------------- */

typedef struct { double c; int i; } knn_item_t;

static int knn_cmp(const void* A, const void* B) {
    const knn_item_t* a = (const knn_item_t*)A;
    const knn_item_t* b = (const knn_item_t*)B;
    if (a->c != b->c) return a->c < b->c ? -1 : 1;
    return a->i < b->i ? -1 : (a->i > b->i ? 1 : 0);
}

/* Neighbour sets of the sparse plan.  Reading: each model spot j keeps the
 * rho observed spots of its angle block with the smallest cost C_ij (ties to
 * the lower index; all of them when the block has at most rho), so that a
 * Sinkhorn update costs rho |J| instead of |I| |J|; every other entry of the
 * plan between observed and model spots is 0, the dustbin row and column
 * stay dense.  nbr: |J| x rho observed indices, -1 past the block's size. */
void orc_knn(const double* Dj, int T, const int* I_off, const double* p, const int* J_off, const double* c,
             const double* r, int rho, int* nbr) {
    int big = 1;
    for (int t = 0; t < T; ++t)
        if (I_off[t + 1] - I_off[t] > big) big = I_off[t + 1] - I_off[t];
    knn_item_t* buf = (knn_item_t*)malloc(sizeof(knn_item_t) * (size_t)big);
    for (int t = 0; t < T; ++t)
        for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
            int n = 0;
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                buf[n].c = orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j]);
                buf[n].i = i;
                ++n;
            }
            qsort(buf, (size_t)n, sizeof(knn_item_t), knn_cmp);
            for (int k = 0; k < rho; ++k) nbr[(long)j * rho + k] = k < n ? buf[k].i : -1;
        }
    free(buf);
}

/* Algorithm BalancedOT (log domain, dustbins as in orc_sinkhorn) with the
 * observed-model entries of the plan restricted to the neighbour sets:
 *   f_i = -eps LSE({(g_j - C_ij)/eps : i in N(j)} u {(g_0 - c_out)/eps})
 *   g_j = -eps LSE({(f_i - C_ij)/eps : i in N(j)} u {f_0 / eps})
 * and the dustbin updates of orc_sinkhorn.  Runs n_iter iterations from
 * f = g = 0. */
int orc_sinkhorn_sparse(const double* Dj, int T, const int* I_off, const double* p, const int* J_off,
                        const double* c, const double* r, double eps, double c_out, int mode, double frac,
                        int n_iter, int rho, double* f, double* g, double* fd, double* gd) {
    int nI = I_off[T], nJ = J_off[T];
    int nd = mode ? T : 1;
    int* nbr = (int*)malloc(sizeof(int) * ((size_t)nJ * rho + 1));
    orc_knn(Dj, T, I_off, p, J_off, c, r, rho, nbr);
    /* per observed spot: the model spots whose neighbour set holds it */
    int* rcount = (int*)calloc((size_t)nI + 1, sizeof(int));
    for (long e = 0; e < (long)nJ * rho; ++e)
        if (nbr[e] >= 0) ++rcount[nbr[e] + 1];
    for (int i = 0; i < nI; ++i) rcount[i + 1] += rcount[i];
    int* rows = (int*)malloc(sizeof(int) * ((size_t)rcount[nI] + 1));
    int* fill = (int*)calloc((size_t)nI + 1, sizeof(int));
    for (int j = 0; j < nJ; ++j)
        for (int k = 0; k < rho; ++k) {
            int i = nbr[(long)j * rho + k];
            if (i >= 0) rows[rcount[i] + fill[i]++] = j;
        }
    double* U = (double*)malloc(sizeof(double) * nd);
    double* O = (double*)malloc(sizeof(double) * nd);
    orc_masses(mode, frac, T, I_off, J_off, U, O);
    for (int i = 0; i < nI; ++i) f[i] = 0.0;
    for (int j = 0; j < nJ; ++j) g[j] = 0.0;
    for (int d = 0; d < nd; ++d) fd[d] = gd[d] = 0.0;
    int big = (nI > nJ ? nI : nJ) + rho + 2;
    double* buf = (double*)malloc(sizeof(double) * big);
    for (int it = 0; it < n_iter; ++it) {
        for (int t = 0; t < T; ++t) {
            int dd = mode ? t : 0;
            for (int i = I_off[t]; i < I_off[t + 1]; ++i) {
                int n = 0;
                for (int e = rcount[i]; e < rcount[i + 1]; ++e) {
                    int j = rows[e];
                    buf[n++] = (g[j] - orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j])) / eps;
                }
                buf[n++] = (gd[dd] - c_out) / eps;
                f[i] = -eps * lse(buf, n);
            }
        }
        for (int d = 0; d < nd; ++d) {
            int j0 = mode ? J_off[d] : 0, j1 = mode ? J_off[d + 1] : nJ;
            int n = 0;
            for (int j = j0; j < j1; ++j) buf[n++] = g[j] / eps;
            buf[n++] = (gd[d] - c_out) / eps;
            fd[d] = eps * logm(U[d]) - eps * lse(buf, n);
        }
        for (int t = 0; t < T; ++t) {
            int dd = mode ? t : 0;
            for (int j = J_off[t]; j < J_off[t + 1]; ++j) {
                int n = 0;
                for (int k = 0; k < rho; ++k) {
                    int i = nbr[(long)j * rho + k];
                    if (i < 0) continue;
                    buf[n++] = (f[i] - orc_pair_cost(p + 3 * i, c + 3 * j, r + 3 * j, Dj[j])) / eps;
                }
                buf[n++] = fd[dd] / eps;
                g[j] = -eps * lse(buf, n);
            }
        }
        for (int d = 0; d < nd; ++d) {
            int i0 = mode ? I_off[d] : 0, i1 = mode ? I_off[d + 1] : nI;
            int n = 0;
            for (int i = i0; i < i1; ++i) buf[n++] = (f[i] - c_out) / eps;
            buf[n++] = (fd[d] - c_out) / eps;
            gd[d] = eps * logm(O[d]) - eps * lse(buf, n);
        }
    }
    free(buf); free(U); free(O); free(nbr); free(rcount); free(rows); free(fill);
    return n_iter;
}
