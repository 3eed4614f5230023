// ray.cuh — one ray of the forward Laue model (Section "Forward model",
// Eqs. ray_mnt, s_mnt, wavelength; cut of Eq. model_spot_cut), shared by the
// forward kernels and the training-scene generator of the set encoder.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace laue {

// Plane point s inside detector k: |(s - centre).a| < half for both in-plane
// axes a1, a2 (for a plane normal to z: |dx| < half and |dy| < half).
__device__ __forceinline__ bool on_detector(const GeomDev& G, int k, float s0, float s1, float s2) {
    float d0 = s0 - G.ctr[k][0], d1 = s1 - G.ctr[k][1], d2 = s2 - G.ctr[k][2];
    float u = fmaf(d0, G.ax1[k][0], fmaf(d1, G.ax1[k][1], d2 * G.ax1[k][2]));
    float v = fmaf(d0, G.ax2[k][0], fmaf(d1, G.ax2[k][1], d2 * G.ax2[k][2]));
    return fabsf(u) < G.half[k] && fabsf(v) < G.half[k];
}

// Detector hit by the ray c + tau r: the smallest tau > 0 whose plane point is
// on its detector; -1 when none.  s receives the point.
__device__ __forceinline__ int hit_detector(const GeomDev& G, const float* r, const float* c, float* s) {
    int det = -1;
    float best = 3.0e38f;
    for (int k = 0; k < G.n_det; ++k) {
        float den = G.nrm[k][0] * r[0] + G.nrm[k][1] * r[1] + G.nrm[k][2] * r[2];
        if (den == 0.0f) continue;
        float num = G.nrm[k][0] * (G.ctr[k][0] - c[0]) + G.nrm[k][1] * (G.ctr[k][1] - c[1]) +
                    G.nrm[k][2] * (G.ctr[k][2] - c[2]);
        float tau = num / den;
        if (!(tau > 0.0f)) continue;
        float s0 = c[0] + tau * r[0], s1 = c[1] + tau * r[1], s2 = c[2] + tau * r[2];
        if (on_detector(G, k, s0, s1, s2) && tau < best) {
            best = tau;
            det = k;
            s[0] = s0;
            s[1] = s1;
            s[2] = s2;
        }
    }
    return det;
}

struct RayOut {
    float r[3];
    float lam;
    float s[3];
    float c[3];
    int det;
};

// u = Gamma_t R_n w_m, r = e - 2 (u.e) u, c = Gamma_t x_n; wavelength of the
// first harmonic in band; detector with the smallest tau > 0 whose square
// holds the spot.  Returns visibility.
__device__ __forceinline__ bool ray_one(const GeomDev& G, float cg, float sg, const float* __restrict__ R,
                                        const float* __restrict__ x, float4 wd, int nh, RayOut& o) {
    float v0 = R[0] * wd.x + R[1] * wd.y + R[2] * wd.z;
    float v1 = R[3] * wd.x + R[4] * wd.y + R[5] * wd.z;
    float v2 = R[6] * wd.x + R[7] * wd.y + R[8] * wd.z;
    // Gamma_t = [[c, 0, s], [0, 1, 0], [-s, 0, c]] (right-handed about +y)
    float u0 = cg * v0 + sg * v2, u1 = v1, u2 = -sg * v0 + cg * v2;
    o.c[0] = cg * x[0] + sg * x[2];
    o.c[1] = x[1];
    o.c[2] = -sg * x[0] + cg * x[2];
    float ue = u0 * G.e[0] + u1 * G.e[1] + u2 * G.e[2];
    o.r[0] = G.e[0] - 2.0f * ue * u0;
    o.r[1] = G.e[1] - 2.0f * ue * u1;
    o.r[2] = G.e[2] - 2.0f * ue * u2;
    float lam0 = 2.0f * wd.w * fabsf(ue);
    bool in_band = false;
    o.lam = lam0;
    for (int n = 1; n <= nh; ++n) {
        float ln = lam0 / (float)n;
        if (ln >= G.lam_min && ln <= G.lam_max) {
            in_band = true;
            o.lam = ln;
            break;
        }
    }
    o.det = hit_detector(G, o.r, o.c, o.s);
    return in_band && o.det >= 0;
}

}  // namespace laue
