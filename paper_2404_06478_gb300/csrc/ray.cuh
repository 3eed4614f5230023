// ray.cuh — one ray of the forward Laue model (Section "Forward model",
// Eqs. ray_mnt, s_mnt, wavelength; cut of Eq. model_spot_cut), shared by the
// forward kernels and the training-scene generator of the set encoder.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace laue {

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
    o.det = -1;
    float best = 3.0e38f;
    for (int k = 0; k < G.n_det; ++k) {
        float den = G.nrm[k][0] * o.r[0] + G.nrm[k][1] * o.r[1] + G.nrm[k][2] * o.r[2];
        if (den == 0.0f) continue;
        float num = G.nrm[k][0] * (G.ctr[k][0] - o.c[0]) + G.nrm[k][1] * (G.ctr[k][1] - o.c[1]) +
                    G.nrm[k][2] * (G.ctr[k][2] - o.c[2]);
        float tau = num / den;
        if (!(tau > 0.0f)) continue;
        float s0 = o.c[0] + tau * o.r[0], s1 = o.c[1] + tau * o.r[1], s2 = o.c[2] + tau * o.r[2];
        float dist = fmaxf(fabsf(s0 - G.ctr[k][0]), fmaxf(fabsf(s1 - G.ctr[k][1]), fabsf(s2 - G.ctr[k][2])));
        if (dist < G.half[k] && tau < best) {
            best = tau;
            o.det = k;
            o.s[0] = s0;
            o.s[1] = s1;
            o.s[2] = s2;
        }
    }
    return in_band && o.det >= 0;
}

}  // namespace laue
