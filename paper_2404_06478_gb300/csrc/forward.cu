// forward.cu — forward Laue model and model-spot cut (paper Eqs. ray_mnt,
// s_mnt, wavelength_lambda and model_spot_cut), and the refresh of a frozen
// model-spot list at new poses.
//
// One thread per (t, n, m) ray, flat index (t*N + n)*M + m, so that the
// compacted list comes out sorted by (t, n, m) without a sort: a count pass,
// an exclusive scan of the per-block counts, and a write pass that recomputes
// each ray and scatters the visible ones.
#include "common.cuh"
#include "kernels.h"
#include "ray.cuh"

namespace laue {

__global__ void __launch_bounds__(kFwdBlock) fwd_count_kernel(FwdArgs a) {
    long long idx = (long long)blockIdx.x * kFwdBlock + threadIdx.x;
    bool vis = false;
    if (idx < a.n_rays) {
        int m = (int)(idx % a.M);
        long long q = idx / a.M;
        int n = (int)(q % a.N);
        int t = (int)(q / a.N);
        float sg, cg;
        sincosf(a.omega[t], &sg, &cg);
        RayOut o;
        vis = ray_one(a.G, cg, sg, a.R + 9 * n, a.x + 3 * n, a.w_d0[m], a.nharm[m], o);
    }
    int cnt = __syncthreads_count(vis);
    if (threadIdx.x == 0) a.blocks[blockIdx.x] = cnt;
}

// Exclusive scan of the per-block counts by one CTA; writes offsets after the
// counts, the total, and J_off[T] = total.
__global__ void __launch_bounds__(1024) fwd_scan_kernel(FwdArgs a) {
    __shared__ int part[1024];
    int nb = a.n_blocks;
    int per = (nb + 1023) / 1024;
    int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    int s = 0;
    for (int b = b0; b < b1; ++b) s += a.blocks[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int acc = 0;
        for (int k = 0; k < 1024; ++k) {
            int v = part[k];
            part[k] = acc;
            acc += v;
        }
        a.ctrl[CTRL_FWD_TOTAL] = acc;
        a.J_off[a.T] = acc;
    }
    __syncthreads();
    int acc = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        a.blocks[nb + b] = acc;
        acc += a.blocks[b];
    }
}

__global__ void __launch_bounds__(kFwdBlock) fwd_write_kernel(FwdArgs a) {
    __shared__ int warp_cnt[kFwdBlock / 32];
    long long idx = (long long)blockIdx.x * kFwdBlock + threadIdx.x;
    bool vis = false;
    RayOut o;
    int m = 0, n = 0, t = 0;
    if (idx < a.n_rays) {
        m = (int)(idx % a.M);
        long long q = idx / a.M;
        n = (int)(q % a.N);
        t = (int)(q / a.N);
        float sg, cg;
        sincosf(a.omega[t], &sg, &cg);
        vis = ray_one(a.G, cg, sg, a.R + 9 * n, a.x + 3 * n, a.w_d0[m], a.nharm[m], o);
    }
    unsigned ball = __ballot_sync(0xffffffffu, vis);
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) warp_cnt[warp] = __popc(ball);
    __syncthreads();
    int before = 0;
    for (int k = 0; k < warp; ++k) before += warp_cnt[k];
    int local = before + __popc(ball & ((1u << lane) - 1u));
    int pos = a.blocks[a.n_blocks + blockIdx.x] + local;
    // J_off[t] = number of visible rays before the first ray of angle t
    if (idx < a.n_rays && n == 0 && m == 0) a.J_off[t] = pos;
    if (vis && pos < a.capacity) {
        a.grain[pos] = n;
        a.plane[pos] = m;
        a.angle[pos] = t;
        a.ray[pos] = make_float4(o.r[0], o.r[1], o.r[2], o.lam);
        a.center[pos] = make_float4(o.c[0], o.c[1], o.c[2], 0.0f);
        a.spot[pos] = make_float4(o.s[0], o.s[1], o.s[2], (float)o.det);
    }
}

// Frozen list at new poses: rays, wavelengths, centres, and the spot position
// on the detector recorded for the spot.
__global__ void refresh_kernel(RefreshArgs a) {
    int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= a.n) return;
    int t = a.angle[j], n = a.grain[j], m = a.plane[j];
    float sg, cg;
    sincosf(a.omega[t], &sg, &cg);
    const float* R = a.R + 9 * n;
    const float* x = a.x + 3 * n;
    float4 wd = a.w_d0[m];
    int nh = a.nharm[m];
    float v0 = R[0] * wd.x + R[1] * wd.y + R[2] * wd.z;
    float v1 = R[3] * wd.x + R[4] * wd.y + R[5] * wd.z;
    float v2 = R[6] * wd.x + R[7] * wd.y + R[8] * wd.z;
    float u0 = cg * v0 + sg * v2, u1 = v1, u2 = -sg * v0 + cg * v2;
    float c0 = cg * x[0] + sg * x[2], c1 = x[1], c2 = -sg * x[0] + cg * x[2];
    const GeomDev& G = a.G;
    float ue = u0 * G.e[0] + u1 * G.e[1] + u2 * G.e[2];
    float r0 = G.e[0] - 2.0f * ue * u0, r1 = G.e[1] - 2.0f * ue * u1, r2 = G.e[2] - 2.0f * ue * u2;
    float lam0 = 2.0f * wd.w * fabsf(ue), lam = lam0;
    for (int k = 1; k <= nh; ++k) {
        float ln = lam0 / (float)k;
        if (ln >= G.lam_min && ln <= G.lam_max) {
            lam = ln;
            break;
        }
    }
    a.ray[j] = make_float4(r0, r1, r2, lam);
    a.center[j] = make_float4(c0, c1, c2, 0.0f);
    float4 sp = a.spot[j];
    int k = (int)sp.w;
    if (k >= 0 && k < G.n_det) {
        float den = G.nrm[k][0] * r0 + G.nrm[k][1] * r1 + G.nrm[k][2] * r2;
        float num = G.nrm[k][0] * (G.ctr[k][0] - c0) + G.nrm[k][1] * (G.ctr[k][1] - c1) +
                    G.nrm[k][2] * (G.ctr[k][2] - c2);
        float tau = den != 0.0f ? num / den : 0.0f;
        a.spot[j] = make_float4(c0 + tau * r0, c1 + tau * r1, c2 + tau * r2, sp.w);
    }
}

cudaError_t launch_forward(const FwdArgs& a, cudaStream_t s) {
    if (a.n_rays == 0) {
        fwd_scan_kernel<<<1, 1024, 0, s>>>(a);
        return cudaGetLastError();
    }
    fwd_count_kernel<<<a.n_blocks, kFwdBlock, 0, s>>>(a);
    fwd_scan_kernel<<<1, 1024, 0, s>>>(a);
    fwd_write_kernel<<<a.n_blocks, kFwdBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_refresh(const RefreshArgs& a, cudaStream_t s) {
    if (a.n > 0) refresh_kernel<<<(a.n + 255) / 256, 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace laue
