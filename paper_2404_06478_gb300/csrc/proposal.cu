// proposal.cu — the learned proposal: a set encoder that reads a
// seed-conditioned set of observed spots and proposes grain poses for the
// single-grain fits.  The paper has no learned component; this is an
// addition beside its candidate scan (Section "Pre-processing"), which stays
// both the fallback and the measure of the proposal's recall.
//
// Kernels:
//   training scenes  grains drawn by Philox4x32-10 (Salmon et al., SC'11),
//                    spots from the forward model (Eqs. ray_mnt, s_mnt,
//                    wavelength, model_spot_cut) with detector noise and
//                    uniform outliers, seeds drawn among the inliers;
//   sets             sample-frame spot axes (u parallel to rhat - e, n =
//                    Gamma_t^T u), the KSET - 1 nearest axes to the seed's in its
//                    rotation window by a three-round radix select, features
//                    in the seed frame (BF16, row-major);
//   network          per-spot layers and the head on the tcgen05 GEMM
//                    (gemm_tc.cu, BF16 operands, FP32 accumulation), masked
//                    mean/max pooling, symmetric multi-hypothesis loss,
//                    backward, Adam.
// Every reduction runs in a fixed order: the same inputs give the same bits.
#include <cuda_bf16.h>

#include "api_internal.h"
#include "gemm_tc.h"
#include "proposal.cuh"
#include "ray.cuh"

namespace laue {
namespace lp {
namespace {

constexpr uint32_t TAG_NOISE = 0, TAG_COUNT = 1, TAG_OUTLIER = 2, TAG_SEED = 3, TAG_SCENE = 4, TAG_GRAIN = 5;
constexpr uint32_t ALL = 0xFFFFFFFFu;
constexpr int kSeedTries = 64;

// ------------------------------------------------------------------ Philox
__device__ __forceinline__ uint4 philox(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}
// (0, 1) uniform: ((x >> 8) + 1/2) 2^-24, exact in FP32
__device__ __forceinline__ float u01(uint32_t x) { return ((float)(x >> 8) + 0.5f) * (1.0f / 16777216.0f); }
// integer in [0, n): ((x >> 8) n) >> 24
__device__ __forceinline__ int uniform_int(uint32_t x, int n) {
    return (int)(((unsigned long long)(x >> 8) * (unsigned long long)n) >> 24);
}
__device__ __forceinline__ void normal_pair(uint32_t a, uint32_t b, float& z1, float& z2) {
    float rad = sqrtf(-2.0f * logf(u01(a)));
    float s, c;
    sincospif(2.0f * u01(b), &s, &c);
    z1 = rad * c;
    z2 = rad * s;
}

// ------------------------------------------------------------------ scenes
struct SceneArgs {
    GeomDev G;
    const float4* w_d0;
    const int* nharm;
    int M;
    const float* omega;
    int T, W, S, Gmax, gmin, gmax;
    float cube, sigma;
    double ratio;
    uint2 key;
    float* R;
    float* x;
    int* n_g;
    int* t0;
    int* counts;  // 2 S W: n_true, n_out
    int* I_off;   // S W + 1
    float* omega_v;
    int capacity;
    float4* p;
    int* label;
    int* ctrl;
};

// Shoemake's uniform rotation from three uniforms (Graphics Gems III, 1992).
__device__ void shoemake(float u1, float u2, float u3, float* R) {
    float a = sqrtf(1.0f - u1), b = sqrtf(u1);
    float s2, c2, s3, c3;
    sincospif(2.0f * u2, &s2, &c2);
    sincospif(2.0f * u3, &s3, &c3);
    float qx = a * s2, qy = a * c2, qz = b * s3, qw = b * c3;
    R[0] = 1 - 2 * (qy * qy + qz * qz);
    R[1] = 2 * (qx * qy - qz * qw);
    R[2] = 2 * (qx * qz + qy * qw);
    R[3] = 2 * (qx * qy + qz * qw);
    R[4] = 1 - 2 * (qx * qx + qz * qz);
    R[5] = 2 * (qy * qz - qx * qw);
    R[6] = 2 * (qx * qz - qy * qw);
    R[7] = 2 * (qy * qz + qx * qw);
    R[8] = 1 - 2 * (qx * qx + qy * qy);
}

__global__ void scene_params_kernel(SceneArgs a) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= a.S * a.Gmax) return;
    int s = idx / a.Gmax, g = idx % a.Gmax;
    if (g == 0) {
        uint4 w = philox(make_uint4((uint32_t)s, ALL, 0u, TAG_SCENE), a.key);
        a.t0[s] = uniform_int(w.x, a.T - a.W + 1);
        a.n_g[s] = a.gmin + uniform_int(w.y, a.gmax - a.gmin + 1);
    }
    uint4 wr = philox(make_uint4((uint32_t)s, (uint32_t)g, 0u, TAG_GRAIN), a.key);
    shoemake(u01(wr.x), u01(wr.y), u01(wr.z), a.R + 9 * (size_t)idx);
    uint4 wx = philox(make_uint4((uint32_t)s, (uint32_t)g, 1u, TAG_GRAIN), a.key);
    a.x[3 * (size_t)idx + 0] = a.cube * (u01(wx.x) - 0.5f);
    a.x[3 * (size_t)idx + 1] = a.cube * (u01(wx.y) - 0.5f);
    a.x[3 * (size_t)idx + 2] = a.cube * (u01(wx.z) - 0.5f);
}

// The noisy spot of (grain g, plane m) at virtual angle v, if it is seen.
__device__ __forceinline__ bool scene_spot(const SceneArgs& a, int v, int s, int g, int m, float cg, float sg,
                                           float4& out) {
    RayOut o;
    size_t gi = (size_t)s * a.Gmax + g;
    if (!ray_one(a.G, cg, sg, a.R + 9 * gi, a.x + 3 * gi, a.w_d0[m], a.nharm[m], o)) return false;
    uint4 w = philox(make_uint4((uint32_t)v, (uint32_t)g, (uint32_t)m, TAG_NOISE), a.key);
    float z1, z2;
    normal_pair(w.x, w.y, z1, z2);
    float X = o.s[0] + a.sigma * z1, Y = o.s[1] + a.sigma * z2;
    int d = o.det;
    if (!(fabsf(X - a.G.ctr[d][0]) < a.G.half[d] && fabsf(Y - a.G.ctr[d][1]) < a.G.half[d])) return false;
    out = make_float4(X, Y, o.s[2], 0.0f);
    return true;
}

__global__ void __launch_bounds__(256) scene_count_kernel(SceneArgs a) {
    int v = blockIdx.x, s = v / a.W, k = v % a.W;
    float w = a.omega[a.t0[s] + k];
    float sg, cg;
    sincosf(w, &sg, &cg);
    int nr = a.n_g[s] * a.M, cnt = 0;
    for (int base = 0; base < nr; base += blockDim.x) {
        int id = base + threadIdx.x;
        bool kept = false;
        if (id < nr) {
            float4 q;
            kept = scene_spot(a, v, s, id / a.M, id % a.M, cg, sg, q);
        }
        cnt += __syncthreads_count(kept);
    }
    if (threadIdx.x == 0) {
        uint4 c = philox(make_uint4((uint32_t)v, ALL, 0u, TAG_COUNT), a.key);
        int n_out = (int)floor(a.ratio * (double)cnt + (double)u01(c.x));
        a.counts[2 * v] = cnt;
        a.counts[2 * v + 1] = n_out;
        a.omega_v[v] = w;
    }
}

// exclusive offsets of the per-angle counts, staged through shared memory in
// chunks of 1024 (one block)
__global__ void __launch_bounds__(1024) scene_scan_kernel(SceneArgs a) {
    __shared__ int cnt[1024];
    __shared__ int carry;
    int nv = a.S * a.W;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < nv; base += 1024) {
        int v = base + threadIdx.x;
        cnt[threadIdx.x] = v < nv ? a.counts[2 * v] + a.counts[2 * v + 1] : 0;
        __syncthreads();
        if (threadIdx.x == 0) {
            int acc = carry, n = min(1024, nv - base);
            for (int k = 0; k < n; ++k) {
                int c = cnt[k];
                cnt[k] = acc;
                acc += c;
            }
            carry = acc;
        }
        __syncthreads();
        if (v < nv) a.I_off[v] = min(cnt[threadIdx.x], a.capacity);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (carry > a.capacity) set_status(a.ctrl, LAUE_ERR_CAPACITY);
        a.I_off[nv] = min(carry, a.capacity);
    }
}

__global__ void __launch_bounds__(256) scene_write_kernel(SceneArgs a) {
    __shared__ int wcnt[8];
    __shared__ int written;
    int v = blockIdx.x, s = v / a.W;
    float sg, cg;
    sincosf(a.omega_v[v], &sg, &cg);
    int nr = a.n_g[s] * a.M;
    int base_pos = a.I_off[v], end = a.I_off[v + 1];
    if (threadIdx.x == 0) written = 0;
    __syncthreads();
    int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    for (int base = 0; base < nr; base += blockDim.x) {
        int id = base + threadIdx.x;
        float4 q = make_float4(0, 0, 0, 0);
        bool kept = false;
        int g = 0;
        if (id < nr) {
            g = id / a.M;
            kept = scene_spot(a, v, s, g, id % a.M, cg, sg, q);
        }
        unsigned ball = __ballot_sync(0xffffffffu, kept);
        if (lane == 0) wcnt[wp] = __popc(ball);
        __syncthreads();
        int before = 0, total = 0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
            if (k < wp) before += wcnt[k];
            total += wcnt[k];
        }
        int pos = base_pos + written + before + __popc(ball & ((1u << lane) - 1u));
        if (kept && pos < end) {
            a.p[pos] = q;
            a.label[pos] = s * a.Gmax + g;
        }
        __syncthreads();
        if (threadIdx.x == 0) written += total;
        __syncthreads();
    }
    int n_true = a.counts[2 * v], n_out = a.counts[2 * v + 1];
    for (int k = threadIdx.x; k < n_out; k += blockDim.x) {
        int pos = base_pos + n_true + k;
        if (pos >= end) break;
        uint4 w = philox(make_uint4((uint32_t)v, ALL, (uint32_t)k, TAG_OUTLIER), a.key);
        int d = min((int)(u01(w.x) * (float)a.G.n_det), a.G.n_det - 1);
        a.p[pos] = make_float4(a.G.ctr[d][0] + a.G.half[d] * (2.0f * u01(w.y) - 1.0f),
                               a.G.ctr[d][1] + a.G.half[d] * (2.0f * u01(w.z) - 1.0f), a.G.ctr[d][2], 0.0f);
        a.label[pos] = -1;
    }
}

__global__ void scene_seeds_kernel(const int* I_off, const int* label, int W, int S, int per_scene, uint2 key,
                                   int* seeds, int* wlo, int* whi) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= S * per_scene) return;
    int s = b / per_scene, j = b % per_scene;
    int lo = I_off[s * W], ns = I_off[(s + 1) * W] - lo;
    int seed = -1;
    for (int q = 0; q < kSeedTries && ns > 0; ++q) {
        uint4 w = philox(make_uint4((uint32_t)s, (uint32_t)j, (uint32_t)q, TAG_SEED), key);
        int i = lo + uniform_int(w.x, ns);
        if (label[i] >= 0) {
            seed = i;
            break;
        }
    }
    seeds[b] = seed;
    wlo[b] = s * W;
    whi[b] = (s + 1) * W;
}

// ------------------------------------------------------------------ sets
// Sample-frame axis of every spot, angle index in .w (as int bits).
__global__ void axes_kernel(const float4* p, const int* I_off, int n_angles, const float* omega, GeomDev G,
                            int cap, float4* axes) {
    int n = min(I_off[n_angles], cap);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        int lo = 0, hi = n_angles;  // largest t with I_off[t] <= i
        while (hi - lo > 1) {
            int mid = (lo + hi) >> 1;
            if (I_off[mid] <= i) lo = mid;
            else hi = mid;
        }
        float4 q = p[i];
        float inv = rsqrtf(q.x * q.x + q.y * q.y + q.z * q.z);
        float u0 = q.x * inv - G.e[0], u1 = q.y * inv - G.e[1], u2 = q.z * inv - G.e[2];
        float nu = sqrtf(u0 * u0 + u1 * u1 + u2 * u2);
        if (nu < 1e-6f) {
            u0 = 1.0f;
            u1 = u2 = 0.0f;
        } else {
            u0 /= nu;
            u1 /= nu;
            u2 /= nu;
        }
        float sg, cg;
        sincosf(omega[lo], &sg, &cg);
        axes[i] = make_float4(cg * u0 - sg * u2, u1, sg * u0 + cg * u2, __int_as_float(lo));
    }
}

struct SetsArgs {
    const float4* p;
    const float4* axes;
    const int* I_off;
    const float* omega;
    int n_angles;
    const int* seeds;
    const int* wlo;
    const int* whi;
    int B;
    const int* label;
    const float* gR;
    const float* gX;
    __nv_bfloat16* X;
    float* F;
    int* nvalid;
    float* Rt;
    float* xt;
    float* svalid;
    int* ids;
    int* ctrl;
};

__device__ __forceinline__ uint32_t dist_key(float4 n, float3 n0) {
    float d = 1.0f - fabsf(n.x * n0.x + n.y * n0.y + n.z * n0.z);
    return __float_as_uint(fmaxf(d, 0.0f));
}

constexpr int kSetThreads = 256;

// Finds, among the keys of [lo, hi) minus i0 that match `prefix` on the
// bits of `pmask`, the bin of bits [sh, sh + nbits) that holds the k-th
// smallest (1-based); updates prefix, pmask and k (rank within the bin).
__device__ void radix_round(const SetsArgs& a, int lo, int hi, int i0, float3 n0, int sh, int nbits,
                            uint32_t& prefix, uint32_t& pmask, int& k, int* hist, int* part) {
    int nb = 1 << nbits;
    for (int j = threadIdx.x; j < nb; j += blockDim.x) hist[j] = 0;
    __syncthreads();
    uint32_t bm = (uint32_t)nb - 1u;
    for (int i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        if (i == i0) continue;
        uint32_t key = dist_key(a.axes[i], n0);
        if ((key & pmask) == prefix) atomicAdd(&hist[(key >> sh) & bm], 1);
    }
    __syncthreads();
    int per = nb / blockDim.x;  // 8 or 4 bins per thread
    int s = 0;
    for (int j = 0; j < per; ++j) s += hist[threadIdx.x * per + j];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int cum = 0, t = 0;
        while (t < (int)blockDim.x && cum + part[t] < k) cum += part[t++];
        int j = t * per;
        while (cum + hist[j] < k) cum += hist[j++];
        part[0] = j;
        part[1] = k - cum;
    }
    __syncthreads();
    uint32_t bin = (uint32_t)part[0];
    k = part[1];
    prefix |= bin << sh;
    pmask |= bm << sh;
    __syncthreads();
}

__global__ void __launch_bounds__(kSetThreads) sets_kernel(SetsArgs a) {
    __shared__ int hist[2048];
    __shared__ int part[kSetThreads];
    __shared__ unsigned long long sel[KSET];
    __shared__ int wcnt[kSetThreads / 32];
    __shared__ int nsel_s, ties_s;
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    const int n_total = a.I_off[a.n_angles];
    for (int b = blockIdx.x; b < a.B; b += gridDim.x) {
        int i0 = a.seeds[b];
        const int wl = min(max(a.wlo[b], 0), a.n_angles), wh = min(max(a.whi[b], wl), a.n_angles);
        if (i0 >= n_total) {
            if (threadIdx.x == 0) set_status(a.ctrl, LAUE_ERR_INVALID_ARG);
            i0 = -1;
        }
        const size_t row0 = (size_t)b * KSET;
        if (i0 < 0) {
            for (int j = threadIdx.x; j < KSET * NF; j += blockDim.x) a.X[row0 * NF + j] = __float2bfloat16_rn(0.0f);
            if (a.ids)
                for (int e = threadIdx.x; e < KSET; e += blockDim.x) a.ids[row0 + e] = -1;
            if (threadIdx.x < 9) a.F[9 * b + threadIdx.x] = 0.0f;
            if (threadIdx.x == 0) {
                a.nvalid[b] = 0;
                if (a.svalid) a.svalid[b] = 0.0f;
            }
            if (a.Rt && threadIdx.x < 9) a.Rt[9 * b + threadIdx.x] = 0.0f;
            if (a.xt && threadIdx.x < 3) a.xt[3 * b + threadIdx.x] = 0.0f;
            __syncthreads();
            continue;
        }
        const float4 s0 = a.axes[i0];
        const float3 n0 = make_float3(s0.x, s0.y, s0.z);
        const int t0 = __float_as_int(s0.w);
        const int lo = a.I_off[wl], hi = a.I_off[wh];
        const int count = hi - lo - ((i0 >= lo && i0 < hi) ? 1 : 0);
        const int K = min(KSET - 1, count);
        uint32_t tau = 0xFFFFFFFFu;
        int k_tie = 0x7FFFFFFF;
        if (count > KSET - 1) {
            uint32_t prefix = 0, pmask = 0;
            int k = KSET - 1;
            radix_round(a, lo, hi, i0, n0, 21, 11, prefix, pmask, k, hist, part);
            radix_round(a, lo, hi, i0, n0, 10, 11, prefix, pmask, k, hist, part);
            radix_round(a, lo, hi, i0, n0, 0, 10, prefix, pmask, k, hist, part);
            tau = prefix;
            k_tie = k;
        }
        // ordered collection: keys < tau, then the first k_tie keys == tau by index
        if (threadIdx.x == 0) {
            nsel_s = 0;
            ties_s = 0;
        }
        for (int e = threadIdx.x; e < KSET; e += blockDim.x) sel[e] = ~0ull;
        __syncthreads();
        for (int base = lo; base < hi; base += blockDim.x) {
            int i = base + threadIdx.x;
            uint32_t key = 0;
            bool in = i < hi && i != i0;
            if (in) key = dist_key(a.axes[i], n0);
            bool lt = in && (count <= KSET - 1 || key < tau);
            bool eq = in && count > KSET - 1 && key == tau;
            unsigned beq = __ballot_sync(0xffffffffu, eq);
            if (lane == 0) wcnt[wp] = __popc(beq);
            __syncthreads();
            int before = 0, tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                if (q < wp) before += wcnt[q];
                tot += wcnt[q];
            }
            int tie_rank = ties_s + before + __popc(beq & ((1u << lane) - 1u));
            bool take = lt || (eq && tie_rank < k_tie);
            __syncthreads();
            unsigned bt = __ballot_sync(0xffffffffu, take);
            if (lane == 0) wcnt[wp] = __popc(bt);
            __syncthreads();
            int bt_before = 0, bt_tot = 0;
            for (int q = 0; q < (int)(blockDim.x >> 5); ++q) {
                if (q < wp) bt_before += wcnt[q];
                bt_tot += wcnt[q];
            }
            int pos = nsel_s + bt_before + __popc(bt & ((1u << lane) - 1u));
            if (take && pos < KSET - 1) sel[pos] = ((unsigned long long)key << 32) | (uint32_t)i;
            __syncthreads();
            if (threadIdx.x == 0) {
                nsel_s += bt_tot;
                ties_s += tot;
            }
            __syncthreads();
        }
        // bitonic sort of the (key, index) pairs, ascending
        for (int size = 2; size <= KSET; size <<= 1) {
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int e = threadIdx.x; e < KSET; e += blockDim.x) {
                    int partner = e ^ stride;
                    if (partner > e) {
                        bool up = (e & size) == 0;
                        unsigned long long x = sel[e], y = sel[partner];
                        if ((x > y) == up) {
                            sel[e] = y;
                            sel[partner] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // seed frame
        float a1x = -n0.y * n0.x, a1y = 1.0f - n0.y * n0.y, a1z = -n0.y * n0.z;
        float na1 = sqrtf(a1x * a1x + a1y * a1y + a1z * a1z);
        if (na1 < 1e-6f) {
            a1x = 1.0f - n0.x * n0.x;
            a1y = -n0.x * n0.y;
            a1z = -n0.x * n0.z;
            na1 = sqrtf(a1x * a1x + a1y * a1y + a1z * a1z);
        }
        a1x /= na1;
        a1y /= na1;
        a1z /= na1;
        float a2x = n0.y * a1z - n0.z * a1y, a2y = n0.z * a1x - n0.x * a1z, a2z = n0.x * a1y - n0.y * a1x;
        const float4 p0 = a.p[i0];
        const float w0 = a.omega[t0];
        for (int e = threadIdx.x; e < KSET; e += blockDim.x) {
            int id = e == 0 ? i0 : (e - 1 < K ? (int)(uint32_t)(sel[e - 1] & 0xFFFFFFFFull) : -1);
            float f[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) f[q] = 0.0f;
            if (id >= 0) {
                float4 n = a.axes[id];
                float dot = n.x * n0.x + n.y * n0.y + n.z * n0.z;
                float sgn = dot < 0.0f ? -1.0f : 1.0f;
                f[0] = sgn * dot;
                f[1] = sgn * (n.x * a1x + n.y * a1y + n.z * a1z);
                f[2] = sgn * (n.x * a2x + n.y * a2y + n.z * a2z);
                int ti = __float_as_int(n.w);
                float dw = a.omega[ti] - w0;
                f[3] = sinf(dw);
                f[4] = cosf(dw);
                float4 q = a.p[id];
                f[5] = q.z / DSCALE;
                f[6] = q.x / HALFS;
                f[7] = q.y / HALFS;
                f[8] = p0.x / HALFS;
                f[9] = p0.y / HALFS;
                f[10] = p0.z / DSCALE;
                f[11] = e == 0 ? 1.0f : 0.0f;
                f[12] = 1.0f;
                f[13] = (float)(ti - t0) / 10.0f;
            }
            __nv_bfloat16* xr = a.X + (row0 + e) * NF;
            uint4* x4 = reinterpret_cast<uint4*>(xr);
            uint32_t w[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                __nv_bfloat162 h2 = __floats2bfloat162_rn(f[2 * q], f[2 * q + 1]);
                w[q] = *reinterpret_cast<uint32_t*>(&h2);
            }
            x4[0] = make_uint4(w[0], w[1], w[2], w[3]);
            x4[1] = make_uint4(w[4], w[5], w[6], w[7]);
#pragma unroll
            for (int q = 2; q < NF / 8; ++q) x4[q] = make_uint4(0, 0, 0, 0);
            if (a.ids) a.ids[row0 + e] = id;
        }
        if (threadIdx.x == 0) {
            float F0[9] = {n0.x, a1x, a2x, n0.y, a1y, a2y, n0.z, a1z, a2z};
            for (int q = 0; q < 9; ++q) a.F[9 * b + q] = F0[q];
            a.nvalid[b] = 1 + K;
            if (a.label) {
                int g = a.label[i0];
                float ok = g >= 0 ? 1.0f : 0.0f;
                a.svalid[b] = ok;
                for (int r = 0; r < 3; ++r)
                    for (int c = 0; c < 3; ++c) {
                        float acc = 0.0f;
                        if (g >= 0)
                            for (int q = 0; q < 3; ++q) acc += F0[3 * q + r] * a.gR[9 * (size_t)g + 3 * q + c];
                        a.Rt[9 * b + 3 * r + c] = acc;
                    }
                for (int q = 0; q < 3; ++q) a.xt[3 * b + q] = g >= 0 ? a.gX[3 * (size_t)g + q] / XSCALE : 0.0f;
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ network
__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }
static_assert(WIDTH == 256 && HEADW == 256, "the pooling and column-sum kernels map 256 threads to the channels");

// masked mean and max (first index on ties) of H3 over the valid rows: FP32
// into pool, rounded to BF16 into poolh (the head's operand; rows B .. Bp - 1
// of poolh are zero).  One CTA per set: thread t reads channels 8 (t % 32)
// .. + 7 of rows t / 32, t / 32 + 8, ... with 16-byte loads; the eight row
// groups are combined in order (sums added; the larger maximum, the lower
// row on ties).
__global__ void __launch_bounds__(256) pool_kernel(const __nv_bfloat16* __restrict__ H3,
                                                   const int* __restrict__ nvalid, int B, int Bp,
                                                   float* __restrict__ pool, __nv_bfloat16* __restrict__ poolh,
                                                   int* __restrict__ amax) {
    __shared__ float s_sum[8][WIDTH], s_best[8][WIDTH];
    __shared__ int s_arg[8][WIDTH];
    const int c8 = (threadIdx.x & 31) * 8, g = threadIdx.x >> 5, c = threadIdx.x;
    for (int b = blockIdx.x; b < Bp; b += gridDim.x) {
        if (b >= B) {
            poolh[(size_t)b * 2 * WIDTH + c] = __float2bfloat16_rn(0.0f);
            poolh[(size_t)b * 2 * WIDTH + WIDTH + c] = __float2bfloat16_rn(0.0f);
            continue;
        }
        const int nv = nvalid[b];
        float sum[8], best[8];
        int arg[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            sum[j] = 0.0f;
            best[j] = 0.0f;
            arg[j] = -1;
        }
#pragma unroll 4
        for (int e = g; e < nv; e += 8) {
            uint4 v = *reinterpret_cast<const uint4*>(H3 + ((size_t)b * KSET + e) * WIDTH + c8);
            const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float h = bf(hv[j]);
                sum[j] += h;
                if (arg[j] < 0 || h > best[j]) {
                    best[j] = h;
                    arg[j] = e;
                }
            }
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            s_sum[g][c8 + j] = sum[j];
            s_best[g][c8 + j] = best[j];
            s_arg[g][c8 + j] = arg[j];
        }
        __syncthreads();
        float tsum = 0.0f, tbest = 0.0f;
        int targ = -1;
        for (int q = 0; q < 8; ++q) {
            tsum += s_sum[q][c];
            const int aq = s_arg[q][c];
            const float bq = s_best[q][c];
            if (aq >= 0 && (targ < 0 || bq > tbest || (bq == tbest && aq < targ))) {
                tbest = bq;
                targ = aq;
            }
        }
        const float mean = nv > 0 ? tsum / (float)nv : 0.0f, mx = nv > 0 ? tbest : 0.0f;
        pool[(size_t)b * 2 * WIDTH + c] = mean;
        pool[(size_t)b * 2 * WIDTH + WIDTH + c] = mx;
        poolh[(size_t)b * 2 * WIDTH + c] = __float2bfloat16_rn(mean);
        poolh[(size_t)b * 2 * WIDTH + WIDTH + c] = __float2bfloat16_rn(mx);
        amax[(size_t)b * WIDTH + c] = targ < 0 ? 0 : targ;
        __syncthreads();
    }
}

// head output O[b][j] = Opad[b][j] + b5[j] (j < NOUT) for the B real sets
__global__ void head_out_kernel(const float* Opad, const float* b5, int B, float* O) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * NOUT) return;
    int b = idx / NOUT, j = idx % NOUT;
    O[idx] = Opad[(size_t)b * NOUTP + j] + b5[j];
}

// dL/dO rounded to BF16 into the zero-padded [Bp][NOUTP] operand of the
// head's backward GEMMs
__global__ void pack_dO_kernel(const float* dO, int B, int Bp, __nv_bfloat16* dOh) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Bp * NOUTP) return;
    int b = idx / NOUTP, j = idx % NOUTP;
    dOh[idx] = __float2bfloat16_rn(b < B && j < NOUT ? dO[(size_t)b * NOUT + j] : 0.0f);
}

// column sums out[n] = sum_m A[m lda + n]: per z-slice partial sums over a
// row range, then the slices added in order
__global__ void colsum_partial_kernel(const float* A, long long lda, int M, int N, int splits, float* part) {
    int n = blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    int mc = (M + splits - 1) / splits, m0 = blockIdx.y * mc, m1 = min(M, m0 + mc);
    float s = 0.0f;
    for (int m = m0; m < m1; ++m) s += A[m * lda + n];
    part[(size_t)blockIdx.y * N + n] = s;
}

// column sums of a BF16 [rows][256] array (the bias gradients sum_m dZ[m][c]):
// blockIdx.x takes rows [x rc, (x+1) rc); thread t adds channels 8 (t % 32)
// .. + 7 of the rows t / 32, t / 32 + 8, ... (four 16-byte loads in flight),
// then the eight row groups are added in order; one partial per (block,
// channel) in part[block][256], added in order by reduce_partials.
constexpr int kColsumSplits = 1024;
__global__ void __launch_bounds__(256) colsum_bf16_kernel(const __nv_bfloat16* A, long long rows, float* part) {
    __shared__ float red[8][WIDTH];
    const int c8 = (threadIdx.x & 31) * 8, g = threadIdx.x >> 5;
    const long long rc = (rows + gridDim.x - 1) / gridDim.x;
    const long long r0 = (long long)blockIdx.x * rc, r1 = min(rows, r0 + rc);
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    long long r = r0 + g;
    for (; r + 24 < r1; r += 32) {
        uint4 v[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) v[u] = *reinterpret_cast<const uint4*>(A + (size_t)(r + 8 * u) * WIDTH + c8);
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&v[u]);
#pragma unroll
            for (int j = 0; j < 8; ++j) acc[j] += bf(hv[j]);
        }
    }
    for (; r < r1; r += 8) {
        uint4 v = *reinterpret_cast<const uint4*>(A + (size_t)r * WIDTH + c8);
        const __nv_bfloat16* hv = reinterpret_cast<const __nv_bfloat16*>(&v);
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[j] += bf(hv[j]);
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[g][c8 + j] = acc[j];
    __syncthreads();
    float t = 0.0f;
    for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
    part[(size_t)blockIdx.x * WIDTH + threadIdx.x] = t;
}

// out[j] = sum_s part[s n + j] for many partials and few outputs: block x
// takes outputs 32 x .. + 31; warp w adds the partials s = w, w + 32, ...
// of output 32 x + lane, then the 32 warp sums are added in order.
constexpr int kReduceThreads = 1024;
__global__ void __launch_bounds__(kReduceThreads) reduce_partials_kernel(const float* __restrict__ part, int splits,
                                                                         int n, float* __restrict__ out) {
    constexpr int W = kReduceThreads / 32;
    __shared__ float red[W][32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, j = blockIdx.x * 32 + lane;
    float t = 0.0f;
    if (j < n)
#pragma unroll 8
        for (int q = w; q < splits; q += W) t += part[(size_t)q * n + j];
    red[w][lane] = t;
    __syncthreads();
    if (w == 0 && j < n) {
        float r = 0.0f;
        for (int q = 0; q < W; ++q) r += red[q][lane];
        out[j] = r;
    }
}

// sum of split-K partials: out[j] = sum_s part[s stride + j], j < n
__global__ void split_reduce_kernel(const float* part, int splits, long long stride, long long n, float* out) {
    long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float s = 0.0f;
    for (int q = 0; q < splits; ++q) s += part[(size_t)q * stride + j];
    out[j] = s;
}

__global__ void count_valid_kernel(const float* svalid, int B, float* inv_nval) {
    __shared__ float red[256];
    float s = 0.0f;
    for (int b = threadIdx.x; b < B; b += blockDim.x) s += svalid[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) inv_nval[0] = 1.0f / fmaxf(red[0], 1.0f);
}

// The 24 proper rotations of the cube, S[r][perm[r]] = sign[r], in the order
// permutations of (0, 1, 2) (lexicographic) x sign triples (+ before -, last
// index fastest), kept when det = +1.  Stored per symmetry and column c as the
// row that holds column c's nonzero and its sign.
__constant__ signed char c_sym_row[24][3] = {
    {0, 1, 2}, {0, 1, 2}, {0, 1, 2}, {0, 1, 2}, {0, 2, 1}, {0, 2, 1},
    {0, 2, 1}, {0, 2, 1}, {1, 0, 2}, {1, 0, 2}, {1, 0, 2}, {1, 0, 2},
    {2, 0, 1}, {2, 0, 1}, {2, 0, 1}, {2, 0, 1}, {1, 2, 0}, {1, 2, 0},
    {1, 2, 0}, {1, 2, 0}, {2, 1, 0}, {2, 1, 0}, {2, 1, 0}, {2, 1, 0}};
__constant__ signed char c_sym_sgn[24][3] = {
    {1, 1, 1}, {1, -1, -1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, 1}, {1, 1, -1},
    {-1, 1, 1}, {-1, -1, -1}, {1, 1, -1}, {-1, 1, 1}, {1, -1, 1}, {-1, -1, -1},
    {1, 1, 1}, {-1, 1, -1}, {-1, -1, 1}, {1, -1, -1}, {1, 1, 1}, {-1, -1, 1},
    {1, -1, -1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, 1}, {1, 1, -1}, {-1, -1, -1}};

__device__ void gram_schmidt(const float* o, float* R) {  // R row-major, columns e1 e2 e3
    float na = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
    float e1[3] = {o[0] / na, o[1] / na, o[2] / na};
    float eb = e1[0] * o[3] + e1[1] * o[4] + e1[2] * o[5];
    float bp[3] = {o[3] - eb * e1[0], o[4] - eb * e1[1], o[5] - eb * e1[2]};
    float nb = sqrtf(bp[0] * bp[0] + bp[1] * bp[1] + bp[2] * bp[2]);
    float e2[3] = {bp[0] / nb, bp[1] / nb, bp[2] / nb};
    float e3[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    for (int r = 0; r < 3; ++r) {
        R[3 * r] = e1[r];
        R[3 * r + 1] = e2[r];
        R[3 * r + 2] = e3[r];
    }
}

__device__ void gram_schmidt_backward(const float* o, const float* dR, float* d6) {
    float na = sqrtf(o[0] * o[0] + o[1] * o[1] + o[2] * o[2]);
    float e1[3] = {o[0] / na, o[1] / na, o[2] / na};
    float eb = e1[0] * o[3] + e1[1] * o[4] + e1[2] * o[5];
    float bp[3] = {o[3] - eb * e1[0], o[4] - eb * e1[1], o[5] - eb * e1[2]};
    float nb = sqrtf(bp[0] * bp[0] + bp[1] * bp[1] + bp[2] * bp[2]);
    float e2[3] = {bp[0] / nb, bp[1] / nb, bp[2] / nb};
    float de1[3], de2[3], de3[3];
    for (int r = 0; r < 3; ++r) {
        de1[r] = dR[3 * r];
        de2[r] = dR[3 * r + 1];
        de3[r] = dR[3 * r + 2];
    }
    // e3 = e1 x e2
    de1[0] += e2[1] * de3[2] - e2[2] * de3[1];
    de1[1] += e2[2] * de3[0] - e2[0] * de3[2];
    de1[2] += e2[0] * de3[1] - e2[1] * de3[0];
    de2[0] += de3[1] * e1[2] - de3[2] * e1[1];
    de2[1] += de3[2] * e1[0] - de3[0] * e1[2];
    de2[2] += de3[0] * e1[1] - de3[1] * e1[0];
    float pe = de2[0] * e2[0] + de2[1] * e2[1] + de2[2] * e2[2];
    float dbp[3] = {(de2[0] - pe * e2[0]) / nb, (de2[1] - pe * e2[1]) / nb, (de2[2] - pe * e2[2]) / nb};
    float q = e1[0] * dbp[0] + e1[1] * dbp[1] + e1[2] * dbp[2];
    for (int r = 0; r < 3; ++r) {
        d6[3 + r] = dbp[r] - q * e1[r];
        de1[r] = de1[r] - eb * dbp[r] - q * o[3 + r];
    }
    float p1 = de1[0] * e1[0] + de1[1] * e1[1] + de1[2] * e1[2];
    for (int r = 0; r < 3; ++r) d6[r] = (de1[r] - p1 * e1[r]) / na;
}

// per set: min over hypotheses of the symmetric rotation error + position
// term, plus BETA times their mean; gradient of the batch mean
__global__ void loss_kernel(const float* O, const float* Rt, const float* xt, const float* svalid,
                            const float* inv_nval, int B, float* dO, float* loss, float* dbest, int* hbest) {
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    float* g = dO + (size_t)b * NOUT;
    if (!(svalid[b] > 0.0f)) {
        for (int q = 0; q < NOUT; ++q) g[q] = 0.0f;
        loss[b] = 0.0f;
        dbest[b] = 0.0f;
        hbest[b] = -1;
        return;
    }
    const float* T = Rt + 9 * (size_t)b;
    const float* xv = xt + 3 * (size_t)b;
    float L[NHYP], dd[NHYP];
    int sb[NHYP];
    for (int h = 0; h < NHYP; ++h) {
        const float* o = O + (size_t)b * NOUT + 9 * h;
        float R[9];
        gram_schmidt(o, R);
        float G[9];  // G[c][k] = sum_i R[i][c] T[i][k]
        for (int c = 0; c < 3; ++c)
            for (int k = 0; k < 3; ++k) G[3 * c + k] = R[c] * T[k] + R[3 + c] * T[3 + k] + R[6 + c] * T[6 + k];
        float best = -1e30f;
        int bs = 0;
        for (int s = 0; s < 24; ++s) {
            float tr = 0.0f;
            for (int c = 0; c < 3; ++c) tr += (float)c_sym_sgn[s][c] * G[3 * c + c_sym_row[s][c]];
            if (tr > best) {
                best = tr;
                bs = s;
            }
        }
        float dx0 = o[6] - xv[0], dx1 = o[7] - xv[1], dx2 = o[8] - xv[2];
        dd[h] = 6.0f - 2.0f * best;
        L[h] = dd[h] + LAMBDA_X * (dx0 * dx0 + dx1 * dx1 + dx2 * dx2);
        sb[h] = bs;
    }
    int hb = 0;
    float mean = 0.0f;
    for (int h = 0; h < NHYP; ++h) {
        mean += L[h];
        if (L[h] < L[hb]) hb = h;
    }
    mean /= (float)NHYP;
    loss[b] = L[hb] + BETA * mean;
    dbest[b] = dd[hb];
    hbest[b] = hb;
    float inv = inv_nval[0];
    for (int h = 0; h < NHYP; ++h) {
        const float* o = O + (size_t)b * NOUT + 9 * h;
        float coef = ((h == hb ? 1.0f : 0.0f) + BETA / (float)NHYP) * inv;
        float R[9], dR[9];
        gram_schmidt(o, R);
        int s = sb[h];
        for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) {
                float ts = (float)c_sym_sgn[s][c] * T[3 * r + c_sym_row[s][c]];
                dR[3 * r + c] = 2.0f * coef * (R[3 * r + c] - ts);
            }
        float d6[6];
        gram_schmidt_backward(o, dR, d6);
        float* gh = g + 9 * h;
        for (int q = 0; q < 6; ++q) gh[q] = d6[q];
        for (int q = 0; q < 3; ++q) gh[6 + q] = 2.0f * LAMBDA_X * coef * (o[6 + q] - xv[q]);
    }
}

// dZ3 = (dmean / nv on valid rows + dmax at the argmax row) where H3 > 0,
// rounded to BF16, row-major.  A CTA takes the sets b = x, x + gridDim.x,
// ...; each thread handles 8 channels of a row with 16-byte loads and
// stores.  The column sums of the CTA's rounded dZ3 rows (its share of the
// bias gradient of layer 3) go to part[x][256], the sets and the eight row
// groups added in order.
constexpr int kPoolBwdBlocks = 1024;
__global__ void __launch_bounds__(256) pool_backward_kernel(const __nv_bfloat16* __restrict__ H3,
                                                            const int* __restrict__ nvalid,
                                                            const int* __restrict__ amax,
                                                            const float* __restrict__ dPool, int B,
                                                            __nv_bfloat16* __restrict__ dZ3,
                                                            float* __restrict__ part) {
    __shared__ float dm_s[WIDTH], dx_s[WIDTH];
    __shared__ int am_s[WIDTH];
    __shared__ float red[8][WIDTH];
    const int c8 = (threadIdx.x & 31) * 8, r0 = threadIdx.x >> 5;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    for (int b = blockIdx.x; b < B; b += gridDim.x) {
        const int nv = nvalid[b];
        for (int c = threadIdx.x; c < WIDTH; c += blockDim.x) {
            dm_s[c] = nv > 0 ? dPool[(size_t)b * 2 * WIDTH + c] / (float)nv : 0.0f;
            dx_s[c] = nv > 0 ? dPool[(size_t)b * 2 * WIDTH + WIDTH + c] : 0.0f;
            am_s[c] = amax[(size_t)b * WIDTH + c];
        }
        __syncthreads();
        // this thread's 8 channels: the per-set constants in registers
        float dm[8], dx[8];
        int am[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            dm[j] = dm_s[c8 + j];
            dx[j] = dx_s[c8 + j];
            am[j] = am_s[c8 + j];
        }
#pragma unroll 4
        for (int e = r0; e < KSET; e += 8) {
            const size_t row = (size_t)b * KSET + e;
            uint4 hv = *reinterpret_cast<const uint4*>(H3 + row * WIDTH + c8);
            const __nv_bfloat16* hh = reinterpret_cast<const __nv_bfloat16*>(&hv);
            __align__(16) __nv_bfloat16 z[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float v = (e < nv ? dm[j] : 0.0f) + (e == am[j] ? dx[j] : 0.0f);
                z[j] = __float2bfloat16_rn(bf(hh[j]) > 0.0f ? v : 0.0f);
                acc[j] += bf(z[j]);
            }
            *reinterpret_cast<uint4*>(dZ3 + row * WIDTH + c8) = *reinterpret_cast<const uint4*>(z);
        }
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[r0][c8 + j] = acc[j];
    __syncthreads();
    float t = 0.0f;
    for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
    part[(size_t)blockIdx.x * WIDTH + threadIdx.x] = t;
}

__global__ void adam_kernel(float* p, float* m, float* v, const float* g, long long n, const int* step, float lr,
                            float b1, float b2, float eps) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float t = (float)(step[0] + 1);
    float gi = g[i];
    float mi = b1 * m[i] + (1.0f - b1) * gi;
    float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    float mh = mi / (1.0f - powf(b1, t)), vh = vi / (1.0f - powf(b2, t));
    p[i] -= lr * mh / (sqrtf(vh) + eps);
}

__global__ void step_kernel(int* step) {
    if (threadIdx.x == 0 && blockIdx.x == 0) step[0] += 1;
}

// BF16 copies of the weights: W1h, W2h, W3h, W4h row-major [out][in], W2t,
// W3t transposed [in][out], W5h row-major with rows NOUT .. NOUTP - 1 zero
constexpr int kRefreshThreads = HEADW * 2 * WIDTH;  // the largest copy (W4)
__global__ void refresh_bf16_kernel(const float* P, __nv_bfloat16* W1h, __nv_bfloat16* W2h, __nv_bfloat16* W3h,
                                    __nv_bfloat16* W2t, __nv_bfloat16* W3t, __nv_bfloat16* W4h,
                                    __nv_bfloat16* W5h) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < WIDTH * NF) W1h[i] = __float2bfloat16_rn(P[oW1 + i]);
    if (i < WIDTH * WIDTH) {
        int o = i / WIDTH, n = i % WIDTH;
        W2h[i] = __float2bfloat16_rn(P[oW2 + i]);
        W3h[i] = __float2bfloat16_rn(P[oW3 + i]);
        W2t[(size_t)n * WIDTH + o] = __float2bfloat16_rn(P[oW2 + i]);
        W3t[(size_t)n * WIDTH + o] = __float2bfloat16_rn(P[oW3 + i]);
    }
    if (i < HEADW * 2 * WIDTH) W4h[i] = __float2bfloat16_rn(P[oW4 + i]);
    if (i < NOUTP * HEADW) W5h[i] = __float2bfloat16_rn(i < NOUT * HEADW ? P[oW5 + i] : 0.0f);
}

// proposals: R = F0 GS(o_h), x = XSCALE o_h[6:9]
__global__ void decode_kernel(const float* O, const float* F, const int* nvalid, int B, float* Rout, float* xout) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= B * NHYP) return;
    int b = idx / NHYP;
    const float* o = O + (size_t)b * NOUT + 9 * (idx % NHYP);
    float Rh[9];
    gram_schmidt(o, Rh);
    const float* F0 = F + 9 * (size_t)b;
    for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c)
            Rout[9 * (size_t)idx + 3 * r + c] =
                nvalid[b] > 0 ? F0[3 * r] * Rh[c] + F0[3 * r + 1] * Rh[3 + c] + F0[3 * r + 2] * Rh[6 + c]
                              : (r == c ? 1.0f : 0.0f);
    for (int q = 0; q < 3; ++q) xout[3 * (size_t)idx + q] = nvalid[b] > 0 ? XSCALE * o[6 + q] : 0.0f;
}

// split-K count of the head's weight gradients (K = Bp rows): the largest
// power of two <= 8 dividing Bp / 64
int head_splits(int Bp) {
    int kb = Bp / 64, s = 1;
    while (s * 2 <= 8 && kb % (s * 2) == 0) s *= 2;
    return s;
}

int splits_for(int B) {
    // K = B KSET rows = B KSET / 64 blocks of 64; the largest power of two <= 128 dividing them
    long long kb = (long long)B * KSET / 64;
    int s = 1;
    while (s * 2 <= kMaxSplits && kb % (s * 2) == 0) s *= 2;
    return s;
}

struct Net {
    float *P, *m, *v, *G, *part;
    __nv_bfloat16 *W1h, *W2h, *W3h, *W2t, *W3t, *W4h, *W5h;
    int* step;
};
Net net_view(void* base) {
    NetLayout L = net_layout();
    char* c = (char*)base;
    Net n;
    n.P = (float*)(c + L.params);
    n.m = (float*)(c + L.adam_m);
    n.v = (float*)(c + L.adam_v);
    n.G = (float*)(c + L.grads);
    n.part = (float*)(c + L.partial);
    n.W1h = (__nv_bfloat16*)(c + L.W1h);
    n.W2h = (__nv_bfloat16*)(c + L.W2h);
    n.W3h = (__nv_bfloat16*)(c + L.W3h);
    n.W2t = (__nv_bfloat16*)(c + L.W2t);
    n.W3t = (__nv_bfloat16*)(c + L.W3t);
    n.W4h = (__nv_bfloat16*)(c + L.W4h);
    n.W5h = (__nv_bfloat16*)(c + L.W5h);
    n.step = (int*)(c + L.step);
    return n;
}

struct Batch {
    BatchLayout L;
    char* c;
    template <class T>
    T* at(size_t off) const {
        return (T*)(c + off);
    }
};

cudaError_t forward_run(const Net& n, const Batch& bt, int B, int* ctrl, cudaStream_t s) {
    const BatchLayout& L = bt.L;
    long long Ms = L.Ms;
    auto bfp = [&](size_t off) { return bt.at<__nv_bfloat16>(off); };
    GemmArgs g{};
    g.M = (int)Ms;
    g.N = WIDTH;
    g.BN = WIDTH;
    g.mode = 1;
    g.ctrl = ctrl;
    cudaError_t e;
    // layer 1: X (K = 64)
    g.K = NF;
    g.bias = n.P + ob1;
    g.Dh = bfp(L.H1);
    if ((e = gemm_tc_run(GemmOperands{bfp(L.X), n.W1h, NF, NF}, g, 1, s)) != cudaSuccess) return e;
    g.K = WIDTH;
    g.bias = n.P + ob2;
    g.Dh = bfp(L.H2);
    if ((e = gemm_tc_run(GemmOperands{bfp(L.H1), n.W2h, WIDTH, WIDTH}, g, 1, s)) != cudaSuccess) return e;
    g.bias = n.P + ob3;
    g.Dh = bfp(L.H3);
    if ((e = gemm_tc_run(GemmOperands{bfp(L.H2), n.W3h, WIDTH, WIDTH}, g, 1, s)) != cudaSuccess) return e;
    const int Bp = L.Bp;
    pool_kernel<<<Bp, 256, 0, s>>>(bfp(L.H3), bt.at<int>(L.nvalid), B, Bp, bt.at<float>(L.pool), bfp(L.poolh),
                                     bt.at<int>(L.amax));
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // head on the tensor cores: H4 = relu(pool W4^T + b4) (BF16), O = H4 W5^T + b5
    GemmArgs hg{};
    hg.M = Bp;
    hg.N = HEADW;
    hg.K = 2 * WIDTH;
    hg.BN = 256;
    hg.mode = 1;
    hg.bias = n.P + ob4;
    hg.Dh = bfp(L.H4h);
    hg.ctrl = ctrl;
    if ((e = gemm_tc_run(GemmOperands{bfp(L.poolh), n.W4h, 2 * WIDTH, 2 * WIDTH}, hg, 1, s)) != cudaSuccess) return e;
    GemmArgs og{};
    og.M = Bp;
    og.N = NOUTP;
    og.K = HEADW;
    og.BN = NOUTP;
    og.mode = 0;
    og.Df = bt.at<float>(L.Opad);
    og.ctrl = ctrl;
    if ((e = gemm_tc_run(GemmOperands{bfp(L.H4h), n.W5h, HEADW, HEADW}, og, 1, s)) != cudaSuccess) return e;
    head_out_kernel<<<(B * NOUT + 255) / 256, 256, 0, s>>>(bt.at<float>(L.Opad), n.P + ob5, B, bt.at<float>(L.O));
    return cudaGetLastError();
}

cudaError_t backward_run(const Net& n, const Batch& bt, int B, int* ctrl, cudaStream_t s) {
    const BatchLayout& L = bt.L;
    long long Ms = L.Ms;
    auto bfp = [&](size_t off) { return bt.at<__nv_bfloat16>(off); };
    cudaError_t e;
    float* dO = bt.at<float>(L.dO);
    const int Bp = L.Bp;
    const int hs = head_splits(Bp);
    // head, on the tensor cores with BF16 operands: dW5 = dO^T H4, db5 = sum dO,
    // dZ4 = (dO W5) * (H4 > 0), dW4 = dZ4^T pool, db4 = sum dZ4, dPool = dZ4 W4
    pack_dO_kernel<<<(Bp * NOUTP + 255) / 256, 256, 0, s>>>(dO, B, Bp, bfp(L.dOh));
    GemmArgs w5{};
    w5.M = NOUTP;
    w5.N = HEADW;
    w5.K = Bp;
    w5.BN = 256;
    w5.mode = 0;
    w5.Df = n.part;
    w5.ctrl = ctrl;
    w5.a_mn = 1;
    w5.b_mn = 1;
    if ((e = gemm_tc_run(GemmOperands{bfp(L.dOh), bfp(L.H4h), NOUTP, HEADW}, w5, hs, s))) return e;
    split_reduce_kernel<<<(NOUT * HEADW + 255) / 256, 256, 0, s>>>(n.part, hs, (long long)NOUTP * HEADW,
                                                                   (long long)NOUT * HEADW, n.G + oW5);
    colsum_partial_kernel<<<dim3(1, 32), NOUT, 0, s>>>(dO, NOUT, B, NOUT, 32, n.part);
    reduce_partials_kernel<<<(NOUT + 31) / 32, kReduceThreads, 0, s>>>(n.part, 32, NOUT, n.G + ob5);
    GemmArgs d4{};
    d4.M = Bp;
    d4.N = HEADW;
    d4.K = NOUTP;
    d4.BN = 256;
    d4.mode = 2;
    d4.mask = bfp(L.H4h);
    d4.Dh = bfp(L.dZ4h);
    d4.ctrl = ctrl;
    d4.b_mn = 1;  // W5 [out][hidden] is the [K][N] operand
    if ((e = gemm_tc_run(GemmOperands{bfp(L.dOh), n.W5h, NOUTP, HEADW}, d4, 1, s))) return e;
    GemmArgs w4{};
    w4.M = HEADW;
    w4.N = 2 * WIDTH;
    w4.K = Bp;
    w4.BN = 256;
    w4.mode = 0;
    w4.Df = n.part;
    w4.ctrl = ctrl;
    w4.a_mn = 1;
    w4.b_mn = 1;
    if ((e = gemm_tc_run(GemmOperands{bfp(L.dZ4h), bfp(L.poolh), HEADW, 2 * WIDTH}, w4, hs, s))) return e;
    split_reduce_kernel<<<(HEADW * 2 * WIDTH + 255) / 256, 256, 0, s>>>(n.part, hs, (long long)HEADW * 2 * WIDTH,
                                                                        (long long)HEADW * 2 * WIDTH, n.G + oW4);
    const int cs4 = Bp / 8 < kColsumSplits ? Bp / 8 : kColsumSplits;
    colsum_bf16_kernel<<<cs4, 256, 0, s>>>(bfp(L.dZ4h), Bp, n.part);
    reduce_partials_kernel<<<WIDTH / 32, kReduceThreads, 0, s>>>(n.part, cs4, WIDTH, n.G + ob4);
    GemmArgs dp{};
    dp.M = Bp;
    dp.N = 2 * WIDTH;
    dp.K = HEADW;
    dp.BN = 256;
    dp.mode = 0;
    dp.Df = bt.at<float>(L.dPool);
    dp.ctrl = ctrl;
    dp.b_mn = 1;  // W4 [hidden][pool] is the [K][N] operand
    if ((e = gemm_tc_run(GemmOperands{bfp(L.dZ4h), n.W4h, HEADW, 2 * WIDTH}, dp, 1, s))) return e;
    // pooling -> dZ3, with the bias gradient of layer 3 (per-set column sums)
    const int pb = B < kPoolBwdBlocks ? B : kPoolBwdBlocks;
    pool_backward_kernel<<<pb, 256, 0, s>>>(bfp(L.H3), bt.at<int>(L.nvalid), bt.at<int>(L.amax),
                                            bt.at<float>(L.dPool), B, bfp(L.dZ3), n.part);
    reduce_partials_kernel<<<WIDTH / 32, kReduceThreads, 0, s>>>(n.part, pb, WIDTH, n.G + ob3);
    if ((e = cudaGetLastError())) return e;
    // dZ2 = (dZ3 W3) * (H2 > 0), dZ1 = (dZ2 W2) * (H1 > 0)
    GemmArgs g{};
    g.M = (int)Ms;
    g.N = WIDTH;
    g.K = WIDTH;
    g.BN = WIDTH;
    g.mode = 2;
    g.ctrl = ctrl;
    g.mask = bfp(L.H2);
    g.Dh = bfp(L.dZ2);
    if ((e = gemm_tc_run(GemmOperands{bfp(L.dZ3), n.W3t, WIDTH, WIDTH}, g, 1, s))) return e;
    g.mask = bfp(L.H1);
    g.Dh = bfp(L.dZ1);
    if ((e = gemm_tc_run(GemmOperands{bfp(L.dZ2), n.W2t, WIDTH, WIDTH}, g, 1, s))) return e;
    // weight gradients dW_l = dZ_l^T H_{l-1}, split K over the spots: both
    // operands are the row-major [spots][channels] arrays, read MN-major
    int splits = splits_for(B);
    GemmArgs w{};
    w.M = WIDTH;
    w.K = (int)Ms;
    w.mode = 0;
    w.Df = n.part;
    w.ctrl = ctrl;
    w.a_mn = 1;
    w.b_mn = 1;
    struct {
        size_t A, Bop;
        int N, bn;
        size_t oW, ob;
    } layers[3] = {{L.dZ3, L.H2, WIDTH, WIDTH, oW3, ob3},
                   {L.dZ2, L.H1, WIDTH, WIDTH, oW2, ob2},
                   {L.dZ1, L.X, NF, NF, oW1, ob1}};
    for (int l = 0; l < 3; ++l) {
        w.N = layers[l].N;
        w.BN = layers[l].bn;
        if ((e = gemm_tc_run(GemmOperands{bfp(layers[l].A), bfp(layers[l].Bop), (uint64_t)WIDTH,
                                          (uint64_t)layers[l].N},
                             w, splits, s)))
            return e;
        long long nw = (long long)WIDTH * layers[l].N;
        split_reduce_kernel<<<(unsigned)((nw + 255) / 256), 256, 0, s>>>(n.part, splits, nw, nw,
                                                                          n.G + layers[l].oW);
        if (l == 0) continue;  // the bias gradient of layer 3 came with dZ3
        colsum_bf16_kernel<<<kColsumSplits, 256, 0, s>>>(bfp(layers[l].A), Ms, n.part);
        reduce_partials_kernel<<<WIDTH / 32, kReduceThreads, 0, s>>>(n.part, kColsumSplits, WIDTH, n.G + layers[l].ob);
        if ((e = cudaGetLastError())) return e;
    }
    return cudaSuccess;
}

}  // namespace
}  // namespace lp
}  // namespace laue

using namespace laue;
using namespace laue::lp;

extern "C" size_t laue_lp_param_count(void) { return kParams; }
extern "C" size_t laue_lp_set_size(void) { return KSET; }
extern "C" size_t laue_lp_net_bytes(void) { return net_layout().total; }
extern "C" size_t laue_lp_batch_bytes(int n_sets) { return n_sets > 0 ? batch_layout(n_sets).total : 0; }

extern "C" long long laue_lp_batch_offset(int n_sets, int region) {
    if (n_sets <= 0) return -1;
    BatchLayout L = batch_layout(n_sets);
    // region 1 (a transposed copy of X) is no longer kept: -1
    const size_t offs[] = {L.X, (size_t)-1, L.F, L.nvalid, L.Rt, L.xt, L.svalid, L.O, L.loss, L.dbest, L.hbest,
                           L.H1, L.H3, L.pool, L.dO, L.dZ3};
    if (region < 0 || region >= (int)(sizeof(offs) / sizeof(offs[0]))) return -1;
    return (long long)offs[region];
}

static int lp_need_ws(laue_handle* h) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    return LAUE_OK;
}

extern "C" int laue_lp_net_init(laue_handle* h, void* net, const float* params_host, void* stream) {
    int rc;
    if ((rc = lp_need_ws(h))) return rc;
    if (!net || !params_host) return laue_fail(h, LAUE_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    Net n = net_view(net);
    NetLayout L = net_layout();
    if ((rc = laue_cuda_check(h, cudaMemsetAsync(net, 0, L.total, s), "net clear"))) return rc;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(n.P, params_host, kParams * 4, cudaMemcpyHostToDevice, s),
                              "net params")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "net init"))) return rc;
    refresh_bf16_kernel<<<(kRefreshThreads + 255) / 256, 256, 0, s>>>(n.P, n.W1h, n.W2h, n.W3h, n.W2t, n.W3t,
                                                                       n.W4h, n.W5h);
    return laue_cuda_check(h, cudaGetLastError(), "net refresh");
}

extern "C" int laue_lp_net_params(laue_handle* h, const void* net, float* params_host, float* grads_host,
                                  void* stream) {
    if (!h || !net) return LAUE_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    Net n = net_view(const_cast<void*>(net));
    int rc;
    if (params_host &&
        (rc = laue_cuda_check(h, cudaMemcpyAsync(params_host, n.P, kParams * 4, cudaMemcpyDeviceToHost, s),
                              "read params")))
        return rc;
    if (grads_host &&
        (rc = laue_cuda_check(h, cudaMemcpyAsync(grads_host, n.G, kParams * 4, cudaMemcpyDeviceToHost, s),
                              "read grads")))
        return rc;
    return laue_cuda_check(h, cudaStreamSynchronize(s), "read net");
}

extern "C" int laue_lp_scene(laue_handle* h, const LaueGeometry* geom, const LaueLattice* lat, const float* omega,
                             int T, int W, int S, int Gmax, int gmin, int gmax, float cube_mm, float sigma_mm,
                             double outlier_ratio, unsigned long long seed, float* grainR, float* grainX,
                             int* scene_i32, int* I_off, float* omega_v, float* p, int* label, int capacity,
                             void* stream) {
    int rc;
    if ((rc = lp_need_ws(h))) return rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if (!lat || !lat->w_d0 || !lat->nharm || lat->M <= 0 || !omega || !grainR || !grainX || !scene_i32 || !I_off ||
        !omega_v || !p || !label)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "null argument");
    if (T < W || W <= 0 || S <= 0 || Gmax <= 0 || gmin < 0 || gmax > Gmax || gmin > gmax || capacity < 0 ||
        !(sigma_mm >= 0.0f) || !(outlier_ratio >= 0.0) || (uintptr_t)p % 16)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "scene sizes");
    if (lat->M > 65535) return laue_fail(h, LAUE_ERR_INVALID_ARG, "too many planes");
    for (int k = 0; k < geom->n_det; ++k)  // the scenes add noise and outliers in the detectors' x and y
        if (geom->det_normal[k][0] != 0.0f || geom->det_normal[k][1] != 0.0f)
            return laue_fail(h, LAUE_ERR_INVALID_ARG, "training scenes need detectors normal to z");
    SceneArgs a;
    a.G = laue_geom_dev(*geom);
    a.w_d0 = (const float4*)lat->w_d0;
    a.nharm = lat->nharm;
    a.M = lat->M;
    a.omega = omega;
    a.T = T;
    a.W = W;
    a.S = S;
    a.Gmax = Gmax;
    a.gmin = gmin;
    a.gmax = gmax;
    a.cube = cube_mm;
    a.sigma = sigma_mm;
    a.ratio = outlier_ratio;
    a.key = make_uint2((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
    a.R = grainR;
    a.x = grainX;
    a.n_g = scene_i32;
    a.t0 = scene_i32 + S;
    a.counts = scene_i32 + 2 * S;
    a.I_off = I_off;
    a.omega_v = omega_v;
    a.capacity = capacity;
    a.p = (float4*)p;
    a.label = label;
    a.ctrl = (int*)h->ws;
    cudaStream_t s = (cudaStream_t)stream;
    int ng = S * Gmax;
    scene_params_kernel<<<(ng + 255) / 256, 256, 0, s>>>(a);
    scene_count_kernel<<<S * W, 256, 0, s>>>(a);
    scene_scan_kernel<<<1, 1024, 0, s>>>(a);
    scene_write_kernel<<<S * W, 256, 0, s>>>(a);
    return laue_cuda_check(h, cudaGetLastError(), "scene launch");
}

extern "C" int laue_lp_scene_seeds(laue_handle* h, const int* I_off, const int* label, int W, int S, int per_scene,
                                   unsigned long long seed, int* seeds, int* wlo, int* whi, void* stream) {
    int rc;
    if ((rc = lp_need_ws(h))) return rc;
    if (!I_off || !label || !seeds || !wlo || !whi || W <= 0 || S <= 0 || per_scene <= 0)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "seeds arguments");
    int B = S * per_scene;
    uint2 key = make_uint2((uint32_t)(seed & 0xFFFFFFFFull), (uint32_t)(seed >> 32));
    scene_seeds_kernel<<<(B + 255) / 256, 256, 0, (cudaStream_t)stream>>>(I_off, label, W, S, per_scene, key, seeds,
                                                                          wlo, whi);
    return laue_cuda_check(h, cudaGetLastError(), "seeds launch");
}

extern "C" int laue_lp_sets(laue_handle* h, const LaueGeometry* geom, const float* p, const int* I_off,
                            const float* omega, int n_angles, int n_cap, const int* seeds, const int* wlo,
                            const int* whi, int n_sets, const int* label, const float* grainR, const float* grainX,
                            void* axes_scratch, void* batch, int* ids, void* stream) {
    int rc;
    if ((rc = lp_need_ws(h))) return rc;
    if ((rc = laue_check_geom(h, geom))) return rc;
    if (!p || !I_off || !omega || !seeds || !wlo || !whi || !axes_scratch || !batch || n_sets <= 0 ||
        n_angles <= 0 || n_cap < 0 || (label && (!grainR || !grainX)) || (uintptr_t)p % 16 ||
        (uintptr_t)axes_scratch % 16 || (uintptr_t)batch % 256)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "sets arguments");
    BatchLayout L = batch_layout(n_sets);
    Batch bt{L, (char*)batch};
    cudaStream_t s = (cudaStream_t)stream;
    GeomDev G = laue_geom_dev(*geom);
    if (n_cap > 0)
        axes_kernel<<<min((n_cap + 255) / 256, h->sm_count * 8), 256, 0, s>>>((const float4*)p, I_off, n_angles,
                                                                              omega, G, n_cap,
                                                                              (float4*)axes_scratch);
    SetsArgs a;
    a.p = (const float4*)p;
    a.axes = (const float4*)axes_scratch;
    a.I_off = I_off;
    a.omega = omega;
    a.n_angles = n_angles;
    a.seeds = seeds;
    a.wlo = wlo;
    a.whi = whi;
    a.B = n_sets;
    a.label = label;
    a.gR = grainR;
    a.gX = grainX;
    a.X = bt.at<__nv_bfloat16>(L.X);
    a.F = bt.at<float>(L.F);
    a.nvalid = bt.at<int>(L.nvalid);
    a.Rt = label ? bt.at<float>(L.Rt) : nullptr;
    a.xt = label ? bt.at<float>(L.xt) : nullptr;
    a.svalid = label ? bt.at<float>(L.svalid) : nullptr;
    a.ids = ids;
    a.ctrl = (int*)h->ws;
    sets_kernel<<<min(n_sets, h->sm_count * 8), kSetThreads, 0, s>>>(a);
    return laue_cuda_check(h, cudaGetLastError(), "sets launch");
}

extern "C" int laue_lp_forward(laue_handle* h, const void* net, void* batch, int n_sets, void* stream) {
    int rc;
    if ((rc = lp_need_ws(h))) return rc;
    if (!net || !batch || n_sets <= 0 || (uintptr_t)batch % 256 || (uintptr_t)net % 256)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "forward arguments");
    Batch bt{batch_layout(n_sets), (char*)batch};
    return laue_cuda_check(h, forward_run(net_view(const_cast<void*>(net)), bt, n_sets, (int*)h->ws,
                                          (cudaStream_t)stream),
                           "forward");
}

extern "C" int laue_lp_train_step(laue_handle* h, void* net, void* batch, int n_sets, float lr, void* stream) {
    int rc;
    if ((rc = lp_need_ws(h))) return rc;
    if (!net || !batch || n_sets <= 0 || !(lr >= 0.0f) || (uintptr_t)batch % 256 || (uintptr_t)net % 256)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "train arguments");
    cudaStream_t s = (cudaStream_t)stream;
    Net n = net_view(net);
    BatchLayout L = batch_layout(n_sets);
    Batch bt{L, (char*)batch};
    int* ctrl = (int*)h->ws;
    if ((rc = laue_cuda_check(h, forward_run(n, bt, n_sets, ctrl, s), "forward"))) return rc;
    count_valid_kernel<<<1, 256, 0, s>>>(bt.at<float>(L.svalid), n_sets, bt.at<float>(L.inv_nval));
    loss_kernel<<<(n_sets + 127) / 128, 128, 0, s>>>(bt.at<float>(L.O), bt.at<float>(L.Rt), bt.at<float>(L.xt),
                                                     bt.at<float>(L.svalid), bt.at<float>(L.inv_nval), n_sets,
                                                     bt.at<float>(L.dO), bt.at<float>(L.loss),
                                                     bt.at<float>(L.dbest), bt.at<int>(L.hbest));
    if ((rc = laue_cuda_check(h, cudaGetLastError(), "loss"))) return rc;
    if ((rc = laue_cuda_check(h, backward_run(n, bt, n_sets, ctrl, s), "backward"))) return rc;
    adam_kernel<<<(unsigned)((kParams + 255) / 256), 256, 0, s>>>(n.P, n.m, n.v, n.G, (long long)kParams, n.step,
                                                                  lr, 0.9f, 0.999f, 1e-8f);
    step_kernel<<<1, 32, 0, s>>>(n.step);
    refresh_bf16_kernel<<<(kRefreshThreads + 255) / 256, 256, 0, s>>>(n.P, n.W1h, n.W2h, n.W3h, n.W2t, n.W3t,
                                                                       n.W4h, n.W5h);
    return laue_cuda_check(h, cudaGetLastError(), "adam");
}

extern "C" int laue_lp_decode(laue_handle* h, const void* batch, int n_sets, float* R_out, float* x_out,
                              void* stream) {
    int rc;
    if ((rc = lp_need_ws(h))) return rc;
    if (!batch || n_sets <= 0 || !R_out || !x_out) return laue_fail(h, LAUE_ERR_INVALID_ARG, "decode arguments");
    BatchLayout L = batch_layout(n_sets);
    Batch bt{L, (char*)const_cast<void*>(batch)};
    int n = n_sets * NHYP;
    decode_kernel<<<(n + 255) / 256, 256, 0, (cudaStream_t)stream>>>(bt.at<float>(L.O), bt.at<float>(L.F),
                                                                     bt.at<int>(L.nvalid), n_sets, R_out, x_out);
    return laue_cuda_check(h, cudaGetLastError(), "decode");
}
