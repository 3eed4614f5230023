// grid.cu — start grid of the single-grain fits (paper Section "Single-grain
// fitting": quasi-uniform starts over orientations and positions, the
// orientations restricted by the crystal symmetry).
//
// Orientations: the super-Fibonacci spiral (Alexa, CVPR 2022), a published
// deterministic quasi-uniform sequence of unit quaternions.  With the cubic
// restriction only the spiral points that lie in the fundamental zone are
// kept, i.e. those whose scalar part is the largest |<q, g>| over the 24
// rotations g of the cubic group (q is then the member of its symmetry class
// nearest the identity).  The quaternion and the zone test are evaluated in
// double precision, one thread per spiral point; kept points are written in
// spiral order (per-block counts, one scan, then ordered writes).  Each kept
// orientation is paired with the k^3 cell centres of the sample cube.
#include "api_internal.h"

namespace laue {

constexpr int kGridBlock = 1024;

__device__ __forceinline__ void spiral_quat(long long i, long long n, double q[4]) {
    const double phi = 1.4142135623730950488, psi = 1.533751168755204288118041;
    const double two_pi = 6.283185307179586476925287;
    double s = (double)i + 0.5;
    double r = sqrt(s / (double)n), rr = sqrt(1.0 - s / (double)n);
    double sa, ca, sb, cb;
    sincos(two_pi * s / phi, &sa, &ca);
    sincos(two_pi * s / psi, &sb, &cb);
    q[0] = r * sa;
    q[1] = r * ca;
    q[2] = rr * sb;
    q[3] = rr * cb;
}

// |<q, g>| over the non-identity rotations of the cubic group, compared with
// |q_w| (the identity's): the 90-degree turns about the axes give
// |q_w +- q_a| / sqrt 2, the 180-degree turns |q_a| and |q_a +- q_b| / sqrt 2,
// the 120-degree turns |q_w +- q_x +- q_y +- q_z| / 2.
__device__ __forceinline__ bool in_cubic_zone(const double q[4]) {
    const double s = 0.70710678118654752440;
    double id = fabs(q[0]);
    for (int a = 1; a <= 3; ++a) {
        if (fabs(q[a]) > id) return false;
        if (s * fabs(q[0] + q[a]) > id || s * fabs(q[0] - q[a]) > id) return false;
        for (int b = a + 1; b <= 3; ++b)
            if (s * fabs(q[a] + q[b]) > id || s * fabs(q[a] - q[b]) > id) return false;
    }
    for (int m = 0; m < 8; ++m) {
        double d = q[0] + ((m & 1) ? -q[1] : q[1]) + ((m & 2) ? -q[2] : q[2]) + ((m & 4) ? -q[3] : q[3]);
        if (0.5 * fabs(d) > id) return false;
    }
    return true;
}

// The dihedral groups D_n (n = 3: trigonal 32, n = 6: hexagonal 622) with
// the n-fold axis along z and a 2-fold axis along x: turns by 2 pi m / n about
// z give |<q, g>| = |q_w cos(pi m/n) + q_z sin(pi m/n)|, the 2-fold turns
// about (cos phi, sin phi, 0), phi = pi m / n, give |q_x cos phi + q_y sin phi|.
__device__ __forceinline__ bool in_dihedral_zone(const double q[4], int n) {
    const double pi = 3.14159265358979323846;
    double id = fabs(q[0]);
    for (int m = 0; m < n; ++m) {
        double s, c;
        sincos(pi * m / n, &s, &c);
        if (m > 0 && fabs(q[0] * c + q[3] * s) > id) return false;
        if (fabs(q[1] * c + q[2] * s) > id) return false;
    }
    return true;
}

__device__ __forceinline__ bool grid_keep(long long i, long long n, int sym, double q[4]) {
    spiral_quat(i, n, q);
    if (sym == 24) return in_cubic_zone(q);
    if (sym == 6) return in_dihedral_zone(q, 3);
    if (sym == 12) return in_dihedral_zone(q, 6);
    return true;
}

__global__ void __launch_bounds__(kGridBlock) grid_count_kernel(long long n, int sym, int* counts) {
    long long i = (long long)blockIdx.x * kGridBlock + threadIdx.x;
    double q[4];
    bool k = i < n && grid_keep(i, n, sym, q);
    int c = __syncthreads_count(k);
    if (threadIdx.x == 0) counts[blockIdx.x] = c;
}

// exclusive scan of the block counts by one CTA; counts[nb] = total
__global__ void __launch_bounds__(1024) grid_scan_kernel(int* counts, int nb, long long* total) {
    __shared__ long long part[1024];
    int per = (nb + 1023) / 1024;
    int b0 = threadIdx.x * per, b1 = min(nb, b0 + per);
    long long s = 0;
    for (int b = b0; b < b1; ++b) s += counts[b];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        long long acc = 0;
        for (int k = 0; k < 1024; ++k) {
            long long v = part[k];
            part[k] = acc;
            acc += v;
        }
        *total = acc;
    }
    __syncthreads();
    long long acc = part[threadIdx.x];
    for (int b = b0; b < b1; ++b) {
        int c = counts[b];
        counts[b] = (int)acc;
        acc += c;
    }
}

__global__ void __launch_bounds__(kGridBlock) grid_write_kernel(long long n, int sym, int k, float cube,
                                                                const int* offsets, long long cap, float* R_out,
                                                                float* x_out) {
    __shared__ int wcnt[kGridBlock / 32];
    long long i = (long long)blockIdx.x * kGridBlock + threadIdx.x;
    double q[4];
    bool kp = i < n && grid_keep(i, n, sym, q);
    unsigned ball = __ballot_sync(0xffffffffu, kp);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) wcnt[w] = __popc(ball);
    __syncthreads();
    if (!kp) return;
    int before = 0;
    for (int v = 0; v < w; ++v) before += wcnt[v];
    long long rank = (long long)offsets[blockIdx.x] + before + __popc(ball & ((1u << lane) - 1u));
    double W = q[0], X = q[1], Y = q[2], Z = q[3];
    float R[9] = {(float)(1 - 2 * (Y * Y + Z * Z)), (float)(2 * (X * Y - W * Z)), (float)(2 * (X * Z + W * Y)),
                  (float)(2 * (X * Y + W * Z)), (float)(1 - 2 * (X * X + Z * Z)), (float)(2 * (Y * Z - W * X)),
                  (float)(2 * (X * Z - W * Y)), (float)(2 * (Y * Z + W * X)), (float)(1 - 2 * (X * X + Y * Y))};
    long long kk = (long long)k * k * k;
    for (long long p = 0; p < kk; ++p) {
        long long s = rank * kk + p;
        if (s >= cap) break;
        long long a = p / ((long long)k * k), b = (p / k) % k, c = p % k;
        for (int e = 0; e < 9; ++e) R_out[9 * s + e] = R[e];
        x_out[3 * s + 0] = (float)((a + 0.5) * (double)cube / k - (double)cube / 2);
        x_out[3 * s + 1] = (float)((b + 0.5) * (double)cube / k - (double)cube / 2);
        x_out[3 * s + 2] = (float)((c + 0.5) * (double)cube / k - (double)cube / 2);
    }
}

size_t start_grid_scratch_bytes(long long n_full) {
    long long nb = (n_full + kGridBlock - 1) / kGridBlock;
    return sizeof(int) * (size_t)(nb + 1) + 64;
}

cudaError_t start_grid_run(long long n_full, int sym, int k, float cube, long long cap, float* R_out, float* x_out,
                           void* scratch, long long* total_dev, cudaStream_t s) {
    int nb = (int)((n_full + kGridBlock - 1) / kGridBlock);
    int* counts = (int*)scratch;
    if (nb > 0) grid_count_kernel<<<nb, kGridBlock, 0, s>>>(n_full, sym, counts);
    grid_scan_kernel<<<1, 1024, 0, s>>>(counts, nb, total_dev);
    if (nb > 0 && cap > 0) grid_write_kernel<<<nb, kGridBlock, 0, s>>>(n_full, sym, k, cube, counts, cap, R_out, x_out);
    return cudaGetLastError();
}

}  // namespace laue

using namespace laue;

extern "C" int laue_start_grid(laue_handle* h, long long n_full, int sym, int k, float cube_mm, long long cap,
                               float* R_out, float* x_out, long long* S_host, void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (n_full < 0 || n_full > (1LL << 40) || (sym != 1 && sym != 6 && sym != 12 && sym != 24) || k < 1 || k > 64 ||
        !(cube_mm >= 0.0f) ||
        cap < 0 || (cap > 0 && (!R_out || !x_out)) || !S_host)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "start_grid: bad arguments");
    if ((n_full + kGridBlock - 1) / kGridBlock > 0x7fffffffLL)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "start_grid: n_full too large");
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    size_t need = kCtrlBytes + 256 + start_grid_scratch_bytes(n_full);
    if (need > h->ws_bytes)
        return laue_fail(h, LAUE_ERR_WORKSPACE, "start_grid: workspace of %zu bytes needed", need);
    cudaStream_t s = (cudaStream_t)stream;
    char* ws = (char*)h->ws;
    long long* total = (long long*)(ws + kCtrlBytes);
    void* scratch = ws + kCtrlBytes + 256;
    int rc;
    if ((rc = laue_cuda_check(h, start_grid_run(n_full, sym, k, cube_mm, cap, R_out, x_out, scratch, total, s),
                              "start_grid launch")))
        return rc;
    long long n_kept = 0;
    if ((rc = laue_cuda_check(h, cudaMemcpyAsync(&n_kept, total, sizeof(long long), cudaMemcpyDeviceToHost, s),
                              "start_grid count")))
        return rc;
    if ((rc = laue_cuda_check(h, cudaStreamSynchronize(s), "start_grid synchronise"))) return rc;
    *S_host = n_kept * (long long)k * k * k;
    return LAUE_OK;
}
