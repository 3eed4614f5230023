// common.cuh — device helpers and the workspace layout shared by the
// LaueOT kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/laueot.h"

namespace laue {

// ---------------------------------------------------------------------------
// status word / control block at the start of the workspace
// ---------------------------------------------------------------------------
enum CtrlSlot {
    CTRL_STATUS = 0,      // first device-side error code (0 = none)
    CTRL_ROW_NEXT = 1,    // tile queue head of the row pass
    CTRL_ROW_DONE = 2,    // finished-CTA ticket of the row pass
    CTRL_COL_NEXT = 3,
    CTRL_COL_DONE = 4,
    CTRL_N_ROW_TILES = 5, // tiles built by the scheduler
    CTRL_N_COL_TILES = 6,
    CTRL_FWD_TOTAL = 7,   // visible spots found by the forward pass
    CTRL_HRV_NEXT = 8,    // harvest passes
    CTRL_HRV_DONE = 9,
    CTRL_HCOL_NEXT = 10,
    CTRL_HCOL_DONE = 11,
    CTRL_GEN_NEXT = 12,   // generic queue / ticket pair for other passes
    CTRL_GEN_DONE = 13,
    CTRL_SF_NEXT = 14,    // single-grain fit start queue / ticket
    CTRL_SF_DONE = 15,
    CTRL_EXACT_ROWS = 16, // row / column log-sum-exps recomputed on the exact path
    CTRL_EXACT_COLS = 17,
    CTRL_SF_PAIRS = 18,   // 64-bit count (slots 18-19) of single-fit pair evaluations
    CTRL_SK_PAIRS = 20,   // 64-bit count (slots 20-21) of pair evaluations of the Sinkhorn passes
    CTRL_SP_DONE = 22,    // finished-CTA ticket of the sparse passes
    CTRL_MS_PAIRS = 24,   // 64-bit count (slots 24-25) of staged pairs the M-step pair kernel visits
    CTRL_SLOTS = 64
};

// single-grain fits: resident CTAs per SM, listed spots per start, cached row
// normalisers per angle block, scratch floats per listed spot ({-r, K} (4),
// centre (3), MM sums (3), tm, kd), scratch floats per near row ({p,
// normaliser} and the row's plan-weighted ray sum u) and the largest capacity
// of the near-row list (observed rows that carry plan mass in one EM step; the
// list holds min(n_obs, kSfNearMax) rows, sf_near_cap)
constexpr int kSfCtasPerSm = 6;
constexpr int kSfCap = 2048;
constexpr int kSfIcap = 4096;
constexpr int kSfSpotFloats = 12;
constexpr int kSfNearFloats = 8;
constexpr int kSfNearMax = 131072;
inline size_t sf_near_cap(int n_obs) {
    size_t c = n_obs < kSfNearMax ? (size_t)(n_obs > 0 ? n_obs : 1) : (size_t)kSfNearMax;
    return (c + 3) / 4 * 4;  // keeps every CTA's slice 16-byte aligned
}
constexpr int kConeGran = 32;  // pairs per cone granule of the pair passes' exact skipping (kGran)
constexpr size_t kCtrlBytes = 4096;  // status + counters + small scalars

// ---------------------------------------------------------------------------
// workspace layout (host computes, device receives pointers)
// ---------------------------------------------------------------------------
struct Layout {
    size_t ctrl;
    size_t row_tiles, col_tiles;  // int4 {t, start, count, pad}
    size_t row_part, col_part;    // float2 (max, sum) per tile, log2 domain
    size_t dust;                  // float: F0, F0n, G0, log2U, log2O, Fmax, Gmax (T each), errors
    size_t ang;                   // int4 per angle: tile ranges of the passes
    size_t obsX, obsY;            // pair-interleaved observed spots (see sinkhorn.cu)
    size_t modX, modY, modZ, modW;// pair-interleaved model spots
    size_t pairoff;               // int: I2_off[T+1], J2_off[T+1] (pair offsets), granule bases (2 x (T+1))
    size_t perm;                  // int: observed and model sort permutations (order -> caller, caller -> order)
    size_t sortbuf;               // sort keys and indices (two buffers each)
    size_t cone;                  // float4 + float per granule of 32 pairs, observed then model
    size_t fwd_blocks;            // int per forward block (count, then offset)
    size_t jsum;                  // float per model spot x 12 (M-step sums)
    size_t gsum;                  // float per grain x 16
    size_t gidx;                  // int: (t, grain) segment table
    size_t sfs;                   // float: per-CTA scratch of the single-grain fits
    size_t spot;                  // SPOT: counts, row pointers, flags, partials, best
    size_t total;
    int max_row_tiles, max_col_tiles, max_fwd_blocks;
    int max_obs_pairs, max_mod_pairs;
    int max_obs_gran, max_mod_gran;
};

constexpr int kMinTile = 64;      // smallest tile (in spot pairs) any launch shape uses
constexpr int kFwdBlock = 256;    // rays per forward block

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

inline Layout make_layout(const LaueProblemDims& d, int sm_count) {
    Layout L{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    int T = d.T > 0 ? d.T : 1;
    L.max_row_tiles = T + (d.n_obs / 2 + kMinTile - 1) / kMinTile + 1;
    L.max_col_tiles = T + (d.n_model / 2 + kMinTile - 1) / kMinTile + 1;
    long long rays = (long long)T * (d.n_grains > 0 ? d.n_grains : 1) * (d.n_planes > 0 ? d.n_planes : 1);
    L.max_fwd_blocks = (int)((rays + kFwdBlock - 1) / kFwdBlock) + 1;
    L.ctrl = take(kCtrlBytes);
    L.row_tiles = take(sizeof(int4) * (size_t)L.max_row_tiles);
    L.col_tiles = take(sizeof(int4) * (size_t)L.max_col_tiles);
    L.row_part = take(sizeof(float2) * (size_t)L.max_row_tiles);
    L.col_part = take(sizeof(float2) * (size_t)L.max_col_tiles);
    L.dust = take(sizeof(float) * (size_t)(8 * T + 16));
    L.ang = take(sizeof(int4) * (size_t)T);
    size_t ip = (size_t)(d.n_obs + T + 2) / 2 + 1, jp = (size_t)(d.n_model + T + 2) / 2 + 1;
    L.max_obs_pairs = (int)ip;
    L.max_mod_pairs = (int)jp;
    L.obsX = take(sizeof(float4) * ip);
    L.obsY = take(sizeof(float4) * ip);
    L.modX = take(sizeof(float4) * jp);
    L.modY = take(sizeof(float4) * jp);
    L.modZ = take(sizeof(float4) * jp);
    L.modW = take(sizeof(float4) * jp);
    L.pairoff = take(sizeof(int) * (size_t)(4 * T + 8));
    size_t nsp = (size_t)d.n_obs + d.n_model + 2;
    L.perm = take(sizeof(int) * 2 * nsp);
    L.sortbuf = take(sizeof(int) * 4 * nsp);
    L.max_obs_gran = (int)((ip + kConeGran - 1) / kConeGran) + T + 1;  // cone granules of kConeGran pairs
    L.max_mod_gran = (int)((jp + kConeGran - 1) / kConeGran) + T + 1;
    L.cone = take((sizeof(float4) + sizeof(float)) * (size_t)(L.max_obs_gran + L.max_mod_gran) + 64);
    L.fwd_blocks = take(sizeof(int) * (size_t)(2 * L.max_fwd_blocks + 2));
    L.jsum = take(sizeof(float) * 12 * (size_t)(d.n_model + 1));
    L.gsum = take(sizeof(float) * 16 * (size_t)(d.n_grains + 1));
    L.gidx = take(sizeof(int) * ((size_t)T * (d.n_grains + 1) + 16));
    // single-grain fits, per CTA (the slices of sf_slice in single.cu)
    size_t sf_ctas = d.n_starts > 0 ? (size_t)sm_count * kSfCtasPerSm : 0;
    L.sfs = take(sizeof(float) * ((size_t)kSfCap * kSfSpotFloats + kSfIcap + kSfNearFloats * sf_near_cap(d.n_obs)) *
                 sf_ctas);
    L.spot = take(d.n_candidates > 0 ? sizeof(int) * (4 * (size_t)d.n_candidates + 16 + 2 * (size_t)sm_count * 4 + 64) +
                                           sizeof(float) * (size_t)(d.n_obs + 1)
                                     : 0);
    L.total = off;
    return L;
}

// ---------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------
#ifdef __CUDACC__

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.6931471805599453f;
constexpr float kNegHuge = -3.0e38f;  // finite stand-in for log(0)

// Hardware approximations (PTX ISA: ex2.approx, lg2.approx, rsqrt.approx).
__device__ __forceinline__ float ex2(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float lg2(float x) {
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsq(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Record the first device-side error in the status word.
__device__ __forceinline__ void set_status(int* ctrl, int code) {
    atomicCAS(ctrl + CTRL_STATUS, 0, code);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// mbarrier + bulk async copy (TMA, non-tensor form).  Addresses and sizes of
// cp.async.bulk must be multiples of 16 bytes: every staged array here is
// float4 rows starting at 256-byte aligned bases.
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(smem_u32(bar)),
        "r"(bytes)
        : "memory");
}
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait on an mbarrier phase: gives up after `limit` polls (each poll
// may suspend the thread for a hardware-defined time) and returns false.
constexpr uint32_t kWaitLimit = 1u << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
    for (uint32_t it = 0; it < kWaitLimit; ++it)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

// Log-sum-exp (base 2) accumulator: value = m + log2(s).
struct Lse2 {
    float m, s;
    __device__ __forceinline__ void init(float v) {
        m = v;
        s = 1.0f;
    }
    __device__ __forceinline__ void merge(float m2, float s2) {
        if (s2 == 0.0f) return;
        if (m2 > m) {
            s = s * ex2(m - m2) + s2;
            m = m2;
        } else {
            s += s2 * ex2(m2 - m);
        }
    }
    __device__ __forceinline__ float value() const { return m + lg2(s); }
};

__device__ __forceinline__ void warp_lse_reduce(float& m, float& s) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        float m2 = __shfl_xor_sync(0xffffffffu, m, o);
        float s2 = __shfl_xor_sync(0xffffffffu, s, o);
        float mm = fmaxf(m, m2);
        s = (s == 0.0f ? 0.0f : s * ex2(m - mm)) + (s2 == 0.0f ? 0.0f : s2 * ex2(m2 - mm));
        m = mm;
    }
}

// Packed pairs of floats for the sm_100+ f32x2 instructions (PTX fma/add/
// mul .rn.f32x2): the low half is the first element.
typedef unsigned long long f2;
__device__ __forceinline__ f2 pk(float a, float b) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ f2 dup(float a) { return pk(a, a); }
__device__ __forceinline__ float lo(f2 v) {
    float a;
    asm("mov.b64 {%0, _}, %1;" : "=f"(a) : "l"(v));
    return a;
}
__device__ __forceinline__ float hi(f2 v) {
    float b;
    asm("mov.b64 {_, %0}, %1;" : "=f"(b) : "l"(v));
    return b;
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ float max3(float a, float b, float c) {
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

#endif  // __CUDACC__

// ---------------------------------------------------------------------------
// deterministic annealing (paper Section "Deterministic annealing"): the one
// temperature schedule of the library, shared by the host drivers and the
// single-grain fit kernel.  eps_k = eps_final * factor^(1 - k/K) for
// 0 <= k < K = ceil(0.75 n_em), then eps_final.  Computed in double so that
// every caller takes the same value.
// ---------------------------------------------------------------------------
__host__ __device__ inline double anneal_eps(double eps_final, int n_em, int k, double factor) {
    int K = (int)ceil(0.75 * (double)n_em);
    if (K < 1 || k >= K) return eps_final;
    return eps_final * pow(factor, 1.0 - (double)k / (double)K);
}

// Outlier cost: the pair cost of two unit rays 3 sigma apart,
// D^2 |a - b|^2 = 4 D^2 sin^2(1.5 sigma_mm / D) (sigma on the detector at
// distance D, read as the angle sigma_mm / D).
__host__ __device__ inline double outlier_cost(double sigma_mm, double D) {
    double s = sin(1.5 * sigma_mm / D);
    return 4.0 * D * D * s * s;
}

}  // namespace laue
