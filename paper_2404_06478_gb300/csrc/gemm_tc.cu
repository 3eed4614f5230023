// gemm_tc.cu — BF16 x BF16 -> FP32 GEMM on the fifth-generation tensor cores
// (tcgen05) for the per-spot layers of the set encoder, with the epilogues
// the encoder's forward and backward passes need fused in.
//
//   D[m][n] = sum_k A[m][k] B[n][k]
//
// Each operand is either K-contiguous (A[m][k], B[n][k]) or MN-contiguous
// (A stored as [k][m], B as [k][n]); the second form lets the weight
// gradients dW = dZ^T H read the activations and errors in the row-major
// layout the forward and backward layers write, with no transposed copies.
//
// One CTA computes one 128 x BN tile (BN = 64, 128 or 256) over a range of K
// (split-K along gridDim.z).  Warp 0, lane 0 streams 128 x 64 and BN x 64
// operand tiles into a two- or four-stage shared-memory ring with TMA
// (cp.async.bulk.tensor, 128-byte swizzle); warp 1, lane 0 issues
// tcgen05.mma (M = 128, N = BN, K = 16 per instruction) into a BN-column
// FP32 accumulator in tensor memory and releases each stage with
// tcgen05.commit; then all four warps read their 32 accumulator lanes with
// tcgen05.ld and run the epilogue:
//   mode 0: FP32 store of the split's partial product, D + split * M * N;
//   mode 1: relu(acc + bias[n]) rounded to BF16, stored row-major and/or
//           transposed (D^T[n][m], leading dimension ldt);
//   mode 2: acc * (mask[m][n] > 0) rounded to BF16, row-major and/or
//           transposed (the ReLU derivative of the back-propagated error).
// Every mbarrier wait is bounded; a wait that runs out records
// LAUE_ERR_TIMEOUT in the status word and the CTA finishes without hanging.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "api_internal.h"
#include "gemm_tc.h"

namespace laue {

namespace {

constexpr int kBM = 128;
constexpr int kBK = 64;  // one 128-byte swizzle row of BF16
constexpr int kThreads = 128;
constexpr uint32_t kAStage = kBM * kBK * 2;

// Shared-memory matrix descriptor of a K-major operand tile stored as rows of
// 128 bytes with the 128-byte swizzle (the layout TMA writes with
// CU_TENSOR_MAP_SWIZZLE_128B): 8-row core groups 1024 bytes apart (stride
// byte offset), leading byte offset unused by this layout, descriptor
// version 1 (bits 46-47), swizzle mode 2 (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_sw128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1u << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Shared-memory matrix descriptor of an MN-major operand tile with the
// 128-byte swizzle.  TMA writes each 64-element (128-byte) MN slice of the
// tile as kBK rows of 128 bytes, one row per k, slices kMnSlice bytes apart:
// 8-row (8 k) core groups 1024 bytes apart (stride byte offset) and the
// 64-element MN repeats kMnSlice bytes apart (leading byte offset).
constexpr uint32_t kMnSlice = 64u * kBK * 2;  // one 64-wide MN slice of a stage
__device__ __forceinline__ uint64_t sdesc_mn128(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((kMnSlice >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(1024u >> 4) << 32;
    d |= (uint64_t)1u << 46;
    d |= (uint64_t)2u << 61;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1),
// BF16 A and B (bits 7-9, 10-12 = 1), A and B major-ness (bits 15, 16:
// 0 K-major, 1 MN-major), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N, int a_mn = 0, int b_mn = 0) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(a_mn & 1) << 15) | ((uint32_t)(b_mn & 1) << 16) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* tm, int x, int y, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], "
        "[%4];" ::"r"(smem_u32(dst)),
        "l"((uint64_t)tm), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 accumulator columns of this thread's lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float* v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
                 : "memory");
}

// The 32 mask values (BF16, 64 bytes) of row m, columns n .. n + 31 (mode 2).
__device__ __forceinline__ void load_mask32(const GemmArgs& a, int m, int n, uint4* mk) {
    const uint4* p = reinterpret_cast<const uint4*>(a.mask + (size_t)m * a.N + n);
#pragma unroll
    for (int q = 0; q < 4; ++q) mk[q] = p[q];
}

// Epilogue arithmetic of 32 accumulator columns n .. n + 31 of one row:
// relu(acc + bias) (mode 1) or acc where the BF16 mask is > 0 (mode 2).
__device__ __forceinline__ void epilogue_math32(const GemmArgs& a, int n, float* v, const uint4* mk) {
    if (a.mode == 1) {
#pragma unroll
        for (int j = 0; j < 32; ++j) v[j] = fmaxf(v[j] + a.bias[n + j], 0.0f);
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 w = mk[q];
            uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                uint32_t lo = ws[h] & 0xFFFFu, hi = ws[h] >> 16;
                if (!(lo != 0u && (lo & 0x8000u) == 0u)) v[8 * q + 2 * h] = 0.0f;
                if (!(hi != 0u && (hi & 0x8000u) == 0u)) v[8 * q + 2 * h + 1] = 0.0f;
            }
        }
    }
}

__device__ __forceinline__ uint4 pack8(const float* v) {
    return make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]), pack_bf16(v[6], v[7]));
}

// Epilogue of 32 accumulator columns of row m with direct stores: four
// 16-byte stores into the row-major output, one BF16 per column into the
// transposed one.
__device__ __forceinline__ void epilogue32(const GemmArgs& a, int m, int n, float* v, const uint4* mk) {
    epilogue_math32(a, n, v, mk);
    if (a.Dh) {
        uint4* dst = reinterpret_cast<uint4*>(a.Dh + (size_t)m * a.N + n);
#pragma unroll
        for (int q = 0; q < 4; ++q) dst[q] = pack8(v + 8 * q);
    }
    if (a.DhT) {
#pragma unroll
        for (int j = 0; j < 32; ++j) a.DhT[(size_t)(n + j) * a.ldt + m] = __float2bfloat16_rn(v[j]);
    }
}

// kStages ring slots: 4 for long K ranges; 2 for K <= 256 (four k-blocks),
// which halves the shared memory so that two CTAs share an SM and one CTA's
// epilogue overlaps the other's loads.
template <int kStages>
__global__ void __launch_bounds__(kThreads, kStages == 2 ? 2 : 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, GemmArgs a) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kStages], empty[kStages], done;
    __shared__ uint32_t tmem_base_s;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sA = smem;
    uint8_t* sB = smem + kStages * kAStage;
    const int BN = a.BN;
    const uint32_t bStage = (uint32_t)BN * kBK * 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int kb0 = blockIdx.z * a.kb_per_split, nkb = a.kb_per_split;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&done, 1);
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"((uint32_t)BN)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kb = 0; kb < nkb; ++kb) {
            int s = kb % kStages;
            uint32_t ph = (uint32_t)(kb / kStages) & 1u;
            if (kb >= kStages && !mbar_wait_bounded(&empty[s], ph ^ 1u)) {
                set_status(a.ctrl, LAUE_ERR_TIMEOUT);
                break;
            }
            mbar_expect_tx(&full[s], kAStage + bStage);
            int kx = (kb0 + kb) * kBK;
            if (a.a_mn) {
                for (int j = 0; j < kBM / 64; ++j)
                    tma_load_2d(sA + s * kAStage + j * kMnSlice, &tmA, m0 + 64 * j, kx, &full[s]);
            } else {
                tma_load_2d(sA + s * kAStage, &tmA, kx, m0, &full[s]);
            }
            if (a.b_mn) {
                for (int j = 0; j < BN / 64; ++j)
                    tma_load_2d(sB + s * bStage + j * kMnSlice, &tmB, n0 + 64 * j, kx, &full[s]);
            } else {
                tma_load_2d(sB + s * bStage, &tmB, kx, n0, &full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer
        const uint32_t idesc = idesc_bf16(kBM, BN, a.a_mn, a.b_mn);
        for (int kb = 0; kb < nkb; ++kb) {
            int s = kb % kStages;
            uint32_t ph = (uint32_t)(kb / kStages) & 1u;
            if (!mbar_wait_bounded(&full[s], ph)) {
                set_status(a.ctrl, LAUE_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            uint32_t aBase = smem_u32(sA + s * kAStage), bBase = smem_u32(sB + s * bStage);
            // K = 16 per instruction: 32 bytes along a K-major row, or two
            // 8-row core groups (2048 bytes) of an MN-major slice
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k) {
                uint64_t ad = a.a_mn ? sdesc_mn128(aBase + 2048u * k) : sdesc_sw128(aBase + 32u * k);
                uint64_t bd = a.b_mn ? sdesc_mn128(bBase + 2048u * k) : sdesc_sw128(bBase + 32u * k);
                tc_mma(tmem, ad, bd, idesc, (kb > 0 || k > 0) ? 1u : 0u);
            }
            tc_commit(&empty[s]);
        }
        tc_commit(&done);
    }
    __syncwarp();

    // epilogue: thread (warp w, lane l) owns accumulator row 32 w + l
    bool ok = mbar_wait_bounded(&done, 0);
    if (!ok && lane == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
    tc_fence_after();
    const int row = warp * 32 + lane;
    const int m = m0 + row;
    for (int c0 = 0; c0 < BN; c0 += 32) {
        float v[32];
        tc_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
        const int n = n0 + c0;
        if (a.mode == 0) {
            float4* dst = reinterpret_cast<float4*>(a.Df + ((size_t)blockIdx.z * a.M + m) * a.N + n);
#pragma unroll
            for (int j = 0; j < 8; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            continue;
        }
        uint4 mk[4];
        if (a.mode == 2) load_mask32(a, m, n, mk);
        epilogue32(a, m, n, v, mk);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"((uint32_t)BN)
                     : "memory");
    }
}

// Persistent, warp-specialised form for the per-spot layers (N = 256,
// K = 64 KB, modes 1 and 2).  The 256 x K weight operand is loaded once per
// CTA and stays in shared memory; 128-row tiles of A stream through a
// four-stage ring; two 256-column FP32 accumulators fill all of tensor
// memory, so the epilogue of one tile runs while the next is multiplied.
// Warp 0 (one lane) loads, warp 1 (one lane) issues the MMAs, warps 2-9
// drain the accumulators: warp w reads tensor-memory lanes 32 (w % 4) ..
// + 31 (the lane quadrant its warp index allows), columns 128 ((w - 2) / 4)
// .. + 127.  In mode 2 each epilogue thread loads its row's 128 mask values
// for the tile before the first accumulator read, so the mask's DRAM latency
// is paid once per tile rather than once per 32 columns.  The row-major
// output goes out through a per-warp shared-memory slot of 32 rows x 32
// columns: a thread writes its row's 64 bytes there (16-byte units swizzled
// by row, conflict-free), then each store instruction of the warp writes 8
// rows x 64 contiguous bytes (full 32-byte sectors) instead of 32 rows x 16
// bytes (half sectors).
constexpr int kPEpiWarps = 8;
constexpr int kPThreads = 64 + 32 * kPEpiWarps;
constexpr int kPStages = 4;
constexpr uint32_t kBBlock = 256u * kBK * 2;  // one 64-wide k-block of the 256-row weight operand

template <int KB>
__global__ void __launch_bounds__(kPThreads, 1)
    gemm_tc_persistent_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                              GemmArgs a, int n_tiles) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t a_full[kPStages], a_empty[kPStages], b_full, acc_full[2], acc_empty[2];
    __shared__ uint32_t tmem_base_s;
    __shared__ __align__(16) uint4 out_slot[kPEpiWarps][32 * 4];
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint8_t* sB = smem;
    uint8_t* sA = smem + KB * kBBlock;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kPStages; ++s) {
            mbar_init(&a_full[s], 1);
            mbar_init(&a_empty[s], 1);
        }
        mbar_init(&b_full, 1);
        for (int b = 0; b < 2; ++b) {
            mbar_init(&acc_full[b], 1);
            mbar_init(&acc_empty[b], 32 * kPEpiWarps);
        }
        fence_mbar_init();
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base_s)),
                     "r"(512u)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_s;

    if (warp == 0 && lane == 0) {
        mbar_expect_tx(&b_full, KB * kBBlock);
        for (int kb = 0; kb < KB; ++kb) tma_load_2d(sB + kb * kBBlock, &tmB, kb * kBK, 0, &b_full);
        int g = 0;
        bool ok = true;
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
            for (int kb = 0; kb < KB; ++kb, ++g) {
                int s = g % kPStages;
                uint32_t ph = (uint32_t)(g / kPStages) & 1u;
                if (g >= kPStages && !mbar_wait_bounded(&a_empty[s], ph ^ 1u)) {
                    set_status(a.ctrl, LAUE_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                mbar_expect_tx(&a_full[s], kAStage);
                tma_load_2d(sA + s * kAStage, &tmA, kb * kBK, tile * kBM, &a_full[s]);
            }
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16(kBM, 256);
        bool ok = mbar_wait_bounded(&b_full, 0);
        if (!ok) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
        tc_fence_after();
        int g = 0, i = 0;
        for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++i) {
            int buf = i & 1, u = i >> 1;
            if (u >= 1 && !mbar_wait_bounded(&acc_empty[buf], (uint32_t)(u & 1) ^ 1u)) {
                set_status(a.ctrl, LAUE_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)buf * 256u;
            for (int kb = 0; kb < KB; ++kb, ++g) {
                int s = g % kPStages;
                uint32_t ph = (uint32_t)(g / kPStages) & 1u;
                if (!mbar_wait_bounded(&a_full[s], ph)) {
                    set_status(a.ctrl, LAUE_ERR_TIMEOUT);
                    ok = false;
                    break;
                }
                tc_fence_after();
                uint32_t aBase = smem_u32(sA + s * kAStage), bBase = smem_u32(sB + kb * kBBlock);
#pragma unroll
                for (int k = 0; k < kBK / 16; ++k)
                    tc_mma(d, sdesc_sw128(aBase + 32u * k), sdesc_sw128(bBase + 32u * k), idesc,
                           (kb > 0 || k > 0) ? 1u : 0u);
                tc_commit(&a_empty[s]);
            }
            tc_commit(&acc_full[buf]);
        }
    } else if (warp >= 2) {
        const int q = warp & 3;
        const int cbeg = 128 * ((warp - 2) >> 2);
        const int row = q * 32 + lane;
        int i = 0;
        for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x, ++i) {
            int buf = i & 1, u = i >> 1;
            const int m = tile * kBM + row;
            uint4 mk[4][4];
            if (a.mode == 2) {
#pragma unroll
                for (int c = 0; c < 4; ++c) load_mask32(a, m, cbeg + 32 * c, mk[c]);
            }
            if (!mbar_wait_bounded(&acc_full[buf], (uint32_t)(u & 1))) {
                if (lane == 0) set_status(a.ctrl, LAUE_ERR_TIMEOUT);
                break;
            }
            tc_fence_after();
            uint4* slot = out_slot[warp - 2];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                const int c0 = cbeg + 32 * c;
                float v[32];
                tc_ld32(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)buf * 256u + (uint32_t)c0, v);
                epilogue_math32(a, c0, v, mk[c]);
                if (a.DhT) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) a.DhT[(size_t)(c0 + j) * a.ldt + m] = __float2bfloat16_rn(v[j]);
                }
                if (a.Dh) {
                    // unit k of row r sits at slot[4 r + (k ^ ((r >> 1) & 3))]
#pragma unroll
                    for (int k = 0; k < 4; ++k) slot[4 * lane + (k ^ ((lane >> 1) & 3))] = pack8(v + 8 * k);
                    __syncwarp();
                    const int k = lane & 3;
#pragma unroll
                    for (int it = 0; it < 4; ++it) {
                        const int r = 8 * it + (lane >> 2);
                        uint4 w = slot[4 * r + (k ^ ((r >> 1) & 3))];
                        *reinterpret_cast<uint4*>(a.Dh + (size_t)(tile * kBM + q * 32 + r) * a.N + c0 + 8 * k) = w;
                    }
                    __syncwarp();
                }
            }
            tc_fence_before();
            mbar_arrive1(&acc_empty[buf]);
        }
    }
    __syncwarp();
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512u) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 lookup_encode() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
        return (PFN_cuTensorMapEncodeTiled_v12000)p;
    return nullptr;
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = lookup_encode();  // thread-safe one-time lookup
    return fn;
}

// 2-D BF16 tensor [rows][cols] with leading dimension ld (elements), box
// 64 columns x box_rows rows, 128-byte swizzle.
bool make_tmap(CUtensorMap* tm, const void* base, uint64_t rows, uint64_t cols, uint64_t ld, uint32_t box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)kBK, box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(tm, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

static int stages_for(int nkb) { return nkb <= 4 ? 2 : 4; }

size_t gemm_tc_smem(int BN, int stages) { return 1024 + (size_t)stages * (kAStage + (size_t)BN * kBK * 2); }

int gemm_tc_check(const GemmOperands& op, const GemmArgs& a, int splits) {
    if (!(a.BN == 64 || a.BN == 128 || a.BN == 256)) return LAUE_ERR_INVALID_ARG;
    if (a.M <= 0 || a.N <= 0 || a.K <= 0 || a.M % kBM || a.N % a.BN || a.K % kBK) return LAUE_ERR_INVALID_ARG;
    if (splits < 1 || (a.K / kBK) % splits) return LAUE_ERR_INVALID_ARG;
    if (op.lda < (uint64_t)(a.a_mn ? a.M : a.K) || op.ldb < (uint64_t)(a.b_mn ? a.N : a.K) || op.lda % 8 ||
        op.ldb % 8)
        return LAUE_ERR_INVALID_ARG;
    if (((uintptr_t)op.A | (uintptr_t)op.B) & 15) return LAUE_ERR_INVALID_ARG;
    if (a.mode == 0 && !a.Df) return LAUE_ERR_INVALID_ARG;
    if (a.mode == 1 && !a.bias) return LAUE_ERR_INVALID_ARG;
    if (a.mode == 2 && !a.mask) return LAUE_ERR_INVALID_ARG;
    if ((a.mode == 1 || a.mode == 2) && !a.Dh && !a.DhT) return LAUE_ERR_INVALID_ARG;
    if (a.mode < 0 || a.mode > 2 || (a.mode != 0 && splits != 1)) return LAUE_ERR_INVALID_ARG;
    if (a.DhT && a.ldt < a.M) return LAUE_ERR_INVALID_ARG;
    if ((a.Dh && ((uintptr_t)a.Dh & 15)) || (a.mask && ((uintptr_t)a.mask & 15)) ||
        (a.Df && ((uintptr_t)a.Df & 15)))
        return LAUE_ERR_INVALID_ARG;
    return LAUE_OK;
}

static int sm_count_current() {
    static int sms[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
    if (!sms[dev]) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) v = 1;
        sms[dev] = v;
    }
    return sms[dev];
}

template <int KB>
static cudaError_t launch_persistent(const CUtensorMap& tA, const CUtensorMap& tB, const GemmArgs& a,
                                     cudaStream_t s) {
    size_t smem = 1024 + (size_t)KB * kBBlock + (size_t)kPStages * kAStage;
    // one CTA per SM: it holds all 512 tensor-memory columns, so a second CTA
    // on the SM would wait in tcgen05.alloc; ask for more than half the SM's
    // shared memory so that the scheduler never co-locates two
    if (smem < 120 * 1024) smem = 120 * 1024;
    cudaError_t e = cudaFuncSetAttribute(gemm_tc_persistent_kernel<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    int n_tiles = a.M / kBM;
    int sms = sm_count_current();
    int grid = n_tiles < sms ? n_tiles : sms;
    gemm_tc_persistent_kernel<KB><<<grid, kPThreads, smem, s>>>(tA, tB, a, n_tiles);
    return cudaGetLastError();
}

cudaError_t gemm_tc_run(const GemmOperands& op, GemmArgs a, int splits, cudaStream_t s) {
    CUtensorMap tA, tB;
    // an MN-major operand is the 2-D array [K][M] (or [K][N]) read in boxes of
    // 64 MN elements x 64 k rows
    bool okA = a.a_mn ? make_tmap(&tA, op.A, (uint64_t)a.K, (uint64_t)a.M, op.lda, kBK)
                      : make_tmap(&tA, op.A, (uint64_t)a.M, (uint64_t)a.K, op.lda, kBM);
    bool okB = a.b_mn ? make_tmap(&tB, op.B, (uint64_t)a.K, (uint64_t)a.N, op.ldb, kBK)
                      : make_tmap(&tB, op.B, (uint64_t)a.N, (uint64_t)a.K, op.ldb, (uint32_t)a.BN);
    if (!okA || !okB) return cudaErrorInvalidValue;
    if (!a.simple && !a.a_mn && !a.b_mn && a.mode != 0 && splits == 1 && a.N == 256 && a.BN == 256) {
        if (a.K == 64) return launch_persistent<1>(tA, tB, a, s);
        if (a.K == 256) return launch_persistent<4>(tA, tB, a, s);
    }
    a.kb_per_split = a.K / kBK / splits;
    int stages = stages_for(a.kb_per_split);
    size_t smem = gemm_tc_smem(a.BN, stages);
    dim3 grid(a.M / kBM, a.N / a.BN, splits);
    cudaError_t e;
    if (stages == 2) {
        e = cudaFuncSetAttribute(gemm_tc_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gemm_tc_kernel<2><<<grid, kThreads, smem, s>>>(tA, tB, a);
    } else {
        e = cudaFuncSetAttribute(gemm_tc_kernel<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        gemm_tc_kernel<4><<<grid, kThreads, smem, s>>>(tA, tB, a);
    }
    return cudaGetLastError();
}

}  // namespace laue

using namespace laue;

extern "C" int laue_gemm_bf16(laue_handle* h, const void* A, long long lda, const void* B, long long ldb, int M,
                              int N, int K, int bn, int splits, int mode, const float* bias, const void* mask,
                              float* D_f32, void* D_bf16, void* DT_bf16, long long ldt, int flags,
                              void* stream) {
    if (!h) return LAUE_ERR_INVALID_ARG;
    if (!h->ws) return laue_fail(h, LAUE_ERR_WORKSPACE, "no workspace set");
    if (!A || !B || lda <= 0 || ldb <= 0) return laue_fail(h, LAUE_ERR_INVALID_ARG, "null or empty operand");
    GemmOperands op{(const __nv_bfloat16*)A, (const __nv_bfloat16*)B, (uint64_t)lda, (uint64_t)ldb};
    GemmArgs a{};
    a.M = M;
    a.N = N;
    a.K = K;
    a.BN = bn;
    a.mode = mode;
    a.bias = bias;
    a.mask = (const __nv_bfloat16*)mask;
    a.Df = D_f32;
    a.Dh = (__nv_bfloat16*)D_bf16;
    a.DhT = (__nv_bfloat16*)DT_bf16;
    a.ldt = ldt;
    a.ctrl = (int*)h->ws;
    a.simple = (flags & 1) ? 1 : 0;
    a.a_mn = (flags & 2) ? 1 : 0;
    a.b_mn = (flags & 4) ? 1 : 0;
    if (gemm_tc_check(op, a, splits) != LAUE_OK)
        return laue_fail(h, LAUE_ERR_INVALID_ARG, "gemm: M %% 128, N %% bn, K %% 64, splits | K/64, ld %% 8, alignment");
    return laue_cuda_check(h, gemm_tc_run(op, a, splits, (cudaStream_t)stream), "gemm launch");
}
