// gemm_tc.h — the tcgen05 BF16 GEMM of the set encoder (gemm_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

namespace laue {

struct GemmOperands {
    const __nv_bfloat16* A;  // [M][lda], K-contiguous; with GemmArgs::a_mn [K][lda], M-contiguous
    const __nv_bfloat16* B;  // [N][ldb], K-contiguous; with GemmArgs::b_mn [K][ldb], N-contiguous
    uint64_t lda, ldb;
};

struct GemmArgs {
    int M, N, K;  // M % 128 == 0, N % BN == 0, K % 64 == 0
    int BN;       // 64, 128 or 256
    int kb_per_split;  // set by gemm_tc_run
    int mode;     // 0: FP32 partials, 1: bias + relu -> BF16, 2: mask -> BF16
    const float* bias;          // mode 1: [N]
    const __nv_bfloat16* mask;  // mode 2: [M][N]
    float* Df;                  // mode 0: [splits][M][N]
    __nv_bfloat16* Dh;          // modes 1, 2: [M][N] or null
    __nv_bfloat16* DhT;         // modes 1, 2: [N][ldt] or null
    long long ldt;
    int* ctrl;                  // status word
    int simple;                 // 1: always the one-tile-per-CTA kernel
    int a_mn, b_mn;             // 1: the operand is stored MN-contiguous (one-tile-per-CTA kernel)
};

size_t gemm_tc_smem(int BN, int stages);
int gemm_tc_check(const GemmOperands& op, const GemmArgs& a, int splits);
cudaError_t gemm_tc_run(const GemmOperands& op, GemmArgs a, int splits, cudaStream_t s);

}  // namespace laue
