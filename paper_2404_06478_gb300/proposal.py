"""Learned proposal over the C ABI: the tensor-core GEMM of the set encoder
(more calls follow in this module as the encoder is built).

Argument marshalling only: every step runs in liblaueot.so.  The paper has no
learned component; this is an addition beside its candidate scan.
"""
from __future__ import annotations

import torch

from . import api


def gemm_bf16(h: api.Handle, A: torch.Tensor, B: torch.Tensor, mode: int = 0, bn: int = 256, splits: int = 1,
              bias: torch.Tensor | None = None, mask: torch.Tensor | None = None, out_f32=None, out=None,
              outT=None, stream=None):
    """D[m][n] = sum_k A[m][k] B[n][k] on the tcgen05 tensor cores (BF16 in,
    FP32 accumulate).  mode 0 writes `splits` FP32 partials into out_f32
    (splits, M, N); mode 1 relu(D + bias) and mode 2 D * (mask > 0) as BF16
    into out (M, N) and/or outT (N, ldt)."""
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
    M, K = A.shape
    N = B.shape[0]
    if h.ws is None:
        h.reserve(1, stream=stream)
    ldt = outT.stride(0) if outT is not None else 0
    rc = h.L.laue_gemm_bf16(h.h, api._ptr(A), A.stride(0), api._ptr(B), B.stride(0), M, N, K, bn, splits, mode,
                            api._ptr(bias), api._ptr(mask), api._ptr(out_f32), api._ptr(out), api._ptr(outT), ldt,
                            api._stream(stream))
    h.check(rc, "gemm_bf16")
