"""The tcgen05 BF16 GEMM of the set encoder against the oracle's FP64
product of the same BF16 operand values (element by element)."""
import numpy as np
import pytest

import oracle.proposal as op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2404_06478_gb300 import api, build, proposal
    build.build()
    dev = torch.device("cuda", 0)
    return dict(torch=torch, api=api, pr=proposal, dev=dev, h=api.Handle(dev))


def _bf(rng, shape, scale=1.0):
    return op.bf16(rng.standard_normal(shape) * scale)


def _dev(env, a, dtype=None):
    torch = env["torch"]
    return torch.tensor(a, dtype=torch.float32).to(dtype or torch.bfloat16).to(env["dev"])


def _bound(A, B, splits):
    """FP32 accumulation error bound: K * 2^-23 * sum_k |a||b| (per split)."""
    K = A.shape[1]
    return (np.abs(A) @ np.abs(B).T) * (K / splits) * 2.0 ** -23 + 1e-30


@pytest.mark.parametrize("M,N,K,bn,splits", [(128, 256, 64, 256, 1), (384, 256, 256, 256, 1),
                                              (256, 128, 512, 128, 2), (128, 64, 1024, 64, 4),
                                              (256, 256, 4096, 256, 8), (640, 128, 192, 128, 3)])
def test_gemm_f32_partials(env, M, N, K, bn, splits):
    torch = env["torch"]
    rng = np.random.default_rng(M * 7 + N + K)
    A, B = _bf(rng, (M, K)), _bf(rng, (N, K))
    D = torch.full((splits, M, N), float("nan"), device=env["dev"])
    env["pr"].gemm_bf16(env["h"], _dev(env, A), _dev(env, B), mode=0, bn=bn, splits=splits, out_f32=D)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    ref = op.gemm_tn(A, B, 0, splits=splits)
    got = D.cpu().numpy().astype(np.float64)
    ks = K // splits
    for s in range(splits):
        bound = _bound(A[:, s * ks:(s + 1) * ks], B[:, s * ks:(s + 1) * ks], 1)
        assert np.all(np.abs(got[s] - ref[s]) <= bound), np.abs(got[s] - ref[s]).max()


@pytest.mark.parametrize("a_mn,b_mn", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("M,N,K,bn,splits", [(256, 256, 8192, 256, 8), (256, 64, 4096, 64, 4),
                                              (384, 128, 192, 128, 1), (128, 256, 64, 256, 1)])
def test_gemm_mn_major_operands(env, a_mn, b_mn, M, N, K, bn, splits):
    """Operands stored MN-contiguous ([K][M], [K][N]) as the weight gradients
    read the row-major activations and errors: the same partial products as
    the K-major form, against the FP64 product of the same BF16 values."""
    torch = env["torch"]
    rng = np.random.default_rng(M + 3 * N + 5 * K + 7 * a_mn + 11 * b_mn)
    A, B = _bf(rng, (M, K)), _bf(rng, (N, K))
    Ad = _dev(env, A.T.copy() if a_mn else A)
    Bd = _dev(env, B.T.copy() if b_mn else B)
    D = torch.full((splits, M, N), float("nan"), device=env["dev"])
    env["pr"].gemm_bf16(env["h"], Ad, Bd, mode=0, bn=bn, splits=splits, out_f32=D, a_mn=a_mn, b_mn=b_mn)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    ref = op.gemm_tn(A, B, 0, splits=splits)
    got = D.cpu().numpy().astype(np.float64)
    ks = K // splits
    for s in range(splits):
        bound = _bound(A[:, s * ks:(s + 1) * ks], B[:, s * ks:(s + 1) * ks], 1)
        assert np.all(np.abs(got[s] - ref[s]) <= bound), np.abs(got[s] - ref[s]).max()


def _bf16_close(got, exact, bound):
    """A BF16 result of an FP32 accumulation: within the accumulation bound
    of the exact value, then rounded (relative 2^-8 covers one rounding).
    relu and the mask are 1-Lipschitz, so the bound carries through them."""
    err = np.abs(got - exact)
    lim = 2.0 ** -8 * np.abs(exact) + bound * (1 + 2.0 ** -8)
    return bool(np.all(err <= lim)), float(np.max(err - lim))


def _mostly_equal(got, ref):
    """Most BF16 results equal the rounded exact value (rounding flips are rare)."""
    return np.mean(got != ref) < 2e-3


@pytest.mark.parametrize("simple", [False, True])
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("M,N,K,bn", [(256, 256, 256, 256), (384, 128, 64, 128), (128, 64, 512, 64),
                                      (640, 256, 64, 256), (49152, 256, 256, 256)])
def test_gemm_bf16_epilogues(env, mode, M, N, K, bn, simple):
    """N = 256 with K = 64 or 256 runs the persistent kernel unless `simple`;
    49152 rows give every persistent CTA several tiles (both accumulators)."""
    torch = env["torch"]
    rng = np.random.default_rng(M + 3 * N + 5 * K + mode)
    A, B = _bf(rng, (M, K)), _bf(rng, (N, K), 0.1)
    bias = rng.standard_normal(N).astype(np.float32).astype(np.float64)
    mask = _bf(rng, (M, N))
    mask[rng.random((M, N)) < 0.1] = 0.0
    ldt = M + 64
    out = torch.full((M, N), float("nan"), dtype=torch.bfloat16, device=env["dev"])
    outT = torch.full((N, ldt), float("nan"), dtype=torch.bfloat16, device=env["dev"])
    env["pr"].gemm_bf16(env["h"], _dev(env, A), _dev(env, B), mode=mode, bn=bn,
                        bias=_dev(env, bias, torch.float32), mask=_dev(env, mask), out=out, outT=outT,
                        simple=simple)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    ref = op.gemm_tn(A, B, mode, bias=bias, mask=mask)
    exact = op.gemm_tn(A, B, mode, bias=bias, mask=mask, round_out=False)
    got = out.float().cpu().numpy()
    gotT = outT.float().cpu().numpy()
    ok, worst = _bf16_close(got, exact, _bound(A, B, 1))
    assert ok, worst
    assert _mostly_equal(got, ref)
    np.testing.assert_array_equal(gotT[:, :M], got.T)
    assert np.isnan(gotT[:, M:]).all()  # columns past M untouched


def test_gemm_large_sampled(env):
    """A per-spot layer at the size of a training batch (2048 sets x 128
    spots), checked on sampled rows."""
    torch = env["torch"]
    M, N, K = 262144, 256, 256
    g = torch.Generator(device="cpu").manual_seed(5)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = (torch.randn(N, K, generator=g) * 0.1).to(torch.bfloat16)
    bias = torch.randn(N, generator=g)
    out = torch.empty(M, N, dtype=torch.bfloat16, device=env["dev"])
    outT = torch.empty(N, M, dtype=torch.bfloat16, device=env["dev"])
    env["pr"].gemm_bf16(env["h"], A.to(env["dev"]), B.to(env["dev"]), mode=1, bias=bias.to(env["dev"]), out=out,
                        outT=outT)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    rows = np.random.default_rng(6).choice(M, 512, replace=False)
    An = A.float().numpy().astype(np.float64)[rows]
    Bn = B.float().numpy().astype(np.float64)
    ref = op.gemm_tn(An, Bn, 1, bias=bias.numpy())
    exact = op.gemm_tn(An, Bn, 1, bias=bias.numpy(), round_out=False)
    got = out.float().cpu().numpy()[rows]
    ok, worst = _bf16_close(got, exact, _bound(An, Bn, 1))
    assert ok, worst
    assert _mostly_equal(got, ref)
    np.testing.assert_array_equal(outT.float().cpu().numpy()[:, rows], got.T)


def test_gemm_rejects_bad_shapes(env):
    torch = env["torch"]
    A = torch.zeros(100, 64, dtype=torch.bfloat16, device=env["dev"])
    B = torch.zeros(256, 64, dtype=torch.bfloat16, device=env["dev"])
    D = torch.zeros(1, 100, 256, device=env["dev"])
    with pytest.raises(RuntimeError):
        env["pr"].gemm_bf16(env["h"], A, B, mode=0, out_f32=D)
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device=env["dev"])
    with pytest.raises(RuntimeError):
        env["pr"].gemm_bf16(env["h"], A, B, mode=0, bn=96, out_f32=D)
    with pytest.raises(RuntimeError):
        env["pr"].gemm_bf16(env["h"], A, B, mode=1, out=torch.zeros(128, 256, dtype=torch.bfloat16,
                                                                        device=env["dev"]))  # no bias
