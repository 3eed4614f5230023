"""Parity of laue_cost_sinkhorn (fused cost + log-domain Sinkhorn, CUDA) with
the FP64 oracle on the same float32 inputs.

Tolerances (derived from the FP32 arithmetic of the kernels): potentials
within 1e-4 * (|f| + eps) (FP32 log-sum-exp over up to a few thousand terms
with hardware ex2/lg2/rsqrt approximations, relative error ~1e-6 per
iteration, accumulated over <= 200 iterations along the shift-neutral
direction); hard assignments bit-exact wherever the oracle's top-two margin
exceeds 1e-3; margins within 1e-4."""
import dataclasses

import numpy as np
import pytest

import oracle
import synthgen as sg
from _cases import GEOM, make_case, to_device

pytestmark = pytest.mark.gpu

TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2404_06478_gb300 import api, build
    build.build()
    dev = torch.device("cuda", 0)
    return dict(torch=torch, api=api, dev=dev, h=api.Handle(dev))


def _run_both(env, case, n_iter, mode=0, eps=None, frac=0.4, cols=False):
    api = env["api"]
    eps = case.cfg.eps if eps is None else eps
    ob, ms = to_device(case, env["dev"])
    out = api.cost_sinkhorn(env["h"], GEOM, ob, ms, eps, case.c_out, n_iter, dust_mode=mode,
                            unmatched_frac=frac, harvest=True, col_harvest=cols)
    env["torch"].cuda.synchronize()
    assert env["h"].device_status() == 0
    gpu = {k: v.cpu().numpy().astype(np.float64) if v.dtype.is_floating_point else v.cpu().numpy()
           for k, v in out.items()}
    fw, obs = case.fw, case.obs
    f, g, fd, gd, _ = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3],
                                      eps, case.c_out, mode, frac, n_iter)
    h = oracle.harvest(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], eps,
                       case.c_out, mode, frac, f, g, fd, gd)
    ref = dict(f=f, g=g, dust=np.concatenate([fd, gd]), **h)
    return gpu, ref, eps


def _check(gpu, ref, eps):
    for k in ("f", "g", "dust"):
        err = np.abs(gpu[k] - ref[k])
        lim = TOL * (np.abs(ref[k]) + eps)
        assert np.all(err <= lim), (k, float((err / lim).max()))
    sure = ref["margin"] > 1e-3
    assert sure.mean() > 0.5
    np.testing.assert_array_equal(gpu["assign"][sure], ref["assign"][sure])
    np.testing.assert_allclose(gpu["margin"], ref["margin"], atol=1e-4)
    assert abs(gpu["marg_err"][0] - ref["row_err"]) < 1e-4


@pytest.mark.parametrize("mode", [0, 1])
def test_sinkhorn_tiny(env, mode):
    case = make_case(sg.CONFIGS["tiny"])
    gpu, ref, eps = _run_both(env, case, 100, mode=mode)
    _check(gpu, ref, eps)


@pytest.mark.parametrize("mode", [0, 1])
def test_sinkhorn_multi_tile_ragged(env, mode):
    """60 grains, 8 angles, |hkl| <= 6, 30% outliers: several row and column
    tiles per angle block with ragged tails, several staged chunks each."""
    case = make_case(sg.CONFIGS["medium"], seed=11, n_grains=60, T=8)
    nI = np.diff(case.obs.I_off)
    nJ = np.diff(case.fw["J_off"])
    assert nI.max() > 256 and nJ.max() > 256 and (nI % 256).min() > 0
    gpu, ref, eps = _run_both(env, case, 60, mode=mode, cols=True)
    _check(gpu, ref, eps)
    np.testing.assert_allclose(gpu["q"], ref["q"], atol=1e-4)


@pytest.mark.parametrize("eps", [0.25, 4.0, 100.0])
def test_sinkhorn_temperatures(env, eps):
    case = make_case(sg.CONFIGS["tiny"], seed=5)
    gpu, ref, _ = _run_both(env, case, 40, eps=eps)
    for k in ("f", "g", "dust"):
        err = np.abs(gpu[k] - ref[k])
        assert np.all(err <= TOL * (np.abs(ref[k]) + eps)), k


def test_sinkhorn_empty_blocks(env):
    """Angle blocks with no observed spots and blocks with no model spots."""
    case = make_case(sg.CONFIGS["tiny"], seed=7)
    obs, fw = case.obs, case.fw
    # drop observed spots of angle 2 and model spots of angle 5
    keep_i = obs.t != 2
    obs.p, obs.t, obs.det, obs.truth = obs.p[keep_i], obs.t[keep_i], obs.det[keep_i], obs.truth[keep_i]
    obs.I_off = np.r_[0, np.cumsum(np.bincount(obs.t, minlength=case.cfg.T))]
    keep_j = fw["t"] != 5
    for k in ("grain", "plane", "ray", "spot", "center", "det", "t"):
        fw[k] = fw[k][keep_j]
    fw["J_off"] = np.r_[0, np.cumsum(np.bincount(fw["t"], minlength=case.cfg.T))]
    for mode in (0, 1):
        gpu, ref, eps = _run_both(env, case, 30, mode=mode)
        _check(gpu, ref, eps)


def test_sinkhorn_no_unmatched_mass(env):
    """unmatched fraction 0 (U from the balance rule only)."""
    case = make_case(sg.CONFIGS["tiny"], seed=8)
    gpu, ref, eps = _run_both(env, case, 30, frac=0.0)
    _check(gpu, ref, eps)


def test_sinkhorn_warm_start_continues(env):
    api, torch = env["api"], env["torch"]
    case = make_case(sg.CONFIGS["tiny"], seed=9)
    ob, ms = to_device(case, env["dev"])
    a = api.cost_sinkhorn(env["h"], GEOM, ob, ms, 1.0, case.c_out, 25)
    b = api.cost_sinkhorn(env["h"], GEOM, ob, ms, 1.0, case.c_out, 15, init=(a["f"], a["g"], a["dust"]))
    fw, obs = case.fw, case.obs
    f, g, fd, gd, _ = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3],
                                      1.0, case.c_out, 0, 0.4, 40)
    np.testing.assert_allclose(b["f"].cpu().numpy(), f, atol=TOL * (np.abs(f).max() + 1))
    np.testing.assert_allclose(b["g"].cpu().numpy(), g, atol=TOL * (np.abs(g).max() + 1))


def test_sinkhorn_exact_fallback_is_taken_and_matches(env):
    """At eps = 0.02 mm^2 the outlier-column term (2^-162 after the shift) and
    every pair of an observed spot far from all model spots underflow the
    shifted fast sum of the row pass, so those rows take the exact
    log-sum-exp path; the device count proves it ran and the potentials still
    equal the oracle's.  The column pass always keeps its unmatched-row term
    (cost 0), so its exact path is reached without dustbins: the unbalanced
    mode at the same temperature, where model spots far from every observed
    spot underflow, again against the oracle."""
    case = make_case(sg.CONFIGS["tiny"], seed=15)
    env["h"].exact_lse_count()  # clear
    gpu, ref, eps = _run_both(env, case, 30, eps=0.02)
    rows, cols = env["h"].exact_lse_count()
    assert rows > 0, (rows, cols)
    for k in ("f", "g", "dust"):
        err = np.abs(gpu[k] - ref[k])
        assert np.all(err <= TOL * (np.abs(ref[k]) + eps)), (k, float((err / (TOL * (np.abs(ref[k]) + eps))).max()))
    gpu, ref = _run_unbalanced(env, case, 30, 0.02, 4.0, 4.0)
    rows, cols = env["h"].exact_lse_count()
    assert rows > 0 and cols > 0, (rows, cols)
    for k in ("f", "g"):
        err = np.abs(gpu[k] - ref[k])
        assert np.all(err <= TOL * (np.abs(ref[k]) + 0.02)), (k, float((err / (TOL * (np.abs(ref[k]) + 0.02))).max()))
    # and at eps = 1 nothing underflows
    _run_both(env, case, 5, eps=1.0)
    assert env["h"].exact_lse_count() == (0, 0)


@pytest.fixture(scope="module")
def batched():
    """The 1000-grain / 90-rotation / 70%-uneven-outlier workload, made by the
    oracle's forward model (model list at the truth)."""
    return make_case(sg.CONFIGS["batched"], seed=0)


def test_sinkhorn_full_size_per_angle_blocks_match_oracle(env, batched):
    """1000 grains, 90 angles, 70% uneven outliers, per-angle dustbins (the
    angle blocks are then independent problems): 20 iterations of the whole
    workload on the GPU in one call; the oracle solves two sampled blocks
    alone.  f, g, the block's dustbin potentials, the hard assignment (where
    the oracle's margin exceeds 1e-3) and the margins agree element by element."""
    from _cases import block_slices, oracle_parallel
    api, torch, dev = env["api"], env["torch"], env["dev"]
    case = batched
    ob, ms = to_device(case, dev)
    n_iter, eps, T = 20, case.cfg.eps, case.cfg.T
    out = api.cost_sinkhorn(env["h"], GEOM, ob, ms, eps, case.c_out, n_iter, dust_mode=1, harvest=True)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    gpu = {k: v.cpu().numpy() for k, v in out.items()}
    nI, nJ = np.diff(case.obs.I_off), np.diff(case.fw["J_off"])
    blocks = [int(t) for t in np.argsort(nI * nJ)[:2]]
    calls = []
    for t in blocks:
        si, sj = block_slices(case, t)
        args = (GEOM.D, case.obs.p[si], [0, si.stop - si.start], [0, sj.stop - sj.start], case.fw["center"][sj],
                case.fw["ray"][sj, :3], eps, case.c_out, 1, 0.4, n_iter)
        calls.append(("sinkhorn", args, {}))
    res = oracle_parallel(calls)
    for t, (f, g, fd, gd, _) in zip(blocks, res):
        si, sj = block_slices(case, t)
        h = oracle.harvest(GEOM.D, case.obs.p[si], [0, si.stop - si.start], [0, sj.stop - sj.start],
                           case.fw["center"][sj], case.fw["ray"][sj, :3], eps, case.c_out, 1, 0.4, f, g, fd, gd)
        for name, got, want in (("f", gpu["f"][si], f), ("g", gpu["g"][sj], g),
                                ("dust", gpu["dust"][[t, T + t]], np.r_[fd, gd])):
            err = np.abs(got.astype(np.float64) - want)
            lim = TOL * (np.abs(want) + eps)
            assert np.all(err <= lim), (t, name, float((err / lim).max()))
        sure = h["margin"] > 1e-3
        assert sure.mean() > 0.5
        a = gpu["assign"][si]
        want_a = np.where(h["assign"] >= 0, h["assign"] + sj.start, -1)
        np.testing.assert_array_equal(a[sure], want_a[sure])
        np.testing.assert_allclose(gpu["margin"][si], h["margin"], atol=1e-4)


def test_sinkhorn_full_size_global_rows_and_marginals(env, batched):
    """The same workload with the global dustbins: one iteration from zero
    gives, for sampled rows, the oracle's row update of their own angle block
    with the dustbin terms at zero; after 200 iterations the row and column
    marginals converge (a property at any size)."""
    api, torch, dev = env["api"], env["torch"], env["dev"]
    case = batched
    ob, ms = to_device(case, dev)
    h = env["h"]
    one = api.cost_sinkhorn(h, GEOM, ob, ms, 1.0, case.c_out, 1, harvest=False)
    f1 = one["f"].cpu().numpy()
    rng = np.random.default_rng(3)
    for t in rng.choice(case.cfg.T, 4, replace=False):
        i0, i1 = case.obs.I_off[t], case.obs.I_off[t + 1]
        j0, j1 = case.fw["J_off"][t], case.fw["J_off"][t + 1]
        sel = rng.choice(np.arange(i0, i1), 16, replace=False)
        fo, *_ = oracle.sinkhorn(GEOM.D, case.obs.p[sel], [0, len(sel)], [0, j1 - j0], case.fw["center"][j0:j1],
                                 case.fw["ray"][j0:j1, :3], 1.0, case.c_out, 0, 0.4, 1)
        np.testing.assert_allclose(f1[sel], fo, atol=TOL * (np.abs(fo).max() + 1.0))
    full = api.cost_sinkhorn(h, GEOM, ob, ms, 1.0, case.c_out, 200, harvest=True, col_harvest=True)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    me = full["marg_err"].cpu().numpy()
    assert me[0] < 1e-2 and me[1] < 1e-4


@pytest.mark.parametrize("shape", [0, 1, 2, 3])
def test_sinkhorn_every_launch_shape(env, shape):
    """Each launch shape of the autotuner (CTA width 256, 128 or 64 spot
    pairs, with and without a register cap) gives the same results."""
    case = make_case(sg.CONFIGS["medium"], seed=12, n_grains=60, T=8)
    env["h"].set_launch_shape(shape, (shape + 1) % 4)
    try:
        gpu, ref, eps = _run_both(env, case, 40, mode=shape % 2, cols=True)
    finally:
        env["h"].set_launch_shape(3, 3)
    _check(gpu, ref, eps)


def test_autotune_picks_valid_shapes(env):
    api = env["api"]
    case = make_case(sg.CONFIGS["medium"], seed=13, n_grains=100, T=12)
    ob, ms = to_device(case, env["dev"])
    h = api.Handle(env["dev"])
    r, c, times = api.autotune(h, GEOM, ob, ms, 1.0, case.c_out, n_iter=2)
    assert 0 <= r < 4 and 0 <= c < 4
    assert all(a > 0 and b > 0 for a, b in times)
    assert times[r][0] == min(a for a, _ in times) and times[c][1] == min(b for _, b in times)


def _run_unbalanced(env, case, n_iter, eps, kappa, lam):
    api = env["api"]
    ob, ms = to_device(case, env["dev"])
    out = api.cost_sinkhorn(env["h"], GEOM, ob, ms, eps, case.c_out, n_iter, dust_mode=2, harvest=True,
                            col_harvest=True, kappa=kappa, lam=lam)
    env["torch"].cuda.synchronize()
    assert env["h"].device_status() == 0
    gpu = {k: v.cpu().numpy().astype(np.float64) if v.dtype.is_floating_point else v.cpu().numpy()
           for k, v in out.items()}
    fw, obs = case.fw, case.obs
    f, g = oracle.sinkhorn_unbalanced(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], eps,
                                      kappa, lam, n_iter)
    h = oracle.harvest_unbalanced(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], eps, f, g)
    return gpu, dict(f=f, g=g, **h)


@pytest.mark.parametrize("kappa,lam", [(2.0, 8.0), (50.0, 0.5)])
def test_sinkhorn_unbalanced_matches_oracle(env, kappa, lam):
    """Unbalanced OT (Algorithm UnbalancedOT, no dustbins, KL-relaxed
    marginals) on 60 grains x 8 angles with ragged multi-tile blocks: f, g
    within the Sinkhorn tolerance, hard assignments (-1 where a row keeps less
    than half its mass) equal where the oracle's margin exceeds 1e-3, column
    masses within 1e-4."""
    case = make_case(sg.CONFIGS["medium"], seed=16, n_grains=60, T=8)
    eps = 1.0
    gpu, ref = _run_unbalanced(env, case, 40, eps, kappa, lam)
    for k in ("f", "g"):
        err = np.abs(gpu[k] - ref[k])
        lim = TOL * (np.abs(ref[k]) + eps)
        assert np.all(err <= lim), (k, float((err / lim).max()))
    sure = (ref["margin"] > 1e-3) & (np.abs(ref["rowmass"] - 0.5) > 1e-3)
    assert sure.mean() > 0.5
    np.testing.assert_array_equal(gpu["assign"][sure], ref["assign"][sure])
    np.testing.assert_allclose(gpu["margin"], ref["margin"], atol=1e-4)
    np.testing.assert_allclose(gpu["q"], ref["q"], atol=1e-4)
    assert (ref["assign"] == -1).any() and (ref["assign"] >= 0).any()


def test_sinkhorn_unbalanced_empty_blocks(env):
    """Unbalanced mode with an angle block that has no observed spots and one
    that has no model spots (their potentials stay 0)."""
    case = make_case(sg.CONFIGS["tiny"], seed=17)
    obs, fw = case.obs, case.fw
    keep_i = obs.t != 3
    obs.p, obs.t, obs.det, obs.truth = obs.p[keep_i], obs.t[keep_i], obs.det[keep_i], obs.truth[keep_i]
    obs.I_off = np.r_[0, np.cumsum(np.bincount(obs.t, minlength=case.cfg.T))]
    keep_j = fw["t"] != 6
    for k in ("grain", "plane", "ray", "spot", "center", "det", "t"):
        fw[k] = fw[k][keep_j]
    fw["J_off"] = np.r_[0, np.cumsum(np.bincount(fw["t"], minlength=case.cfg.T))]
    gpu, ref = _run_unbalanced(env, case, 30, 1.0, 5.0, 5.0)
    for k in ("f", "g"):
        err = np.abs(gpu[k] - ref[k])
        assert np.all(err <= TOL * (np.abs(ref[k]) + 1.0)), k


@pytest.mark.parametrize("eps,mode", [(0.25, 0), (1.0, 1), (1.0, 2), (2000.0, 0)])
def test_sinkhorn_skipping_is_bit_identical(env, eps, mode):
    """The exact underflow skipping (direction-ordered spots, cone bounds per
    run of 128 pairs) changes no bit of the potentials, the dustbins or the
    read-out.  Workload: the 1000-grain density on 4 angles (about 14k
    observed and 8k model spots per block, so a tile's cone spans a few degrees
    of a detector).  At eps <= 1 mm^2 a host model of the cone bounds (32-pair
    granules, the default 64-pair tiles) predicts that the row pass keeps about
    a quarter of its pairs, and the column pass keeps somewhat more; at
    eps = 2000 none can be skipped."""
    api, torch = env["api"], env["torch"]
    case = make_case(sg.CONFIGS["batched"], seed=0, T=4)
    ob, ms = to_device(case, env["dev"])
    h = env["h"]
    h.reserve(case.cfg.T, n_obs=int(case.obs.I_off[-1]), n_model=int(case.fw["J_off"][-1]))
    runs = {}
    try:
        for skip in (False, True):
            h.set_pair_skipping(skip)
            h.counters()
            out = api.cost_sinkhorn(h, GEOM, ob, ms, eps, case.c_out, 30, dust_mode=mode, harvest=True,
                                    col_harvest=True, kappa=3.0, lam=3.0)
            torch.cuda.synchronize()
            assert h.device_status() == 0
            runs[skip] = (out, h.counters()["pass_pairs"])
    finally:
        h.set_pair_skipping(True)
    (a, pa), (b, pb) = runs[False], runs[True]
    for k in a:
        assert torch.equal(a[k], b[k]), k
    nI, nJ = np.diff(case.obs.I_off), np.diff(case.fw["J_off"])
    dense = 2 * 30 * int(np.sum((nI + nI % 2) * (nJ + nJ % 2)))
    assert pa == dense
    if eps <= 1.0:
        assert pb < 0.5 * pa, (pb, pa)
    else:
        assert pb == pa
