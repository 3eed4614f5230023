"""Parity of laue_forward / laue_refresh (CUDA) with the FP64 oracle."""
import dataclasses

import numpy as np
import pytest

import oracle
import synthgen as sg
from _cases import GEOM, f32, planes32

pytestmark = pytest.mark.gpu

MARGIN = 1e-5   # visibility decisions closer than this (relative) to a threshold may differ


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2404_06478_gb300 import api, build
    build.build()
    dev = torch.device("cuda", 0)
    return dict(torch=torch, api=api, dev=dev, h=api.Handle(dev))


def _gpu_forward(env, cfg, R, x, om, capacity=None):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    lat = api.Lattice.cubic(cfg.a, cfg.hmax, cfg.centering, device=dev)
    ms = api.forward(env["h"], GEOM, lat, torch.tensor(R, device=dev), torch.tensor(x, device=dev),
                     torch.tensor(om, device=dev), capacity=capacity)
    n = ms.n
    g = lambda t: t[:n].cpu().numpy()
    return dict(n=n, J_off=ms.J_off.cpu().numpy(), grain=g(ms.grain), plane=g(ms.plane), angle=g(ms.angle),
                ray=g(ms.ray), center=g(ms.center), spot=g(ms.spot)), ms, lat


def _compare(cfg, R, x, om, gpu):
    P = planes32(cfg)
    ref = oracle.forward(GEOM, P, R, x, om, with_all=True)
    T, N, M = ref["vis_all"].shape
    vis_gpu = np.zeros((T, N, M), bool)
    vis_gpu[gpu["angle"], gpu["grain"], gpu["plane"]] = True
    sure = ref["margin_all"] > MARGIN
    np.testing.assert_array_equal(vis_gpu[sure], ref["vis_all"][sure].astype(bool))
    # sorted by (t, n, m) and consistent offsets
    key = (gpu["angle"].astype(np.int64) * N + gpu["grain"]) * M + gpu["plane"]
    assert np.all(np.diff(key) > 0)
    np.testing.assert_array_equal(np.searchsorted(gpu["angle"], np.arange(T + 1)), gpu["J_off"])
    # values on spots visible on both sides
    rk = (ref["t"].astype(np.int64) * N + ref["grain"]) * M + ref["plane"]
    common, ig, ir = np.intersect1d(key, rk, return_indices=True)
    assert len(common) >= 0.999 * len(rk)
    np.testing.assert_allclose(gpu["ray"][ig, :3], ref["ray"][ir, :3], atol=2e-6)
    np.testing.assert_allclose(gpu["ray"][ig, 3], ref["ray"][ir, 3], rtol=2e-6)
    np.testing.assert_allclose(gpu["center"][ig, :3], ref["center"][ir], atol=2e-5)
    np.testing.assert_allclose(gpu["spot"][ig, :3], ref["spot"][ir], atol=5e-4)
    np.testing.assert_array_equal(gpu["spot"][ig, 3].astype(int), ref["det"][ir])
    return len(common)


@pytest.mark.parametrize("name,n_grains,T", [("tiny", None, None), ("medium", 60, 12), ("medium", 7, 5)])
def test_forward_parity(env, name, n_grains, T):
    cfg = sg.CONFIGS[name]
    if n_grains:
        cfg = dataclasses.replace(cfg, n_grains=n_grains, T=T)
    rng = np.random.default_rng(3)
    R, x = sg.random_grains(cfg, rng)
    R, x, om = f32(R), f32(x), f32(sg.omegas(cfg))
    gpu, _, _ = _gpu_forward(env, cfg, R, x, om)
    assert _compare(cfg, R, x, om, gpu) > 0


def test_forward_full_size_sampled(env):
    """1000 grains x 90 angles x 433 directions (39M rays): the (grain, angle)
    pairs of a random sample match the oracle run on that grain and angle."""
    cfg = sg.CONFIGS["batched"]
    rng = np.random.default_rng(4)
    R, x = sg.random_grains(cfg, rng)
    R, x, om = f32(R), f32(x), f32(sg.omegas(cfg))
    gpu, _, _ = _gpu_forward(env, cfg, R, x, om)
    assert 600_000 < gpu["n"] < 800_000
    P = planes32(cfg)
    for k in range(40):
        n, t = int(rng.integers(cfg.n_grains)), int(rng.integers(cfg.T))
        ref = oracle.forward(GEOM, P, R[n:n + 1], x[n:n + 1], om[t:t + 1], with_all=True)
        sel = (gpu["grain"] == n) & (gpu["angle"] == t)
        vis = np.zeros(len(P.w), bool)
        vis[gpu["plane"][sel]] = True
        sure = ref["margin_all"][0, 0] > MARGIN
        np.testing.assert_array_equal(vis[sure], ref["vis_all"][0, 0][sure].astype(bool))
        common = np.intersect1d(gpu["plane"][sel], ref["plane"])
        gi = {m: i for i, m in enumerate(gpu["plane"][sel])}
        ri = {m: i for i, m in enumerate(ref["plane"])}
        for m in common:
            np.testing.assert_allclose(gpu["ray"][sel][gi[m], :3], ref["ray"][ri[m], :3], atol=2e-6)
            np.testing.assert_allclose(gpu["spot"][sel][gi[m], :3], ref["spot"][ri[m]], atol=5e-4)


def test_forward_edge_cases(env):
    cfg = sg.CONFIGS["tiny"]
    om = f32(sg.omegas(cfg))
    # no grains: empty list, zero offsets
    gpu, _, _ = _gpu_forward(env, cfg, np.zeros((0, 3, 3)), np.zeros((0, 3)), om)
    assert gpu["n"] == 0 and not gpu["J_off"].any()
    # one angle
    rng = np.random.default_rng(5)
    R, x = sg.random_grains(cfg, rng)
    R, x = f32(R), f32(x)
    gpu, _, _ = _gpu_forward(env, cfg, R, x, om[:1])
    _compare(cfg, R, x, om[:1], gpu)
    # capacity overflow reports the needed size and keeps offsets valid
    from paper_2404_06478_gb300 import api
    with pytest.raises(api.LaueError) as ei:
        _gpu_forward(env, cfg, R, x, om, capacity=5)
    assert ei.value.code == -2


def test_refresh_matches_oracle(env):
    torch = env["torch"]
    cfg = dataclasses.replace(sg.CONFIGS["medium"], n_grains=20, T=8)
    rng = np.random.default_rng(6)
    R, x = sg.random_grains(cfg, rng)
    R, x, om = f32(R), f32(x), f32(sg.omegas(cfg))
    gpu, ms, lat = _gpu_forward(env, cfg, R, x, om)
    R2, x2 = f32(sg.random_rotations(cfg.n_grains, rng)), f32(x + rng.normal(size=x.shape))
    dev = env["dev"]
    env["api"].refresh(env["h"], GEOM, lat, torch.tensor(R2, device=dev), torch.tensor(x2, device=dev),
                       torch.tensor(om, device=dev), ms)
    ray, ce = oracle.refresh(GEOM, planes32(cfg), R2, x2, om, gpu["J_off"], gpu["grain"], gpu["plane"])
    n = ms.n
    np.testing.assert_allclose(ms.ray[:n, :3].cpu().numpy(), ray[:, :3], atol=2e-6)
    np.testing.assert_allclose(ms.center[:n, :3].cpu().numpy(), ce, atol=2e-5)
