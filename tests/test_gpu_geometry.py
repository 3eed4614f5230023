"""Parity on a two-detector geometry like the paper's experimental setups
(Appendix "Experimental details": forward and backscatter detectors at
different sample distances): the transmission detector at 125 mm, offset
10 mm along x, the backscatter detector at 165 mm and tilted by 8 degrees,
each with its own cost length (C_ij = D_j^2 |rhat - r_j|^2, D_j the distance
of the detector model spot j hits).  Every stage of the path runs on this
geometry against the FP64 oracle with the same per-detector lengths:
forward model, dense E-step (global and per-angle dustbins), unbalanced and
sparse E-steps, plain and adjoint M-steps, the adjoint gradient, single-grain
fits, the SPOT matrix selection, the EM driver and laue_index.  Tolerances are
those of the axis-aligned tests."""
import math

import numpy as np
import pytest

import oracle
import synthgen as sg
from _cases import f32, geom32, make_case, planes32, to_device

pytestmark = pytest.mark.gpu

TILT = geom32(sg.tilted_geometry())
TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2404_06478_gb300 import api, build
    build.build()
    dev = torch.device("cuda", 0)
    return dict(torch=torch, api=api, dev=dev, h=api.Handle(dev))


def _rotvec(w):
    th = float(np.linalg.norm(w))
    if th == 0:
        return np.eye(3)
    k = np.asarray(w) / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def _mis_deg(A, B):
    M = np.einsum("nji,njk->nik", A, B)
    ax = np.stack([M[:, 2, 1] - M[:, 1, 2], M[:, 0, 2] - M[:, 2, 0], M[:, 1, 0] - M[:, 0, 1]], -1) / 2
    return np.degrees(np.arctan2(np.linalg.norm(ax, axis=1), (np.trace(M, axis1=1, axis2=2) - 1) / 2))


def _cubic():
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            S = np.zeros((3, 3))
            for r, c in enumerate(perm):
                S[r, c] = signs[r]
            if np.linalg.det(S) > 0:
                out.append(S)
    return out


def _t(env, a, dtype=None):
    torch = env["torch"]
    return torch.tensor(np.asarray(a), dtype=dtype or torch.float32, device=env["dev"]).contiguous()


def _Dj(case):
    return oracle.cost_lengths(TILT, case.fw["det"])


def test_forward_parity_tilted(env):
    api = env["api"]
    cfg = sg.CONFIGS["medium"]
    import dataclasses
    cfg = dataclasses.replace(cfg, n_grains=60, T=12)
    rng = np.random.default_rng(3)
    R, x = sg.random_grains(cfg, rng)
    R, x, om = f32(R), f32(x), f32(sg.omegas(cfg))
    lat = api.Lattice.cubic(cfg.a, cfg.hmax, cfg.centering, device=env["dev"])
    ms = api.forward(env["h"], TILT, lat, _t(env, R), _t(env, x), _t(env, om))
    n = ms.n
    ref = oracle.forward(TILT, planes32(cfg), R, x, om, with_all=True)
    T, N, M = ref["vis_all"].shape
    ang, gr, pl = (a[:n].cpu().numpy() for a in (ms.angle, ms.grain, ms.plane))
    vis = np.zeros((T, N, M), bool)
    vis[ang, gr, pl] = True
    sure = ref["margin_all"] > 1e-5
    np.testing.assert_array_equal(vis[sure], ref["vis_all"][sure].astype(bool))
    key = (ang.astype(np.int64) * N + gr) * M + pl
    rk = (ref["t"].astype(np.int64) * N + ref["grain"]) * M + ref["plane"]
    common, ig, ir = np.intersect1d(key, rk, return_indices=True)
    assert len(common) >= 0.999 * len(rk)
    spot = ms.spot[:n].cpu().numpy()
    np.testing.assert_allclose(spot[ig, :3], ref["spot"][ir], atol=5e-4)
    np.testing.assert_array_equal(spot[ig, 3].astype(int), ref["det"][ir])
    assert np.bincount(ref["det"], minlength=2).min() > 100


@pytest.mark.parametrize("mode", [0, 1])
def test_estep_tilted(env, mode):
    api = env["api"]
    case = make_case(sg.CONFIGS["medium"], seed=11, n_grains=60, T=8, geom=TILT)
    eps = case.cfg.eps
    ob, ms = to_device(case, env["dev"])
    out = api.cost_sinkhorn(env["h"], TILT, ob, ms, eps, case.c_out, 60, dust_mode=mode, harvest=True,
                            col_harvest=True)
    env["torch"].cuda.synchronize()
    assert env["h"].device_status() == 0
    fw, obs = case.fw, case.obs
    geo = (_Dj(case), obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3])
    f, g, fd, gd, _ = oracle.sinkhorn(*geo, eps, case.c_out, mode, 0.4, 60)
    h = oracle.harvest(*geo, eps, case.c_out, mode, 0.4, f, g, fd, gd)
    for name, got, want in (("f", out["f"], f), ("g", out["g"], g), ("dust", out["dust"], np.r_[fd, gd])):
        got = got.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want) <= TOL * (np.abs(want) + eps)), name
    sure = h["margin"] > 1e-3
    assert sure.mean() > 0.5
    np.testing.assert_array_equal(out["assign"].cpu().numpy()[sure], h["assign"][sure])
    np.testing.assert_allclose(out["q"].cpu().numpy(), h["q"], atol=1e-4)
    # the per-detector lengths matter: the single-D oracle differs
    f1, *_ = oracle.sinkhorn(TILT.D, *geo[1:], eps, case.c_out, mode, 0.4, 60)
    assert np.abs(f1 - f).max() > 100 * TOL * (np.abs(f).max() + eps)


def test_unbalanced_and_sparse_tilted(env):
    api = env["api"]
    case = make_case(sg.CONFIGS["tiny"], seed=12, geom=TILT)
    eps = case.cfg.eps
    ob, ms = to_device(case, env["dev"])
    fw, obs = case.fw, case.obs
    geo = (_Dj(case), obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3])
    ub = api.cost_sinkhorn(env["h"], TILT, ob, ms, eps, case.c_out, 40, dust_mode=2, harvest=False, kappa=4.0,
                           lam=4.0)
    sp = api.cost_sinkhorn_sparse(env["h"], TILT, ob, ms, eps, case.c_out, 60, rho=8, harvest=False,
                                  neighbours=True)
    env["torch"].cuda.synchronize()
    assert env["h"].device_status() == 0
    fu, gu = oracle.sinkhorn_unbalanced(*geo, eps, 4.0, 4.0, 40)
    fs, gs, fds, gds = oracle.sinkhorn_sparse(*geo, eps, case.c_out, 0, 0.4, 60, 8)
    nbr = oracle.knn(*geo, 8)
    np.testing.assert_array_equal(sp["nbr"].cpu().numpy(), nbr)
    for got, want in ((ub["f"], fu), (ub["g"], gu), (sp["f"], fs), (sp["g"], gs)):
        got = got.cpu().numpy().astype(np.float64)
        assert np.all(np.abs(got - want) <= TOL * (np.abs(want) + eps))


def _estep_case(seed, n_grains=None, T=None, eps=1.0, name="tiny"):
    case = make_case(sg.CONFIGS[name], seed=seed, n_grains=n_grains, T=T, geom=TILT)
    rng = np.random.default_rng(seed + 100)
    R0 = f32(np.array([_rotvec(rng.normal(size=3) * math.radians(0.2) / math.sqrt(3)) @ a for a in case.R]))
    x0 = f32(case.x + rng.normal(size=case.x.shape) * 0.1)
    fw = oracle.forward(TILT, case.planes, R0, x0, case.om)
    for k in ("ray", "spot", "center"):
        fw[k] = f32(fw[k])
    case.fw = fw
    obs = case.obs
    f, g, *_ = oracle.sinkhorn(_Dj(case), obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], eps,
                               case.c_out, 0, 0.4, 100)
    return case, R0, x0, f32(f), f32(g), eps


@pytest.mark.parametrize("kind", ["plain", "adjoint"])
def test_msteps_tilted(env, kind):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    case, R0, x0, f, g, eps = _estep_case(31, n_grains=40, T=10, name="medium")
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    R = _t(env, R0.reshape(-1, 9))
    x = _t(env, x0)
    fn = api.mstep if kind == "plain" else api.mstep_adjoint
    fn(env["h"], TILT, lat, ob, ms, _t(env, f), _t(env, g), eps, _t(env, case.om), R, x)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    Rg = R.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
    xg = x.cpu().numpy().astype(np.float64)
    fw, obs = case.fw, case.obs
    args = (TILT, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"], fw["center"],
            fw["ray"][:, :3], f, g, eps, R0, x0)
    if kind == "plain":
        Ro, xo, _ = oracle.mstep(*args, det=fw["det"])
    else:
        Ro, xo, _ = oracle.mstep_adjoint(*args, n_steps=4, lam=1e-3, det=fw["det"])
    assert np.all(_mis_deg(Rg, Ro) < 1e-3), _mis_deg(Rg, Ro).max()
    assert np.abs(xg - xo).max() < 1e-3
    assert np.abs(xo - x0).max() > 1e-3


def test_objective_grad_tilted(env):
    api = env["api"]
    case, R0, x0, f, g, eps = _estep_case(32, eps=2.0, name="adjoint")
    ob, ms = to_device(case, env["dev"])
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=env["dev"])
    grad, val = api.objective_grad(env["h"], TILT, lat, ob, ms, _t(env, f), _t(env, g), eps, _t(env, case.om),
                                   _t(env, R0.reshape(-1, 9)), _t(env, x0))
    grad = grad.cpu().numpy().astype(np.float64)
    fw, obs = case.fw, case.obs
    ref = oracle.grain_grad(TILT, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"],
                            f, g, eps, R0, x0, det=fw["det"])
    for part in (slice(0, 3), slice(3, 6)):
        gr, gg = ref[:, part], grad[:, part]
        lim = 1e-3 * np.abs(gr).max(axis=1, keepdims=True) + 1e-4 * np.abs(gr).max()
        assert np.all(np.abs(gg - gr) <= lim), float((np.abs(gg - gr) / lim).max())


def test_single_fit_and_spot_tilted(env):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    case = make_case(sg.CONFIGS["tiny"], seed=33, geom=TILT)
    rng = np.random.default_rng(34)
    near_R = f32(np.array([_rotvec(rng.normal(size=3) * math.radians(1.0) / math.sqrt(3)) @ a for a in case.R]))
    near_x = f32(case.x + rng.normal(size=case.x.shape) * 0.3)
    ob = api.ObsSpots.from_numpy(case.obs.p, case.obs.I_off, device=dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    Ro, xo, keep, unm = api.single_fit(env["h"], TILT, lat, ob, _t(env, case.om), _t(env, near_R), _t(env, near_x),
                                       1.0, 20, case.c_out)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    Rg = Ro.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
    xg = xo.cpu().numpy().astype(np.float64)
    Rr, xr, kr, ur = oracle.single_fit(TILT, case.planes, case.om, case.obs.p, case.obs.I_off, near_R, near_x, 1.0,
                                       20, case.c_out)
    assert kr.all() and keep.cpu().numpy().all()
    assert np.all(_mis_deg(Rg, Rr) < 1e-3)
    assert np.abs(xg - xr).max() < 1e-3
    np.testing.assert_allclose(unm.cpu().numpy(), ur, atol=1e-6)
    # SPOT on the truth plus random candidates: the truth is selected, k* = 5
    rnd_R, rnd_x = sg.random_grains(case.cfg, rng)
    cR = np.concatenate([f32(rnd_R), case.R])
    cx = np.concatenate([f32(rnd_x), case.x])
    order, gains, ks = api.prototype_select(env["h"], TILT, lat, ob, _t(env, case.om), _t(env, cR), _t(env, cx), 1.0,
                                            case.c_out, len(cR))
    torch.cuda.synchronize()
    Lbar = oracle.spot_matrix(TILT, case.planes, case.om, case.obs.p, case.obs.I_off, cR, cx, 1.0, case.c_out)
    o_ref, g_ref, _ = oracle.spot_greedy(Lbar, len(cR))
    gains = gains.cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(gains[:len(g_ref)], g_ref, atol=1e-4 * g_ref.max())
    assert ks == oracle.kstar(g_ref) == len(case.R)
    assert sorted(order.cpu().numpy()[:ks].tolist()) == sorted(o_ref[:ks].tolist())


def test_em_and_index_tilted(env):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    from paper_2404_06478_gb300.em import EMConfig, EMSolver
    case = make_case(sg.CONFIGS["tiny"], seed=35, geom=TILT)
    rng = np.random.default_rng(36)
    R0 = f32(np.array([_rotvec(rng.normal(size=3) * math.radians(0.3) / math.sqrt(3)) @ a for a in case.R]))
    x0 = f32(case.x + rng.normal(size=case.x.shape) * 0.1)
    fw = oracle.forward(TILT, case.planes, R0, x0, case.om)
    for k in ("ray", "spot", "center"):
        fw[k] = f32(fw[k])
    case.fw = fw
    ref = oracle.em(TILT, case.planes, case.om, case.obs.p, case.obs.I_off, fw["J_off"], fw["grain"], fw["plane"],
                    R0, x0, eps_final=1.0, n_em=12, n_sinkhorn=60, c_out=case.c_out, det=fw["det"])
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    cfg = EMConfig(eps_final=1.0, n_em=12, n_sinkhorn=60, c_out=case.c_out)
    solver = EMSolver(env["h"], TILT, lat, ob, ms, _t(env, case.om), cfg)
    R, x = _t(env, R0.reshape(-1, 9)), _t(env, x0)
    solver.run(R, x)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    Rg = R.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
    assert np.all(_mis_deg(Rg, ref["R"]) < 1e-3)
    assert np.abs(x.cpu().numpy() - ref["x"]).max() < 1e-3
    # laue_index from starts near the truth and random starts recovers every grain
    near_R = f32(np.array([_rotvec(rng.normal(size=3) * math.radians(1.0) / math.sqrt(3)) @ a for a in case.R]))
    near_x = f32(case.x + rng.normal(size=case.x.shape) * 0.3)
    rnd_R, rnd_x = sg.random_grains(case.cfg, rng)
    sR = np.concatenate([near_R, f32(rnd_R)])
    sx = np.concatenate([near_x, f32(rnd_x)])
    Rk, xk, _ = api.index(env["h"], TILT, lat, ob, _t(env, case.om), _t(env, sR), _t(env, sx), 1.0, case.c_out, 16)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    Rk = Rk.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
    xk = xk.cpu().numpy().astype(np.float64)
    assert len(Rk) == len(case.R)
    for n in range(len(case.R)):
        # misorientation up to the cubic symmetry of the crystal
        d = np.min([_mis_deg(np.repeat(case.R[n:n + 1], len(Rk), 0), Rk @ S[None]) for S in _cubic()], axis=0)
        k = int(np.argmin(d))
        assert d[k] < 0.5 and np.linalg.norm(xk[k] - case.x[n]) < 0.5, (n, d[k])
