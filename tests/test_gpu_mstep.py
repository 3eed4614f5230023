"""Parity of laue_mstep (Newton on positions, MM/Wahba on orientations) and
laue_objective_grad (adjoint of the OT-weighted cost) with the FP64 oracle.

Both sides get the same float32 inputs and the same E-step potentials (the
oracle's, rounded to float32).  Pose tolerance: 1e-3 deg misorientation and
1e-3 mm.  Gradient tolerance: 1e-3 of the largest component per grain plus
1e-4 of the largest over all grains (FP32 sums of Q-weighted terms)."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synthgen as sg
from _cases import GEOM, f32, make_case, planes32, to_device

pytestmark = pytest.mark.gpu


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


def _misorientation_deg(A, B):
    """Angle of A^T B, well conditioned near 0: atan2(|axial part|, (tr - 1)/2)."""
    M = np.einsum("nji,njk->nik", A, B)
    ax = np.stack([M[:, 2, 1] - M[:, 1, 2], M[:, 0, 2] - M[:, 2, 0], M[:, 1, 0] - M[:, 0, 1]], -1) / 2
    c = (np.trace(M, axis1=1, axis2=2) - 1) / 2
    return np.degrees(np.arctan2(np.linalg.norm(ax, axis=1), c))


def _estep_case(cfg, seed, n_grains=None, T=None, eps=1.0, rot_deg=0.2, dx=0.1):
    """Observed spots from the truth, model list frozen at perturbed poses,
    oracle potentials of a 100-iteration E-step at those poses."""
    case = make_case(cfg, seed=seed, n_grains=n_grains, T=T)
    rng = np.random.default_rng(seed + 100)
    R0 = f32(np.array([_rotvec(rng.normal(size=3) * math.radians(rot_deg) / math.sqrt(3)) @ a for a in case.R]))
    x0 = f32(case.x + rng.normal(size=case.x.shape) * dx)
    fw = oracle.forward(GEOM, case.planes, R0, x0, case.om)
    for k in ("ray", "spot", "center"):
        fw[k] = f32(fw[k])
    case.fw = fw
    obs = case.obs
    f, g, fd, gd, _ = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3],
                                      eps, case.c_out, 0, 0.4, 100)
    return case, R0, x0, f32(f), f32(g), eps


def _gpu_mstep(env, case, R0, x0, f, g, eps, n_newton=4, n_mm=4):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    R = torch.tensor(R0.reshape(-1, 9), dtype=torch.float32, device=dev).contiguous()
    x = torch.tensor(x0, dtype=torch.float32, device=dev).contiguous()
    norms = torch.zeros(len(x0), 2, device=dev)
    api.mstep(env["h"], GEOM, lat, ob, ms, torch.tensor(f, dtype=torch.float32, device=dev),
              torch.tensor(g, dtype=torch.float32, device=dev), eps, torch.tensor(case.om, dtype=torch.float32,
                                                                                 device=dev),
              R, x, n_newton=n_newton, n_mm=n_mm, step_norms=norms)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    return R.cpu().numpy().reshape(-1, 3, 3).astype(np.float64), x.cpu().numpy().astype(np.float64), norms


@pytest.mark.parametrize("name,n_grains,T,seed", [("tiny", None, None, 1), ("medium", 40, 10, 2)])
def test_mstep_parity(env, name, n_grains, T, seed):
    case, R0, x0, f, g, eps = _estep_case(sg.CONFIGS[name], seed, n_grains, T)
    Rg, xg, _ = _gpu_mstep(env, case, R0, x0, f, g, eps)
    fw, obs = case.fw, case.obs
    Ro, xo, st = oracle.mstep(GEOM, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"],
                              fw["center"], fw["ray"][:, :3], f, g, eps, R0, x0)
    assert np.all(_misorientation_deg(Rg, Ro) < 1e-3)
    assert np.abs(xg - xo).max() < 1e-3
    # the step actually moved the grains
    assert np.abs(xo - x0).max() > 1e-3


def test_mstep_newton_only_and_mm_only(env):
    case, R0, x0, f, g, eps = _estep_case(sg.CONFIGS["tiny"], 3)
    fw, obs = case.fw, case.obs
    for nn, nm in ((2, 0), (0, 3)):
        Rg, xg, _ = _gpu_mstep(env, case, R0, x0, f, g, eps, n_newton=nn, n_mm=nm)
        Ro, xo, _ = oracle.mstep(GEOM, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"],
                                 fw["plane"], fw["center"], fw["ray"][:, :3], f, g, eps, R0, x0, n_newton=nn,
                                 n_mm=nm)
        assert np.all(_misorientation_deg(Rg, Ro) < 1e-3)
        assert np.abs(xg - xo).max() < 1e-3


def _gpu_grad(env, case, R, x, f, g, eps):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()
    grad, val = api.objective_grad(env["h"], GEOM, lat, ob, ms, t(f), t(g), eps, t(case.om), t(R.reshape(-1, 9)),
                                   t(x))
    return grad.cpu().numpy().astype(np.float64), val.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("name,n_grains,T", [("tiny", None, None), ("adjoint", None, None)])
def test_objective_grad_parity(env, name, n_grains, T):
    """Gradient of sum Q C w.r.t. axis-angle and position (50 grains, 20
    rotations for the adjoint configuration)."""
    case, R0, x0, f, g, eps = _estep_case(sg.CONFIGS[name], 4, n_grains, T, eps=2.0)
    fw, obs = case.fw, case.obs
    ref = oracle.grain_grad(GEOM, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"],
                            f, g, eps, R0, x0)
    val_ref = oracle.grain_objective(GEOM, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"],
                                     fw["plane"], fw["center"], fw["ray"][:, :3], f, g, eps, R0, x0)
    grad, val = _gpu_grad(env, case, R0, x0, f, g, eps)
    for part in (slice(0, 3), slice(3, 6)):
        gr, gg = ref[:, part], grad[:, part]
        lim = 1e-3 * np.abs(gr).max(axis=1, keepdims=True) + 1e-4 * np.abs(gr).max()
        assert np.all(np.abs(gg - gr) <= lim), float((np.abs(gg - gr) / lim).max())
    np.testing.assert_allclose(val, val_ref, rtol=1e-4, atol=1e-4 * np.abs(val_ref).max())


def test_autograd_function_matches_oracle(env):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    from paper_2404_06478_gb300.autograd import ot_weighted_cost
    case, R0, x0, f, g, eps = _estep_case(sg.CONFIGS["tiny"], 5, eps=2.0)
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()
    w = torch.zeros(len(x0), 3, device=dev, requires_grad=True)
    x = t(x0).requires_grad_(True)
    E = ot_weighted_cost(w, x, t(R0.reshape(-1, 9)), env["h"], GEOM, lat, ob, ms, t(f), t(g), eps, t(case.om))
    E.sum().backward()
    fw, obs = case.fw, case.obs
    ref = oracle.grain_grad(GEOM, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"],
                            f, g, eps, R0, x0)
    gw, gx = w.grad.cpu().numpy(), x.grad.cpu().numpy()
    np.testing.assert_allclose(gw, ref[:, :3], rtol=1e-3, atol=1e-4 * np.abs(ref[:, :3]).max())
    np.testing.assert_allclose(gx, ref[:, 3:], rtol=1e-3, atol=1e-4 * np.abs(ref[:, 3:]).max())


def test_autograd_function_at_nonzero_axis_angle(env):
    """The same function at w != 0, where the axis-angle chain rule
    (laue_axis_angle_vjp) matters: dE/dw and dE/dx equal FP64 central
    differences of the oracle's objective in w and x (Q held at the plan of the
    poses R(w) = exp([w]x) R0, x), with an upstream gradient gout != 1."""
    torch, api, dev = env["torch"], env["api"], env["dev"]
    from paper_2404_06478_gb300.autograd import ot_weighted_cost
    case, Rb, x0, f, g, eps = _estep_case(sg.CONFIGS["tiny"], 6, eps=2.0)
    rng = np.random.default_rng(61)
    w0 = f32(rng.normal(size=(len(x0), 3)) * 0.3)
    R0 = f32(np.array([_rotvec(-w) @ a for w, a in zip(w0, Rb)]))  # so that R(w0) ~ Rb
    Rw = np.array([_rotvec(w) @ a for w, a in zip(w0, R0)])
    fw = oracle.forward(GEOM, case.planes, Rw, x0, case.om)
    # the model list of the E-step case, refreshed at R(w0) (same labels)
    ray, ce = oracle.refresh(GEOM, case.planes, Rw, x0, case.om, case.fw["J_off"], case.fw["grain"],
                             case.fw["plane"])
    case.fw["ray"], case.fw["center"] = f32(ray), f32(ce)
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()
    w = t(w0).requires_grad_(True)
    x = t(x0).requires_grad_(True)
    gout = f32(rng.uniform(0.5, 2.0, size=len(x0)))
    E = ot_weighted_cost(w, x, t(R0.reshape(-1, 9)), env["h"], GEOM, lat, ob, ms, t(f), t(g), eps, t(case.om))
    (E * t(gout)).sum().backward()
    obs, cf = case.obs, case.fw
    args = (GEOM, case.planes, case.om, obs.p, obs.I_off, cf["J_off"], cf["grain"], cf["plane"], ce, ray[:, :3],
            f, g, eps)
    h = 1e-6
    FD = np.zeros((len(x0), 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Rp = np.array([_rotvec(w + e[:3]) @ a for w, a in zip(w0, R0)])
        Rm = np.array([_rotvec(w - e[:3]) @ a for w, a in zip(w0, R0)])
        FD[:, k] = (oracle.grain_objective(*args, Rp, x0 + e[3:]) - oracle.grain_objective(*args, Rm, x0 - e[3:])) / (2 * h)
    FD *= gout[:, None]
    gw, gx = w.grad.cpu().numpy(), x.grad.cpu().numpy()
    assert fw["J_off"][-1] > 0
    np.testing.assert_allclose(gw, FD[:, :3], rtol=1e-3, atol=1e-4 * np.abs(FD[:, :3]).max())
    np.testing.assert_allclose(gx, FD[:, 3:], rtol=1e-3, atol=1e-4 * np.abs(FD[:, 3:]).max())


@pytest.mark.parametrize("name,n_grains,T,seed", [("tiny", None, None, 21), ("medium", 40, 10, 22)])
def test_mstep_adjoint_parity(env, name, n_grains, T, seed):
    """The adjoint M-step (damped Gauss-Newton on the OT-weighted cost, plan
    held at the E-step) equals the oracle's: 4 steps from poses 0.2 deg /
    0.1 mm off the truth, within 1e-3 deg and 1e-3 mm, and it moves the grains."""
    torch, api, dev = env["torch"], env["api"], env["dev"]
    case, R0, x0, f, g, eps = _estep_case(sg.CONFIGS[name], seed, n_grains, T)
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev).contiguous()
    R, x = t(R0.reshape(-1, 9)), t(x0)
    norms = torch.zeros(len(x0), 2, device=dev)
    api.mstep_adjoint(env["h"], GEOM, lat, ob, ms, t(f), t(g), eps, t(case.om), R, x, n_steps=4, lam=1e-3,
                      step_norms=norms)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    Rg = R.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
    xg = x.cpu().numpy().astype(np.float64)
    fw, obs = case.fw, case.obs
    Ro, xo, no = oracle.mstep_adjoint(GEOM, case.planes, case.om, obs.p, obs.I_off, fw["J_off"], fw["grain"],
                                      fw["plane"], fw["center"], fw["ray"][:, :3], f, g, eps, R0, x0, n_steps=4,
                                      lam=1e-3)
    assert np.all(_misorientation_deg(Rg, Ro) < 1e-3), _misorientation_deg(Rg, Ro).max()
    assert np.abs(xg - xo).max() < 1e-3
    assert np.abs(xo - x0).max() > 1e-3
    # the steps shrink: the last step is far below the first move
    assert float(norms[:, 0].max()) < 0.5 * np.abs(xo - x0).max() + 1e-4


@pytest.mark.parametrize("adjoint", [False, True])
def test_mstep_skipping_is_bit_identical(env, adjoint):
    """The M-step pair passes skip, by the cone bounds, the observed granules
    whose every plan entry is below 2^-40, the entries their sums leave out:
    poses and step norms are bit-identical with the skipping on or off, and
    fewer pairs are visited.  Workload: the 1000-grain density on 4 angles
    with potentials from 30 Sinkhorn iterations at eps = 1 mm^2 (checked
    elsewhere against the oracle)."""
    torch, api, dev, h = env["torch"], env["api"], env["dev"], env["h"]
    case = make_case(sg.CONFIGS["batched"], seed=0, T=4)
    ob, ms = to_device(case, dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    om = torch.tensor(case.om, dtype=torch.float32, device=dev)
    pot = api.cost_sinkhorn(h, GEOM, ob, ms, 1.0, case.c_out, 30, harvest=False)
    runs = {}
    try:
        for skip in (False, True):
            h.set_pair_skipping(skip)
            R = torch.tensor(case.R.reshape(-1, 9), dtype=torch.float32, device=dev).contiguous()
            x = torch.tensor(case.x, dtype=torch.float32, device=dev).contiguous()
            norms = torch.zeros(len(case.x), 2, device=dev)
            h.counters()
            if adjoint:
                api.mstep_adjoint(h, GEOM, lat, ob, ms, pot["f"], pot["g"], 1.0, om, R, x, n_steps=2,
                                  step_norms=norms)
            else:
                api.mstep(h, GEOM, lat, ob, ms, pot["f"], pot["g"], 1.0, om, R, x, n_newton=2, n_mm=2,
                          step_norms=norms)
            torch.cuda.synchronize()
            assert h.device_status() == 0
            runs[skip] = (R, x, norms, h.counters()["mstep_pairs"])
    finally:
        h.set_pair_skipping(True)
    (Ra, xa, na, pa), (Rb, xb, nb, pb) = runs[False], runs[True]
    assert torch.equal(Ra, Rb) and torch.equal(xa, xb) and torch.equal(na, nb)
    nI, nJ = np.diff(case.obs.I_off), np.diff(case.fw["J_off"])
    dense = int(np.sum((nI + nI % 2) * (nJ + nJ % 2)))
    assert pa > 0 and pa % dense == 0, (pa, dense)
    assert pb < 0.5 * pa, (pb, pa)
