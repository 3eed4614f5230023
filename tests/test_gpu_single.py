"""Parity of laue_single_fit (batched SingleLaueOT + f_out filter) with the
FP64 oracle.  Fits that converge are compared pose by pose (1e-3 deg,
1e-3 mm); the keep decisions must agree wherever the oracle's unmatched
fraction is not within 0.05 of the threshold."""
import math

import numpy as np
import pytest

import oracle
import synthgen as sg
from _cases import GEOM, f32, make_case

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
    k = np.asarray(w) / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def _mis_deg(A, B):
    M = np.einsum("nji,njk->nik", A, B)
    ax = np.stack([M[:, 2, 1] - M[:, 1, 2], M[:, 0, 2] - M[:, 2, 0], M[:, 1, 0] - M[:, 0, 1]], -1) / 2
    return np.degrees(np.arctan2(np.linalg.norm(ax, axis=1), (np.trace(M, axis1=1, axis2=2) - 1) / 2))


def _gpu_fit(env, case, R0, x0, k_max=20):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    ob = api.ObsSpots.from_numpy(case.obs.p, case.obs.I_off, device=dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev)
    Ro, xo, keep, unm = api.single_fit(env["h"], GEOM, lat, ob, t(case.om), t(R0), t(x0), 1.0, k_max, case.c_out)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    return (Ro.cpu().numpy().reshape(-1, 3, 3).astype(np.float64), xo.cpu().numpy().astype(np.float64),
            keep.cpu().numpy(), unm.cpu().numpy().astype(np.float64))


def test_single_fit_parity_tiny(env):
    case = make_case(sg.CONFIGS["tiny"], seed=3)
    rng = np.random.default_rng(17)
    near_R = f32(np.array([_rotvec(rng.normal(size=3) * math.radians(1.0) / math.sqrt(3)) @ a for a in case.R]))
    near_x = f32(case.x + rng.normal(size=case.x.shape) * 0.3)
    rnd_R, rnd_x = sg.random_grains(case.cfg, rng)
    R0 = np.concatenate([near_R, f32(rnd_R)])
    x0 = np.concatenate([near_x, f32(rnd_x)])
    Rg, xg, kg, ug = _gpu_fit(env, case, R0, x0)
    Ro, xo, ko, uo = oracle.single_fit(GEOM, case.planes, case.om, case.obs.p, case.obs.I_off, R0, x0, 1.0, 20,
                                       case.c_out)
    n = len(near_R)
    assert ko[:n].all() and kg[:n].all()
    assert np.all(_mis_deg(Rg[:n], Ro[:n]) < 1e-3)
    assert np.abs(xg[:n] - xo[:n]).max() < 1e-3
    sure = np.abs(uo - 0.1) > 0.05
    np.testing.assert_array_equal(kg[sure], ko[sure])
    np.testing.assert_allclose(ug[:n], uo[:n], atol=1e-6)


def test_single_fit_medium_blocks(env):
    """60 rotations, |hkl| <= 6, 40 grains: angle blocks of ~700 observed spots
    (several warps per block row), ~470 listed spots per start."""
    case = make_case(sg.CONFIGS["medium"], seed=5, n_grains=40, T=60)
    rng = np.random.default_rng(23)
    R0 = f32(np.array([_rotvec(rng.normal(size=3) * math.radians(0.7) / math.sqrt(3)) @ a for a in case.R[:6]]))
    x0 = f32(case.x[:6] + rng.normal(size=(6, 3)) * 0.2)
    Rg, xg, kg, ug = _gpu_fit(env, case, R0, x0, k_max=8)
    Ro, xo, ko, uo = oracle.single_fit(GEOM, case.planes, case.om, case.obs.p, case.obs.I_off, R0, x0, 1.0, 8,
                                       case.c_out)
    conv = ko.astype(bool)
    assert conv.sum() >= 4
    assert np.all(_mis_deg(Rg[conv], Ro[conv]) < 1e-3)
    assert np.abs(xg[conv] - xo[conv]).max() < 1e-3


def test_single_fit_edge_cases(env):
    case = make_case(sg.CONFIGS["tiny"], seed=4)
    # no starts
    Rg, xg, kg, ug = _gpu_fit(env, case, np.zeros((0, 3, 3)), np.zeros((0, 3)))
    assert len(kg) == 0
    # a start far outside the sample: its spots still fall on the detectors,
    # nothing matches, the filter rejects it
    Rg, xg, kg, ug = _gpu_fit(env, case, case.R[:1], np.array([[40.0, 0.0, 0.0]]), k_max=3)
    assert not kg[0]
