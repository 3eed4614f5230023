"""Parity of laue_prototype_select (sparse grain-to-spot matrix, greedy
facility-location selection, k*) with the FP64 oracle's naive greedy.

The increments must agree within 1e-4 of the largest increment; k* must be
equal; the chosen prototypes must agree up to exchanging a grain with its
near-duplicate (several greedy orders are then equally valid: the test compares
which true grain each pick covers, and checks the increments)."""
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


def _gpu_select(env, case, cR, cx, eps_s, k_max):
    torch, api, dev = env["torch"], env["api"], env["dev"]
    ob = api.ObsSpots.from_numpy(case.obs.p, case.obs.I_off, device=dev)
    lat = api.Lattice.cubic(case.cfg.a, case.cfg.hmax, case.cfg.centering, device=dev)
    t = lambda a: torch.tensor(np.asarray(a), dtype=torch.float32, device=dev)
    order, gains, ks = api.prototype_select(env["h"], GEOM, lat, ob, t(case.om), t(cR), t(cx), eps_s, case.c_out,
                                            k_max)
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    return order.cpu().numpy(), gains.cpu().numpy().astype(np.float64), ks


@pytest.mark.parametrize("name,n_grains,T,seed", [("tiny", None, None, 5), ("medium", 25, 20, 6)])
def test_spot_parity(env, name, n_grains, T, seed):
    case = make_case(sg.CONFIGS[name], seed=seed, n_grains=n_grains, T=T)
    rng = np.random.default_rng(seed + 50)
    R, x = case.R, case.x
    n = len(R)
    dup_R = f32(np.array([_rotvec(rng.normal(size=3) * 0.003) @ a for a in R]))
    dup_x = f32(x + rng.normal(size=x.shape) * 0.05)
    rnd_R, rnd_x = sg.random_grains(case.cfg, rng)
    cR = np.concatenate([dup_R, f32(rnd_R), R])
    cx = np.concatenate([dup_x, f32(rnd_x), x])
    k_max = len(cR)
    order, gains, ks = _gpu_select(env, case, cR, cx, 1.0, k_max)
    Lbar = oracle.spot_matrix(GEOM, case.planes, case.om, case.obs.p, case.obs.I_off, cR, cx, 1.0, case.c_out)
    o_ref, g_ref, F_ref = oracle.spot_greedy(Lbar, k_max)
    k_ref = oracle.kstar(g_ref)
    np.testing.assert_allclose(gains, g_ref, atol=1e-4 * g_ref.max())
    assert ks == k_ref == n
    cover = lambda o: sorted(int(v) % n for v in o[:n])
    assert cover(order) == cover(o_ref) == list(range(n))
    assert sorted(order.tolist()) == list(range(k_max))


def test_spot_edge_cases(env):
    case = make_case(sg.CONFIGS["tiny"], seed=7)
    # fewer steps than candidates, one candidate, zero candidates
    order, gains, ks = _gpu_select(env, case, case.R, case.x, 1.0, 3)
    assert len(order) == 3 and len(set(order.tolist())) == 3 and ks in (2, 3)
    order, gains, ks = _gpu_select(env, case, case.R[:1], case.x[:1], 1.0, 1)
    assert order.tolist() == [0] and ks == 1
    order, gains, ks = _gpu_select(env, case, np.zeros((0, 3, 3)), np.zeros((0, 3)), 1.0, 0)
    assert ks == 0
