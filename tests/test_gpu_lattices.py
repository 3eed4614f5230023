"""Non-cubic lattices on the GPU path: the trigonal and hexagonal start grids
against the oracle's, the forward model of a ruby (R-3c) cell against the
oracle's, and end-to-end indexing of a ruby polycrystal from the library's
trigonal start grid."""
import dataclasses
import math

import numpy as np
import pytest

import oracle
import synthgen as sg
from _cases import GEOM, f32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2404_06478_gb300 import api, build
    build.build()
    dev = torch.device("cuda", 0)
    return dict(torch=torch, api=api, dev=dev, h=api.Handle(dev))


def _ruby():
    c = sg.RUBY
    B = oracle.reciprocal_basis(c.a, c.b, c.c, c.alpha, c.beta, c.gamma)
    return B, sg.ruby_hkl(4, 12)


def _d3():
    def rot(w):
        th = float(np.linalg.norm(w))
        k = np.asarray(w) / th
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
        return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K
    out = [np.eye(3), rot([0, 0, 2 * math.pi / 3]), rot([0, 0, 4 * math.pi / 3])]
    for q in range(3):
        phi = math.pi * q / 3
        out.append(rot(np.array([math.cos(phi), math.sin(phi), 0.0]) * math.pi))
    return out


@pytest.mark.parametrize("sym", [6, 12])
def test_dihedral_start_grids_match_oracle(env, sym):
    R, x = env["api"].start_grid(env["h"], 120000, sym=sym, k=2, cube_mm=4.0)
    env["torch"].cuda.synchronize()
    Ro, xo = oracle.start_grid(120000, sym=sym, k=2, cube=4.0)
    assert R.shape[0] == len(Ro)
    np.testing.assert_allclose(R.cpu().numpy().reshape(-1, 3, 3), Ro, atol=2e-6)
    np.testing.assert_allclose(x.cpu().numpy(), xo, atol=1e-6)


def test_ruby_forward_matches_oracle(env):
    """The forward model with the ruby plane table (general B, R-3c
    reflections): the same visible spots as the oracle's, positions within
    1e-3 mm (20 grains, 15 rotations)."""
    torch, api, dev = env["torch"], env["api"], env["dev"]
    B, hkl = _ruby()
    P = oracle.reflections_hkl(B, hkl)
    P32 = oracle.Planes(f32(P.w), f32(P.d0), P.nharm, P.hkl0)
    rng = np.random.default_rng(3)
    R = f32(sg.random_rotations(20, rng))
    x = f32(rng.uniform(-2.5, 2.5, (20, 3)))
    om = f32(np.radians(np.arange(15) * 24.0))
    fw = oracle.forward(GEOM, P32, R, x, om)
    lat = api.Lattice.from_hkl(B, hkl, device=dev)
    ms = api.forward(env["h"], GEOM, lat, torch.tensor(R.reshape(-1, 9), dtype=torch.float32, device=dev),
                     torch.tensor(x, dtype=torch.float32, device=dev), torch.tensor(om, dtype=torch.float32, device=dev))
    torch.cuda.synchronize()
    assert ms.n == fw["J_off"][-1]
    np.testing.assert_array_equal(ms.J_off.cpu().numpy(), fw["J_off"])
    np.testing.assert_array_equal(ms.plane[:ms.n].cpu().numpy(), fw["plane"])
    np.testing.assert_allclose(ms.spot[:ms.n, :3].cpu().numpy(), fw["spot"], atol=1e-3)


def test_ruby_polycrystal_indexed_from_the_trigonal_grid(env):
    """5 ruby grains, 12 rotations over 180 deg, 0.5 mm noise, 10% outliers:
    laue_index from the library's start grid restricted to the fundamental zone
    of the trigonal group (600k spiral points, 100k orientations) finds every
    grain within 0.5 deg (symmetry aware) and 0.3 mm."""
    torch, api, dev = env["torch"], env["api"], env["dev"]
    B, hkl = _ruby()
    P = oracle.reflections_hkl(B, hkl)
    cfg = dataclasses.replace(sg.CONFIGS["tiny"], n_grains=5, T=12, hmax=4)
    rng = np.random.default_rng(8)
    R, x = sg.random_grains(cfg, rng)
    om = sg.omegas(cfg)
    fw = oracle.forward(GEOM, P, R, x, om)
    obs = sg.observe(GEOM, cfg, fw["t"], fw["det"], fw["spot"], rng)
    ob = api.ObsSpots.from_numpy(obs.p, obs.I_off, device=dev)
    lat = api.Lattice.from_hkl(B, hkl, device=dev)
    omt = torch.tensor(om, dtype=torch.float32, device=dev)
    c_out = api.c_out_for(0.5, GEOM.D)
    Rf, xf, _ = api.index(env["h"], GEOM, lat, ob, omt, None, None, 1.0, c_out, 40, n_em=20, n_sinkhorn=100,
                          k_single=30, anneal_single=400.0, recut_single=True,
                          grid=dict(n_full=600_000, sym=6, k=1, cube_mm=5.0))
    torch.cuda.synchronize()
    assert env["h"].device_status() == 0
    Rf = Rf.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
    xf = xf.cpu().numpy().astype(np.float64)
    assert len(Rf) == 5
    syms = _d3()
    for n in range(5):
        best, dx = 180.0, 1e9
        for k in range(len(Rf)):
            for S in syms:
                M = (Rf[k] @ S).T @ R[n]
                ang = math.degrees(math.acos(max(-1.0, min(1.0, (np.trace(M) - 1) / 2))))
                if ang < best:
                    best, dx = ang, float(np.linalg.norm(xf[k] - x[n]))
        assert best < 0.5 and dx < 0.3, (n, best, dx)
