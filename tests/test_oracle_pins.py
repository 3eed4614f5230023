"""Pins of the FP64 oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a worked
example printed in the paper or derived from Bragg's law, closed forms,
invariants, a library routine (LAPACK, the Hungarian algorithm, an LP solver)
or brute force on tiny inputs.  None of these runs on a GPU.
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

import oracle
import synthgen as sg

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GEOM = sg.Geometry()
TINY = sg.CONFIGS["tiny"]


def _rotvec(w):
    th = float(np.linalg.norm(w))
    if th == 0.0:
        return np.eye(3)
    k = np.asarray(w) / th
    K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]])
    return np.eye(3) + math.sin(th) * K + (1 - math.cos(th)) * K @ K


def _cubic_group():
    mats = []
    for perm in itertools.permutations(range(3)):
        for signs in itertools.product([1, -1], repeat=3):
            S = np.zeros((3, 3))
            for r, c in enumerate(perm):
                S[r, c] = signs[r]
            if np.linalg.det(S) > 0:
                mats.append(S)
    return mats


@pytest.fixture(scope="module")
def tiny():
    planes = oracle.reflections(TINY.a, TINY.hmax, TINY.centering)
    rng = sg.workload_seed(TINY)
    R, x = sg.random_grains(TINY, rng)
    om = sg.omegas(TINY)
    fw = oracle.forward(GEOM, planes, R, x, om)
    obs = sg.observe(GEOM, TINY, fw["t"], fw["det"], fw["spot"], rng)
    return dict(planes=planes, R=R, x=x, om=om, fw=fw, obs=obs)


# ---------------------------------------------------------------- reflections

def test_reflection_table_covers_every_allowed_hkl_once():
    """Brute force: every allowed hkl within the bound is n * g0 of exactly one
    direction (up to the Friedel sign), n <= nharm, and no two directions are
    parallel."""
    for hmax, count in ((4, 145), (6, 433)):
        P = oracle.reflections(2.87, hmax, 1)
        assert len(P.w) == count
        g0 = P.hkl0
        seen = {}
        for m in range(len(g0)):
            for n in range(1, P.nharm[m] + 1):
                for s in (1, -1):
                    key = tuple(int(v) for v in s * n * g0[m])
                    seen[key] = seen.get(key, 0) + 1
        allowed = {(h, k, l) for h, k, l in itertools.product(range(-hmax, hmax + 1), repeat=3)
                   if (h, k, l) != (0, 0, 0) and (h + k + l) % 2 == 0}
        assert set(seen) == allowed
        assert all(v == 1 for v in seen.values())
        W = P.w
        cosines = np.abs(W @ W.T) - np.eye(len(W))
        assert cosines.max() < 1 - 1e-9
        np.testing.assert_allclose(P.d0, 2.87 / np.linalg.norm(g0, axis=1), rtol=1e-14)


# -------------------------------------------------------------------- forward

def test_forward_worked_example():
    gold = json.load(open(os.path.join(GOLD, "forward_worked_example.json")))
    P = oracle.reflections(gold["lattice_a"], 4, 1)
    m = [i for i, h in enumerate(P.hkl0) if list(h) == gold["hkl0"]]
    assert len(m) == 1
    sub = oracle.Planes(P.w[m], P.d0[m], P.nharm[m], P.hkl0[m])
    assert sub.d0[0] == pytest.approx(gold["d0"], rel=1e-12)
    fw = oracle.forward(GEOM, sub, np.eye(3)[None], np.zeros((1, 3)), np.zeros(1))
    assert fw["J_off"][-1] == 1
    assert fw["ray"][0, 3] == pytest.approx(gold["lambda"], rel=1e-12)
    np.testing.assert_allclose(fw["ray"][0, :3], gold["ray"], atol=1e-12)
    np.testing.assert_allclose(fw["spot"][0], gold["spot"], atol=1e-9)
    assert fw["det"][0] == gold["detector"]


def test_gamma_is_rotation_about_y():
    G0 = oracle.gamma(0.0)
    np.testing.assert_allclose(G0, np.eye(3), atol=0)
    for om in (0.3, 2.0, -1.1):
        G = oracle.gamma(om)
        np.testing.assert_allclose(G @ G.T, np.eye(3), atol=1e-15)
        assert np.linalg.det(G) == pytest.approx(1.0, abs=1e-15)
        np.testing.assert_allclose(G @ [0, 1, 0], [0, 1, 0], atol=1e-15)
        # right-handed: a small positive rotation about y takes +z towards +x
    assert (oracle.gamma(0.1) @ [0, 0, 1])[0] > 0


def test_forward_spots_satisfy_laue_and_bragg(tiny):
    """Every visible spot: unit ray; Laue condition k_out = k_in - 2(k_in.g)g with
    g = Gamma R w_m; Bragg n lambda = 2 d sin(theta) with theta read from the
    scattering angle; spot on its detector plane, inside the square, on the ray
    from the grain centre."""
    fw, P, R, x, om = tiny["fw"], tiny["planes"], tiny["R"], tiny["x"], tiny["om"]
    e = np.array(GEOM.beam)
    assert fw["J_off"][-1] > 100
    for j in range(fw["J_off"][-1]):
        t, n, m = fw["t"][j], fw["grain"][j], fw["plane"][j]
        r, lam = fw["ray"][j, :3], fw["ray"][j, 3]
        assert np.linalg.norm(r) == pytest.approx(1.0, abs=1e-14)
        Gm = oracle.gamma(om[t])
        g = Gm @ R[n] @ P.w[m]
        np.testing.assert_allclose(r, e - 2 * (e @ g) * g, atol=1e-13)
        theta = 0.5 * math.acos(np.clip(e @ r, -1, 1))
        ok = [k for k in range(1, P.nharm[m] + 1)
              if abs(k * lam - 2 * P.d0[m] * math.sin(theta)) < 1e-9]
        assert ok, (j, lam)
        assert GEOM.lam_min <= lam <= GEOM.lam_max
        det = GEOM.detectors[fw["det"][j]]
        s = fw["spot"][j]
        assert s[2] == pytest.approx(det.centre[2], abs=1e-9)
        assert abs(s[0]) < det.half and abs(s[1]) < det.half
        c = Gm @ x[n]
        np.testing.assert_allclose(fw["center"][j], c, atol=1e-13)
        d = s - c
        assert np.linalg.norm(np.cross(d, r)) < 1e-9 and d @ r > 0


def test_forward_invariant_under_cubic_symmetry(tiny):
    """The spot multiset of a cubic grain does not change under R -> R S for the
    24 proper rotations of the cube (Section 'Pre-processing': the search is
    restricted by the crystal symmetries)."""
    P, R, x, om = tiny["planes"], tiny["R"], tiny["x"], tiny["om"]
    base = oracle.forward(GEOM, P, R[:2], x[:2], om)
    key = lambda fw: np.array(sorted(map(tuple, np.round(
        np.c_[fw["t"], fw["grain"], fw["spot"], fw["ray"][:, 3]], 8))))
    k0 = key(base)
    for S in _cubic_group():
        fw = oracle.forward(GEOM, P, R[:2] @ S, x[:2], om)
        np.testing.assert_allclose(key(fw), k0, atol=2e-8)


def test_sigma_conversion_matches_paper():
    gold = json.load(open(os.path.join(GOLD, "sigma_conversion.json")))
    for case in gold["cases"]:
        deg = math.degrees(case["sigma_mm"] / case["distance_mm"])
        assert round(deg, gold["printed_digits"]) == case["sigma_deg"]


def test_outlier_cost_is_three_sigma_pair_cost():
    """c_out is the pair cost of a ray 3 sigma away: ~9 sigma_mm^2 for small
    angles, and exactly D^2 |a - b|^2 for unit rays 3 sigma_ang apart."""
    c = oracle.c_out_for(0.5, 200.0)
    assert c == pytest.approx(9 * 0.25, rel=1e-5)
    ang = 3 * 0.5 / 200.0
    a = np.array([0, 0, 1.0]); b = np.array([math.sin(ang), 0, math.cos(ang)])
    assert c == pytest.approx(200.0 ** 2 * np.sum((a - b) ** 2), rel=1e-9)


# ----------------------------------------------------------------------- cost

def test_noiseless_truth_has_zero_cost(tiny):
    fw = tiny["fw"]
    for j in range(fw["J_off"][-1]):
        C = oracle.pair_cost(fw["spot"][j], fw["center"][j], fw["ray"][j, :3], GEOM.D)
        assert C < 1e-20


def test_cost_is_angle_between_rays():
    rng = np.random.default_rng(5)
    for _ in range(50):
        p = rng.normal(size=3) * 100; c = rng.normal(size=3)
        r = rng.normal(size=3); r /= np.linalg.norm(r)
        a = (p - c) / np.linalg.norm(p - c)
        ang = math.atan2(np.linalg.norm(np.cross(a, r)), a @ r)
        assert oracle.pair_cost(p, c, r, 200.0) == pytest.approx(
            2 * 200.0 ** 2 * (1 - math.cos(ang)), rel=1e-9, abs=1e-9)


# ------------------------------------------------------------------- Sinkhorn

def _plan(D, p, I_off, J_off, c, r, eps, cout, f, g):
    """Dense real-pair block of the plan from potentials (for the tests)."""
    Q = np.zeros((len(p), len(c)))
    T = len(I_off) - 1
    for t in range(T):
        for i in range(I_off[t], I_off[t + 1]):
            for j in range(J_off[t], J_off[t + 1]):
                Q[i, j] = math.exp((f[i] + g[j] - oracle.pair_cost(p[i], c[j], r[j], D)) / eps)
    return Q


@pytest.mark.parametrize("mode", [0, 1])
def test_sinkhorn_marginals_converge(tiny, mode):
    fw, obs = tiny["fw"], tiny["obs"]
    cout = oracle.c_out_for(0.5, GEOM.D)
    f, g, fd, gd, it = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"],
                                       fw["ray"][:, :3], 1.0, cout, mode, 0.4, 5000, 1e-12)
    assert it < 5000
    h = oracle.harvest(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3],
                       1.0, cout, mode, 0.4, f, g, fd, gd)
    assert h["row_err"] < 1e-10 and h["col_err"] < 1e-10


def test_sinkhorn_single_pair_closed_form():
    """|I| = |J| = 1 in one block: U = O = 1 and the 2 x 2 extended plan has
    Q_11 Q_00 / (Q_10 Q_01) = exp(-(C + c_out - c_out - 0)/eps), hence
    Q_11 = 1 / (1 + exp(C / (2 eps)))."""
    p = np.array([[3.0, -2.0, -200.0]]); c = np.array([[0.5, 0.2, -0.1]])
    r = np.array([[0.02, -0.01, -1.0]]); r /= np.linalg.norm(r)
    C = oracle.pair_cost(p[0], c[0], r[0], 200.0)
    for eps in (0.5, 2.0, 10.0):
        f, g, fd, gd, _ = oracle.sinkhorn(200.0, p, [0, 1], [0, 1], c, r, eps, 2.25, 0, 0.4,
                                          10000, 1e-14)
        Q11 = math.exp((f[0] + g[0] - C) / eps)
        assert Q11 == pytest.approx(1 / (1 + math.exp(C / (2 * eps))), rel=1e-10)


def test_sinkhorn_large_eps_is_independent_coupling():
    """One angle block, eps -> inf: Q -> a b^T / sum(a) on the extended matrix."""
    rng = np.random.default_rng(1)
    nI, nJ = 7, 5
    p = np.c_[rng.uniform(-50, 50, (nI, 2)), -200 * np.ones(nI)]
    c = rng.uniform(-2, 2, (nJ, 3))
    r = np.c_[rng.normal(size=(nJ, 2)) * 0.2, -np.ones(nJ)]
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    U, O = oracle.masses(0, 0.4, [0, nI], [0, nJ])
    f, g, fd, gd, _ = oracle.sinkhorn(200.0, p, [0, nI], [0, nJ], c, r, 1e12, 2.25, 0, 0.4, 5000, 1e-13)
    Q = _plan(200.0, p, [0, nI], [0, nJ], c, r, 1e12, 2.25, f, g)
    np.testing.assert_allclose(Q, 1.0 / (nI + U[0]), rtol=1e-6)


def test_sinkhorn_small_eps_matches_hungarian():
    """eps -> 0: the plan's row argmax equals the optimal assignment of the
    capacity-expanded square problem (rows: observed + U copies of the
    unmatched-model source; columns: model + O copies of the outlier sink),
    solved by the Hungarian algorithm and checked by brute force when tiny."""
    from scipy.optimize import linear_sum_assignment
    rng = np.random.default_rng(7)
    for trial in range(6):
        T = 2
        nIt = [rng.integers(2, 5) for _ in range(T)]
        nJt = [rng.integers(2, 4) for _ in range(T)]
        I_off = np.r_[0, np.cumsum(nIt)]; J_off = np.r_[0, np.cumsum(nJt)]
        nI, nJ = I_off[-1], J_off[-1]
        c = rng.uniform(-2, 2, (nJ, 3))
        r = np.c_[rng.normal(size=(nJ, 2)) * 0.1, -np.ones(nJ)]
        r /= np.linalg.norm(r, axis=1, keepdims=True)
        p = np.zeros((nI, 3))
        for t in range(T):
            for i in range(I_off[t], I_off[t + 1]):
                j = rng.integers(J_off[t], J_off[t + 1])
                tau = (-200 - c[j, 2]) / r[j, 2]
                p[i] = c[j] + tau * r[j] + np.r_[rng.normal(size=2) * 1.5, 0]
        cout = 2.25
        U, O = oracle.masses(0, 0.4, I_off, J_off)
        U, O = int(U[0]), int(O[0])
        BIG = 1e6
        n = nI + U
        Cm = np.full((n, n), BIG)
        for t in range(T):
            for i in range(I_off[t], I_off[t + 1]):
                for j in range(J_off[t], J_off[t + 1]):
                    Cm[i, j] = oracle.pair_cost(p[i], c[j], r[j], 200.0)
        Cm[:nI, nJ:] = cout
        Cm[nI:, :nJ] = 0.0
        Cm[nI:, nJ:] = cout
        rows, cols = linear_sum_assignment(Cm)
        ref = np.where(cols[:nI] < nJ, cols[:nI], -1)
        if n <= 8:
            best = min(itertools.permutations(range(n)), key=lambda s: sum(Cm[a, s[a]] for a in range(n)))
            assert sum(Cm[a, best[a]] for a in range(n)) == pytest.approx(Cm[rows, cols].sum())
        # unique optimum required for an argmax comparison
        eps = 0.01
        f, g, fd, gd, _ = oracle.sinkhorn(200.0, p, I_off, J_off, c, r, eps, cout, 0, 0.4, 200000, 1e-9)
        h = oracle.harvest(200.0, p, I_off, J_off, c, r, eps, cout, 0, 0.4, f, g, fd, gd)
        np.testing.assert_array_equal(h["assign"], ref)


def test_per_angle_equals_global_for_one_block(tiny):
    fw, obs = tiny["fw"], tiny["obs"]
    t0 = 3
    i0, i1 = obs.I_off[t0], obs.I_off[t0 + 1]
    j0, j1 = fw["J_off"][t0], fw["J_off"][t0 + 1]
    args = (GEOM.D, obs.p[i0:i1], [0, i1 - i0], [0, j1 - j0], fw["center"][j0:j1],
            fw["ray"][j0:j1, :3], 1.0, 2.25)
    a = oracle.sinkhorn(*args, 0, 0.4, 50)
    b = oracle.sinkhorn(*args, 1, 0.4, 50)
    for u, v in zip(a[:4], b[:4]):
        np.testing.assert_array_equal(u, v)


# --------------------------------------------------------------------- M-step

def test_sym3_eig_matches_lapack():
    rng = np.random.default_rng(3)
    for _ in range(20):
        A = rng.normal(size=(3, 3)); A = A + A.T
        ev, V = oracle.sym3_eig(A)
        np.testing.assert_allclose(ev, np.linalg.eigvalsh(A), atol=1e-12)
        np.testing.assert_allclose(A @ V, V @ np.diag(ev), atol=1e-11)


def test_svd3_matches_lapack():
    rng = np.random.default_rng(4)
    for k in range(20):
        B = rng.normal(size=(3, 3))
        if k % 4 == 0:
            B[:, 2] = B[:, 0] + B[:, 1]  # rank 2
        U, S, V = oracle.svd3(B)
        np.testing.assert_allclose(S, np.linalg.svd(B, compute_uv=False), atol=1e-12)
        np.testing.assert_allclose(U @ np.diag(S) @ V.T, B, atol=1e-12)
        np.testing.assert_allclose(U.T @ U, np.eye(3), atol=1e-12)


def test_wahba_recovers_rotation_exactly():
    """Kabsch: noiseless correspondences a_k = R b_k give R back, including
    the determinant correction when the unconstrained optimum is a reflection."""
    rng = np.random.default_rng(2)
    for _ in range(10):
        Rt = sg.random_rotations(1, rng)[0]
        b = rng.normal(size=(6, 3)); a = b @ Rt.T
        w = rng.uniform(0.5, 2, 6)
        B = (w[:, None, None] * a[:, :, None] * b[:, None, :]).sum(0)
        np.testing.assert_allclose(oracle.wahba(B), Rt, atol=1e-12)
    # planar data: rank 2, the reflection branch must be excluded
    b = np.c_[rng.normal(size=(5, 2)), np.zeros(5)]
    Rt = sg.random_rotations(1, rng)[0]
    B = (Rt @ b.T) @ b
    Rh = oracle.wahba(B)
    assert np.linalg.det(Rh) == pytest.approx(1.0)
    np.testing.assert_allclose(Rh @ b.T, Rt @ b.T, atol=1e-12)
    # rank 1 keeps R (returns None)
    assert oracle.wahba(np.outer([1, 2, 3], [0, 1, 0])) is None


def _noiseless_assignment(seed=0):
    planes = oracle.reflections(TINY.a, TINY.hmax, TINY.centering)
    rng = np.random.default_rng(seed)
    R, x = sg.random_grains(TINY, rng)
    om = sg.omegas(TINY)
    fw = oracle.forward(GEOM, planes, R, x, om)
    # observed = the true spots themselves, in model order (no noise/outliers)
    p = fw["spot"].copy()
    I_off = fw["J_off"].copy()
    return planes, R, x, om, fw, p, I_off


def test_newton_recovers_true_position_with_ground_truth_plan():
    """Q = the true assignment (pure assignment problem: no dustbin mass, small
    eps): Newton moves a displaced grain back to the true x within 3 steps."""
    planes, R, x, om, fw, p, I_off = _noiseless_assignment(0)
    c, r = fw["center"], fw["ray"][:, :3]
    f, g, fd, gd, _ = oracle.sinkhorn(GEOM.D, p, I_off, fw["J_off"], c, r, 0.05, 2.25, 0, 0.0,
                                      2000, 1e-12)
    Q = _plan(GEOM.D, p, I_off, fw["J_off"], c, r, 0.05, 2.25, f, g)
    np.testing.assert_allclose(np.diag(Q), 1.0, atol=1e-9)
    rng = np.random.default_rng(11)
    x0 = x + rng.normal(size=x.shape) * 0.2
    R1, x1, st = oracle.mstep(GEOM, planes, om, p, I_off, fw["J_off"], fw["grain"], fw["plane"],
                              c, r, f, g, 0.05, R, x0, n_newton=3, n_mm=0)
    np.testing.assert_allclose(x1, x, atol=1e-7)


def test_newton_gradient_matches_finite_differences():
    """The Newton objective Phi(x) = sum Q rhat.r: the gradient the step uses is
    checked through the adjoint's x-part (dE/dx = -2 D^2 dPhi/dx)."""
    planes, R, x, om, fw, p, I_off = _noiseless_assignment(1)
    rng = np.random.default_rng(12)
    p = p + np.c_[rng.normal(size=(len(p), 2)) * 0.5, np.zeros(len(p))]
    c, r = fw["center"], fw["ray"][:, :3]
    args = (GEOM, planes, om, p, I_off, fw["J_off"], fw["grain"], fw["plane"])
    f, g, fd, gd, _ = oracle.sinkhorn(GEOM.D, p, I_off, fw["J_off"], c, r, 2.0, 2.25, 0, 0.4, 100)
    G = oracle.grain_grad(*args, f, g, 2.0, R, x)
    h = 1e-6
    FD = np.zeros_like(G)
    for k in range(6):
        e = np.zeros(6); e[k] = h
        Rp = np.array([_rotvec(e[:3]) @ a for a in R]); Rm = np.array([_rotvec(-e[:3]) @ a for a in R])
        Ep = oracle.grain_objective(*args, c, r, f, g, 2.0, Rp, x + e[3:])
        Em = oracle.grain_objective(*args, c, r, f, g, 2.0, Rm, x - e[3:])
        FD[:, k] = (Ep - Em) / (2 * h)
    assert np.abs(G - FD).max() <= 1e-7 * np.abs(G).max()


def test_mm_never_decreases_objective(tiny):
    """Majorisation-minimisation is monotone (appendix 'Grain rotation')."""
    P, R, x, om, fw, obs = (tiny[k] for k in ("planes", "R", "x", "om", "fw", "obs"))
    rng = np.random.default_rng(9)
    Rp = np.array([_rotvec(rng.normal(size=3) * 0.01) @ a for a in R])
    ray, ce = oracle.refresh(GEOM, P, Rp, x, om, fw["J_off"], fw["grain"], fw["plane"])
    f, g, fd, gd, _ = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], ce, ray[:, :3], 3.0,
                                      2.25, 0, 0.4, 100)
    for k_mm in (1, 2, 4):
        _, _, st = oracle.mstep(GEOM, P, om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"],
                                ce, ray[:, :3], f, g, 3.0, Rp, x, n_newton=0, n_mm=k_mm)
        assert np.all(st[:, 5] >= st[:, 4] - 1e-9 * np.abs(st[:, 4]))


def test_em_fixed_point_at_noiseless_truth():
    """Noiseless data, grains at the truth, plan without dustbin mass: the EM
    step leaves the poses where they are."""
    planes, R, x, om, fw, p, I_off = _noiseless_assignment(2)
    out = oracle.em(GEOM, planes, om, p, I_off, fw["J_off"], fw["grain"], fw["plane"], R, x,
                    eps_final=1e-4, n_em=2, n_sinkhorn=300, c_out=2.25, mode=0, frac=0.0)
    np.testing.assert_allclose(out["x"], x, atol=1e-9)
    np.testing.assert_allclose(out["R"], R, atol=1e-10)
    np.testing.assert_array_equal(out["assign"], np.arange(len(p)))


def test_em_recovers_perturbed_grains(tiny):
    """Tiny workload with noise and outliers: EM from poses perturbed by
    ~0.2 deg / 0.1 mm ends within 0.05 deg of the true orientations; with 0.5 mm
    spot noise over 10 rotations the positions are noise-limited (< 0.5 mm)."""
    P, R, x, om, fw, obs = (tiny[k] for k in ("planes", "R", "x", "om", "fw", "obs"))
    rng = np.random.default_rng(21)
    Rp = np.array([_rotvec(rng.normal(size=3) * 0.002) @ a for a in R])
    xp = x + rng.normal(size=x.shape) * 0.1
    out = oracle.em(GEOM, P, om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"], Rp, xp,
                    eps_final=1.0, n_em=10, n_sinkhorn=100, c_out=oracle.c_out_for(0.5, GEOM.D))
    for Ra, Rb in zip(out["R"], R):
        ang = math.degrees(math.acos(np.clip((np.trace(Ra.T @ Rb) - 1) / 2, -1, 1)))
        assert ang < 0.05
    assert np.abs(out["x"] - x).max() < 0.5


# ----------------------------------------------------------------------- SPOT

def test_spot_closed_form_equals_lp():
    """f(S) = sum_i max_{n in S} Lbar_in equals the LP max <Lbar, P> over plans
    with P 1 = a and support on S (source weights free)."""
    from scipy.optimize import linprog
    rng = np.random.default_rng(0)
    nI, Nc = 6, 4
    Lbar = np.maximum(0, rng.normal(size=(nI, Nc)))
    for S in ([0], [1, 3], [0, 2, 3]):
        nv = nI * len(S)
        cvec = -np.array([Lbar[i, n] for i in range(nI) for n in S])
        A = np.zeros((nI, nv))
        for i in range(nI):
            A[i, i * len(S):(i + 1) * len(S)] = 1
        res = linprog(cvec, A_eq=A, b_eq=np.ones(nI), bounds=(0, None), method="highs")
        order, gain, F = oracle.spot_greedy(Lbar[:, S], len(S))
        assert -res.fun == pytest.approx(F[-1], rel=1e-12)


def test_spot_greedy_submodular_guarantees():
    """Greedy gains are non-increasing (submodularity), each prefix is the
    greedy answer for the smaller cardinality, and the value is at least
    (1 - 1/e) of the exhaustive optimum (Nemhauser et al.)."""
    rng = np.random.default_rng(1)
    for trial in range(5):
        nI, Nc = 15, 10
        Lbar = np.maximum(0, rng.normal(size=(nI, Nc)) + 0.3)
        order, gain, F = oracle.spot_greedy(Lbar, Nc)
        assert np.all(np.diff(gain) <= 1e-12)
        for k in range(1, 5):
            o2, _, _ = oracle.spot_greedy(Lbar, k)
            np.testing.assert_array_equal(o2, order[:k])
            best = max(np.maximum.reduce([Lbar[:, n] for n in S]).sum()
                       for S in itertools.combinations(range(Nc), k))
            assert F[k - 1] >= (1 - 1 / math.e) * best - 1e-12
            # the first step is exact
            if k == 1:
                assert F[0] == pytest.approx(best)


def test_kstar_finds_true_count_on_duplicates(tiny):
    """Candidates = the true grains, perturbed duplicates and random grains: the
    largest drop of the greedy increments sits at the true grain count."""
    P, R, x, om, obs = (tiny[k] for k in ("planes", "R", "x", "om", "obs"))
    rng = np.random.default_rng(5)
    dup_R = np.array([_rotvec(rng.normal(size=3) * 0.003) @ a for a in R])
    dup_x = x + rng.normal(size=x.shape) * 0.05
    rnd_R, rnd_x = sg.random_grains(TINY, rng)
    cR = np.concatenate([dup_R, rnd_R, R]); cx = np.concatenate([dup_x, rnd_x, x])
    Lbar = oracle.spot_matrix(GEOM, P, om, obs.p, obs.I_off, cR, cx, 1.0, 2.25)
    order, gain, F = oracle.spot_greedy(Lbar, len(cR))
    k = oracle.kstar(gain)
    assert k == len(R)
    chosen = order[:k] % len(R)
    assert sorted(chosen) == list(range(len(R)))


# ------------------------------------------------------------ single-grain fit

def test_single_fit_recovers_near_starts_and_filter_rejects_random(tiny):
    """Algorithm SingleLaueOT: a start within ~1 deg / 0.5 mm of a true grain
    converges to it and passes the f_out filter; random starts fail it."""
    P, R, x, om, obs = (tiny[k] for k in ("planes", "R", "x", "om", "obs"))
    rng = np.random.default_rng(31)
    R0 = np.array([_rotvec(rng.normal(size=3) * math.radians(1.0) / math.sqrt(3)) @ a for a in R])
    x0 = x + rng.normal(size=x.shape) * 0.5
    Ro, xo, keep, unm = oracle.single_fit(GEOM, P, om, obs.p, obs.I_off, R0, x0, 1.0, 20, 2.25)
    for Ra, Rb in zip(Ro, R):
        assert math.degrees(math.acos(np.clip((np.trace(Ra.T @ Rb) - 1) / 2, -1, 1))) < 0.1
    assert keep.all() and np.abs(xo - x).max() < 0.5
    Rr, xr = sg.random_grains(TINY, rng)
    _, _, keep_r, unm_r = oracle.single_fit(GEOM, P, om, obs.p, obs.I_off, Rr, xr, 1.0, 20, 2.25)
    assert not keep_r.any() and unm_r.min() > 0.5


def test_adjoint_gradient_fd_50_grains_20_rotations():
    """The adjoint configuration (50 grains, 20 rotations): the oracle's analytic
    gradient of sum Q C equals FP64 central differences with h = 1e-6."""
    cfg = sg.CONFIGS["adjoint"]
    P = oracle.reflections(cfg.a, cfg.hmax, cfg.centering)
    rng = sg.workload_seed(cfg)
    R, x = sg.random_grains(cfg, rng)
    om = sg.omegas(cfg)
    fw = oracle.forward(GEOM, P, R, x, om)
    obs = sg.observe(GEOM, cfg, fw["t"], fw["det"], fw["spot"], rng)
    c, r = fw["center"], fw["ray"][:, :3]
    f, g, fd, gd, _ = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], c, r, 2.0, 2.25, 0, 0.4, 30)
    args = (GEOM, P, om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"])
    G = oracle.grain_grad(*args, f, g, 2.0, R, x)
    h = 1e-6
    FD = np.zeros_like(G)
    for k in range(6):
        e = np.zeros(6); e[k] = h
        Rp = np.array([_rotvec(e[:3]) @ a for a in R]); Rm = np.array([_rotvec(-e[:3]) @ a for a in R])
        Ep = oracle.grain_objective(*args, c, r, f, g, 2.0, Rp, x + e[3:])
        Em = oracle.grain_objective(*args, c, r, f, g, 2.0, Rm, x - e[3:])
        FD[:, k] = (Ep - Em) / (2 * h)
    assert np.abs(G - FD).max() <= 1e-6 * np.abs(G).max()


# ------------------------------------------------ corners pinned by hand

def test_spot_matrix_by_hand_two_angles():
    """Grain-to-spot matrix (App. "Selection of prototypes", read as the gain
    over the outlier baseline) on a constructed case whose value follows from
    geometry alone.  The grain sits at the origin with R = I.  At omega = 0 its
    (0,0,-2) reflection sends the ray r = (0,0,-1) straight back to (0,0,-200).
    Observed spot 0 (angle 0) lies at (200 tan(th), 0, -200), so its ray estimate
    makes the angle th with r and C = 4 D^2 sin^2(th/2); every other model spot
    of that angle is far away, so Lbar = (c_out - C)/eps_s to rounding.
    Observed spot 1 has the same coordinates at angle 1 (omega = 30 deg), where no
    model spot is near: it must get 0 (it would get spot 0's value if spots of
    another angle counted).  Observed spot 2 (angle 0) is far from every spot: 0.
    A mis-signed baseline gives 0 for spot 0 instead of a positive gain."""
    P = oracle.reflections(2.87, 4, 1)
    om = np.array([0.0, math.radians(30.0)])
    R, x = np.eye(3)[None], np.zeros((1, 3))
    th = math.radians(0.1)
    p0 = np.array([200.0 * math.tan(th), 0.0, -200.0])
    far = np.array([60.0, -50.0, -200.0])
    fw = oracle.forward(GEOM, P, R, x, om)
    J = fw["J_off"]
    # preconditions read off the forward model: the straight-back spot exists at
    # angle 0, every other spot is > 15 mm from p0 (both angles) and from `far`
    s0 = fw["spot"][J[0]:J[1]]
    k0 = np.argmin(np.linalg.norm(s0 - [0, 0, -200.0], axis=1))
    np.testing.assert_allclose(s0[k0], [0, 0, -200.0], atol=1e-9)
    np.testing.assert_allclose(fw["ray"][J[0] + k0, :3], [0, 0, -1.0], atol=1e-12)
    others0 = np.delete(s0, k0, axis=0)
    assert np.linalg.norm(others0 - p0, axis=1).min() > 15.0
    assert np.linalg.norm(fw["spot"][J[1]:J[2]] - p0, axis=1).min() > 15.0
    assert np.linalg.norm(s0 - far, axis=1).min() > 15.0
    pobs = np.array([p0, p0, far])
    I_off = [0, 2, 3]  # spots 0 and 2 at angle 0, spot 1 at angle 1
    pobs = pobs[[0, 2, 1]]
    eps_s, c_out, D = 1.0, oracle.c_out_for(0.5, GEOM.D), GEOM.D
    L = oracle.spot_matrix(GEOM, P, om, pobs, I_off, R, x, eps_s, c_out)
    C = 4.0 * D * D * math.sin(th / 2) ** 2
    assert L.shape == (3, 1)
    assert L[0, 0] == pytest.approx((c_out - C) / eps_s, rel=1e-12)
    assert L[0, 0] > 0.5
    assert L[1, 0] == 0.0  # far spot at angle 0
    assert L[2, 0] == 0.0  # same coordinates as spot 0, but at angle 1


def test_masses_balance_when_model_spots_outnumber_observed():
    """Masses of the dustbins (Eq. estep_obj balance T_a = T_b - b^T 1 + a^T 1):
    with |J| > |I| + ceil(frac |J|) the outlier mass would be negative, so the
    unmatched mass rises to |J| - |I| and the outlier mass is 0.  Both readings
    keep total row mass = total column mass; Sinkhorn then meets every marginal
    (the outlier column carries nothing)."""
    I_off, J_off = [0, 2, 3], [0, 6, 10]
    U, O = oracle.masses(0, 0.4, I_off, J_off)
    assert (U[0], O[0]) == (7.0, 0.0)           # ceil(4) + 3 - 10 < 0 -> U = 10 - 3
    assert 3 + U[0] == 10 + O[0]
    Up, Op = oracle.masses(1, 0.4, I_off, J_off)  # per angle: (6, 2) and (4, 1)
    np.testing.assert_array_equal(Up, [4.0, 3.0])
    np.testing.assert_array_equal(Op, [0.0, 0.0])
    Uq, Oq = oracle.masses(0, 0.4, [0, 8], [0, 5])  # the ordinary branch
    assert (Uq[0], Oq[0]) == (2.0, 5.0)
    rng = np.random.default_rng(3)
    p = np.c_[rng.uniform(-20, 20, (3, 2)), -200 * np.ones(3)]
    c = rng.uniform(-1, 1, (10, 3))
    r = np.c_[rng.normal(size=(10, 2)) * 0.05, -np.ones(10)]
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    for mode in (0, 1):
        f, g, fd, gd, it = oracle.sinkhorn(200.0, p, I_off, J_off, c, r, 50.0, 2.25, mode, 0.4, 20000, 1e-13)
        h = oracle.harvest(200.0, p, I_off, J_off, c, r, 50.0, 2.25, mode, 0.4, f, g, fd, gd)
        assert h["row_err"] < 1e-10 and h["col_err"] < 1e-10
        assert np.all(h["assign"] >= 0)  # the outlier column has no mass to take


def test_refresh_equals_forward_at_the_same_pose(tiny):
    """Refreshing a frozen list (§"Assignments with outlier and missing spots")
    gives the forward model's rays, wavelengths and centres for every spot of the
    list, both at the pose that made the list and at a new pose (for the spots the
    forward model also lists there)."""
    P, fw, om = tiny["planes"], tiny["fw"], tiny["om"]
    R, x = tiny["R"], tiny["x"]
    ray, ce = oracle.refresh(GEOM, P, R, x, om, fw["J_off"], fw["grain"], fw["plane"])
    np.testing.assert_allclose(ray, fw["ray"], rtol=0, atol=1e-13)
    np.testing.assert_allclose(ce, fw["center"], rtol=0, atol=1e-13)
    rng = np.random.default_rng(4)
    R2 = np.array([_rotvec(rng.normal(size=3) * 0.01) @ a for a in R])
    x2 = x + rng.normal(size=x.shape) * 0.2
    ray2, ce2 = oracle.refresh(GEOM, P, R2, x2, om, fw["J_off"], fw["grain"], fw["plane"])
    fw2 = oracle.forward(GEOM, P, R2, x2, om)
    key2 = {(t, n, m): j for j, (t, n, m) in enumerate(zip(fw2["t"], fw2["grain"], fw2["plane"]))}
    hits = 0
    for j, k in enumerate(zip(fw["t"], fw["grain"], fw["plane"])):
        if k in key2:
            hits += 1
            np.testing.assert_allclose(ray2[j], fw2["ray"][key2[k]], rtol=0, atol=1e-13)
            np.testing.assert_allclose(ce2[j], fw2["center"][key2[k]], rtol=0, atol=1e-13)
    assert hits > 0.8 * len(fw["t"])


# ------------------------------------------------------------ start grid

def _mat_to_quat(R):
    """Unit quaternions (w >= 0) of rotation matrices (Shepperd's method)."""
    out = np.zeros((len(R), 4))
    for n, M in enumerate(R):
        tr = np.trace(M)
        cand = [1 + tr, 1 + 2 * M[0, 0] - tr, 1 + 2 * M[1, 1] - tr, 1 + 2 * M[2, 2] - tr]
        k = int(np.argmax(cand))
        v = math.sqrt(cand[k]) / 2
        if k == 0:
            q = [v, (M[2, 1] - M[1, 2]) / (4 * v), (M[0, 2] - M[2, 0]) / (4 * v), (M[1, 0] - M[0, 1]) / (4 * v)]
        elif k == 1:
            q = [(M[2, 1] - M[1, 2]) / (4 * v), v, (M[0, 1] + M[1, 0]) / (4 * v), (M[0, 2] + M[2, 0]) / (4 * v)]
        elif k == 2:
            q = [(M[0, 2] - M[2, 0]) / (4 * v), (M[0, 1] + M[1, 0]) / (4 * v), v, (M[1, 2] + M[2, 1]) / (4 * v)]
        else:
            q = [(M[1, 0] - M[0, 1]) / (4 * v), (M[0, 2] + M[2, 0]) / (4 * v), (M[1, 2] + M[2, 1]) / (4 * v), v]
        q = np.array(q)
        out[n] = q if q[0] >= 0 else -q
    return out


def test_start_grid_is_uniform_and_in_the_cubic_fundamental_zone():
    """Section "Single-grain fitting": quasi-uniform starts restricted by the
    lattice symmetry.  (1) The full spiral's second moments are those of the
    uniform distribution on the unit quaternions, E[q_a q_b] = delta_ab / 4.
    (2) With the cubic restriction, every kept orientation lies in the cubic
    fundamental zone as it is usually written in Rodrigues space (|r_i| <=
    sqrt(2) - 1 and |r_1| + |r_2| + |r_3| <= 1, r = q_v / q_w), and 1/24 of the
    spiral is kept.  (3) Every rotation has a start within the covering radius
    of a set of that size (symmetry aware).  (4) Positions: the k^3 cell centres."""
    R, x = oracle.start_grid(96000, sym=1, k=1)
    q = _mat_to_quat(R)
    M = np.einsum("na,nb->ab", q * np.sign(q[:, :1] + 1e-300), q * np.sign(q[:, :1] + 1e-300)) / len(q)
    np.testing.assert_allclose(M, np.eye(4) / 4, atol=2e-3)
    np.testing.assert_allclose(x, 0.0, atol=0)
    Rz, _ = oracle.start_grid(96000, sym=24, k=1)
    assert abs(len(Rz) - 96000 / 24) < 0.02 * 96000 / 24
    qz = _mat_to_quat(Rz)
    rod = qz[:, 1:] / qz[:, :1]
    assert np.all(np.abs(rod) <= math.sqrt(2) - 1 + 1e-9)
    assert np.all(np.abs(rod).sum(axis=1) <= 1 + 1e-9)
    # covering: 4000 kept orientations in a zone of volume pi^2/24 (quaternion
    # half-angle balls); no rotation is farther than 2x the ideal radius
    rng = np.random.default_rng(5)
    probes = sg.random_rotations(300, rng)
    syms = np.array(_cubic_group())
    worst = 0.0
    for P in probes:
        M = np.einsum("kji,jl->kil", Rz, P)
        best = np.full(len(Rz), 180.0)
        for S in syms:
            c = np.clip((np.trace(M @ S, axis1=1, axis2=2) - 1) / 2, -1, 1)
            best = np.minimum(best, np.degrees(np.arccos(c)))
        worst = max(worst, best.min())
    ideal = 2 * math.degrees((math.pi ** 2 / 24 / len(Rz) / (4 / 3 * math.pi)) ** (1 / 3))
    assert worst < 2 * ideal, (worst, ideal)
    Rk, xk = oracle.start_grid(2400, sym=24, k=3, cube=6.0)
    assert len(Rk) == 27 * len(oracle.start_grid(2400, sym=24, k=1)[0])
    np.testing.assert_allclose(np.unique(xk[:, 0]), [-2.0, 0.0, 2.0], atol=1e-12)
    np.testing.assert_allclose(Rk[0], Rk[26], atol=0)


# ------------------------------------------------------- adjoint M-step

def _one_grain_noiseless(seed=7, T=6):
    """One grain, |hkl| <= 4, its noiseless spots as the observed spots."""
    P = oracle.reflections(2.87, 4, 1)
    rng = np.random.default_rng(seed)
    R = sg.random_rotations(1, rng)
    x = rng.uniform(-2, 2, size=(1, 3))
    om = np.radians(np.arange(T) * 30.0)
    fw = oracle.forward(GEOM, P, R, x, om)
    return P, R, x, om, fw


def test_adjoint_gn_gradient_matches_finite_differences(tiny):
    """The gradient of orc_grain_gn at a pose away from the E-step pose (Q held
    at the E-step plan) equals FP64 central differences of the objective."""
    P, fw, obs, om = tiny["planes"], tiny["fw"], tiny["obs"], tiny["om"]
    c, r = fw["center"], fw["ray"][:, :3]
    f, g, *_ = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], c, r, 2.0, 2.25, 0, 0.4, 30)
    rng = np.random.default_rng(8)
    R1 = np.array([_rotvec(rng.normal(size=3) * 0.004) @ a for a in tiny["R"]])
    x1 = tiny["x"] + rng.normal(size=tiny["x"].shape) * 0.1
    args = (GEOM, P, om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"], c, r, f, g, 2.0)
    G, H, val = oracle.grain_gn(*args, R1, x1)
    np.testing.assert_allclose(val, oracle.grain_objective(*args, R1, x1), rtol=1e-12)
    h = 1e-6
    FD = np.zeros_like(G)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Rp = np.array([_rotvec(e[:3]) @ a for a in R1])
        Rm = np.array([_rotvec(-e[:3]) @ a for a in R1])
        FD[:, k] = (oracle.grain_objective(*args, Rp, x1 + e[3:]) - oracle.grain_objective(*args, Rm, x1 - e[3:])) / (2 * h)
    assert np.abs(G - FD).max() <= 1e-6 * np.abs(G).max()
    # the matrix is symmetric positive semi-definite
    np.testing.assert_allclose(H, H.transpose(0, 2, 1), atol=1e-9 * np.abs(H).max())
    assert np.linalg.eigvalsh(H).min() > -1e-9 * np.abs(H).max()


def test_adjoint_gn_matrix_is_jacobian_product_on_noiseless_pairs():
    """Where every observed spot sits on its model spot (noiseless, plan = the
    true matching), the Gauss-Newton matrix is exactly 2 D^2 sum_j J_j^T J_j
    with J_j the Jacobian of the residual rhat_j - r_j in (phi, x), here taken
    by FP64 central differences."""
    P, R, x, om, fw = _one_grain_noiseless()
    p, J_off = fw["spot"], fw["J_off"]
    c, r = fw["center"], fw["ray"][:, :3]
    nJ = int(J_off[-1])
    eps = 1e-4  # the plan is the identity matching to double precision
    f, g = np.zeros(nJ), np.zeros(nJ)
    args = (GEOM, P, om, p, J_off, J_off, fw["grain"], fw["plane"], c, r, f, g, eps)
    G, H, val = oracle.grain_gn(*args, R, x)
    assert np.abs(G).max() < 1e-6 and val[0] < 1e-12

    def residuals(dtheta):
        Rn = _rotvec(dtheta[:3]) @ R[0]
        ray, ce = oracle.refresh(GEOM, P, Rn[None], x + dtheta[3:], om, J_off, fw["grain"], fw["plane"])
        d = p - ce
        return (d / np.linalg.norm(d, axis=1, keepdims=True) - ray[:, :3]).ravel()

    h = 1e-6
    J = np.zeros((3 * nJ, 6))
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        J[:, k] = (residuals(e) - residuals(-e)) / (2 * h)
    want = 2 * GEOM.D ** 2 * J.T @ J
    np.testing.assert_allclose(H[0], want, rtol=1e-6, atol=1e-6 * np.abs(want).max())


def test_adjoint_mstep_converges_on_noiseless_data():
    """Started 0.5 deg and 0.3 mm from a noiseless grain, with the plan held at
    the true matching, the damped Gauss-Newton M-step returns to the truth."""
    P, R, x, om, fw = _one_grain_noiseless(seed=9)
    p, J_off = fw["spot"], fw["J_off"]
    nJ = int(J_off[-1])
    f, g = np.zeros(nJ), np.zeros(nJ)
    rng = np.random.default_rng(10)
    R0 = (_rotvec(rng.normal(size=3) * math.radians(0.5) / math.sqrt(3)) @ R[0])[None]
    x0 = x + rng.normal(size=3) * 0.3 / math.sqrt(3)
    Ro, xo, norms = oracle.mstep_adjoint(GEOM, P, om, p, J_off, J_off, fw["grain"], fw["plane"], fw["center"],
                                         fw["ray"][:, :3], f, g, 1e-4, R0, x0, n_steps=8)
    M = Ro[0].T @ R[0]
    assert math.degrees(math.acos(min(1.0, (np.trace(M) - 1) / 2))) < 1e-6
    assert np.abs(xo - x).max() < 1e-8


# ------------------------------------------------------- unbalanced OT

def test_unbalanced_fixed_point_is_the_marginal_kl_condition(tiny):
    """Problem (B) of App. "Optimal transport variants": at the optimum the
    potentials and the plan's marginals satisfy f_i = -kappa log(sum_j Q_ij)
    and g_j = -lambda log(sum_i Q_ij) (a = b = 1), the first-order conditions
    of the KL-relaxed marginals; the converged log-domain iteration meets them
    to 1e-9 (kappa on the observed rows, lambda on the model columns)."""
    fw, obs = tiny["fw"], tiny["obs"]
    for kappa, lam in ((2.0, 8.0), (20.0, 0.5)):
        f, g = oracle.sinkhorn_unbalanced(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3],
                                          4.0, kappa, lam, 3000)
        h = oracle.harvest_unbalanced(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], 4.0, f,
                                      g)
        # rows whose every plan entry underflows double precision are skipped
        okr, okc = h["rowmass"] > 1e-280, h["q"] > 1e-280
        assert okr.mean() > 0.8 and okc.mean() > 0.8
        np.testing.assert_allclose(f[okr], -kappa * np.log(h["rowmass"][okr]), atol=1e-9 * max(1.0, np.abs(f).max()))
        np.testing.assert_allclose(g[okc], -lam * np.log(h["q"][okc]), atol=1e-9 * max(1.0, np.abs(g).max()))


def test_unbalanced_large_kappa_lambda_is_balanced():
    """kappa, lambda -> infinity gives balanced OT: on a square block with no
    dustbin mass (frac = 0, |I| = |J|), the converged unbalanced iteration with
    kappa = lambda = 1e12 gives BalancedOT's plan (potentials equal up to the
    shift f + s, g - s that leaves a balanced plan unchanged), and the plan's
    marginals are 1."""
    rng = np.random.default_rng(2)
    n = 9
    p = np.c_[rng.uniform(-30, 30, (n, 2)), -200 * np.ones(n)]
    c = rng.uniform(-1, 1, (n, 3))
    r = np.c_[rng.normal(size=(n, 2)) * 0.1, -np.ones(n)]
    r /= np.linalg.norm(r, axis=1, keepdims=True)
    eps = 200.0
    fu, gu = oracle.sinkhorn_unbalanced(200.0, p, [0, n], [0, n], c, r, eps, 1e12, 1e12, 500)
    fb, gb, fd, gd, _ = oracle.sinkhorn(200.0, p, [0, n], [0, n], c, r, eps, 2.25, 0, 0.0, 500)
    # the same plan: the potentials differ by one constant shift (f + s, g - s)
    shift = np.mean(fu - fb)
    np.testing.assert_allclose(fu - fb, shift, atol=1e-5)
    np.testing.assert_allclose(gu - gb, -shift, atol=1e-5)
    h = oracle.harvest_unbalanced(200.0, p, [0, n], [0, n], c, r, eps, fu, gu)
    np.testing.assert_allclose(h["rowmass"], 1.0, atol=1e-8)
    np.testing.assert_allclose(h["q"], 1.0, atol=1e-8)


# ------------------------------------------------------- general lattices

def test_reflections_from_hkl_list_equal_the_cubic_table():
    """The general builder (reciprocal basis + list of allowed reflections)
    with B = I / a and the body-centred list reproduces the cubic table (entries,
    spacings, harmonics, order) that its own pins fix."""
    for hmax in (4, 6):
        P = oracle.reflections(2.87, hmax, 1)
        Q = oracle.reflections_hkl(np.eye(3) / 2.87, sg.bcc_hkl(hmax))
        np.testing.assert_array_equal(Q.hkl0, P.hkl0)
        np.testing.assert_array_equal(Q.nharm, P.nharm)
        np.testing.assert_allclose(Q.w, P.w, atol=1e-14)
        np.testing.assert_allclose(Q.d0, P.d0, rtol=1e-14)


def test_hexagonal_reciprocal_basis_and_spacings_closed_form():
    """Hexagonal cell (ruby): |b1| = |b2| = 2 / (a sqrt 3) at 60 degrees, b3 =
    (0, 0, 1/c); every entry's spacing obeys the textbook
    1/d^2 = 4 (h^2 + hk + k^2) / (3 a^2) + l^2 / c^2."""
    c = sg.RUBY
    B = oracle.reciprocal_basis(c.a, c.b, c.c, c.alpha, c.beta, c.gamma)
    b1, b2, b3 = B[:, 0], B[:, 1], B[:, 2]
    assert np.linalg.norm(b1) == pytest.approx(2 / (c.a * math.sqrt(3)), rel=1e-12)
    assert np.linalg.norm(b2) == pytest.approx(2 / (c.a * math.sqrt(3)), rel=1e-12)
    assert math.degrees(math.acos(b1 @ b2 / (np.linalg.norm(b1) * np.linalg.norm(b2)))) == pytest.approx(60.0, abs=1e-9)
    np.testing.assert_allclose(b3, [0, 0, 1 / c.c], atol=1e-15)
    P = oracle.reflections_hkl(B, sg.ruby_hkl(4, 12))
    h, k, l = P.hkl0[:, 0].astype(float), P.hkl0[:, 1].astype(float), P.hkl0[:, 2].astype(float)
    inv_d2 = 4 * (h * h + h * k + k * k) / (3 * c.a ** 2) + l * l / c.c ** 2
    np.testing.assert_allclose(P.d0, 1 / np.sqrt(inv_d2), rtol=1e-12)
    assert len(P.d0) > 50 and P.nharm.max() >= 2


def _d3():
    """The trigonal group 32 with the 3-fold axis along z and a 2-fold axis
    along x (hexagonal a1), as matrices."""
    out = []
    for q in range(3):
        out.append(_rotvec([0, 0, 2 * math.pi * q / 3]))
    for q in range(3):
        phi = math.pi * q / 3
        out.append(_rotvec(np.array([math.cos(phi), math.sin(phi), 0.0]) * math.pi))
    return out


def test_ruby_spots_are_invariant_under_the_trigonal_group():
    """With the ruby plane table, a grain at R and at R S for S in the trigonal
    group 32 make the same spots (the reflection list carries the crystal's
    symmetry); a 90-degree turn about c, which is not a symmetry of the cell,
    makes different ones."""
    c = sg.RUBY
    B = oracle.reciprocal_basis(c.a, c.b, c.c, c.alpha, c.beta, c.gamma)
    P = oracle.reflections_hkl(B, sg.ruby_hkl(4, 12))
    rng = np.random.default_rng(31)
    R = sg.random_rotations(1, rng)[0]
    x = np.array([0.3, -0.7, 1.1])
    om = np.radians(np.arange(8) * 22.5)

    def spots(Rm):
        fw = oracle.forward(GEOM, P, Rm[None], x[None], om)
        key = np.c_[fw["t"], np.round(fw["spot"], 6)]
        return key[np.lexsort(key.T[::-1])]

    ref = spots(R)
    assert len(ref) > 20
    for S in _d3():
        np.testing.assert_allclose(spots(R @ S), ref, atol=1e-6)
    other = spots(R @ _rotvec([0, 0, math.pi / 2]))
    assert other.shape != ref.shape or np.abs(other - ref).max() > 1.0


@pytest.mark.parametrize("sym,n_axis", [(6, 3), (12, 6)])
def test_start_grid_dihedral_fundamental_zone(sym, n_axis):
    """Start grids for the trigonal (32) and hexagonal (622) groups keep 1/6 and
    1/12 of the spiral, and every kept orientation lies in the group's
    fundamental zone as it is written in Rodrigues space: |r_z| <= tan(pi / 2n)
    for the n-fold axis along z and |r . a| <= 1 for every 2-fold axis a in the
    xy plane at multiples of pi / n from x."""
    R, _ = oracle.start_grid(60000, sym=sym, k=1)
    assert abs(len(R) - 60000 / sym) < 0.03 * 60000 / sym
    q = _mat_to_quat(R)
    rod = q[:, 1:] / q[:, :1]
    assert np.all(np.abs(rod[:, 2]) <= math.tan(math.pi / (2 * n_axis)) + 1e-9)
    for m in range(n_axis):
        phi = math.pi * m / n_axis
        assert np.all(np.abs(rod[:, 0] * math.cos(phi) + rod[:, 1] * math.sin(phi)) <= 1 + 1e-9)


# ----------------------------------------------- sparse assignment (rho-NN)

def test_knn_sets_are_the_rho_nearest_by_angle(tiny):
    """Section "Working with sparse assignment matrices": each model spot keeps
    its rho nearest observed spots of the same angle block.  Checked by brute
    force on the angle between each ray estimate and the model ray (the cost is
    2 D^2 (1 - cos) of that angle), ties to the lower index."""
    fw, obs = tiny["fw"], tiny["obs"]
    rho = 6
    nbr = oracle.knn(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], rho)
    for j in range(0, len(fw["t"]), 7):
        t = fw["t"][j]
        i0, i1 = obs.I_off[t], obs.I_off[t + 1]
        d = obs.p[i0:i1] - fw["center"][j]
        cosang = d @ fw["ray"][j, :3] / np.linalg.norm(d, axis=1)
        ang = np.arccos(np.clip(cosang, -1, 1))
        want = np.lexsort((np.arange(i0, i1), ang))[:rho] + i0
        np.testing.assert_array_equal(nbr[j][:len(want)], want)


def test_sparse_sinkhorn_limits(tiny):
    """With rho at least the largest block the sparse plan is the dense one
    (same potentials); with rho = 32 at eps = 1 mm^2 every left-out entry is
    below exp(-100), so the potentials agree with the dense ones to 1e-9."""
    fw, obs = tiny["fw"], tiny["obs"]
    args = (GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], 1.0, 2.25, 0, 0.4, 40)
    fd_, gd_, fdd, gdd, _ = oracle.sinkhorn(*args)
    big = int(np.diff(obs.I_off).max())
    fs, gs, fds, gds = oracle.sinkhorn_sparse(*args, rho=big)
    np.testing.assert_allclose(fs, fd_, atol=1e-12)
    np.testing.assert_allclose(gs, gd_, atol=1e-12)
    np.testing.assert_allclose(np.r_[fds, gds], np.r_[fdd, gdd], atol=1e-12)
    fs, gs, _, _ = oracle.sinkhorn_sparse(*args, rho=32)
    np.testing.assert_allclose(fs, fd_, atol=1e-9)
    np.testing.assert_allclose(gs, gd_, atol=1e-9)
    fs, gs, _, _ = oracle.sinkhorn_sparse(*args, rho=1)
    assert np.abs(fs - fd_).max() > 1e-6  # a one-neighbour support is a different plan


# ------------------------------------- tilted detectors, per-detector lengths

TILT = sg.tilted_geometry()


@pytest.fixture(scope="module")
def tilted():
    planes = oracle.reflections(TINY.a, TINY.hmax, TINY.centering)
    rng = np.random.default_rng(21)
    R, x = sg.random_grains(TINY, rng)
    om = sg.omegas(TINY)
    fw = oracle.forward(TILT, planes, R, x, om)
    obs = sg.observe(TILT, TINY, fw["t"], fw["det"], fw["spot"], rng)
    return dict(planes=planes, R=R, x=x, om=om, fw=fw, obs=obs)


def _plane_coords(det, s):
    a1, a2 = det.axes()
    d = np.asarray(s, np.float64) - np.asarray(det.centre)
    n = np.asarray(det.normal, np.float64) / np.linalg.norm(det.normal)
    return d @ a1, d @ a2, d @ n


def test_tilted_forward_spots_lie_on_their_detector(tilted):
    """Appendix "Experimental details": two detectors at different distances,
    here one offset and one tilted.  Every visible spot lies on its detector's
    plane, inside its square (in-plane axes), on the ray from the grain centre
    at positive parameter, and no detector closer along the ray holds it;
    both detectors receive spots; and every ray the forward model rejects
    while in band misses both squares (brute force over all (t, n, m))."""
    fw, P, R, x, om = tilted["fw"], tilted["planes"], tilted["R"], tilted["x"], tilted["om"]
    counts = np.bincount(fw["det"], minlength=2)
    assert counts.min() > 10, counts
    for j in range(fw["J_off"][-1]):
        det = TILT.detectors[fw["det"][j]]
        u, v, w = _plane_coords(det, fw["spot"][j])
        assert abs(w) < 1e-9 and abs(u) < det.half and abs(v) < det.half
        d = fw["spot"][j] - fw["center"][j]
        r = fw["ray"][j, :3]
        assert np.linalg.norm(np.cross(d, r)) < 1e-9 and d @ r > 0
    full = oracle.forward(TILT, P, R, x, om, with_all=True)
    e = np.array(TILT.beam)
    for t in range(len(om)):
        Gm = oracle.gamma(om[t])
        for n in range(len(R)):
            c = Gm @ x[n]
            for m in range(len(P.w)):
                g = Gm @ R[n] @ P.w[m]
                r = e - 2 * (e @ g) * g
                hits = []
                for k, det in enumerate(TILT.detectors):
                    nv = np.asarray(det.normal) / np.linalg.norm(det.normal)
                    den = nv @ r
                    if den == 0:
                        continue
                    tau = nv @ (np.asarray(det.centre) - c) / den
                    if tau <= 0:
                        continue
                    u, v, _ = _plane_coords(det, c + tau * r)
                    if abs(u) < det.half and abs(v) < det.half:
                        hits.append(tau)
                lam0 = 2 * P.d0[m] * abs(e @ g)
                in_band = any(TILT.lam_min <= lam0 / k <= TILT.lam_max for k in range(1, P.nharm[m] + 1))
                want = bool(hits) and in_band
                if full["margin_all"][t, n, m] > 1e-9:
                    assert bool(full["vis_all"][t, n, m]) == want, (t, n, m)


def test_cost_length_is_each_detectors_distance():
    """The pair cost is the squared displacement on the detector the model ray
    hits: for a ray along a detector's normal (to the foot of the
    perpendicular) and an observed spot displaced by delta in the plane, the
    rays differ by the angle atan(delta / D_k), so the cost with that
    detector's length is 4 D_k^2 sin^2(atan(delta / D_k) / 2) = delta^2 (1 -
    O(delta^2 / D_k^2)); with the geometry's single D it would be about
    (D / D_k)^2 delta^2."""
    Ls = oracle.cost_lengths(TILT, [0, 1, -1])
    np.testing.assert_allclose(Ls, [125.0, 165.0, TILT.D])
    for k, det in enumerate(TILT.detectors):
        nv = np.asarray(det.normal, np.float64) / np.linalg.norm(det.normal)
        foot = nv * (nv @ np.asarray(det.centre))
        r = foot / np.linalg.norm(foot)
        a1, a2 = det.axes()
        for delta, ax in ((0.3, a1), (0.5, a2)):
            p = foot + delta * ax
            C = oracle.pair_cost(p, np.zeros(3), r, Ls[k])
            exact = 4 * Ls[k] ** 2 * math.sin(0.5 * math.atan(delta / Ls[k])) ** 2
            assert C == pytest.approx(exact, rel=1e-10), (k, C, exact)
            assert C == pytest.approx(delta ** 2, rel=1e-4)
            assert abs(np.linalg.norm(foot) - Ls[k]) < 1e-9


def test_tilted_gradient_and_mstep_fixed_point(tilted):
    """With per-detector lengths the adjoint gradient of sum Q_ij D_j^2 |rhat -
    r|^2 equals central differences of the objective (Q held), and the plain
    M-step (Newton on x, MM on R) run to convergence with Q held stops where
    that gradient vanishes: its weights Q_ij (D_j / D)^2 are the objective's."""
    P, fw, obs, om = tilted["planes"], tilted["fw"], tilted["obs"], tilted["om"]
    c, r = fw["center"], fw["ray"][:, :3]
    Dj = oracle.cost_lengths(TILT, fw["det"])
    assert len(set(Dj.tolist())) == 2
    f, g, *_ = oracle.sinkhorn(Dj, obs.p, obs.I_off, fw["J_off"], c, r, 2.0, 2.25, 0, 0.4, 30)
    rng = np.random.default_rng(9)
    R1 = np.array([_rotvec(rng.normal(size=3) * 0.004) @ a for a in tilted["R"]])
    x1 = tilted["x"] + rng.normal(size=tilted["x"].shape) * 0.1
    args = (TILT, P, om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"], c, r, f, g, 2.0)
    G, H, val = oracle.grain_gn(*args, R1, x1, det=fw["det"])
    np.testing.assert_allclose(val, oracle.grain_objective(*args, R1, x1, det=fw["det"]), rtol=1e-12)
    h = 1e-6
    FD = np.zeros_like(G)
    for k in range(6):
        e = np.zeros(6)
        e[k] = h
        Rp = np.array([_rotvec(e[:3]) @ a for a in R1])
        Rm = np.array([_rotvec(-e[:3]) @ a for a in R1])
        FD[:, k] = (oracle.grain_objective(*args, Rp, x1 + e[3:], det=fw["det"]) -
                    oracle.grain_objective(*args, Rm, x1 - e[3:], det=fw["det"])) / (2 * h)
    assert np.abs(G - FD).max() <= 1e-6 * np.abs(G).max()
    # the M-step's fixed point with Q held at the E-step plan
    Rk, xk = tilted["R"].copy(), tilted["x"].copy()
    G0, *_ = oracle.grain_gn(*args, Rk, xk, det=fw["det"])
    for _ in range(40):
        Rk, xk, _ = oracle.mstep(TILT, P, om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"], c, r,
                                 f, g, 2.0, Rk, xk, n_newton=8, n_mm=20, tol_x=1e-14, tol_R=1e-15,
                                 det=fw["det"])
    # MM maximises sum Q D_j^2 rhat(x).r(R) over R: the rotation part of the
    # gradient vanishes at (Rk, xk); Newton maximises it over x with the E-step
    # rays, i.e. the x part vanishes at (R_E, xk) where the rays are r(R_E)
    Gk, *_ = oracle.grain_gn(*args, Rk, xk, det=fw["det"])
    Gx, *_ = oracle.grain_gn(*args, tilted["R"], xk, det=fw["det"])
    assert np.abs(Gk[:, :3]).max() <= 1e-7 * np.abs(G0[:, :3]).max(), (Gk[:, :3], G0[:, :3])
    assert np.abs(Gx[:, 3:]).max() <= 1e-7 * np.abs(G0[:, 3:]).max(), (Gx[:, 3:], G0[:, 3:])
    # without the (D_j / D)^2 weights the fixed point is elsewhere
    Ru, xu = tilted["R"].copy(), tilted["x"].copy()
    for _ in range(40):
        Ru, xu, _ = oracle.mstep(TILT, P, om, obs.p, obs.I_off, fw["J_off"], fw["grain"], fw["plane"], c, r,
                                 f, g, 2.0, Ru, xu, n_newton=8, n_mm=20, tol_x=1e-14, tol_R=1e-15)
    Gu, *_ = oracle.grain_gn(*args, Ru, xu, det=fw["det"])
    assert np.abs(Gu[:, :3]).max() > 1e3 * np.abs(Gk[:, :3]).max()


def test_observe_on_tilted_detectors(tilted):
    """The detected spots of the tilted geometry lie on their detector plane
    and inside its square; the noise is in the plane."""
    obs = tilted["obs"]
    for i in range(len(obs.p)):
        det = TILT.detectors[obs.det[i]]
        u, v, w = _plane_coords(det, obs.p[i])
        assert abs(w) < 1e-9 and abs(u) < det.half and abs(v) < det.half
