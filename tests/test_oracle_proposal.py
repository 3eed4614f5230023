"""Pins of the learned-proposal oracle (oracle/proposal.py).

The paper has no learned component, so nothing here is a value the paper
prints: each test ties the oracle to finite differences, closed forms,
invariants, a library routine or published known-answer vectors.  None of
these runs on a GPU.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import oracle.proposal as op
import synthgen as sg

GOLD = os.path.join(os.path.dirname(__file__), "golden")
GEOM = sg.Geometry()
BATCHED = sg.CONFIGS["batched"]


@pytest.fixture(scope="module")
def planes():
    return oracle.reflections(BATCHED.a, BATCHED.hmax, BATCHED.centering)


def test_philox_known_answers():
    kat = json.load(open(os.path.join(GOLD, "philox4x32_kat.json")))
    for v in kat["vectors"]:
        c = np.array([int(h, 16) for h in v["counter"]], np.uint32)
        k = np.array([int(h, 16) for h in v["key"]], np.uint32)
        out = op.philox4x32(c, k)
        assert ["%08x" % w for w in out] == v["out"]


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(10000) * 10.0 ** rng.integers(-6, 6, 10000),
                        [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, -(1.0 + 2 ** -8), 65504.0]])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(op.bf16(x), want)


def test_axes_are_plane_normals(planes):
    """Noiseless spots of a grain at the origin: the axis is +-R w_m."""
    rng = np.random.default_rng(1)
    R = sg.random_rotations(6, rng)
    x = np.zeros((6, 3))
    om = sg.omegas(BATCHED)[:12]
    f = oracle.forward(GEOM, planes, R, x, om)
    n = op.spot_axes(f["spot"], f["t"], om)
    want = np.einsum("nij,nj->ni", R.reshape(-1, 3, 3)[f["grain"]], planes.w[f["plane"]])
    dots = np.abs((n * want).sum(1))
    assert len(dots) > 100
    np.testing.assert_allclose(dots, 1.0, atol=1e-12)


def test_seed_frame():
    rng = np.random.default_rng(2)
    for _ in range(50):
        n0 = rng.standard_normal(3)
        n0 /= np.linalg.norm(n0)
        F = op.seed_frame(n0)
        np.testing.assert_allclose(F.T @ F, np.eye(3), atol=1e-14)
        assert np.linalg.det(F) == pytest.approx(1.0, abs=1e-14)
        np.testing.assert_allclose(F[:, 0], n0, atol=1e-15)
        # a1 lies in the plane of +y and n0, on the +y side
        assert abs(F[:, 1] @ np.cross(n0, [0.0, 1.0, 0.0])) < 1e-14
        assert F[1, 1] > 0
    F = op.seed_frame(np.array([0.0, 1.0, 0.0]))
    np.testing.assert_allclose(F.T @ F, np.eye(3), atol=1e-14)


def _scene(planes, n_grains, T=20, seed=3, sigma=0.5):
    rng = np.random.default_rng(seed)
    R = sg.random_rotations(n_grains, rng)
    x = rng.uniform(-2.5, 2.5, (n_grains, 3))
    om = sg.omegas(BATCHED)[:T]
    f = oracle.forward(GEOM, planes, R, x, om)
    p = f["spot"].copy()
    p[:, :2] += sigma * rng.standard_normal((len(p), 2))
    return R, x, om, p, f["t"], f["grain"]


def test_sets_take_the_nearest_axes(planes):
    R, x, om, p, t, g = _scene(planes, 8)
    rng = np.random.default_rng(4)
    seeds = rng.choice(len(p), 20, replace=False)
    wlo = np.maximum(t[seeds] - 4, 0)
    whi = np.minimum(t[seeds] + 6, len(om))
    X, ids, F = op.make_sets(p, t, om, seeds, wlo, whi)
    n = op.spot_axes(p, t, om)
    for b, i0 in enumerate(seeds):
        assert ids[b, 0] == i0
        cand = np.nonzero((t >= wlo[b]) & (t < whi[b]) & (np.arange(len(p)) != i0))[0]
        d = 1.0 - np.abs(n[cand] @ n[i0])
        k = min(op.KSET - 1, len(cand))
        got = ids[b, 1:1 + k]
        assert (ids[b, 1 + k:] == -1).all()
        dg = 1.0 - np.abs(n[got] @ n[i0])
        # the k smallest distances (a library partition), in ascending order
        np.testing.assert_array_equal(np.sort(dg), np.sort(np.partition(d, k - 1)[:k]))
        assert (np.diff(dg) >= 0).all()
        np.testing.assert_allclose(X[b, 0, 0:3], [1.0, 0.0, 0.0], atol=1e-14)
        np.testing.assert_allclose(np.linalg.norm(X[b, :1 + k, 0:3], axis=1), 1.0, atol=1e-12)
        assert (X[b, :1 + k, 0] >= 0).all()
        assert X[b, 0, 11] == 1 and X[b, 1:, 11].sum() == 0
        assert X[b, :1 + k, 12].sum() == 1 + k
        # feature 0 is the cosine of the angle between the axes
        np.testing.assert_allclose(X[b, 1:1 + k, 0], 1.0 - dg, atol=1e-12)


def test_gram_schmidt_closed_forms():
    rng = np.random.default_rng(5)
    o = rng.standard_normal((100, 6))
    Rh = op.gram_schmidt(o)
    np.testing.assert_allclose(np.einsum("nji,njk->nik", Rh, Rh), np.broadcast_to(np.eye(3), (100, 3, 3)),
                               atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(Rh), 1.0, atol=1e-13)
    R = sg.random_rotations(100, rng).reshape(-1, 3, 3)
    o6 = np.concatenate([R[:, :, 0] * 3.0, R[:, :, 1] * 0.5 + R[:, :, 0] * 2.0], 1)
    np.testing.assert_allclose(op.gram_schmidt(o6), R, atol=1e-13)


def test_gram_schmidt_backward_finite_differences():
    rng = np.random.default_rng(6)
    o = rng.standard_normal((5, 6))
    dR = rng.standard_normal((5, 3, 3))
    g = op.gram_schmidt_backward(o, dR)
    h = 1e-6
    for n in range(5):
        for k in range(6):
            op_ = o.copy(); op_[n, k] += h
            om_ = o.copy(); om_[n, k] -= h
            fd = ((op.gram_schmidt(op_)[n] - op.gram_schmidt(om_)[n]) * dR[n]).sum() / (2 * h)
            assert g[n, k] == pytest.approx(fd, rel=1e-6, abs=1e-8)


def _exact_encoding(Rloc, xt):
    o = np.concatenate([Rloc[:, :, 0], Rloc[:, :, 1], xt], 1)
    return np.tile(o, (1, op.NHYP))


def test_loss_zero_at_truth_and_symmetric():
    rng = np.random.default_rng(7)
    B = 16
    Rloc = sg.random_rotations(B, rng).reshape(-1, 3, 3)
    xt = rng.uniform(-1, 1, (B, 3))
    valid = np.ones(B)
    loss, dO, d, _ = op.set_loss(_exact_encoding(Rloc, xt), Rloc, xt, valid)
    assert loss == pytest.approx(0.0, abs=1e-13)
    np.testing.assert_allclose(dO, 0.0, atol=1e-12)
    O = rng.standard_normal((B, op.NOUT))
    base = op.set_loss(O, Rloc, xt, valid)[0]
    for S in op.cubic_group():
        assert op.set_loss(O, Rloc @ S, xt, valid)[0] == pytest.approx(base, rel=1e-13)
    # a symmetric copy of the truth is a zero-loss answer too
    S = op.cubic_group()[7]
    assert op.set_loss(_exact_encoding(Rloc @ S, xt), Rloc, xt, valid)[0] == pytest.approx(0.0, abs=1e-13)
    # the rotation error is 2 (3 - tr) = 8 sin^2(theta / 2) of the misorientation
    th = 0.3
    Rz = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    _, _, d, _ = op.set_loss(_exact_encoding(Rloc @ Rz, xt), Rloc, xt, valid)
    np.testing.assert_allclose(d, 8 * math.sin(th / 2) ** 2, rtol=1e-12)


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(8)
    B = 6
    Rloc = sg.random_rotations(B, rng).reshape(-1, 3, 3)
    xt = rng.uniform(-1, 1, (B, 3))
    valid = np.array([1, 1, 0, 1, 1, 1.0])
    O = rng.standard_normal((B, op.NOUT))
    _, dO, _, _ = op.set_loss(O, Rloc, xt, valid)
    assert np.all(dO[2] == 0)
    h = 1e-6
    for b in range(B):
        for k in rng.choice(op.NOUT, 12, replace=False):
            Op = O.copy(); Op[b, k] += h
            Om = O.copy(); Om[b, k] -= h
            fd = (op.set_loss(Op, Rloc, xt, valid)[0] - op.set_loss(Om, Rloc, xt, valid)[0]) / (2 * h)
            assert dO[b, k] == pytest.approx(fd, rel=1e-5, abs=1e-9)


def _sets(rng, B):
    X = np.zeros((B, op.KSET, op.NF))
    X[:, :, :14] = rng.standard_normal((B, op.KSET, 14))
    nvalid = rng.integers(1, op.KSET + 1, B)
    for b in range(B):
        X[b, :, 12] = (np.arange(op.KSET) < nvalid[b]).astype(float)
        X[b, nvalid[b]:, :] = 0.0
    return X


def test_network_gradient_finite_differences():
    rng = np.random.default_rng(9)
    P = op.init_params(rng)
    for k in P:
        if k.startswith("b"):
            P[k] = 0.1 * rng.standard_normal(P[k].shape)
    B = 3
    X = _sets(rng, B)
    Rloc = sg.random_rotations(B, rng).reshape(-1, 3, 3)
    xt = rng.uniform(-1, 1, (B, 3))
    valid = np.ones(B)

    def L(P):
        O, _ = op.forward(P, X, bf16_ops=False)
        return op.set_loss(O, Rloc, xt, valid)[0]

    O, cache = op.forward(P, X, bf16_ops=False)
    _, dO, _, _ = op.set_loss(O, Rloc, xt, valid)
    G = op.backward(P, cache, dO)
    h = 1e-6
    for name, _ in op.PARAM_SHAPES:
        flat = P[name].reshape(-1)
        for idx in rng.choice(flat.size, 6, replace=False):
            Pp = {k: v.copy() for k, v in P.items()}
            Pm = {k: v.copy() for k, v in P.items()}
            Pp[name].reshape(-1)[idx] += h
            Pm[name].reshape(-1)[idx] -= h
            fd = (L(Pp) - L(Pm)) / (2 * h)
            assert G[name].reshape(-1)[idx] == pytest.approx(fd, rel=1e-4, abs=1e-8), (name, idx)


def test_network_permutation_invariance_and_padding():
    rng = np.random.default_rng(10)
    P = op.init_params(rng)
    X = _sets(rng, 2)
    O, _ = op.forward(P, X, bf16_ops=False)
    Xp = X.copy()
    n0 = int(X[0, :, 12].sum())
    perm = rng.permutation(n0)
    Xp[0, :n0] = X[0, perm]
    Xp[1, int(X[1, :, 12].sum()):, :13] = 0.0  # padding content is ignored
    Op, _ = op.forward(P, Xp, bf16_ops=False)
    np.testing.assert_allclose(Op, O, rtol=1e-12, atol=1e-12)


def test_bf16_forward_close_to_exact():
    rng = np.random.default_rng(11)
    P = op.init_params(rng)
    X = _sets(rng, 4)
    O64, _ = op.forward(P, X, bf16_ops=False)
    O16, _ = op.forward(P, X, bf16_ops=True)
    assert np.linalg.norm(O16 - O64) / np.linalg.norm(O64) < 2e-2


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(12)
    P = {"w": rng.standard_normal(50)}
    G = {"w": rng.standard_normal(50)}
    M = {"w": np.zeros(50)}
    V = {"w": np.zeros(50)}
    p0 = P["w"].copy()
    op.adam(P, G, M, V, 1, 1e-3)
    np.testing.assert_allclose(P["w"], p0 - 1e-3 * G["w"] / (np.abs(G["w"]) + 1e-8), rtol=1e-12)
    # constant gradient: every step moves by lr (bias correction exact)
    P2, G2 = {"w": np.zeros(3)}, {"w": np.array([2.0, -0.5, 1e-3])}
    M2, V2 = {"w": np.zeros(3)}, {"w": np.zeros(3)}
    for s in range(1, 6):
        op.adam(P2, G2, M2, V2, s, 0.01, eps=0.0)
    np.testing.assert_allclose(P2["w"], -0.05 * np.sign(G2["w"]), rtol=1e-12)


def test_scene_params_distribution():
    S, G = 400, 8
    key = np.array([3, 4], np.uint32)
    t0, n_g, R, x = op.scene_params(S, G, 2, 6, 90, 10, key, 5.0)
    assert t0.min() >= 0 and t0.max() <= 80 and n_g.min() >= 2 and n_g.max() <= 6
    assert set(n_g.tolist()) == {2, 3, 4, 5, 6}
    Rf = R.reshape(-1, 3, 3)
    np.testing.assert_allclose(np.einsum("nji,njk->nik", Rf, Rf), np.broadcast_to(np.eye(3), Rf.shape), atol=1e-12)
    np.testing.assert_allclose(np.linalg.det(Rf), 1.0, atol=1e-12)
    # uniform on SO(3): E[R] = 0 and E[tr R] = 0 (Haar measure)
    assert np.abs(Rf.mean(0)).max() < 0.05
    assert abs(np.trace(Rf, axis1=1, axis2=2).mean()) < 0.06
    assert np.abs(x).max() <= 2.5 and abs(x.mean()) < 0.1


def test_training_scene_noiseless_matches_forward(planes):
    S, G, W = 3, 4, 10
    key = np.array([17, 99], np.uint32)
    om = sg.omegas(BATCHED)
    t0, n_g, R, x = op.scene_params(S, G, 0, G, len(om), W, key, 5.0)
    n_g = np.array([4, 0, 2])
    p, lab, I_off, omega_v = op.training_scene(GEOM, planes, om, t0, W, R, x, n_g, key, 0.0, 0.7)
    assert I_off[-1] == len(p)
    for v in range(S * W):
        s = v // W
        assert omega_v[v] == om[t0[s] + v % W]
        sl = slice(I_off[v], I_off[v + 1])
        inl = lab[sl] >= 0
        f = oracle.forward(GEOM, planes, R[s, :n_g[s]].reshape(-1, 9), x[s, :n_g[s]], np.array([omega_v[v]]))
        assert inl.sum() == len(f["spot"])
        np.testing.assert_array_equal(lab[sl][inl], s * G + f["grain"])
        np.testing.assert_allclose(p[sl][inl], f["spot"], atol=1e-12)
        n_out = int((~inl).sum())
        u = op.uniform01(op.philox4x32(np.array([v, op.ALL, 0, op.TAG_COUNT], np.uint32), key)[0])
        assert n_out == math.floor(0.7 * inl.sum() + u)
        po = p[sl][~inl]
        assert np.all(np.abs(po[:, :2]) < 128.0) and np.all(np.abs(np.abs(po[:, 2]) - 200.0) == 0)
    assert (lab[I_off[W]:I_off[2 * W]] < 0).all()
    seeds = op.scene_seeds(lab, I_off, W, 5, key)
    for s in range(S):
        for j in range(5):
            i = seeds[s * 5 + j]
            if n_g[s] == 0:
                assert i == -1
            else:
                assert I_off[s * W] <= i < I_off[(s + 1) * W] and lab[i] >= 0


def test_training_scene_noise_statistics(planes):
    S, G, W = 2, 30, 10
    key = np.array([5, 6], np.uint32)
    om = sg.omegas(BATCHED)
    t0, n_g, R, x = op.scene_params(S, G, G, G, len(om), W, key, 0.0)
    p0, l0, _, _ = op.training_scene(GEOM, planes, om, t0, W, R, x, n_g, key, 0.0, 0.0)
    p1, l1, _, _ = op.training_scene(GEOM, planes, om, t0, W, R, x, n_g, key, 0.5, 0.0)
    # same counter -> same spot; keep the spots that stayed on the detector
    assert len(p1) <= len(p0) and len(p1) > 0.95 * len(p0)
    d = []
    j = 0
    for i in range(len(p0)):
        if j < len(p1) and l0[i] == l1[j] and np.linalg.norm(p1[j, :2] - p0[i, :2]) < 5.0:
            d.append(p1[j, :2] - p0[i, :2])
            j += 1
    d = np.array(d)
    assert len(d) > 0.95 * len(p1)
    assert abs(d.mean()) < 0.05 and d.std() == pytest.approx(0.5, rel=0.05)


def test_bf16_mode_equals_exact_mode_when_no_rounding_occurs():
    """The BF16 data path (weights, activations, pooled features and the
    back-propagated errors the GEMMs read, rounded to BF16) is the FP64 path
    with rounding points added.  On a network and sets whose every such
    quantity has at most 8 significant bits (signed permutation weights,
    dyadic inputs and biases, 8 valid spots per set so that the mean divides
    by a power of two, head weights with one dyadic entry per row of W4 and
    per column of W5) no rounding changes a value, so both modes give the same
    outputs and the same gradients bit for bit; the FP64 mode is itself
    pinned by finite differences above."""
    rng = np.random.default_rng(29)
    B = 3
    P = {}
    for name, shape in op.PARAM_SHAPES:
        P[name] = np.zeros(shape)
    # per-spot layers: one signed power-of-two entry per row
    P["W1"][np.arange(op.WIDTH), rng.integers(0, 14, op.WIDTH)] = rng.choice([-1.0, 1.0, 0.5], op.WIDTH)
    for name in ("W2", "W3"):
        perm = rng.permutation(op.WIDTH)
        P[name][np.arange(op.WIDTH), perm] = rng.choice([-1.0, 1.0], op.WIDTH)
    for name in ("b1", "b2", "b3"):
        P[name] = rng.integers(-2, 3, op.WIDTH) / 16.0
    # head: W4 takes one pooled feature per hidden unit (one dyadic entry per
    # row, distinct columns) and no bias, so the hidden activations stay
    # exact; W5 one dyadic entry per column, so that every error sent back
    # has a single term and few significant bits as well
    dy = [-0.25, -0.125, 0.125, 0.25]
    P["W4"][np.arange(op.HEAD), rng.permutation(2 * op.WIDTH)[:op.HEAD]] = rng.choice(dy, op.HEAD)
    rows, cols = P["W5"].shape
    P["W5"][rng.integers(0, rows, cols), np.arange(cols)] = rng.choice(dy, cols)
    X = np.zeros((B, op.KSET, op.NF))
    X[:, :, :14] = rng.integers(-8, 9, (B, op.KSET, 14)) / 16.0
    X[:, :, 12] = 0.0
    X[:, :8, 12] = 1.0  # 8 valid spots per set: the mean divides by a power of two
    O64, c64 = op.forward(P, X, bf16_ops=False)
    O16, c16 = op.forward(P, X, bf16_ops=True)
    np.testing.assert_array_equal(O16, O64)
    for k in ("H1", "H2", "H3"):
        np.testing.assert_array_equal(c16[k], c64[k])
    assert np.count_nonzero(c64["H3"]) > 0.2 * c64["H3"].size
    dO = rng.integers(-4, 5, O64.shape) / 64.0
    G64 = op.backward(P, c64, dO)
    G16 = op.backward(P, c16, dO)
    for k in G64:
        np.testing.assert_array_equal(G16[k], G64[k], err_msg=k)
    assert all(np.count_nonzero(G64[k]) > 0 for k in ("W1", "W2", "W3", "W4", "W5"))
    assert np.count_nonzero(c64["H4"]) > 0.2 * c64["H4"].size
