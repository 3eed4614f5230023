"""The learned proposal's kernels against the oracle (oracle/proposal.py):
training scenes, seed-conditioned sets, network forward, gradients, Adam
and decoding.  Inputs are drawn on the host; nothing the oracle reads comes
from the GPU."""
import numpy as np
import pytest

import oracle
import oracle.proposal as op
import synthgen as sg

pytestmark = pytest.mark.gpu

GEOM = sg.Geometry()
BATCHED = sg.CONFIGS["batched"]
OMEGA = sg.omegas(BATCHED)


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2404_06478_gb300 import api, build, proposal
    build.build()
    dev = torch.device("cuda", 0)
    h = api.Handle(dev)
    lat = api.Lattice.cubic(BATCHED.a, BATCHED.hmax, BATCHED.centering, device=dev)
    planes = oracle.reflections(BATCHED.a, BATCHED.hmax, BATCHED.centering)
    return dict(torch=torch, api=api, pr=proposal, dev=dev, h=h, lat=lat, planes=planes)


def _key(seed):
    return np.array([seed & 0xFFFFFFFF, seed >> 32], np.uint32)


def test_scene_matches_oracle(env):
    torch, pr, h = env["torch"], env["pr"], env["h"]
    S, W, G, per = 3, 10, 6, 5
    seed = 0x1234567890AB
    sc = pr.Scenes(h, S, W, G, per, capacity=20000)
    omega = torch.tensor(OMEGA, dtype=torch.float32, device=env["dev"])
    sc.generate(GEOM, env["lat"], omega, seed, gmin=0, gmax=G, cube_mm=5.0, sigma_mm=0.5, outlier_ratio=0.7)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    t0, n_g, R, x = op.scene_params(S, G, 0, G, len(OMEGA), W, _key(seed), 5.0)
    si = sc.scene_i32.cpu().numpy()
    np.testing.assert_array_equal(si[:S], n_g)
    np.testing.assert_array_equal(si[S:2 * S], t0)
    np.testing.assert_allclose(sc.grainR.cpu().numpy().reshape(S, G, 3, 3), R, atol=2e-6)
    np.testing.assert_allclose(sc.grainX.cpu().numpy().reshape(S, G, 3), x, atol=2e-6)
    p, lab, I_off, omega_v = op.training_scene(GEOM, env["planes"], OMEGA, t0, W, R, x, n_g, _key(seed), 0.5, 0.7)
    gI = sc.I_off.cpu().numpy()
    gp = sc.p4.cpu().numpy()[:, :3]
    gl = sc.label.cpu().numpy()
    np.testing.assert_allclose(sc.omega_v.cpu().numpy(), omega_v, atol=1e-6)
    flips = 0
    for v in range(S * W):
        a, b = slice(gI[v], gI[v + 1]), slice(I_off[v], I_off[v + 1])
        if gI[v + 1] - gI[v] != I_off[v + 1] - I_off[v] or not np.array_equal(gl[a], lab[b]):
            flips += 1  # an FP32 / FP64 visibility or edge decision within rounding of a boundary
            continue
        np.testing.assert_allclose(gp[a], p[b], atol=2e-3)
    assert flips <= 1
    if flips == 0:
        seeds = op.scene_seeds(lab, I_off, W, per, _key(seed))
        np.testing.assert_array_equal(sc.seeds.cpu().numpy(), seeds)
        np.testing.assert_array_equal(sc.wlo.cpu().numpy(), np.repeat(np.arange(S) * W, per))


def _host_scene(env, S=4, W=10, G=20, per=8, seed=77, sigma=0.5, ratio=0.7, gmin=None):
    key = _key(seed)
    t0, n_g, R, x = op.scene_params(S, G, G if gmin is None else gmin, G, len(OMEGA), W, key, 5.0)
    p, lab, I_off, omega_v = op.training_scene(GEOM, env["planes"], OMEGA, t0, W, R, x, n_g, key, sigma, ratio)
    seeds = op.scene_seeds(lab, I_off, W, per, key)
    wlo = np.repeat(np.arange(S) * W, per)
    return dict(p=p, lab=lab, I_off=I_off, omega_v=omega_v, seeds=seeds, wlo=wlo, whi=wlo + W,
                R=R.reshape(-1, 3, 3), x=x.reshape(-1, 3), t=np.repeat(np.arange(S * W), np.diff(I_off)))


def _upload_sets(env, d, batch):
    torch, pr, dev = env["torch"], env["pr"], env["dev"]
    p4 = np.zeros((len(d["p"]), 4), np.float32)
    p4[:, :3] = d["p"]
    t = lambda a, dt=torch.int32: torch.tensor(np.asarray(a), dtype=dt, device=dev)
    axes = torch.empty(len(p4), 4, dtype=torch.float32, device=dev)
    pr.make_sets(env["h"], GEOM, t(p4, torch.float32), t(d["I_off"]), t(d["omega_v"], torch.float32),
                 t(d["seeds"]), t(d["wlo"]), t(d["whi"]), batch, axes, label=t(d["lab"]),
                 grainR=t(d["R"].reshape(-1, 9), torch.float32), grainX=t(d["x"], torch.float32))


def test_sets_match_oracle(env):
    torch, pr, h = env["torch"], env["pr"], env["h"]
    d = _host_scene(env)
    B = len(d["seeds"])
    batch = pr.Batch(h, B)
    _upload_sets(env, d, batch)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    X, ids, F = op.make_sets(d["p"], d["t"], d["omega_v"], d["seeds"], d["wlo"], d["whi"])
    Rt, xt = op.set_targets(F, d["R"][np.maximum(d["lab"][np.maximum(d["seeds"], 0)], 0)],
                            d["x"][np.maximum(d["lab"][np.maximum(d["seeds"], 0)], 0)])
    gids = batch.ids.cpu().numpy().reshape(B, op.KSET)
    gX = batch.features().float().cpu().numpy()
    n = op.spot_axes(d["p"], d["t"], d["omega_v"])
    for b in range(B):
        i0 = d["seeds"][b]
        assert gids[b, 0] == ids[b, 0] == i0
        if i0 < 0:
            assert (gids[b] == -1).all() and not gX[b].any()
            continue
        a, o = set(gids[b][gids[b] >= 0].tolist()), set(ids[b][ids[b] >= 0].tolist())
        assert len(a) == len(o)
        # membership may differ only at the selection boundary (distances equal in FP32)
        dist = lambda i: 1.0 - abs(n[i] @ n[i0])
        kth = max(dist(i) for i in o if i != i0)
        for i in a ^ o:
            assert abs(dist(i) - kth) < 1e-6
        for e, i in enumerate(gids[b]):
            if i < 0:
                assert not gX[b, e].any()
                continue
            if i not in o:
                continue
            eo = int(np.nonzero(ids[b] == i)[0][0])
            want = op.bf16(X[b, eo])
            np.testing.assert_allclose(gX[b, e], want, rtol=2 ** -7, atol=1e-6)
    np.testing.assert_allclose(batch.frames().cpu().numpy(), F, atol=2e-6)
    valid = d["lab"][np.maximum(d["seeds"], 0)] >= 0
    np.testing.assert_array_equal(batch.region("svalid", torch.float32, (B,)).cpu().numpy(),
                                  (valid & (d["seeds"] >= 0)).astype(np.float32))
    np.testing.assert_allclose(batch.region("Rt", torch.float32, (B, 3, 3)).cpu().numpy()[valid], Rt[valid],
                               atol=3e-6)
    np.testing.assert_allclose(batch.region("xt", torch.float32, (B, 3)).cpu().numpy()[valid], xt[valid],
                               atol=2e-6)


def _oracle_batch(env, B=24, seed=5):
    """Host sets (oracle features, BF16-rounded), targets and parameters."""
    d = _host_scene(env, S=3, per=B // 3, G=12, seed=seed)
    X, ids, F = op.make_sets(d["p"], d["t"], d["omega_v"], d["seeds"], d["wlo"], d["whi"])
    X = op.bf16(X)
    g = d["lab"][np.maximum(d["seeds"], 0)]
    valid = ((d["seeds"] >= 0) & (g >= 0)).astype(np.float64)
    Rt, xt = op.set_targets(F, d["R"][np.maximum(g, 0)], d["x"][np.maximum(g, 0)])
    return X, F, Rt, xt, valid


def _load_batch(env, batch, X, Rt, xt, valid):
    torch = env["torch"]
    B = X.shape[0]
    dev = env["dev"]
    batch.features().copy_(torch.tensor(X, dtype=torch.float32).to(torch.bfloat16))
    batch.region("nvalid", torch.int32, (B,)).copy_(torch.tensor(X[:, :, 12].sum(1), dtype=torch.int32))
    batch.region("Rt", torch.float32, (B, 3, 3)).copy_(torch.tensor(Rt, dtype=torch.float32))
    batch.region("xt", torch.float32, (B, 3)).copy_(torch.tensor(xt, dtype=torch.float32))
    batch.region("svalid", torch.float32, (B,)).copy_(torch.tensor(valid, dtype=torch.float32))


def _oracle_params(env, seed):
    P = env["pr"].unpack_params(env["pr"].init_params(seed))
    Pd = {k: v.astype(np.float64) for k, v in P.items()}
    rng = np.random.default_rng(seed + 1)
    for k in Pd:
        if k.startswith("b"):
            Pd[k] = (0.05 * rng.standard_normal(Pd[k].shape)).astype(np.float32).astype(np.float64)
    vec = np.concatenate([Pd[k].astype(np.float32).reshape(-1) for k, _ in env["pr"].PARAM_SHAPES])
    return Pd, vec


def test_forward_matches_oracle(env):
    torch, pr, h = env["torch"], env["pr"], env["h"]
    X, F, Rt, xt, valid = _oracle_batch(env)
    B = X.shape[0]
    Pd, vec = _oracle_params(env, 3)
    net = pr.Network(h, params=vec)
    batch = pr.Batch(h, B)
    _load_batch(env, batch, X, Rt, xt, valid)
    O = pr.forward(h, net, batch).cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    Oo, _ = op.forward(Pd, X, bf16_ops=True)
    scale = np.abs(Oo).max()
    assert np.abs(O - Oo).max() < 3e-3 * scale, np.abs(O - Oo).max() / scale
    H3 = batch.region("H3", torch.bfloat16, (B * op.KSET, 256)).float().cpu().numpy()
    _, cache = op.forward(Pd, X, bf16_ops=True)
    # activations: BF16 values equal up to rare one-step rounding flips
    assert np.mean(H3 != cache["H3"]) < 1e-2


@pytest.mark.parametrize("B", [24, 96, 384, 2046])
def test_gradients_match_oracle(env, B):
    """B = 96 and up take the split reductions of the head's weight
    gradients; 384 sets spread the weight-gradient GEMMs over split-K
    partials and every persistent CTA over several tiles; 2046 sets are the
    size of a training batch (the bench's 2048 rounded to three scenes)."""
    torch, pr, h = env["torch"], env["pr"], env["h"]
    X, F, Rt, xt, valid = _oracle_batch(env, B=B, seed=9)
    B = X.shape[0]
    Pd, vec = _oracle_params(env, 4)
    net = pr.Network(h, params=vec)
    batch = pr.Batch(h, B)
    _load_batch(env, batch, X, Rt, xt, valid)
    pr.train_step(h, net, batch, lr=0.0)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    G = pr.unpack_params(net.grads())
    np.testing.assert_array_equal(net.params(), vec)  # lr = 0 leaves the parameters
    O, cache = op.forward(Pd, X, bf16_ops=True)
    loss, dO, dbest, hbest = op.set_loss(O, Rt, xt, valid)
    Go = op.backward(Pd, cache, dO)
    gl = batch.region("loss", torch.float32, (B,)).cpu().numpy()
    Lset_o = np.zeros(B)
    Oh = O.reshape(B, op.NHYP, 9)
    for b in range(B):
        if valid[b]:
            Lset_o[b] = op.set_loss(O[b:b + 1], Rt[b:b + 1], xt[b:b + 1], np.ones(1))[0]
    # The GPU's per-spot activations differ from the oracle's in rare one-ulp
    # rounding flips (FP32 against FP64 accumulation); a flip upstream of a
    # later rounding point (the BF16 pooled features and head activations) can
    # move that value by a whole ulp (2^-8 relative), and a set whose loss is
    # ill-conditioned (nearly parallel 6-D rotation columns) amplifies it.  So
    # almost every set agrees to 5e-3 and every set to 5e-2; the same holds for
    # the best hypothesis, which a near tie can flip.
    rel = np.abs(gl - Lset_o) / np.maximum(np.abs(Lset_o), 2e-2)
    assert np.mean(rel > 5e-3) <= 0.03 and rel.max() < 5e-2, (np.mean(rel > 5e-3), rel.max())
    hb = batch.region("hbest", torch.int32, (B,)).cpu().numpy()[valid > 0]
    assert np.mean(hb != hbest[valid > 0]) <= 0.03
    for k, _ in pr.PARAM_SHAPES:
        err = np.linalg.norm(G[k] - Go[k]) / max(np.linalg.norm(Go[k]), 1e-30)
        assert err < 2e-2, (k, err)


def test_adam_step_matches_oracle(env):
    torch, pr, h = env["torch"], env["pr"], env["h"]
    X, F, Rt, xt, valid = _oracle_batch(env, seed=11)
    B = X.shape[0]
    Pd, vec = _oracle_params(env, 5)
    net = pr.Network(h, params=vec)
    batch = pr.Batch(h, B)
    _load_batch(env, batch, X, Rt, xt, valid)
    pr.train_step(h, net, batch, lr=1e-3)
    torch.cuda.synchronize()
    P1 = pr.unpack_params(net.params())
    O, cache = op.forward(Pd, X, bf16_ops=True)
    _, dO, _, _ = op.set_loss(O, Rt, xt, valid)
    Go = op.backward(Pd, cache, dO)
    Po = {k: v.copy() for k, v in Pd.items()}
    op.adam(Po, Go, {k: np.zeros_like(v) for k, v in Pd.items()}, {k: np.zeros_like(v) for k, v in Pd.items()},
            1, 1e-3)
    for k, _ in pr.PARAM_SHAPES:
        big = np.abs(Go[k]) > 1e-3 * np.abs(Go[k]).max()
        diff = np.abs(P1[k] - Po[k])[big]
        # first Adam step moves every weight by lr * g / (|g| + eps): sign of g
        assert np.mean(diff > 1e-6) < 0.02, (k, np.mean(diff > 1e-6))


def test_decode_matches_oracle(env):
    torch, pr, h = env["torch"], env["pr"], env["h"]
    B = 16
    rng = np.random.default_rng(21)
    O = rng.standard_normal((B, op.NOUT)).astype(np.float32)
    F = sg.random_rotations(B, rng).reshape(B, 3, 3).astype(np.float32)
    batch = pr.Batch(h, B)
    batch.outputs().copy_(torch.tensor(O))
    batch.frames().copy_(torch.tensor(F))
    nv = np.full(B, 5, np.int32)
    nv[3] = 0
    batch.region("nvalid", torch.int32, (B,)).copy_(torch.tensor(nv))
    R, x = pr.decode(h, batch)
    Ro, xo = op.decode(O.astype(np.float64), F.astype(np.float64))
    R = R.cpu().numpy().reshape(B, op.NHYP, 3, 3)
    x = x.cpu().numpy().reshape(B, op.NHYP, 3)
    keep = nv > 0
    np.testing.assert_allclose(R[keep], Ro[keep], atol=2e-5)
    np.testing.assert_allclose(x[keep], xo[keep], atol=2e-5)
    np.testing.assert_allclose(R[3], np.broadcast_to(np.eye(3), (op.NHYP, 3, 3)))


def test_training_reduces_the_loss(env):
    """A short run on single-grain scenes (the easiest case) must learn."""
    torch, pr, h = env["torch"], env["pr"], env["h"]
    S, W, per = 32, 10, 8
    sc = pr.Scenes(h, S, W, 1, per, capacity=S * W * 60)
    omega = torch.tensor(OMEGA, dtype=torch.float32, device=env["dev"])
    net = pr.Network(h, seed=0)
    batch = pr.Batch(h, S * per)
    first, last = [], []
    for it in range(400):
        sc.generate(GEOM, env["lat"], omega, seed=1000 + it, gmin=1, gmax=1, outlier_ratio=0.0)
        sc.sets(GEOM, batch)
        pr.train_step(h, net, batch, lr=1e-3)
        d = batch.region("dbest", torch.float32, (S * per,))
        v = batch.region("svalid", torch.float32, (S * per,))
        m = float((d * v).sum() / v.sum().clamp(min=1))
        (first if it < 50 else last if it >= 350 else []).append(m)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    assert np.mean(last) < 0.8 * np.mean(first), (np.mean(first), np.mean(last))


def test_sets_edge_cases(env):
    """Empty sets (seed -1), windows with fewer candidates than a set holds,
    a window holding only the seed, duplicated spots (equal distances: the
    lower index wins) and windows clipped at the ends of the scan."""
    torch, pr, h = env["torch"], env["pr"], env["h"]
    rng = np.random.default_rng(31)
    T = 6
    counts = np.array([3, 1, 0, 200, 150, 2])
    I_off = np.concatenate([[0], np.cumsum(counts)])
    n = int(I_off[-1])
    p = np.zeros((n, 3))
    p[:, 0] = rng.uniform(-120, 120, n)
    p[:, 1] = rng.uniform(-120, 120, n)
    p[:, 2] = np.where(rng.random(n) < 0.8, -200.0, 200.0)
    # duplicates: spots 10..19 repeat spot 9 of angle 3 exactly (equal distances)
    p[10:20] = p[9]
    t = np.repeat(np.arange(T), counts)
    om = np.radians(np.arange(T) * 4.0)
    seeds = np.array([-1, 0, 3, 9, 100, 350, 353, 9])
    wlo = np.array([0, 0, 1, 3, 0, 4, 5, 0])
    whi = np.array([6, 1, 2, 4, 6, 6, 6, 6])
    dev = env["dev"]
    p4 = np.zeros((n, 4), np.float32)
    p4[:, :3] = p
    ti = lambda a: torch.tensor(np.asarray(a), dtype=torch.int32, device=dev)
    batch = pr.Batch(h, len(seeds))
    axes = torch.empty(n, 4, dtype=torch.float32, device=dev)
    pr.make_sets(h, GEOM, torch.tensor(p4, device=dev), ti(I_off), torch.tensor(om, dtype=torch.float32,
                                                                                 device=dev),
                 ti(seeds), ti(wlo), ti(whi), batch, axes)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    X, ids, F = op.make_sets(p4[:, :3].astype(np.float64), t, om, seeds, wlo, whi)
    gids = batch.ids.cpu().numpy().reshape(len(seeds), op.KSET)
    nval = batch.region("nvalid", torch.int32, (len(seeds),)).cpu().numpy()
    for b in range(len(seeds)):
        assert nval[b] == (ids[b] >= 0).sum()
        if b in (0, 1, 2, 6):  # fewer candidates than the set holds: the whole window
            np.testing.assert_array_equal(np.sort(gids[b][gids[b] >= 0]), np.sort(ids[b][ids[b] >= 0]))
    assert nval[0] == 0 and nval[1] == 3 and nval[2] == 1
    # the duplicates of spot 9 are at distance 0 from seed 9 and come first, by index
    assert set(gids[3][1:11].tolist()) == set(range(10, 20))
    assert list(gids[7][1:11]) == list(range(10, 20))
    X0 = batch.features().float().cpu().numpy()
    assert not X0[0].any()


def test_sets_full_size_sampled(env):
    """Sets of the 1000-grain, 90-rotation, 70%-outlier workload (about 132k
    candidate spots per window) on sampled seeds: the oracle's set and the
    GPU's agree up to ties at the selection boundary, features match."""
    torch, pr, h = env["torch"], env["pr"], env["h"]
    from _cases import make_case
    case = make_case(BATCHED, seed=0)
    p, I_off = case.obs.p, case.obs.I_off
    t = np.repeat(np.arange(BATCHED.T), np.diff(I_off))
    rng = np.random.default_rng(41)
    seeds = rng.choice(len(p), 12, replace=False)
    seeds[0] = I_off[1] - 1   # a seed in the first angles: window clipped at the start
    seeds[1] = len(p) - 1     # and at the end
    ob = env["api"].ObsSpots.from_numpy(p, I_off, device=env["dev"])
    om = torch.tensor(case.om, dtype=torch.float32, device=env["dev"])
    batch = pr.Batch(h, len(seeds))
    pr.propose(h, pr.Network(h, seed=0), GEOM, ob, om, seeds, batch=batch)
    torch.cuda.synchronize()
    assert h.device_status() == 0
    T = BATCHED.T
    tt = np.searchsorted(I_off, seeds, side="right") - 1
    lo = np.clip(tt - 4, 0, T)
    hi = np.clip(lo + 10, 0, T)
    lo = np.clip(hi - 10, 0, T)
    X, ids, F = op.make_sets(p, t, case.om, seeds, lo, hi)
    n = op.spot_axes(p, t, case.om)
    gids = batch.ids.cpu().numpy().reshape(len(seeds), op.KSET)
    gX = batch.features().float().cpu().numpy()
    for b, i0 in enumerate(seeds):
        a, o = set(gids[b].tolist()), set(ids[b].tolist())
        dist = lambda i: 1.0 - abs(n[i] @ n[i0])
        kth = max(dist(i) for i in o if i != i0)
        for i in a ^ o:
            assert abs(dist(i) - kth) < 2e-6
        for e, i in enumerate(gids[b]):
            if i in o:
                eo = int(np.nonzero(ids[b] == i)[0][0])
                np.testing.assert_allclose(gX[b, e], op.bf16(X[b, eo]), rtol=2 ** -7, atol=1e-6)
    np.testing.assert_allclose(batch.frames().cpu().numpy(), F, atol=2e-6)
