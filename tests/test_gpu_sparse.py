"""Parity of laue_cost_sinkhorn_sparse (the E-step on the rho-nearest-
neighbour support, paper Section "Working with sparse assignment matrices")
with the FP64 oracle on the same float32 inputs.

The neighbour sets are integer results decided by float comparisons: the
kernel ranks costs computed in float32, the oracle in float64.  The float32
cost D^2 |rhat - r|^2 carries an absolute error of about 1e-7 in each
component of rhat - r, i.e. about 2e-7 sqrt(3) D sqrt(C) in C; two costs
closer than 4e-6 D sqrt(C) (about 5x that) are a near tie that either
precision may order either way.  So a listed set must equal the oracle's
except at near ties, where it must still be valid: k distinct spots of the
block whose float64 costs are increasing and whose largest is within the
near-tie distance of the oracle's k-th smallest.  Potentials within
1e-4 (|f| + eps) as for the dense E-step
(float32 log-sum-exps over at most a few hundred terms per spot); hard
assignments bit-exact where the reference margin exceeds 1e-3; margins and
marginal errors within 1e-4."""
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


def _geo(case):
    fw = case.fw
    return case.obs.p, case.obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3]


def _near(C):
    """Near-tie distance of float32 costs around C (mm^2)."""
    return 4e-6 * GEOM.D * np.sqrt(np.maximum(C, 0.0)) + 1e-9


def _check_neighbours(got, want, p, I_off, J_off, c, r, rows):
    """got/want: neighbour lists of model spots `rows` (-1 padded).  Rows that
    differ must be valid near-tie alternatives; returns how many differ."""
    t_of_j = np.repeat(np.arange(len(I_off) - 1), np.diff(J_off))
    n_diff = 0
    for g_row, w_row, j in zip(got, want, rows):
        if np.array_equal(g_row, w_row):
            continue
        n_diff += 1
        t = t_of_j[j]
        i0, i1 = int(I_off[t]), int(I_off[t + 1])
        k = int((w_row >= 0).sum())
        sel = g_row[:k]
        assert np.all(g_row[k:] == -1) and np.all((sel >= i0) & (sel < i1)) and len(set(sel.tolist())) == k, j
        cost = oracle.pair_costs(p[i0:i1], c[j], r[j], GEOM.D)
        cg = cost[sel - i0]
        assert np.all(np.diff(cg) >= -_near(cg[1:])), (j, cg)
        kth = np.sort(cost)[k - 1]
        assert cg.max() <= kth + _near(kth), (j, cg.max(), kth)
    return n_diff


def _reference(case, eps, mode, rho, n_iter, frac=0.4):
    """Oracle potentials on the sparse support plus the read-out defined on
    them: row argmax over the support and the outlier column (ties to the
    lowest model index, the outlier column only when strictly larger), the
    top-two margin, the column masses and the marginal errors."""
    p, I_off, J_off, c, r = _geo(case)
    D, c_out = GEOM.D, case.c_out
    f, g, fd, gd = oracle.sinkhorn_sparse(D, p, I_off, J_off, c, r, eps, c_out, mode, frac, n_iter, rho)
    nbr = oracle.knn(D, p, I_off, J_off, c, r, rho)
    T, nI, nJ = len(I_off) - 1, int(I_off[-1]), int(J_off[-1])
    rows = [[] for _ in range(nI)]
    for j in range(nJ):
        for i in nbr[j]:
            if i >= 0:
                rows[i].append(j)
    t_of_i = np.repeat(np.arange(T), np.diff(I_off))
    t_of_j = np.repeat(np.arange(T), np.diff(J_off))
    assign = np.full(nI, -1, np.int64)
    margin = np.zeros(nI)
    row_err = 0.0
    for i in range(nI):
        dd = t_of_i[i] if mode else 0
        js = np.array(sorted(rows[i]), np.int64)
        v = (g[js] - oracle.pair_costs(p[i], c[js], r[js], D)) / eps
        dv = (gd[dd] - c_out) / eps
        b1, b2, arg = -np.inf, -np.inf, -1
        for jj, x in zip(js, v):
            if x > b1:
                b1, b2, arg = x, b1, int(jj)
            elif x > b2:
                b2 = x
        if dv > b1:
            b1, b2, arg = dv, b1, -1
        elif dv > b2:
            b2 = dv
        assign[i] = arg
        margin[i] = np.exp(f[i] / eps + b1) - (np.exp(f[i] / eps + b2) if np.isfinite(b2) else 0.0)
        row_err = max(row_err, abs(np.exp(f[i] / eps + np.logaddexp.reduce(np.r_[v, dv])) - 1.0))
    U, O = oracle.masses(mode, frac, I_off, J_off)
    for d in range(T if mode else 1):
        if U[d] > 0:
            j0, j1 = (J_off[d], J_off[d + 1]) if mode else (0, nJ)
            fnext = eps * np.log(U[d]) - eps * np.logaddexp.reduce(np.r_[g[j0:j1] / eps, (gd[d] - c_out) / eps])
            row_err = max(row_err, abs(np.exp((fd[d] - fnext) / eps) - 1.0))
    q = np.zeros(nJ)
    col_err = 0.0
    for j in range(nJ):
        ii = nbr[j][nbr[j] >= 0]
        if len(ii):
            cost = oracle.pair_costs(p[ii], c[j], r[j], D)
            q[j] = np.exp((f[ii] + g[j] - cost) / eps).sum()
        dd = t_of_j[j] if mode else 0
        col_err = max(col_err, abs(q[j] + np.exp((g[j] + fd[dd]) / eps) - 1.0))
    return dict(f=f, g=g, dust=np.r_[fd, gd], nbr=nbr, assign=assign, margin=margin, q=q,
                marg_err=np.array([row_err, col_err]))


def _run(env, case, eps, mode, rho, n_iter, init=None):
    api = env["api"]
    ob, ms = to_device(case, env["dev"])
    out = api.cost_sinkhorn_sparse(env["h"], GEOM, ob, ms, eps, case.c_out, n_iter, rho=rho, dust_mode=mode,
                                   harvest=True, col_harvest=True, neighbours=True, init=init)
    env["torch"].cuda.synchronize()
    assert env["h"].device_status() == 0
    return {k: v.cpu().numpy() for k, v in out.items()}


def _compare(gpu, ref, eps, case):
    p, I_off, J_off, c, r = _geo(case)
    assert _check_neighbours(gpu["nbr"], ref["nbr"], p, I_off, J_off, c, r, range(len(ref["nbr"]))) == 0
    for k in ("f", "g", "dust"):
        err = np.abs(gpu[k].astype(np.float64) - ref[k])
        lim = TOL * (np.abs(ref[k]) + eps)
        assert np.all(err <= lim), (k, float((err / lim).max()))
    sure = ref["margin"] > 1e-3
    assert sure.mean() > 0.5
    np.testing.assert_array_equal(gpu["assign"][sure], ref["assign"][sure])
    np.testing.assert_allclose(gpu["margin"], ref["margin"], atol=1e-4)
    np.testing.assert_allclose(gpu["q"], ref["q"], atol=1e-4)
    np.testing.assert_allclose(gpu["marg_err"], ref["marg_err"], atol=1e-4)


@pytest.mark.parametrize("mode,rho", [(0, 8), (1, 8), (0, 1), (1, 32)])
def test_sparse_tiny_matches_oracle(env, mode, rho):
    case = make_case(sg.CONFIGS["tiny"])
    eps = case.cfg.eps
    _compare(_run(env, case, eps, mode, rho, 100), _reference(case, eps, mode, rho, 100), eps, case)


@pytest.mark.parametrize("mode", [0, 1])
def test_sparse_multi_tile_ragged_matches_oracle(env, mode):
    """60 grains, 8 angles: blocks of about 600 observed spots (two 512-spot
    row tiles, the second ragged) and 470 model spots (one ragged column
    tile)."""
    case = make_case(sg.CONFIGS["medium"], seed=11, n_grains=60, T=8)
    nI, nJ = np.diff(case.obs.I_off), np.diff(case.fw["J_off"])
    assert nI.max() > 512 and (nI % 512).min() > 0 and (nJ % 512).min() > 0
    rho, eps = 16, case.cfg.eps
    _compare(_run(env, case, eps, mode, rho, 40), _reference(case, eps, mode, rho, 40), eps, case)


def test_sparse_full_support_equals_dense(env):
    """With rho at least the largest observed block every pair is in the
    support: the sparse E-step is the dense one (laue_cost_sinkhorn)."""
    api, torch = env["api"], env["torch"]
    case = make_case(sg.CONFIGS["tiny"], seed=3)
    assert np.diff(case.obs.I_off).max() <= 64
    eps = case.cfg.eps
    ob, ms = to_device(case, env["dev"])
    for mode in (0, 1):
        sp = _run(env, case, eps, mode, 64, 80)
        de = api.cost_sinkhorn(env["h"], GEOM, ob, ms, eps, case.c_out, 80, dust_mode=mode, harvest=True)
        torch.cuda.synchronize()
        for k in ("f", "g", "dust"):
            want = de[k].cpu().numpy().astype(np.float64)
            assert np.all(np.abs(sp[k] - want) <= TOL * (np.abs(want) + eps)), k
        sure = de["margin"].cpu().numpy() > 1e-3
        np.testing.assert_array_equal(sp["assign"][sure], de["assign"].cpu().numpy()[sure])


def test_sparse_edge_cases(env):
    """An angle block with no observed spots, zero iterations, and a warm
    start that continues a run (30 + 30 iterations = 60)."""
    case = make_case(sg.CONFIGS["tiny"], seed=4)
    eps, rho = case.cfg.eps, 8
    # drop the observed spots of angle 2
    I_off = case.obs.I_off.copy()
    keep = np.r_[0:I_off[2], I_off[3]:I_off[-1]]
    n2 = I_off[3] - I_off[2]
    case.obs.p = case.obs.p[keep]
    case.obs.I_off = np.r_[I_off[:3], I_off[3:] - n2].astype(I_off.dtype)
    for mode in (0, 1):
        _compare(_run(env, case, eps, mode, rho, 50), _reference(case, eps, mode, rho, 50), eps, case)
    zero = _run(env, case, eps, 0, rho, 0)
    assert np.all(zero["f"] == 0) and np.all(zero["g"] == 0)
    import torch
    a = _run(env, case, eps, 1, rho, 30)
    dev = env["dev"]
    b = _run(env, case, eps, 1, rho, 30,
             init=(torch.tensor(a["f"], device=dev), torch.tensor(a["g"], device=dev),
                   torch.tensor(a["dust"], device=dev)))
    ref = _reference(case, eps, 1, rho, 60)
    for k in ("f", "g"):
        assert np.all(np.abs(b[k] - ref[k]) <= TOL * (np.abs(ref[k]) + eps)), k


def test_sparse_full_size_per_angle_blocks_match_oracle(env):
    """1000 grains, 90 angles, 70% uneven outliers, per-angle dustbins, rho =
    32: the whole workload in one call on the GPU, the oracle on the two
    smallest blocks alone.  The neighbour lists equal the oracle's except at
    near ties (at most 0.1% of the model spots, each a valid alternative); f,
    g and the dustbin potentials agree element by element."""
    from _cases import block_slices, oracle_parallel
    case = make_case(sg.CONFIGS["batched"], seed=0)
    eps, rho, n_iter, T = case.cfg.eps, 32, 30, case.cfg.T
    gpu = _run(env, case, eps, 1, rho, n_iter)
    nI, nJ = np.diff(case.obs.I_off), np.diff(case.fw["J_off"])
    blocks = [int(t) for t in np.argsort(nI * nJ)[:2]]
    calls = []
    for t in blocks:
        si, sj = block_slices(case, t)
        geo = (GEOM.D, case.obs.p[si], [0, si.stop - si.start], [0, sj.stop - sj.start], case.fw["center"][sj],
               case.fw["ray"][sj, :3])
        calls.append(("sinkhorn_sparse", geo + (eps, case.c_out, 1, 0.4, n_iter, rho), {}))
        calls.append(("knn", geo + (rho,), {}))
    res = oracle_parallel(calls)
    for k, t in enumerate(blocks):
        si, sj = block_slices(case, t)
        f, g, fd, gd = res[2 * k]
        nbr = res[2 * k + 1]
        want_nbr = np.where(nbr >= 0, nbr + si.start, -1)
        p, I_off, J_off, c, r = _geo(case)
        n_diff = _check_neighbours(gpu["nbr"][sj], want_nbr, p, I_off, J_off, c, r, range(sj.start, sj.stop))
        assert n_diff <= 1e-3 * (sj.stop - sj.start), n_diff
        for name, got, want in (("f", gpu["f"][si], f), ("g", gpu["g"][sj], g),
                                ("dust", gpu["dust"][[t, T + t]], np.r_[fd, gd])):
            err = np.abs(got.astype(np.float64) - want)
            lim = TOL * (np.abs(want) + eps)
            assert np.all(err <= lim), (t, name, float((err / lim).max()))


def test_sparse_full_size_global_fixed_point(env):
    """The same workload with global dustbins: the neighbour lists of sampled
    model spots are the rho nearest of their block (up to near ties), and
    after the last column update each sampled g_j is the sparse column update
    of the returned f over its listed support and the outlier-column
    potential (a property at any size)."""
    case = make_case(sg.CONFIGS["batched"], seed=0)
    eps, rho = case.cfg.eps, 32
    gpu = _run(env, case, eps, 0, rho, 50)
    p, I_off, J_off, c, r = _geo(case)
    fd = float(gpu["dust"][0])
    rng = np.random.default_rng(5)
    t_of_j = np.repeat(np.arange(len(I_off) - 1), np.diff(J_off))
    for j in rng.choice(int(J_off[-1]), 24, replace=False):
        t = t_of_j[j]
        i0, i1 = I_off[t], I_off[t + 1]
        cost = oracle.pair_costs(p[i0:i1], c[j], r[j], GEOM.D)
        order = np.lexsort((np.arange(i1 - i0), cost))[:rho]
        want = np.full(rho, -1)
        want[:len(order)] = order + i0
        _check_neighbours(gpu["nbr"][j:j + 1], want[None], p, I_off, J_off, c, r, [j])
        ii = gpu["nbr"][j][gpu["nbr"][j] >= 0]
        v = (gpu["f"][ii].astype(np.float64) - cost[ii - i0]) / eps
        want_g = -eps * np.logaddexp.reduce(np.r_[v, fd / eps])
        assert abs(gpu["g"][j] - want_g) <= TOL * (abs(want_g) + eps), (j, gpu["g"][j], want_g)
    me = gpu["marg_err"]
    assert 0 <= me[1] < 1e-4  # columns exact after the column update
