"""The no-allocation E-step (laue_cost_sinkhorn_noalloc) against the
workspace-based laue_cost_sinkhorn and against the FP64 oracle.

The no-allocation variant exists for callers that cannot allocate device
memory (code running under stream capture, real-time loops, plugins whose
host framework owns all device memory); it uses a fixed device array of the
library instead of a caller workspace.  This file is collected last so that a
run stopping at the first failure has run every other test first."""
import numpy as np
import pytest

import oracle
import synthgen as sg
from _cases import GEOM, make_case, to_device

pytestmark = pytest.mark.gpu

TOL = 1e-4  # potentials: 1e-4 * (|f| + eps), as in the Sinkhorn parity tests


def test_no_alloc_matches_workspace_entry_point_twice():
    import torch
    from paper_2404_06478_gb300 import api, build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    case = make_case(sg.CONFIGS["medium"], seed=11, n_grains=60, T=8)
    ob, ms = to_device(case, dev)
    eps, n_iter = 1.0, 60
    h = api.Handle(dev)
    ref = api.cost_sinkhorn(h, GEOM, ob, ms, eps, case.c_out, n_iter, harvest=True, col_harvest=True)
    torch.cuda.synchronize()
    fw, obs = case.fw, case.obs
    of, og, ofd, ogd, _ = oracle.sinkhorn(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3],
                                          eps, case.c_out, 0, 0.4, n_iter)
    oh = oracle.harvest(GEOM.D, obs.p, obs.I_off, fw["J_off"], fw["center"], fw["ray"][:, :3], eps, case.c_out,
                        0, 0.4, of, og, ofd, ogd)
    orc = dict(f=of, g=og, dust=np.concatenate([ofd, ogd]))
    nI, nJ = int(ob.p.shape[0]), ms.n
    for call in range(2):
        f = torch.full((nI,), float("nan"), device=dev)
        g = torch.full((nJ,), float("nan"), device=dev)
        dust = torch.zeros(2, device=dev)
        assign = torch.full((nI,), -7, dtype=torch.int32, device=dev)
        margin = torch.zeros(nI, device=dev)
        merr = torch.zeros(2, device=dev)
        q = torch.zeros(nJ, device=dev)
        status = torch.full((1,), 99, dtype=torch.int32, device=dev)
        rc = api.cost_sinkhorn_noalloc(GEOM, ob, ms, eps, case.c_out, n_iter, f, g, dust, assign, margin, merr, q,
                                       status)
        torch.cuda.synchronize()
        assert rc == 0
        assert int(status.item()) == 0
        for name, got in (("f", f), ("g", g), ("dust", dust)):
            r = ref[name].double().cpu().numpy()
            d = np.abs(got.double().cpu().numpy() - r)
            assert np.all(d <= TOL * (np.abs(r) + eps)), (call, name, float(d.max()))
        np.testing.assert_array_equal(assign.cpu().numpy(), ref["assign"].cpu().numpy())
        # and against the oracle itself
        for name, got in (("f", f), ("g", g), ("dust", dust)):
            r = orc[name]
            d = np.abs(got.double().cpu().numpy() - r)
            assert np.all(d <= TOL * (np.abs(r) + eps)), (call, "oracle", name, float(d.max()))
        sure = oh["margin"] > 1e-3
        np.testing.assert_array_equal(assign.cpu().numpy()[sure], oh["assign"][sure])
        np.testing.assert_allclose(margin.cpu().numpy(), ref["margin"].cpu().numpy(), atol=1e-4)
        np.testing.assert_allclose(q.cpu().numpy(), ref["q"].cpu().numpy(), atol=1e-4)


def test_no_alloc_rejects_problems_beyond_its_scratch():
    import torch
    from paper_2404_06478_gb300 import api, build
    from paper_2404_06478_gb300 import _native as N
    build.build()
    dev = torch.device("cuda", 0)
    case = make_case(sg.CONFIGS["tiny"], seed=2)
    ob, ms = to_device(case, dev)
    big = api.ObsSpots(ob.p, ob.I_off)
    o_s = big.struct()
    o_s.n = 8_000_000  # rejected on the host before any kernel reads the arrays
    prm = api.ot_params(1.0, case.c_out, 5)
    g_s, m_s = api.geometry_struct(GEOM), ms.struct()
    f = torch.zeros(8, device=dev)
    g = torch.zeros(8, device=dev)
    rc = N.lib().laue_cost_sinkhorn_noalloc(api.ctypes.byref(g_s), api.ctypes.byref(o_s), api.ctypes.byref(m_s),
                                            api.ctypes.byref(prm), api._ptr(f), api._ptr(g), None, None, None, None,
                                            None, None, api._stream())
    assert rc == N.LAUE_ERR_CAPACITY
