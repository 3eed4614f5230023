"""The C-ABI library builds, loads and exports every entry point its header
declares; host-side helpers agree with the oracle.  No GPU needed."""
import re
import os
import ctypes

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def native():
    from paper_2404_06478_gb300 import build
    build.build()
    from paper_2404_06478_gb300 import _native
    return _native


def _declared():
    text = open(os.path.join(ROOT, "include", "laueot.h")).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*|size_t|long long|double)\s+(laue_\w+)\s*\(", text, re.M)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("laue_forward", "laue_cost_sinkhorn", "laue_mstep", "laue_prototype_select", "laue_index"):
        assert must in names


def test_library_exports_every_declared_symbol(native):
    L = native.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(native.exported_symbols()) == _declared()


def test_reflection_table_matches_oracle(native):
    import oracle
    from paper_2404_06478_gb300 import api
    for hmax, cen in ((4, 1), (6, 1), (3, 2), (3, 0)):
        w, nh, hk = api.reflections(2.87, hmax, cen)
        P = oracle.reflections(2.87, hmax, cen)
        np.testing.assert_array_equal(hk, P.hkl0)
        np.testing.assert_array_equal(nh, P.nharm)
        np.testing.assert_allclose(w[:, :3], P.w, atol=1e-7)
        np.testing.assert_allclose(w[:, 3], P.d0, rtol=1e-7)


def test_invalid_arguments_rejected_without_gpu(native):
    L = native.lib()
    M = ctypes.c_int(0)
    assert L.laue_reflections(2.87, 0, 1, 0, None, None, None, ctypes.byref(M)) == native.LAUE_ERR_INVALID_ARG
    assert L.laue_reflections(-1.0, 4, 1, 0, None, None, None, ctypes.byref(M)) == native.LAUE_ERR_INVALID_ARG
    assert L.laue_reflections(2.87, 4, 1, 0, None, None, None, ctypes.byref(M)) == native.LAUE_ERR_CAPACITY
    assert M.value == 145
    assert L.laue_create(None, 0) == native.LAUE_ERR_INVALID_ARG


def test_set_encoder_sizes_match_the_oracle(native):
    import oracle.proposal as op
    from paper_2404_06478_gb300 import proposal as pr
    L = native.lib()
    assert L.laue_lp_set_size() == op.KSET == pr.KSET
    assert L.laue_lp_param_count() == sum(int(np.prod(s)) for _, s in op.PARAM_SHAPES)
    assert [n for n, _ in op.PARAM_SHAPES] == [n for n, _ in pr.PARAM_SHAPES]


def test_index_retries_once_with_the_missing_workspace():
    """The SPOT matrix's size is known only after the single-grain fits.  When
    laue_index reports that it does not fit, the binding adds the missing
    bytes named in the library's message to the workspace and calls again.
    Host logic only: a stand-in library answers the calls, tensors stay on
    the CPU."""
    import torch
    from paper_2404_06478_gb300 import api
    from paper_2404_06478_gb300 import _native as N

    class FakeLib:
        def __init__(self):
            self.calls, self.ws_sizes = 0, []

        def laue_index_workspace_size(self, h, T, nI, S, n_max, M, out):
            out._obj.value = 1000
            return 0

        def laue_set_workspace(self, h, ptr, nbytes, stream):
            self.ws_sizes.append(nbytes)
            return 0

        def laue_index(self, *args):
            self.calls += 1
            if self.calls == 1:
                return N.LAUE_ERR_CAPACITY
            args[12]._obj.value = 2
            return 0

        def laue_last_error(self, h):
            return b"prototype_select: 300 nonzeros need 5000 more workspace bytes"

    class FakeHandle:
        def __init__(self):
            self.h, self.L, self.ws = None, FakeLib(), None

        def check(self, rc, what=""):
            if rc < 0:
                raise api.LaueError(rc, what)
            return rc

    h = FakeHandle()
    geom = __import__("synthgen").Geometry()
    lat = api.Lattice(torch.zeros(8, 4), torch.zeros(8, dtype=torch.int32))
    obs = api.ObsSpots(torch.zeros(10, 4), torch.tensor([0, 10], dtype=torch.int32))
    api._stream_saved = api._stream
    try:
        api._stream = lambda stream=None: None
        R, x, a = api.index(h, geom, lat, obs, torch.zeros(1), torch.zeros(3, 9), torch.zeros(3, 3), 1.0, 2.25, 4)
    finally:
        api._stream = api._stream_saved
    assert h.L.calls == 2
    assert h.L.ws_sizes[0] == 1000 + 256
    assert h.L.ws_sizes[1] == 1000 + 256 + 5000 + (1 << 20)
    assert R.shape == (2, 9) and x.shape == (2, 3) and a.shape == (10,)


def test_host_constants_match_oracle(native):
    """laue_c_out and laue_anneal_eps (host functions of the library) agree with
    the oracle's outlier cost and annealing schedule."""
    import oracle
    from paper_2404_06478_gb300 import api
    for sigma, D in ((0.5, 200.0), (0.143, 160.0), (1.2, 350.0)):
        assert api.c_out_for(sigma, D) == pytest.approx(oracle.c_out_for(sigma, D), rel=1e-14)
    for n_em in (1, 4, 20, 30):
        for k in range(n_em + 2):
            for fac in (100.0, 1000.0, 1.0):
                assert api.anneal_eps(1.5, n_em, k, fac) == pytest.approx(oracle.eps_schedule(1.5, n_em, k, fac),
                                                                           rel=1e-14)
    L = native.lib()
    assert L.laue_c_out(-1.0, 200.0) < 0 and L.laue_anneal_eps(1.0, -1, 0, 100.0) < 0


def test_general_lattice_tables_match_oracle(native):
    """laue_reciprocal_basis and laue_reflections_hkl (host functions) agree with
    the oracle's: the hexagonal ruby cell with its R-3c reflections, and a
    cubic cell given as a list.  Lines whose multiples are not 1..n of a base
    are rejected."""
    import oracle
    import synthgen as sg
    from paper_2404_06478_gb300 import api
    c = sg.RUBY
    B = api.reciprocal_basis(c.a, c.b, c.c, c.alpha, c.beta, c.gamma)
    Bo = oracle.reciprocal_basis(c.a, c.b, c.c, c.alpha, c.beta, c.gamma)
    np.testing.assert_allclose(B, Bo, atol=1e-15)
    for Bm, hkl in ((Bo, sg.ruby_hkl(4, 12)), (np.eye(3) / 2.87, sg.bcc_hkl(6)),
                    (oracle.reciprocal_basis(5.0, 6.0, 7.0, 80.0, 95.0, 105.0), sg.bcc_hkl(3))):
        w, nh, h0 = api.reflections_hkl(Bm, hkl)
        P = oracle.reflections_hkl(Bm, hkl)
        np.testing.assert_array_equal(h0, P.hkl0)
        np.testing.assert_array_equal(nh, P.nharm)
        np.testing.assert_allclose(w[:, :3], P.w, atol=1e-7)
        np.testing.assert_allclose(w[:, 3], P.d0, rtol=1e-7)
    with pytest.raises(Exception):
        api.reflections_hkl(np.eye(3), [[1, 0, 0], [3, 0, 0]])  # 1x and 3x without 2x
    with pytest.raises(ValueError):
        oracle.reflections_hkl(np.eye(3), [[1, 0, 0], [3, 0, 0]])
    with pytest.raises(Exception):
        api.reciprocal_basis(5.0, 5.0, 5.0, 10.0, 10.0, 170.0)  # angles that close no cell


@pytest.mark.parametrize("B", [1, 24, 128, 2048, 3001])
def test_set_encoder_batch_regions_are_disjoint(native, B):
    """The batch buffer's public regions lie inside laue_lp_batch_bytes, are
    256-byte aligned and do not overlap; region 1 (a transposed copy of the
    features that the weight gradients no longer need) is reported as -1."""
    L = native.lib()
    K, W, NOUT = 128, 256, 72
    sizes = {0: B * K * 64 * 2, 2: B * 9 * 4, 3: B * 4, 4: B * 9 * 4, 5: B * 3 * 4, 6: B * 4, 7: B * NOUT * 4,
             8: B * 4, 9: B * 4, 10: B * 4, 11: B * K * W * 2, 12: B * K * W * 2, 13: B * 2 * W * 4,
             14: B * NOUT * 4, 15: B * K * W * 2}
    total = L.laue_lp_batch_bytes(B)
    assert L.laue_lp_batch_offset(B, 1) == -1
    assert L.laue_lp_batch_offset(B, 16) == -1 and L.laue_lp_batch_offset(B, -1) == -1
    spans = sorted((L.laue_lp_batch_offset(B, r), sizes[r]) for r in sizes)
    for off, size in spans:
        assert off >= 0 and off % 256 == 0 and off + size <= total
    for (o1, s1), (o2, _) in zip(spans, spans[1:]):
        assert o1 + s1 <= o2
