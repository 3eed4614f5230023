"""The library's start grid (laue_start_grid) against the oracle's: the same
super-Fibonacci orientations, the same cubic fundamental-zone selection in the
same order, the same cell-centre positions."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("n_full,sym,k,cube", [(240000, 24, 1, 5.0), (48000, 24, 2, 5.0), (20000, 1, 3, 4.0),
                                               (1, 1, 1, 5.0), (0, 24, 1, 5.0)])
def test_start_grid_matches_oracle(n_full, sym, k, cube):
    import torch
    from paper_2404_06478_gb300 import api, build
    build.build()
    dev = torch.device("cuda", 0)
    h = api.Handle(dev)
    R, x = api.start_grid(h, n_full, sym=sym, k=k, cube_mm=cube)
    torch.cuda.synchronize()
    Ro, xo = oracle.start_grid(n_full, sym=sym, k=k, cube=cube)
    assert R.shape[0] == len(Ro)
    if len(Ro):
        np.testing.assert_allclose(R.cpu().numpy().reshape(-1, 3, 3), Ro, atol=2e-6)
        np.testing.assert_allclose(x.cpu().numpy(), xo, atol=1e-6)
