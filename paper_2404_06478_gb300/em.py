"""Multi-grain Sinkhorn-EM driver (paper Algorithm LaueOT, Section "The LaueOT
solver") over the C ABI, with deterministic annealing (Section "Deterministic
annealing") and optional capture of the whole solve as one CUDA graph.

The solve is one laue_em call.  Each EM step: refresh the frozen model list
at the current poses (laue_refresh), E-step at temperature eps_k
(laue_cost_sinkhorn, fixed number of Sinkhorn iterations from f = g = 0),
M-step (laue_mstep, or laue_mstep_adjoint).  A final E-step at the last poses
gives the hard assignment.  The temperature schedule starts at anneal_factor
eps_final and cools geometrically to eps_final at step ceil(0.75 n_em), then
holds.  The host only enqueues work: no step reads device data back.
"""
from __future__ import annotations

import dataclasses

import torch

from . import api


def eps_schedule(eps_final: float, n_em: int, k: int, factor: float = 100.0) -> float:
    """The library's annealing schedule (laue_anneal_eps); factor 1 means no
    annealing."""
    return api.anneal_eps(eps_final, n_em, k, factor)


@dataclasses.dataclass
class EMConfig:
    eps_final: float = 1.0
    n_em: int = 20
    n_sinkhorn: int = 100
    c_out: float = 2.25
    dust_mode: int = 0
    unmatched_frac: float = 0.4
    n_newton: int = 4
    n_mm: int = 4
    tol_x: float = 1e-6
    tol_R: float = 1e-9
    hreg: float = 1e-3
    anneal_factor: float = 100.0  # eps_init / eps_final
    mstep: str = "plain"          # "plain": laue_mstep; "adjoint": laue_mstep_adjoint
    lm_damping: float = 1e-3      # Levenberg-Marquardt damping of the adjoint M-step


class EMSolver:
    """Runs Algorithm LaueOT for fixed observed spots and a frozen model list
    through one laue_em call (refresh, E-step and M-step of every annealed
    step, then the final E-step with the read-out).

    R (N, 9) and x (N, 3) float32 device tensors are updated in place."""

    def __init__(self, h: api.Handle, geom, lat: api.Lattice, obs: api.ObsSpots, model: api.ModelSpots,
                 omega: torch.Tensor, cfg: EMConfig):
        self.h, self.geom, self.lat, self.obs, self.model = h, geom, lat, obs, model
        self.omega = omega.contiguous().float()
        self.cfg = cfg
        self.graph = None
        self.out = None

    def em(self, R, x, k_first=0, k_last=None, out=None):
        """laue_em over steps k_first .. k_last (default: the whole solve)."""
        c = self.cfg
        hreg = c.lm_damping if c.mstep == "adjoint" else c.hreg
        return api.em(self.h, self.geom, self.lat, self.obs, self.model, self.omega, R, x, c.eps_final, c.n_em,
                      c.n_sinkhorn, c.c_out, k_first=k_first, k_last=k_last, anneal=c.anneal_factor,
                      dust_mode=c.dust_mode, unmatched_frac=c.unmatched_frac, mstep=c.mstep, n_newton=c.n_newton,
                      n_mm=c.n_mm, tol_x=c.tol_x, tol_R=c.tol_R, hreg=hreg, out=out)

    def reserve(self, n_grains):
        """Size the workspace for every call of the solve (before any capture)."""
        h, obs, model = self.h, self.obs, self.model
        h.reserve(obs.T, n_obs=int(obs.p.shape[0]), n_model=model.n, n_grains=int(n_grains),
                  n_planes=int(self.lat.w_d0.shape[0]))

    def run(self, R, x, use_graph=False):
        """Full annealed solve; returns the final plan read-out (assign,
        margin, f, g, dust)."""
        self.reserve(x.shape[0])
        if not use_graph:
            return self.em(R, x)
        if self.graph is None:
            self._R, self._x = R, x
            self.out = api.em_outputs(self.obs, self.model, self.cfg.dust_mode)  # allocated before the capture
            s = torch.cuda.Stream()
            s.wait_stream(torch.cuda.current_stream())
            with torch.cuda.stream(s):
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=s):
                    self.em(self._R, self._x, out=self.out)
            torch.cuda.current_stream().wait_stream(s)
            self.graph = g
        if R.data_ptr() != self._R.data_ptr():
            self._R.copy_(R)
            self._x.copy_(x)
        self.graph.replay()
        if R.data_ptr() != self._R.data_ptr():
            R.copy_(self._R)
            x.copy_(self._x)
        return self.out


def step_graph(solver: EMSolver, R, x, k):
    """CUDA graph of one EM iteration (annealed step k < n_em: refresh, E-step
    with read-out, M-step) on the tensors R, x; returns (graph, outputs)."""
    solver.reserve(x.shape[0])
    out = api.em_outputs(solver.obs, solver.model, solver.cfg.dust_mode)  # allocated before the capture
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            solver.em(R, x, k_first=k, k_last=k, out=out)
    torch.cuda.current_stream().wait_stream(s)
    return g, out
