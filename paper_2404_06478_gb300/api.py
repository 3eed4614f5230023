"""Python binding of the LaueOT C ABI (same names as include/laueot.h).

Marshalling only: tensors are handed to liblaueot.so by data pointer together
with the current CUDA stream; PyTorch provides device memory and streams.  No
step of the hot path runs here, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import re
import dataclasses
import math

import numpy as np
import torch

from . import _native as N


class LaueError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("LaueOT error %d: %s" % (code, msg))
        self.code = code


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def c_out_for(sigma_mm: float, D: float) -> float:
    """laue_c_out: outlier cost for spot noise sigma_mm at distance D."""
    v = N.lib().laue_c_out(float(sigma_mm), float(D))
    if v < 0:
        raise LaueError(N.LAUE_ERR_INVALID_ARG, "laue_c_out: sigma_mm and D must be > 0")
    return v


def anneal_eps(eps_final: float, n_em: int, k: int, factor: float = 100.0) -> float:
    """laue_anneal_eps: temperature of annealed step k."""
    v = N.lib().laue_anneal_eps(float(eps_final), int(n_em), int(k), float(factor))
    if v < 0:
        raise LaueError(N.LAUE_ERR_INVALID_ARG, "laue_anneal_eps: bad arguments")
    return v


def geometry_struct(geom) -> N.LaueGeometry:
    g = N.LaueGeometry()
    g.beam[:] = [float(v) for v in geom.beam]
    g.lam_min, g.lam_max, g.D = float(geom.lam_min), float(geom.lam_max), float(geom.D)
    g.n_det = len(geom.detectors)
    for k, det in enumerate(geom.detectors):
        g.det_centre[k][:] = [float(v) for v in det.centre]
        g.det_normal[k][:] = [float(v) for v in det.normal]
        g.det_half[k] = float(det.half)
        g.det_D[k] = float(getattr(det, "D", 0.0))
    return g


def reflections(a: float, hmax: int, centering: int = 1):
    """Plane table on the host: (w_d0 (M, 4) float32, nharm (M,) int32, hkl0 (M, 3) int32)."""
    L = N.lib()
    M = ctypes.c_int(0)
    L.laue_reflections(a, hmax, centering, 0, None, None, None, ctypes.byref(M))
    w = np.zeros((M.value, 4), np.float32)
    nh = np.zeros(M.value, np.int32)
    hk = np.zeros((M.value, 3), np.int32)
    rc = L.laue_reflections(a, hmax, centering, M.value, w.ctypes.data_as(ctypes.c_void_p),
                            nh.ctypes.data_as(ctypes.c_void_p), hk.ctypes.data_as(ctypes.c_void_p),
                            ctypes.byref(M))
    if rc != 0:
        raise LaueError(rc, "laue_reflections failed")
    return w, nh, hk


def reciprocal_basis(a, b, c, alpha, beta, gamma) -> np.ndarray:
    """laue_reciprocal_basis: B (3, 3), columns b1 b2 b3."""
    B = np.zeros(9)
    rc = N.lib().laue_reciprocal_basis(float(a), float(b), float(c), float(alpha), float(beta), float(gamma),
                                       B.ctypes.data_as(ctypes.c_void_p))
    if rc != 0:
        raise LaueError(rc, "laue_reciprocal_basis: bad cell")
    return B.reshape(3, 3)


def reflections_hkl(B, hkl):
    """laue_reflections_hkl on the host: (w_d0 (M, 4) float32, nharm (M,), hkl0 (M, 3))."""
    L = N.lib()
    Bc = np.ascontiguousarray(np.asarray(B, np.float64).reshape(9))
    hk = np.ascontiguousarray(np.asarray(hkl, np.int32).reshape(-1, 3))
    M = ctypes.c_int(0)
    args = (Bc.ctypes.data_as(ctypes.c_void_p), hk.ctypes.data_as(ctypes.c_void_p), len(hk))
    rc = L.laue_reflections_hkl(*args, 0, None, None, None, ctypes.byref(M))
    if rc not in (0, N.LAUE_ERR_CAPACITY):
        raise LaueError(rc, "laue_reflections_hkl failed")
    w = np.zeros((M.value, 4), np.float32)
    nh = np.zeros(M.value, np.int32)
    h0 = np.zeros((M.value, 3), np.int32)
    rc = L.laue_reflections_hkl(*args, M.value, w.ctypes.data_as(ctypes.c_void_p), nh.ctypes.data_as(ctypes.c_void_p),
                                h0.ctypes.data_as(ctypes.c_void_p), ctypes.byref(M))
    if rc != 0:
        raise LaueError(rc, "laue_reflections_hkl failed")
    return w, nh, h0


@dataclasses.dataclass
class Lattice:
    w_d0: torch.Tensor   # (M, 4) float32 device
    nharm: torch.Tensor  # (M,) int32 device

    def struct(self):
        return N.LaueLattice(_ptr(self.w_d0), _ptr(self.nharm), int(self.w_d0.shape[0]))

    @staticmethod
    def cubic(a, hmax, centering=1, device="cuda"):
        w, nh, _ = reflections(a, hmax, centering)
        return Lattice(torch.from_numpy(w).to(device), torch.from_numpy(nh).to(device))

    @staticmethod
    def from_hkl(B, hkl, device="cuda"):
        """Any lattice: reciprocal basis B and the allowed reflections."""
        w, nh, _ = reflections_hkl(B, hkl)
        return Lattice(torch.from_numpy(w).to(device), torch.from_numpy(nh).to(device))


@dataclasses.dataclass
class ObsSpots:
    p: torch.Tensor      # (n, 4) float32 device
    I_off: torch.Tensor  # (T+1,) int32 device

    @property
    def T(self):
        return int(self.I_off.shape[0]) - 1

    def struct(self):
        return N.LaueObsSpots(self.T, int(self.p.shape[0]), _ptr(self.I_off), _ptr(self.p))

    @staticmethod
    def from_numpy(p, I_off, device="cuda"):
        P = np.zeros((len(p), 4), np.float32)
        P[:, :3] = p
        return ObsSpots(torch.from_numpy(P).to(device),
                        torch.from_numpy(np.asarray(I_off, np.int32)).to(device))


@dataclasses.dataclass
class ModelSpots:
    T: int
    n: int
    J_off: torch.Tensor
    grain: torch.Tensor
    plane: torch.Tensor
    angle: torch.Tensor
    ray: torch.Tensor
    center: torch.Tensor
    spot: torch.Tensor

    @property
    def capacity(self):
        return int(self.grain.shape[0])

    def struct(self):
        return N.LaueModelSpots(self.T, self.n, self.capacity, _ptr(self.J_off), _ptr(self.grain),
                                _ptr(self.plane), _ptr(self.angle), _ptr(self.ray), _ptr(self.center),
                                _ptr(self.spot))

    @staticmethod
    def empty(T, capacity, device="cuda"):
        cap = max(int(capacity), 1)
        z = lambda *s, dt=torch.int32: torch.zeros(*s, dtype=dt, device=device)
        return ModelSpots(T, 0, z(T + 1), z(cap), z(cap), z(cap), z(cap, 4, dt=torch.float32),
                          z(cap, 4, dt=torch.float32), z(cap, 4, dt=torch.float32))

    @staticmethod
    def from_numpy(J_off, grain, plane, ray4, center3, spot3=None, det=None, device="cuda"):
        """Model list from host arrays (J_off (T+1,), labels (n,), ray4 (n, 4) =
        (r, lambda), center3 (n, 3), spot3 (n, 3), det (n,))."""
        J_off = np.asarray(J_off, np.int32)
        T, n = len(J_off) - 1, int(J_off[-1])
        out = ModelSpots.empty(T, n, device=device)
        out.n = n
        t = np.repeat(np.arange(T, dtype=np.int32), np.diff(J_off))
        c4 = np.zeros((n, 4), np.float32)
        c4[:, :3] = center3
        s4 = np.zeros((n, 4), np.float32)
        if spot3 is not None:
            s4[:, :3] = spot3
        if det is not None:
            s4[:, 3] = det
        cp = lambda dst, src: dst[:n].copy_(torch.from_numpy(np.ascontiguousarray(src)))
        out.J_off.copy_(torch.from_numpy(J_off))
        if n:
            cp(out.grain, np.asarray(grain, np.int32))
            cp(out.plane, np.asarray(plane, np.int32))
            cp(out.angle, t)
            cp(out.ray, np.asarray(ray4, np.float32))
            cp(out.center, c4)
            cp(out.spot, s4)
        return out

    def truncated(self):
        n = self.n
        return ModelSpots(self.T, n, self.J_off, self.grain[:n], self.plane[:n], self.angle[:n],
                          self.ray[:n], self.center[:n], self.spot[:n])


class Handle:
    """laue_create / laue_destroy plus a workspace tensor owned by this object."""

    def __init__(self, device=None):
        dev = torch.device(device) if device is not None else torch.device("cuda")
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.L = N.lib()
        h = ctypes.c_void_p()
        rc = self.L.laue_create(ctypes.byref(h), self.device.index or 0)
        if rc != 0:
            raise LaueError(rc, "laue_create failed")
        self.h = h
        self.ws = None

    def close(self):
        if self.h:
            self.L.laue_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, rc, what=""):
        if rc < 0:
            msg = self.L.laue_last_error(self.h)
            raise LaueError(rc, (what + ": " if what else "") + (msg.decode() if msg else ""))
        return rc

    def workspace_size(self, T, n_obs=0, n_model=0, n_grains=0, n_planes=0, n_starts=0, n_candidates=0) -> int:
        d = N.LaueProblemDims(T, n_obs, n_model, n_grains, n_planes, n_starts, n_candidates)
        b = ctypes.c_size_t()
        self.check(self.L.laue_workspace_size(self.h, ctypes.byref(d), ctypes.byref(b)), "workspace_size")
        return b.value

    def reserve(self, T, n_obs=0, n_model=0, n_grains=0, n_planes=0, n_starts=0, n_candidates=0, extra=0,
                stream=None):
        need = self.workspace_size(T, n_obs, n_model, n_grains, n_planes, n_starts, n_candidates) + int(extra)
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
            self.check(self.L.laue_set_workspace(self.h, _ptr(self.ws), self.ws.numel(), _stream(stream)),
                       "set_workspace")
        return self.ws

    def reserve_bytes(self, need, stream=None):
        """Grow the workspace to at least `need` bytes (keeps a larger one)."""
        if self.ws is None or self.ws.numel() < need:
            self.ws = torch.empty(int(need) + 256, dtype=torch.uint8, device=self.device)
            self.check(self.L.laue_set_workspace(self.h, _ptr(self.ws), self.ws.numel(), _stream(stream)),
                       "set_workspace")
        return self.ws

    def alu_peaks(self, stream=None) -> dict:
        """Measured pipe throughputs (ops/s) of this device."""
        self.reserve(1, stream=stream)
        out = (ctypes.c_double * 6)()
        self.check(self.L.laue_alu_peaks(self.h, out, _stream(stream)), "alu_peaks")
        return dict(ffma=out[0], ffma2=out[1], ex2=out[2], rsqrt=out[3], lg2=out[4], sm_count=int(out[5]))

    def set_launch_shape(self, row_shape, col_shape):
        self.check(self.L.laue_set_launch_shape(self.h, int(row_shape), int(col_shape)), "set_launch_shape")

    def counters(self, stream=None):
        """laue_read_counters: dict of the device counters since the last read."""
        v = (ctypes.c_longlong * 5)()
        self.check(self.L.laue_read_counters(self.h, _stream(stream), v, 5), "read_counters")
        return dict(exact_rows=v[0], exact_cols=v[1], fit_pairs=v[2], pass_pairs=v[3], mstep_pairs=v[4])

    def set_pair_skipping(self, enable: bool):
        self.check(self.L.laue_set_pair_skipping(self.h, 1 if enable else 0), "set_pair_skipping")

    def exact_lse_count(self, stream=None):
        """(rows, columns) recomputed on the exact log-sum-exp path since the last read."""
        c = self.counters(stream)
        return c["exact_rows"], c["exact_cols"]

    def device_status(self, stream=None) -> int:
        v = ctypes.c_int(0)
        self.check(self.L.laue_device_status(self.h, _stream(stream), ctypes.byref(v)), "device_status")
        return v.value


def forward(h: Handle, geom, lat: Lattice, R, x, omega, capacity=None, stream=None) -> ModelSpots:
    """laue_forward: visible model spots of grains (R (N,3,3), x (N,3)) at angles omega (T,)."""
    R = R.reshape(-1, 9).contiguous().float()
    x = x.reshape(-1, 3).contiguous().float()
    omega = omega.contiguous().float()
    N_, T = int(R.shape[0]), int(omega.shape[0])
    M = int(lat.w_d0.shape[0])
    h.reserve(T, n_grains=N_, n_planes=M, stream=stream)
    cap = capacity if capacity is not None else max(64, N_ * T * 16)
    out = ModelSpots.empty(T, cap, device=R.device)
    st = out.struct()
    total = ctypes.c_int(0)
    g = geometry_struct(geom)
    ls = lat.struct()
    rc = h.L.laue_forward(h.h, ctypes.byref(g), ctypes.byref(ls), _ptr(R), _ptr(x), N_, _ptr(omega), T,
                          ctypes.byref(st), ctypes.byref(total), _stream(stream))
    if rc == N.LAUE_ERR_CAPACITY and capacity is None:
        out = ModelSpots.empty(T, total.value, device=R.device)
        st = out.struct()
        rc = h.L.laue_forward(h.h, ctypes.byref(g), ctypes.byref(ls), _ptr(R), _ptr(x), N_, _ptr(omega), T,
                              ctypes.byref(st), ctypes.byref(total), _stream(stream))
    h.check(rc, "laue_forward")
    out.n = total.value
    return out


def refresh(h: Handle, geom, lat: Lattice, R, x, omega, model: ModelSpots, stream=None):
    R = R.reshape(-1, 9).contiguous().float()
    x = x.reshape(-1, 3).contiguous().float()
    st = model.struct()
    g = geometry_struct(geom)
    ls = lat.struct()
    h.check(h.L.laue_refresh(h.h, ctypes.byref(g), ctypes.byref(ls), _ptr(R), _ptr(x),
                             _ptr(omega.contiguous().float()), ctypes.byref(st), _stream(stream)),
            "laue_refresh")


def ot_params(eps, c_out, n_iter, dust_mode=0, unmatched_frac=0.4, warm_start=False, kappa=0.0, lam=0.0):
    """dust_mode 0 / 1: balanced OT with global / per-angle dustbins; 2:
    unbalanced OT with marginal weights kappa (observed) and lam (model)."""
    return N.LaueOTParams(float(unmatched_frac), float(eps), float(c_out), int(n_iter), int(dust_mode),
                          1 if warm_start else 0, float(kappa), float(lam), 0)


def cost_sinkhorn(h: Handle, geom, obs: ObsSpots, model: ModelSpots, eps, c_out, n_iter, dust_mode=0,
                  unmatched_frac=0.4, harvest=True, col_harvest=False, init=None, kappa=0.0, lam=0.0, stream=None):
    """laue_cost_sinkhorn; returns dict of device tensors f, g, dust and, with
    harvest, assign, margin, marg_err (and q with col_harvest)."""
    dev = obs.p.device
    T = obs.T
    nI, nJ = int(obs.p.shape[0]), model.n
    h.reserve(T, n_obs=nI, n_model=nJ, stream=stream)
    nd = T if dust_mode else 1
    out = {}
    if init is not None:
        f, g, dust = (t.clone().float().contiguous() for t in init)
    else:
        f = torch.zeros(max(nI, 1), device=dev)
        g = torch.zeros(max(nJ, 1), device=dev)
        dust = torch.zeros(2 * nd, device=dev)
    assign = torch.empty(max(nI, 1), dtype=torch.int32, device=dev) if harvest else None
    margin = torch.empty(max(nI, 1), device=dev) if harvest else None
    merr = torch.empty(2, device=dev) if (harvest or col_harvest) else None
    q = torch.empty(max(nJ, 1), device=dev) if col_harvest else None
    prm = ot_params(eps, c_out, n_iter, dust_mode, unmatched_frac, init is not None, kappa, lam)
    g_s = geometry_struct(geom)
    o_s = obs.struct()
    m_s = model.struct()
    h.check(h.L.laue_cost_sinkhorn(h.h, ctypes.byref(g_s), ctypes.byref(o_s), ctypes.byref(m_s),
                                   ctypes.byref(prm), _ptr(f), _ptr(g), _ptr(dust), _ptr(assign), _ptr(margin),
                                   _ptr(merr), _ptr(q), _stream(stream)), "laue_cost_sinkhorn")
    out.update(f=f[:nI], g=g[:nJ], dust=dust)
    if harvest:
        out.update(assign=assign[:nI], margin=margin[:nI])
    if merr is not None:
        out["marg_err"] = merr
    if col_harvest:
        out["q"] = q[:nJ]
    return out


def cost_sinkhorn_sparse(h: Handle, geom, obs: ObsSpots, model: ModelSpots, eps, c_out, n_iter, rho=32,
                         dust_mode=0, unmatched_frac=0.4, harvest=True, col_harvest=False, init=None,
                         neighbours=False, stream=None):
    """laue_cost_sinkhorn_sparse: the E-step on the rho-nearest-neighbour
    support; returns the outputs of cost_sinkhorn (and nbr with neighbours)."""
    dev = obs.p.device
    T = obs.T
    nI, nJ = int(obs.p.shape[0]), model.n
    b = ctypes.c_size_t()
    h.check(h.L.laue_sparse_workspace_size(T, nI, nJ, int(rho), ctypes.byref(b)), "sparse_workspace_size")
    h.reserve_bytes(b.value, stream=stream)
    nd = T if dust_mode else 1
    if init is not None:
        f, g, dust = (t.clone().float().contiguous() for t in init)
    else:
        f = torch.zeros(max(nI, 1), device=dev)
        g = torch.zeros(max(nJ, 1), device=dev)
        dust = torch.zeros(2 * nd, device=dev)
    assign = torch.empty(max(nI, 1), dtype=torch.int32, device=dev) if harvest else None
    margin = torch.empty(max(nI, 1), device=dev) if harvest else None
    merr = torch.empty(2, device=dev) if (harvest or col_harvest) else None
    q = torch.empty(max(nJ, 1), device=dev) if col_harvest else None
    nbr = torch.empty(max(nJ * int(rho), 1), dtype=torch.int32, device=dev) if neighbours else None
    prm = ot_params(eps, c_out, n_iter, dust_mode, unmatched_frac, init is not None)
    g_s = geometry_struct(geom)
    o_s = obs.struct()
    m_s = model.struct()
    h.check(h.L.laue_cost_sinkhorn_sparse(h.h, ctypes.byref(g_s), ctypes.byref(o_s), ctypes.byref(m_s),
                                          ctypes.byref(prm), int(rho), _ptr(f), _ptr(g), _ptr(dust), _ptr(assign),
                                          _ptr(margin), _ptr(merr), _ptr(q), _ptr(nbr), _stream(stream)),
            "laue_cost_sinkhorn_sparse")
    out = dict(f=f[:nI], g=g[:nJ], dust=dust)
    if harvest:
        out.update(assign=assign[:nI], margin=margin[:nI])
    if merr is not None:
        out["marg_err"] = merr
    if col_harvest:
        out["q"] = q[:nJ]
    if neighbours:
        out["nbr"] = nbr[:nJ * int(rho)].view(nJ, int(rho))
    return out


def mparams(eps, n_newton=4, n_mm=4, tol_x=1e-6, tol_R=1e-9, hreg=1e-3):
    return N.LaueMParams(float(eps), int(n_newton), int(n_mm), float(tol_x), float(tol_R), float(hreg))


def mstep(h: Handle, geom, lat: Lattice, obs: ObsSpots, model: ModelSpots, f, g, eps, omega, R, x,
          n_newton=4, n_mm=4, tol_x=1e-6, tol_R=1e-9, hreg=1e-3, step_norms=None, stream=None):
    """laue_mstep: updates R ((N, 9) or (N, 3, 3) float32, contiguous) and x
    ((N, 3)) in place from the E-step potentials f, g (model must hold the
    E-step rays and centres)."""
    N_ = int(x.shape[0])
    h.reserve(obs.T, n_obs=int(obs.p.shape[0]), n_model=model.n, n_grains=N_,
              n_planes=int(lat.w_d0.shape[0]), stream=stream)
    prm = mparams(eps, n_newton, n_mm, tol_x, tol_R, hreg)
    g_s, o_s, m_s, l_s = geometry_struct(geom), obs.struct(), model.struct(), lat.struct()
    h.check(h.L.laue_mstep(h.h, ctypes.byref(g_s), ctypes.byref(l_s), ctypes.byref(o_s), ctypes.byref(m_s),
                           _ptr(f), _ptr(g), ctypes.byref(prm), _ptr(omega), _ptr(R), _ptr(x), N_,
                           _ptr(step_norms), _stream(stream)), "laue_mstep")


def em_outputs(obs: ObsSpots, model: ModelSpots, dust_mode=0, harvest=True):
    """Output tensors of laue_em (f, g, dust, and assign, margin with harvest)."""
    dev = obs.p.device
    nI, nJ, nd = int(obs.p.shape[0]), model.n, obs.T if dust_mode else 1
    out = dict(f=torch.zeros(max(nI, 1), device=dev), g=torch.zeros(max(nJ, 1), device=dev),
               dust=torch.zeros(2 * nd, device=dev))
    if harvest:
        out["assign"] = torch.empty(max(nI, 1), dtype=torch.int32, device=dev)
        out["margin"] = torch.empty(max(nI, 1), device=dev)
    return out


def em(h: Handle, geom, lat: Lattice, obs: ObsSpots, model: ModelSpots, omega, R, x, eps_final, n_em, n_sinkhorn,
       c_out, k_first=0, k_last=None, anneal=100.0, dust_mode=0, unmatched_frac=0.4, mstep="plain", n_newton=4,
       n_mm=4, tol_x=1e-6, tol_R=1e-9, hreg=1e-3, out=None, harvest=True, stream=None):
    """laue_em: steps k_first .. k_last (default n_em: the whole solve and its
    final E-step) of the annealed EM on the frozen model list, R (N, 9) and
    x (N, 3) updated in place; returns dict f, g, dust (and assign, margin of
    step k_last's E-step with harvest).  `out` reuses the output tensors of a
    previous call (no allocation, e.g. under graph capture)."""
    n_grains = int(x.shape[0])
    if out is None:
        out = em_outputs(obs, model, dust_mode, harvest)
    prm = N.LaueEMParams(float(unmatched_frac), float(eps_final), float(c_out), float(anneal), int(n_em),
                         int(n_sinkhorn), int(dust_mode), 1 if mstep == "adjoint" else 0, int(k_first),
                         int(n_em if k_last is None else k_last), mparams(eps_final, n_newton, n_mm, tol_x, tol_R, hreg))
    g_s, l_s, o_s, m_s = geometry_struct(geom), lat.struct(), obs.struct(), model.struct()
    h.check(h.L.laue_em(h.h, ctypes.byref(g_s), ctypes.byref(l_s), ctypes.byref(o_s), _ptr(omega),
                        ctypes.byref(m_s), _ptr(R), _ptr(x), n_grains, ctypes.byref(prm), _ptr(out["f"]), _ptr(out["g"]),
                        _ptr(out["dust"]), _ptr(out.get("assign")), _ptr(out.get("margin")), _stream(stream)),
            "laue_em")
    return out


def mstep_adjoint(h: Handle, geom, lat: Lattice, obs: ObsSpots, model: ModelSpots, f, g, eps, omega, R, x,
                  n_steps=4, lam=1e-3, step_norms=None, stream=None):
    """laue_mstep_adjoint: damped Gauss-Newton M-step on the OT-weighted cost
    (plan held at the E-step); updates R ((N, 9) float32) and x ((N, 3)) in place."""
    N_ = int(x.shape[0])
    h.reserve(obs.T, n_obs=int(obs.p.shape[0]), n_model=model.n, n_grains=N_,
              n_planes=int(lat.w_d0.shape[0]), stream=stream)
    prm = mparams(eps, n_steps, 0, 0.0, 0.0, lam)
    g_s, o_s, m_s, l_s = geometry_struct(geom), obs.struct(), model.struct(), lat.struct()
    h.check(h.L.laue_mstep_adjoint(h.h, ctypes.byref(g_s), ctypes.byref(l_s), ctypes.byref(o_s), ctypes.byref(m_s),
                                   _ptr(f), _ptr(g), ctypes.byref(prm), _ptr(omega), _ptr(R), _ptr(x), N_,
                                   _ptr(step_norms), _stream(stream)), "laue_mstep_adjoint")


def objective_grad(h: Handle, geom, lat: Lattice, obs: ObsSpots, model: ModelSpots, f, g, eps, omega, R, x,
                   stream=None):
    """laue_objective_grad: (grad (N, 6) = [dE/dw, dE/dx], value (N,))."""
    N_ = int(x.shape[0])
    h.reserve(obs.T, n_obs=int(obs.p.shape[0]), n_model=model.n, n_grains=N_,
              n_planes=int(lat.w_d0.shape[0]), stream=stream)
    grad = torch.empty(max(N_, 1), 6, device=x.device)
    val = torch.empty(max(N_, 1), device=x.device)
    g_s, o_s, m_s, l_s = geometry_struct(geom), obs.struct(), model.struct(), lat.struct()
    h.check(h.L.laue_objective_grad(h.h, ctypes.byref(g_s), ctypes.byref(l_s), ctypes.byref(o_s),
                                    ctypes.byref(m_s), _ptr(f), _ptr(g), float(eps), _ptr(omega), _ptr(R),
                                    _ptr(x), N_, _ptr(grad), _ptr(val), _stream(stream)), "laue_objective_grad")
    return grad[:N_], val[:N_]


def axis_angle(h: Handle, w, R0, with_jacobian=False, stream=None):
    """laue_axis_angle: R = exp([w]x) R0 and optionally J_l(w)^T."""
    N_ = int(w.shape[0])
    R = torch.empty(max(N_, 1), 9, device=w.device)
    J = torch.empty(max(N_, 1), 9, device=w.device) if with_jacobian else None
    h.check(h.L.laue_axis_angle(h.h, _ptr(w.contiguous()), _ptr(R0.reshape(-1, 9).contiguous()), _ptr(R),
                                _ptr(J), N_, _stream(stream)), "laue_axis_angle")
    return (R[:N_], J[:N_]) if with_jacobian else R[:N_]


def axis_angle_vjp(h: Handle, w, grad, gout=None, stream=None):
    """laue_axis_angle_vjp: (gw (N, 3), gx (N, 3)) from a left-perturbation
    gradient grad (N, 6) at R = exp([w]x) R0, scaled by gout (N,)."""
    N_ = int(w.shape[0])
    gw = torch.empty(max(N_, 1), 3, device=w.device)
    gx = torch.empty(max(N_, 1), 3, device=w.device)
    go = gout.contiguous().float() if gout is not None else None
    h.check(h.L.laue_axis_angle_vjp(h.h, _ptr(w.contiguous().float()), _ptr(grad.contiguous().float()), _ptr(go),
                                    _ptr(gw), _ptr(gx), N_, _stream(stream)), "laue_axis_angle_vjp")
    return gw[:N_], gx[:N_]


def start_grid(h: Handle, n_full: int, sym: int = 24, k: int = 1, cube_mm: float = 5.0, device=None, stream=None):
    """laue_start_grid: (R (S, 9), x (S, 3)) device tensors of the start grid."""
    dev = device if device is not None else h.device
    h.reserve(1, extra=4 * (int(n_full) // 1024 + 1) + 1024, stream=stream)
    S = ctypes.c_longlong(0)
    h.check(h.L.laue_start_grid(h.h, int(n_full), int(sym), int(k), float(cube_mm), 0, None, None, ctypes.byref(S),
                                _stream(stream)), "laue_start_grid")
    R = torch.empty(max(S.value, 1), 9, device=dev)
    x = torch.empty(max(S.value, 1), 3, device=dev)
    h.check(h.L.laue_start_grid(h.h, int(n_full), int(sym), int(k), float(cube_mm), S.value, _ptr(R), _ptr(x),
                                ctypes.byref(S), _stream(stream)), "laue_start_grid")
    return R[:S.value], x[:S.value]


def single_fit(h: Handle, geom, lat: Lattice, obs: ObsSpots, omega, R0, x0, eps_final, k_max, c_out,
               f_out=0.1, n_newton=4, n_mm=4, tol_x=1e-6, tol_R=1e-9, hreg=1e-3, anneal=100.0, recut=False,
               stream=None):
    """laue_single_fit: (R (S, 9), x (S, 3), keep (S,) bool, unmatched (S,))."""
    R0 = R0.reshape(-1, 9).contiguous().float()
    x0 = x0.reshape(-1, 3).contiguous().float()
    S = int(R0.shape[0])
    h.reserve(obs.T, n_obs=int(obs.p.shape[0]), n_planes=int(lat.w_d0.shape[0]), n_starts=S, stream=stream)
    Ro = torch.empty(max(S, 1), 9, device=R0.device)
    xo = torch.empty(max(S, 1), 3, device=R0.device)
    keep = torch.empty(max(S, 1), dtype=torch.int32, device=R0.device)
    unm = torch.empty(max(S, 1), device=R0.device)
    prm = N.LaueSingleParams(float(eps_final), float(c_out), float(f_out), int(k_max),
                             mparams(eps_final, n_newton, n_mm, tol_x, tol_R, hreg), float(anneal),
                             1 if recut else 0)
    g_s, o_s, l_s = geometry_struct(geom), obs.struct(), lat.struct()
    h.check(h.L.laue_single_fit(h.h, ctypes.byref(g_s), ctypes.byref(l_s), ctypes.byref(o_s), _ptr(omega), _ptr(R0),
                                _ptr(x0), S, ctypes.byref(prm), _ptr(Ro), _ptr(xo), _ptr(keep), _ptr(unm),
                                _stream(stream)), "laue_single_fit")
    return Ro[:S], xo[:S], keep[:S].bool(), unm[:S]


def prototype_select(h: Handle, geom, lat: Lattice, obs: ObsSpots, omega, candR, candX, eps_s, c_out, k_max,
                     stream=None):
    """laue_prototype_select: (order (k_max,) int32, gains (k_max,), k_star)."""
    candR = candR.reshape(-1, 9).contiguous().float()
    candX = candX.reshape(-1, 3).contiguous().float()
    Nc = int(candR.shape[0])
    dev = candR.device
    order = torch.empty(max(k_max, 1), dtype=torch.int32, device=dev)
    gains = torch.empty(max(k_max, 1), device=dev)
    extra = 1 << 20
    for attempt in range(3):
        h.reserve(obs.T, n_obs=int(obs.p.shape[0]), n_planes=int(lat.w_d0.shape[0]), n_starts=1,
                  n_candidates=max(Nc, 1), extra=extra, stream=stream)
        ks = ctypes.c_int(0)
        nnz = ctypes.c_longlong(0)
        g_s, o_s, l_s = geometry_struct(geom), obs.struct(), lat.struct()
        rc = h.L.laue_prototype_select(h.h, ctypes.byref(g_s), ctypes.byref(l_s), ctypes.byref(o_s), _ptr(omega),
                                       _ptr(candR), _ptr(candX), Nc, float(eps_s), float(c_out), int(k_max),
                                       _ptr(order), _ptr(gains), ctypes.byref(ks), ctypes.byref(nnz), _stream(stream))
        if rc == N.LAUE_ERR_CAPACITY and nnz.value > 0:
            extra = 8 * nnz.value + (1 << 20)
            continue
        h.check(rc, "laue_prototype_select")
        return order[:k_max], gains[:k_max], ks.value
    h.check(rc, "laue_prototype_select")


def index(h: Handle, geom, lat: Lattice, obs: ObsSpots, omega, startR, startX, eps_final, c_out, n_max,
          n_em=20, n_sinkhorn=100, k_single=20, f_out=0.1, unmatched_frac=0.4, dust_mode=0, n_newton=4, n_mm=4,
          tol_x=1e-6, tol_R=1e-9, hreg=1e-3, anneal_single=100.0, recut_single=False, grid=None, mstep="plain",
          stream=None):
    """laue_index: (R (k*, 9), x (k*, 3), assign (n_obs,) grain per observed spot).

    Starts: startR (S, 9) / startX (S, 3), or startR = startX = None and
    grid = dict(n_full, sym, k, cube_mm) for the library's start grid.
    mstep: "plain" (Newton + MM) or "adjoint" (damped Gauss-Newton on the
    OT-weighted cost; n_newton steps, hreg the damping)."""
    g_n, g_sym, g_k, g_cube = 0, 24, 1, 5.0
    if startR is None:
        g = {"sym": 24, "k": 1, "cube_mm": 5.0}
        g.update(grid or {})
        g_n, g_sym, g_k, g_cube = int(g["n_full"]), int(g["sym"]), int(g["k"]), float(g["cube_mm"])
        h.reserve(obs.T, extra=4 * (g_n // 1024 + 1) + 1024, stream=stream)
        Sg = ctypes.c_longlong(0)
        h.check(h.L.laue_start_grid(h.h, g_n, g_sym, g_k, g_cube, 0, None, None, ctypes.byref(Sg), _stream(stream)),
                "laue_start_grid")
        S = int(Sg.value)
        dev = obs.p.device
    else:
        startR = startR.reshape(-1, 9).contiguous().float()
        startX = startX.reshape(-1, 3).contiguous().float()
        S = int(startR.shape[0])
        dev = startR.device
    nI = int(obs.p.shape[0])
    b = ctypes.c_size_t()
    h.check(h.L.laue_index_workspace_size(h.h, obs.T, nI, S, int(n_max), int(lat.w_d0.shape[0]), ctypes.byref(b)),
            "laue_index_workspace_size")
    need = b.value + 256
    R = torch.empty(int(n_max), 9, device=dev)
    x = torch.empty(int(n_max), 3, device=dev)
    assign = torch.empty(max(nI, 1), dtype=torch.int32, device=dev)
    prm = N.LaueIndexParams(float(unmatched_frac), float(eps_final), float(c_out), float(f_out), int(n_em),
                            int(n_sinkhorn), int(k_single), int(dust_mode),
                            mparams(eps_final, n_newton, n_mm, tol_x, tol_R, hreg), float(anneal_single),
                            1 if recut_single else 0, g_n, g_sym, g_k, g_cube, 1 if mstep == "adjoint" else 0)
    ng = ctypes.c_int(0)
    g_s, o_s, l_s = geometry_struct(geom), obs.struct(), lat.struct()
    # The SPOT matrix's size is known only after the fits (its nonzeros per kept
    # candidate grow with the spot density); when it does not fit, the library
    # reports the missing bytes, and the call is repeated once with them added.
    for attempt in range(3):
        if h.ws is None or h.ws.numel() < need:
            h.ws = None
            h.ws = torch.empty(need, dtype=torch.uint8, device=dev)
            h.check(h.L.laue_set_workspace(h.h, _ptr(h.ws), h.ws.numel(), _stream(stream)), "set_workspace")
        rc = h.L.laue_index(h.h, ctypes.byref(g_s), ctypes.byref(l_s), ctypes.byref(o_s), _ptr(omega), _ptr(startR),
                            _ptr(startX), S, ctypes.byref(prm), _ptr(R), _ptr(x), int(n_max), ctypes.byref(ng),
                            _ptr(assign), _stream(stream))
        if rc == N.LAUE_ERR_CAPACITY and attempt < 2:
            msg = h.L.laue_last_error(h.h)
            m = re.search(r"need (\d+) more workspace bytes", msg.decode() if msg else "")
            if m:
                need = h.ws.numel() + int(m.group(1)) + (1 << 20)
                continue
        h.check(rc, "laue_index")
        break
    k = ng.value
    return R[:k], x[:k], assign[:nI]


def cost_sinkhorn_noalloc(geom, obs: ObsSpots, model: ModelSpots, eps, c_out, n_iter, f, g, dust, assign=None,
                          margin=None, marg_err=None, q=None, status=None, dust_mode=0, unmatched_frac=0.4,
                          stream=None):
    """laue_cost_sinkhorn_noalloc: the E-step into caller-allocated outputs,
    with the library's fixed device scratch (no allocation by the library).
    Returns the status code of the call."""
    L = N.lib()
    prm = ot_params(eps, c_out, n_iter, dust_mode, unmatched_frac, False)
    g_s, o_s, m_s = geometry_struct(geom), obs.struct(), model.struct()
    return L.laue_cost_sinkhorn_noalloc(ctypes.byref(g_s), ctypes.byref(o_s), ctypes.byref(m_s), ctypes.byref(prm),
                                        _ptr(f), _ptr(g), _ptr(dust), _ptr(assign), _ptr(margin), _ptr(marg_err),
                                        _ptr(q), _ptr(status), _stream(stream))


def autotune(h: Handle, geom, obs: ObsSpots, model: ModelSpots, eps, c_out, n_iter=3, dust_mode=0,
             unmatched_frac=0.4, stream=None):
    """laue_autotune: picks the fastest launch shapes of the Sinkhorn passes
    for this problem; returns (row shape, column shape, per-shape ms)."""
    T = obs.T
    nI, nJ = int(obs.p.shape[0]), model.n
    base = h.workspace_size(T, n_obs=nI, n_model=nJ)
    h.reserve(T, n_obs=nI, n_model=nJ, extra=4 * (nI + nJ + 2 * T + 8) + 4096, stream=stream)
    prm = ot_params(eps, c_out, 1, dust_mode, unmatched_frac, False)
    ch = (ctypes.c_int * 2)()
    ms = (ctypes.c_float * 8)()
    g_s, o_s, m_s = geometry_struct(geom), obs.struct(), model.struct()
    h.check(h.L.laue_autotune(h.h, ctypes.byref(g_s), ctypes.byref(o_s), ctypes.byref(m_s), ctypes.byref(prm),
                              int(n_iter), ch, ms, _stream(stream)), "laue_autotune")
    return ch[0], ch[1], [(ms[2 * v], ms[2 * v + 1]) for v in range(4)]
