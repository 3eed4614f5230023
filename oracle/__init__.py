"""FP64 CPU oracle for the LaueOT Sinkhorn-EM hot path (arXiv 2404.06478).

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the tests, the smoke check and the
benchmark's CPU-baseline leg import this package.  The arithmetic lives in
plain C (``laue_oracle.c``, FP64 loops over the paper's definitions); this
module compiles it with gcc and marshals numpy arrays through ctypes.  It shares
no code with the CUDA path.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "laue_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liblaue_oracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)
_B = ctypes.POINTER(ctypes.c_byte)


def build(force: bool = False) -> str:
    """Compile the oracle into a shared library next to its source."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp.%d" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
        # OpenMP (threads over angle blocks in the Sinkhorn updates) where gcc has it
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            L.orc_forward.restype = ctypes.c_long
            L.orc_pair_cost.restype = ctypes.c_double
            L.orc_eps_schedule.restype = ctypes.c_double
            L.orc_eps_schedule_f.restype = ctypes.c_double
            L.orc_start_grid.restype = ctypes.c_long
            _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _i(a):
    return a.ctypes.data_as(_I) if a is not None else None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a.reshape(shape) if shape is not None else a


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def pack_geom(geom) -> np.ndarray:
    g = [*geom.beam, geom.lam_min, geom.lam_max, geom.D, len(geom.detectors)]
    for det in geom.detectors:
        g += [*det.centre, *det.normal, det.half, float(getattr(det, "D", 0.0))]
    return np.asarray(g, dtype=np.float64)


def cost_lengths(geom, det):
    """Cost length D_j of each model spot: the distance of the detector it
    hits (det[j]), the geometry's D where that detector sets none."""
    det = _i32(det)
    out = np.zeros(max(len(det), 1))
    lib().orc_cost_lengths(_d(pack_geom(geom)), len(det), _i(det), _d(out))
    return out[:len(det)]


def _Dj(D, nJ):
    """Per-model-spot cost lengths from a scalar or an array."""
    if np.ndim(D) == 0:
        return np.full(max(nJ, 1), float(D))
    D = _f64(D)
    assert len(D) == nJ, (len(D), nJ)
    return D if nJ else np.zeros(1)


def _det(det):
    return None if det is None else _i(_i32(det))


def c_out_for(sigma_mm: float, D: float) -> float:
    """Outlier cost: the pair cost of a ray 3 sigma away (sigma_ang = sigma_mm / D)."""
    half = 1.5 * sigma_mm / D
    return 4.0 * D * D * math.sin(half) ** 2


@dataclasses.dataclass
class Planes:
    w: np.ndarray      # (M, 3) unit crystal directions
    d0: np.ndarray     # (M,) spacing of the base reflection (Angstrom)
    nharm: np.ndarray  # (M,) number of allowed harmonics
    hkl0: np.ndarray   # (M, 3) base reflection


def reflections(a: float, hmax: int, centering: int = 1) -> Planes:
    L = lib()
    cap = (2 * hmax + 1) ** 3
    w = np.zeros((cap, 3)); d0 = np.zeros(cap)
    nh = np.zeros(cap, np.int32); hkl = np.zeros((cap, 3), np.int32)
    M = L.orc_reflections(ctypes.c_double(a), hmax, centering, cap, _d(w), _d(d0), _i(nh), _i(hkl))
    if M < 0:
        raise ValueError("reflection multipliers are not an arithmetic progression")
    return Planes(w[:M].copy(), d0[:M].copy(), nh[:M].copy(), hkl[:M].copy())


def forward(geom, planes: Planes, R, x, omega, with_all: bool = False):
    """Forward model + cut; returns dict of the visible spot list sorted by
    (t, grain, plane)."""
    L = lib()
    g = pack_geom(geom)
    R = _f64(R, (-1, 9)); x = _f64(x, (-1, 3)); omega = _f64(omega)
    N, M, T = len(R), len(planes.w), len(omega)
    w = _f64(planes.w); d0 = _f64(planes.d0); nh = _i32(planes.nharm)
    vis = np.zeros(T * N * M, np.int8) if with_all else None
    mrg = np.zeros(T * N * M) if with_all else None
    J_off = np.zeros(T + 1, np.int32)
    args = lambda cap, gr, pl, ray, sp, dt, ce: (
        _d(g), _d(w), _d(d0), _i(nh), M, _d(R), _d(x), N, _d(omega), T, ctypes.c_long(cap),
        _i(J_off), _i(gr), _i(pl), _d(ray), _d(sp), _i(dt), _d(ce),
        vis.ctypes.data_as(_B) if vis is not None else None, _d(mrg))
    z = np.zeros(1, np.int32); zd = np.zeros(4)
    J = L.orc_forward(*args(0, z, z, zd, zd, z, zd))
    gr = np.zeros(J, np.int32); pl = np.zeros(J, np.int32); dt = np.zeros(J, np.int32)
    ray = np.zeros((J, 4)); sp = np.zeros((J, 3)); ce = np.zeros((J, 3))
    L.orc_forward(*args(J, gr, pl, ray, sp, dt, ce))
    out = dict(J_off=J_off.astype(np.int64), grain=gr, plane=pl, ray=ray, spot=sp, det=dt, center=ce,
               t=np.repeat(np.arange(T), np.diff(J_off)))
    if with_all:
        out["vis_all"] = vis.reshape(T, N, M)
        out["margin_all"] = mrg.reshape(T, N, M)
    return out


def refresh(geom, planes: Planes, R, x, omega, J_off, grain, plane):
    L = lib()
    g = pack_geom(geom)
    R = _f64(R, (-1, 9)); x = _f64(x, (-1, 3)); omega = _f64(omega)
    J_off = _i32(J_off); grain = _i32(grain); plane = _i32(plane)
    J = int(J_off[-1])
    ray = np.zeros((J, 4)); ce = np.zeros((J, 3))
    L.orc_refresh(_d(g), _d(_f64(planes.w)), _d(_f64(planes.d0)), _i(_i32(planes.nharm)), _d(R), _d(x),
                  _d(omega), len(omega), _i(J_off), _i(grain), _i(plane), _d(ray), _d(ce))
    return ray, ce


def pair_cost(p, c, r, D):
    return lib().orc_pair_cost(_d(_f64(p)), _d(_f64(c)), _d(_f64(r)), ctypes.c_double(D))


def pair_costs(p, c, r, D):
    """orc_pair_cost of the rows of (n, 3) arrays p, c, r (broadcast to n)."""
    p, c, r = np.broadcast_arrays(np.asarray(p, np.float64).reshape(-1, 3), np.asarray(c, np.float64).reshape(-1, 3),
                                  np.asarray(r, np.float64).reshape(-1, 3))
    p, c, r = (np.ascontiguousarray(a) for a in (p, c, r))
    out = np.zeros(len(p))
    lib().orc_pair_costs(len(p), _d(p), _d(c), _d(r), ctypes.c_double(D), _d(out))
    return out


def masses(mode, frac, I_off, J_off):
    T = len(I_off) - 1
    nd = T if mode else 1
    U = np.zeros(nd); O = np.zeros(nd)
    lib().orc_masses(mode, ctypes.c_double(frac), T, _i(_i32(I_off)), _i(_i32(J_off)), _d(U), _d(O))
    return U, O


def sinkhorn(D, p, I_off, J_off, c, r, eps, c_out, mode=0, frac=0.4, n_iter=100, tol=0.0, init=None):
    """Log-domain BalancedOT; returns (f, g, fd, gd, iterations)."""
    L = lib()
    p = _f64(p, (-1, 3)); c = _f64(c, (-1, 3)); r = _f64(r, (-1, 3))
    I_off = _i32(I_off); J_off = _i32(J_off)
    T = len(I_off) - 1
    nd = T if mode else 1
    if init is None:
        f = np.zeros(len(p)); g = np.zeros(len(c)); fd = np.zeros(nd); gd = np.zeros(nd); warm = 0
    else:
        f, g, fd, gd = [np.array(a, dtype=np.float64) for a in init]; warm = 1
    it = L.orc_sinkhorn(_d(_Dj(D, len(c))), T, _i(I_off), _d(p), _i(J_off), _d(c), _d(r),
                        ctypes.c_double(eps), ctypes.c_double(c_out), mode, ctypes.c_double(frac),
                        n_iter, ctypes.c_double(tol), warm, _d(f), _d(g), _d(fd), _d(gd))
    return f, g, fd, gd, it


def harvest(D, p, I_off, J_off, c, r, eps, c_out, mode, frac, f, g, fd, gd):
    """Returns dict(assign, margin, row_err, col_err, q, v)."""
    L = lib()
    p = _f64(p, (-1, 3)); c = _f64(c, (-1, 3)); r = _f64(r, (-1, 3))
    I_off = _i32(I_off); J_off = _i32(J_off)
    T = len(I_off) - 1
    nI, nJ = len(p), len(c)
    assign = np.zeros(nI, np.int32); margin = np.zeros(nI); err = np.zeros(2)
    q = np.zeros(nJ); v = np.zeros((nJ, 3))
    L.orc_harvest(_d(_Dj(D, nJ)), T, _i(I_off), _d(p), _i(J_off), _d(c), _d(r),
                  ctypes.c_double(eps), ctypes.c_double(c_out), mode, ctypes.c_double(frac),
                  _d(_f64(f)), _d(_f64(g)), _d(_f64(fd)), _d(_f64(gd)),
                  _i(assign), _d(margin), _d(err), _d(q), _d(v))
    return dict(assign=assign, margin=margin, row_err=err[0], col_err=err[1], q=q, v=v)


def mstep(geom, planes, omega, p, I_off, J_off, grain, plane, cE, rE, f, g, eps, R, x,
          n_newton=4, n_mm=4, tol_x=1e-6, tol_R=1e-9, hreg=1e-3, det=None):
    """One M-step (Newton on x, then MM on R); returns (R, x, stats (N, 8))."""
    L = lib()
    R = _f64(R, (-1, 9)).copy(); x = _f64(x, (-1, 3)).copy()
    N = len(R)
    stats = np.zeros((N, 8))
    omega = _f64(omega)
    L.orc_mstep(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(omega), len(omega), _i(_i32(I_off)),
                _d(_f64(p, (-1, 3))), _i(_i32(J_off)), _i(_i32(grain)), _i(_i32(plane)), _det(det), N,
                _d(_f64(cE, (-1, 3))), _d(_f64(rE, (-1, 3))), _d(_f64(f)), _d(_f64(g)),
                ctypes.c_double(eps), n_newton, n_mm, ctypes.c_double(tol_x), ctypes.c_double(tol_R),
                ctypes.c_double(hreg), _d(R), _d(x), _d(stats))
    return R.reshape(-1, 3, 3), x, stats


def eps_schedule(eps_final, n_em, k, factor=100.0):
    return lib().orc_eps_schedule_f(ctypes.c_double(eps_final), n_em, k, ctypes.c_double(factor))


def em(geom, planes, omega, p, I_off, J_off, grain, plane, R, x, eps_final, n_em, n_sinkhorn,
       c_out, mode=0, frac=0.4, n_newton=4, n_mm=4, tol_x=1e-6, tol_R=1e-9, hreg=1e-3, mstep="plain",
       det=None):
    """Algorithm LaueOT with a fixed number of EM steps; returns dict.  mstep
    "adjoint" takes the damped Gauss-Newton M-step (hreg its damping)."""
    L = lib()
    R = _f64(R, (-1, 9)).copy(); x = _f64(x, (-1, 3)).copy()
    N = len(R); omega = _f64(omega); T = len(omega)
    nI = int(I_off[-1]); nJ = int(J_off[-1]); nd = T if mode else 1
    f = np.zeros(nI); g = np.zeros(nJ); fd = np.zeros(nd); gd = np.zeros(nd)
    assign = np.zeros(nI, np.int32); margin = np.zeros(nI)
    L.orc_em(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(_f64(planes.d0)), _i(_i32(planes.nharm)),
             _d(omega), T, _i(_i32(I_off)), _d(_f64(p, (-1, 3))), _i(_i32(J_off)), _i(_i32(grain)),
             _i(_i32(plane)), _det(det), N, _d(R), _d(x), ctypes.c_double(eps_final), n_em, n_sinkhorn,
             ctypes.c_double(c_out), mode, ctypes.c_double(frac), n_newton, n_mm,
             ctypes.c_double(tol_x), ctypes.c_double(tol_R), ctypes.c_double(hreg), 1 if mstep == "adjoint" else 0,
             _d(f), _d(g), _d(fd), _d(gd), _i(assign), _d(margin))
    return dict(R=R.reshape(-1, 3, 3), x=x, f=f, g=g, fd=fd, gd=gd, assign=assign, margin=margin)


def single_fit(geom, planes, omega, p, I_off, R0, x0, eps_final, k_max, c_out,
               n_newton=4, n_mm=4, tol_x=1e-6, tol_R=1e-9, hreg=1e-3, f_out=0.1, anneal=100.0, recut=False):
    L = lib()
    R0 = _f64(R0, (-1, 9)); x0 = _f64(x0, (-1, 3))
    S = len(R0); omega = _f64(omega)
    Ro = np.zeros_like(R0); xo = np.zeros_like(x0)
    keep = np.zeros(S, np.int32); unm = np.zeros(S)
    L.orc_single_fit(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(_f64(planes.d0)),
                     _i(_i32(planes.nharm)), len(planes.w), _d(omega), len(omega), _i(_i32(I_off)),
                     _d(_f64(p, (-1, 3))), S, _d(R0), _d(x0), ctypes.c_double(eps_final), k_max,
                     ctypes.c_double(c_out), n_newton, n_mm, ctypes.c_double(tol_x),
                     ctypes.c_double(tol_R), ctypes.c_double(hreg), ctypes.c_double(f_out),
                     ctypes.c_double(anneal), 1 if recut else 0, _d(Ro), _d(xo), _i(keep), _d(unm))
    return Ro.reshape(-1, 3, 3), xo, keep.astype(bool), unm


def spot_matrix(geom, planes, omega, p, I_off, R, x, eps_s, c_out):
    L = lib()
    R = _f64(R, (-1, 9)); x = _f64(x, (-1, 3)); omega = _f64(omega)
    Nc = len(R); nI = int(I_off[-1])
    Lbar = np.zeros((nI, Nc))
    L.orc_spot_matrix(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(_f64(planes.d0)),
                      _i(_i32(planes.nharm)), len(planes.w), _d(omega), len(omega), _i(_i32(I_off)),
                      _d(_f64(p, (-1, 3))), Nc, _d(R), _d(x), ctypes.c_double(eps_s),
                      ctypes.c_double(c_out), _d(Lbar))
    return Lbar


def spot_greedy(Lbar, kmax):
    Lbar = _f64(Lbar)
    nI, Nc = Lbar.shape
    order = np.zeros(kmax, np.int32); gain = np.zeros(kmax); F = np.zeros(kmax)
    k = lib().orc_spot_greedy(nI, Nc, _d(Lbar), kmax, _i(order), _d(gain), _d(F))
    return order[:k], gain[:k], F[:k]


def kstar(gain):
    gain = _f64(gain)
    return lib().orc_kstar(len(gain), _d(gain))


def grain_objective(geom, planes, omega, p, I_off, J_off, grain, plane, cE, rE, f, g, eps, R, x, det=None):
    L = lib()
    R = _f64(R, (-1, 9)); x = _f64(x, (-1, 3)); N = len(R); omega = _f64(omega)
    En = np.zeros(N)
    L.orc_grain_objective(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(omega), len(omega),
                          _i(_i32(I_off)), _d(_f64(p, (-1, 3))), _i(_i32(J_off)), _i(_i32(grain)),
                          _i(_i32(plane)), _det(det), N, _d(_f64(cE, (-1, 3))), _d(_f64(rE, (-1, 3))),
                          _d(_f64(f)), _d(_f64(g)), ctypes.c_double(eps), _d(R), _d(x), _d(En))
    return En


def grain_grad(geom, planes, omega, p, I_off, J_off, grain, plane, f, g, eps, R, x, det=None):
    L = lib()
    R = _f64(R, (-1, 9)); x = _f64(x, (-1, 3)); N = len(R); omega = _f64(omega)
    grad = np.zeros((N, 6))
    L.orc_grain_grad(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(omega), len(omega),
                     _i(_i32(I_off)), _d(_f64(p, (-1, 3))), _i(_i32(J_off)), _i(_i32(grain)),
                     _i(_i32(plane)), _det(det), N, _d(_f64(f)), _d(_f64(g)), ctypes.c_double(eps), _d(R),
                     _d(x), _d(grad))
    return grad


def sym3_eig(A):
    A = _f64(A, (9,)); ev = np.zeros(3); V = np.zeros(9)
    lib().orc_sym3_eig(_d(A), _d(ev), _d(V))
    return ev, V.reshape(3, 3)


def svd3(B):
    B = _f64(B, (9,)); U = np.zeros(9); S = np.zeros(3); V = np.zeros(9)
    lib().orc_svd3(_d(B), _d(U), _d(S), _d(V))
    return U.reshape(3, 3), S, V.reshape(3, 3)


def wahba(B):
    B = _f64(B, (9,)); R = np.zeros(9)
    ok = lib().orc_wahba(_d(B), _d(R))
    return (R.reshape(3, 3) if ok else None)


def gamma(omega):
    G = np.zeros(9)
    lib().orc_gamma(ctypes.c_double(omega), _d(G))
    return G.reshape(3, 3)


def start_grid(n_full, sym=24, k=1, cube=5.0):
    """Start grid of the single-grain fits: super-Fibonacci orientations
    (restricted to the cubic fundamental zone when sym = 24) x k^3 cell
    centres of the sample cube.  Returns (R (S, 3, 3), x (S, 3))."""
    L = lib()
    n = L.orc_start_grid(ctypes.c_long(n_full), sym, k, ctypes.c_double(cube), ctypes.c_long(0), None, None)
    R = np.zeros((max(n, 1), 9)); x = np.zeros((max(n, 1), 3))
    L.orc_start_grid(ctypes.c_long(n_full), sym, k, ctypes.c_double(cube), ctypes.c_long(n), _d(R), _d(x))
    return R[:n].reshape(-1, 3, 3), x[:n]


def grain_gn(geom, planes, omega, p, I_off, J_off, grain, plane, cE, rE, f, g, eps, R, x, det=None):
    """Gradient (N, 6), Gauss-Newton matrix (N, 6, 6) and value (N,) of the
    OT-weighted cost at the pose (R, x), Q held at the E-step plan."""
    L = lib()
    R = _f64(R, (-1, 9)); x = _f64(x, (-1, 3))
    N = len(R)
    grad = np.zeros((N, 6)); H = np.zeros((N, 36)); val = np.zeros(N)
    L.orc_grain_gn(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(_f64(omega)), len(omega), _i(_i32(I_off)),
                   _d(_f64(p, (-1, 3))), _i(_i32(J_off)), _i(_i32(grain)), _i(_i32(plane)), _det(det), N,
                   _d(_f64(cE, (-1, 3))), _d(_f64(rE, (-1, 3))), _d(_f64(f)), _d(_f64(g)), ctypes.c_double(eps),
                   _d(R), _d(x), _d(grad), _d(H), _d(val))
    return grad, H.reshape(-1, 6, 6), val


def mstep_adjoint(geom, planes, omega, p, I_off, J_off, grain, plane, cE, rE, f, g, eps, R, x, n_steps=4,
                  lam=1e-3, det=None):
    """Adjoint M-step (damped Gauss-Newton with Q held); returns (R, x, step_norms)."""
    L = lib()
    R = _f64(R, (-1, 9)).copy(); x = _f64(x, (-1, 3)).copy()
    N = len(R)
    norms = np.zeros((N, 2))
    L.orc_mstep_adjoint(_d(pack_geom(geom)), _d(_f64(planes.w)), _d(_f64(omega)), len(omega), _i(_i32(I_off)),
                        _d(_f64(p, (-1, 3))), _i(_i32(J_off)), _i(_i32(grain)), _i(_i32(plane)), _det(det), N,
                        _d(_f64(cE, (-1, 3))), _d(_f64(rE, (-1, 3))), _d(_f64(f)), _d(_f64(g)), ctypes.c_double(eps),
                        n_steps, ctypes.c_double(lam), _d(R), _d(x), _d(norms))
    return R.reshape(-1, 3, 3), x, norms


def sinkhorn_unbalanced(D, p, I_off, J_off, c, r, eps, kappa, lam, n_iter=100):
    """Algorithm UnbalancedOT (log domain, no dustbins); returns (f, g)."""
    p = _f64(p, (-1, 3)); c = _f64(c, (-1, 3)); r = _f64(r, (-1, 3))
    I_off = _i32(I_off); J_off = _i32(J_off)
    T = len(I_off) - 1
    f = np.zeros(int(I_off[-1])); g = np.zeros(int(J_off[-1]))
    lib().orc_sinkhorn_unbalanced(_d(_Dj(D, len(c))), T, _i(I_off), _d(p), _i(J_off), _d(c), _d(r),
                                  ctypes.c_double(eps), ctypes.c_double(kappa), ctypes.c_double(lam), n_iter,
                                  _d(f), _d(g))
    return f, g


def harvest_unbalanced(D, p, I_off, J_off, c, r, eps, f, g):
    """(assign, margin, row mass, column mass q) of the unbalanced plan."""
    p = _f64(p, (-1, 3)); c = _f64(c, (-1, 3)); r = _f64(r, (-1, 3))
    I_off = _i32(I_off); J_off = _i32(J_off)
    T = len(I_off) - 1
    nI, nJ = int(I_off[-1]), int(J_off[-1])
    assign = np.zeros(nI, np.int32); margin = np.zeros(nI); rows = np.zeros(nI); q = np.zeros(nJ)
    lib().orc_harvest_unbalanced(_d(_Dj(D, nJ)), T, _i(I_off), _d(p), _i(J_off), _d(c), _d(r),
                                 ctypes.c_double(eps), _d(_f64(f)), _d(_f64(g)), _i(assign), _d(margin), _d(rows),
                                 _d(q))
    return dict(assign=assign, margin=margin, rowmass=rows, q=q)


def set_threads(n):
    """Threads of the oracle's Sinkhorn updates; returns the number in effect
    (1 without OpenMP)."""
    return int(lib().orc_set_threads(int(n)))


def reciprocal_basis(a, b, c, alpha, beta, gamma):
    """Reciprocal basis B (3, 3), columns b1 b2 b3 (Angstrom^-1, no 2 pi)."""
    B = np.zeros(9)
    lib().orc_reciprocal_basis(*(ctypes.c_double(v) for v in (a, b, c, alpha, beta, gamma)), _d(B))
    return B.reshape(3, 3)


def reflections_hkl(B, hkl):
    """Plane table from a reciprocal basis and a list of allowed reflections
    (n, 3); raises ValueError when a line's multiples are not 1..n of a base."""
    L = lib()
    B = _f64(B, (9,))
    hkl = np.ascontiguousarray(np.asarray(hkl, np.int32).reshape(-1, 3))
    n = L.orc_reflections_hkl(_d(B), _i(hkl), len(hkl), 0, None, None, None, None)
    if n < 0:
        raise ValueError("harmonics of some line are not the multiples 1..n of its base reflection")
    w = np.zeros((max(n, 1), 3)); d0 = np.zeros(max(n, 1)); nh = np.zeros(max(n, 1), np.int32)
    h0 = np.zeros((max(n, 1), 3), np.int32)
    L.orc_reflections_hkl(_d(B), _i(hkl), len(hkl), n, _d(w), _d(d0), _i(nh), _i(h0))
    return Planes(w[:n], d0[:n], nh[:n], h0[:n])


def knn(D, p, I_off, J_off, c, r, rho):
    """Neighbour sets of the sparse plan: (|J|, rho) observed indices, -1 padded."""
    p = _f64(p, (-1, 3)); c = _f64(c, (-1, 3)); r = _f64(r, (-1, 3))
    I_off = _i32(I_off); J_off = _i32(J_off)
    nbr = np.zeros((max(int(J_off[-1]), 1), rho), np.int32)
    lib().orc_knn(_d(_Dj(D, int(J_off[-1]))), len(I_off) - 1, _i(I_off), _d(p), _i(J_off), _d(c), _d(r), rho, _i(nbr))
    return nbr[:int(J_off[-1])]


def sinkhorn_sparse(D, p, I_off, J_off, c, r, eps, c_out, mode=0, frac=0.4, n_iter=100, rho=32):
    """BalancedOT restricted to the rho-nearest-neighbour support; (f, g, fd, gd)."""
    p = _f64(p, (-1, 3)); c = _f64(c, (-1, 3)); r = _f64(r, (-1, 3))
    I_off = _i32(I_off); J_off = _i32(J_off)
    T = len(I_off) - 1
    nd = T if mode else 1
    f = np.zeros(int(I_off[-1])); g = np.zeros(int(J_off[-1])); fd = np.zeros(nd); gd = np.zeros(nd)
    lib().orc_sinkhorn_sparse(_d(_Dj(D, int(J_off[-1]))), T, _i(I_off), _d(p), _i(J_off), _d(c), _d(r), ctypes.c_double(eps),
                              ctypes.c_double(c_out), mode, ctypes.c_double(frac), n_iter, rho, _d(f), _d(g), _d(fd),
                              _d(gd))
    return f, g, fd, gd
