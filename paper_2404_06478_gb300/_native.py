"""ctypes declarations of the C ABI in include/laueot.h.

Argument marshalling only: every step of the hot path runs in liblaueot.so.
Importing this module fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblaueot.so")

LAUE_OK = 0
LAUE_WARN_NOT_CONVERGED = 1
LAUE_ERR_INVALID_ARG = -1
LAUE_ERR_CAPACITY = -2
LAUE_ERR_CUDA = -3
LAUE_ERR_NUMERIC = -4
LAUE_ERR_TIMEOUT = -5
LAUE_ERR_UNIMPLEMENTED = -6
LAUE_ERR_WORKSPACE = -7

_vp = ctypes.c_void_p
_i = ctypes.c_int
_f = ctypes.c_float
_d = ctypes.c_double
_pi = ctypes.POINTER(ctypes.c_int)


class LaueGeometry(ctypes.Structure):
    _fields_ = [("beam", _f * 3), ("lam_min", _f), ("lam_max", _f), ("D", _f), ("n_det", _i),
                ("det_centre", (_f * 3) * 4), ("det_normal", (_f * 3) * 4), ("det_half", _f * 4),
                ("det_D", _f * 4)]


class LaueLattice(ctypes.Structure):
    _fields_ = [("w_d0", _vp), ("nharm", _vp), ("M", _i)]


class LaueObsSpots(ctypes.Structure):
    _fields_ = [("T", _i), ("n", _i), ("I_off", _vp), ("p", _vp)]


class LaueModelSpots(ctypes.Structure):
    _fields_ = [("T", _i), ("n", _i), ("capacity", _i), ("J_off", _vp), ("grain", _vp), ("plane", _vp),
                ("angle", _vp), ("ray", _vp), ("center", _vp), ("spot", _vp)]


class LaueOTParams(ctypes.Structure):
    _fields_ = [("unmatched_frac", _d), ("eps", _f), ("c_out", _f), ("n_iter", _i), ("dust_mode", _i),
                ("warm_start", _i), ("kappa", _f), ("lambda_", _f), ("pad_", _i)]


class LaueMParams(ctypes.Structure):
    _fields_ = [("eps", _f), ("n_newton", _i), ("n_mm", _i), ("tol_x", _f), ("tol_R", _f), ("hreg", _f)]


class LaueProblemDims(ctypes.Structure):
    _fields_ = [("T", _i), ("n_obs", _i), ("n_model", _i), ("n_grains", _i), ("n_planes", _i), ("n_starts", _i),
                ("n_candidates", _i)]


class LaueSingleParams(ctypes.Structure):
    _fields_ = [("eps_final", _f), ("c_out", _f), ("f_out", _f), ("k_max", _i), ("mstep", LaueMParams),
                ("anneal", _f), ("recut", _i)]


class LaueEMParams(ctypes.Structure):
    _fields_ = [("unmatched_frac", ctypes.c_double), ("eps_final", _f), ("c_out", _f), ("anneal", _f),
                ("n_em", _i), ("n_sinkhorn", _i), ("dust_mode", _i), ("mstep_kind", _i), ("k_first", _i),
                ("k_last", _i), ("mstep", LaueMParams)]


class LaueIndexParams(ctypes.Structure):
    _fields_ = [("unmatched_frac", _d), ("eps_final", _f), ("c_out", _f), ("f_out", _f), ("n_em", _i),
                ("n_sinkhorn", _i), ("k_single", _i), ("dust_mode", _i), ("mstep", LaueMParams),
                ("anneal_single", _f), ("recut_single", _i), ("grid_n", ctypes.c_longlong), ("grid_sym", _i),
                ("grid_k", _i), ("grid_cube", _f), ("mstep_kind", _i)]


_P = ctypes.POINTER
_lib = None

# name -> argtypes (all return int unless noted)
SIGNATURES = {
    "laue_create": [_P(_vp), _i],
    "laue_destroy": [_vp],
    "laue_last_error": [_vp],
    "laue_workspace_size": [_vp, _P(LaueProblemDims), _P(ctypes.c_size_t)],
    "laue_set_workspace": [_vp, _vp, ctypes.c_size_t, _vp],
    "laue_device_status": [_vp, _vp, _pi],
    "laue_reflections": [_d, _i, _i, _i, _vp, _vp, _vp, _pi],
    "laue_reciprocal_basis": [_d, _d, _d, _d, _d, _d, _vp],
    "laue_reflections_hkl": [_vp, _vp, _i, _i, _vp, _vp, _vp, _pi],
    "laue_alu_peaks": [_vp, _vp, _vp],
    "laue_forward": [_vp, _P(LaueGeometry), _P(LaueLattice), _vp, _vp, _i, _vp, _i, _P(LaueModelSpots), _pi, _vp],
    "laue_refresh": [_vp, _P(LaueGeometry), _P(LaueLattice), _vp, _vp, _vp, _P(LaueModelSpots), _vp],
    "laue_cost_sinkhorn": [_vp, _P(LaueGeometry), _P(LaueObsSpots), _P(LaueModelSpots), _P(LaueOTParams),
                           _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "laue_cost_sinkhorn_noalloc": [_P(LaueGeometry), _P(LaueObsSpots), _P(LaueModelSpots), _P(LaueOTParams),
                                   _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "laue_autotune": [_vp, _P(LaueGeometry), _P(LaueObsSpots), _P(LaueModelSpots), _P(LaueOTParams), _i, _vp,
                      _vp, _vp],
    "laue_set_launch_shape": [_vp, _i, _i],
    "laue_set_pair_skipping": [_vp, _i],
    "laue_em": [_vp, _P(LaueGeometry), _P(LaueLattice), _P(LaueObsSpots), _vp, _P(LaueModelSpots), _vp, _vp, _i,
                _P(LaueEMParams), _vp, _vp, _vp, _vp, _vp, _vp],
    "laue_sparse_workspace_size": [_i, _i, _i, _i, _P(ctypes.c_size_t)],
    "laue_cost_sinkhorn_sparse": [_vp, _P(LaueGeometry), _P(LaueObsSpots), _P(LaueModelSpots), _P(LaueOTParams),
                                  _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp],
    "laue_read_counters": [_vp, _vp, _P(ctypes.c_longlong), _i],
    "laue_mstep": [_vp, _P(LaueGeometry), _P(LaueLattice), _P(LaueObsSpots), _P(LaueModelSpots), _vp, _vp,
                   _P(LaueMParams), _vp, _vp, _vp, _i, _vp, _vp],
    "laue_mstep_adjoint": [_vp, _P(LaueGeometry), _P(LaueLattice), _P(LaueObsSpots), _P(LaueModelSpots), _vp,
                           _vp, _P(LaueMParams), _vp, _vp, _vp, _i, _vp, _vp],
    "laue_objective_grad": [_vp, _P(LaueGeometry), _P(LaueLattice), _P(LaueObsSpots), _P(LaueModelSpots),
                            _vp, _vp, _f, _vp, _vp, _vp, _i, _vp, _vp, _vp],
    "laue_axis_angle": [_vp, _vp, _vp, _vp, _vp, _i, _vp],
    "laue_axis_angle_vjp": [_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp],
    "laue_start_grid": [_vp, ctypes.c_longlong, _i, _i, _f, ctypes.c_longlong, _vp, _vp, _P(ctypes.c_longlong), _vp],
    "laue_single_fit": [_vp, _P(LaueGeometry), _P(LaueLattice), _P(LaueObsSpots), _vp, _vp, _vp, _i,
                        _P(LaueSingleParams), _vp, _vp, _vp, _vp, _vp],
    "laue_prototype_select": [_vp, _P(LaueGeometry), _P(LaueLattice), _P(LaueObsSpots), _vp, _vp, _vp, _i,
                              _f, _f, _i, _vp, _vp, _pi, _P(ctypes.c_longlong), _vp],
    "laue_index_workspace_size": [_vp, _i, _i, _i, _i, _i, _P(ctypes.c_size_t)],
    "laue_index": [_vp, _P(LaueGeometry), _P(LaueLattice), _P(LaueObsSpots), _vp, _vp, _vp, _i,
                   _P(LaueIndexParams), _vp, _vp, _i, _pi, _vp, _vp],
    "laue_lp_net_init": [_vp, _vp, _vp, _vp],
    "laue_lp_net_params": [_vp, _vp, _vp, _vp, _vp],
    "laue_lp_scene": [_vp, _P(LaueGeometry), _P(LaueLattice), _vp, _i, _i, _i, _i, _i, _i, _f, _f, _d,
                      ctypes.c_ulonglong, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp],
    "laue_lp_scene_seeds": [_vp, _vp, _vp, _i, _i, _i, ctypes.c_ulonglong, _vp, _vp, _vp, _vp],
    "laue_lp_sets": [_vp, _P(LaueGeometry), _vp, _vp, _vp, _i, _i, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp, _vp,
                     _vp],
    "laue_lp_forward": [_vp, _vp, _vp, _i, _vp],
    "laue_lp_train_step": [_vp, _vp, _vp, _i, _f, _vp],
    "laue_lp_decode": [_vp, _vp, _i, _vp, _vp, _vp],
    "laue_gemm_bf16": [_vp, _vp, ctypes.c_longlong, _vp, ctypes.c_longlong, _i, _i, _i, _i, _i, _i, _vp, _vp,
                       _vp, _vp, _vp, ctypes.c_longlong, _i, _vp],
}


# host helpers that return sizes and offsets rather than a status
SIZE_FUNCTIONS = [
    ("laue_lp_param_count", [], ctypes.c_size_t),
    ("laue_lp_set_size", [], ctypes.c_size_t),
    ("laue_lp_net_bytes", [], ctypes.c_size_t),
    ("laue_lp_batch_bytes", [_i], ctypes.c_size_t),
    ("laue_lp_batch_offset", [_i, _i], ctypes.c_longlong),
    ("laue_c_out", [_d, _d], _d),
    ("laue_anneal_eps", [_d, _i, _i, _d], _d),
]


def lib():
    """The loaded library; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(
                "liblaueot.so is missing: build it with paper_2404_06478_gb300.build.build() "
                "(there is no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_char_p if name == "laue_last_error" else ctypes.c_int
        for name, args, res in SIZE_FUNCTIONS:
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def exported_symbols():
    return list(SIGNATURES) + [n for n, _, _ in SIZE_FUNCTIONS]
