"""Seeded parity cases shared by the GPU tests.

Inputs are produced by the oracle's forward model and synthgen's noise and
outliers, rounded once to float32; both the CUDA path and the oracle then see
exactly the same numbers (the oracle reads them back as float64)."""
import dataclasses

import numpy as np

import oracle
import synthgen as sg

GEOM = sg.Geometry()


def f32(a):
    return np.asarray(a, np.float64).astype(np.float32).astype(np.float64)


@dataclasses.dataclass
class Case:
    cfg: sg.Config
    planes: oracle.Planes      # float32-rounded
    R: np.ndarray
    x: np.ndarray
    om: np.ndarray
    fw: dict                   # model list (float32-rounded vectors)
    obs: sg.Observed           # float32-rounded positions
    c_out: float
    geom: sg.Geometry = GEOM


def geom32(geom):
    """The geometry with every number rounded to float32 (what the CUDA path
    receives), so that both sides see the same detectors."""
    r = lambda v: float(np.float32(v))
    dets = tuple(sg.Detector(tuple(r(v) for v in d.centre), tuple(r(v) for v in d.normal), r(d.half), r(d.D))
                 for d in geom.detectors)
    return sg.Geometry(tuple(r(v) for v in geom.beam), r(geom.lam_min), r(geom.lam_max), r(geom.D), dets)


def planes32(cfg):
    P = oracle.reflections(cfg.a, cfg.hmax, cfg.centering)
    return oracle.Planes(f32(P.w), f32(P.d0), P.nharm, P.hkl0)


def make_case(cfg, seed=None, n_grains=None, T=None, outlier_frac=None, sigma=None, geom=GEOM):
    if n_grains is not None or T is not None:
        cfg = dataclasses.replace(cfg, n_grains=n_grains or cfg.n_grains, T=T or cfg.T)
    rng = np.random.default_rng(cfg.seed if seed is None else seed)
    R, x = sg.random_grains(cfg, rng)
    R, x = f32(R), f32(x)
    om = f32(sg.omegas(cfg))
    P = planes32(cfg)
    fw = oracle.forward(geom, P, R, x, om)
    for k in ("ray", "spot", "center"):
        fw[k] = f32(fw[k])
    obs = sg.observe(geom, cfg, fw["t"], fw["det"], fw["spot"], rng, sigma_mm=sigma,
                     outlier_frac=outlier_frac)
    obs.p = f32(obs.p)
    return Case(cfg, P, R, x, om, fw, obs, float(np.float32(oracle.c_out_for(cfg.sigma_mm, geom.D))), geom)


def to_device(case, dev):
    import torch
    from paper_2404_06478_gb300 import api
    ob = api.ObsSpots.from_numpy(case.obs.p, case.obs.I_off, device=dev)
    fw = case.fw
    ms = api.ModelSpots.from_numpy(fw["J_off"], fw["grain"], fw["plane"], fw["ray"], fw["center"],
                                   fw["spot"], fw["det"], device=dev)
    return ob, ms


def _oracle_call(args):
    name, a, kw = args
    return getattr(oracle, name)(*a, **kw)


def oracle_parallel(calls, workers=None):
    """Runs oracle functions [(name, args, kwargs), ...] in a pool of spawned
    processes (spawned, not forked: the parent may hold a CUDA context)."""
    import concurrent.futures
    import multiprocessing
    import os
    workers = workers or min(len(calls), os.cpu_count() or 1)
    if workers <= 1:
        return [_oracle_call(c) for c in calls]
    with concurrent.futures.ProcessPoolExecutor(workers, mp_context=multiprocessing.get_context("spawn")) as ex:
        return list(ex.map(_oracle_call, calls))


def block_slices(case, t):
    """Observed and model index ranges of angle block t."""
    return (slice(int(case.obs.I_off[t]), int(case.obs.I_off[t + 1])),
            slice(int(case.fw["J_off"][t]), int(case.fw["J_off"][t + 1])))
