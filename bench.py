"""Benchmark of the LaueOT Sinkhorn-EM hot path on GB300.

Workload: 1000 grains, |hkl| <= 6 bcc (a = 2.87 A), 90 rotations over 360 deg,
0.5 mm spot noise, 70% outliers with uneven per-angle Poisson counts, eps =
1 mm^2, 200 Sinkhorn iterations per EM step (synthetic, seeded).  One step =
one EM iteration: refresh of the frozen model list at the current poses, the
fused cost + Sinkhorn E-step (all angle blocks in each persistent launch), the
plan read-out, and the M-step (Newton on positions, MM on orientations).

Metric: cost-pair evaluations per second in Sinkhorn (2 * sum_t |I_t| |J_t| per
iteration).  Prints one JSON line.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cost-pair evals/s in Sinkhorn-EM at 1000 grains; time-to-index vs plain form"
UNIT = "pairs/s"


# DRAM bytes of one row-pass launch on the 1000-grain workload, counted by ncu
# (dram__bytes_read.sum + dram__bytes_write.sum) for the current kernels; None
# after a kernel change until it is captured again
SK_PASS_DRAM_BYTES = 42244608


def max_over_ranks(value, world, device):
    """The largest value over the ranks: the job's step time is the slowest
    replica's."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(units_per_rank, world, ms):
    """Whole-job throughput: every rank processes units_per_rank per step
    (weak scaling), the job takes the slowest rank's ms."""
    return units_per_rank * world / (ms / 1e3)


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self.proc = None
        self.thread = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append([s.strip() for s in line.split(",")])

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for s in self.samples:
            try:
                sm.append(float(s[1]))
                smax = float(s[2])
                for k, nm in enumerate(names):
                    if s[5 + k].lower().startswith("active"):
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload(dev, seed, api, sg, torch, grains=None, angles=None):
    import dataclasses
    cfg = sg.CONFIGS["batched"]
    if grains or angles:
        cfg = dataclasses.replace(cfg, n_grains=grains or cfg.n_grains, T=angles or cfg.T)
    geom = sg.Geometry()
    rng = np.random.default_rng(seed)
    R, x = sg.random_grains(cfg, rng)
    om = sg.omegas(cfg)
    h = api.Handle(dev)
    lat = api.Lattice.cubic(cfg.a, cfg.hmax, cfg.centering, device=dev)
    om_t = torch.tensor(om, dtype=torch.float32, device=dev)
    truth = api.forward(h, geom, lat, torch.tensor(R, device=dev), torch.tensor(x, device=dev), om_t)
    t_j = truth.angle[:truth.n].cpu().numpy()
    det = truth.spot[:truth.n, 3].cpu().numpy().astype(int)
    s = truth.spot[:truth.n, :3].cpu().numpy().astype(np.float64)
    obs = sg.observe(geom, cfg, t_j, det, s, rng)
    truth_grain = truth.grain[:truth.n].cpu().numpy()
    # starting poses (prototype stand-ins): truth perturbed by ~0.1 deg / 0.05 mm
    ang = rng.normal(size=(cfg.n_grains, 3)) * np.radians(0.1) / np.sqrt(3)
    th = np.linalg.norm(ang, axis=1, keepdims=True)
    k = ang / np.maximum(th, 1e-30)
    K = np.zeros((cfg.n_grains, 3, 3))
    K[:, 0, 1], K[:, 0, 2], K[:, 1, 2] = -k[:, 2], k[:, 1], -k[:, 0]
    K = K - K.transpose(0, 2, 1)
    s_ = np.sin(th)[:, :, None]
    c_ = (1 - np.cos(th))[:, :, None]
    dR = np.eye(3)[None] + s_ * K + c_ * (K @ K)
    R0 = dR @ R
    x0 = x + rng.normal(size=x.shape) * 0.05
    R0_t = torch.tensor(R0, dtype=torch.float32, device=dev).reshape(-1, 9).contiguous()
    x0_t = torch.tensor(x0, dtype=torch.float32, device=dev).contiguous()
    model = api.forward(h, geom, lat, R0_t, x0_t, om_t).truncated()
    ob = api.ObsSpots.from_numpy(obs.p, obs.I_off, device=dev)
    nI = np.diff(obs.I_off)
    nJ = np.diff(model.J_off.cpu().numpy())
    pairs_half = int(np.sum(nI.astype(np.int64) * nJ))
    return dict(cfg=cfg, geom=geom, h=h, lat=lat, om=om_t, obs=obs, ob=ob, model=model, R0=R0_t, x0=x0_t,
                R_true=R.reshape(-1, 3, 3), x_true=x, truth_grain=truth_grain, pairs_half=pairs_half, nI=int(nI.sum()), nJ=int(nJ.sum()), c_out=api.c_out_for(cfg.sigma_mm, geom.D))


def em_step(W, api, R, x, stream=None):
    """One EM iteration at eps_final (the last annealed step k = n_em - 1 of
    Algorithm LaueOT: refresh, E-step with read-out, M-step) in one laue_em
    call; the outputs are allocated once, so the call can be captured."""
    cfg, h = W["cfg"], W["h"]
    if "em_out" not in W:
        W["em_out"] = api.em_outputs(W["ob"], W["model"])
    k = cfg.n_em - 1
    return api.em(h, W["geom"], W["lat"], W["ob"], W["model"], W["om"], R, x, cfg.eps, cfg.n_em, cfg.n_sinkhorn,
                  W["c_out"], k_first=k, k_last=k, out=W["em_out"], stream=stream)


def oracle_workload(seed=0):
    """The 1000-grain workload built by the oracle's forward model (same seeds
    and generator as the GPU workload), for the CPU-baseline legs."""
    import oracle
    import synthgen as sg
    cfg = sg.CONFIGS["batched"]
    geom = sg.Geometry()
    rng = np.random.default_rng(seed)
    R, x = sg.random_grains(cfg, rng)
    om = sg.omegas(cfg)
    P = oracle.reflections(cfg.a, cfg.hmax, cfg.centering)
    fw = oracle.forward(geom, P, R, x, om)
    obs = sg.observe(geom, cfg, fw["t"], fw["det"], fw["spot"], rng)
    return dict(cfg=cfg, geom=geom, fw=fw, obs=obs, c_out=oracle.c_out_for(cfg.sigma_mm, geom.D))


def cpu_baseline_sample(OW, threads=1, blocks=(0, 45)):
    """The FP64 oracle's Sinkhorn on a bounded sample of the 1000-grain
    workload: one full iteration (row + column update) over the given angle
    blocks, on `threads` host threads (OpenMP over angle blocks)."""
    import oracle
    obs, fw = OW["obs"], OW["fw"]
    J_off = fw["J_off"]
    used = oracle.set_threads(threads)
    sel_i = np.concatenate([np.arange(obs.I_off[t], obs.I_off[t + 1]) for t in blocks])
    sel_j = np.concatenate([np.arange(J_off[t], J_off[t + 1]) for t in blocks])
    I_off = np.r_[0, np.cumsum([obs.I_off[t + 1] - obs.I_off[t] for t in blocks])]
    J_o = np.r_[0, np.cumsum([J_off[t + 1] - J_off[t] for t in blocks])]
    pairs = 2 * int(np.sum(np.diff(I_off) * np.diff(J_o)))
    t0 = time.perf_counter()
    oracle.sinkhorn(OW["geom"].D, obs.p[sel_i], I_off, J_o, fw["center"][sel_j], fw["ray"][sel_j, :3],
                    OW["cfg"].eps, OW["c_out"], 0, 0.4, 1)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    cpu = _cpu_model()
    return dict(value=pairs / dt, unit=UNIT, cores=used, kind="oracle", cpu_model=cpu, nproc=os.cpu_count(),
                sample="FP64 C oracle on %d thread(s) (OpenMP over angle blocks): 1 Sinkhorn iteration (row + column "
                       "update) on %d of the 90 angle blocks of the 1000-grain workload, %d pair evaluations in %.1f s"
                       % (used, len(blocks), pairs, dt))


def _cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part", "processor name")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


def _found_count(Rk, xk, R, x, tol_deg=0.5, tol_mm=0.5):
    """True grains with a found grain within tol (cubic symmetry aware)."""
    import itertools
    syms = []
    for perm in itertools.permutations(range(3)):
        for sgn in itertools.product([1, -1], repeat=3):
            S = np.zeros((3, 3))
            for r, c in enumerate(perm):
                S[r, c] = sgn[r]
            if np.linalg.det(S) > 0:
                syms.append(S)
    n = 0
    for g in range(len(R)):
        if len(Rk) == 0:
            break
        M = np.einsum("kji,jl->kil", Rk, R[g])
        best = np.full(len(Rk), 180.0)
        for S in syms:
            tr = np.trace(M @ S, axis1=1, axis2=2)
            best = np.minimum(best, np.degrees(np.arccos(np.clip((tr - 1) / 2, -1, 1))))
        n += bool(np.any((best < tol_deg) & (np.linalg.norm(xk - x[g], axis=1) < tol_mm)))
    return n


def proposal_bench(dev, api, sg, torch, peaks):
    """The learned proposal: training throughput, the tensor-core GEMM of the
    per-spot layers against its roofline, time-to-index of the plain and the
    learned form on a workload both recover, and the oracle beside it."""
    import dataclasses
    import time
    from paper_2404_06478_gb300 import proposal as pr
    h = api.Handle(dev)
    geom = sg.Geometry()
    cfgB = sg.CONFIGS["batched"]
    lat = api.Lattice.cubic(cfgB.a, cfgB.hmax, cfgB.centering, device=dev)
    omega = torch.tensor(sg.omegas(cfgB), dtype=torch.float32, device=dev)
    out = {}
    # training: 20000 steps of 2048 sets (64 single-grain scenes x 32 seeds)
    steps = 20000
    pr.train(h, geom, lat, omega, steps=20, seed=1)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    net = pr.train(h, geom, lat, omega, steps=steps, gmin=1, gmax=1, seed=7)
    e1.record()
    torch.cuda.synchronize()
    tr_s = e0.elapsed_time(e1) / 1e3
    out["train"] = dict(steps=steps, sets_per_step=2048, seconds=tr_s, sets_per_s=steps * 2048 / tr_s,
                        ms_per_step=tr_s * 1e3 / steps, data="single-grain scenes simulated on the GPU")
    # the per-spot GEMMs at training-batch size (inputs > L2)
    Ms = 2048 * 128
    A = torch.randn(Ms, 256, device=dev).to(torch.bfloat16)
    B = (torch.randn(256, 256, device=dev) * 0.05).to(torch.bfloat16)
    bias = torch.zeros(256, device=dev)
    D = torch.empty(Ms, 256, dtype=torch.bfloat16, device=dev)
    # weight-gradient operands: errors and activations as the layers store
    # them, row-major [spots][channels], read MN-major by the GEMM
    dZ = torch.randn(Ms, 256, device=dev).to(torch.bfloat16)
    Hp = torch.randn(Ms, 256, device=dev).to(torch.bfloat16)
    part = torch.empty(64, 256, 256, device=dev)

    def timed(fn, reps=20):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps / 1e3

    t_fwd = timed(lambda: pr.gemm_bf16(h, A, B, mode=1, bias=bias, out=D))
    # context for write-heavy kernels: a plain fill of the same output bytes
    t_fill = timed(lambda: D.fill_(1.0))
    t_wg = timed(lambda: pr.gemm_bf16(h, dZ, Hp, mode=0, splits=64, out_f32=part, a_mn=True, b_mn=True))
    fl = 2.0 * Ms * 256 * 256
    # the method's bytes: A read and one output written
    by_fwd = Ms * 256 * 2 + Ms * 256 * 2 + 256 * 256 * 2
    by_wg = 2 * 256 * Ms * 2 + 64 * 256 * 256 * 4
    hbm, bf = peaks.get("hbm_gbs", 6800.0), peaks.get("bf16_tflops", 1900.0)
    out["gemm"] = dict(
        kernel="gemm_tc_kernel (tcgen05, TMA, TMEM)",
        forward_layer=dict(shape="M=%d N=256 K=256, bias+ReLU, BF16 out row-major" % Ms,
                           us=t_fwd * 1e6, tflops=fl / t_fwd / 1e12, tensor_frac_of_measured=fl / t_fwd / 1e12 / bf,
                           roofline=dict(bound="hbm", achieved=by_fwd / t_fwd / 1e9, peak=hbm, unit="GB/s",
                                         frac=by_fwd / t_fwd / 1e9 / hbm, traffic=None,
                                         algorithmic_bytes=by_fwd)),
        weight_grad=dict(shape="M=256 N=256 K=%d, split-K 64, FP32 partials, both operands MN-major" % Ms,
                         us=t_wg * 1e6,
                         tflops=fl / t_wg / 1e12, tensor_frac_of_measured=fl / t_wg / 1e12 / bf,
                         roofline=dict(bound="hbm", achieved=by_wg / t_wg / 1e9, peak=hbm, unit="GB/s",
                                       frac=by_wg / t_wg / 1e9 / hbm, traffic=None, algorithmic_bytes=by_wg)),
        peaks_basis="MEASURED_PEAKS.json (hbm_gbs %.1f, bf16_tflops %.1f)" % (hbm, bf),
        write_only_GBs=D.numel() * 2 / t_fill / 1e9,
        write_note="a plain fill (torch) of the output array runs at write_only_GBs: half of the forward "
                   "layer's bytes are HBM writes")
    del A, B, D, dZ, Hp, part
    out["time_to_index"] = index_bench(dev, api, sg, torch, h, net, geom, lat, omega)
    assert h.device_status() == 0
    return out


def _medium_workload(dev, api, sg, torch, h, seed=0, grains=None):
    """The 100-grain / 60-rotation / 30%-outlier workload (|hkl| <= 6), spots
    from the CUDA forward model."""
    import dataclasses
    cfg = sg.CONFIGS["medium"]
    if grains:
        cfg = dataclasses.replace(cfg, n_grains=grains)
    geom = sg.Geometry()
    rng = np.random.default_rng(seed)
    R, x = sg.random_grains(cfg, rng)
    om_t = torch.tensor(sg.omegas(cfg), dtype=torch.float32, device=dev)
    lat = api.Lattice.cubic(cfg.a, cfg.hmax, cfg.centering, device=dev)
    tr = api.forward(h, geom, lat, torch.tensor(R, device=dev), torch.tensor(x, device=dev), om_t)
    obs = sg.observe(geom, cfg, tr.angle[:tr.n].cpu().numpy(), tr.spot[:tr.n, 3].cpu().numpy().astype(int),
                     tr.spot[:tr.n, :3].cpu().numpy().astype(np.float64), rng)
    ob = api.ObsSpots.from_numpy(obs.p, obs.I_off, device=dev)
    return dict(cfg=cfg, geom=geom, lat=lat, om=om_t, ob=ob, obs=obs, R=R, x=x, nI=len(obs.p),
                c_out=api.c_out_for(cfg.sigma_mm, geom.D))


def index_bench(dev, api, sg, torch, h, net, geom, lat_b, omega_b):
    """Time-to-index (one laue_index call, from the start set to the final
    EM) on the 100-grain configuration in the plain form (the library's start
    grid, Newton + MM M-step), the plain form with the adjoint M-step, and the
    learned-proposal forms; the single-grain fit kernel against its ALU
    roofline; the learned proposal at the 1000-grain density."""
    from paper_2404_06478_gb300 import proposal as pr
    out = {}
    M = _medium_workload(dev, api, sg, torch, h)
    cfg = M["cfg"]
    grid = dict(n_full=1_200_000, sym=24, k=1, cube_mm=cfg.cube_mm)
    fit = dict(k_single=40, anneal_single=1000.0, recut_single=True)
    em = dict(n_em=cfg.n_em, n_sinkhorn=cfg.n_sinkhorn)

    def run(form):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if form.startswith("learned"):
            seeds = np.random.default_rng(5).choice(M["nI"], 2500, replace=False)
            R0, x0 = pr.propose(h, net, geom, M["ob"], M["om"], seeds)
            starts = int(R0.shape[0])
        else:
            R0 = x0 = None
        Rf, xf, _ = api.index(h, geom, M["lat"], M["ob"], M["om"], R0, x0, cfg.eps, M["c_out"], 200,
                              grid=grid if R0 is None else None, mstep="adjoint" if "adjoint" in form else "plain",
                              **fit, **em)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        assert h.device_status() == 0
        Rk = Rf.cpu().numpy().reshape(-1, 3, 3).astype(np.float64)
        xk = xf.cpu().numpy().astype(np.float64)
        found = _found_count(Rk, xk, M["R"], M["x"], 0.5, 0.1)
        return dict(seconds=dt, k_star=len(Rk), grains_found=found, recall=found / cfg.n_grains,
                    starts=starts if R0 is not None else None)

    forms = {f: run(f) for f in ("plain", "plain_adjoint", "learned_adjoint", "learned")}
    # the single-grain fit kernel alone on the same grid, with its pair evaluations counted on the device
    Rg, xg = api.start_grid(h, grid["n_full"], 24, 1, cfg.cube_mm)
    h.counters()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    api.single_fit(h, geom, M["lat"], M["ob"], M["om"], Rg, xg, cfg.eps, fit["k_single"], M["c_out"],
                   anneal=fit["anneal_single"], recut=True)
    e1.record()
    torch.cuda.synchronize()
    fit_s = e0.elapsed_time(e1) / 1e3
    pairs = h.counters()["fit_pairs"]
    pk = h.alu_peaks()
    peak = min(max(pk["ffma"], pk["ffma2"]) / 13.0, pk["ex2"], pk["rsqrt"])
    plain_s = forms["plain"]["seconds"]
    out["medium"] = dict(
        workload="100 grains, |hkl|<=6 bcc, 60 rotations over 360 deg, 0.5 mm noise, 30% outliers; eps 1 mm^2, "
                 "30 EM steps x 200 Sinkhorn iterations; found = within 0.5 deg and 0.1 mm of the truth",
        start_grid="1.2M super-Fibonacci points restricted to the cubic fundamental zone (%d orientations) at the "
                   "cube centre; fits of 40 steps annealed from 1000 eps with visible spots re-listed every step"
                   % int(Rg.shape[0]),
        learned_starts="2500 random seed spots x 8 hypotheses of the set encoder",
        forms=forms,
        speedup_vs_plain={f: plain_s / v["seconds"] for f, v in forms.items()},
        fit_kernel=dict(kernel="single_fit_kernel", starts=int(Rg.shape[0]), seconds=fit_s,
                        starts_per_s=int(Rg.shape[0]) / fit_s, pair_evaluations=pairs,
                        roofline=dict(bound="alu", achieved=pairs / fit_s, peak=peak, unit="pairs/s",
                                      frac=pairs / fit_s / peak,
                                      peak_basis="min(FP32 lane-ops/s / 13, MUFU ex2/s, MUFU rsqrt/s) measured by "
                                                 "laue_alu_peaks; one pair evaluation = one cost and one exponential")))
    del Rg, xg
    # 5 grains (the learned form's working density) in the 90-rotation geometry
    W5 = build_workload(dev, 5, api, sg, torch, grains=5)
    res5 = {}
    for form in ("plain", "learned_adjoint"):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if form == "plain":
            R0 = x0 = None
        else:
            seeds = np.random.default_rng(5).choice(W5["nI"], 2500, replace=False)
            R0, x0 = pr.propose(h, net, geom, W5["ob"], W5["om"], seeds)
        Rf, xf, _ = api.index(h, geom, W5["lat"], W5["ob"], W5["om"], R0, x0, W5["cfg"].eps, W5["c_out"], 50,
                              grid=dict(n_full=4_800_000, sym=24, k=1, cube_mm=5.0) if R0 is None else None,
                              mstep="plain" if form == "plain" else "adjoint", n_em=20, n_sinkhorn=100, k_single=8,
                              f_out=0.3)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        found = _found_count(Rf.cpu().numpy().reshape(-1, 3, 3).astype(np.float64),
                             xf.cpu().numpy().astype(np.float64), W5["R_true"], W5["x_true"])
        res5[form] = dict(seconds=dt, grains_found=found, k_star=int(Rf.shape[0]))
    out["five_grains"] = dict(workload="5 grains, |hkl|<=6 bcc, 90 rotations over 360 deg, 70% uneven outliers; "
                                       "found = within 0.5 deg and 0.5 mm of the truth",
                              plain=res5["plain"], learned_adjoint=res5["learned_adjoint"],
                              speedup=res5["plain"]["seconds"] / res5["learned_adjoint"]["seconds"],
                              plain_starts="4.8M super-Fibonacci points restricted to the cubic fundamental zone "
                                           "(200k orientations) at the cube centre")
    del W5
    # 1000 grains: the fit kernel's rate on a bounded sample of grid starts, and the
    # set encoder's hypotheses against the seeds' own grains
    W = build_workload(dev, 0, api, sg, torch)
    Rg, xg = api.start_grid(h, 1_200_000, 24, 1, 5.0)
    n_s = 600
    h.counters()
    torch.cuda.synchronize()
    e0.record()
    _, _, keep, _ = api.single_fit(h, geom, W["lat"], W["ob"], W["om"], Rg[:n_s].contiguous(), xg[:n_s].contiguous(),
                                   W["cfg"].eps, 40, W["c_out"], anneal=1000.0, recut=True)
    e1.record()
    torch.cuda.synchronize()
    s1000 = e0.elapsed_time(e1) / 1e3
    p1000 = h.counters()["fit_pairs"]
    seeds = np.random.default_rng(6).choice(np.nonzero(W["obs"].truth >= 0)[0], 2000, replace=False)
    Rp, _ = pr.propose(h, net, geom, W["ob"], W["om"], seeds)
    Rp = Rp.cpu().numpy().reshape(len(seeds), 8, 3, 3).astype(np.float64)
    gtrue = W["truth_grain"][W["obs"].truth[seeds]]
    good = 0
    for k, g in enumerate(gtrue):
        M_ = np.einsum("hji,jl->hil", Rp[k], W["R_true"][g])
        best = 180.0
        for S_ in _cubic_group():
            c = np.clip((np.trace(M_ @ S_, axis1=1, axis2=2) - 1) / 2, -1, 1)
            best = min(best, float(np.degrees(np.arccos(c)).min()))
        good += best < 3.0
    out["thousand_grains"] = dict(
        workload="1000 grains, 90 rotations, 70% uneven outliers",
        fit_sample=dict(starts=n_s, seconds=s1000, starts_per_s=n_s / s1000, pair_evaluations=p1000,
                        pairs_per_s=p1000 / s1000, kept_fraction=float(keep.float().mean().item()),
                        projected_seconds_for_the_50k_grid=50000 * s1000 / n_s),
        proposal_quality=dict(seeds=len(seeds), within_3deg_of_seed_grain=good / len(seeds),
                              note="fraction of true-spot seeds with one of the 8 hypotheses within 3 deg of the "
                                   "seed's own grain (chance is about 1%)"))
    return out


def _cubic_group():
    import itertools
    out = []
    for perm in itertools.permutations(range(3)):
        for sgn in itertools.product([1, -1], repeat=3):
            S = np.zeros((3, 3))
            for r, c in enumerate(perm):
                S[r, c] = sgn[r]
            if np.linalg.det(S) > 0:
                out.append(S)
    return out


def proposal_cpu_baseline():
    """The oracle's set encoder (FP64, BF16-emulating) forward + backward on a
    bounded sample of 8 sets, timed on one host core."""
    import time
    import oracle.proposal as op
    rng = np.random.default_rng(0)
    P = op.init_params(rng)
    B = 8
    X = np.zeros((B, op.KSET, op.NF))
    X[:, :, :14] = rng.standard_normal((B, op.KSET, 14))
    X[:, :, 12] = 1.0
    Rt = np.stack([np.eye(3)] * B)
    xt = np.zeros((B, 3))
    t0 = time.perf_counter()
    O, cache = op.forward(P, X, bf16_ops=True)
    _, dO, _, _ = op.set_loss(O, Rt, xt, np.ones(B))
    op.backward(P, cache, dO)
    dt = time.perf_counter() - t0
    return dict(value=B / dt, unit="sets/s (forward + backward)", cores=1, kind="oracle",
                sample="%d sets of 128 spots" % B)


def run_reference(args):
    """The reference arm: the FP64 oracle (the paper gives no program) timed
    on the host cores on a bounded sample of the same workload, whose inputs
    the oracle's own forward model builds.  Rank 0 only."""
    rank, world, local = _dist_env()
    if rank != 0:
        return 0
    OW = oracle_workload(0)
    vals, samples = [], []
    for _ in range(max(1, args.steps)):
        r = cpu_baseline_sample(OW, threads=os.cpu_count() or 1, blocks=tuple(range(0, 90, 3)))
        vals.append(r["value"])
        samples.append(r)
    v = float(np.mean(vals))
    r = samples[-1]
    line = dict(impl="reference", metric=METRIC, value=v, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, higher_is_better=True, dtype="f64", data="synthetic",
                config=dict(workload="1000 grains, 90 rotations, 70% uneven outliers, |hkl|<=6; oracle sample"),
                cpu_baseline=dict(kind="oracle", cores=r["cores"], value=v, cpu_model=r["cpu_model"],
                                  sample=r["sample"] + " (per step)"),
                e2e=dict(value=v, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--grains", type=int, default=None, help="smaller case for profiling (not a bench line)")
    ap.add_argument("--angles", type=int, default=None, help="smaller case for profiling (not a bench line)")
    ap.add_argument("--no-proposal", action="store_true", help="skip the learned-proposal measurements")
    ap.add_argument("--only-proposal-train", type=int, default=0,
                    help="run only this many set-encoder training steps (profiling; not a bench line)")
    ap.add_argument("--only-fit-grid", type=int, default=0,
                    help="run only the single-grain fits of the 100-grain workload from a start grid of this many "
                         "spiral points (profiling; not a bench line)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.only_proposal_train:
        import torch
        from paper_2404_06478_gb300 import api, build, proposal as pr
        import synthgen as sg
        build.build()
        dev = torch.device("cuda", 0)
        h = api.Handle(dev)
        cfgB = sg.CONFIGS["batched"]
        lat = api.Lattice.cubic(cfgB.a, cfgB.hmax, cfgB.centering, device=dev)
        omega = torch.tensor(sg.omegas(cfgB), dtype=torch.float32, device=dev)
        t0 = time.perf_counter()
        pr.train(h, sg.Geometry(), lat, omega, steps=args.only_proposal_train, seed=3)
        torch.cuda.synchronize()
        assert h.device_status() == 0
        print(json.dumps(dict(proposal_train_steps=args.only_proposal_train, sets_per_step=2048,
                              seconds=time.perf_counter() - t0)))
        return 0
    if args.only_fit_grid:
        import torch
        from paper_2404_06478_gb300 import api, build
        import synthgen as sg
        build.build()
        dev = torch.device("cuda", 0)
        h = api.Handle(dev)
        M = _medium_workload(dev, api, sg, torch, h)
        Rg, xg = api.start_grid(h, args.only_fit_grid, 24, 1, M["cfg"].cube_mm)
        h.counters()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        api.single_fit(h, M["geom"], M["lat"], M["ob"], M["om"], Rg, xg, M["cfg"].eps, 40, M["c_out"], anneal=1000.0,
                       recut=True)
        torch.cuda.synchronize()
        assert h.device_status() == 0
        print(json.dumps(dict(fit_starts=int(Rg.shape[0]), seconds=time.perf_counter() - t0,
                              pair_evaluations=h.counters()["fit_pairs"])))
        return 0
    rank, world, local = _dist_env()
    import torch
    import torch.distributed as dist
    if world > 1 and not dist.is_initialized():
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    from paper_2404_06478_gb300 import api, build
    import synthgen as sg
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    W = build_workload(dev, rank, api, sg, torch, args.grains, args.angles)
    stream = torch.cuda.current_stream()
    # the project's autotuner picks the launch shapes of the Sinkhorn passes for this problem
    tuned = api.autotune(W["h"], W["geom"], W["ob"], W["model"], W["cfg"].eps, W["c_out"], n_iter=3)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)  # > L2 (129 MB)
    R = W["R0"].clone()
    x = W["x0"].clone()
    for _ in range(args.warmup):
        em_step(W, api, R.clone(), x.clone())
    torch.cuda.synchronize()
    # per-launch duration of the dominant kernel: differential timing of the
    # Sinkhorn passes (n2 - n1 iterations = 2 (n2 - n1) launches of the pair passes)
    cfg = W["cfg"]
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    n1, n2 = 20, 120
    W["h"].counters()  # clear
    ev[0].record(stream)
    api.cost_sinkhorn(W["h"], W["geom"], W["ob"], W["model"], cfg.eps, W["c_out"], n1, harvest=False)
    ev[1].record(stream)
    c1 = W["h"].counters()["pass_pairs"]
    ev[2].record(stream)
    api.cost_sinkhorn(W["h"], W["geom"], W["ob"], W["model"], cfg.eps, W["c_out"], n2, harvest=False)
    ev[3].record(stream)
    torch.cuda.synchronize()
    c2 = W["h"].counters()["pass_pairs"]
    per_launch_ms = (ev[2].elapsed_time(ev[3]) - ev[0].elapsed_time(ev[1])) / (2 * (n2 - n1))
    # pairs the passes evaluated after the exact underflow skipping, per launch
    evaluated_per_launch = (c2 - c1) / (2.0 * (n2 - n1))

    # the whole EM iteration captured once as a CUDA graph on static pose buffers
    Rs, xs = W["R0"].clone(), W["x0"].clone()
    cap_stream = torch.cuda.Stream()
    cap_stream.wait_stream(stream)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.stream(cap_stream):
        with torch.cuda.graph(graph, stream=cap_stream):
            em_step(W, api, Rs, xs)
    stream.wait_stream(cap_stream)
    torch.cuda.synchronize()

    clocks = ClockSampler(local)
    clocks.start()
    times = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        Rs.copy_(W["R0"])
        xs.copy_(W["x0"])
        graph.replay()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ms = max_over_ranks(float(np.mean(times)), world, dev)
    pairs_step = 2 * W["pairs_half"] * cfg.n_sinkhorn
    value = job_value(pairs_step, world, ms)

    # end to end through the C ABI with host buffers: H2D of the step's inputs
    # from pinned memory, the step, D2H of its results
    p_host = W["ob"].p.cpu().pin_memory()
    R_host = W["R0"].cpu().pin_memory()
    x_host = W["x0"].cpu().pin_memory()
    a_host = torch.empty(W["nI"], dtype=torch.int32).pin_memory()
    Ro_host = torch.empty_like(R_host).pin_memory()
    xo_host = torch.empty_like(x_host).pin_memory()
    e2e_times = []
    for k in range(max(2, args.steps // 2)):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        W["ob"].p.copy_(p_host, non_blocking=True)
        Rk = R_host.to(dev, non_blocking=True)
        xk = x_host.to(dev, non_blocking=True)
        out = em_step(W, api, Rk, xk)
        a_host.copy_(out["assign"], non_blocking=True)
        Ro_host.copy_(Rk, non_blocking=True)
        xo_host.copy_(xk, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_times.append(e0.elapsed_time(e1))
    e2e_ms = float(np.mean(e2e_times))
    h2d = p_host.numel() * 4 + R_host.numel() * 4 + x_host.numel() * 4
    d2h = a_host.numel() * 4 + Ro_host.numel() * 4 + xo_host.numel() * 4

    # the adjoint of the OT-weighted cost at the same size: gradient with
    # respect to every grain's axis-angle and position, costs recomputed
    out_sk = api.cost_sinkhorn(W["h"], W["geom"], W["ob"], W["model"], cfg.eps, W["c_out"], cfg.n_sinkhorn,
                               harvest=False)
    api.objective_grad(W["h"], W["geom"], W["lat"], W["ob"], W["model"], out_sk["f"], out_sk["g"], cfg.eps,
                       W["om"], W["R0"], W["x0"])
    torch.cuda.synchronize()
    ea, eb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ea.record(stream)
    for _ in range(5):
        api.objective_grad(W["h"], W["geom"], W["lat"], W["ob"], W["model"], out_sk["f"], out_sk["g"], cfg.eps,
                           W["om"], W["R0"], W["x0"])
    eb.record(stream)
    torch.cuda.synchronize()
    adj_ms = ea.elapsed_time(eb) / 5
    adjoint = dict(ms_per_call=adj_ms, pairs_per_s=W["pairs_half"] / (adj_ms / 1e3),
                   grains=cfg.n_grains, note="gradient of sum_ij Q_ij C_ij wrt each grain's axis-angle and "
                                             "position (Q from 200 Sinkhorn iterations, costs recomputed)")

    # the sparse E-step (each model spot keeps its rho = 32 nearest observed
    # spots) at the same size: set-up (neighbour lists and their transpose)
    # and per-iteration time, HBM roofline of the passes, and how often its
    # hard assignment equals the dense plan's
    rho = 32
    sp_kw = dict(rho=rho, harvest=True)
    api.cost_sinkhorn_sparse(W["h"], W["geom"], W["ob"], W["model"], cfg.eps, W["c_out"], 2, **sp_kw)
    torch.cuda.synchronize()
    es = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    es[0].record(stream)
    api.cost_sinkhorn_sparse(W["h"], W["geom"], W["ob"], W["model"], cfg.eps, W["c_out"], 0, **sp_kw)
    es[1].record(stream)
    es[2].record(stream)
    sp = api.cost_sinkhorn_sparse(W["h"], W["geom"], W["ob"], W["model"], cfg.eps, W["c_out"], cfg.n_sinkhorn,
                                  **sp_kw)
    es[3].record(stream)
    torch.cuda.synchronize()
    assert W["h"].device_status() == 0
    sp_setup_ms = es[0].elapsed_time(es[1])
    sp_total_ms = es[2].elapsed_time(es[3])
    sp_iter_ms = (sp_total_ms - sp_setup_ms) / cfg.n_sinkhorn
    dn = api.cost_sinkhorn(W["h"], W["geom"], W["ob"], W["model"], cfg.eps, W["c_out"], cfg.n_sinkhorn,
                           harvest=True)
    torch.cuda.synchronize()
    sure = dn["margin"] > 1e-3
    agree = float((sp["assign"][sure] == dn["assign"][sure]).float().mean())
    nnz = W["nJ"] * rho
    sp_bytes = 16.0 * nnz + 8.0 * (W["nI"] + W["nJ"])  # {index, e2} records of both passes, potentials
    hbm_peak = None
    pk_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        hbm_peak = json.load(open(pk_path)).get("hbm_gbs")
    sparse = dict(rho=rho, setup_ms=sp_setup_ms, ms_per_iteration=sp_iter_ms, ms_200_iterations=sp_total_ms,
                  dense_ms_per_iteration=2 * per_launch_ms,
                  speedup_per_iteration=2 * per_launch_ms / sp_iter_ms,
                  assign_agreement_with_dense=agree,
                  roofline=dict(bound="hbm", bytes_per_iteration=sp_bytes,
                                achieved_gbs=sp_bytes / (sp_iter_ms / 1e3) / 1e9, peak_gbs=hbm_peak,
                                frac=(sp_bytes / (sp_iter_ms / 1e3) / 1e9 / hbm_peak) if hbm_peak else None,
                                note="algorithmic bytes: 8-byte {index, e2} record per support entry in each of "
                                     "the two passes plus one potential read and written per spot; gathers of "
                                     "the other side's potentials hit L2"),
                  note="paper Section 'Working with sparse assignment matrices'; agreement over rows whose dense "
                       "top-two margin exceeds 1e-3")

    # refresh 1; Sinkhorn: schedule, pack, dust init, G maxima, 2 per iteration, clear, harvest,
    # finish; M-step: schedule, pack, dust init, G maxima, segment count + scan, init, 2 per Newton step,
    # MM pair + MM grain, norms
    launches_per_step = 1 + (4 + 2 * cfg.n_sinkhorn + 3) + (4 + 2 + 1 + 2 * 4 + 2 + 1)
    # roofline: the algorithmic pair evaluation is 13 FP32 lane-ops (3 sub,
    # 3 for |d|^2, 3 for d.r, 1 for the cosine, 1 fold with the potential, 1
    # running-maximum update, 1 accumulate), 1 MUFU rsqrt and 1 MUFU ex2; the
    # peak is the slowest of the three pipes, each measured on this device by
    # laue_alu_peaks.  The kernel itself spends 14 (it forms |rhat - r|^2 from
    # the difference vector, which keeps the small costs of matched pairs free
    # of cancellation, and needs no running maximum): frac_kernel_ops.
    pk_ = W["h"].alu_peaks()
    fp32 = max(pk_["ffma"], pk_["ffma2"])
    peak = min(fp32 / 13.0, pk_["ex2"], pk_["rsqrt"])
    peak14 = min(fp32 / 14.0, pk_["ex2"], pk_["rsqrt"])
    bound_by = min((fp32 / 13.0, "fp32"), (pk_["ex2"], "mufu_ex2"), (pk_["rsqrt"], "mufu_rsqrt"))[1]
    achieved = evaluated_per_launch / (per_launch_ms / 1e3)
    line = dict(
        metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps, warmup=args.warmup,
        ms_per_step=ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic",
        config=dict(workload="%d grains, |hkl|<=6 bcc, %d rotations over 360 deg, 0.5 mm noise, "
                             "70%% uneven Poisson outliers, eps=1 mm^2, 200 Sinkhorn iterations per EM step"
                             % (cfg.n_grains, cfg.T),
                    grains=cfg.n_grains, angles=cfg.T, observed=W["nI"], model_spots=W["nJ"],
                    pairs_per_half_iteration=W["pairs_half"],
                    step="one EM iteration (refresh, 200 Sinkhorn iterations with read-out, M-step), replayed as "
                         "one CUDA graph",
                    l2="256 MB buffer written between timed steps", parallelism="replicas" if world > 1 else "1 GPU",
                    autotuned_shapes={"row": tuned[0], "col": tuned[1],
                                      "ms_per_pass": [[round(r, 3), round(c, 3)] for r, c in tuned[2]]}),
        roofline=dict(bound="alu", achieved=achieved, peak=peak, unit="pairs/s", frac=achieved / peak,
                      frac_kernel_ops=achieved / peak14,
                      traffic=SK_PASS_DRAM_BYTES if (cfg.n_grains == 1000 and SK_PASS_DRAM_BYTES) else None,
                      traffic_unit="bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum of one row-pass "
                                   "launch, ncu capture of this workload; profiles/sk_row_kernel_dram_1000grains_"
                                   "90angles.md)",
                      kernel="sk_row_kernel+sk_col_kernel (per launch; evaluated pairs after the exact skipping)",
                      peak_basis="min(FP32 lane-ops/s / 13, MUFU ex2/s, MUFU rsqrt/s), measured by "
                                 "laue_alu_peaks; binding pipe: %s" % bound_by,
                      pipes={k: v for k, v in pk_.items()}),
        clocks=clk,
        e2e=dict(value=pairs_step / (e2e_ms / 1e3), unit=UNIT, h2d_bytes_per_step=int(h2d),
                 d2h_bytes_per_step=int(d2h)),
        gpu_launches=launches_per_step * args.steps,
        em_iterations_per_s=1e3 / ms,
        pairs=dict(dense_equivalent_per_s=value, evaluated_per_s=value * evaluated_per_launch / W["pairs_half"],
                   evaluated_fraction=evaluated_per_launch / W["pairs_half"],
                   note="value counts 2 sum_t |I_t||J_t| pair evaluations per Sinkhorn iteration (the dense "
                        "plan); the passes skip (tile, chunk) combinations whose plan entries all underflow to "
                        "exactly 0 in FP32 (potentials bit-identical), and evaluate the fraction shown"),
        adjoint=adjoint,
        sparse_estep=sparse,
    )
    if rank == 0 and not args.no_proposal:
        peaks = {}
        pk_path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")
        if os.path.exists(pk_path):
            peaks = json.load(open(pk_path))
        line["proposal"] = proposal_bench(dev, api, sg, torch, peaks)
        if not args.no_cpu_baseline:
            line["proposal"]["cpu_baseline"] = proposal_cpu_baseline()
    if rank == 0 and not args.no_cpu_baseline:
        OW = oracle_workload(0)
        one = cpu_baseline_sample(OW, threads=1)
        allc = cpu_baseline_sample(OW, threads=os.cpu_count() or 1, blocks=tuple(range(0, 90, 3)))
        line["cpu_baseline"] = dict(allc, single_thread=dict(value=one["value"], cores=1, sample=one["sample"]))
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
