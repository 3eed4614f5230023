"""Learned proposal over the C ABI: the tensor-core GEMM of the set encoder
(more calls follow in this module as the encoder is built).

Argument marshalling only: every step runs in liblaueot.so.  The paper has no
learned component; this is an addition beside its candidate scan.
"""
from __future__ import annotations

import torch

from . import api


def gemm_bf16(h: api.Handle, A: torch.Tensor, B: torch.Tensor, mode: int = 0, bn: int = 256, splits: int = 1,
              bias: torch.Tensor | None = None, mask: torch.Tensor | None = None, out_f32=None, out=None,
              outT=None, simple: bool = False, a_mn: bool = False, b_mn: bool = False, stream=None):
    """D[m][n] = sum_k A[m][k] B[n][k] on the tcgen05 tensor cores (BF16 in,
    FP32 accumulate).  A is (M, K) and B (N, K), or, with a_mn / b_mn, the
    stored arrays (K, M) / (K, N) read MN-major.  mode 0 writes `splits` FP32
    partials into out_f32 (splits, M, N); mode 1 relu(D + bias) and mode 2
    D * (mask > 0) as BF16 into out (M, N) and/or outT (N, ldt)."""
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16 and A.is_cuda and B.is_cuda
    K, M = A.shape if a_mn else A.shape[::-1]
    N = B.shape[1] if b_mn else B.shape[0]
    if h.ws is None:
        h.reserve(1, stream=stream)
    ldt = outT.stride(0) if outT is not None else 0
    flags = (1 if simple else 0) | (2 if a_mn else 0) | (4 if b_mn else 0)
    rc = h.L.laue_gemm_bf16(h.h, api._ptr(A), A.stride(0), api._ptr(B), B.stride(0), M, N, K, bn, splits, mode,
                            api._ptr(bias), api._ptr(mask), api._ptr(out_f32), api._ptr(out), api._ptr(outT), ldt,
                            flags, api._stream(stream))
    h.check(rc, "gemm_bf16")


# ---------------------------------------------------------------- set encoder
NF, NHYP, NOUT = 64, 8, 72
KSET = 128  # spots per set; equals laue_lp_set_size() of the library (checked by the tests)
REGIONS = dict(X=0, F=2, nvalid=3, Rt=4, xt=5, svalid=6, O=7, loss=8, dbest=9, hbest=10, H1=11, H3=12,
               pool=13, dO=14, dZ3=15)
PARAM_SHAPES = [("W1", (256, 64)), ("b1", (256,)), ("W2", (256, 256)), ("b2", (256,)), ("W3", (256, 256)),
                ("b3", (256,)), ("W4", (256, 512)), ("b4", (256,)), ("W5", (72, 256)), ("b5", (72,))]


def _aligned(nbytes, device, align=256):
    """A uint8 device buffer of nbytes whose data pointer is `align`-aligned."""
    raw = torch.empty(nbytes + align, dtype=torch.uint8, device=device)
    off = (-raw.data_ptr()) % align
    return raw, raw[off:off + nbytes]


def init_params(seed: int):
    """He-normal weights for the ReLU layers, 1/fan_in variance for the output
    layer, zero biases (FP32 vector in the library's parameter order)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for name, shape in PARAM_SHAPES:
        if name.startswith("b"):
            out.append(np.zeros(shape, np.float32))
        else:
            gain = 1.0 if name == "W5" else 2.0
            out.append((rng.standard_normal(shape) * (gain / shape[1]) ** 0.5).astype(np.float32))
    return np.concatenate([a.reshape(-1) for a in out])


def unpack_params(vec):
    """Parameter vector -> dict of arrays in PARAM_SHAPES order."""
    out, o = {}, 0
    for name, shape in PARAM_SHAPES:
        n = 1
        for d in shape:
            n *= d
        out[name] = vec[o:o + n].reshape(shape)
        o += n
    return out


class Network:
    """Parameters, Adam state and gradients of the set encoder in one device
    buffer owned by this object."""

    def __init__(self, h: api.Handle, params=None, seed: int = 0, stream=None):
        import ctypes
        import numpy as np
        self.h, self.L = h, h.L
        if h.ws is None:
            h.reserve(1, stream=stream)
        self.n_params = int(self.L.laue_lp_param_count())
        self._raw, self.buf = _aligned(int(self.L.laue_lp_net_bytes()), h.device)
        vec = init_params(seed) if params is None else np.ascontiguousarray(params, np.float32)
        assert vec.size == self.n_params
        h.check(self.L.laue_lp_net_init(h.h, api._ptr(self.buf), vec.ctypes.data_as(ctypes.c_void_p),
                                        api._stream(stream)), "lp_net_init")

    def params(self, stream=None):
        import ctypes
        import numpy as np
        out = np.zeros(self.n_params, np.float32)
        self.h.check(self.L.laue_lp_net_params(self.h.h, api._ptr(self.buf), out.ctypes.data_as(ctypes.c_void_p),
                                               None, api._stream(stream)), "lp_net_params")
        return out

    def grads(self, stream=None):
        import ctypes
        import numpy as np
        out = np.zeros(self.n_params, np.float32)
        self.h.check(self.L.laue_lp_net_params(self.h.h, api._ptr(self.buf), None, out.ctypes.data_as(ctypes.c_void_p),
                                               api._stream(stream)), "lp_net_params")
        return out


class Batch:
    """Device buffer for n_sets seed-conditioned sets and their activations."""

    def __init__(self, h: api.Handle, n_sets: int):
        self.h, self.L, self.n = h, h.L, int(n_sets)
        if h.ws is None:
            h.reserve(1)
        self._raw, self.buf = _aligned(int(self.L.laue_lp_batch_bytes(self.n)), h.device)
        self.ids = torch.empty(self.n * KSET, dtype=torch.int32, device=h.device)

    def region(self, name, dtype, shape):
        off = int(self.L.laue_lp_batch_offset(self.n, REGIONS[name]))
        item = torch.empty(0, dtype=dtype).element_size()
        n = 1
        for d in shape:
            n *= d
        return self.buf[off:off + n * item].view(dtype).view(*shape)

    def outputs(self):
        return self.region("O", torch.float32, (self.n, NOUT))

    def features(self):
        return self.region("X", torch.bfloat16, (self.n, KSET, NF))

    def frames(self):
        return self.region("F", torch.float32, (self.n, 3, 3))


def make_sets(h: api.Handle, geom, p4: torch.Tensor, I_off: torch.Tensor, omega: torch.Tensor, seeds, wlo, whi,
              batch: Batch, axes: torch.Tensor, label=None, grainR=None, grainX=None, stream=None):
    """Seed-conditioned sets of spots p4 (n, 4) sorted by angle (I_off)."""
    import ctypes
    n_angles = omega.numel()
    g = api.geometry_struct(geom)
    rc = h.L.laue_lp_sets(h.h, ctypes.byref(g), api._ptr(p4), api._ptr(I_off), api._ptr(omega), n_angles, p4.shape[0],
                          api._ptr(seeds), api._ptr(wlo), api._ptr(whi), batch.n, api._ptr(label), api._ptr(grainR),
                          api._ptr(grainX), api._ptr(axes), api._ptr(batch.buf), api._ptr(batch.ids),
                          api._stream(stream))
    h.check(rc, "lp_sets")


def forward(h: api.Handle, net: Network, batch: Batch, stream=None):
    h.check(h.L.laue_lp_forward(h.h, api._ptr(net.buf), api._ptr(batch.buf), batch.n, api._stream(stream)),
            "lp_forward")
    return batch.outputs()


def train_step(h: api.Handle, net: Network, batch: Batch, lr: float, stream=None):
    h.check(h.L.laue_lp_train_step(h.h, api._ptr(net.buf), api._ptr(batch.buf), batch.n, float(lr),
                                   api._stream(stream)), "lp_train_step")


def decode(h: api.Handle, batch: Batch, stream=None):
    """Proposals (n_sets * 8, 9) rotations and (n_sets * 8, 3) positions."""
    R = torch.empty(batch.n * NHYP, 9, dtype=torch.float32, device=h.device)
    x = torch.empty(batch.n * NHYP, 3, dtype=torch.float32, device=h.device)
    h.check(h.L.laue_lp_decode(h.h, api._ptr(batch.buf), batch.n, api._ptr(R), api._ptr(x), api._stream(stream)),
            "lp_decode")
    return R, x


class Scenes:
    """Device buffers of a batch of training scenes (S scenes of W angles,
    at most Gmax grains each) and of their seeds."""

    def __init__(self, h: api.Handle, S: int, W: int, Gmax: int, per_scene: int, capacity: int):
        dev = h.device
        if h.ws is None:
            h.reserve(1)
        self.h, self.S, self.W, self.Gmax, self.per_scene, self.capacity = h, S, W, Gmax, per_scene, capacity
        self.grainR = torch.empty(S * Gmax, 9, dtype=torch.float32, device=dev)
        self.grainX = torch.empty(S * Gmax, 3, dtype=torch.float32, device=dev)
        self.scene_i32 = torch.empty(4 * S * W + 2 * S, dtype=torch.int32, device=dev)
        self.I_off = torch.empty(S * W + 1, dtype=torch.int32, device=dev)
        self.omega_v = torch.empty(S * W, dtype=torch.float32, device=dev)
        self.p4 = torch.empty(capacity, 4, dtype=torch.float32, device=dev)
        self.label = torch.empty(capacity, dtype=torch.int32, device=dev)
        self.axes = torch.empty(capacity, 4, dtype=torch.float32, device=dev)
        B = S * per_scene
        self.seeds = torch.empty(B, dtype=torch.int32, device=dev)
        self.wlo = torch.empty(B, dtype=torch.int32, device=dev)
        self.whi = torch.empty(B, dtype=torch.int32, device=dev)

    def generate(self, geom, lat: api.Lattice, omega: torch.Tensor, seed: int, gmin: int, gmax: int,
                 cube_mm=5.0, sigma_mm=0.5, outlier_ratio=0.7, stream=None):
        import ctypes
        h = self.h
        g = api.geometry_struct(geom)
        ls = lat.struct()
        rc = h.L.laue_lp_scene(h.h, ctypes.byref(g), ctypes.byref(ls), api._ptr(omega), omega.numel(), self.W, self.S, self.Gmax, gmin,
                               gmax, float(cube_mm), float(sigma_mm), float(outlier_ratio), int(seed),
                               api._ptr(self.grainR), api._ptr(self.grainX), api._ptr(self.scene_i32),
                               api._ptr(self.I_off), api._ptr(self.omega_v), api._ptr(self.p4), api._ptr(self.label),
                               self.capacity, api._stream(stream))
        h.check(rc, "lp_scene")
        rc = h.L.laue_lp_scene_seeds(h.h, api._ptr(self.I_off), api._ptr(self.label), self.W, self.S,
                                     self.per_scene, int(seed), api._ptr(self.seeds), api._ptr(self.wlo),
                                     api._ptr(self.whi), api._stream(stream))
        h.check(rc, "lp_scene_seeds")

    def sets(self, geom, batch: Batch, stream=None):
        make_sets(self.h, geom, self.p4, self.I_off, self.omega_v, self.seeds, self.wlo, self.whi, batch, self.axes,
                  label=self.label, grainR=self.grainR, grainX=self.grainX, stream=stream)


def propose(h: api.Handle, net: Network, geom, obs: api.ObsSpots, omega: torch.Tensor, seeds, window: int = 10,
            batch: Batch | None = None, stream=None):
    """Candidate poses from the set encoder: for each seed spot (indices into
    obs, chosen by the caller) the set of its window of `window` rotation
    angles starting window//2 - 1 before the seed's angle (clipped to the
    scan), the network's 8 hypotheses decoded to (R, x).  Returns R (n*8, 9)
    and x (n*8, 3) on the device."""
    import numpy as np
    dev = h.device
    seeds = np.asarray(seeds, np.int64)
    I_off = obs.I_off.cpu().numpy().astype(np.int64)
    T = len(I_off) - 1
    t = np.searchsorted(I_off, seeds, side="right") - 1
    lo = np.clip(t - (window // 2 - 1), 0, T)
    hi = np.clip(lo + window, 0, T)
    lo = np.clip(hi - window, 0, T)
    n = len(seeds)
    if batch is None or batch.n != n:
        batch = Batch(h, n)
    ti = lambda a: torch.tensor(a, dtype=torch.int32, device=dev)
    axes = torch.empty(obs.p.shape[0], 4, dtype=torch.float32, device=dev)
    make_sets(h, geom, obs.p, obs.I_off, omega, ti(seeds), ti(lo), ti(hi), batch, axes, stream=stream)
    forward(h, net, batch, stream=stream)
    return decode(h, batch, stream=stream)


def train(h: api.Handle, geom, lat: api.Lattice, omega: torch.Tensor, steps: int, gmin: int = 1, gmax: int = 1,
          S: int = 64, per_scene: int = 32, W: int = 10, lr: float = 1e-3, seed: int = 0, net: Network | None = None,
          cube_mm: float = 5.0, sigma_mm: float = 0.5, outlier_ratio: float = 0.7, stream=None):
    """Trains the set encoder on scenes the forward model simulates: every
    step draws S fresh scenes of gmin..gmax grains (Philox keyed by seed and
    step), builds per_scene seed-conditioned sets per scene and takes one
    Adam step with a cosine-decayed learning rate.  Returns the network."""
    import math
    net = net if net is not None else Network(h, seed=seed, stream=stream)
    cap = S * W * (max(gmax, 1) * 48 + 64)
    sc = Scenes(h, S, W, max(gmax, 1), per_scene, cap)
    batch = Batch(h, S * per_scene)
    for it in range(steps):
        lr_t = lr * 0.5 * (1.0 + math.cos(math.pi * it / max(steps, 1)))
        sc.generate(geom, lat, omega, (int(seed) << 32) + it + 1, gmin, gmax, cube_mm, sigma_mm, outlier_ratio,
                    stream=stream)
        sc.sets(geom, batch, stream=stream)
        train_step(h, net, batch, lr_t, stream=stream)
    return net
