"""FP64 oracle of the learned proposal: a set encoder that maps a
seed-conditioned set of observed spots to candidate grain poses.

TEST INFRASTRUCTURE, NOT PRODUCT CODE: only the tests, the smoke check and the
benchmark's CPU-baseline leg import this module.  It shares no code with the
CUDA path.

The paper has no learned component.  This network is an addition beside the
paper's candidate scan (Section "Pre-processing", single-grain fits from a
grid of starts), which stays both its fallback and the measure of its recall.
What it computes is fixed here, in plain numpy:

* Spot axes.  A spot p recorded at rotation angle omega_t is read as a ray
  from a grain at the origin: rhat = p / |p|.  Bragg reflection off a plane
  with unit normal u turns the beam e into r = e - 2 (u.e) u (Eq. ray_mnt), so
  u is parallel to r - e; the sample-frame axis is n = Gamma_t^T u with Gamma_t
  the rotation about +y (Section "Forward model").  For a grain at the origin
  and no noise, n = +-R w_m exactly: the plane normal of the reflection.
* Seed-conditioned sets.  A seed spot i0 with axis n0 and the KSET-1 spots of
  its rotation window whose axes are closest to n0 (distance 1 - |n.n0|, ties
  by index), described in the seed frame F0 = [n0, a1, n0 x a1] where a1 is
  the unit part of +y orthogonal to n0.
* The network.  A per-spot MLP of three 256-wide ReLU layers, masked mean and
  max pooling over the set, a two-layer head that emits NHYP hypotheses of
  (6-D rotation, 3-D position).  The 6-D output is turned into a rotation by
  Gram-Schmidt.  Every layer (the per-spot layers and the head) is BF16 with
  FP32 accumulation on the GPU; with ``bf16=True`` this oracle rounds the
  same operands (all weights, the per-spot activations, the pooled features,
  the head's hidden activations and the back-propagated errors the GEMMs
  read) to BF16 and accumulates in FP64.
* The loss.  Per set and hypothesis the cubic-symmetry-aware rotation error
  min_S ||Rhat - R_loc S||_F^2 (S over the 24 proper rotations of the cube,
  R_loc = F0^T R) plus LAMBDA_X ||xhat - x / XSCALE||^2; the set loss is the
  best hypothesis plus BETA times the mean over hypotheses.
* Adam (Kingma and Ba, 2015) with bias correction.
* Philox4x32-10 (Salmon, Moraes, Dror and Shaw, SC'11), the counter-based
  generator that draws the noise, outliers and seeds of a training scene.

Parity of the network is unpinned against the paper (the paper has no such
network); the pins in the tests tie it to finite differences, closed forms,
invariants and published known-answer vectors.
"""
from __future__ import annotations

import itertools
import math

import numpy as np

KSET = 128          # spots per set: the seed + 127 neighbours
NF = 64             # feature width (14 used, the rest zero)
WIDTH = 256         # per-spot MLP width
HEAD = 256          # head hidden width
NHYP = 8            # hypotheses per set
NOUT = 9 * NHYP
XSCALE = 2.5        # position scale (mm): half the sample cube
LAMBDA_X = 0.1
BETA = 0.05
DSCALE = 200.0      # detector-distance scale of the features (mm)
HALF = 128.0        # detector half-width scale of the features (mm)


# ------------------------------------------------------------------ BF16
def bf16(a):
    """Round to the nearest BF16 value (ties to even), returned as float64."""
    f = np.ascontiguousarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    out = r.astype(np.uint32).view(np.float32)
    nan = np.isnan(f)
    if nan.any():
        out = np.where(nan, f, out)
    return out.astype(np.float64)


# ------------------------------------------------------------------ geometry
def cubic_group():
    """The 24 proper rotations of the cube (signed permutation matrices, det +1)."""
    out = []
    for perm in itertools.permutations(range(3)):
        for sgn in itertools.product([1, -1], repeat=3):
            S = np.zeros((3, 3))
            for r, c in enumerate(perm):
                S[r, c] = sgn[r]
            if np.linalg.det(S) > 0:
                out.append(S)
    return np.array(out)


def spot_axes(p, t, omega, beam=(0.0, 0.0, 1.0)):
    """Sample-frame axes (n, 3) of spots p (n, 3) at angle indices t."""
    p = np.asarray(p, np.float64).reshape(-1, 3)
    e = np.asarray(beam, np.float64)
    r = p / np.linalg.norm(p, axis=1, keepdims=True)
    u = r - e
    nu = np.linalg.norm(u, axis=1, keepdims=True)
    bad = nu[:, 0] < 1e-9
    u = u / np.where(nu > 0, nu, 1.0)
    u[bad] = (1.0, 0.0, 0.0)
    w = np.asarray(omega, np.float64)[np.asarray(t)]
    c, s = np.cos(w), np.sin(w)
    # lab = Gamma sample with Gamma = [[c, 0, s], [0, 1, 0], [-s, 0, c]]
    return np.stack([c * u[:, 0] - s * u[:, 2], u[:, 1], s * u[:, 0] + c * u[:, 2]], 1)


def seed_frame(n0):
    """Columns n0, a1 (the part of +y orthogonal to n0, or of +x if n0 ~ y), n0 x a1."""
    n0 = np.asarray(n0, np.float64)
    y = np.array([0.0, 1.0, 0.0])
    a1 = y - (y @ n0) * n0
    if np.linalg.norm(a1) < 1e-6:
        x = np.array([1.0, 0.0, 0.0])
        a1 = x - (x @ n0) * n0
    a1 /= np.linalg.norm(a1)
    return np.stack([n0, a1, np.cross(n0, a1)], 1)


def make_sets(p, t, omega, seeds, wlo, whi, beam=(0.0, 0.0, 1.0)):
    """Seed-conditioned sets.

    p (n, 3) spots, t (n,) angle indices, omega (T,) radians, seeds (B,)
    spot indices (or -1: an empty set), wlo/whi (B,) the angle window
    [wlo, whi) of each seed.  Returns X (B, KSET, NF) features, ids (B, KSET)
    spot indices (-1 for padding) and F (B, 3, 3) seed frames.

    Features of element i (seed first, then neighbours by distance):
      0-2  sign(n.n0) F0^T n      3-4  sin, cos of omega_i - omega_0
      5    p_z / 200              6-7  p_x / 128, p_y / 128
      8-10 the seed's p / (128, 128, 200)
      11   1 for the seed         12   1 for a valid element
      13   (t_i - t_0) / 10
    """
    p = np.asarray(p, np.float64).reshape(-1, 3)
    t = np.asarray(t, np.int64)
    n = spot_axes(p, t, omega, beam)
    B = len(seeds)
    X = np.zeros((B, KSET, NF))
    ids = -np.ones((B, KSET), np.int64)
    F = np.zeros((B, 3, 3))
    for b, i0 in enumerate(seeds):
        if i0 < 0:
            continue
        F0 = seed_frame(n[i0])
        F[b] = F0
        cand = np.nonzero((t >= wlo[b]) & (t < whi[b]))[0]
        cand = cand[cand != i0]
        d = 1.0 - np.abs(n[cand] @ n[i0])
        order = np.lexsort((cand, d))[:KSET - 1]
        sel = np.concatenate([[i0], cand[order]])
        ids[b, :len(sel)] = sel
        v = n[sel] @ F0
        sgn = np.where(n[sel] @ n[i0] < 0.0, -1.0, 1.0)
        v *= sgn[:, None]
        w0 = omega[t[i0]]
        dw = np.asarray(omega)[t[sel]] - w0
        k = len(sel)
        X[b, :k, 0:3] = v
        X[b, :k, 3] = np.sin(dw)
        X[b, :k, 4] = np.cos(dw)
        X[b, :k, 5] = p[sel, 2] / DSCALE
        X[b, :k, 6] = p[sel, 0] / HALF
        X[b, :k, 7] = p[sel, 1] / HALF
        X[b, :k, 8] = p[i0, 0] / HALF
        X[b, :k, 9] = p[i0, 1] / HALF
        X[b, :k, 10] = p[i0, 2] / DSCALE
        X[b, 0, 11] = 1.0
        X[b, :k, 12] = 1.0
        X[b, :k, 13] = (t[sel] - t[i0]) / 10.0
    return X, ids, F


def set_targets(F, R, x):
    """Targets of the sets: R_loc = F0^T R (B, 3, 3) and x / XSCALE (B, 3)."""
    return np.einsum("bji,bjk->bik", F, R), np.asarray(x) / XSCALE


# ------------------------------------------------------------------ network
PARAM_SHAPES = [("W1", (WIDTH, NF)), ("b1", (WIDTH,)), ("W2", (WIDTH, WIDTH)), ("b2", (WIDTH,)),
                ("W3", (WIDTH, WIDTH)), ("b3", (WIDTH,)), ("W4", (HEAD, 2 * WIDTH)), ("b4", (HEAD,)),
                ("W5", (NOUT, HEAD)), ("b5", (NOUT,))]
BF16_WEIGHTS = ("W1", "W2", "W3", "W4", "W5")  # BF16 operands on the GPU


def init_params(rng):
    """He-normal weights for the ReLU layers, 1/fan_in variance for the output
    layer, zero biases; FP32-representable values."""
    P = {}
    for name, shape in PARAM_SHAPES:
        if name.startswith("b"):
            P[name] = np.zeros(shape)
        else:
            gain = 1.0 if name == "W5" else 2.0
            w = rng.standard_normal(shape) * math.sqrt(gain / shape[1])
            P[name] = w.astype(np.float32).astype(np.float64)
    return P


def _relu(z):
    return np.maximum(z, 0.0)


def forward(P, X, bf16_ops=True):
    """Network forward over sets X (B, KSET, NF).  Returns (O (B, NOUT), cache)."""
    rnd = bf16 if bf16_ops else (lambda a: np.asarray(a, np.float64))
    B = X.shape[0]
    valid = X[:, :, 12] > 0.5
    x0 = rnd(X.reshape(B * KSET, NF))
    W = {k: (rnd(P[k]) if k in BF16_WEIGHTS else P[k]) for k in P}
    Z1 = x0 @ W["W1"].T + P["b1"]
    H1 = rnd(_relu(Z1))
    Z2 = H1 @ W["W2"].T + P["b2"]
    H2 = rnd(_relu(Z2))
    Z3 = H2 @ W["W3"].T + P["b3"]
    H3 = rnd(_relu(Z3))
    H3s = H3.reshape(B, KSET, WIDTH)
    nv = valid.sum(1)
    mean = (H3s * valid[:, :, None]).sum(1) / np.maximum(nv, 1)[:, None]
    masked = np.where(valid[:, :, None], H3s, -np.inf)
    amax = np.argmax(masked, axis=1)  # first index on ties
    mx = np.take_along_axis(H3s, amax[:, None, :], 1)[:, 0, :]
    mx = np.where(nv[:, None] > 0, mx, 0.0)
    Pool = rnd(np.concatenate([mean, mx], 1))
    Z4 = Pool @ W["W4"].T + P["b4"]
    H4 = rnd(_relu(Z4))
    O = H4 @ W["W5"].T + P["b5"]
    cache = dict(x0=x0, W=W, H1=H1, H2=H2, H3=H3, valid=valid, nv=nv, amax=amax, Pool=Pool, Z4=Z4, H4=H4,
                 bf16_ops=bf16_ops)
    return O, cache


def gram_schmidt(o6):
    """Rotation (..., 3, 3) with columns e1 = a/|a|, e2 = unit part of b
    orthogonal to e1, e3 = e1 x e2, from o6 = (a, b)."""
    a, b = o6[..., 0:3], o6[..., 3:6]
    e1 = a / np.linalg.norm(a, axis=-1, keepdims=True)
    bp = b - (e1 * b).sum(-1, keepdims=True) * e1
    e2 = bp / np.linalg.norm(bp, axis=-1, keepdims=True)
    return np.stack([e1, e2, np.cross(e1, e2)], -1)


def gram_schmidt_backward(o6, dR):
    """Gradient with respect to o6 of <dR, gram_schmidt(o6)>."""
    a, b = o6[..., 0:3], o6[..., 3:6]
    na = np.linalg.norm(a, axis=-1, keepdims=True)
    e1 = a / na
    eb = (e1 * b).sum(-1, keepdims=True)
    bp = b - eb * e1
    nb = np.linalg.norm(bp, axis=-1, keepdims=True)
    e2 = bp / nb
    de1, de2, de3 = dR[..., :, 0], dR[..., :, 1], dR[..., :, 2]
    de1 = de1 + np.cross(e2, de3)
    de2 = de2 + np.cross(de3, e1)
    dbp = (de2 - (de2 * e2).sum(-1, keepdims=True) * e2) / nb
    db = dbp - (e1 * dbp).sum(-1, keepdims=True) * e1
    de1 = de1 - eb * dbp - (e1 * dbp).sum(-1, keepdims=True) * b
    da = (de1 - (de1 * e1).sum(-1, keepdims=True) * e1) / na
    return np.concatenate([da, db], -1)


_SYM = cubic_group()


def set_loss(O, Rloc, xt, set_valid):
    """Mean over valid sets of min_h L_h + BETA mean_h L_h; returns (loss,
    dO, per-set best rotation error d (B,), best hypothesis (B,))."""
    B = O.shape[0]
    Oh = O.reshape(B, NHYP, 9)
    Rh = gram_schmidt(Oh[..., :6])                       # B,H,3,3
    RS = np.einsum("bij,sjk->bsik", Rloc, _SYM)           # B,24,3,3
    tr = np.einsum("bhij,bsij->bhs", Rh, RS)              # B,H,24
    sbest = np.argmax(tr, axis=2)                         # first on ties
    d = 6.0 - 2.0 * np.take_along_axis(tr, sbest[..., None], 2)[..., 0]
    dxv = Oh[..., 6:9] - xt[:, None, :]
    L = d + LAMBDA_X * (dxv ** 2).sum(-1)
    hbest = np.argmin(L, axis=1)
    Lset = L[np.arange(B), hbest] + BETA * L.mean(1)
    nval = max(int(set_valid.sum()), 1)
    loss = float((Lset * set_valid).sum() / nval)
    coef = np.full((B, NHYP), BETA / NHYP)
    coef[np.arange(B), hbest] += 1.0
    coef *= (set_valid / nval)[:, None]
    Sb = RS[np.arange(B)[:, None], sbest]                 # B,H,3,3
    dR = 2.0 * (Rh - Sb) * coef[..., None, None]
    do6 = gram_schmidt_backward(Oh[..., :6], dR)
    dx = 2.0 * LAMBDA_X * dxv * coef[..., None]
    dO = np.concatenate([do6, dx], -1).reshape(B, NOUT)
    return loss, dO, d[np.arange(B), hbest], hbest


def backward(P, cache, dO):
    """Gradients of all parameters given dL/dO.  With bf16 operands the
    back-propagated errors that a GEMM reads are rounded to BF16 (as the GPU
    stores them; the output bias takes dL/dO unrounded) and every product
    accumulates in FP64."""
    rnd = bf16 if cache["bf16_ops"] else (lambda a: np.asarray(a, np.float64))
    W = cache["W"]
    G = {}
    H4, Z4, Pool = cache["H4"], cache["Z4"], cache["Pool"]
    dOr = rnd(dO)
    G["W5"] = dOr.T @ H4
    G["b5"] = dO.sum(0)
    dZ4 = rnd((dOr @ W["W5"]) * (Z4 > 0))
    G["W4"] = dZ4.T @ Pool
    G["b4"] = dZ4.sum(0)
    dPool = dZ4 @ W["W4"]
    B = dO.shape[0]
    valid, nv, amax = cache["valid"], cache["nv"], cache["amax"]
    dH3 = valid[:, :, None] * (dPool[:, None, :WIDTH] / np.maximum(nv, 1)[:, None, None])
    hasv = nv > 0
    bi, ci = np.nonzero(np.broadcast_to(hasv[:, None], (B, WIDTH)))
    dH3[bi, amax[bi, ci], ci] += dPool[bi, WIDTH + ci]
    dH3 = dH3.reshape(B * KSET, WIDTH)
    H1, H2, H3, x0 = cache["H1"], cache["H2"], cache["H3"], cache["x0"]
    dZ3 = rnd(dH3 * (H3 > 0))
    G["W3"] = dZ3.T @ H2
    G["b3"] = dZ3.sum(0)
    dZ2 = rnd((dZ3 @ W["W3"]) * (H2 > 0))
    G["W2"] = dZ2.T @ H1
    G["b2"] = dZ2.sum(0)
    dZ1 = rnd((dZ2 @ W["W2"]) * (H1 > 0))
    G["W1"] = dZ1.T @ x0
    G["b1"] = dZ1.sum(0)
    return G


def adam(P, G, Mo, Vo, step, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam step (in place) with bias correction; step counts from 1."""
    for k in P:
        Mo[k] = b1 * Mo[k] + (1.0 - b1) * G[k]
        Vo[k] = b2 * Vo[k] + (1.0 - b2) * G[k] ** 2
        mh = Mo[k] / (1.0 - b1 ** step)
        vh = Vo[k] / (1.0 - b2 ** step)
        P[k] = P[k] - lr * mh / (np.sqrt(vh) + eps)


def decode(O, F, xscale=XSCALE):
    """Proposals of the sets: R (B, NHYP, 3, 3) = F0 Rhat and x (B, NHYP, 3)."""
    B = O.shape[0]
    Oh = O.reshape(B, NHYP, 9)
    Rh = gram_schmidt(Oh[..., :6])
    return np.einsum("bij,bhjk->bhik", F, Rh), xscale * Oh[..., 6:9]


# ------------------------------------------------------------------ Philox
_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85


def philox4x32(counter, key):
    """Philox4x32-10 of (4,) uint32 counter words and (2,) key words; arrays
    broadcast over leading dimensions.  Returns (..., 4) uint32."""
    c = [np.asarray(counter[..., i], np.uint64) for i in range(4)]
    k = [np.asarray(key[..., 0], np.uint64), np.asarray(key[..., 1], np.uint64)]
    mask = np.uint64(0xFFFFFFFF)
    for _ in range(10):
        p0 = np.uint64(_M0) * c[0]
        p1 = np.uint64(_M1) * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & mask
        hi1, lo1 = p1 >> np.uint64(32), p1 & mask
        c = [(hi1 ^ c[1] ^ k[0]) & mask, lo1, (hi0 ^ c[3] ^ k[1]) & mask, lo0]
        k = [(k[0] + np.uint64(_W0)) & mask, (k[1] + np.uint64(_W1)) & mask]
    return np.stack(c, -1).astype(np.uint32)


def uniform01(x):
    """(0, 1) uniform from a uint32: (x >> 8 + 0.5) / 2^24."""
    return ((np.asarray(x, np.uint64) >> np.uint64(8)).astype(np.float64) + 0.5) / 16777216.0


def normal_pair(x0, x1):
    """Two standard normals from two uint32 words (Box-Muller on the (0, 1)
    uniforms above)."""
    u1, u2 = uniform01(x0), uniform01(x1)
    rad = np.sqrt(-2.0 * np.log(u1))
    return rad * np.cos(2.0 * math.pi * u2), rad * np.sin(2.0 * math.pi * u2)


TAG_NOISE, TAG_COUNT, TAG_OUTLIER, TAG_SEED, TAG_SCENE, TAG_GRAIN = 0, 1, 2, 3, 4, 5
ALL = 0xFFFFFFFF


def uniform_int(x, n):
    """Integer in [0, n) from a uint32 word: ((x >> 8) n) >> 24 (exact)."""
    return int((int(x) >> 8) * int(n)) >> 24


def shoemake(u1, u2, u3):
    """Uniform rotation from three uniforms (Shoemake, Graphics Gems III,
    1992): q = (sqrt(1-u1) sin 2 pi u2, sqrt(1-u1) cos 2 pi u2,
    sqrt(u1) sin 2 pi u3, sqrt(u1) cos 2 pi u3) as (x, y, z, w)."""
    a, b = math.sqrt(1.0 - u1), math.sqrt(u1)
    qx, qy = a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2)
    qz, qw = b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)
    return np.array([
        [1 - 2 * (qy * qy + qz * qz), 2 * (qx * qy - qz * qw), 2 * (qx * qz + qy * qw)],
        [2 * (qx * qy + qz * qw), 1 - 2 * (qx * qx + qz * qz), 2 * (qy * qz - qx * qw)],
        [2 * (qx * qz - qy * qw), 2 * (qy * qz + qx * qw), 1 - 2 * (qx * qx + qy * qy)]])


def scene_params(S, Gmax, gmin, gmax, T, W, key, cube):
    """Per scene s: window start t0 = uniform_int(word 0, T - W + 1) and grain
    count n_g = gmin + uniform_int(word 1, gmax - gmin + 1) from counter
    (s, ALL, 0, TAG_SCENE); per grain g < Gmax: R = shoemake of words 0-2 of
    (s, g, 0, TAG_GRAIN), x = cube (u - 1/2) from words 0-2 of
    (s, g, 1, TAG_GRAIN)."""
    key = np.asarray(key, np.uint32)
    t0 = np.zeros(S, np.int64)
    n_g = np.zeros(S, np.int64)
    R = np.zeros((S, Gmax, 3, 3))
    x = np.zeros((S, Gmax, 3))
    for s in range(S):
        w = philox4x32(np.array([s, ALL, 0, TAG_SCENE], np.uint32), key)
        t0[s] = uniform_int(w[0], T - W + 1)
        n_g[s] = gmin + uniform_int(w[1], gmax - gmin + 1)
        for g in range(Gmax):
            wr = philox4x32(np.array([s, g, 0, TAG_GRAIN], np.uint32), key)
            R[s, g] = shoemake(uniform01(wr[0]), uniform01(wr[1]), uniform01(wr[2]))
            wx = philox4x32(np.array([s, g, 1, TAG_GRAIN], np.uint32), key)
            x[s, g] = cube * (uniform01(wx[:3]) - 0.5)
    return t0, n_g, R, x


def training_scene(geom, planes, omega, t0, W, R, x, n_g, key, sigma, outlier_ratio):
    """Training scenes built from the forward model (FP64).  Scene s covers
    the W rotation angles omega[t0[s]:t0[s]+W]: virtual angle v = s W + k
    has omega_v = omega[t0[s] + k] and holds grains R[s, :n_g[s]],
    x[s, :n_g[s]] (R (S, Gmax, 3, 3), x (S, Gmax, 3)).

    At virtual angle v, every spot of the forward model (Eqs. ray_mnt, s_mnt,
    wavelength, model_spot_cut) of grain g and plane m gets detector noise
    sigma * (z1, z2) with (z1, z2) = normal_pair of Philox words 0, 1 of
    counter (v, g, m, TAG_NOISE); spots pushed off their detector are
    dropped.  Then floor(ratio * n_true_v + u) outliers follow (u from word 0
    of (v, ALL, 0, TAG_COUNT)); outlier k takes detector floor(u0 n_det) and
    position centre + half (2 u1 - 1, 2 u2 - 1) from words 0-2 of
    (v, ALL, k, TAG_OUTLIER).  Order: true spots by (g, m), then outliers.
    Returns p (n, 3), label (n,) global grain s Gmax + g or -1, I_off
    (S W + 1,) and omega_v (S W,)."""
    from . import forward as orc_forward
    key = np.asarray(key, np.uint32)
    S, Gmax = R.shape[0], R.shape[1]
    omega_v = np.concatenate([np.asarray(omega)[t0[s]:t0[s] + W] for s in range(S)])
    P, L = [], []
    for v in range(S * W):
        s = v // W
        ng = int(n_g[s])
        if ng > 0:
            f = orc_forward(geom, planes, R[s, :ng].reshape(-1, 9), x[s, :ng], np.array([omega_v[v]]))
            g, m, sp, det = f["grain"], f["plane"], f["spot"], f["det"]
        else:
            g = m = det = np.zeros(0, np.int64)
            sp = np.zeros((0, 3))
        ctr = np.stack([np.full(len(g), v), g, m, np.full(len(g), TAG_NOISE)], 1).astype(np.uint32)
        words = philox4x32(ctr, np.broadcast_to(key, (len(g), 2)))
        z1, z2 = normal_pair(words[:, 0], words[:, 1])
        p = sp.copy()
        p[:, 0] += sigma * z1
        p[:, 1] += sigma * z2
        keep = np.ones(len(p), bool)
        for i in range(len(p)):
            d = geom.detectors[int(det[i])]
            keep[i] = abs(p[i, 0] - d.centre[0]) < d.half and abs(p[i, 1] - d.centre[1]) < d.half
        p, g = p[keep], g[keep]
        cw = philox4x32(np.array([v, ALL, 0, TAG_COUNT], np.uint32), key)
        n_out = int(math.floor(outlier_ratio * len(p) + uniform01(cw[0])))
        po = np.zeros((n_out, 3))
        if n_out:
            ctr = np.stack([np.full(n_out, v), np.full(n_out, ALL), np.arange(n_out),
                            np.full(n_out, TAG_OUTLIER)], 1).astype(np.uint32)
            wo = philox4x32(ctr, np.broadcast_to(key, (n_out, 2)))
            nd = len(geom.detectors)
            dk = np.minimum((uniform01(wo[:, 0]) * nd).astype(np.int64), nd - 1)
            for i in range(n_out):
                d = geom.detectors[int(dk[i])]
                po[i] = (d.centre[0] + d.half * (2.0 * uniform01(wo[i, 1]) - 1.0),
                         d.centre[1] + d.half * (2.0 * uniform01(wo[i, 2]) - 1.0), d.centre[2])
        P.append(np.concatenate([p, po]))
        L.append(np.concatenate([s * Gmax + g, -np.ones(n_out, np.int64)]))
    cnt = np.array([len(a) for a in L])
    I_off = np.concatenate([[0], np.cumsum(cnt)])
    return np.concatenate(P), np.concatenate(L), I_off, omega_v


def scene_seeds(label, I_off, W, per_scene, key, tries=64):
    """Seed of set j of scene s: the first inlier among spots chosen
    uniformly (uniform_int(word 0 of (s, j, q, TAG_SEED), n_s), q = 0, 1,
    ...) within the scene; -1 when none of `tries` draws is an inlier."""
    key = np.asarray(key, np.uint32)
    S = (len(I_off) - 1) // W
    out = -np.ones(S * per_scene, np.int64)
    for s in range(S):
        lo, hi = int(I_off[s * W]), int(I_off[(s + 1) * W])
        ns = hi - lo
        for j in range(per_scene):
            if ns == 0:
                continue
            for q in range(tries):
                w = philox4x32(np.array([s, j, q, TAG_SEED], np.uint32), key)
                i = lo + uniform_int(w[0], ns)
                if label[i] >= 0:
                    out[s * per_scene + j] = i
                    break
    return out


def gemm_tn(A, B, mode=0, bias=None, mask=None, splits=1, round_out=True):
    """Reference of the tensor-core GEMM: D = A B^T in FP64 over the given
    operand values.  mode 0 returns the `splits` partial products over equal
    K ranges (splits, M, N); mode 1 bf16(relu(D + bias)); mode 2
    bf16(D where mask > 0, else 0); round_out=False skips the BF16 rounding."""
    A = np.asarray(A, np.float64)
    B = np.asarray(B, np.float64)
    K = A.shape[1]
    if mode == 0:
        ks = K // splits
        return np.stack([A[:, s * ks:(s + 1) * ks] @ B[:, s * ks:(s + 1) * ks].T for s in range(splits)])
    D = A @ B.T
    rnd = bf16 if round_out else (lambda a: a)
    if mode == 1:
        return rnd(np.maximum(D + np.asarray(bias, np.float64)[None, :], 0.0))
    return rnd(np.where(np.asarray(mask) > 0, D, 0.0))
