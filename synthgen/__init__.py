"""Seeded synthetic inputs for the LaueOT hot path.

This module is shared by the tests, the benchmark and the oracle's callers.  It
holds no arithmetic of the indexing method: it only draws random numbers, holds
the experiment configurations, and assembles observed-spot lists out of true
spot positions that a forward model (either one) has already produced.

Workload shapes follow the paper's simulations (Section "Simulations and
experiments": white beam, two flat detectors, rotation about one axis, Gaussian
spot noise, uniform outliers) with the sizes of the configurations below.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


@dataclasses.dataclass(frozen=True)
class Detector:
    """Flat square detector: centre (mm), plane normal, half side (mm) and
    cost length D (mm; 0 takes the geometry's D).  Its in-plane axes are
    a1 = (y x n)/|y x n| (x when n is along y) and a2 = n x a1, and it holds
    the plane points s with |(s - centre).a| < half for both axes."""

    centre: tuple
    normal: tuple
    half: float
    D: float = 0.0

    def axes(self):
        n = np.asarray(self.normal, np.float64)
        n = n / np.linalg.norm(n)
        a1 = np.array([n[2], 0.0, -n[0]])
        a1 = a1 / np.linalg.norm(a1) if np.linalg.norm(a1) > 1e-12 else np.array([1.0, 0.0, 0.0])
        return a1, np.cross(n, a1)


def tilted_geometry():
    """Two detectors at the distances of the paper's CoNiGa tomography
    (backscatter at 165 mm, transmission at 125 mm), the backscatter plane
    tilted by 8 degrees about x and the transmission plane offset 10 mm along
    x; each detector's cost length is its distance."""
    a = math.radians(8.0)
    return Geometry(D=165.0, detectors=(
        Detector((10.0, 0.0, 125.0), (0.0, 0.0, 1.0), 128.0, 125.0),
        Detector((0.0, 165.0 * math.sin(a), -165.0 * math.cos(a)), (0.0, -math.sin(a), math.cos(a)), 128.0, 165.0),
    ))


@dataclasses.dataclass(frozen=True)
class Geometry:
    """Beam direction, wavelength band (Angstrom), cost length scale D (mm) and
    flat square detectors.  Default: beam +z, band [1, 4], transmission detector
    at z=+200 mm (index 0) and backscatter detector at z=-200 mm (index 1),
    both 256 x 256 mm."""

    beam: tuple = (0.0, 0.0, 1.0)
    lam_min: float = 1.0
    lam_max: float = 4.0
    D: float = 200.0
    detectors: tuple = (
        Detector((0.0, 0.0, 200.0), (0.0, 0.0, 1.0), 128.0),
        Detector((0.0, 0.0, -200.0), (0.0, 0.0, 1.0), 128.0),
    )


@dataclasses.dataclass(frozen=True)
class Config:
    name: str
    n_grains: int
    hmax: int
    T: int
    span_deg: float
    sigma_mm: float
    outlier_frac: float
    outlier_mode: str = "uniform"  # or "poisson_uneven"
    a: float = 2.87                 # cubic lattice constant (Angstrom)
    centering: int = 1              # 0 = P, 1 = I (h+k+l even), 2 = F
    cube_mm: float = 5.0
    eps: float = 1.0                # final entropic temperature (mm^2)
    n_sinkhorn: int = 100
    n_em: int = 20
    n_orient_scan: int = 5000
    n_pos_scan: int = 125
    seed: int = 0


CONFIGS = {
    # 5 grains, |hkl| <= 4, 10 rotations over 180 deg, 10% outliers
    "tiny": Config("tiny", 5, 4, 10, 180.0, 0.5, 0.10, n_sinkhorn=100, n_em=20,
                   n_orient_scan=5000, n_pos_scan=125),
    # 100 grains, |hkl| <= 6, 60 rotations over 360 deg, 30% outliers
    "medium": Config("medium", 100, 6, 60, 360.0, 0.5, 0.30, n_sinkhorn=200, n_em=30,
                     n_orient_scan=200000, n_pos_scan=512),
    # 1000 grains, 90 rotations over 360 deg, 70% outliers, uneven per angle
    "batched": Config("batched", 1000, 6, 90, 360.0, 0.5, 0.70, outlier_mode="poisson_uneven",
                      n_sinkhorn=200, n_em=30),
    # gradient check: 50 grains, 20 rotations
    "adjoint": Config("adjoint", 50, 6, 20, 360.0, 0.5, 0.30, n_sinkhorn=100, n_em=20),
}


@dataclasses.dataclass(frozen=True)
class Cell:
    """Unit cell (Angstrom, degrees)."""
    a: float
    b: float
    c: float
    alpha: float
    beta: float
    gamma: float


# Ruby (corundum, space group R-3c) in its hexagonal setting
RUBY = Cell(4.759, 4.759, 12.991, 90.0, 90.0, 120.0)


def ruby_hkl(hmax: int = 4, lmax: int = 12) -> np.ndarray:
    """Reflections (h, k, l) with |h|, |k|, |h + k| <= hmax (the bound on the
    three hexagonal a-axis indices, which the crystal's rotations permute) and
    |l| <= lmax, allowed by the reflection conditions of R-3c on hexagonal
    axes: -h + k + l divisible by 3 (rhombohedral centring), and l even on the
    three zones with one a-axis index zero (h = 0, k = 0 or h + k = 0: the c
    glides that the 3-fold axis relates).  Input data of the crystal, not part
    of the indexing method."""
    out = []
    for h in range(-hmax, hmax + 1):
        for k in range(-hmax, hmax + 1):
            if abs(h + k) > hmax:
                continue
            for l in range(-lmax, lmax + 1):
                if h == 0 and k == 0 and l == 0:
                    continue
                if (-h + k + l) % 3 != 0:
                    continue
                if (h == 0 or k == 0 or h + k == 0) and l % 2 != 0:
                    continue
                out.append((h, k, l))
    return np.array(out, np.int32)


def bcc_hkl(hmax: int) -> np.ndarray:
    """Reflections of a body-centred cubic lattice, |h|, |k|, |l| <= hmax, h+k+l even."""
    r = range(-hmax, hmax + 1)
    return np.array([(h, k, l) for h in r for k in r for l in r
                     if (h, k, l) != (0, 0, 0) and (h + k + l) % 2 == 0], np.int32)


def omegas(cfg: Config) -> np.ndarray:
    """Rotation angles omega_t = t * span / T (radians)."""
    return np.radians(cfg.span_deg) * np.arange(cfg.T, dtype=np.float64) / cfg.T


def quat_to_matrix(q: np.ndarray) -> np.ndarray:
    """Unit quaternions (w, x, y, z) -> rotation matrices (n, 3, 3)."""
    q = np.asarray(q, dtype=np.float64)
    q = q / np.linalg.norm(q, axis=-1, keepdims=True)
    w, x, y, z = q[..., 0], q[..., 1], q[..., 2], q[..., 3]
    R = np.empty(q.shape[:-1] + (3, 3))
    R[..., 0, 0] = 1 - 2 * (y * y + z * z)
    R[..., 0, 1] = 2 * (x * y - w * z)
    R[..., 0, 2] = 2 * (x * z + w * y)
    R[..., 1, 0] = 2 * (x * y + w * z)
    R[..., 1, 1] = 1 - 2 * (x * x + z * z)
    R[..., 1, 2] = 2 * (y * z - w * x)
    R[..., 2, 0] = 2 * (x * z - w * y)
    R[..., 2, 1] = 2 * (y * z + w * x)
    R[..., 2, 2] = 1 - 2 * (x * x + y * y)
    return R


def random_rotations(n: int, rng: np.random.Generator) -> np.ndarray:
    """Uniform rotations on SO(3) (Shoemake's subgroup algorithm)."""
    u1, u2, u3 = rng.random((3, n))
    a, b = np.sqrt(1 - u1), np.sqrt(u1)
    q = np.stack([a * np.sin(2 * np.pi * u2), a * np.cos(2 * np.pi * u2),
                  b * np.sin(2 * np.pi * u3), b * np.cos(2 * np.pi * u3)], axis=-1)
    return quat_to_matrix(q)


def random_grains(cfg: Config, rng: np.random.Generator):
    """Orientations uniform on SO(3), positions uniform in a cube centred at 0."""
    R = random_rotations(cfg.n_grains, rng)
    x = rng.uniform(-cfg.cube_mm / 2, cfg.cube_mm / 2, size=(cfg.n_grains, 3))
    return R, x


def super_fibonacci(n: int) -> np.ndarray:
    """Deterministic quasi-uniform rotations: the super-Fibonacci spiral of
    Alexa (CVPR 2022), returned as (n, 3, 3) matrices."""
    phi = math.sqrt(2.0)
    psi = 1.533751168755204288118041  # real root of psi^4 = psi + 4
    s = np.arange(n, dtype=np.float64) + 0.5
    r = np.sqrt(s / n)
    Rr = np.sqrt(1.0 - s / n)
    alpha = 2 * np.pi * s / phi
    beta = 2 * np.pi * s / psi
    q = np.stack([r * np.sin(alpha), r * np.cos(alpha), Rr * np.sin(beta), Rr * np.cos(beta)], -1)
    return quat_to_matrix(q)


def position_grid(k: int, cube_mm: float) -> np.ndarray:
    """k^3 cell-centred lattice over the sample cube."""
    c = (np.arange(k) + 0.5) / k * cube_mm - cube_mm / 2
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()], -1)


@dataclasses.dataclass
class Observed:
    """Observed spots sorted by angle: p (I, 3) mm, t (I,), det (I,),
    truth (I,) index of the true spot it came from or -1 for an outlier,
    I_off (T+1,)."""

    p: np.ndarray
    t: np.ndarray
    det: np.ndarray
    truth: np.ndarray
    I_off: np.ndarray


def observe(geom: Geometry, cfg: Config, t_true, det_true, s_true, rng: np.random.Generator,
            sigma_mm: float | None = None, outlier_frac: float | None = None) -> Observed:
    """Detected spots from true spot positions: iid N(0, sigma^2) noise on the
    detector's x and y, spots pushed off the detector dropped, outliers uniform
    on a uniformly chosen detector's square.  Outlier counts: 'uniform' draws
    round(f * #true) outliers over uniformly chosen angles; 'poisson_uneven'
    draws per angle a Poisson count of mean f * |true_t| * m_t / 1.25 with
    m_t ~ U(0.5, 2).  Within an angle the spot order is a random permutation."""
    sigma = cfg.sigma_mm if sigma_mm is None else sigma_mm
    frac = cfg.outlier_frac if outlier_frac is None else outlier_frac
    t_true = np.asarray(t_true, dtype=np.int64)
    det_true = np.asarray(det_true, dtype=np.int64)
    s_true = np.asarray(s_true, dtype=np.float64).reshape(-1, 3)
    n_true = len(t_true)
    z = rng.standard_normal((n_true, 2))
    ax = [d.axes() for d in geom.detectors]
    A1 = np.array([ax[k][0] for k in det_true]).reshape(-1, 3)
    A2 = np.array([ax[k][1] for k in det_true]).reshape(-1, 3)
    ctr = np.array([geom.detectors[k].centre for k in det_true], np.float64).reshape(-1, 3)
    p = s_true + sigma * (z[:, :1] * A1 + z[:, 1:] * A2)
    half = np.array([geom.detectors[k].half for k in det_true]) if n_true else np.zeros(0)
    keep = ((np.abs(np.sum((p - ctr) * A1, 1)) < half) & (np.abs(np.sum((p - ctr) * A2, 1)) < half)
            if n_true else np.zeros(0, bool))
    p, t_in, d_in = p[keep], t_true[keep], det_true[keep]
    truth = np.nonzero(keep)[0]
    T = cfg.T
    if cfg.outlier_mode == "poisson_uneven":
        per_t = np.bincount(t_true, minlength=T).astype(np.float64)
        m_t = rng.uniform(0.5, 2.0, size=T)
        counts = rng.poisson(frac * per_t * m_t / 1.25)
        t_out = np.repeat(np.arange(T), counts)
    else:
        n_out = int(round(frac * n_true))
        t_out = rng.integers(0, T, size=n_out)
    n_out = len(t_out)
    d_out = rng.integers(0, len(geom.detectors), size=n_out)
    uv = rng.uniform(-1.0, 1.0, size=(n_out, 2))
    p_out = np.zeros((n_out, 3))
    for k, det in enumerate(geom.detectors):
        sel = d_out == k
        a1, a2 = ax[k]
        p_out[sel] = (np.asarray(det.centre, np.float64) + det.half * uv[sel, :1] * a1 +
                      det.half * uv[sel, 1:] * a2)
    P = np.concatenate([p, p_out])
    Tt = np.concatenate([t_in, t_out]).astype(np.int64)
    Dd = np.concatenate([d_in, d_out]).astype(np.int64)
    truth = np.concatenate([truth, -np.ones(n_out, np.int64)])
    key = rng.permutation(len(P))
    order = key[np.argsort(Tt[key], kind="stable")]
    I_off = np.zeros(T + 1, np.int64)
    np.cumsum(np.bincount(Tt, minlength=T), out=I_off[1:])
    return Observed(P[order], Tt[order], Dd[order], truth[order], I_off)


def workload_seed(cfg: Config, repeat: int = 0) -> np.random.Generator:
    """Generator for a configuration: seed 0 for the data, 1, 2, 3 for repeats."""
    return np.random.default_rng(cfg.seed + repeat)
