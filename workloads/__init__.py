"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module only draws input spectra; it holds none of the correlation
arithmetic.  Every generator works in FP64 with ``numpy.random.default_rng``
and rounds the result to FP32, so the GPU path and the oracle read identical
FP32 arrays.  Stacks are m x n row-major: row j is perturbation step t_j,
column is the spectral variable nu (the layout of the paper's input matrix,
Sec. 3).

The paper's own speed-test data (``sim2ddata``) and its Raman dataset are not
available, so band-shaped synthetic spectra stand in for them:

* ``c1``: m=11, n=500, three Lorentzian bands whose amplitudes are
  a_b sin(2 pi t + phi_b) with lags 0/30/60 degrees, noise sigma 0.01.
* ``c2``: m=64, n=4096, 50 Lorentzian bands with sigmoid amplitude in t
  (random midpoint and slope), constant baseline 10, noise sigma 1e-3.
* ``c3``: m=128, hetero, raw spectra on jittered non-uniform axes ~1.3x denser
  than the 8192 / 2048-point target grids, Gaussian bands; stack-2 amplitudes
  are phase-lagged, correlated copies of stack-1 latent signals.
* ``c4``: m=256, n=32768, the c2 generator with 400 bands.
* ``c5``: 512 problems with m ~ U{8..200}, n1, n2 log-uniform in
  [256, 8192], even indices homo and odd indices hetero.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _lorentz(nu: np.ndarray, c: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Band profiles, one row per band: 1 / (1 + ((nu - c)/g)^2)."""
    return 1.0 / (1.0 + ((nu[None, :] - c[:, None]) / g[:, None]) ** 2)


def _gauss(nu: np.ndarray, c: np.ndarray, w: np.ndarray) -> np.ndarray:
    return np.exp(-((nu[None, :] - c[:, None]) ** 2) / (2.0 * w[:, None] ** 2))


def random_stack(m: int, n: int, seed: int, offset: float = 0.0, scale: float = 1.0) -> np.ndarray:
    """Unstructured N(offset, scale^2) stack, for small edge-case tests."""
    rng = np.random.default_rng(seed)
    return (offset + scale * rng.standard_normal((m, n))).astype(np.float32)


def step_stack(m: int, n: int, seed: int, offset: float = 1.0, noise: float = 1e-3) -> np.ndarray:
    """Every variable jumps once, at a step between m/4 and 3m/4, by a random
    amplitude, plus a little noise.  The discrete Hilbert transform of such a
    step grows like (2/pi) ln m near the jump, so it is larger than the
    dynamic spectrum itself for most variables once m is a few dozen."""
    rng = np.random.default_rng(seed)
    t = np.arange(m)[:, None]
    t0 = rng.integers(m // 4, max(m // 4 + 1, 3 * m // 4), size=n)[None, :]
    amp = rng.uniform(0.5, 2.0, size=n)[None, :] * rng.choice([-1.0, 1.0], size=n)[None, :]
    y = offset + amp * (t >= t0) + noise * rng.standard_normal((m, n))
    return y.astype(np.float32)


def sinusoid_bands(m: int, n: int, phases_deg, seed: int, noise: float = 0.0,
                   centers=None, widths=None, amps=None, one_period: bool = True):
    """Lorentzian bands with amplitudes a_b sin(2 pi t_j + phi_b), t_j = j/m.

    Returns (stack, centers, widths, amps)."""
    rng = np.random.default_rng(seed)
    nb = len(phases_deg)
    nu = np.arange(n, dtype=np.float64)
    c = np.asarray(centers, np.float64) if centers is not None else rng.uniform(0.1 * n, 0.9 * n, nb)
    g = np.asarray(widths, np.float64) if widths is not None else rng.uniform(5, 20, nb)
    a = np.asarray(amps, np.float64) if amps is not None else rng.uniform(0.5, 1.5, nb)
    t = np.arange(m, dtype=np.float64) / (m if one_period else (m - 1))
    ph = np.deg2rad(np.asarray(phases_deg, np.float64))
    amp_t = a[None, :] * np.sin(2 * np.pi * t[:, None] + ph[None, :])  # m x nb
    y = amp_t @ _lorentz(nu, c, g)
    if noise > 0:
        y = y + noise * rng.standard_normal((m, n))
    return y.astype(np.float32), c, g, a


def c1(seed: int = 0) -> np.ndarray:
    """m=11, n=500, three bands with phase lags 0/30/60 deg, noise 0.01."""
    y, _, _, _ = sinusoid_bands(11, 500, [0.0, 30.0, 60.0], seed, noise=0.01,
                                centers=np.random.default_rng(seed + 100).uniform(50, 450, 3))
    return y


def sigmoid_bands(m: int, n: int, nbands: int, seed: int, baseline: float = 10.0,
                  noise: float = 1e-3) -> np.ndarray:
    """Lorentzian bands with sigmoid amplitudes A_b / (1 + exp(-(t - t0_b)/s_b)), t = j/(m-1)."""
    rng = np.random.default_rng(seed)
    nu = np.arange(n, dtype=np.float64)
    c = rng.uniform(0, n, nbands)
    g = rng.uniform(5, 20, nbands)
    A = rng.uniform(0.1, 1.0, nbands)
    t0 = rng.uniform(0.0, 1.0, nbands)
    s = rng.uniform(0.02, 0.2, nbands)
    t = np.arange(m, dtype=np.float64) / (m - 1)
    amp_t = A[None, :] / (1.0 + np.exp(-(t[:, None] - t0[None, :]) / s[None, :]))
    y = amp_t @ _lorentz(nu, c, g) + baseline
    if noise > 0:
        y = y + noise * rng.standard_normal((m, n))
    return y.astype(np.float32)


def c2(seed: int = 1) -> np.ndarray:
    """m=64, n=4096, 50 bands, baseline offset 10, noise 1e-3."""
    return sigmoid_bands(64, 4096, 50, seed)


def c4(seed: int = 3) -> np.ndarray:
    """m=256, n=32768, 400 bands (the c2 generator)."""
    return sigmoid_bands(256, 32768, 400, seed)


@dataclass
class RawHetero:
    """Raw spectra of a hetero pair on non-uniform axes (inputs of the preprocessing step)."""
    x1: np.ndarray
    y1: np.ndarray
    x2: np.ndarray
    y2: np.ndarray
    n1_out: int
    n2_out: int
    alpha: float = 0.5


def jittered_axis(n_raw: int, x_first: float, x_last: float, rng) -> np.ndarray:
    """Strictly increasing axis: uniform grid with U(-0.4h, 0.4h) jitter, endpoints fixed."""
    h = (x_last - x_first) / (n_raw - 1)
    x = x_first + h * np.arange(n_raw, dtype=np.float64)
    x[1:-1] += rng.uniform(-0.4 * h, 0.4 * h, n_raw - 2)
    x[0], x[-1] = x_first, x_last  # exactly, not x_first + h (n_raw - 1)
    return x


def hetero_raw(m: int, n1_out: int, n2_out: int, seed: int, density: float = 1.3,
               nbands1: int = 40, nbands2: int = 12, corr: float = 0.8,
               noise: float = 1e-3) -> RawHetero:
    """Raw hetero pair: Gaussian bands, stack-2 amplitudes lag stack-1 latents by U(0, 90) deg."""
    rng = np.random.default_rng(seed)
    n1_raw = int(round(density * n1_out))
    n2_raw = int(round(density * n2_out))
    x1 = jittered_axis(n1_raw, 0.0, float(n1_out - 1), rng)
    x2 = jittered_axis(n2_raw, 0.0, float(n2_out - 1), rng)
    t = np.arange(m, dtype=np.float64) / m
    ph1 = rng.uniform(0, 2 * np.pi, nbands1)
    lat1 = np.sin(2 * np.pi * t[:, None] + ph1[None, :])  # m x nb1
    a1 = rng.uniform(0.5, 1.5, nbands1)
    c1_ = rng.uniform(0, n1_out - 1, nbands1)
    w1 = rng.uniform(5, 20, nbands1)
    y1 = (lat1 * a1) @ _gauss(x1, c1_, w1)
    src = rng.integers(0, nbands1, nbands2)
    lag = np.deg2rad(rng.uniform(0, 90, nbands2))
    own = np.sin(2 * np.pi * t[:, None] + rng.uniform(0, 2 * np.pi, nbands2)[None, :])
    lat2 = corr * np.sin(2 * np.pi * t[:, None] + ph1[src][None, :] - lag[None, :]) \
        + math.sqrt(1 - corr * corr) * own
    a2 = rng.uniform(0.5, 1.5, nbands2)
    c2_ = rng.uniform(0, n2_out - 1, nbands2)
    w2 = rng.uniform(5, 20, nbands2)
    y2 = (lat2 * a2) @ _gauss(x2, c2_, w2)
    y1 = y1 + noise * rng.standard_normal(y1.shape)
    y2 = y2 + noise * rng.standard_normal(y2.shape)
    return RawHetero(x1, y1.astype(np.float32), x2, y2.astype(np.float32), n1_out, n2_out)


def c3(seed: int = 2) -> RawHetero:
    """m=128, n1=8192, n2=2048 targets, raw axes ~1.3x denser, alpha=0.5."""
    return hetero_raw(128, 8192, 2048, seed)


@dataclass
class Problem:
    m: int
    n1: int
    n2: int
    homo: bool
    seed: int


@dataclass
class BatchSpec:
    problems: list = field(default_factory=list)

    @property
    def total_outputs(self) -> int:
        return sum(p.n1 * p.n2 for p in self.problems)


def c5_spec(count: int = 512, seed: int = 4, m_lo: int = 8, m_hi: int = 200,
            n_lo: int = 256, n_hi: int = 8192, n_fixed: int = 0) -> BatchSpec:
    """Shapes of the batched workload: m ~ U{m_lo..m_hi}, n log-uniform, even = homo.
    n_fixed > 0 gives every stack n_fixed variables and keeps every other draw
    (a smaller case with the same m mix, for profiling)."""
    rng = np.random.default_rng(seed)
    spec = BatchSpec()
    for i in range(count):
        m = int(rng.integers(m_lo, m_hi + 1))
        n1 = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        n2r = int(round(math.exp(rng.uniform(math.log(n_lo), math.log(n_hi)))))
        if n_fixed > 0:
            n1 = n2r = n_fixed
        homo = (i % 2 == 0)
        spec.problems.append(Problem(m, n1, n1 if homo else n2r, homo, seed * 100003 + i))
    return spec


def batch_inputs(spec: BatchSpec, nbands: int = 20):
    """Stacks for every problem of a batch: list of (y1, y2 or None)."""
    out = []
    for p in spec.problems:
        y1 = sigmoid_bands(p.m, p.n1, nbands, p.seed, baseline=1.0)
        y2 = None if p.homo else sigmoid_bands(p.m, p.n2, nbands, p.seed + 7, baseline=1.0)
        out.append((y1, y2))
    return out


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """Seeded sorted sample of max(count, 2) distinct row indices (all n when
    count >= n) that always includes the first and the last row."""
    if count >= n:
        return np.arange(n, dtype=np.int32)
    rng = np.random.default_rng(seed)
    inner = rng.choice(np.arange(1, n - 1), size=max(count - 2, 0), replace=False)
    return np.array(sorted({0, n - 1} | set(inner.tolist())), dtype=np.int32)

