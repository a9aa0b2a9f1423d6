"""Seeded synthetic inputs for harmonic summing: noise planes, injected
harmonic signals and detection thresholds.

This module holds none of the harmonic-summing arithmetic (no stretch, no
level sums, no comparison).  It only draws the inputs that both the CUDA path
and the FP64 oracle are given, so that both see the same bytes.

Plane recipe (the paper's filter-output plane, Section III, is detected
power; no real data is available, so noise and signals are synthetic):
  * noise: iid Exponential(mean 1) per point, drawn from numpy's Philox
    counter-based generator keyed by the seed, row by row, in binary32;
  * signals: a fundamental at (z0, f0) with harmonics at (h*z0, h*f0),
    h = 1..H, each with an amplitude drawn from U[3, 8], added where the
    harmonic lies inside the plane;
  * thresholds: for unit-mean exponential noise a sum of k independent points
    is Gamma(k, 1); the level-k threshold T_k solves Q(k, T_k) = p_fa with Q the
    regularised upper incomplete gamma function, so every level has the same
    per-point false-alarm probability.  The same value is used for every row.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Signal:
    z0: int
    f0: int
    amps: np.ndarray  # amplitude of harmonic h = 1..len(amps)


@dataclass
class Workload:
    name: str
    n_templates: int
    n_bins: int
    H: int
    seed: int
    p_fa: float
    n_signals: int
    f0_range: tuple
    z0_range: tuple
    signals: list = field(default_factory=list)


def small_plane(seed: int = 0) -> Workload:
    """21 templates (z = -10..10) x 65,536 bins, H = 8, p_fa = 1e-6, 5 signals."""
    return Workload("plane 21x65536 H=8 fp32", 21, 65536, 8, seed, 1e-6, 5,
                    (500, 8000), (-1, 1))


def ska_plane(seed: int = 1) -> Workload:
    """85 templates (z = -42..42) x 2^21 bins, H = 16, p_fa = 1e-8, 50 signals."""
    return Workload("plane 85x2^21 H=16 fp32", 85, 1 << 21, 16, seed, 1e-8, 50,
                    (10_000, 100_001), (-2, 2))


def beam_lengths(n_beams: int = 64, seed: int = 3, lo_log2: float = 18.0,
                 hi_log2: float = 22.0) -> np.ndarray:
    """Bin counts drawn log-uniform in [2^lo, 2^hi], rounded to integers."""
    rng = np.random.Generator(np.random.Philox(seed))
    u = rng.uniform(lo_log2, hi_log2, size=n_beams)
    return np.rint(2.0 ** u).astype(np.int64)


def noise(n_templates: int, n_bins: int, seed: int, out: np.ndarray | None = None,
          row_offset: int = 0) -> np.ndarray:
    """iid Exponential(mean 1) binary32 plane, drawn row by row.

    out may be a preallocated float32 [n_templates][n_bins] array (for example
    a pinned host buffer).  Row r uses the Philox stream keyed by
    (seed, r + row_offset), so any row can be regenerated on its own."""
    if out is None:
        out = np.empty((n_templates, n_bins), np.float32)

    def row(r):
        rng = np.random.Generator(np.random.Philox(key=[seed, r + row_offset]))
        out[r, :] = rng.standard_exponential(n_bins, dtype=np.float32)

    if n_templates * n_bins < (1 << 22):
        for r in range(n_templates):
            row(r)
    else:
        # rows are independent streams; numpy releases the GIL while filling
        with ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 1)) as ex:
            list(ex.map(row, range(n_templates)))
    return out


def sparse_points(n_templates: int, n_bins: int, count: int, seed: int):
    """`count` distinct (row, bin) positions of an n_templates x n_bins plane,
    drawn uniformly without replacement, and an Exponential(mean 1) binary32
    value for each: (rows int64, bins int64, values float32)."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x5A]))
    flat = rng.choice(n_templates * n_bins, size=count, replace=False)
    vals = rng.standard_exponential(count, dtype=np.float32)
    return flat // n_bins, flat % n_bins, vals


def sparse(n_templates: int, n_bins: int, count: int, seed: int,
           ld: int | None = None) -> np.ndarray:
    """A plane [n_templates][ld] (ld >= n_bins, the row pitch) that is zero
    except at the positions and values of sparse_points; the padding bins
    [n_bins, ld) stay zero.  The zeros are not written, so a very large
    plane costs memory only where a value lies."""
    ld = n_bins if ld is None else ld
    if ld < n_bins:
        raise ValueError("row pitch below the bin count")
    out = np.zeros((n_templates, ld), np.float32)
    rows, bins, vals = sparse_points(n_templates, n_bins, count, seed)
    out[rows, bins] = vals
    return out


def draw_signals(wl: Workload, H_inj: int | None = None) -> list:
    """Random fundamentals with per-harmonic amplitudes U[3, 8]."""
    H_inj = wl.H if H_inj is None else H_inj
    rng = np.random.Generator(np.random.Philox(key=[wl.seed, 0x5157]))
    sigs = []
    for _ in range(wl.n_signals):
        f0 = int(rng.integers(wl.f0_range[0], wl.f0_range[1]))
        z0 = int(rng.integers(wl.z0_range[0], wl.z0_range[1] + 1))
        amps = rng.uniform(3.0, 8.0, size=H_inj).astype(np.float32)
        sigs.append(Signal(z0, f0, amps))
    return sigs


def inject(plane: np.ndarray, signals: list) -> np.ndarray:
    """Add each signal's harmonics at (h*z0, h*f0) where they fit (in place)."""
    nt, n = plane.shape
    Z = (nt - 1) // 2
    for s in signals:
        for h, a in enumerate(s.amps, start=1):
            z, f = h * s.z0, h * s.f0
            if -Z <= z <= Z and 0 <= f < n:
                plane[z + Z, f] = np.float32(plane[z + Z, f] + a)
    return plane


def level_thresholds(p_fa: float, H: int) -> np.ndarray:
    """T_k with Q(k, T_k) = p_fa for k = 1..H (float64)."""
    from scipy.special import gammainccinv
    return np.array([gammainccinv(k, p_fa) for k in range(1, H + 1)], np.float64)


def thresholds(p_fa: float, H: int, n_templates: int) -> np.ndarray:
    """Threshold array TA[k-1][row], binary32, the same for every row."""
    t = level_thresholds(p_fa, H).astype(np.float32)
    return np.ascontiguousarray(np.repeat(t[:, None], n_templates, axis=1))


def make_plane(wl: Workload, out: np.ndarray | None = None) -> np.ndarray:
    """Noise plus injected signals for a workload (signals kept on wl)."""
    plane = noise(wl.n_templates, wl.n_bins, wl.seed, out=out)
    wl.signals = draw_signals(wl)
    inject(plane, wl.signals)
    return plane


def random_plane(n_templates: int, n_bins: int, seed: int, *, lo: float = 0.0,
                 hi: float = 1.0) -> np.ndarray:
    """Uniform [lo, hi) binary32 plane (for signed or edge-case inputs)."""
    rng = np.random.Generator(np.random.Philox(key=[seed, 0x0DD]))
    return rng.uniform(lo, hi, size=(n_templates, n_bins)).astype(np.float32)
