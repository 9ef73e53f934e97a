"""Seeded synthetic inputs shaped like the test problems of arXiv 2003.07968.

This module feeds both the CUDA path and the FP64 oracle with the SAME
arrays.  It holds no arithmetic of the method itself: only random numbers
(SplitMix64), initial density fields (the tanh droplet of Eq. ISD, the
ellipse of Eq. REL, a flat liquid band) and workload recipes.  The
coexistence densities used to initialise the fields come from a table that
``oracle/write_coexistence_table.py`` writes (Maxwell equal-area rule).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np

SEED = 2003007968
_HERE = os.path.dirname(os.path.abspath(__file__))
_TABLE = os.path.join(_HERE, "coexistence_cs.json")
_table_cache = None

_GOLDEN_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_MIX1 = np.uint64(0xBF58476D1CE4E5B9)
_MIX2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """n outputs of SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) started at
    state ``seed``; output k uses state seed + (offset + k + 1) * gamma."""
    with np.errstate(over="ignore"):
        k = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GOLDEN_GAMMA
        z = (z ^ (z >> np.uint64(30))) * _MIX1
        z = (z ^ (z >> np.uint64(27))) * _MIX2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo: float = 0.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    """Uniform doubles in [lo, hi) from the top 53 bits of SplitMix64."""
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0**-53)
    return lo + (hi - lo) * u


def randint(seed: int, n: int, lo: int, hi: int, offset: int = 0) -> np.ndarray:
    """Integers uniform on {lo, ..., hi} (inclusive)."""
    u = uniform(seed, n, 0.0, 1.0, offset)
    return np.minimum(lo + np.floor(u * (hi - lo + 1)).astype(np.int64), hi)


def coexistence(T: float) -> tuple[float, float]:
    """(rho_g, rho_l) of the Maxwell rule at reduced temperature T, linearly
    interpolated in the stored table (0.55 <= T <= 0.95)."""
    global _table_cache
    if _table_cache is None:
        with open(_TABLE) as fh:
            _table_cache = json.load(fh)
    t = np.asarray(_table_cache["T"])
    if not (t[0] <= T <= t[-1]):
        raise ValueError(f"T={T} outside the coexistence table [{t[0]}, {t[-1]}]")
    return (float(np.interp(T, t, _table_cache["rho_g"])),
            float(np.interp(T, t, _table_cache["rho_l"])))


def flat_band(nx: int = 64, ny: int = 64, T: float = 0.8, rows=(16, 47),
              noise: float = 1e-3, seed: int = SEED + 1) -> np.ndarray:
    """Liquid band in rows ``rows[0]..rows[1]`` (inclusive), vapour elsewhere,
    at the coexistence densities of T, plus uniform noise in [-noise, noise)."""
    rg, rl = coexistence(T)
    rho = np.full((ny, nx), rg)
    rho[rows[0]:rows[1] + 1, :] = rl
    if noise:
        rho += uniform(seed, nx * ny, -noise, noise).reshape(ny, nx)
    return rho


def band(nx: int, ny: int, T: float, y1: float, y2: float, W: float = 5.0,
         densities=None) -> np.ndarray:
    """Flat liquid band between rows y1 and y2 with the tanh interface
    profile of Eq. (ISD) (width W) on both sides, vapour elsewhere."""
    rg, rl = densities if densities is not None else coexistence(T)
    y = np.arange(ny, dtype=np.float64)[:, None] * np.ones((1, nx))
    prof = 0.5 * (np.tanh(2.0 * (y - y1) / W) - np.tanh(2.0 * (y - y2) / W))
    return rg + (rl - rg) * prof


def droplet(nx: int, ny: int, R: float, T: float, W: float = 5.0, center=None,
            densities=None) -> np.ndarray:
    """Circular droplet with the tanh profile of Eq. (ISD), centred on node
    (nx//2, ny//2)."""
    rg, rl = densities if densities is not None else coexistence(T)
    x0, y0 = (nx // 2, ny // 2) if center is None else center
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    return 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh(2.0 * (r - R) / W)


def ellipse(nx: int, ny: int, r_max: float, r_min: float, T: float, W: float = 5.0,
            densities=None) -> np.ndarray:
    """Elliptic droplet, Eq. (ISD) with R_0(theta) of Eq. (REL); semi-axis
    r_max along x and r_min along y."""
    rg, rl = densities if densities is not None else coexistence(T)
    x0, y0 = nx // 2, ny // 2
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    r = np.sqrt((x - x0) ** 2 + (y - y0) ** 2)
    theta = np.arctan2(y - y0, x - x0)
    e = math.sqrt(1.0 - (r_min / r_max) ** 2)
    r0 = r_min / np.sqrt(1.0 - (e * np.cos(theta)) ** 2)
    return 0.5 * (rl + rg) - 0.5 * (rl - rg) * np.tanh(2.0 * (r - r0) / W)


def batch_recipe(n: int = 512, side=(64, 512), rfrac=(0.15, 0.35), T=(0.6, 0.9),
                 seed: int = SEED + 4) -> list[dict]:
    """Uneven batch of independent droplet lattices: square sides uniform on
    {side[0]..side[1]}, radius = side * U(rfrac), T uniform on T."""
    sides = randint(seed, n, side[0], side[1], offset=0)
    fr = uniform(seed, n, rfrac[0], rfrac[1], offset=n)
    ts = uniform(seed, n, T[0], T[1], offset=2 * n)
    return [dict(nx=int(s), ny=int(s), R=float(s * f), T=float(t))
            for s, f, t in zip(sides, fr, ts)]


def serving_stream(n: int = 1000, rate: float = 200.0, side=(128, 2048),
                   steps=(1000, 50000), T=(0.6, 0.9), seed: int = SEED + 5) -> list[dict]:
    """Finite Poisson arrival stream of solve requests: inter-arrival times
    exponential with the given rate, kind droplet/flat band 50/50, square
    sides uniform on {side}, step counts uniform on {steps}, T uniform."""
    gaps = -np.log1p(-uniform(seed, n, 0.0, 1.0, offset=0)) / rate
    kinds = uniform(seed, n, 0.0, 1.0, offset=n) < 0.5
    sides = randint(seed, n, side[0], side[1], offset=2 * n)
    nst = randint(seed, n, steps[0], steps[1], offset=3 * n)
    ts = uniform(seed, n, T[0], T[1], offset=4 * n)
    rf = uniform(seed, n, 0.15, 0.35, offset=5 * n)
    t_arr = np.cumsum(gaps)
    return [dict(t_arrival=float(a), kind="droplet" if k else "band", nx=int(s), ny=int(s),
                 steps=int(m), T=float(t), R=float(s * f))
            for a, k, s, m, t, f in zip(t_arr, kinds, sides, nst, ts, rf)]


def request_field(req: dict) -> np.ndarray:
    """Initial density field of one serving request."""
    if req["kind"] == "droplet":
        return droplet(req["nx"], req["ny"], req["R"], req["T"])
    ny = req["ny"]
    return band(req["nx"], ny, req["T"], ny / 4.0, 3.0 * ny / 4.0)
