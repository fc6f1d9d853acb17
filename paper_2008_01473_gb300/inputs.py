"""Seeded synthetic inputs shared by the CUDA path, the tests and the benchmark.

This module holds none of the method's arithmetic: it only lays out initial
density fields (tanh droplets as in Eq. 31, flat slabs, noisy uniform states)
from densities and geometry that the caller supplies, plus a counter-based
SplitMix64 noise stream. Both the oracle and the CUDA path are fed the same
arrays.

SplitMix64 (Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): state s_0 = mix(seed) and the i-th output is
mix(s_0 + (i + 1) * 0x9E3779B97F4A7C15), where mix is the published
xor-shift-multiply finaliser. Node (x, y) of case c takes counter
i = (c * ny + y) * nx + x, and a uniform double in [0, 1) is
(out >> 11) * 2^-53.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix_uniform(seed: int, case: int, nx: int, ny: int) -> np.ndarray:
    """U[0, 1) doubles of shape (ny, nx) for one case."""
    s0 = _mix(np.array([seed & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    idx = (np.uint64(case) * np.uint64(ny) + np.arange(ny, dtype=np.uint64)[:, None]) * np.uint64(nx) \
        + np.arange(nx, dtype=np.uint64)[None, :]
    with np.errstate(over="ignore"):
        z = s0 + (idx + np.uint64(1)) * _GOLDEN
    out = _mix(z)
    return (out >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def droplet(nx: int, ny: int, radius: float, rho_l: float, rho_g: float, width: float = 5.0,
            noise: float = 0.0, seed: int = 0, case: int = 0) -> np.ndarray:
    """Eq. 31 tanh droplet centred at (nx/2, ny/2), plus additive U[-noise, noise]."""
    y, x = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64),
                       indexing="ij")
    r0 = np.sqrt((x - nx / 2.0) ** 2 + (y - ny / 2.0) ** 2)
    rho = 0.5 * (rho_l + rho_g) - 0.5 * (rho_l - rho_g) * np.tanh(2.0 * (r0 - radius) / width)
    if noise:
        rho = rho + noise * (2.0 * splitmix_uniform(seed, case, nx, ny) - 1.0)
    return np.ascontiguousarray(rho)


def slab(nx: int, ny: int, rho_l: float, rho_g: float, width: float = 5.0,
         noise: float = 0.0, seed: int = 0, case: int = 0) -> np.ndarray:
    """Flat liquid slab between x = nx/4 and x = 3nx/4 with tanh edges of width W."""
    x = np.arange(nx, dtype=np.float64)
    prof = rho_g + 0.5 * (rho_l - rho_g) * (np.tanh(2.0 * (x - nx / 4.0) / width)
                                             - np.tanh(2.0 * (x - 3.0 * nx / 4.0) / width))
    rho = np.repeat(prof[None, :], ny, axis=0)
    if noise:
        rho = rho + noise * (2.0 * splitmix_uniform(seed, case, nx, ny) - 1.0)
    return np.ascontiguousarray(rho)


def spinodal(nx: int, ny: int, rho_mean: float, rel_noise: float, seed: int = 0,
             case: int = 0) -> np.ndarray:
    """Uniform mean density times (1 + U[-rel_noise, rel_noise])."""
    u = splitmix_uniform(seed, case, nx, ny)
    return np.ascontiguousarray(rho_mean * (1.0 + rel_noise * (2.0 * u - 1.0)))
