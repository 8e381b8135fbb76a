"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle callers.

This module holds only input generation: a counter-based random generator
(SplitMix64, Steele, Lea & Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014) and the initial conditions / grids the paper and the
benchmark workloads use.  It contains none of the solver's arithmetic, so both
the CUDA path and the CPU oracle can be fed from it without sharing code.

Grid convention (one reading of the paper, stated once here and used by both
sides): a periodic line of ``n`` stored nodes has ``N = n`` intervals and
``h = L / n``; a non-periodic line (Neumann or Dirichlet) of ``n`` stored nodes
has both walls as nodes, ``N = n - 1`` intervals and ``h = L / (n - 1)``.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Outputs ``offset .. offset+count-1`` of the SplitMix64 stream started at ``seed``."""
    idx = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, count: int, offset: int = 0) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of SplitMix64."""
    return (splitmix64(seed, count, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


def uniform_noise(shape, amp: float, seed: int, mean: float = 0.0) -> np.ndarray:
    """``mean + amp * U[-1, 1]`` on ``shape`` (row-major fill order)."""
    count = int(np.prod(shape))
    return (mean + amp * (2.0 * uniform01(seed, count) - 1.0)).reshape(shape)


def gaussian_noise(shape, amp: float, seed: int, mean: float = 0.0) -> np.ndarray:
    """``mean + amp * N(0, 1)`` by Box-Muller on pairs of SplitMix64 uniforms."""
    count = int(np.prod(shape))
    m = (count + 1) // 2
    u = uniform01(seed, 2 * m)
    u1 = 1.0 - u[0::2]          # (0, 1]: log is finite
    u2 = u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    z = np.concatenate([r * np.cos(2 * np.pi * u2), r * np.sin(2 * np.pi * u2)])[:count]
    return (mean + amp * z).reshape(shape)


def gaussian_noise_block(shape, rows: int, cols: int, amp: float, seed: int, mean: float = 0.0, row0: int = 0,
                         col0: int = 0) -> np.ndarray:
    """The block of rows row0 .. row0+rows-1 and columns col0 .. col0+cols-1 of
    ``gaussian_noise(shape, ...)`` without drawing the rest of the field (a crop of a large
    initial state).  Needs (row0 + rows) * shape[1] <= half the field, where every value of the
    block is the cosine half of its Box-Muller pair."""
    ny, nx = shape
    m = (ny * nx + 1) // 2
    k0, k1 = row0 * nx, (row0 + rows) * nx
    if row0 + rows > ny or col0 + cols > nx or k1 > m:
        raise ValueError("the block must lie within the first half of the field")
    u = uniform01(seed, 2 * (k1 - k0), offset=2 * k0)
    z = np.sqrt(-2.0 * np.log(1.0 - u[0::2])) * np.cos(2 * np.pi * u[1::2])
    return (mean + amp * z).reshape(rows, nx)[:, col0:col0 + cols].copy()


def three_phase_mixture(shape, seed: int):
    """A random three-phase mixture for the two-component (vector) model: per node, phase fractions
    (p1, p2, p3) ~ Dirichlet(1, 1, 1) (normalised Exp(1) draws from SplitMix64 uniforms), placed at
    the fractions' barycentre of the three phase values, the cube roots of unity of the (u1, u2)
    plane.  Returns (u1, u2) of ``shape``."""
    count = int(np.prod(shape))
    e = -np.log(1.0 - uniform01(seed, 3 * count).reshape(count, 3))   # Exp(1), finite
    p = e / e.sum(axis=1, keepdims=True)
    ang = np.array([0.0, 2.0 * np.pi / 3.0, -2.0 * np.pi / 3.0])
    return (p @ np.cos(ang)).reshape(shape), (p @ np.sin(ang)).reshape(shape)


def spacing(n: int, length: float, periodic: bool) -> float:
    """Node spacing for ``n`` stored nodes on a line of ``length``."""
    return length / n if periodic else length / (n - 1)


def nodes(n: int, length: float, periodic: bool, start: float = 0.0) -> np.ndarray:
    return start + spacing(n, length, periodic) * np.arange(n)


def paper_ic_1d(n: int, periodic: bool = True) -> np.ndarray:
    """Initial state of the 1D refinement and ripening runs (Eq. CH1D_initial), x in [0, 2pi]."""
    x = nodes(n, 2 * np.pi, periodic)
    return np.cos(2 * x) + 0.01 * np.exp(np.cos(x + 0.1))


def paper_ic_2d(nx: int, ny: int, periodic: bool = True) -> np.ndarray:
    """Initial state of the 2D runs (Eq. CH2D_initial) on [0, 2pi]^2, shape (ny, nx)."""
    x = nodes(nx, 2 * np.pi, periodic)[None, :]
    y = nodes(ny, 2 * np.pi, periodic)[:, None]
    s = np.sin(x) + np.sin(y)
    return 2 * np.exp(s - 2) + 2.2 * np.exp(-s - 2) - 1


def mode_ic(nx: int, ny: int, kx: int, ky: int, amp: float, periodic: bool = True) -> np.ndarray:
    """A single small Fourier mode ``amp * sin(kx x) sin(ky y)`` (or ``sin(kx x)`` when ny == 1)."""
    x = nodes(nx, 2 * np.pi, periodic)[None, :]
    if ny == 1:
        return (amp * np.sin(kx * x)).reshape(1, nx)
    y = nodes(ny, 2 * np.pi, periodic)[:, None]
    return amp * np.sin(kx * x) * np.sin(ky * y)
