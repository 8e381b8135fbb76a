"""The 1D modified-Helmholtz inverse by fast convolution (Sec. 3.1.2 Eq. L_Inverse / Iu, Sec. 3.2 Eq. IL, IR, homogeneous).

Test infrastructure only (see ``oracle/__init__.py``).

H_c[v] = L^{-1}[v] with L = I - c d_xx = I - d_xx / alpha^2, alpha = c^{-1/2}:

    L^{-1}[v](x) = I[v](x) + B_a e^{-alpha (x - a)} + B_b e^{-alpha (b - x)},
    I[v] = I^L + I^R,   I^L_j = d I^L_{j-1} + J^L_j,   I^R_j = d I^R_{j+1} + J^R_j,

on nodes a = x_0 < ... < x_N = b with uniform h, d = e^{-alpha h}, mu = e^{-alpha (b - a)} = d^N.

Readings (the paper leaves these open):
* Grid: periodic lines store N nodes (node N is node 0); Neumann / Dirichlet
  lines store N + 1 nodes with both walls as nodes.
* Stencils: centred -M/2..M/2 about x_j; on non-periodic lines a stencil that
  would leave [x_0, x_N] is shifted inward to keep M + 1 nodes, integrating
  over the same cell.  Periodic stencils wrap.
* B_a, B_b: periodic is Eq. homogeneous.  Neumann and Dirichlet are the
  "analogous" 2x2 systems of Sec. 3.2, obtained the same way from
  L^{-1}(a), L^{-1}(b) and L^{-1}_x = alpha (I^R - I^L) + homogeneous part:
      Neumann   (L^{-1}v)_x = 0 at a, b:  B_a - mu B_b = I_0,   -mu B_a + B_b = I_N
      Dirichlet  L^{-1}v    = 0 at a, b:  B_a + mu B_b = -I_0,   mu B_a + B_b = -I_N
  with I_0 = I^R_0 and I_N = I^L_N.  (The periodic slope condition is printed
  with +B_a mu on the right; the slope of B_a e^{-alpha(x-a)} at b is
  -alpha mu B_a, and only that sign yields the printed B_a = I_N/(1-mu),
  B_b = I_0/(1-mu), which is what is used.)
"""
from __future__ import annotations

from functools import lru_cache

import numpy as np
from scipy.signal import lfilter

from .weights import local_weights

PERIODIC, NEUMANN, DIRICHLET = "periodic", "neumann", "dirichlet"


def intervals(n: int, bc: str) -> int:
    """Number of intervals N for n stored nodes."""
    return n if bc == PERIODIC else n - 1


def stencil_nodes(j: int, N: int, M: int, bc: str):
    """Node indices (in 0..N) of the M+1 point stencil used at node j."""
    if bc == PERIODIC:
        return [(j + o) % N for o in range(-M // 2, M // 2 + 1)]
    start = min(max(j - M // 2, 0), N - M)
    return list(range(start, start + M + 1))


def _offsets(j: int, nodes_j, M: int, bc: str):
    """Stencil offsets relative to node j (periodic stencils are always centred)."""
    if bc == PERIODIC:
        return tuple(range(-M // 2, M // 2 + 1))
    return tuple(m - j for m in nodes_j)


@lru_cache(maxsize=256)
def _gather_tables(n: int, nu: float, M: int, bc: str):
    """Index and weight tables: J^L_j = sum_k WL[j,k] v[idxL[j,k]], same for R."""
    N = intervals(n, bc)
    if N < M:
        raise ValueError(f"line of {n} nodes is too short for quadrature order M={M}")
    idxL = np.zeros((N + 1, M + 1), dtype=np.int64)
    idxR = np.zeros((N + 1, M + 1), dtype=np.int64)
    WL = np.zeros((N + 1, M + 1))
    WR = np.zeros((N + 1, M + 1))
    cacheL, cacheR = {}, {}
    for j in range(1, N + 1):                      # J^L_j, j = 1..N (Eq. IL)
        nodes_j = stencil_nodes(j, N, M, bc)
        offs = _offsets(j, nodes_j, M, bc)
        if offs not in cacheL:
            cacheL[offs] = local_weights(nu, offs, "L")
        idxL[j] = nodes_j
        WL[j] = cacheL[offs]
    for j in range(0, N):                          # J^R_j, j = 0..N-1 (Eq. IR)
        nodes_j = stencil_nodes(j, N, M, bc)
        offs = _offsets(j, nodes_j, M, bc)
        if offs not in cacheR:
            cacheR[offs] = local_weights(nu, offs, "R")
        idxR[j] = nodes_j
        WR[j] = cacheR[offs]
    return idxL, WL, idxR, WR


def line_constants(c: float, h: float, n: int, bc: str):
    alpha = c ** -0.5
    nu = alpha * h
    d = np.exp(-nu)
    N = intervals(n, bc)
    mu = np.exp(-nu * N)
    return alpha, nu, d, mu, N


def local_integrals(v: np.ndarray, c: float, h: float, bc: str, M: int):
    """J^L_j (j = 1..N) and J^R_j (j = 0..N-1) for stored nodes ``v`` (last axis), as arrays over nodes 0..N.

    Periodic stencil indices are already reduced mod N, so node N reads node 0."""
    n = v.shape[-1]
    _, nu, _, _, N = line_constants(c, h, n, bc)
    idxL, WL, idxR, WR = _gather_tables(n, float(nu), M, bc)
    JL = np.einsum("...jk,jk->...j", v[..., idxL], WL)
    JR = np.einsum("...jk,jk->...j", v[..., idxR], WR)
    JL[..., 0] = 0.0
    JR[..., N] = 0.0
    return JL, JR


def boundary_coefficients(I0, IN, mu: float, bc: str):
    """B_a, B_b from the 2x2 boundary system (Eq. homogeneous and its Neumann/Dirichlet analogues)."""
    if bc == PERIODIC:
        return IN / (1 - mu), I0 / (1 - mu)
    if bc == NEUMANN:
        return (I0 + mu * IN) / (1 - mu ** 2), (IN + mu * I0) / (1 - mu ** 2)
    if bc == DIRICHLET:
        return -(I0 - mu * IN) / (1 - mu ** 2), -(IN - mu * I0) / (1 - mu ** 2)
    raise ValueError(bc)


def helmholtz_inverse(f: np.ndarray, c: float, h: float, bc: str, M: int, axis: int = -1) -> np.ndarray:
    """H_c[f] along ``axis``: one application of L^{-1} = (I - c d_xx)^{-1} to every line."""
    f = np.moveaxis(np.asarray(f, dtype=np.float64), axis, -1)
    n = f.shape[-1]
    _, _, d, mu, N = line_constants(c, h, n, bc)
    IL, IR = particular_recurrence(f, c, h, bc, M)
    I0 = IR[..., 0]
    IN = IL[..., N]
    Ba, Bb = boundary_coefficients(I0, IN, mu, bc)
    j = np.arange(N + 1)
    out = IL + IR + Ba[..., None] * d ** j + Bb[..., None] * d ** (N - j)
    if bc == PERIODIC:
        out = out[..., :N]
    return np.moveaxis(out, -1, axis)


def particular_recurrence(f: np.ndarray, c: float, h: float, bc: str, M: int):
    """I^L and I^R over nodes 0..N by the exponential recurrences (Eq. IL, IR), last axis."""
    n = f.shape[-1]
    _, _, d, _, N = line_constants(c, h, n, bc)
    JL, JR = local_integrals(f, c, h, bc, M)          # over nodes 0..N
    # Eq. IL: I^L_0 = 0, I^L_j = d I^L_{j-1} + J^L_j.  lfilter([1], [1, -d]) is exactly
    # y_k = x_k + d y_{k-1} with zero initial state.
    IL = np.zeros_like(JL)
    IL[..., 1:] = lfilter([1.0], [1.0, -d], JL[..., 1:], axis=-1)
    # Eq. IR: I^R_N = 0, I^R_j = d I^R_{j+1} + J^R_j (the same filter run backwards).
    IR = np.zeros_like(JR)
    IR[..., :N] = lfilter([1.0], [1.0, -d], JR[..., :N][..., ::-1], axis=-1)[..., ::-1]
    return IL, IR


def particular_direct(f: np.ndarray, c: float, h: float, bc: str, M: int) -> np.ndarray:
    """O(N^2) direct sum I_j = sum_{i<=j} d^{j-i} J^L_i + sum_{i>=j} d^{i-j} J^R_i on nodes 0..N (pin for Eq. IL/IR)."""
    f = np.asarray(f, dtype=np.float64)
    n = f.shape[-1]
    _, _, d, _, N = line_constants(c, h, n, bc)
    JL, JR = local_integrals(f, c, h, bc, M)
    out = np.zeros_like(JL)
    for jj in range(N + 1):
        for i in range(1, jj + 1):
            out[..., jj] += d ** (jj - i) * JL[..., i]
        for i in range(jj, N):
            out[..., jj] += d ** (i - jj) * JR[..., i]
    return out
