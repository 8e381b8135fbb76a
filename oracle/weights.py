"""Local quadrature weights of the fast convolution (Sec. 3.2, Eq. IL / IR and the M=2 weights P, Q, R).

Test infrastructure only (see ``oracle/__init__.py``).

The local integrals are

    J^L_j = (alpha/2) int_{x_{j-1}}^{x_j} e^{-alpha (x_j - x')} v(x') dx'
          = (nu/2) int_0^1 e^{-nu t} v(x_j - t h) dt,
    J^R_j = (alpha/2) int_{x_j}^{x_{j+1}} e^{-alpha (x' - x_j)} v(x') dx'
          = (nu/2) int_0^1 e^{-nu t} v(x_j + t h) dt,            nu = alpha h.

v is replaced by its Lagrange interpolant through M+1 nodes x_{j+o}, o in a
stencil of integer offsets.  The weight of node x_{j+o} is therefore

    wL_o = (nu/2) int_0^1 e^{-nu t} l_o(-t) dt,    wR_o = (nu/2) int_0^1 e^{-nu t} l_o(+t) dt,

with l_o the Lagrange basis polynomial on the stencil offsets.  The factor 1/2
sits inside the weights (reading: the paper's M=2 formulas P, Q, R sum to
1 - d, i.e. they omit the 1/2 of Eq. IL; here it is kept so that J matches
Eq. IL exactly).  The paper gives no formula for M = 4, 6 ("pre-computed");
the reading is the same definition with the centred stencil -M/2..M/2, which
reduces to P, Q, R at M = 2.

Here the integral is evaluated by composite Gauss-Legendre quadrature of the
definition itself, with l_o evaluated by its product formula: slow and direct.
"""
from __future__ import annotations

import numpy as np


def lagrange_basis(offsets, o_index: int, s: np.ndarray) -> np.ndarray:
    """l_o(s) = prod_{k != o} (s - x_k) / (x_o - x_k) on the integer nodes ``offsets``."""
    xo = offsets[o_index]
    out = np.ones_like(s, dtype=np.float64)
    for k, xk in enumerate(offsets):
        if k != o_index:
            out = out * (s - xk) / (xo - xk)
    return out


def _gauss_legendre_01(nu: float):
    """Composite Gauss-Legendre nodes/weights on [0, 1], panels fine enough for e^{-nu t}."""
    panels = 1 + int(np.ceil(nu / 8.0))
    xg, wg = np.polynomial.legendre.leggauss(40)
    t_all, w_all = [], []
    for p in range(panels):
        a, b = p / panels, (p + 1) / panels
        t_all.append(a + (b - a) * (xg + 1) / 2)
        w_all.append(wg * (b - a) / 2)
    return np.concatenate(t_all), np.concatenate(w_all)


def local_weights(nu: float, offsets, side: str) -> np.ndarray:
    """Weights (one per offset) of J^L (side='L') or J^R (side='R') for a given stencil."""
    offsets = [int(o) for o in offsets]
    t, w = _gauss_legendre_01(nu)
    sgn = -1.0 if side == "L" else 1.0
    kern = (nu / 2.0) * np.exp(-nu * t)
    return np.array([np.sum(w * kern * lagrange_basis(offsets, i, sgn * t))
                     for i in range(len(offsets))])


def paper_m2_pqr(nu: float):
    """The paper's M=2 weights P, Q, R exactly as printed in Sec. 3.2 (no factor 1/2)."""
    d = np.exp(-nu)
    P = 1 - (1 - d) / nu
    Q = -d + (1 - d) / nu
    R = (1 - d) / nu ** 2 - (1 + d) / (2 * nu)
    return P, Q, R
