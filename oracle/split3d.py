"""Three-dimensional splitting of the stage solve (the extension Sec. 5 remarks on), FP64.

Test infrastructure only (see ``oracle/__init__.py``).

The paper builds the 2D iteration of Sec. 5.1 from the factorization of (I - c Lap) into line
operators and says the splitting extends to three dimensions; it does not write the 3D form.
The reading taken here, for one factor I - c Lap with L_a = I - c d_aa on each axis a:

    L_x L_y L_z = I - c Lap + c^2 (dxx dyy + dxx dzz + dyy dzz) - c^3 dxx dyy dzz,

so I - c Lap = L_x L_y L_z - P.  With the line inverse H_a = L_a^{-1} and D_a = I - H_a
(= -c H_a d_aa), and M^{-1} = H_x H_y H_z,

    M^{-1} P = D_x D_y H_z + D_x D_z H_y + D_y D_z H_x + D_x D_y D_z
             = D_x D_y + D_x D_z + D_y D_z - 2 D_x D_y D_z  =: X,

hence I - c Lap = M (I - X).  In 2D the same steps give X = D_x D_y, the operator of
Eq. CH_2D_Doperator1.  The stage equation v - tau F(v) = r then takes the 2D iteration of
Sec. 5.1 with X in place of D_x D_y (``oracle/solver.py`` states the 2D form):

    v^{k+1} = Y + M_o^{-1}[ beta (M_i^{-1} G - G + X_i G) ] + (X_o + X_i - X_o X_i) v^k,
    Y = M_o^{-1} M_i^{-1} r,   G = G(v^k) as in 1D and 2D.

Arrays are indexed [z, y, x] (x fastest).  Grids follow the 2D conventions: periodic lines
store N nodes with h = L/N, Neumann lines N nodes with h = L/(N-1).  Dirichlet walls are not
covered here.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .helmholtz import helmholtz_inverse
from .solver import G, StageResult, stage_params

PERIODIC, NEUMANN = "periodic", "neumann"


@dataclass
class Problem3D:
    nx: int
    ny: int
    nz: int
    Lx: float = 2 * np.pi
    Ly: float = 2 * np.pi
    Lz: float = 2 * np.pi
    bc: str = PERIODIC
    eps: float = 0.1
    M: int = 4
    tol: float = 1e-10
    max_iter: int = 1000

    def h(self, axis: str) -> float:
        n, L = {"x": (self.nx, self.Lx), "y": (self.ny, self.Ly), "z": (self.nz, self.Lz)}[axis]
        return L / n if self.bc == PERIODIC else L / (n - 1)


_AXIS = {"x": 2, "y": 1, "z": 0}


def H(prob: Problem3D, f: np.ndarray, c: float, axis: str) -> np.ndarray:
    """The line inverse (I - c d_aa)^{-1} along one axis (Sec. 3, Eq. IL/IR with the boundary
    correction), applied to every line of that axis."""
    return helmholtz_inverse(f, c, prob.h(axis), prob.bc, prob.M, axis=_AXIS[axis])


def D(prob: Problem3D, f: np.ndarray, c: float, axis: str) -> np.ndarray:
    """D_a = I - H_a."""
    return f - H(prob, f, c, axis)


def M_inv(prob: Problem3D, f: np.ndarray, c: float) -> np.ndarray:
    """(L_x L_y L_z)^{-1} f = H_x H_y H_z f."""
    return H(prob, H(prob, H(prob, f, c, "z"), c, "y"), c, "x")


def X(prob: Problem3D, f: np.ndarray, c: float) -> np.ndarray:
    """X f = (D_x D_y + D_x D_z + D_y D_z - 2 D_x D_y D_z) f, the splitting remainder M^{-1} P."""
    dz = D(prob, f, c, "z")
    dy = D(prob, f, c, "y")
    dydz = D(prob, dz, c, "y")
    return D(prob, dy, c, "x") + D(prob, dz, c, "x") + dydz - 2.0 * D(prob, dydz, c, "x")


def stage_rhs_inverse(prob: Problem3D, r: np.ndarray, sp) -> np.ndarray:
    """Y = M_o^{-1} M_i^{-1} r."""
    return M_inv(prob, M_inv(prob, r, sp.c_in), sp.c_out)


def fixed_point_map(prob: Problem3D, Y: np.ndarray, v: np.ndarray, sp) -> np.ndarray:
    """One fixed-point iteration of the 3D split stage (the module's reading of Sec. 5.1)."""
    g = G(v, sp.lam)
    inner = sp.beta * (M_inv(prob, g, sp.c_in) - g + X(prob, g, sp.c_in))
    xi = X(prob, v, sp.c_in)
    return Y + M_inv(prob, inner, sp.c_out) + X(prob, v, sp.c_out) + xi - X(prob, xi, sp.c_out)


def stage_solve(prob: Problem3D, r: np.ndarray, v0: np.ndarray, tau: float) -> StageResult:
    """Solve v - tau F(v) = r by the lagged fixed-point iteration; stop at ||v^{k+1} - v^k||_inf
    < tol (Sec. 4.4) or max_iter; the first guess is v0."""
    sp = stage_params(tau, prob.eps)
    Y = stage_rhs_inverse(prob, r, sp)
    v = np.array(v0, dtype=np.float64)
    res, hist = np.inf, []
    for k in range(1, prob.max_iter + 1):
        v_new = fixed_point_map(prob, Y, v, sp)
        res = float(np.max(np.abs(v_new - v)))
        hist.append(res)
        v = v_new
        if res < prob.tol:
            return StageResult(v, k, res, True, hist)
    return StageResult(v, prob.max_iter, res, False, hist)


class Solver3D:
    """BE and BDF2 (BE start, restarted whenever dt changes) in the physical variable u;
    internally v = u + 1, as the 1D and 2D oracle."""

    def __init__(self, prob: Problem3D):
        self.prob = prob
        self.v_prev = None
        self.dt_prev = None

    def step(self, u: np.ndarray, dt: float, scheme: str):
        v = np.asarray(u, dtype=np.float64) + 1.0
        if scheme == "be" or (scheme == "bdf2" and (self.v_prev is None or self.dt_prev != dt)):
            res = stage_solve(self.prob, v, v, dt)
        elif scheme == "bdf2":
            res = stage_solve(self.prob, (4.0 * v - self.v_prev) / 3.0, v, 2.0 * dt / 3.0)
        else:
            raise ValueError(scheme)
        self.v_prev, self.dt_prev = v, dt
        return res.v - 1.0, res


def mass(prob: Problem3D, u: np.ndarray) -> float:
    """Trapezoid-weighted sum h_x h_y h_z sum w u (weights 1/2 on non-periodic boundary nodes)."""
    def w(n):
        a = np.ones(n)
        if prob.bc != PERIODIC:
            a[0] = a[-1] = 0.5
        return a
    wt = w(prob.nz)[:, None, None] * w(prob.ny)[None, :, None] * w(prob.nx)[None, None, :]
    return float(prob.h("x") * prob.h("y") * prob.h("z") * np.sum(wt * u))


__all__ = ["Problem3D", "H", "D", "M_inv", "X", "stage_rhs_inverse", "fixed_point_map", "stage_solve", "Solver3D",
           "mass"]
