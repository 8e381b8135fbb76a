"""The sixth-order (functionalized) Cahn-Hilliard model of the paper's last section, 1D and 2D, FP64.

Test infrastructure only (see ``oracle/__init__.py``).

Eq. FCH0 in v = u + 1 (Eq. FCH): v_t = Lap[(eps^2 Lap - f'(v) + eta eps^2)(eps^2 Lap v - f(v))],
f(v) = v^3 - 3v^2 + 2v.  Expanded, v_t = eps^4 Lap^3 v + Lap g(v) with
    g(v) = -eps^2 Lap f - eps^2 f' Lap v + f f' + eta eps^4 Lap v - eta eps^2 f.
Readings (the paper leaves these open, or prints them with a slip):
* BE follows the PDE: (I - dt eps^4 Lap^3) v^{n+1} = v^n + dt Lap g(v^{n+1}).  Eq. FCH_BE prints
  the last four bracket terms with the opposite signs, which would make eta eps^4 Lap^2 v
  dissipative where the PDE makes it anti-dissipative; the PDE is taken.
* Completing the cube with a = (dt eps^4)^(1/3): I - dt eps^4 Lap^3 = (I - a Lap)^3 + 3a Lap - 3a^2 Lap^2,
  and H = (I - a Lap)^{-1} (the line inverse of Sec. 3 with c = a) gives H Lap = (H - I)/a.  With
  D = H - I the lagged iteration v^{k+1} = H^3[v^n + dt Lap g(v^k) - (3a Lap - 3a^2 Lap^2) v^k]
  becomes, with no explicit derivative,
    v^{k+1} = H z,
    z = H^2 v^n + (3 + c_eta) D^2 v - 3 H D v - c_f D^2 f + c_p H D p,
  c_eta = dt eta eps^4 / a^2, c_f = dt eps^2 / a^2, c_p = dt / a, and the pointwise part
  p = -eps^2 f' Lap v + f f' - eta eps^2 f.
* The product f' Lap v needs Lap v.  The iterate is v^{k+1} = H z with z from the same
  iteration, so Lap v^{k+1} = (v^{k+1} - z)/a exactly for the discrete H; it is kept with the
  iterate.  The first iteration of a run (initial data, no z yet) takes Lap(H v^n) = (H v^n - v^n)/a
  in its place; the fixed point does not depend on it.
Stopping: ||v^{k+1} - v^k||_inf < tol (Sec. 4.4) or max_iter.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .helmholtz import helmholtz_inverse
from .solver import Problem


@dataclass
class FchResult:
    v: np.ndarray
    lap_v: np.ndarray
    iters: int
    residual: float
    converged: bool
    history: list   # ||v^{k+1} - v^k||_inf after each iteration


def f_v(v):
    """f(v) = v^3 - 3v^2 + 2v (f(u) = u^3 - u in v = u + 1)."""
    return v ** 3 - 3 * v ** 2 + 2 * v


def fp_v(v):
    """f'(v) = 3v^2 - 6v + 2."""
    return 3 * v ** 2 - 6 * v + 2


def _H(prob: Problem, f: np.ndarray, a: float) -> np.ndarray:
    return helmholtz_inverse(f, a, prob.hx, prob.bc, prob.M, axis=1)


def fch_be_step(prob: Problem, vn: np.ndarray, dt: float, eta: float, lap_vn=None) -> FchResult:
    """One BE step of Eq. FCH by the iteration of the module docstring; lap_vn is Lap v^n from the
    previous step (None for initial data)."""
    eps = prob.eps
    a = (dt * eps ** 4) ** (1.0 / 3.0)
    c_eta, c_f, c_p = dt * eta * eps ** 4 / a ** 2, dt * eps ** 2 / a ** 2, dt / a
    H = lambda g: _H(prob, g, a)
    h_vn = H(vn)
    h2_vn = H(h_vn)
    v = np.array(vn, dtype=np.float64)
    lap = np.array(lap_vn if lap_vn is not None else (h_vn - vn) / a, dtype=np.float64)
    res, hist = np.inf, []
    for k in range(1, prob.max_iter + 1):
        f, fp = f_v(v), fp_v(v)
        p = -eps ** 2 * fp * lap + f * fp - eta * eps ** 2 * f
        dv = H(v) - v
        hdv = H(dv)
        df = H(f) - f
        hdf = H(df)
        dp = H(p) - p
        hdp = H(dp)
        z = h2_vn + (3 + c_eta) * (hdv - dv) - 3 * hdv - c_f * (hdf - df) + c_p * hdp
        v_new = H(z)
        lap = (v_new - z) / a
        res = float(np.max(np.abs(v_new - v)))
        hist.append(res)
        v = v_new
        if res < prob.tol:
            return FchResult(v, lap, k, res, True, hist)
    return FchResult(v, lap, prob.max_iter, res, False, hist)


class FchSolver:
    """BE steps of Eq. FCH in the physical variable u (internally v = u + 1), 1D."""

    def __init__(self, prob: Problem, eta: float):
        if prob.dim != 1:
            raise ValueError("the FCH oracle is one-dimensional")
        self.prob, self.eta = prob, eta
        self.lap = None

    def step(self, u: np.ndarray, dt: float):
        res = fch_be_step(self.prob, np.asarray(u, dtype=np.float64) + 1.0, dt, self.eta, self.lap)
        self.lap = res.lap_v
        return res.v - 1.0, res


# ---- 2D (the paper's section is the 2D model, solved "by the procedure of Sec. 5.1") ----------
#
# Reading (the paper gives the cube and refers to the 2D splitting for the rest).  Sec. 5.1 replaces
# I - a Lap by the split product M = L_x L_y, L = I - a d_aa, and absorbs the remainder in the
# iteration: I - a Lap = M (I - X) with X = D_x D_y, D_a = H_a - I, H_a = L_a^{-1} (its sign does
# not matter in the product).  All of these commute, so (I - a Lap)^3 = M^3 (I - X)^3 and the BE
# equation (I - a Lap)^3 v = R(v) = v^n + dt Lap g(v) - (3a Lap - 3a^2 Lap^2) v becomes the lagged
#     v^{k+1} = M^{-3} R(v^k) + (1 - (1 - X)^3) v^k,
# the 2D iteration of Sec. 5.1 with three equal factors (it reduces to the 1D one above for X = 0).
# Every Lap comes with an M^{-1}: K = M^{-1} a Lap = D_x H_y + H_x D_y = 2 M^{-1} - H_x - H_y, so
#     v^{k+1} = M^{-1} W^{k+1},
#     W^{k+1} = M^{-2} v^n - 3 M^{-1} K v + (3 + c_eta) K^2 v - c_f K^2 f + c_p M^{-1} K p
#               + (3X - 3X^2 + X^3) W^k,
# with c_eta, c_f, c_p and p as in 1D.  Keeping the iterate as v = M^{-1} W (the lagged term commutes
# with M^{-1}, so (1 - (1-X)^3) v^k = M^{-1} (1 - (1-X)^3) W^k) gives Lap v = K W / a exactly for the
# discrete operators, which the product f' Lap v needs (in 1D, W is z and K W = v - z).  The first
# step starts from W^0 = v^n (v^0 = M^{-1} v^n, Lap v^0 = K v^n / a); later steps carry W.  The
# fixed point does not depend on the start.  One iteration is 26 line sweeps.


@dataclass
class Fch2DResult:
    v: np.ndarray
    w: np.ndarray          # W of the last iterate (v = M^{-1} W)
    lap_v: np.ndarray
    iters: int
    residual: float
    converged: bool
    history: list


def fch2d_be_step(prob: Problem, vn: np.ndarray, dt: float, eta: float, w0=None) -> Fch2DResult:
    """One BE step of Eq. FCH on a 2D grid (ny, nx) by the iteration above; w0 is W from the
    previous step (None for initial data)."""
    eps = prob.eps
    a = (dt * eps ** 4) ** (1.0 / 3.0)
    c_eta, c_f, c_p = dt * eta * eps ** 4 / a ** 2, dt * eps ** 2 / a ** 2, dt / a

    def Hx(g):
        return helmholtz_inverse(g, a, prob.hx, prob.bc, prob.M, axis=1)

    def Hy(g):
        return helmholtz_inverse(g, a, prob.hy, prob.bc, prob.M, axis=0)

    def parts(g):
        """(H_x g, H_y g, M^{-1} g = H_x H_y g)"""
        hy = Hy(g)
        return Hx(g), hy, Hx(hy)

    def K(g):
        """K g = M^{-1} a Lap g = 2 M^{-1} g - H_x g - H_y g, and M^{-1} g"""
        hx, hy, m = parts(g)
        return 2 * m - hx - hy, m

    def X(g):
        """X g = D_x D_y g = M^{-1} g - H_x g - H_y g + g"""
        hx, hy, m = parts(g)
        return m - hx - hy + g

    vn = np.asarray(vn, dtype=np.float64)
    m2_vn = Hx(Hy(Hx(Hy(vn))))
    W = np.array(vn if w0 is None else w0, dtype=np.float64)
    hxw, hyw, v = parts(W)
    lap = (2 * v - hxw - hyw) / a
    xw = v - hxw - hyw + W
    res, hist = np.inf, []
    for k in range(1, prob.max_iter + 1):
        f, fp = f_v(v), fp_v(v)
        p = -eps ** 2 * fp * lap + f * fp - eta * eps ** 2 * f
        kv, _ = K(v)
        kkv, mkv = K(kv)
        kf, _ = K(f)
        kkf, _ = K(kf)
        kp, _ = K(p)
        mkp = Hx(Hy(kp))
        x2w = X(xw)
        x3w = X(x2w)
        W_new = (m2_vn - 3 * mkv + (3 + c_eta) * kkv - c_f * kkf + c_p * mkp
                 + 3 * xw - 3 * x2w + x3w)
        hxw, hyw, v_new = parts(W_new)
        lap = (2 * v_new - hxw - hyw) / a
        xw = v_new - hxw - hyw + W_new
        res = float(np.max(np.abs(v_new - v)))
        hist.append(res)
        v, W = v_new, W_new
        if res < prob.tol:
            return Fch2DResult(v, W, lap, k, res, True, hist)
    return Fch2DResult(v, W, lap, prob.max_iter, res, False, hist)


class Fch2DSolver:
    """BE steps of Eq. FCH in the physical variable u (internally v = u + 1), 2D (ny, nx)."""

    def __init__(self, prob: Problem, eta: float):
        if prob.dim != 2:
            raise ValueError("the 2D FCH oracle needs ny > 1")
        self.prob, self.eta = prob, eta
        self.w = None

    def step(self, u: np.ndarray, dt: float):
        res = fch2d_be_step(self.prob, np.asarray(u, dtype=np.float64) + 1.0, dt, self.eta, self.w)
        self.w = res.w
        return res.v - 1.0, res


__all__ = ["f_v", "fp_v", "fch_be_step", "FchSolver", "FchResult", "fch2d_be_step", "Fch2DSolver",
           "Fch2DResult"]
