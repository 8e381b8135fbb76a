"""The sixth-order (functionalized) Cahn-Hilliard model of the paper's last section, 1D, FP64.

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


__all__ = ["f_v", "fp_v", "fch_be_step", "FchSolver", "FchResult"]
