"""Adaptive time-step control of Sec. 5 (Algorithm 1) over the oracle's time schemes.

Test infrastructure only: the CUDA path never imports this module.

One call advances u by one accepted step. Two local truncation error (LTE) estimates of Sec. 5
are available:
- "richardson": Backward Euler by Richardson extrapolation (Algorithm 1, step 1). One BE step of
  size dt and two of size dt/2, eta = (1/2) ||u_dt - u_dt/2||_inf.
- "sdc2": BE-SDC2. One SDC2 step from a fresh start; eta = ||u^[1] - u^[0]||_inf, the
  difference of its first-order level [0] (BE) and its second-order level [1].
- "bdf2": BE-BDF2. One BE step and one variable-step BDF2 step over the same interval, from the
  previous accepted state; eta = ||u_BDF2 - u_BE||_inf.

Readings (the algorithm leaves these open):
- **Accepted solution.** Richardson keeps the two-half-step solution, SDC2 level [1] and BDF2 the
  BDF2 solution: in each case the more accurate of the two.
- **BDF2 with varying steps.** Steps change size nearly every time, so BE-BDF2 uses the
  variable-step BDF2 formula (bdf2_variable below); with equal steps it is the fixed-step Eq. BDF2.
  Its history is the state before the last accepted step and that step's size, kept in an
  AdaptiveHistory. Without history (the first step) the attempt uses the BE-SDC2 estimate.
- **N_it.** The largest fixed-point iteration count of the stage solves of the attempt;
  N_maxit is the problem's max_iter.
- **Limits.** The proposed next step is clipped to [dt_min, dt_max]. A rejected step that would
  fall below dt_min is an error.
- **eta = 0.** Then sqrt(sigma_tol / eta) is taken as infinite, so the growth factor is the cap.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .solver import OracleSolver, stage_solve


@dataclass
class AdaptiveInfo:
    dt_used: float
    dt_next: float
    eta: float
    rejections: int
    max_iters: int


def decide(eta: float, tol: float, n_it: int, n_maxit: int, dt: float, theta: float = 0.8, gamma: float = 1.3):
    """Step-size decision of Algorithm 1: (accepted, next dt) for an attempt of size dt whose LTE
    estimate is eta.  A step that meets the tolerance is kept unless its fixed-point iteration hit
    the cap; it grows by the LTE proposal theta sqrt(tol/eta), at most by gamma when the iteration
    used under 70% of its cap and not at all above that.  A failed step shrinks by gamma when the
    iteration hit its cap or eta exceeds twice the tolerance, and takes the LTE proposal otherwise."""
    ratio = math.inf if eta == 0.0 else math.sqrt(tol / eta)
    if eta <= tol:
        frac = n_it / n_maxit
        if frac < 0.7:
            return True, dt * min(theta * ratio, gamma)
        if frac < 1.0:
            return True, dt * min(theta * ratio, 1.0)
        return False, dt / gamma
    if eta / tol > 2.0:
        return False, dt / gamma
    return False, dt * theta * ratio


@dataclass
class AdaptiveHistory:
    """The state before the last accepted step and that step's size (BE-BDF2 only)."""
    u_prev: np.ndarray | None = None
    dt_prev: float | None = None


def bdf2_variable(dt: float, dt_prev: float):
    """Variable-step BDF2 as one stage v - tau F(v) = a_n u^n + a_prev u^{n-1}: (tau, a_n, a_prev).

    With omega = dt / dt_prev it is the quadratic through (t_{n-1}, u^{n-1}), (t_n, u^n),
    (t_{n+1}, u^{n+1}) whose slope at t_{n+1} is F(u^{n+1}):
      tau = dt (1 + omega) / (1 + 2 omega),
      a_n = (1 + omega)^2 / (1 + 2 omega),  a_prev = -omega^2 / (1 + 2 omega).
    """
    om = dt / dt_prev
    return dt * (1.0 + om) / (1.0 + 2.0 * om), (1.0 + om) ** 2 / (1.0 + 2.0 * om), -om * om / (1.0 + 2.0 * om)


def _attempt(solver: OracleSolver, u: np.ndarray, dt: float, estimator: str, history: AdaptiveHistory | None):
    """One attempt of size dt: (candidate solution, eta, N_it)."""
    if estimator == "richardson":
        u_full, i_full = solver.step(u, dt, "be")
        u_half, i_h1 = solver.step(u, 0.5 * dt, "be")
        u_half, i_h2 = solver.step(u_half, 0.5 * dt, "be")
        eta = 0.5 * float(np.max(np.abs(u_full - u_half)))
        return u_half, eta, max(max(i_full.iters), max(i_h1.iters), max(i_h2.iters))
    if estimator == "bdf2" and history.u_prev is not None:
        u_be, i_be = solver.step(u, dt, "be")
        tau, a_n, a_prev = bdf2_variable(dt, history.dt_prev)
        v = np.asarray(u, dtype=np.float64) + 1.0
        r = a_n * v + a_prev * (np.asarray(history.u_prev, dtype=np.float64) + 1.0)
        res = stage_solve(solver.prob, r, v, tau)
        u_bdf = res.v - 1.0
        return u_bdf, float(np.max(np.abs(u_bdf - u_be))), max(max(i_be.iters), res.iters)
    if estimator in ("sdc2", "bdf2"):
        solver.sdc_v0 = None                     # fresh start: level [0] from u itself
        u1, info = solver.step(u, dt, "sdc2")
        u0 = solver.sdc_v0 - 1.0                 # level [0] (BE) value, physical variable
        return u1, float(np.max(np.abs(u1 - u0))), max(info.iters)
    raise ValueError(estimator)


def adaptive_step(solver: OracleSolver, u: np.ndarray, dt: float, tol: float, dt_min: float, dt_max: float,
                  theta: float = 0.8, gamma: float = 1.3, estimator: str = "richardson",
                  history: AdaptiveHistory | None = None):
    """Advance u by one accepted step whose LTE estimate meets tol (Algorithm 1).

    estimator "bdf2" needs a history, which an accepted step updates."""
    if estimator not in ("richardson", "sdc2", "bdf2"):
        raise ValueError(estimator)
    if estimator == "bdf2" and history is None:
        raise ValueError("the BE-BDF2 estimate needs an AdaptiveHistory")
    rejections = 0
    while True:
        cand, eta, n_it = _attempt(solver, u, dt, estimator, history)
        ok, dt_next = decide(eta, tol, n_it, solver.prob.max_iter, dt, theta, gamma)
        dt_next = min(max(dt_next, dt_min), dt_max)
        if ok:
            if history is not None:
                history.u_prev, history.dt_prev = np.array(u, dtype=np.float64), dt
            return cand, AdaptiveInfo(dt, dt_next, eta, rejections, n_it)
        rejections += 1
        if dt <= dt_min:
            raise RuntimeError("adaptive step: dt reached dt_min without meeting the LTE tolerance")
        dt = dt_next
