"""Adaptive time-step control of Sec. 5 (Algorithm 1) over the oracle's time schemes.

Test infrastructure only: the CUDA path never imports this module.

One call advances u by one accepted step. The local truncation error (LTE) estimate is
Richardson extrapolation with Backward Euler (Algorithm 1, step 1): one BE step of size dt and
two of size dt/2, eta = (1/2) ||u_dt - u_dt/2||_inf.

Readings (the algorithm leaves these open):
- **Accepted solution.** The two-half-step solution, the more accurate of the two.
- **N_it.** The largest fixed-point iteration count of the three stage solves of the attempt;
  N_maxit is the problem's max_iter.
- **Limits.** The proposed next step is clipped to [dt_min, dt_max]. A rejected step that would
  fall below dt_min is an error.
- **eta = 0.** Then sqrt(sigma_tol / eta) is taken as infinite, so the growth factor is the cap.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from .solver import OracleSolver


@dataclass
class AdaptiveInfo:
    dt_used: float
    dt_next: float
    eta: float
    rejections: int
    max_iters: int


def decide(eta: float, tol: float, n_it: int, n_maxit: int, dt: float, theta: float = 0.8, gamma: float = 1.3):
    """Algorithm 1, step 2: (accepted, next dt) for an attempt of size dt with LTE estimate eta."""
    ratio = math.inf if eta == 0.0 else math.sqrt(tol / eta)
    if eta <= tol:                                    # case (I)
        frac = n_it / n_maxit
        if frac < 0.7:
            return True, dt * min(theta * ratio, gamma)
        if frac < 1.0:
            return True, dt * min(theta * ratio, 1.0)
        return False, dt / gamma                      # step fails: the iteration hit its cap
    if eta / tol > 2.0:                               # case (II): step fails
        return False, dt / gamma
    return False, dt * theta * ratio


def adaptive_step(solver: OracleSolver, u: np.ndarray, dt: float, tol: float, dt_min: float, dt_max: float,
                  theta: float = 0.8, gamma: float = 1.3):
    """Advance u by one accepted BE step whose Richardson LTE estimate meets tol (Algorithm 1)."""
    rejections = 0
    while True:
        u_full, i_full = solver.step(u, dt, "be")
        u_half, i_h1 = solver.step(u, 0.5 * dt, "be")
        u_half, i_h2 = solver.step(u_half, 0.5 * dt, "be")
        eta = 0.5 * float(np.max(np.abs(u_full - u_half)))
        n_it = max(max(i_full.iters), max(i_h1.iters), max(i_h2.iters))
        ok, dt_next = decide(eta, tol, n_it, solver.prob.max_iter, dt, theta, gamma)
        dt_next = min(max(dt_next, dt_min), dt_max)
        if ok:
            return u_half, AdaptiveInfo(dt, dt_next, eta, rejections, n_it)
        rejections += 1
        if dt <= dt_min:
            raise RuntimeError("adaptive step: dt reached dt_min without meeting the LTE tolerance")
        dt = dt_next
