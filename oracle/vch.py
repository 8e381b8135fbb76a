"""Vector Cahn-Hilliard (VCH): two components, three phases (Eq. CH_vector, Sec. 5.2).

Test infrastructure only (see ``oracle/__init__.py``).

u = (u1, u2) with u_t = -Lap[eps^2 Lap u - grad_u W(u)] and W(u) = prod_i |u - z_i|^2 over the
cube roots of unity z_i of the (u1, u2) plane (Eq. CH_vector_reaction).  With z = u1 + i u2,
W = |z^3 - 1|^2 and grad W = 2 (z^3 - 1) conj(3 z^2) read as (Re, Im).

The scheme follows Sec. 5.2.  The state is translated about z3 = (-1/2, -sqrt(3)/2),
v = u - z3 (Eq. CH_vector_linearize).  Since the Hessian of W at every z_i is 18 I (Eq. Jacobian),
each component sees the scalar scheme's linear operator with 18 in place of 2:
- Factorization regime, tau >= eps^2/81 (Eq. CH_vector_fixed1):
  c = 9 tau +- sqrt(81 tau^2 - eps^2 tau), so c1 + c2 = 18 tau and c1 c2 = eps^2 tau.
- Completed square, tau < eps^2/81 (Eq. CH_vector_fixed2): c1 = c2 = sqrt(eps^2 tau).

Readings:
- **The lagged term.** Eq. CH_vector_BE prints the right side as v^n + Lap grad W~ without a
  factor dt; the BE step of Eq. CH_vector_linearize carries tau Lap grad W~, which is used here.
  The linear part moved to the left is s v with s = (c1 + c2)/tau, so the lagged term of
  component j is G_j(v) = [grad W(v + z3)]_j - s v_j.  That is W~ of Eq. CH_vector_linearize in
  the factorization regime, and the scalar scheme's completed-square form otherwise.
- **Iteration.** Each component takes the scalar fixed-point map (``solver.fixed_point_map``)
  with that G. Both components' G come from the previous iterate (a Jacobi sweep). Stopping uses
  the larger of the two components' max-norm changes.
- **Boundary conditions.** They apply to v. Dirichlet walls therefore hold u = z3, and periodic
  and Neumann lines are unaffected by the translation.
- **Schemes.** BE, and BDF2 with a BE start, restarted whenever dt changes (as for the scalar
  model).
- **Energy.** The scalar edge / trapezoid rule over both components, with W(u) in place of F(u)
  (Eq. EnergyFunctional_vector).
- **Adaptive steps** (``vch_adaptive_step``): Algorithm 1 with the Richardson or BE-BDF2 estimate,
  as in the paper's vector run (Sec. 6.2.2); readings in its docstring.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .solver import DD, M_inv, PERIODIC, Problem, StepInfo, _edge_sq, trapezoid_weights

Z3 = (-0.5, -np.sqrt(3.0) / 2.0)


def cube_roots():
    """The three minima z_1, z_2, z_3 of W: cube roots of unity as (u1, u2) pairs."""
    return [(np.cos(t), np.sin(t)) for t in (0.0, 2 * np.pi / 3, -2 * np.pi / 3)]


def W(u1, u2):
    """W(u) = |z^3 - 1|^2, z = u1 + i u2 (Eq. CH_vector_reaction)."""
    z = np.asarray(u1, dtype=np.float64) + 1j * np.asarray(u2, dtype=np.float64)
    return np.abs(z ** 3 - 1.0) ** 2


def grad_W(u1, u2):
    """(dW/du1, dW/du2) = (Re, Im) of 2 (z^3 - 1) conj(3 z^2)."""
    z = np.asarray(u1, dtype=np.float64) + 1j * np.asarray(u2, dtype=np.float64)
    g = 2.0 * (z ** 3 - 1.0) * np.conj(3.0 * z ** 2)
    return g.real, g.imag


@dataclass
class VchStageParams:
    regime: str
    c_in: float
    c_out: float
    beta: float     # tau / c_in
    s: float        # (c1 + c2) / tau: the linear part moved to the left


def vch_stage_params(tau: float, eps: float) -> VchStageParams:
    """Eq. CH_vector_fixed1 / CH_vector_fixed2 with dt -> tau."""
    if 81.0 * tau >= eps ** 2:
        disc = np.sqrt(81.0 * tau * tau - eps * eps * tau)
        c1, c2 = 9.0 * tau + disc, 9.0 * tau - disc
        regime = "factor"
    else:
        c1 = c2 = np.sqrt(eps * eps * tau)
        regime = "square"
    c_in, c_out = max(c1, c2), min(c1, c2)
    return VchStageParams(regime, c_in, c_out, tau / c_in, (c1 + c2) / tau)


def G_vec(v1: np.ndarray, v2: np.ndarray, s: float):
    """Lagged terms G_j = [grad W(v + z3)]_j - s v_j."""
    w1, w2 = grad_W(v1 + Z3[0], v2 + Z3[1])
    return w1 - s * v1, w2 - s * v2


def _component_map(prob: Problem, Y: np.ndarray, v: np.ndarray, g: np.ndarray, sp: VchStageParams) -> np.ndarray:
    """The scalar fixed-point map of one component with its lagged term g given."""
    inner = sp.beta * (M_inv(prob, g, sp.c_in) - g + DD(prob, g, sp.c_in))
    out = Y + M_inv(prob, inner, sp.c_out)
    if prob.dim == 2:
        ddi = DD(prob, v, sp.c_in)
        out = out + DD(prob, v, sp.c_out) + ddi - DD(prob, ddi, sp.c_out)
    return out


@dataclass
class VchStageResult:
    v1: np.ndarray
    v2: np.ndarray
    iters: int
    residual: float
    converged: bool


def vch_stage_solve(prob: Problem, r1, r2, v01, v02, tau: float) -> VchStageResult:
    """Solve v - tau F(v) = r for both components by the lagged fixed-point iteration."""
    sp = vch_stage_params(tau, prob.eps)
    Y1 = M_inv(prob, M_inv(prob, r1, sp.c_in), sp.c_out)
    Y2 = M_inv(prob, M_inv(prob, r2, sp.c_in), sp.c_out)
    v1, v2 = np.array(v01, dtype=np.float64), np.array(v02, dtype=np.float64)
    res = np.inf
    for k in range(1, prob.max_iter + 1):
        g1, g2 = G_vec(v1, v2, sp.s)
        n1 = _component_map(prob, Y1, v1, g1, sp)
        n2 = _component_map(prob, Y2, v2, g2, sp)
        res = float(max(np.max(np.abs(n1 - v1)), np.max(np.abs(n2 - v2))))
        v1, v2 = n1, n2
        if res < prob.tol:
            return VchStageResult(v1, v2, k, res, True)
    return VchStageResult(v1, v2, prob.max_iter, res, False)


class VchSolver:
    """BE and BDF2 steps of the vector model in the physical variable u = (u1, u2)."""

    def __init__(self, prob: Problem):
        self.prob = prob
        self.prev = None       # v^{n-1} (both components) for BDF2
        self.dt_prev = None

    def step(self, u1: np.ndarray, u2: np.ndarray, dt: float, scheme: str):
        info = StepInfo()
        v1 = np.asarray(u1, dtype=np.float64) - Z3[0]
        v2 = np.asarray(u2, dtype=np.float64) - Z3[1]
        if scheme == "be" or (scheme == "bdf2" and (self.prev is None or self.dt_prev != dt)):
            res = vch_stage_solve(self.prob, v1, v2, v1, v2, dt)
        elif scheme == "bdf2":
            p1, p2 = self.prev
            res = vch_stage_solve(self.prob, (4.0 * v1 - p1) / 3.0, (4.0 * v2 - p2) / 3.0, v1, v2, 2.0 * dt / 3.0)
        else:
            raise ValueError(scheme)
        info.iters.append(res.iters)
        info.residual = res.residual
        info.converged = res.converged
        self.prev, self.dt_prev = (v1, v2), dt
        return res.v1 + Z3[0], res.v2 + Z3[1], info


def vch_energy(prob: Problem, u1: np.ndarray, u2: np.ndarray) -> float:
    """Discrete VCH energy (Eq. EnergyFunctional_vector) by the scalar edge / trapezoid rule."""
    u1 = np.asarray(u1, dtype=np.float64).reshape(prob.ny, prob.nx)
    u2 = np.asarray(u2, dtype=np.float64).reshape(prob.ny, prob.nx)
    wx = trapezoid_weights(prob.nx, prob.bc)
    pot = W(u1, u2)
    eps2 = prob.eps ** 2
    if prob.dim == 1:
        grad = sum(np.sum(_edge_sq(u[0], 0, prob.bc)) for u in (u1, u2)) / prob.hx ** 2
        return prob.hx * (0.5 * eps2 * grad + np.sum(wx * pot[0]))
    wy = trapezoid_weights(prob.ny, prob.bc)
    gx = sum(np.sum(wy[:, None] * _edge_sq(u, 1, prob.bc)) for u in (u1, u2)) / prob.hx ** 2
    gy = sum(np.sum(wx[None, :] * _edge_sq(u, 0, prob.bc)) for u in (u1, u2)) / prob.hy ** 2
    return prob.hx * prob.hy * (0.5 * eps2 * (gx + gy) + np.sum(wy[:, None] * wx[None, :] * pot))


def vch_adaptive_step(solver: VchSolver, u1, u2, dt: float, tol: float, dt_min: float, dt_max: float,
                      theta: float = 0.8, gamma: float = 1.3, estimator: str = "bdf2", history: dict | None = None):
    """One accepted step of the vector model under Algorithm 1 (Sec. 5), as the paper runs it in
    Sec. 6.2.2.  Returns (u1, u2, AdaptiveInfo).

    Readings:
    - **Estimators.** "richardson": BE with two half steps, eta = (1/2) max|u_dt - u_dt/2| over both
      components; the half-step solution is kept.  "bdf2" (BE-BDF2): one BE step and one
      variable-step BDF2 step from the previous accepted state; eta = max|u_BDF2 - u_BE| and the
      BDF2 solution is kept.
    - **First step.** The vector model has no SDC2 here, so a BE-BDF2 step without history takes
      the Richardson estimate.
    - **History.** ``history`` is a dict holding the previous accepted state ("u1", "u2") and its
      step ("dt"); an accepted step updates it.
    """
    from .adaptive import AdaptiveInfo, bdf2_variable, decide
    if estimator not in ("richardson", "bdf2"):
        raise ValueError(estimator)
    if estimator == "bdf2" and history is None:
        raise ValueError("the BE-BDF2 estimate needs a history dict")
    prob = solver.prob
    rejections = 0
    while True:
        if estimator == "bdf2" and history.get("u1") is not None:
            b1, b2, ib = VchSolver(prob).step(u1, u2, dt, "be")
            tau, a_n, a_prev = bdf2_variable(dt, history["dt"])
            v1, v2 = np.asarray(u1, dtype=np.float64) - Z3[0], np.asarray(u2, dtype=np.float64) - Z3[1]
            p1, p2 = history["u1"] - Z3[0], history["u2"] - Z3[1]
            res = vch_stage_solve(prob, a_n * v1 + a_prev * p1, a_n * v2 + a_prev * p2, v1, v2, tau)
            c1, c2 = res.v1 + Z3[0], res.v2 + Z3[1]
            eta = float(max(np.max(np.abs(c1 - b1)), np.max(np.abs(c2 - b2))))
            n_it = max(ib.iters[0], res.iters)
        else:
            f1, f2, i1 = VchSolver(prob).step(u1, u2, dt, "be")
            h1, h2, i2 = VchSolver(prob).step(u1, u2, 0.5 * dt, "be")
            c1, c2, i3 = VchSolver(prob).step(h1, h2, 0.5 * dt, "be")
            eta = 0.5 * float(max(np.max(np.abs(f1 - c1)), np.max(np.abs(f2 - c2))))
            n_it = max(i1.iters[0], i2.iters[0], i3.iters[0])
        ok, dt_next = decide(eta, tol, n_it, prob.max_iter, dt, theta, gamma)
        dt_next = min(max(dt_next, dt_min), dt_max)
        if ok:
            if history is not None:
                history.update(u1=np.array(u1, dtype=np.float64), u2=np.array(u2, dtype=np.float64), dt=dt)
            return c1, c2, AdaptiveInfo(dt, dt_next, eta, rejections, n_it)
        rejections += 1
        if dt <= dt_min:
            raise RuntimeError("adaptive step: dt reached dt_min without meeting the LTE tolerance")
        dt = dt_next


__all__ = ["Z3", "cube_roots", "W", "grad_W", "vch_stage_params", "G_vec", "vch_stage_solve", "VchSolver",
           "vch_energy", "vch_adaptive_step", "PERIODIC"]
