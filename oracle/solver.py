"""Stage parameters, fixed-point stage solves, time schemes and discrete energy / mass (Sec. 3-5).

Test infrastructure only (see ``oracle/__init__.py``).

Every stage of every scheme solves  v - tau F(v) = r  with
F(v) = -eps^2 Lap^2 v + Lap f(v - 1),  f(v - 1) = v^3 - 3v^2 + 2v  (Eq. CahnHilliard_v),
in the shifted variable v = u + 1 (Sec. 3).

Readings (the paper leaves these open, or prints them with a slip):
* One G for both regimes.  The linear part of f moved to the left is s v with
  (I - c1 Lap)(I - c2 Lap) = I - s tau Lap + eps^2 tau Lap^2, so c1 c2 = eps^2 tau,
  c1 + c2 = s tau and the lagged term is G(v) = v^3 - 3v^2 + (2 - (c1+c2)/tau) v.
  Factorization regime (tau >= eps^2, Eq. CH_BE_fixed2_factor): c = tau +- sqrt(tau^2 - eps^2 tau),
  G = f~.  Completed square (tau < eps^2, Eq. CH_BE_fixed_complete): c1 = c2 = sqrt(eps^2 tau),
  G = f(v-1) - 2 sqrt(eps^2/tau) v.  (Eq. CH_BE_fixed_complete prints
  f~ - 2(1 + sqrt(eps^2/dt)) v, whose fixed point is not Eq. CH_BE; the sign read
  here agrees with the 2D Eq. CH_BE_2D and the SDC Eq. SDC2_fixed.)
* The inner inversion (the one that carries Lap G through Remark Laplacian) is
  the larger c, so beta = tau / c_in <= 1.
* 1D iteration:  v^{k+1} = H_o[ H_i[r + beta G(v^k)] - beta G(v^k) ].
* 2D iteration (Sec. 5.1, generalised to c_o != c_i):
      v^{k+1} = Y + M_o^{-1}[ beta (M_i^{-1} G - G + D_ix D_iy G) ]
                  + (D_ox D_oy + D_ix D_iy - D_ox D_oy D_ix D_iy) v^k,
  Y = M_o^{-1} M_i^{-1} r, M^{-1} = H_x H_y, D = I - H.  With c_o = c_i it is
  Eq. CH_BE_2D_3 with C1, C2 of Eq. CH_2D_Doperator1/2.
* Stopping: ||v^{k+1} - v^k||_inf < tol (Sec. 4.4) or k = max_iter; the
  result is v^{k+1}; the first guess is the previous time level (or stage).
* SDIRK in stage-value form: V_i - eta dt F(V_i) = v^n + dt sum_{l<i} a_il K_l,
  K_l = (V_l - R_l)/(eta dt), v^{n+1} = V_s (both tableaus are stiffly accurate).
  SDIRK2 tableau from Sec. 4.2; SDIRK3 is Alexander's three-stage L-stable
  method with eta the root of x^3 - 3x^2 + 3x/2 - 1/6 near 0.4359 (the value
  Sec. 4.4 quotes).
* BDF2 (Eq. BDF2) starts with one BE step and restarts that way whenever dt
  changes.  The paper does not say how BDF2 starts; a BE start reproduces its
  BDF2 refinement column (Table CH_refinement_second) digit for digit, while
  an SDIRK2 start does not.
* SDC2 (Sec. 4.3, Eq. IDC_BE_j with P = 1, Eq. SDC_fixed): level [0] is a BE
  trajectory and level [1] solves
      v1_{n+1} - dt F(v1_{n+1}) = v1_n - (dt/2)(F0_{n+1} - F0_n),
  both advanced together one step at a time (the paper runs level [0] over all
  of [0, T] first; advancing both levels together gives the same numbers).
  F0_{n+1} = (v0_{n+1} - v0_n)/dt is the level-[0] BE identity; F0 at the
  first step is F(v^n) taken inside the inverse through Remark Laplacian /
  biLaplacian: M_o^{-1}M_i^{-1}F(v) = -(eps^2/(c_i c_o)) E_o E_i v + (1/c_i) M_o^{-1} E_i f(v-1),
  E = M^{-1} - I + D_x D_y (E = H - I in 1D).  This reproduces the paper's SDC2
  refinement column (Table CH_refinement_second) digit for digit.
* Energy (Eq. EnergyFunctional): h_x h_y [ sum over grid edges of
  eps^2/2 (forward difference / h)^2 weighted by the trapezoid weight of the
  other direction + sum over nodes of trapezoid-weighted F(u) ], F(u) = (u^2-1)^2/4;
  trapezoid weights are 1/2 on non-periodic wall nodes.  Mass = h_x h_y sum w u.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .helmholtz import PERIODIC, helmholtz_inverse


@dataclass
class Problem:
    """A CH instance: dim 1 uses shape (1, nx); dim 2 uses shape (ny, nx), x along the last axis."""
    nx: int
    ny: int = 1
    Lx: float = 2 * np.pi
    Ly: float = 2 * np.pi
    bc: str = PERIODIC
    eps: float = 0.18
    M: int = 4
    tol: float = 1e-10
    max_iter: int = 500

    @property
    def dim(self) -> int:
        return 1 if self.ny == 1 else 2

    @property
    def hx(self) -> float:
        return self.Lx / (self.nx if self.bc == PERIODIC else self.nx - 1)

    @property
    def hy(self) -> float:
        return self.Ly / (self.ny if self.bc == PERIODIC else self.ny - 1)


@dataclass
class StageParams:
    regime: str
    c_in: float
    c_out: float
    beta: float
    lam: float


def stage_params(tau: float, eps: float) -> StageParams:
    """Regime switch and Helmholtz parameters (Sec. 3.1.2; Sec. 4.1-4.2 with dt -> tau)."""
    if tau >= eps ** 2:
        disc = np.sqrt(tau * tau - eps * eps * tau)
        c1, c2 = tau + disc, tau - disc
        regime = "factor"
    else:
        c1 = c2 = np.sqrt(eps * eps * tau)
        regime = "square"
    c_in, c_out = max(c1, c2), min(c1, c2)
    return StageParams(regime, c_in, c_out, tau / c_in, 2.0 - (c1 + c2) / tau)


def G(v: np.ndarray, lam: float) -> np.ndarray:
    """Lagged nonlinear term v^3 - 3v^2 + lam v."""
    return v ** 3 - 3 * v ** 2 + lam * v


@dataclass
class StageResult:
    v: np.ndarray
    iters: int
    residual: float
    converged: bool
    history: list = field(default_factory=list)   # residual after each iteration

    def contraction(self, last: int = 5) -> float:
        """Observed contraction factor: geometric mean of the last residual ratios."""
        h = [r for r in self.history if r > 0]
        if len(h) < 2:
            return 0.0
        h = h[-(last + 1):]
        return float((h[-1] / h[0]) ** (1.0 / (len(h) - 1)))


def _H(prob: Problem, f: np.ndarray, c: float, axis: str) -> np.ndarray:
    if axis == "x":
        return helmholtz_inverse(f, c, prob.hx, prob.bc, prob.M, axis=1)
    return helmholtz_inverse(f, c, prob.hy, prob.bc, prob.M, axis=0)


def M_inv(prob: Problem, f: np.ndarray, c: float) -> np.ndarray:
    """(L_x L_y)^{-1} f = H_x H_y f in 2D, H_x f in 1D (Eq. 2D_Helmholtz)."""
    if prob.dim == 1:
        return _H(prob, f, c, "x")
    return _H(prob, _H(prob, f, c, "y"), c, "x")


def DD(prob: Problem, f: np.ndarray, c: float) -> np.ndarray:
    """D_x D_y f with D = I - H (Eq. CH_2D_Doperator1); zero in 1D."""
    if prob.dim == 1:
        return np.zeros_like(f)
    dy = f - _H(prob, f, c, "y")
    return dy - _H(prob, dy, c, "x")


def stage_rhs_inverse(prob: Problem, r: np.ndarray, sp: StageParams) -> np.ndarray:
    """Y = M_o^{-1} M_i^{-1} r."""
    return M_inv(prob, M_inv(prob, r, sp.c_in), sp.c_out)


def fixed_point_map(prob: Problem, Y: np.ndarray, v: np.ndarray, sp: StageParams) -> np.ndarray:
    """One fixed-point iteration (1D: Eq. CH_BE_fixed2_factor / _complete; 2D: Sec. 5.1)."""
    g = G(v, sp.lam)
    inner = sp.beta * (M_inv(prob, g, sp.c_in) - g + DD(prob, g, sp.c_in))
    out = Y + M_inv(prob, inner, sp.c_out)
    if prob.dim == 2:
        ddi = DD(prob, v, sp.c_in)
        out = out + DD(prob, v, sp.c_out) + ddi - DD(prob, ddi, sp.c_out)
    return out


def inverse_of_F(prob: Problem, v: np.ndarray, sp: StageParams) -> np.ndarray:
    """M_o^{-1} M_i^{-1} F(v) without explicit derivatives (Remark Laplacian, Remark biLaplacian)."""
    def E(f, c):
        return M_inv(prob, f, c) - f + DD(prob, f, c)
    f = v ** 3 - 3 * v ** 2 + 2 * v
    return (-(prob.eps ** 2) / (sp.c_in * sp.c_out) * E(E(v, sp.c_in), sp.c_out)
            + M_inv(prob, E(f, sp.c_in), sp.c_out) / sp.c_in)


def stage_solve(prob: Problem, r: np.ndarray, v0: np.ndarray, tau: float, Y: np.ndarray = None) -> StageResult:
    """Solve v - tau F(v) = r by the lagged fixed-point iteration (Y = M_o^{-1}M_i^{-1} r if given)."""
    sp = stage_params(tau, prob.eps)
    if Y is None:
        Y = stage_rhs_inverse(prob, r, sp)
    v = np.array(v0, dtype=np.float64)
    res = np.inf
    hist = []
    for k in range(1, prob.max_iter + 1):
        v_new = fixed_point_map(prob, Y, v, sp)
        res = float(np.max(np.abs(v_new - v)))
        hist.append(res)
        v = v_new
        if res < prob.tol:
            return StageResult(v, k, res, True, hist)
    return StageResult(v, prob.max_iter, res, False, hist)


ETA2 = 1.0 - np.sqrt(2.0) / 2.0


def _alexander_eta() -> float:
    """Root of x^3 - 3x^2 + 3x/2 - 1/6 in (0.4, 0.5) by bisection."""
    lo, hi = 0.4, 0.5
    p = lambda x: x ** 3 - 3 * x ** 2 + 1.5 * x - 1.0 / 6.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if p(lo) * p(mid) <= 0:
            hi = mid
        else:
            lo = mid
    return 0.5 * (lo + hi)


ETA3 = _alexander_eta()

SDIRK2 = np.array([[ETA2, 0.0], [1.0 - ETA2, ETA2]])
SDIRK3 = np.array([
    [ETA3, 0.0, 0.0],
    [(1.0 - ETA3) / 2.0, ETA3, 0.0],
    [-(6 * ETA3 ** 2 - 16 * ETA3 + 1) / 4.0, (6 * ETA3 ** 2 - 20 * ETA3 + 5) / 4.0, ETA3],
])


@dataclass
class StepInfo:
    iters: list = field(default_factory=list)
    residual: float = 0.0
    converged: bool = True
    contraction: float = 0.0      # largest observed contraction factor over the stages


class OracleSolver:
    """Time stepping in the physical variable u; internally v = u + 1."""

    def __init__(self, prob: Problem):
        self.prob = prob
        self.v_prev = None      # v^{n-1} for BDF2 / BDF3
        self.dt_prev = None
        self.v_prev2 = None     # v^{n-2} for BDF3
        self.dt_prev2 = None
        self.sdc_v0 = None      # level-[0] value v0_n for SDC2
        self.sdc_F0 = None      # level-[0] F0_n (a field) for SDC2

    def _record(self, info: StepInfo, res: StageResult):
        info.iters.append(res.iters)
        info.residual = max(info.residual, res.residual)
        info.converged = info.converged and res.converged
        info.contraction = max(info.contraction, res.contraction())

    def _sdirk(self, v: np.ndarray, dt: float, A: np.ndarray, info: StepInfo) -> np.ndarray:
        eta = A[0, 0]
        K = []
        guess = v
        for i in range(A.shape[0]):
            R = v + dt * sum(A[i, l] * K[l] for l in range(i)) if i else v.copy()
            res = stage_solve(self.prob, R, guess, eta * dt)
            self._record(info, res)
            K.append((res.v - R) / (eta * dt))
            guess = res.v
        return guess

    def _sdc2(self, v: np.ndarray, dt: float, info: StepInfo) -> np.ndarray:
        prob = self.prob
        sp = stage_params(dt, prob.eps)
        start = self.sdc_v0 is None or self.dt_prev != dt
        v0n = v if start else self.sdc_v0
        lvl0 = stage_solve(prob, v0n, v0n, dt)                 # level [0]: BE
        self._record(info, lvl0)
        F1 = (lvl0.v - v0n) / dt
        if start:
            Y = stage_rhs_inverse(prob, v, sp) - 0.5 * dt * (stage_rhs_inverse(prob, F1, sp)
                                                            - inverse_of_F(prob, v0n, sp))
        else:
            Y = stage_rhs_inverse(prob, v - 0.5 * dt * (F1 - self.sdc_F0), sp)
        lvl1 = stage_solve(prob, None, lvl0.v, dt, Y=Y)        # level [1]
        self._record(info, lvl1)
        self.sdc_v0, self.sdc_F0 = lvl0.v, F1
        return lvl1.v

    def step(self, u: np.ndarray, dt: float, scheme: str):
        info = StepInfo()
        v = np.asarray(u, dtype=np.float64) + 1.0
        if scheme == "be":
            res = stage_solve(self.prob, v, v, dt)
            self._record(info, res)
            v_new = res.v
        elif scheme == "sdirk2":
            v_new = self._sdirk(v, dt, SDIRK2, info)
        elif scheme == "sdirk3":
            v_new = self._sdirk(v, dt, SDIRK3, info)
        elif scheme == "bdf2":
            if self.v_prev is None or self.dt_prev != dt:
                res = stage_solve(self.prob, v, v, dt)
                self._record(info, res)
                v_new = res.v
            else:
                r = (4.0 * v - self.v_prev) / 3.0
                res = stage_solve(self.prob, r, v, 2.0 * dt / 3.0)
                self._record(info, res)
                v_new = res.v
        elif scheme == "bdf3":
            # Eq. BDF3: tau = 6 dt / 11, r = (18 v^n - 9 v^{n-1} + 2 v^{n-2}) / 11; its two
            # starting steps (and a restart after any dt change) are SDIRK2 steps (Sec. 4.4)
            if self.v_prev is None or self.v_prev2 is None or self.dt_prev != dt or self.dt_prev2 != dt:
                v_new = self._sdirk(v, dt, SDIRK2, info)
            else:
                r = (18.0 * v - 9.0 * self.v_prev + 2.0 * self.v_prev2) / 11.0
                res = stage_solve(self.prob, r, v, 6.0 * dt / 11.0)
                self._record(info, res)
                v_new = res.v
        elif scheme == "sdc2":
            v_new = self._sdc2(v, dt, info)
        else:
            raise ValueError(scheme)
        if scheme != "sdc2":
            self.sdc_v0 = None
        self.v_prev2, self.dt_prev2 = self.v_prev, self.dt_prev
        self.v_prev, self.dt_prev = v, dt
        return v_new - 1.0, info


def trapezoid_weights(n: int, bc: str) -> np.ndarray:
    w = np.ones(n)
    if bc != PERIODIC:
        w[0] = w[-1] = 0.5
    return w


def _edge_sq(u: np.ndarray, axis: int, bc: str) -> np.ndarray:
    if bc == PERIODIC:
        return (np.roll(u, -1, axis=axis) - u) ** 2
    return np.diff(u, axis=axis) ** 2


def energy(prob: Problem, u: np.ndarray) -> float:
    """Discrete CH free energy (Eq. EnergyFunctional) by the edge / trapezoid rule above."""
    u = np.asarray(u, dtype=np.float64).reshape(prob.ny, prob.nx)
    wx = trapezoid_weights(prob.nx, prob.bc)
    F = 0.25 * (u ** 2 - 1.0) ** 2
    eps2 = prob.eps ** 2
    if prob.dim == 1:
        grad = np.sum(_edge_sq(u[0], 0, prob.bc)) / prob.hx ** 2
        return prob.hx * (0.5 * eps2 * grad + np.sum(wx * F[0]))
    wy = trapezoid_weights(prob.ny, prob.bc)
    gx = np.sum(wy[:, None] * _edge_sq(u, 1, prob.bc)) / prob.hx ** 2
    gy = np.sum(wx[None, :] * _edge_sq(u, 0, prob.bc)) / prob.hy ** 2
    return prob.hx * prob.hy * (0.5 * eps2 * (gx + gy) + np.sum(wy[:, None] * wx[None, :] * F))


def mass(prob: Problem, u: np.ndarray) -> float:
    """Trapezoid-weighted integral of u."""
    u = np.asarray(u, dtype=np.float64).reshape(prob.ny, prob.nx)
    wx = trapezoid_weights(prob.nx, prob.bc)
    if prob.dim == 1:
        return prob.hx * float(np.sum(wx * u[0]))
    wy = trapezoid_weights(prob.ny, prob.bc)
    return prob.hx * prob.hy * float(np.sum(wy[:, None] * wx[None, :] * u))
