"""Pins for the adaptive step-size control (Sec. 5, Algorithm 1) in the oracle: properties of the
Richardson, BE-SDC2 and BE-BDF2 LTE estimates, of the variable-step BDF2 formula and of the
controller that hold independently of the oracle's code."""
import numpy as np
import pytest

from oracle.adaptive import adaptive_step, decide
from oracle.solver import OracleSolver, Problem
from paper_1611_04214_gb300.inputs import paper_ic_1d


def test_richardson_estimate_scales_as_dt_squared():
    # BE has local error O(dt^2); eta = |u_dt - u_dt/2| / 2 estimates it, so halving dt divides
    # eta by a factor that tends to 4 (the stiff initial transient keeps it a little below).
    prob = Problem(nx=128, eps=0.18, M=6, tol=1e-13, max_iter=3000)
    u = paper_ic_1d(128)[None, :]
    etas = []
    for dt in (2e-4, 1e-4, 5e-5):
        s = OracleSolver(prob)
        full, _ = s.step(u, dt, "be")
        half, _ = s.step(u, dt / 2, "be")
        half, _ = s.step(half, dt / 2, "be")
        etas.append(0.5 * np.abs(full - half).max())
    r1, r2 = etas[0] / etas[1], etas[1] / etas[2]
    assert 3.6 < r1 < 4.2 and 3.75 < r2 < 4.15 and r2 > r1, (r1, r2)   # -> 4 from below


def test_controller_cases_of_algorithm_1():
    tol, dt = 1e-4, 0.5
    # (I) accurate, few iterations: grow by theta sqrt(tol/eta), capped at gamma = 1.3
    ok, nxt = decide(tol / 100, tol, 10, 600, dt)
    assert ok and nxt == pytest.approx(dt * 1.3)
    ok, nxt = decide(tol / 1.2, tol, 10, 600, dt)
    assert ok and nxt == pytest.approx(dt * 0.8 * np.sqrt(1.2))
    # (I) accurate but 0.7 <= N_it / N_maxit < 1: no growth beyond 1
    ok, nxt = decide(tol / 100, tol, 500, 600, dt)
    assert ok and nxt == pytest.approx(dt)
    # (I) iteration cap reached: fail, dt / gamma
    ok, nxt = decide(tol / 100, tol, 600, 600, dt)
    assert not ok and nxt == pytest.approx(dt / 1.3)
    # (II) inaccurate: fail; far off -> dt / gamma, near -> theta sqrt(tol/eta)
    ok, nxt = decide(3 * tol, tol, 10, 600, dt)
    assert not ok and nxt == pytest.approx(dt / 1.3)
    ok, nxt = decide(1.5 * tol, tol, 10, 600, dt)
    assert not ok and nxt == pytest.approx(dt * 0.8 * np.sqrt(1 / 1.5))


def test_adaptive_steps_meet_the_tolerance_and_grow_in_slow_phases():
    # From the stiff initial state the accepted steps must satisfy eta <= tol, and the step
    # size must grow as the fast spinodal transient decays.
    prob = Problem(nx=128, eps=0.18, M=6, tol=1e-11, max_iter=600)
    s = OracleSolver(prob)
    u = paper_ic_1d(128)[None, :]
    dt, t, tol = 1e-3, 0.0, 1e-4
    dts = []
    for _ in range(25):
        u, info = adaptive_step(s, u, dt, tol, 1e-6, 10.0)
        assert info.eta <= tol
        t += info.dt_used
        dts.append(info.dt_used)
        dt = info.dt_next
    assert dts[-1] > 2 * dts[0]


def test_sdc2_level_difference_scales_as_dt_squared():
    # Level [0] (BE) has local error O(dt^2) and level [1] O(dt^3), so their difference after one
    # step from the same state falls like dt^2.
    prob = Problem(nx=128, eps=0.18, M=6, tol=1e-13, max_iter=3000)
    u = paper_ic_1d(128)[None, :]
    etas = []
    for dt in (2e-4, 1e-4, 5e-5):
        s = OracleSolver(prob)
        u1, info = s.step(u, dt, "sdc2")
        etas.append(np.abs(u1 - (s.sdc_v0 - 1.0)).max())
    r1, r2 = etas[0] / etas[1], etas[1] / etas[2]
    assert 3.5 < r1 < 4.2 and 3.7 < r2 < 4.15, (r1, r2)


def test_variable_bdf2_exact_on_quadratics():
    # BDF2 with any step ratio reproduces every polynomial of degree <= 2 in t: with u = p(t),
    # u' = p'(t), the stage relation u^{n+1} - tau u'(t_{n+1}) = a_n u^n + a_prev u^{n-1} holds.
    from oracle.adaptive import bdf2_variable
    rng = np.random.default_rng(5)
    for _ in range(20):
        dt, dt_prev, t = rng.uniform(0.05, 2.0), rng.uniform(0.05, 2.0), rng.uniform(-1.0, 1.0)
        tau, a_n, a_prev = bdf2_variable(dt, dt_prev)
        for c in ([1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0], list(rng.normal(size=3))):
            p = np.polynomial.Polynomial(c)
            lhs = p(t + dt) - tau * p.deriv()(t + dt)
            rhs = a_n * p(t) + a_prev * p(t - dt_prev)
            assert abs(lhs - rhs) < 1e-12 * (1 + abs(lhs))
    # equal steps give the fixed-step scheme: tau = 2dt/3, r = (4 u^n - u^{n-1}) / 3
    tau, a_n, a_prev = bdf2_variable(0.3, 0.3)
    assert (tau, a_n, a_prev) == pytest.approx((0.2, 4.0 / 3.0, -1.0 / 3.0), rel=1e-15)


def test_bdf2_estimate_scales_as_dt_squared():
    # u_BDF2 - u_BE is dominated by BE's local error, O(dt^2).
    from oracle.adaptive import AdaptiveHistory, _attempt
    prob = Problem(nx=128, eps=0.18, M=6, tol=1e-13, max_iter=3000)
    u0 = paper_ic_1d(128)[None, :]
    etas = []
    for dt in (2e-4, 1e-4, 5e-5):
        s = OracleSolver(prob)
        u1, _ = s.step(u0, dt, "be")
        _, eta, _ = _attempt(s, u1, dt, "bdf2", AdaptiveHistory(u0, dt))
        etas.append(eta)
    r1, r2 = etas[0] / etas[1], etas[1] / etas[2]
    assert 3.5 < r1 < 4.2 and 3.7 < r2 < 4.15, (r1, r2)


def test_bdf2_controller_keeps_history_and_needs_it():
    from oracle.adaptive import AdaptiveHistory
    prob = Problem(nx=64, eps=0.18, M=6, tol=1e-12, max_iter=600)
    s = OracleSolver(prob)
    u = paper_ic_1d(64)[None, :]
    with pytest.raises(ValueError):
        adaptive_step(s, u, 1e-3, 1e-4, 1e-8, 1.0, estimator="bdf2")
    h = AdaptiveHistory()
    u1, info1 = adaptive_step(s, u, 1e-3, 1e-4, 1e-8, 1.0, estimator="bdf2", history=h)
    assert h.dt_prev == info1.dt_used and np.array_equal(h.u_prev, u)
    u2, info2 = adaptive_step(s, u1, info1.dt_next, 1e-4, 1e-8, 1.0, estimator="bdf2", history=h)
    assert h.dt_prev == info2.dt_used and np.array_equal(h.u_prev, u1)
    assert 0 < info2.eta <= 1e-4
