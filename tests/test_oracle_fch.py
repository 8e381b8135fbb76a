"""Pins of the 1D FCH oracle (``oracle/fch.py``) against things other than itself.

* A small mode about u = -1 decays in one BE step by the linearised rate of Eq. FCH0:
  1 / (1 + dt k^2 (eps^2 k^2 + 2)(eps^2 k^2 + 2 - eta eps^2)), periodic and, for cosine modes
  with nodes on the walls, Neumann.
* The converged step solves the BE equation of the PDE with the discrete Laplacian the line
  inverse implies (symbol (1/h(k) - 1)/a, measured by FFT of H's impulse response), evaluated
  pointwise and by FFT, independently of the iteration's rearrangement; the printed signs of
  Eq. FCH_BE do not.
* Periodic mass is conserved to rounding.
* About the wells the lagged iteration multiplies a mode by
  m(x) = h [(3 + c_eta - 2 c_f) x^2 h^2 + 3 x h^2 - c_p x h^2 (2 eps^2 x / a + 4 - 2 eta eps^2)],
  x = a k^2, h = 1/(1 + x) (the lagged zero-order part f f' = 4v of p dominates): at the paper's
  dt = 0.1 (eps = 0.18) m = -1.04 at k = 4 and the iteration diverges; at dt = 0.05 it contracts.
"""
import numpy as np
import pytest

from oracle.fch import FchSolver, f_v, fp_v, fch_be_step
from oracle.helmholtz import helmholtz_inverse
from oracle.solver import Problem
from paper_1611_04214_gb300.inputs import paper_ic_1d


def _x(n):
    return 2 * np.pi * np.arange(n) / n


@pytest.mark.parametrize("k,dt", [(1, 0.05), (2, 0.05), (3, 0.01)])
def test_small_mode_decays_at_the_linear_rate(k, dt):
    n, eps, eta, amp = 128, 0.18, 1.0, 1e-7
    prob = Problem(nx=n, eps=eps, M=6, tol=1e-16, max_iter=400)
    u0 = (-1.0 + amp * np.cos(k * _x(n)))[None, :]
    u1, res = FchSolver(prob, eta).step(u0, dt)
    k2 = float(k * k)
    rate = 1.0 / (1.0 + dt * k2 * (eps ** 2 * k2 + 2) * (eps ** 2 * k2 + 2 - eta * eps ** 2))
    np.testing.assert_allclose(u1 + 1.0, rate * (u0 + 1.0), rtol=0, atol=1e-4 * amp)


@pytest.mark.parametrize("m", [2, 4, 6])
def test_neumann_cosine_mode_decays_at_the_linear_rate(m):
    # cos(m x / 2) on [0, 2pi] with nodes on both walls is a Neumann mode (wavenumber m / 2): the
    # walls' boundary correction and shifted stencils must reproduce the same linear rate.
    from paper_1611_04214_gb300.inputs import nodes
    n, eps, eta, amp, dt = 129, 0.18, 1.0, 1e-7, 0.05
    prob = Problem(nx=n, eps=eps, M=6, tol=1e-16, max_iter=400, bc="neumann")
    kap2 = (m / 2.0) ** 2
    u0 = (-1.0 + amp * np.cos(0.5 * m * nodes(n, 2 * np.pi, False)))[None, :]
    u1, res = FchSolver(prob, eta).step(u0, dt)
    rate = 1.0 / (1.0 + dt * kap2 * (eps ** 2 * kap2 + 2) * (eps ** 2 * kap2 + 2 - eta * eps ** 2))
    np.testing.assert_allclose(u1 + 1.0, rate * (u0 + 1.0), rtol=0, atol=1e-6 * amp)


def _discrete_lap(prob, a):
    """Apply the Laplacian implied by the line inverse H = (I - a Lap_h)^{-1} (periodic, by FFT)."""
    n = prob.nx
    delta = np.zeros((1, n))
    delta[0, 0] = 1.0
    hk = np.fft.fft(helmholtz_inverse(delta, a, prob.hx, prob.bc, prob.M, axis=1)[0])
    sym = -(1.0 / hk.real - 1.0) / a                  # symbol of Lap_h (real, <= 0)
    return lambda w: np.real(np.fft.ifft(sym * np.fft.fft(w)))


@pytest.mark.parametrize("eta", [1.0, 3.0])
def test_converged_step_solves_the_pde_be_equation(eta):
    n, eps, dt = 128, 0.18, 0.05
    prob = Problem(nx=n, eps=eps, M=6, tol=1e-13, max_iter=3000)
    vn = paper_ic_1d(n) + 1.0
    res = fch_be_step(prob, vn[None, :], dt, eta)
    assert res.converged
    a = (dt * eps ** 4) ** (1.0 / 3.0)
    lap = _discrete_lap(prob, a)
    v = res.v[0]
    assert np.abs(lap(v) - res.lap_v[0]).max() < 1e-9 * np.abs(lap(v)).max()   # Lap v carried exactly
    f, fp = f_v(v), fp_v(v)

    def residual(sign):
        g = sign * (-eps ** 2 * lap(f) - eps ** 2 * fp * lap(v) + eta * eps ** 4 * lap(v) - eta * eps ** 2 * f) + f * fp
        return v - vn - dt * eps ** 4 * lap(lap(lap(v))) - dt * lap(g)

    # the PDE's signs: solved to the iteration's tolerance (times the operator's scale)
    assert np.abs(residual(+1.0)).max() < 1e-9
    # the printed signs of the last four bracket terms are not what the step solves
    assert np.abs(residual(-1.0)).max() > 1e-3


def test_periodic_mass_conserved():
    n = 128
    prob = Problem(nx=n, eps=0.18, M=6, tol=1e-12, max_iter=2000)
    s = FchSolver(prob, 1.0)
    u = paper_ic_1d(n)[None, :]
    m0 = u.mean()
    for _ in range(4):
        u, res = s.step(u, 0.1)
        assert res.converged
    assert abs(u.mean() - m0) < 1e-13


def _well_factor(k, dt, eps, eta):
    a = (dt * eps ** 4) ** (1.0 / 3.0)
    x, c_eta, c_f, c_p = a * k * k, dt * eta * eps ** 4 / a ** 2, dt * eps ** 2 / a ** 2, dt / a
    h = 1.0 / (1.0 + x)
    return h * ((3 + c_eta - 2 * c_f) * x * x * h * h + 3 * x * h * h
                - c_p * x * h * h * (2 * eps ** 2 * x / a + 4 - 2 * eta * eps ** 2))


@pytest.mark.parametrize("dt", [0.1, 0.05])
def test_iteration_factor_about_the_wells(dt):
    # A k = 4 mode about u = -1 as the step's start: the residual of the lagged iteration changes
    # by |m| per iteration, growing at the paper's dt = 0.1 and shrinking at dt = 0.05.
    n, eps, eta, k = 128, 0.18, 1.0, 4
    m = _well_factor(k, dt, eps, eta)
    prob = Problem(nx=n, eps=eps, M=6, tol=1e-30, max_iter=30)
    res = fch_be_step(prob, (1e-9 * np.cos(k * _x(n)))[None, :], dt, eta)
    h = res.history
    ratio = (h[-1] / h[-11]) ** 0.1
    assert abs(ratio - abs(m)) < 0.02 * abs(m), (ratio, m)
    assert (h[-1] > h[0]) == (abs(m) > 1.0)
