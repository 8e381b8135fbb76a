"""Pins of the 2D FCH oracle (``oracle/fch.py``, ``fch2d_be_step``) against things other than itself.

* A small mode about u = -1 decays in one BE step by the linearised rate of Eq. FCH0 with
  k^2 = kx^2 + ky^2, periodic, and for cosine modes with nodes on the walls, Neumann.
* The converged step solves the PDE's BE equation with the discrete Laplacian the split line
  inverses imply (the sum of the two 1D symbols (1/h(k) - 1)/a, measured by FFT of H's impulse
  response), evaluated by FFT independently of the iteration's rearrangement, on a non-square
  grid with different spacings in x and y; the printed signs of Eq. FCH_BE do not solve it.
  The carried Lap v equals that Laplacian of the iterate.
* Periodic mass is conserved to rounding.
* Data constant in y reproduce the 1D oracle (H_y leaves them unchanged and the splitting
  remainder vanishes), step after step.
* Transposing the data of a square grid transposes the step.
* About the wells the lagged 2D iteration multiplies a mode of W by
  phi = -3 m^2 K + (3 + c_eta - 2 c_f) m K^2 + c_p m K (-2 eps^2 K / a + (4 - 2 eta eps^2) m)
        + 1 - (1 - X)^3,
  m = h_x h_y, K = 2m - h_x - h_y, X = (h_x - 1)(h_y - 1), h = 1 / (1 + a k^2) per axis; the
  residual history shows that factor (it is the 1D factor for ky = 0).
"""
import numpy as np
import pytest

from oracle.fch import Fch2DSolver, FchSolver, f_v, fp_v, fch2d_be_step
from oracle.helmholtz import helmholtz_inverse
from oracle.solver import Problem
from paper_1611_04214_gb300.inputs import nodes, paper_ic_1d, paper_ic_2d, uniform_noise

EPS, ETA = 0.18, 1.0


def _rate(k2, dt, eps=EPS, eta=ETA):
    return 1.0 / (1.0 + dt * k2 * (eps ** 2 * k2 + 2) * (eps ** 2 * k2 + 2 - eta * eps ** 2))


@pytest.mark.parametrize("kx,ky", [(1, 1), (2, 1), (2, 2)])
def test_small_mode_decays_at_the_linear_rate(kx, ky):
    n, amp, dt = 32, 1e-7, 0.05
    x = 2 * np.pi * np.arange(n) / n
    prob = Problem(nx=n, ny=n, eps=EPS, M=6, tol=1e-16, max_iter=300)
    v0 = amp * np.cos(ky * x)[:, None] * np.cos(kx * x)[None, :]
    res = fch2d_be_step(prob, v0, dt, ETA)
    np.testing.assert_allclose(res.v, _rate(kx * kx + ky * ky, dt) * v0, rtol=0, atol=1e-5 * amp)


@pytest.mark.parametrize("mx,my", [(2, 2), (4, 2)])
def test_neumann_cosine_mode_decays_at_the_linear_rate(mx, my):
    # cos(mx x / 2) cos(my y / 2) on [0, 2pi]^2 with nodes on the walls is a Neumann mode
    n, amp, dt = 65, 1e-7, 0.05
    x = nodes(n, 2 * np.pi, False)
    prob = Problem(nx=n, ny=n, eps=EPS, M=6, tol=1e-16, max_iter=300, bc="neumann")
    v0 = amp * np.cos(0.5 * my * x)[:, None] * np.cos(0.5 * mx * x)[None, :]
    res = fch2d_be_step(prob, v0, dt, ETA)
    np.testing.assert_allclose(res.v, _rate(0.25 * (mx * mx + my * my), dt) * v0, rtol=0, atol=1e-5 * amp)


def _symbol(n, h, a):
    delta = np.zeros((1, n))
    delta[0, 0] = 1.0
    hk = np.fft.fft(helmholtz_inverse(delta, a, h, "periodic", 6, axis=1)[0])
    return -(1.0 / hk.real - 1.0) / a


def test_converged_step_solves_the_pde_be_equation():
    nx, ny, dt = 32, 24, 0.05
    prob = Problem(nx=nx, ny=ny, Lx=2 * np.pi, Ly=1.5 * np.pi, eps=EPS, M=6, tol=1e-13, max_iter=3000)
    vn = paper_ic_2d(nx, ny) + 1.0
    res = fch2d_be_step(prob, vn, dt, ETA)
    assert res.converged
    a = (dt * EPS ** 4) ** (1.0 / 3.0)
    S = _symbol(ny, prob.hy, a)[:, None] + _symbol(nx, prob.hx, a)[None, :]

    def lap(w):
        return np.real(np.fft.ifft2(S * np.fft.fft2(w)))

    v = res.v
    assert np.abs(lap(v) - res.lap_v).max() < 1e-11 * np.abs(lap(v)).max()
    f, fp = f_v(v), fp_v(v)

    def residual(sign):
        g = sign * (-EPS ** 2 * lap(f) - EPS ** 2 * fp * lap(v) + ETA * EPS ** 4 * lap(v) - ETA * EPS ** 2 * f) + f * fp
        return v - vn - dt * EPS ** 4 * lap(lap(lap(v))) - dt * lap(g)

    assert np.abs(residual(+1.0)).max() < 1e-9
    assert np.abs(residual(-1.0)).max() > 1e-3
    assert abs(v.mean() - vn.mean()) < 1e-14


def test_y_constant_data_reproduce_the_1d_oracle():
    n, dt = 64, 0.05
    u = paper_ic_1d(n)
    s2 = Fch2DSolver(Problem(nx=n, ny=8, eps=EPS, M=6, tol=1e-13, max_iter=3000), ETA)
    s1 = FchSolver(Problem(nx=n, eps=EPS, M=6, tol=1e-13, max_iter=3000), ETA)
    u2, u1 = np.tile(u, (8, 1)), u[None, :]
    for _ in range(2):
        u2, r2 = s2.step(u2, dt)
        u1, r1 = s1.step(u1, dt)
        assert r2.converged and r1.converged
        assert np.abs(u2 - u1).max() < 1e-11


def test_transpose_symmetry():
    n, dt = 24, 0.05
    v = uniform_noise((n, n), 0.3, seed=7, mean=0.1) + 1.0
    prob = Problem(nx=n, ny=n, eps=EPS, M=4, tol=1e-13, max_iter=3000)
    a = fch2d_be_step(prob, v, dt, ETA)
    b = fch2d_be_step(prob, v.T, dt, ETA)
    assert a.converged and b.converged
    assert np.abs(a.v - b.v.T).max() < 1e-12


def _phi(kx, ky, dt, eps=EPS, eta=ETA):
    a = (dt * eps ** 4) ** (1.0 / 3.0)
    c_eta, c_f, c_p = dt * eta * eps ** 4 / a ** 2, dt * eps ** 2 / a ** 2, dt / a
    hx, hy = 1.0 / (1.0 + a * kx * kx), 1.0 / (1.0 + a * ky * ky)
    m = hx * hy
    K, X = 2 * m - hx - hy, (hx - 1) * (hy - 1)
    return (-3 * m * m * K + (3 + c_eta - 2 * c_f) * m * K * K
            + c_p * m * K * (-2 * eps ** 2 * K / a + (4 - 2 * eta * eps ** 2) * m) + 1 - (1 - X) ** 3)


@pytest.mark.parametrize("kx,ky", [(4, 1), (3, 2), (4, 0)])
def test_iteration_factor_about_the_wells(kx, ky):
    # the paper's dt = 0.1: the 2D modes (4, 1) and (3, 2) contract (0.92, 0.75), the axis mode
    # (4, 0) grows (1.04) as in 1D
    n, dt = 64, 0.1
    x = 2 * np.pi * np.arange(n) / n
    prob = Problem(nx=n, ny=n, eps=EPS, M=6, tol=1e-30, max_iter=30)
    res = fch2d_be_step(prob, 1e-9 * np.cos(ky * x)[:, None] * np.cos(kx * x)[None, :], dt, ETA)
    h = res.history
    ratio = (h[-1] / h[-11]) ** 0.1
    m = abs(_phi(kx, ky, dt))
    assert abs(ratio - m) < 1e-3 * m, (ratio, m)
    assert (h[-1] > h[0]) == (m > 1.0)
