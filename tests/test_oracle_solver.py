"""Pins for the oracle's stage solves and time schemes (Sec. 3-5), against things other than
the oracle itself: the paper's printed refinement tables and regime-switch values, textbook
stability functions of each scheme on a single Fourier mode, a spectral (FFT) solve of the
unsplit stage equation, Runge-Kutta order conditions, and the paper's invariants."""
import json
import os

import numpy as np
import pytest

from oracle.solver import (ETA2, ETA3, SDIRK2, SDIRK3, OracleSolver, Problem, energy, mass,
                           stage_params, stage_solve)
from paper_1611_04214_gb300.inputs import mode_ic, paper_ic_1d, paper_ic_2d, uniform_noise

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_refinement_1d.json")


def _load_golden():
    with open(GOLDEN) as fh:
        return json.load(fh)


def _run_1d(scheme, dt, n=512, M=6, T=1.0, tol=1e-12):
    prob = Problem(nx=n, eps=0.18, M=M, tol=tol, max_iter=3000)
    s = OracleSolver(prob)
    u = paper_ic_1d(n)[None, :]
    for _ in range(int(round(T / dt))):
        u, info = s.step(u, dt, scheme)
        assert info.converged
    return u[0]


@pytest.mark.parametrize("scheme", ["bdf2", "sdirk2", "sdc2", "sdirk3", "bdf3"])
def test_refinement_tables_reproduced(scheme):
    # Tables CH_refinement_second / CH_refinement_third: successive errors at dt = 0.05, 0.025, 0.0125.
    # BDF3 starts with two SDIRK2 steps (Sec. 4.4); that start reproduces its column.
    g = _load_golden()
    dts = g["dt"][:4]
    us = [_run_1d(scheme, dt) for dt in dts]
    errs = [np.abs(us[i] - us[i + 1]).max() for i in range(3)]
    np.testing.assert_allclose(errs, g["errors"][scheme][:3], rtol=2e-4)


def test_regime_switch_values():
    # Sec. 4.4 prints the switch time steps for eps = 0.18: the factorization regime starts where
    # the stage coefficient tau reaches eps^2 (BDF2: tau = 2dt/3, SDIRK2: tau = eta dt, SDC2: tau = dt).
    g = _load_golden()["regime_switch_dt"]
    eps2 = g["eps"] ** 2
    assert round(1.5 * eps2, 4) == g["bdf2"]
    assert round(eps2 / ETA2, 4) == g["sdirk2"]
    assert round(eps2, 4) == g["sdc2"]
    assert stage_params(eps2 * 0.999, g["eps"]).regime == "square"
    assert stage_params(eps2 * 1.001, g["eps"]).regime == "factor"


def test_stage_params_factor_the_operator():
    for tau, eps in [(0.1, 0.18), (1e-4, 0.05), (0.0324, 0.18)]:
        sp = stage_params(tau, eps)
        # (1 + c1 k^2)(1 + c2 k^2) = 1 + s tau k^2 + eps^2 tau k^4 with s = 2 - lam.
        assert np.isclose(sp.c_in * sp.c_out, eps * eps * tau, rtol=1e-12)
        assert np.isclose(sp.c_in + sp.c_out, (2 - sp.lam) * tau, rtol=1e-12)
        assert sp.beta <= 1.0 + 1e-15
        if sp.regime == "factor":
            assert abs(sp.lam) < 1e-12          # G = f~ (Eq. CH_BE_fixed2_factor)


def test_sdirk_tableaus():
    # SDIRK2: eta is the root of 1/2 - 2 eta + eta^2 (Sec. 4.2); SDIRK3: eta ~ 0.4359 (Sec. 4.4)
    # and the third-order conditions hold.
    assert abs(0.5 - 2 * ETA2 + ETA2 ** 2) < 1e-15
    assert round(ETA3, 4) == 0.4359
    for A, order in ((SDIRK2, 2), (SDIRK3, 3)):
        b, c = A[-1], A.sum(axis=1)
        assert np.isclose(b.sum(), 1) and np.isclose(b @ c, 0.5)
        if order == 3:
            assert np.isclose(b @ c ** 2, 1 / 3) and np.isclose(b @ A @ c, 1 / 6)


def _scalar_scheme(scheme, lam, dt, steps):
    """The scheme applied to y' = lam y, y(0) = 1 (textbook forms)."""
    z = lam * dt
    if scheme == "be":
        return (1 / (1 - z)) ** steps
    if scheme in ("sdirk2", "sdirk3"):
        A = SDIRK2 if scheme == "sdirk2" else SDIRK3
        s = A.shape[0]
        R = 1 + z * A[-1] @ np.linalg.solve(np.eye(s) - z * A, np.ones(s))
        return R ** steps
    if scheme == "bdf2":        # BE start, then (3 y_{n+1} - 4 y_n + y_{n-1}) = 2 z y_{n+1}
        ys = [1.0, 1 / (1 - z)]
        while len(ys) <= steps:
            ys.append((4 * ys[-1] - ys[-2]) / (3 - 2 * z))
        return ys[steps]
    if scheme == "bdf3":        # two SDIRK2 steps, then 11 y_{n+1} - 18 y_n + 9 y_{n-1} - 2 y_{n-2} = 6 z y_{n+1}
        s = SDIRK2.shape[0]
        R2 = 1 + z * SDIRK2[-1] @ np.linalg.solve(np.eye(s) - z * SDIRK2, np.ones(s))
        ys = [1.0, R2, R2 * R2]
        while len(ys) <= steps:
            ys.append((18 * ys[-1] - 9 * ys[-2] + 2 * ys[-3]) / (11 - 6 * z))
        return ys[steps]
    if scheme == "sdc2":        # level 0 BE; level 1 trapezoid correction with F0 = lam y0
        y0, y1 = 1.0, 1.0
        for _ in range(steps):
            y0n = y0 / (1 - z)
            y1 = (y1 - 0.5 * z * (y0n - y0)) / (1 - z)
            y0 = y0n
        return y1
    raise ValueError(scheme)


@pytest.mark.parametrize("scheme", ["be", "bdf2", "sdirk2", "sdirk3", "sdc2", "bdf3"])
@pytest.mark.parametrize("dt", [4e-3, 0.08])      # square and factorization regimes (eps = 0.18)
def test_single_mode_matches_scalar_scheme_1d(scheme, dt):
    # A small mode a sin(kx) about u = 0 evolves by y' = (k^2 - eps^2 k^4) y (f(u) ~ -u); the
    # spatial error of the line inverse is O(h^M), far below the tolerance used here.
    n, k, a, eps, steps = 96, 3, 1e-6, 0.18, 4
    prob = Problem(nx=n, eps=eps, M=6, tol=1e-15, max_iter=5000)
    s = OracleSolver(prob)
    u0 = mode_ic(n, 1, k, 0, a)
    u = u0
    for _ in range(steps):
        u, _ = s.step(u, dt, scheme)
    lam = k * k - eps * eps * k ** 4
    np.testing.assert_allclose(u, _scalar_scheme(scheme, lam, dt, steps) * u0, rtol=0, atol=2e-6 * a)


@pytest.mark.parametrize("scheme,dt", [("be", 4e-3), ("sdirk2", 4e-3), ("be", 0.05)])
def test_single_mode_matches_scalar_scheme_2d(scheme, dt):
    # In 2D the converged split iteration must solve the unsplit equation: a mode
    # sin(kx x) sin(ky y) evolves with lam = |k|^2 - eps^2 |k|^4 (splitting error removed).
    nx, ny, kx, ky, a, eps = 64, 56, 2, 3, 1e-6, 0.18
    prob = Problem(nx=nx, ny=ny, eps=eps, M=6, tol=1e-15, max_iter=4000)
    s = OracleSolver(prob)
    u0 = mode_ic(nx, ny, kx, ky, a)
    u, info = s.step(u0, dt, scheme)
    k2 = kx * kx + ky * ky
    lam = k2 - eps * eps * k2 * k2
    np.testing.assert_allclose(u, _scalar_scheme(scheme, lam, dt, 1) * u0, rtol=0, atol=3e-5 * a)


def _spectral_stage_solve(r, tau, eps, shape, tol=1e-13):
    """Fourier-space fixed point for the unsplit periodic stage equation v - tau F(v) = r on [0,2pi]^d."""
    ks = [np.fft.fftfreq(n, 1.0 / n) for n in shape]
    K2 = sum(np.meshgrid(*[k ** 2 for k in ks], indexing="ij"))
    sp = stage_params(tau, eps)
    denom = (1 + sp.c_in * K2) * (1 + sp.c_out * K2)
    v = r.copy()
    for _ in range(20000):
        g = v ** 3 - 3 * v ** 2 + sp.lam * v
        vn = np.real(np.fft.ifftn((np.fft.fftn(r) - tau * K2 * np.fft.fftn(g)) / denom))
        if np.abs(vn - v).max() < tol:
            return vn
        v = vn
    raise AssertionError("spectral fixed point did not converge")


@pytest.mark.parametrize("dim,dt", [(1, 0.01), (1, 0.06), (2, 0.01), (2, 0.05)])
def test_nonlinear_stage_matches_spectral_solve(dim, dt):
    # The converged stage of the line-sweep iteration equals an FFT solve of the same continuous
    # nonlinear equation (no splitting, exact symbols) up to the quadrature error, which must fall
    # at order ~M (M = 6) when the grid is doubled.
    eps = 0.18
    diffs = []
    for n in ((128, 256) if dim == 1 else (32, 64)):
        if dim == 1:
            prob = Problem(nx=n, eps=eps, M=6, tol=1e-13, max_iter=5000)
            v_n = paper_ic_1d(n)[None, :] + 1
            shape = (n,)
        else:
            prob = Problem(nx=n, ny=n, eps=eps, M=6, tol=1e-12, max_iter=5000)
            v_n = paper_ic_2d(n, n) + 1
            shape = (n, n)
        res = stage_solve(prob, v_n, v_n, dt)
        assert res.converged
        ref = _spectral_stage_solve(v_n.reshape(shape), dt, eps, shape)
        diffs.append(np.abs(res.v.reshape(shape) - ref).max())
    assert np.log2(diffs[0] / diffs[1]) > 4.5, diffs
    assert diffs[1] < (1e-7 if dim == 1 else 1e-5), diffs


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("scheme,dt", [("be", 2e-3), ("be", 0.02), ("bdf2", 0.01), ("sdirk2", 0.01)])
def test_energy_decays_and_mass(bc, scheme, dt):
    # Lemma of Sec. 3.1.1 (and the paper's observation for the higher-order schemes): energy does
    # not increase; mass is conserved exactly for periodic lines and to discretization error for Neumann.
    nx, ny = 40, 36
    prob = Problem(nx=nx, ny=ny, bc=bc, eps=0.1, M=4, tol=1e-12, max_iter=4000)
    u = uniform_noise((ny, nx), 0.05, seed=0)
    s = OracleSolver(prob)
    m0, e_prev = mass(prob, u), energy(prob, u)
    for _ in range(3):
        u, info = s.step(u, dt, scheme)
        assert info.converged
        e = energy(prob, u)
        assert e <= e_prev + 1e-12 * abs(e_prev)
        e_prev = e
    drift = abs(mass(prob, u) - m0) / (prob.Lx * prob.Ly)      # per unit area
    assert drift < (1e-14 if bc == "periodic" else 1e-3)


def test_dirichlet_walls_and_energy():
    # Per-inversion Dirichlet lines hold v = 0 (u = -1) at the walls; with an initial state that
    # satisfies the wall value the energy still decays.
    nx, ny = 36, 30
    prob = Problem(nx=nx, ny=ny, bc="dirichlet", eps=0.1, M=4, tol=1e-12, max_iter=4000)
    u = uniform_noise((ny, nx), 0.05, seed=1, mean=0.1)
    u[0, :] = u[-1, :] = -1
    u[:, 0] = u[:, -1] = -1
    s = OracleSolver(prob)
    e_prev = energy(prob, u)
    for _ in range(3):
        u, _ = s.step(u, 2e-3, "be")
        assert np.abs(u[0, :] + 1).max() < 1e-12 and np.abs(u[:, -1] + 1).max() < 1e-12
        e = energy(prob, u)
        assert e <= e_prev + 1e-12 * abs(e_prev)
        e_prev = e


def test_iteration_cap_reports_not_converged():
    prob = Problem(nx=64, eps=0.18, M=4, tol=1e-14, max_iter=2)
    res = stage_solve(prob, paper_ic_1d(64)[None, :] + 1, paper_ic_1d(64)[None, :] + 1, 0.1)
    assert not res.converged and res.iters == 2


def test_energy_and_mass_closed_forms():
    # u = cos x on a periodic line: E = eps^2/2 * pi (+O(h^2)) + int (cos^2 - 1)^2/4, mass = 0.
    n, eps = 256, 0.1
    prob = Problem(nx=n, eps=eps)
    x = 2 * np.pi * np.arange(n) / n
    u = np.cos(x)[None, :]
    exact = eps ** 2 / 2 * np.pi + 3 * np.pi / 16
    assert abs(energy(prob, u) - exact) < 1e-4
    assert abs(mass(prob, u)) < 1e-12


def test_ripening_time_be_dt10_matches_paper():
    # Sec. 6.1, Table 1DCH_ripeninglargedt: 1D periodic, 128 nodes, eps = 0.18, u0 of Eq.
    # CH1D_initial, tolerance 1e-11; BE with dt = 10 ripens (u(pi) < 0 first) at t = 8250.00.
    # 825 steps deep in the factorization regime (tau / eps^2 = 309).
    n = 128
    prob = Problem(nx=n, eps=0.18, M=6, tol=1e-11, max_iter=4000)
    s = OracleSolver(prob)
    u = paper_ic_1d(n)[None, :]
    k = 0
    while True:
        u, info = s.step(u, 10.0, "be")
        assert info.converged
        k += 1
        if u[0, n // 2] < 0 or k > 1000:
            break
    assert k * 10.0 == 8250.0
