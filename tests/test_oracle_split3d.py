"""Pins of the 3D split oracle (``oracle/split3d.py``) against things other than itself.

* The splitting remainder X: on a periodic Fourier mode every operator is a number, and
  M^{-1} (I - c Lap_h) = I - X must hold with Lap_h the discrete Laplacian implied by H itself
  (symbol (1/h_a - 1)/c per axis).  A wrong coefficient of the triple term fails it.
* A field constant along z: D_z of it is 0 (H reproduces constants on periodic and Neumann lines),
  so X reduces to D_x D_y and the 3D step equals the pinned 2D oracle's step on every slab.
* A small Fourier mode about u = 0 evolves with the textbook stability function of the scheme at
  lam = |k|^2 - eps^2 |k|^4: the converged split iteration solves the unsplit equation.
* The converged nonlinear stage equals an FFT solve of the same continuous equation up to the
  quadrature error, which falls at order ~M.
"""
import numpy as np
import pytest

from oracle.solver import OracleSolver, Problem, stage_params
from oracle.split3d import H, M_inv, Problem3D, Solver3D, X, mass, stage_solve
from paper_1611_04214_gb300.inputs import uniform_noise


def _grid(n, L, periodic=True):
    return L * np.arange(n) / (n if periodic else n - 1)


def _mode(prob, k, amp=1.0):
    z = _grid(prob.nz, prob.Lz)[:, None, None]
    y = _grid(prob.ny, prob.Ly)[None, :, None]
    x = _grid(prob.nx, prob.Lx)[None, None, :]
    return amp * np.sin(k[0] * x) * np.sin(k[1] * y) * np.sin(k[2] * z)


@pytest.mark.parametrize("nu", [0.05, 0.4, 2.0])
def test_remainder_x_symbol(nu):
    prob = Problem3D(nx=24, ny=20, nz=16, M=4)
    k = (2, 3, 1)
    f = _mode(prob, k)
    c = (prob.h("x") / nu) ** 2
    # the symbol of each line inverse on this mode, measured by applying it
    sym = {a: float(np.sum(H(prob, f, c, a) * f) / np.sum(f * f)) for a in "xyz"}
    for a in "xyz":   # the mode is an eigenfunction of each H_a
        assert np.abs(H(prob, f, c, a) - sym[a] * f).max() < 1e-13
    lap = sum((1.0 / sym[a] - 1.0) / c for a in "xyz")            # -Lap_h symbol
    expected = 1.0 - sym["x"] * sym["y"] * sym["z"] * (1.0 + c * lap)   # 1 - M^{-1}(I - c Lap_h)
    got = X(prob, f, c)
    assert np.abs(got - expected * f).max() < 1e-13 * max(1.0, abs(expected))
    # and M^{-1} is the product of the three symbols
    assert np.abs(M_inv(prob, f, c) - sym["x"] * sym["y"] * sym["z"] * f).max() < 1e-13


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
@pytest.mark.parametrize("scheme", ["be", "bdf2"])
def test_z_constant_field_reduces_to_2d(bc, scheme):
    nx, ny, nz, eps = 20, 16, 6, 0.12
    u2 = uniform_noise((ny, nx), 0.05, seed=3, mean=0.05)
    u3 = np.repeat(u2[None, :, :], nz, axis=0)
    p2 = Problem(nx=nx, ny=ny, Lx=2.0, Ly=1.5, bc=bc, eps=eps, M=4, tol=1e-13, max_iter=3000)
    p3 = Problem3D(nx=nx, ny=ny, nz=nz, Lx=2.0, Ly=1.5, Lz=0.7, bc=bc, eps=eps, M=4, tol=1e-13, max_iter=3000)
    s2, s3 = OracleSolver(p2), Solver3D(p3)
    for _ in range(3):
        u2, _ = s2.step(u2, 2e-3, scheme)
        u3, res = s3.step(u3, 2e-3, scheme)
        assert res.converged
    assert np.abs(u3 - u2[None]).max() < 1e-11


def _scalar(scheme, lam, dt, steps):
    z = lam * dt
    if scheme == "be":
        return (1 / (1 - z)) ** steps
    ys = [1.0, 1 / (1 - z)]                      # BDF2 with a BE start
    while len(ys) <= steps:
        ys.append((4 * ys[-1] - ys[-2]) / (3 - 2 * z))
    return ys[steps]


@pytest.mark.parametrize("scheme,dt,steps", [("be", 4e-3, 2), ("be", 0.05, 1), ("bdf2", 4e-3, 3)])
def test_single_mode_matches_scalar_scheme_3d(scheme, dt, steps):
    n, a, eps = 32, 1e-6, 0.18
    k = (1, 2, 2)
    prob = Problem3D(nx=n, ny=n, nz=n, eps=eps, M=6, tol=1e-15, max_iter=4000)
    u0 = _mode(prob, k, a)
    s = Solver3D(prob)
    u = u0
    for _ in range(steps):
        u, _ = s.step(u, dt, scheme)
    k2 = float(sum(q * q for q in k))
    lam = k2 - eps * eps * k2 * k2
    np.testing.assert_allclose(u, _scalar(scheme, lam, dt, steps) * u0, rtol=0, atol=3e-5 * a)


def _spectral_stage_solve(r, tau, eps, shape, tol=1e-13):
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


def test_nonlinear_stage_matches_spectral_solve_3d():
    eps, dt, diffs = 0.3, 0.01, []
    for n in (12, 24):
        prob = Problem3D(nx=n, ny=n, nz=n, eps=eps, M=6, tol=1e-12, max_iter=3000)
        z = _grid(n, 2 * np.pi)[:, None, None]
        y = _grid(n, 2 * np.pi)[None, :, None]
        x = _grid(n, 2 * np.pi)[None, None, :]
        v_n = 1.0 + 0.3 * np.cos(x) * np.sin(y + 0.2) + 0.2 * np.cos(z + y) - 0.1 * np.sin(2 * x - z)
        res = stage_solve(prob, v_n, v_n, dt)
        assert res.converged
        diffs.append(np.abs(res.v - _spectral_stage_solve(v_n, dt, eps, v_n.shape)).max())
    assert np.log2(diffs[0] / diffs[1]) > 4.5, diffs
    assert diffs[1] < 1e-5, diffs


def test_periodic_mass_conserved_3d():
    prob = Problem3D(nx=16, ny=14, nz=12, eps=0.15, M=4, tol=1e-13, max_iter=3000)
    u = 0.05 * np.random.default_rng(1).standard_normal((12, 14, 16))
    m0 = mass(prob, u)
    s = Solver3D(prob)
    for scheme in ("be", "bdf2", "bdf2"):
        u, res = s.step(u, 5e-3, scheme)
        assert res.converged
    assert abs(mass(prob, u) - m0) < 1e-12
