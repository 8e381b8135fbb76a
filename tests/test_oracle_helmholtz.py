"""Pins for the oracle's quadrature weights and line inverse (Sec. 3.2), each against something
other than the oracle itself: the paper's printed M=2 weights, closed-form integrals, an O(N^2)
direct sum, exact polynomial solutions of u - c u'' = p, and trigonometric closed forms."""
import numpy as np
import pytest
from scipy.special import gammainc, gamma

from oracle.helmholtz import (DIRICHLET, NEUMANN, PERIODIC, boundary_coefficients,
                              helmholtz_inverse, line_constants, particular_direct,
                              particular_recurrence, stencil_nodes)
from oracle.weights import local_weights, paper_m2_pqr

BCS = [PERIODIC, NEUMANN, DIRICHLET]


@pytest.mark.parametrize("nu", [1e-3, 0.05, 0.3, 1.0, 4.0, 25.0])
def test_m2_weights_match_printed_pqr(nu):
    # Sec. 3.2: J^L ~ P v_j + Q v_{j-1} + R (v_{j+1} - 2 v_j + v_{j-1}); our weights carry the 1/2.
    # The printed closed forms cancel catastrophically for small nu (R = (1-d)/nu^2 - (1+d)/(2nu)),
    # so the tolerance is the rounding error of evaluating them: ~1e-16 / nu^2.
    P, Q, R = paper_m2_pqr(nu)
    tol = 4e-16 / nu ** 2
    wl = 2 * local_weights(nu, (-1, 0, 1), "L")
    wr = 2 * local_weights(nu, (-1, 0, 1), "R")
    np.testing.assert_allclose(wl, [Q + R, P - 2 * R, R], rtol=1e-12, atol=tol)
    np.testing.assert_allclose(wr, [R, P - 2 * R, Q + R], rtol=1e-12, atol=tol)


@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("nu", [0.01, 0.27, 2.0, 12.0])
def test_weights_exact_on_monomials(M, nu):
    # sum_o w_o p(o) = (nu/2) int_0^1 e^{-nu t} p(-/+t) dt for deg p <= M, for centred and shifted
    # stencils; the right side is the lower incomplete gamma function (closed form).
    for offs in [tuple(range(-M // 2, M // 2 + 1)), tuple(range(0, M + 1)), tuple(range(-M, 1)),
                 tuple(range(-1, M))]:
        for side, sgn in (("L", -1.0), ("R", 1.0)):
            w = local_weights(nu, offs, side)
            for k in range(M + 1):
                lower_gamma = gammainc(k + 1, nu) * gamma(k + 1)
                exact = 0.5 * nu * sgn ** k * lower_gamma / nu ** (k + 1)
                got = float(np.dot(w, np.array(offs, dtype=float) ** k))
                assert abs(got - exact) <= 1e-12 * max(1.0, abs(exact)), (offs, side, k)


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("M", [2, 4, 6])
def test_recurrences_equal_direct_sum(bc, M):
    # Eq. IL / IR are exact identities: the recurrences equal the O(N^2) direct sum.
    rng = np.random.default_rng(1)
    n = 23
    h = 2 * np.pi / (n if bc == PERIODIC else n - 1)
    f = rng.uniform(0, 2, size=(3, n))
    IL, IR = particular_recurrence(f, 0.02, h, bc, M)
    np.testing.assert_allclose(IL + IR, particular_direct(f, 0.02, h, bc, M), rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("bc", [PERIODIC, NEUMANN])
@pytest.mark.parametrize("c", [1e-5, 1e-2, 10.0])
def test_constants_are_fixed(bc, c):
    n = 37
    h = 2 * np.pi / (n if bc == PERIODIC else n - 1)
    np.testing.assert_allclose(helmholtz_inverse(np.full((2, n), 1.7), c, h, bc, 4), 1.7, rtol=1e-12)


def _exact_poly_solution(coef, c, L, bc, x):
    """u - c u'' = p on [0, L] with homogeneous Neumann or Dirichlet conditions, closed form."""
    p = np.polynomial.Polynomial(coef)
    up = p.copy()
    term = p
    while term.degree() >= 2:
        term = c * term.deriv(2)
        up = up + term
    alpha = c ** -0.5
    mu = np.exp(-alpha * L)
    if bc == NEUMANN:     # u'(0) = u'(L) = 0 with u = up + A e^{-alpha x} + B e^{-alpha (L - x)}
        A = np.array([[-alpha, alpha * mu], [-alpha * mu, alpha]])
        rhs = -np.array([up.deriv()(0.0), up.deriv()(L)])
    else:                 # u(0) = u(L) = 0
        A = np.array([[1.0, mu], [mu, 1.0]])
        rhs = -np.array([up(0.0), up(L)])
    a, b = np.linalg.solve(A, rhs)
    return up(x) + a * np.exp(-alpha * x) + b * np.exp(-alpha * (L - x))


@pytest.mark.parametrize("bc", [NEUMANN, DIRICHLET])
@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("c", [3e-4, 0.05, 2.0])
def test_polynomials_exact_nonperiodic(bc, M, c):
    # The quadrature is exact for degree <= M and the recurrences and boundary solve are exact,
    # so the discrete inverse equals the continuous solution at the nodes (covers the shifted
    # wall stencils and the Neumann / Dirichlet B formulas).
    rng = np.random.default_rng(M)
    n, L = 29, 3.0
    x = np.linspace(0, L, n)
    coef = rng.uniform(-1, 1, size=M + 1)
    got = helmholtz_inverse(np.polynomial.Polynomial(coef)(x), c, L / (n - 1), bc, M)
    exact = _exact_poly_solution(coef, c, L, bc, x)
    np.testing.assert_allclose(got, exact, rtol=0, atol=1e-11 * max(1.0, np.abs(exact).max()))


@pytest.mark.parametrize("M", [2, 4, 6])
def test_periodic_trig_converges_at_order_M(M):
    # Periodic L^{-1}[sin kx] = sin kx / (1 + c k^2); the error falls at least like h^M.
    c, k = 0.01, 3
    errs = []
    for n in (48, 96, 192):
        x = 2 * np.pi * np.arange(n) / n
        got = helmholtz_inverse(np.sin(k * x), c, 2 * np.pi / n, PERIODIC, M)
        errs.append(np.abs(got - np.sin(k * x) / (1 + c * k * k)).max())
    orders = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert np.all(orders > M - 0.3), (errs, orders)


def test_periodic_is_circulant_and_large_c_projects_to_mean():
    rng = np.random.default_rng(3)
    n = 40
    h = 2 * np.pi / n
    f = rng.uniform(size=n)
    a = helmholtz_inverse(f, 0.05, h, PERIODIC, 4)
    b = helmholtz_inverse(np.roll(f, 7), 0.05, h, PERIODIC, 4)
    np.testing.assert_allclose(np.roll(a, 7), b, rtol=1e-13, atol=1e-14)
    far = helmholtz_inverse(f, 1e10, h, PERIODIC, 4)
    np.testing.assert_allclose(far, f.mean(), rtol=0, atol=1e-6)   # k != 0 modes are damped to O(nu)


def test_neumann_commutes_with_reflection():
    rng = np.random.default_rng(4)
    n = 31
    f = rng.uniform(size=n)
    h = 1.0 / (n - 1)
    a = helmholtz_inverse(f, 0.003, h, NEUMANN, 6)
    b = helmholtz_inverse(f[::-1], 0.003, h, NEUMANN, 6)
    np.testing.assert_allclose(a[::-1], b, rtol=1e-12, atol=1e-14)


def test_boundary_systems_satisfied():
    # B_a, B_b solve the 2x2 systems written from L^{-1}(a), L^{-1}(b) and L^{-1}_x (Sec. 3.2).
    # L^{-1}_x(b) = alpha(-I_N - mu B_a + B_b): the slope of B_a e^{-alpha(x-a)} at b is
    # -alpha mu B_a.  (The paper prints +B_a mu there; with that sign its own printed
    # solution B_a = I_N/(1-mu), B_b = I_0/(1-mu) would not follow.)
    I0, IN, mu = 0.3, -0.7, 0.2
    Ba, Bb = boundary_coefficients(I0, IN, mu, PERIODIC)
    assert np.isclose(I0 + Ba + Bb * mu, IN + Ba * mu + Bb)
    assert np.isclose(I0 - Ba + Bb * mu, -IN - Ba * mu + Bb)
    Ba, Bb = boundary_coefficients(I0, IN, mu, NEUMANN)
    assert np.isclose(I0 - Ba + mu * Bb, 0) and np.isclose(-IN - mu * Ba + Bb, 0)
    Ba, Bb = boundary_coefficients(I0, IN, mu, DIRICHLET)
    assert np.isclose(I0 + Ba + mu * Bb, 0) and np.isclose(IN + mu * Ba + Bb, 0)


def test_stencils_stay_inside_and_wrap():
    N, M = 10, 6
    for j in range(N + 1):
        nodes = stencil_nodes(j, N, M, NEUMANN)
        assert len(nodes) == M + 1 and min(nodes) >= 0 and max(nodes) <= N
    assert stencil_nodes(0, N, 4, PERIODIC) == [8, 9, 0, 1, 2]


def test_line_constants():
    alpha, nu, d, mu, N = line_constants(0.25, 0.1, 11, NEUMANN)
    assert alpha == 2.0 and np.isclose(nu, 0.2) and N == 10 and np.isclose(mu, d ** 10)
