"""Pins for the vector Cahn-Hilliard oracle (Eq. CH_vector, Sec. 5.2) that do not depend on its code:
- W written as the product over the three roots;
- finite differences;
- the Hessian 18 I of Eq. Jacobian;
- the continuous linear growth rate of a Fourier mode;
- conservation, energy decay and temporal order."""
import numpy as np
import pytest

from oracle.solver import Problem
from oracle.vch import (VchSolver, W, Z3, cube_roots, grad_W, vch_energy, vch_stage_params,
                        vch_stage_solve)
from paper_1611_04214_gb300.inputs import nodes, paper_ic_2d, uniform_noise


def _W_product(u1, u2):
    # Eq. CH_vector_reaction as printed: the product of squared distances to the three roots
    out = np.ones_like(np.asarray(u1, dtype=np.float64))
    for a, b in cube_roots():
        out = out * ((u1 - a) ** 2 + (u2 - b) ** 2)
    return out


def test_potential_is_the_product_over_the_roots():
    rng = np.random.default_rng(1)
    u1, u2 = rng.uniform(-2, 2, 200), rng.uniform(-2, 2, 200)
    assert np.allclose(W(u1, u2), _W_product(u1, u2), rtol=1e-12, atol=1e-12)
    for a, b in cube_roots():
        assert W(a, b) < 1e-28
    assert Z3 == pytest.approx(cube_roots()[2], abs=1e-15)


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(2)
    u1, u2 = rng.uniform(-1.5, 1.5, 50), rng.uniform(-1.5, 1.5, 50)
    h = 1e-6
    d1 = (_W_product(u1 + h, u2) - _W_product(u1 - h, u2)) / (2 * h)
    d2 = (_W_product(u1, u2 + h) - _W_product(u1, u2 - h)) / (2 * h)
    g1, g2 = grad_W(u1, u2)
    assert np.allclose(g1, d1, rtol=1e-6, atol=1e-6)
    assert np.allclose(g2, d2, rtol=1e-6, atol=1e-6)


def test_hessian_at_every_root_is_18_identity():
    # Eq. Jacobian
    h = 1e-6
    for a, b in cube_roots():
        H = np.empty((2, 2))
        for j, (da, db) in enumerate(((h, 0.0), (0.0, h))):
            gp = grad_W(a + da, b + db)
            gm = grad_W(a - da, b - db)
            H[:, j] = [(gp[0] - gm[0]) / (2 * h), (gp[1] - gm[1]) / (2 * h)]
        assert np.allclose(H, 18.0 * np.eye(2), atol=1e-6), H


@pytest.mark.parametrize("tau", [1e-3, 1.2644e-3, 1.2645e-3, 0.01, 1.0])
def test_stage_parameters_factor_the_operator(tau):
    # (I - c1 Lap)(I - c2 Lap) must equal I - s tau Lap + eps^2 tau Lap^2 with s = 18 in the
    # factorization regime (Eq. CH_vector_fixed1) and s = 2 sqrt(eps^2/tau) otherwise
    # (Eq. CH_vector_fixed2); the switch sits at tau = eps^2/81.
    eps = 0.32
    sp = vch_stage_params(tau, eps)
    assert sp.c_in * sp.c_out == pytest.approx(eps * eps * tau, rel=1e-12)
    assert sp.c_in + sp.c_out == pytest.approx(sp.s * tau, rel=1e-12)
    if tau >= eps * eps / 81:
        assert sp.regime == "factor" and sp.s == pytest.approx(18.0, rel=1e-12)
    else:
        assert sp.regime == "square" and sp.s == pytest.approx(2 * np.sqrt(eps * eps / tau), rel=1e-12)
    assert sp.beta == pytest.approx(tau / sp.c_in) and sp.beta <= 1.0
    # continuity at the switch
    t0 = eps * eps / 81
    a, b = vch_stage_params(t0 * (1 + 1e-12), eps), vch_stage_params(t0 * (1 - 1e-12), eps)
    assert a.c_in == pytest.approx(b.c_in, rel=1e-5) and a.s == pytest.approx(b.s, rel=1e-5)


@pytest.mark.parametrize("root", [2, 0])
@pytest.mark.parametrize("tau", [0.01, 5e-4])
def test_small_mode_decays_at_the_linear_rate_1d(root, tau):
    # About any root z_i the linearized model is v_t = -eps^2 v'''' + 18 v'' per component, so
    # one BE step multiplies cos(kx) by 1 / (1 + tau (18 k^2 + eps^2 k^4)).
    n, eps, k, delta = 256, 0.32, 2, 1e-6
    prob = Problem(nx=n, eps=eps, M=6, tol=1e-17, max_iter=200)
    x = nodes(n, 2 * np.pi, True)[None, :]
    a, b = cube_roots()[root]
    u1 = a + delta * np.cos(k * x)
    u2 = b + 0.5 * delta * np.cos(k * x)
    n1, n2, _ = VchSolver(prob).step(u1, u2, tau, "be")
    expect = 1.0 / (1.0 + tau * (18 * k * k + eps * eps * k ** 4))
    for comp, amp in ((n1 - a, delta), (n2 - b, 0.5 * delta)):
        proj = 2.0 / n * np.sum(comp * np.cos(k * x))
        assert proj / amp == pytest.approx(expect, rel=2e-5)


def test_small_mode_decays_at_the_linear_rate_2d():
    nx = ny = 96
    eps, tau, delta = 0.32, 0.02, 1e-6
    prob = Problem(nx=nx, ny=ny, eps=eps, M=6, tol=1e-17, max_iter=300)
    x = nodes(nx, 2 * np.pi, True)[None, :]
    y = nodes(ny, 2 * np.pi, True)[:, None]
    mode = np.cos(2 * x) * np.cos(y)
    u1, u2 = Z3[0] + delta * mode, Z3[1] - delta * mode
    n1, n2, _ = VchSolver(prob).step(u1, u2, tau, "be")
    k2 = 5.0
    expect = 1.0 / (1.0 + tau * (18 * k2 + eps * eps * k2 * k2))
    for comp, amp in ((n1 - Z3[0], delta), (n2 - Z3[1], -delta)):
        proj = 4.0 / (nx * ny) * np.sum(comp * mode)
        assert proj / amp == pytest.approx(expect, rel=5e-5)


@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_mass_conserved_and_energy_decreases(bc):
    # Eq. CH_vector conserves each component's integral and dissipates the energy of
    # Eq. EnergyFunctional_vector.  Mass is exact on periodic lines; with Neumann walls it holds
    # to discretization error (as for the scalar model).
    from oracle.solver import mass
    n = 48
    prob = Problem(nx=n, ny=n, bc=bc, eps=0.32, M=4, tol=1e-11, max_iter=1000)
    u1 = uniform_noise((n, n), 0.3, seed=11)
    u2 = uniform_noise((n, n), 0.3, seed=12)
    s = VchSolver(prob)
    m0 = (mass(prob, u1), mass(prob, u2))
    e_prev = vch_energy(prob, u1, u2)
    for step in range(4):
        u1, u2, info = s.step(u1, u2, 2e-3, "bdf2")
        assert info.converged
        e = vch_energy(prob, u1, u2)
        assert e < e_prev
        e_prev = e
    scale = prob.Lx * prob.Ly
    bound = 1e-10 if bc == "periodic" else 1e-3
    assert abs(mass(prob, u1) - m0[0]) < bound * scale
    assert abs(mass(prob, u2) - m0[1]) < bound * scale


def test_temporal_order_be_and_bdf2():
    # Successive errors against a fine reference fall by ~2 (BE) and ~4 (BDF2) per halving of dt.
    n, T = 64, 0.02
    prob = Problem(nx=n, eps=0.32, M=6, tol=1e-14, max_iter=2000)
    x = nodes(n, 2 * np.pi, True)
    # within 0.1 of z3, where |Hess W - 18 I| < 13 keeps the lagged iteration contracting
    u10 = Z3[0] + 0.1 * np.cos(x)
    u20 = Z3[1] + 0.1 * np.sin(2 * x)

    def run(dt, scheme):
        s = VchSolver(prob)
        a, b = u10[None, :], u20[None, :]
        for _ in range(int(round(T / dt))):
            a, b, _ = s.step(a, b, dt, scheme)
        return a, b

    ref = run(T / 256, "bdf2")
    for scheme, lo, hi in (("be", 1.8, 2.2), ("bdf2", 3.4, 5.0)):   # BDF2 nears 4 from above
        errs = []
        for dt in (T / 8, T / 16, T / 32):
            a, b = run(dt, scheme)
            errs.append(max(np.abs(a - ref[0]).max(), np.abs(b - ref[1]).max()))
        r = [errs[i] / errs[i + 1] for i in range(2)]
        assert all(lo < q < hi for q in r), (scheme, errs, r)


def test_paper_initial_state_stage_converges():
    # The paper's VCH run (Sec. 6.2.2): eps = 0.32, 64^2 nodes on [0, 2pi]^2, u1 from Eq. CH2D_initial,
    # u2 = sin(y); one BE stage of the fixed-point solve at dt = 1e-4 reaches N_tol = 1e-6 within
    # N_maxit = 400.  (At dt = 1e-3 this state, far from the wells, makes the lagged iteration
    # diverge: a step Algorithm 1 would reject.)
    n = 64
    prob = Problem(nx=n, ny=n, eps=0.32, M=4, tol=1e-6, max_iter=400)
    y = nodes(n, 2 * np.pi, True)[:, None]
    u1 = paper_ic_2d(n, n)
    u2 = np.sin(y) * np.ones((1, n))
    v1, v2 = u1 - Z3[0], u2 - Z3[1]
    res = vch_stage_solve(prob, v1, v2, v1, v2, 1e-4)
    assert res.converged and res.iters < 400


def test_dirichlet_walls_hold_z3():
    # Boundary conditions apply to v = u - z3, so homogeneous Dirichlet walls hold u = z3 after a step.
    n = 64
    prob = Problem(nx=n, bc="dirichlet", eps=0.32, M=4, tol=1e-12, max_iter=500)
    x = nodes(n, 2 * np.pi, False)[None, :]
    u1 = Z3[0] + 0.1 * np.sin(x / 2)
    u2 = Z3[1] + 0.05 * np.sin(x)
    n1, n2, info = VchSolver(prob).step(u1, u2, 1e-3, "be")
    assert info.converged
    for a, z in ((n1, Z3[0]), (n2, Z3[1])):
        assert abs(a[0, 0] - z) < 1e-13 and abs(a[0, -1] - z) < 1e-13


@pytest.mark.parametrize("estimator", ["richardson", "bdf2"])
def test_vch_lte_estimates_scale_as_dt_squared(estimator):
    # Both estimates are dominated by BE's local error, O(dt^2): halving dt divides eta by a factor
    # that tends to 4 (from below here: the stiff modes are not yet asymptotic).
    from oracle.vch import vch_adaptive_step
    n = 64
    prob = Problem(nx=n, eps=0.32, M=6, tol=1e-14, max_iter=3000)
    x = nodes(n, 2 * np.pi, True)[None, :]
    u1, u2 = Z3[0] + 0.1 * np.cos(x), Z3[1] + 0.1 * np.sin(2 * x)
    etas = []
    for dt in (5e-5, 2.5e-5, 1.25e-5):
        hist = None
        if estimator == "bdf2":
            p1, p2, _ = VchSolver(prob).step(u1, u2, dt, "be")      # history: one BE step of the same size
            hist, a1, a2 = {"u1": u1, "u2": u2, "dt": dt}, p1, p2
        else:
            a1, a2 = u1, u2
        _, _, info = vch_adaptive_step(VchSolver(prob), a1, a2, dt, 1.0, 1e-9, 1.0, estimator=estimator,
                                       history=hist)
        etas.append(info.eta)
    r1, r2 = etas[0] / etas[1], etas[1] / etas[2]
    assert 3.5 < r1 < 4.1 and 3.7 < r2 < 4.1 and r2 > r1, (r1, r2)


def test_vch_adaptive_run_keeps_mass_and_lowers_energy():
    from oracle.solver import mass
    from oracle.vch import vch_adaptive_step
    n = 48
    prob = Problem(nx=n, ny=n, eps=0.32, M=4, tol=1e-10, max_iter=400)
    x = nodes(n, 2 * np.pi, True)[None, :]
    y = nodes(n, 2 * np.pi, True)[:, None]
    u1 = Z3[0] + 0.1 * np.cos(x) * np.cos(y)
    u2 = Z3[1] + 0.1 * np.sin(x + y)
    e0, m0 = vch_energy(prob, u1, u2), (mass(prob, u1), mass(prob, u2))
    hist, dt, t = {}, 1e-4, 0.0
    s = VchSolver(prob)
    for _ in range(6):
        u1, u2, info = vch_adaptive_step(s, u1, u2, dt, 1e-4, 1e-8, 0.1, estimator="bdf2", history=hist)
        assert info.eta <= 1e-4
        t += info.dt_used
        dt = info.dt_next
    assert t > 6e-4                      # the controller grew the step
    assert vch_energy(prob, u1, u2) < e0
    assert abs(mass(prob, u1) - m0[0]) < 1e-9 and abs(mass(prob, u2) - m0[1]) < 1e-9
