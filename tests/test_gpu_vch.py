"""GPU: vector Cahn-Hilliard steps (Sec. 5.2) through the C ABI against the oracle.

FP64 parity element by element:
- 1D and 2D; periodic, Neumann and Dirichlet lines; BE and BDF2;
- ragged sizes spanning several row / column tiles;
- both stage regimes (tau >= eps^2/81 and below).

FP32 parity within the FP32 stopping floor.  The paper's configuration (eps = 0.32, 64^2 nodes,
u1 from Eq. CH2D_initial, u2 = sin y): parity, conserved mass, decreasing energy.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.solver import Problem, mass  # noqa: E402
from oracle.vch import VchSolver, Z3, vch_energy  # noqa: E402
from paper_1611_04214_gb300.inputs import nodes, paper_ic_2d, uniform_noise  # noqa: E402

from _parity import check_fp32  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


def _state(nx, ny, bc, seed):
    # smooth states near z3 that satisfy the walls (cosines for Neumann, half-sines for
    # Dirichlet), plus small noise on lines (1D).  In 2D the lagged iteration contracts slowly
    # on modes that are stiff in both directions (the splitting terms of Sec. 5.1), so 2D states
    # carry no grid-scale noise.
    periodic = bc == "periodic"
    x = nodes(nx, 2 * np.pi, periodic)[None, :]
    y = nodes(ny, 2 * np.pi, periodic)[:, None] if ny > 1 else np.zeros((1, 1))
    if bc == "dirichlet":
        p1 = 0.1 * np.sin(x / 2) * np.sin(y if ny > 1 else 1.0) + 0.05 * np.sin(3 * x / 2)
        p2 = 0.1 * np.sin(x) * (np.sin(y / 2) if ny > 1 else 1.0) + 0.05 * np.sin(x / 2)
    else:
        p1 = 0.1 * np.cos(x) * np.cos(2 * y) + 0.05 * np.cos(3 * x)
        p2 = 0.1 * np.cos(2 * x) * np.cos(y) + 0.05 * np.cos(3 * y)
    noise = 0.01 if ny == 1 else 0.0
    u1 = Z3[0] + p1 + uniform_noise((ny, nx), noise, seed=seed) * (1 if noise else 0)
    u2 = Z3[1] + p2 + uniform_noise((ny, nx), noise, seed=seed + 1) * (1 if noise else 0)
    if bc == "dirichlet":
        u1[..., 0] = u1[..., -1] = Z3[0]
        u2[..., 0] = u2[..., -1] = Z3[1]
    return u1, u2


def _run_both(nx, ny, bc, scheme, dt, steps, precision="fp64", tol=1e-13, M=4, eps=0.32, u0=None, oracle_tol=None):
    from paper_1611_04214_gb300.molt import Solver
    prob = Problem(nx=nx, ny=ny, bc=bc, eps=eps, M=M, tol=tol if oracle_tol is None else oracle_tol, max_iter=2000)
    u1, u2 = u0 if u0 is not None else _state(nx, ny, bc, seed=nx + ny)
    o = VchSolver(prob)
    r1, r2 = u1, u2
    dtype = torch.float64 if precision == "fp64" else torch.float32
    shape = (ny, nx) if ny > 1 else (nx,)
    g1 = torch.tensor(u1.reshape(shape), dtype=dtype, device="cuda")
    g2 = torch.tensor(u2.reshape(shape), dtype=dtype, device="cuda")
    iters_g, iters_o = [], []
    with Solver(nx=nx, ny=ny, bc=bc, eps=eps, quad_order=M, precision=precision, tol=tol, max_iter=2000) as s:
        for _ in range(steps):
            info = s.vch_step(g1, g2, dt, scheme)
            r1, r2, oinfo = o.step(r1, r2, dt, scheme)
            assert oinfo.converged
            iters_g.append(info.iters[0])
            iters_o.append(oinfo.iters[0])
        out = (g1.double().cpu().numpy().reshape(ny, nx), g2.double().cpu().numpy().reshape(ny, nx))
    return out, (r1.reshape(ny, nx), r2.reshape(ny, nx)), iters_g, iters_o, prob


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
@pytest.mark.parametrize("scheme", ["be", "bdf2"])
@pytest.mark.parametrize("dt", [5e-3, 5e-4])
def test_vch_fp64_parity_1d(bc, scheme, dt):
    (g1, g2), (o1, o2), ig, io, _ = _run_both(333, 1, bc, scheme, dt, 4, M=6)
    assert max(np.abs(g1 - o1).max(), np.abs(g2 - o2).max()) < 1e-11
    assert all(abs(a - b) <= 1 for a, b in zip(ig, io)), (ig, io)


@pytest.mark.parametrize("bc,dims,dt", [("periodic", (200, 136), 2e-3), ("neumann", (200, 136), 2e-3),
                                        ("dirichlet", (160, 136), 5e-4)])
@pytest.mark.parametrize("scheme", ["be", "bdf2"])
def test_vch_fp64_parity_2d(bc, dims, dt, scheme):
    (g1, g2), (o1, o2), ig, io, _ = _run_both(dims[0], dims[1], bc, scheme, dt, 3, tol=1e-12)
    assert max(np.abs(g1 - o1).max(), np.abs(g2 - o2).max()) < 1e-10
    assert all(abs(a - b) <= 2 for a, b in zip(ig, io)), (ig, io)


def test_vch_fp64_parity_2d_square_regime():
    (g1, g2), (o1, o2), _, _, _ = _run_both(160, 144, "periodic", "bdf2", 5e-4, 3, tol=1e-12)
    assert max(np.abs(g1 - o1).max(), np.abs(g2 - o2).max()) < 1e-10


# (1000, 1) and (256, 200) run the generic kernels; (1024, 1) and (1024, 40) the pipelined row
# kernel (vector passes a and 2); (64, 288) the TMA column kernel (vector pass 1) over three tiles
@pytest.mark.parametrize("dims", [(1000, 1), (256, 200), (1024, 1), (1024, 40), (64, 288)])
@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_vch_fp32_parity(dims, bc):
    from paper_1611_04214_gb300 import molt
    nx, ny = dims
    t0 = molt.molt_column_tma_launches()
    (g1, g2), (o1, o2), _, _, _ = _run_both(nx, ny, bc, "bdf2", 2e-3, 3, precision="fp32", tol=1e-7,
                                            oracle_tol=1e-13)
    # FP32 fixed points (the FP32 solve stops at its rounding floor) against a tightly converged
    # FP64 oracle, held to 1e-6 of max|u|
    check_fp32(f"vch_fp32_{nx}x{ny}_{bc}_bdf2_3steps", np.stack([g1, g2]), np.stack([o1, o2]),
               max(np.abs(o1).max(), np.abs(o2).max()))
    if dims == (64, 288):
        assert molt.molt_column_tma_launches() > t0


def test_vch_paper_configuration():
    # Sec. 6.2.2: eps = 0.32, dx = dy = 2pi/64, N_tol = 1e-6, N_maxit = 400; u1 from Eq. CH2D_initial,
    # u2 = sin(y).  Steps of dt = 1e-4 from that far-from-equilibrium state.
    n = 64
    y = nodes(n, 2 * np.pi, True)[:, None]
    u1 = paper_ic_2d(n, n)
    u2 = np.sin(y) * np.ones((1, n))
    (g1, g2), (o1, o2), _, _, prob = _run_both(n, n, "periodic", "bdf2", 1e-4, 5, tol=1e-12, u0=(u1, u2))
    assert max(np.abs(g1 - o1).max(), np.abs(g2 - o2).max()) < 1e-10
    assert abs(mass(prob, g1) - mass(prob, u1)) < 1e-10
    assert abs(mass(prob, g2) - mass(prob, u2)) < 1e-10
    assert vch_energy(prob, g1, g2) < vch_energy(prob, u1, u2)


def test_vch_arguments_and_scalar_state():
    from paper_1611_04214_gb300 import molt
    n = 96
    with molt.Solver(nx=n, ny=n, bc="periodic", eps=0.32, precision="fp64", tol=1e-12) as s, \
            molt.Solver(nx=n, ny=n, bc="periodic", eps=0.32, precision="fp64", tol=1e-12) as fresh:
        a = torch.zeros(n, n, dtype=torch.float64, device="cuda")
        with pytest.raises(molt.MoltError):
            s.vch_step(a, a, 1e-3)
        with pytest.raises(molt.MoltError) as ei:
            s.vch_step(a, a.clone(), 1e-3, "sdirk2")
        assert ei.value.status == molt.MOLT_ERR_UNSUPPORTED
        u1, u2 = (torch.tensor(x, device="cuda") for x in _state(n, n, "periodic", 3))
        s.vch_step(u1, u2, 1e-3, "bdf2")
        # a scalar step after vector steps matches a fresh solver bit for bit
        u = torch.tensor(uniform_noise((n, n), 0.05, seed=4), device="cuda")
        v = u.clone()
        for _ in range(2):
            a_info = s.step(u, 1e-4, "bdf2", raise_on_nonconvergence=False)
            b_info = fresh.step(v, 1e-4, "bdf2", raise_on_nonconvergence=False)
            assert a_info.iters == b_info.iters
        assert torch.equal(u, v)


def test_vch_three_phase_mixture_crop_fixed_iterations():
    # The shape of the 4096^2 three-phase workload on a 96 x 80 Neumann crop with its node spacing
    # (2pi/4095), eps = 0.03 and a Dirichlet(1, 1, 1) mixture: one BE start and two BDF2 steps of
    # dt = 1e-6, each stage capped at 40 fixed-point iterations (the grid-scale mixture contracts
    # slowly), on both sides the same iterations.
    from paper_1611_04214_gb300.inputs import three_phase_mixture
    from paper_1611_04214_gb300.molt import Solver
    nx, ny, h = 96, 80, 2 * np.pi / 4095
    prob = Problem(nx=nx, ny=ny, Lx=(nx - 1) * h, Ly=(ny - 1) * h, bc="neumann", eps=0.03, M=4, tol=1e-14,
                   max_iter=40)
    u1, u2 = three_phase_mixture((ny, nx), seed=7)
    o = VchSolver(prob)
    r1, r2 = u1, u2
    g1 = torch.tensor(u1, device="cuda")
    g2 = torch.tensor(u2, device="cuda")
    with Solver(nx=nx, ny=ny, Lx=prob.Lx, Ly=prob.Ly, bc="neumann", eps=0.03, quad_order=4, precision="fp64",
                tol=1e-14, max_iter=40) as s:
        for _ in range(3):
            info = s.vch_step(g1, g2, 1e-6, "bdf2", raise_on_nonconvergence=False)
            r1, r2, oinfo = o.step(r1, r2, 1e-6, "bdf2")
            assert info.iters[0] == oinfo.iters[0] == 40
        got = (g1.cpu().numpy(), g2.cpu().numpy())
    assert max(np.abs(got[0] - r1).max(), np.abs(got[1] - r2).max()) < 1e-11


@pytest.mark.parametrize("bc", ["neumann", "periodic"])
def test_vch_fp32_three_phase_mixture_fixed_iterations(bc):
    # FP32 on the shape of the 4096^2 three-phase workload (96 x 80 crop, node spacing 2pi/4095,
    # eps = 0.03, Dirichlet(1, 1, 1) mixture, one BE start and two BDF2 steps of dt = 1e-6), each
    # stage capped at 40 fixed-point iterations on both sides, against the FP64 oracle.
    from paper_1611_04214_gb300.inputs import three_phase_mixture
    from paper_1611_04214_gb300.molt import Solver
    nx, ny = 96, 80
    h = 2 * np.pi / 4095 if bc == "neumann" else 2 * np.pi / 4096
    Lx, Ly = ((nx - 1) * h, (ny - 1) * h) if bc == "neumann" else (nx * h, ny * h)
    prob = Problem(nx=nx, ny=ny, Lx=Lx, Ly=Ly, bc=bc, eps=0.03, M=4, tol=1e-30, max_iter=40)
    u1, u2 = three_phase_mixture((ny, nx), seed=7)
    u1 = u1.astype(np.float32).astype(np.float64)
    u2 = u2.astype(np.float32).astype(np.float64)
    o = VchSolver(prob)
    r1, r2 = u1, u2
    g1 = torch.tensor(u1, dtype=torch.float32, device="cuda")
    g2 = torch.tensor(u2, dtype=torch.float32, device="cuda")
    with Solver(nx=nx, ny=ny, Lx=Lx, Ly=Ly, bc=bc, eps=0.03, quad_order=4, precision="fp32", tol=1e-30,
                max_iter=40) as s:
        for _ in range(3):
            info = s.vch_step(g1, g2, 1e-6, "bdf2", raise_on_nonconvergence=False)
            r1, r2, oinfo = o.step(r1, r2, 1e-6, "bdf2")
            assert info.iters[0] == oinfo.iters[0] == 40
        got = np.stack([g1.double().cpu().numpy(), g2.double().cpu().numpy()])
    # Known miss (tests/_parity.py): on this grid-scale mixture the lagged term carries the linear
    # part s v with s = (c1 + c2)/tau = 73 and each stage runs 40 iterations; rounding only the
    # oracle's own iterate v = u - z3 to FP32 after every iteration already gives 1.5 x (periodic)
    # and 0.55 x (Neumann) the target, every sweep output rounded gives 5.2 x and 2.6 x.
    guard = {"periodic": 12.0, "neumann": 5.5}[bc]
    check_fp32(f"vch_fp32_mixture_crop96x80_{bc}_bdf2_40it", got, np.stack([r1, r2]),
               max(np.abs(r1).max(), np.abs(r2).max()),
               known_miss=(guard, "FP32 rounding over 120 iterations of a grid-scale mixture, s = 73"))


@pytest.mark.parametrize("estimator", ["richardson", "bdf2"])
@pytest.mark.parametrize("bc", ["periodic", "neumann"])
def test_vch_adaptive_matches_oracle(estimator, bc):
    # Algorithm 1 for the vector model (Sec. 6.2.2) in FP64 on a 48 x 40 grid: the GPU controller
    # takes the oracle's decisions, step sizes and rejections step for step, and its fields match.
    from oracle.vch import vch_adaptive_step
    from paper_1611_04214_gb300.molt import Solver
    nx, ny = 48, 40
    prob = Problem(nx=nx, ny=ny, bc=bc, eps=0.32, M=4, tol=1e-12, max_iter=400)
    u1, u2 = _state(nx, ny, bc, seed=5)
    hist, dt = {}, 2e-4
    o1, o2 = u1.copy(), u2.copy()
    g1 = torch.tensor(u1, device="cuda")
    g2 = torch.tensor(u2, device="cuda")
    with Solver(nx=nx, ny=ny, bc=bc, eps=0.32, quad_order=4, precision="fp64", tol=1e-12, max_iter=400) as s:
        for _ in range(5):
            gi = s.vch_step_adaptive(g1, g2, dt, 1e-4, 1e-8, 0.1, estimator=estimator)
            o1, o2, oi = vch_adaptive_step(VchSolver(prob), o1, o2, dt, 1e-4, 1e-8, 0.1, estimator=estimator,
                                           history=hist if estimator == "bdf2" else None)
            assert gi["rejections"] == oi.rejections
            assert abs(gi["dt_used"] - oi.dt_used) <= 1e-12 * oi.dt_used
            assert abs(gi["dt_next"] - oi.dt_next) <= 1e-6 * oi.dt_next
            assert abs(gi["eta"] - oi.eta) <= 1e-6 * oi.eta + 1e-14
            dt = oi.dt_next
        got = (g1.cpu().numpy(), g2.cpu().numpy())
    assert max(np.abs(got[0] - o1).max(), np.abs(got[1] - o2).max()) < 1e-10
