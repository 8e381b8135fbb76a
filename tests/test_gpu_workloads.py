"""GPU parity on the benchmark workloads themselves, element by element against the FP64 oracle.

* The 8192^2 SDIRK3 workload (eps = 0.02, dt = 5e-5, M = 4, u0 = 0.1 + 0.05 N(0,1)) at its full
  row length: a 8192 x 288 strip of its initial state with its node spacing, periodic and
  Dirichlet (u = -1 on the walls).  The row passes run the persistent pipelined row kernel with
  512 threads per 8192-node line; the column passes run the TMA column kernels over three tiles
  with a ragged tail.  One SDIRK3 step at the bench's fixed 10 fixed-point iterations per stage
  on both sides.
* The 1024^2 crop of the same problem (top-left block of the 8192^2 initial state, same h, eps,
  dt, posed with the same boundary condition on its own edges), FP32 and FP64, two SDIRK3 steps
  at 10 iterations per stage.
* The 1024^2 Neumann BDF2 workload (eps = 0.05, dt = 1e-4, u0 = 0.05 U[-1, 1]) iterated to the
  tolerance 1e-6 on a 128^2 crop with its node spacing: the fixed point is reached, so this is
  the converged step, with mass and energy checked along the way.  On this white-noise state the
  lagged 2D iteration contracts its highest mixed modes with rho = 0.9996 (measured by the
  oracle on this run), which puts the FP32 fixed point at about 2^-24 max|w| / (1 - rho) from
  the FP64 one: that case is checked against that bound and recorded (tests/_parity.py).
"""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.solver import OracleSolver, Problem, energy, mass  # noqa: E402
from paper_1611_04214_gb300.inputs import gaussian_noise_block, uniform_noise  # noqa: E402

from _parity import check_fp32, check_fp64, record  # noqa: E402

N3, EPS3, DT3, M3, ITERS3 = 8192, 0.02, 5e-5, 4, 10

# Known miss (tests/_parity.py): the Dirichlet variant's FP32 error after 30 to 60 fixed
# iterations is about 2.5e-6 of max|u|, as on the periodic variant, but its walls at u = -1 make
# max|u| four times the periodic one while the scale max|u + 1| stays the same; the oracle's own
# arithmetic with every sweep output rounded to FP32 lands at 2.2 x on the 1024^2 crop.
CH2D8192_DIRICHLET_MISS = (3.0, "FP32 rounding of the iteration at |u| = 1 walls, 60 fixed iterations")


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


def _ch2d8192_block(rows, cols, bc):
    """Top-left rows x cols block of the 8192^2 initial state, with its node spacing and lengths."""
    u = gaussian_noise_block((N3, N3), rows, cols, 0.05, seed=0, mean=0.1)
    h = 2 * np.pi / N3 if bc == "periodic" else 2 * np.pi / (N3 - 1)
    if bc == "dirichlet":
        u[0, :] = u[-1, :] = -1
        u[:, 0] = u[:, -1] = -1
    Lx = h * cols if bc == "periodic" else h * (cols - 1)
    Ly = h * rows if bc == "periodic" else h * (rows - 1)
    return u, Lx, Ly


@functools.lru_cache(maxsize=8)
def _oracle_fixed(rows, cols, bc, steps):
    """The oracle's SDIRK3 steps from the FP32-rounded start, ITERS3 iterations per stage."""
    u0, Lx, Ly = _ch2d8192_block(rows, cols, bc)
    start = u0.astype(np.float32).astype(np.float64)
    prob = Problem(nx=cols, ny=rows, Lx=Lx, Ly=Ly, bc=bc, eps=EPS3, M=M3, tol=1e-30, max_iter=ITERS3)
    o = OracleSolver(prob)
    u, iters = start, []
    for _ in range(steps):
        u, info = o.step(u, DT3, "sdirk3")
        iters.append(list(info.iters))
    return u, iters


def _gpu_fixed(rows, cols, bc, steps, precision):
    from paper_1611_04214_gb300.molt import Solver
    u0, Lx, Ly = _ch2d8192_block(rows, cols, bc)
    with Solver(nx=cols, ny=rows, Lx=Lx, Ly=Ly, bc=bc, eps=EPS3, quad_order=M3, precision=precision,
                tol=1e-30, max_iter=ITERS3) as s:
        u = torch.tensor(u0.astype(np.float32), device="cuda").to(s.dtype)
        iters = [s.step(u, DT3, "sdirk3", raise_on_nonconvergence=False).iters for _ in range(steps)]
        torch.cuda.synchronize()
        return u.double().cpu().numpy(), iters


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_ch2d8192_full_rows_fixed_iterations(bc):
    rows, cols = 288, N3
    got, ig = _gpu_fixed(rows, cols, bc, 1, "fp32")
    ref, io = _oracle_fixed(rows, cols, bc, 1)
    assert ig == io == [[ITERS3] * 3], (ig, io)
    check_fp32(f"ch2d8192_rows8192x288_sdirk3_{bc}_1step_10it", got, ref, np.abs(ref + 1).max(),
               known_miss=CH2D8192_DIRICHLET_MISS if bc == "dirichlet" else None)


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_ch2d8192_crop_1024(bc, precision):
    n = 1024
    got, ig = _gpu_fixed(n, n, bc, 2, precision)
    ref, io = _oracle_fixed(n, n, bc, 2)
    assert ig == io == [[ITERS3] * 3] * 2, (ig, io)
    case = f"ch2d8192_crop1024_sdirk3_{bc}_2steps_10it"
    scale = np.abs(ref + 1).max()
    if precision == "fp64":
        check_fp64(case + "_fp64", got, ref, 1e-11 * scale)
    else:
        check_fp32(case, got, ref, scale, known_miss=CH2D8192_DIRICHLET_MISS if bc == "dirichlet" else None)


# ---- the Neumann BDF2 workload, iterated to its tolerance on a 128^2 crop ----
N2, EPS2, DT2, TOL2, CROP2, STEPS2 = 1024, 0.05, 1e-4, 1e-6, 128, 3


def _ch2d1024_problem():
    h = 2 * np.pi / (N2 - 1)
    L = h * (CROP2 - 1)
    u0 = uniform_noise((CROP2, CROP2), 0.05, seed=0)
    return u0, L


@functools.lru_cache(maxsize=1)
def _oracle_ch2d1024():
    u0, L = _ch2d1024_problem()
    prob = Problem(nx=CROP2, ny=CROP2, Lx=L, Ly=L, bc="neumann", eps=EPS2, M=4, tol=TOL2, max_iter=20000)
    o = OracleSolver(prob)
    u = u0.astype(np.float32).astype(np.float64)
    iters, rho, conv = [], 0.0, []
    for _ in range(STEPS2):
        u, info = o.step(u, DT2, "bdf2")
        iters.append(info.iters[0])
        rho = max(rho, info.contraction)
        conv.append(info.residual < TOL2)
    return u, iters, rho, conv, prob


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_ch2d1024_crop_converged_steps(precision):
    from paper_1611_04214_gb300.molt import Solver
    u0, L = _ch2d1024_problem()
    ref, io, rho, conv, prob = _oracle_ch2d1024()
    assert all(conv), io        # the oracle reaches the tolerance at every step
    with Solver(nx=CROP2, ny=CROP2, Lx=L, Ly=L, bc="neumann", eps=EPS2, quad_order=4, precision=precision,
                tol=TOL2, max_iter=20000) as s:
        u = torch.tensor(u0.astype(np.float32), device="cuda").to(s.dtype)
        m0, e_prev = s.mass(u), s.energy(u)
        ig, monotone = [], True
        for _ in range(STEPS2):
            info = s.step(u, DT2, "bdf2")          # raises unless the stage reached its tolerance
            ig.append(info.iters[0])
            e = s.energy(u)
            monotone &= e <= e_prev * (1 + (1e-13 if precision == "fp64" else 1e-6))
            e_prev = e
        drift = abs(s.mass(u) - m0)
        got = u.double().cpu().numpy()
    scale = np.abs(ref + 1).max()
    case = f"ch2d1024_crop128_neumann_bdf2_tol1e-6_{STEPS2}steps"
    record(case + f"_{precision}_invariants", drift, 0, 0, "invariants", rho, iters_gpu=ig, iters_oracle=io,
           energy_monotone=bool(monotone))
    assert monotone
    # Neumann mass is conserved only to the discretization level of the local quadrature on rough
    # data; the GPU's drift is the oracle's
    start = u0.astype(np.float32).astype(np.float64)
    drift_ref = abs(mass(prob, ref) - mass(prob, start))
    assert abs(drift - drift_ref) <= (1e-10 if precision == "fp64" else 1e-6) * L * L + 1e-3 * drift_ref, \
        (drift, drift_ref)
    if precision == "fp64":
        # iteration counts equal up to a tie at the tolerance; one iteration more or less moves the
        # iterate by less than the tolerance
        assert all(abs(a - b) <= 1 for a, b in zip(ig, io)), (ig, io)
        check_fp64(case + "_fp64", got, ref, 2 * TOL2, iters_gpu=ig, iters_oracle=io)
    else:
        check_fp32(case, got, ref, scale, rho, rho_limited_w=np.abs(ref).max(), iters_gpu=ig, iters_oracle=io)
    assert energy(prob, got) <= energy(prob, u0.astype(np.float32).astype(np.float64))


def test_autotuned_solver_keeps_parity():
    # After molt_autotune (whatever kernel families it keeps on this GPU) the SDIRK3 workload's
    # 1024 x 288 periodic block still meets the FP32 bar against the oracle, and every sweep of a
    # step was tuned.
    from paper_1611_04214_gb300.molt import Solver
    rows, cols = 288, 1024
    u0, Lx, Ly = _ch2d8192_block(rows, cols, "periodic")
    with Solver(nx=cols, ny=rows, Lx=Lx, Ly=Ly, bc="periodic", eps=EPS3, quad_order=M3, precision="fp32",
                tol=1e-30, max_iter=ITERS3) as s:
        table = s.autotune()
        assert [(t["pass"], t["axis"]) for t in table] == [(0, "x"), (0, "y"), (1, "y"), (2, "x"), (3, "y"), (4, "x"),
                                                           (7, "y"), (8, "x")]
        assert all(t["chosen"] != "default" for t in table), table
        record("autotune_1024x288_periodic", 0.0, 0.0, 0.0, "autotune", None, table=table)
        u = torch.tensor(u0.astype(np.float32), device="cuda")
        iters = s.step(u, DT3, "sdirk3", raise_on_nonconvergence=False).iters
        got = u.double().cpu().numpy()
    ref, io = _oracle_fixed(rows, cols, "periodic", 1)
    assert [iters] == io
    check_fp32("ch2d8192_rows1024x288_sdirk3_periodic_autotuned", got, ref, np.abs(ref + 1).max())
