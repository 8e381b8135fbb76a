"""GPU: BE steps of the sixth-order model on independent 1D lines (molt_fch1d_*) against the 1D
FCH oracle (``oracle/fch.py``).

* Fixed iteration counts (tol below reach) on both sides, FP64, periodic and Neumann, four
  different lines per field (a ragged line of 200 nodes spans 13 chunks of 16 with a tail of 8):
  held to 1e-11 of max|v|.
* Fixed iteration counts with M = 2, 4 and eta = 1, 3 (FP64, 1e-11 of max|v|).
* Converged steps, FP64, to the same tolerance on both sides: iteration counts within 2 and the
  fields within 1e-10 (the iteration contracts with rho = 0.95 at dt = 0.05, eps = 0.18, so each
  side's distance to the fixed point is below tol rho / (1 - rho) = 2e-12).
* Converged steps, FP32 (the FP32 stopping rule): the rho-limited bar of tests/_parity.py,
  72 ulp max|v| / (1 - rho), since rho = 0.95 puts the FP32 fixed point's rounding level above
  the strict 1e-6.
* 4096 lines of 1024 nodes (the launch grid of a large field) made of 8 distinct lines repeated:
  every copy equals its first copy, and the 8 match the oracle (the stopping rule's max over all
  lines is the max over the 8).
* A small mode about u = -1 decays by the linearised rate of Eq. FCH0 (the oracle's pin, on
  the GPU path), and periodic mass is kept.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.fch import FchSolver as OracleFch  # noqa: E402
from oracle.solver import Problem  # noqa: E402
from paper_1611_04214_gb300.inputs import paper_ic_1d, uniform_noise  # noqa: E402

from _parity import check_fp32, check_fp64  # noqa: E402

EPS, ETA, DT = 0.18, 1.0, 0.05


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


def _lines(n, periodic):
    ic = paper_ic_1d(n, periodic)
    return np.stack([ic, 0.9 * ic[::-1], uniform_noise((1, n), 0.3, seed=3, mean=-0.1)[0],
                     uniform_noise((1, n), 0.05, seed=4, mean=0.2)[0]])


def _run_both(u0, bc, steps, tol, max_iter, precision="fp64", oracle_tol=None, dt=DT, M=6, eta=ETA):
    from paper_1611_04214_gb300.molt import Fch1D
    lines, n = u0.shape
    prob = Problem(nx=n, eps=EPS, M=M, tol=oracle_tol or tol, max_iter=max_iter, bc=bc)
    o = OracleFch(prob, eta)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    ref, its_o, its_g, rho = u0.astype(np.float64), [], [], 0.0
    with Fch1D(n, lines, bc=bc, eps=EPS, eta=eta, quad_order=M, tol=tol, max_iter=max_iter,
               precision=precision) as s:
        u = torch.tensor(u0, dtype=dtype, device="cuda")
        for _ in range(steps):
            its_g.append(s.step(u, dt, raise_on_nonconvergence=False).iters[0])
            ref, res = o.step(ref, dt)
            its_o.append(res.iters)
            h = res.history
            if len(h) > 8:
                rho = max(rho, max(h[i + 1] / h[i] for i in range(len(h) // 2, len(h) - 1)))
        torch.cuda.synchronize()
        launches = s.kernel_launches()
        got = u.double().cpu().numpy()
    return got, ref, its_g, its_o, rho, launches


@pytest.mark.parametrize("bc,n", [("periodic", 200), ("neumann", 136)])
def test_fch_fixed_iterations_fp64(bc, n):
    u0 = _lines(n, bc == "periodic")
    got, ref, ig, io, _, launches = _run_both(u0, bc, 2, 1e-30, 25)
    assert ig == io == [25, 25], (ig, io)
    assert launches > 2 * 25 * 14
    check_fp64(f"fch1d_{n}x4_{bc}_2steps_25it_fp64", got, ref, 1e-11 * np.abs(ref + 1).max())


@pytest.mark.parametrize("eta", [1.0, 3.0])
@pytest.mark.parametrize("M", [2, 4])
@pytest.mark.parametrize("bc,n", [("periodic", 200), ("neumann", 136)])
def test_fch_orders_and_eta_fp64(bc, n, M, eta):
    # the quadrature orders M = 2, 4 and a stronger eta (both contract at dt = 0.05, rho <= 0.95)
    u0 = _lines(n, bc == "periodic")
    got, ref, ig, io, _, _ = _run_both(u0, bc, 1, 1e-30, 15, M=M, eta=eta)
    assert ig == io == [15], (ig, io)
    check_fp64(f"fch1d_{n}x4_{bc}_M{M}_eta{eta:g}_1step_15it_fp64", got, ref, 1e-11 * np.abs(ref + 1).max())


@pytest.mark.parametrize("bc,n", [("periodic", 200), ("neumann", 136)])
def test_fch_converged_fp64(bc, n):
    u0 = _lines(n, bc == "periodic")
    got, ref, ig, io, rho, _ = _run_both(u0, bc, 3, 1e-13, 3000)
    assert all(abs(a - b) <= 2 for a, b in zip(ig, io)), (ig, io)
    assert rho < 0.97, rho
    check_fp64(f"fch1d_{n}x4_{bc}_3steps_converged_fp64", got, ref, 1e-10, iters_gpu=ig, iters_oracle=io)


@pytest.mark.parametrize("bc,n", [("periodic", 200), ("neumann", 136)])
def test_fch_converged_fp32(bc, n):
    u0 = _lines(n, bc == "periodic").astype(np.float32)
    got, ref, ig, io, rho, _ = _run_both(u0, bc, 3, 1e-10, 3000, precision="fp32", oracle_tol=1e-13)
    assert max(ig) < 3000, ig
    check_fp32(f"fch1d_{n}x4_{bc}_3steps_converged_fp32", got, ref, np.abs(ref + 1).max(), rho,
               rho_limited_w=np.abs(ref + 1).max(), iters_gpu=ig, iters_oracle=io)


def test_fch_many_lines_fp64():
    from paper_1611_04214_gb300.molt import Fch1D
    n, distinct, copies = 1024, 8, 512
    base = np.concatenate([_lines(n, True), 0.5 * _lines(n, True)[:, ::-1]])
    prob = Problem(nx=n, eps=EPS, M=6, tol=1e-12, max_iter=3000)
    ref, res = OracleFch(prob, ETA).step(base, DT)
    with Fch1D(n, distinct * copies, eps=EPS, eta=ETA, quad_order=6, tol=1e-12, max_iter=3000) as s:
        u = torch.tensor(np.tile(base, (copies, 1)), dtype=torch.float64, device="cuda")
        info = s.step(u, DT)
        torch.cuda.synchronize()
        got = u.cpu().numpy().reshape(copies, distinct, n)
    assert abs(info.iters[0] - res.iters) <= 2, (info.iters, res.iters)
    assert np.abs(got - got[:1]).max() <= 1e-14
    check_fp64("fch1d_1024x4096_periodic_1step_converged_fp64", got[0], ref, 1e-9,
               iters_gpu=info.iters, iters_oracle=[res.iters])


def test_fch_small_mode_rate_and_mass():
    from paper_1611_04214_gb300.molt import Fch1D
    n, k, amp = 128, 2, 1e-7
    x = 2 * np.pi * np.arange(n) / n
    u0 = np.stack([-1.0 + amp * np.cos(k * x), paper_ic_1d(n)])
    with Fch1D(n, 2, eps=EPS, eta=ETA, quad_order=6, tol=1e-13, max_iter=3000) as s:
        u = torch.tensor(u0, dtype=torch.float64, device="cuda")
        s.step(u, DT)
        torch.cuda.synchronize()
        got = u.cpu().numpy()
    k2 = float(k * k)
    rate = 1.0 / (1.0 + DT * k2 * (EPS ** 2 * k2 + 2) * (EPS ** 2 * k2 + 2 - ETA * EPS ** 2))
    assert np.abs(got[0] + 1.0 - rate * (u0[0] + 1.0)).max() < 1e-4 * amp
    assert abs(got[1].mean() - u0[1].mean()) < 1e-13
