"""GPU: BE steps of the sixth-order model on a 2D grid (molt_fch2d_*) against the 2D FCH oracle
(``oracle/fch.py``, ``fch2d_be_step``), FP64.

* Fixed iteration counts on both sides (tol below reach), periodic on a non-square domain and
  Neumann, and 288-row columns that span three column tiles with a ragged tail: held to 1e-11 of
  max|v|.
* Converged periodic steps to the same tolerance on both sides: iteration counts within 2 and the
  fields within 1e-9.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.fch import Fch2DSolver as Oracle2D  # noqa: E402
from oracle.solver import Problem  # noqa: E402
from paper_1611_04214_gb300.inputs import paper_ic_2d, uniform_noise  # noqa: E402

from _parity import check_fp64  # noqa: E402

EPS, ETA, DT = 0.18, 1.0, 0.05


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


def _field(ny, nx, bc, seed):
    return 0.8 * paper_ic_2d(nx, ny, bc == "periodic") + uniform_noise((ny, nx), 0.05, seed=seed)


def _run_both(u0, bc, steps, tol, max_iter, Ly, precision="fp64", oracle_tol=None, M=6):
    from paper_1611_04214_gb300.molt import Fch2D
    ny, nx = u0.shape
    prob = Problem(nx=nx, ny=ny, Lx=2 * np.pi, Ly=Ly, bc=bc, eps=EPS, M=M, tol=oracle_tol or tol, max_iter=max_iter)
    o = Oracle2D(prob, ETA)
    dtype = torch.float32 if precision == "fp32" else torch.float64
    ref, ig, io, rho = u0.astype(np.float64), [], [], 0.0
    with Fch2D(nx, ny, Ly=Ly, bc=bc, eps=EPS, eta=ETA, quad_order=M, tol=tol, max_iter=max_iter,
               precision=precision) as s:
        u = torch.tensor(u0, dtype=dtype, device="cuda")
        for _ in range(steps):
            ig.append(s.step(u, DT, raise_on_nonconvergence=False).iters[0])
            ref, res = o.step(ref, DT)
            io.append(res.iters)
            h = res.history
            if len(h) > 8:
                rho = max(rho, max(h[i + 1] / h[i] for i in range(len(h) // 2, len(h) - 1)))
        torch.cuda.synchronize()
        got = u.double().cpu().numpy()
    return got, ref, ig, io, rho


@pytest.mark.parametrize("bc,shape", [("periodic", (48, 64)), ("neumann", (36, 40)), ("periodic", (288, 64))])
def test_fch2d_fixed_iterations_fp64(bc, shape):
    ny, nx = shape
    u0 = _field(ny, nx, bc, seed=11)
    got, ref, ig, io, _ = _run_both(u0, bc, 2, 1e-30, 8, Ly=1.5 * np.pi)
    assert ig == io == [8, 8], (ig, io)
    check_fp64(f"fch2d_{nx}x{ny}_{bc}_2steps_8it_fp64", got, ref, 1e-11 * np.abs(ref + 1).max())


def test_fch2d_converged_fp64():
    ny, nx = 32, 32
    u0 = paper_ic_2d(nx, ny)
    got, ref, ig, io, _ = _run_both(u0, "periodic", 2, 1e-12, 5000, Ly=2 * np.pi)
    assert all(abs(a - b) <= 2 for a, b in zip(ig, io)), (ig, io)
    check_fp64("fch2d_32x32_periodic_2steps_converged_fp64", got, ref, 1e-9, iters_gpu=ig, iters_oracle=io)
