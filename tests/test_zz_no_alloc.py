"""The allocation-free column sweep (molt_helmholtz_columns_noalloc) against the solver's column
sweep (molt_helmholtz_apply, axis 1), both through the C ABI.

The entry point exists for callers that cannot call cudaMalloc (code under a memory manager
that owns all device memory, or latency-critical loops that must not allocate): its scan
scratch is a static device array shared by every call.  Two calls in a row with different
inputs check that no state leaks from one call into the next.  This file is collected last so
that a failure here comes after every other test has run."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
@pytest.mark.parametrize("shape", [(300, 96), (1000, 100)])   # pipelined and general column kernels
def test_noalloc_columns_match_solver_sweep(bc, shape):
    from paper_1611_04214_gb300.inputs import spacing, uniform_noise
    from paper_1611_04214_gb300.molt import (Solver, molt_helmholtz_columns_noalloc,
                                             molt_helmholtz_columns_noalloc_status)
    ny, nx = shape
    L = 2 * np.pi
    h = spacing(ny, L, bc == "periodic")
    with Solver(nx=nx, ny=ny, bc=bc, quad_order=4, precision="fp32", eps=0.1, Lx=L, Ly=L) as s:
        for call, (nu, seed) in enumerate([(0.08, 1), (1.5, 2)]):
            c = (h / nu) ** 2
            f = torch.tensor(uniform_noise((ny, nx), 1.0, seed=seed, mean=1.0), dtype=torch.float32, device="cuda")
            ref = torch.empty_like(f)
            got = torch.full_like(f, float("nan"))
            s.helmholtz_apply(1, c, f, ref)
            molt_helmholtz_columns_noalloc(nx, ny, L, bc, 4, c, f, got)
            assert molt_helmholtz_columns_noalloc_status() == 0, call   # every tile copy arrived
            torch.cuda.synchronize()
            r, g = ref.double().cpu().numpy(), got.double().cpu().numpy()
            assert np.all(np.isfinite(g)), call
            assert np.abs(g - r).max() <= 1e-6 * np.abs(r).max(), call


def test_noalloc_rejects_oversized_grid():
    from paper_1611_04214_gb300.molt import MoltError, molt_helmholtz_columns_noalloc
    ny, nx = 8192, 8192            # 64 tiles x 8192 columns exceeds the 4 MiB static scratch
    f = torch.zeros((ny, nx), dtype=torch.float32, device="cuda")
    out = torch.empty_like(f)
    with pytest.raises(MoltError, match="static scratch"):
        molt_helmholtz_columns_noalloc(nx, ny, 1.0, "periodic", 4, 1e-6, f, out)
