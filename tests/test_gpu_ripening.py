"""GPU: the 1D ripening experiment of Sec. 6.1 against the times the paper prints.

1D CH on [0, 2pi], periodic, 128 nodes, eps = 0.18, u0 of Eq. CH1D_initial, M = 6, fixed-point
tolerance 1e-11 (Sec. 6.1).  The ripening time is the first step time at which the midpoint value
u(pi, t) is negative.  Table 1DCH_ripeninglargedt prints, for fixed steps dt = 10 and dt = 1:
BE 8250.00 / 8296.00 and BDF2 8290.00 / 8303.00.  These are whole-run results of the method
(hundreds to thousands of steps in the factorization regime, tau / eps^2 up to 309), so they pin
every part of the solver at once; the FP64 oracle gives the same steps at dt = 10.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_1611_04214_gb300.inputs import paper_ic_1d  # noqa: E402

# (scheme, dt) -> ripening time printed in Table 1DCH_ripeninglargedt
PAPER_RIPENING = {("be", 10.0): 8250.0, ("bdf2", 10.0): 8290.0, ("be", 1.0): 8296.0, ("bdf2", 1.0): 8303.0}


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


def _ripening(scheme, dt, precision, t_max=12000.0):
    from paper_1611_04214_gb300.molt import Solver
    n = 128
    dtype = torch.float64 if precision == "fp64" else torch.float32
    tol = 1e-11 if precision == "fp64" else 1e-9
    with Solver(nx=n, ny=1, bc="periodic", eps=0.18, quad_order=6, precision=precision, tol=tol,
                max_iter=20000) as s:
        u = torch.tensor(paper_ic_1d(n), dtype=dtype, device="cuda")
        k = 0
        while k * dt < t_max:
            info = s.step(u, dt, scheme, raise_on_nonconvergence=False)
            assert info.status == 0, (scheme, dt, k, info.iters)
            k += 1
            if u[n // 2].item() < 0:
                return k * dt
    return None


@pytest.mark.parametrize("scheme,dt", sorted(PAPER_RIPENING))
def test_ripening_time_matches_paper_fp64(scheme, dt):
    assert _ripening(scheme, dt, "fp64") == PAPER_RIPENING[(scheme, dt)]

