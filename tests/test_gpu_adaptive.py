"""GPU: adaptive step-size control (Sec. 5, Algorithm 1) with the Richardson (BE), BE-SDC2 and
BE-BDF2 LTE estimates.

1. Parity: from the stiff 1D initial state the GPU controller (FP64) takes the same accept /
   reject decisions and step sizes as the oracle's, and the fields agree to rounding.
2. The paper's experiment (Sec. 6.1, Table 1DCH_ripening_adaptive): 1D periodic, 128 nodes,
   eps = 0.18, tolerance 1e-11, N_maxit = 600, sigma_tol = 1e-3.  The paper prints ripening times
   between 8276.08 and 8320.03 for its adaptive runs; it does not state the initial step or the
   step bounds, so the check is that band, widened to 8250-8350.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.adaptive import AdaptiveHistory, adaptive_step  # noqa: E402
from oracle.solver import OracleSolver, Problem  # noqa: E402
from paper_1611_04214_gb300.inputs import paper_ic_1d  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


@pytest.mark.parametrize("estimator", ["richardson", "sdc2", "bdf2"])
def test_adaptive_controller_matches_oracle(estimator):
    from paper_1611_04214_gb300.molt import Solver
    n, tol_lte = 128, 1e-4
    prob = Problem(nx=n, eps=0.18, M=6, tol=1e-12, max_iter=600)
    o = OracleSolver(prob)
    hist = AdaptiveHistory()
    u_ref = paper_ic_1d(n)[None, :]
    with Solver(nx=n, ny=1, bc="periodic", eps=0.18, quad_order=6, precision="fp64", tol=1e-12, max_iter=600) as s:
        u = torch.tensor(paper_ic_1d(n), dtype=torch.float64, device="cuda")
        dt_gpu = dt_ref = 2e-3
        for _ in range(15):
            info = s.step_adaptive(u, dt_gpu, tol_lte, 1e-8, 10.0, estimator=estimator)
            u_ref, rinfo = adaptive_step(o, u_ref, dt_ref, tol_lte, 1e-8, 10.0, estimator=estimator,
                                        history=hist)
            assert info["rejections"] == rinfo.rejections
            assert info["dt_used"] == pytest.approx(rinfo.dt_used, rel=1e-9)
            assert info["eta"] == pytest.approx(rinfo.eta, rel=1e-6)
            dt_gpu, dt_ref = info["dt_next"], rinfo.dt_next
        got = u.cpu().numpy()
    assert np.abs(got - u_ref[0]).max() < 1e-10


@pytest.mark.parametrize("estimator", ["richardson", "sdc2", "bdf2"])
def test_adaptive_ripening_within_paper_band(estimator):
    from paper_1611_04214_gb300.molt import Solver
    n = 128
    with Solver(nx=n, ny=1, bc="periodic", eps=0.18, quad_order=6, precision="fp64", tol=1e-11, max_iter=600) as s:
        u = torch.tensor(paper_ic_1d(n), dtype=torch.float64, device="cuda")
        t, dt, steps = 0.0, 1e-3, 0
        while t < 12000.0 and steps < 200000:
            info = s.step_adaptive(u, dt, 1e-3, 1e-8, 1e3, estimator=estimator)
            t += info["dt_used"]
            dt = info["dt_next"]
            steps += 1
            if u[n // 2].item() < 0:
                break
    assert 8250.0 <= t <= 8350.0, (t, steps)


def test_bdf2_history_dropped_by_a_plain_step():
    # Without a previous accepted state BE-BDF2 takes a BE-SDC2 attempt, so it matches a solver
    # stepping with BE-SDC2; with one it does not.
    from paper_1611_04214_gb300.molt import Solver
    n = 128
    kw = dict(nx=n, ny=1, bc="periodic", eps=0.18, quad_order=6, precision="fp64", tol=1e-12, max_iter=600)
    with Solver(**kw) as sa, Solver(**kw) as sb:
        u = torch.tensor(paper_ic_1d(n), dtype=torch.float64, device="cuda")
        v = u.clone()

        def both(dt):
            a = sa.step_adaptive(u, dt, 1e-2, 1e-8, 1.0, estimator="bdf2")
            b = sb.step_adaptive(v, dt, 1e-2, 1e-8, 1.0, estimator="sdc2")
            return a, b

        a, b = both(1e-3)                      # first call: no history
        assert a["eta"] == pytest.approx(b["eta"], rel=1e-12)
        sa.step(u, 1e-3, "be")                 # a plain step drops the history
        sb.step(v, 1e-3, "be")
        a, b = both(1e-3)
        assert a["eta"] == pytest.approx(b["eta"], rel=1e-12)
        assert torch.allclose(u, v, rtol=0, atol=1e-14)
        a, b = both(a["dt_next"])              # history kept from the last call: BDF2
        assert abs(a["eta"] - b["eta"]) > 1e-3 * b["eta"]


def test_adaptive_rejects_unknown_estimator():
    from paper_1611_04214_gb300 import molt
    with molt.Solver(nx=64, ny=1, bc="periodic", eps=0.18, precision="fp64") as s:
        u = torch.zeros(64, dtype=torch.float64, device="cuda")
        a = molt._Adaptive(1e-3, 1e-8, 1.0, 0.8, 1.3, 7)
        assert s._lib.molt_step_adaptive(s._h, s._field(u), 1e-3, molt.ctypes.byref(a), None, None) \
            == molt.MOLT_ERR_ARG
