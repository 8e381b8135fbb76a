"""GPU: the tensor-core row sweep (molt_helmholtz_rows_tc) against the FP64 oracle and against
the FP32 row sweep.

The chunk products run on FP16 high / low splits of the operands (three products accumulated in
FP32 in tensor memory).  Each split represents its operand to about 2^-22 relative, and the 144
window terms of a chunk row add in the tensor core's FP32 accumulator, so the sweep is held to
16 * 2^-22 (3.8e-6) of max|H f|, on lines of every supported length, quadrature order and decay.
Measured on a GB300 it sits at 1.5e-6 to 1.8e-6, against 1.4e-7 to 5.4e-7 for the FP32 sweep, so it
misses the FP32 sweeps' 1e-6 bar: the autotuner's accuracy gate keeps it out of the production
path (each record carries both errors).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.helmholtz import helmholtz_inverse  # noqa: E402
from paper_1611_04214_gb300.inputs import spacing, uniform_noise  # noqa: E402

from _parity import record  # noqa: E402

FP16_SPLIT_BAR = 16 * 2.0 ** -22


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


@pytest.mark.parametrize("n,nlines", [(1024, 16), (2048, 12), (8192, 8)])
@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("nu", [0.02, 0.3, 2.0])
def test_rows_tc_matches_oracle(n, nlines, M, nu):
    from paper_1611_04214_gb300.molt import Solver
    h = spacing(n, 2 * np.pi, True)
    c = (h / nu) ** 2
    f = uniform_noise((nlines, n), 1.0, seed=n + M, mean=1.0)
    with Solver(nx=n, ny=nlines, bc="periodic", quad_order=M, precision="fp32", eps=0.1) as s:
        fin = torch.tensor(f, dtype=torch.float32, device="cuda")
        out = torch.empty_like(fin)
        ref32 = torch.empty_like(fin)
        s.helmholtz_rows_tc(c, fin, out)
        s.helmholtz_apply(0, c, fin, ref32)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
        fp32 = ref32.double().cpu().numpy()
    ref = helmholtz_inverse(f.astype(np.float32).astype(np.float64), c, h, "periodic", M, axis=1)
    scale = np.abs(ref).max()
    err = float(np.abs(got - ref).max())
    record(f"rows_tc_{n}x{nlines}_M{M}_nu{nu}", err, 1e-6 * scale, FP16_SPLIT_BAR * scale, "fp16-split", None,
           fp32_sweep_err=float(np.abs(fp32 - ref).max() / scale))
    assert err <= FP16_SPLIT_BAR * scale, (err, scale)


def test_rows_tc_rejects_unsupported():
    from paper_1611_04214_gb300.molt import MoltError, Solver
    with Solver(nx=1000, ny=8, bc="periodic", precision="fp32") as s:
        a = torch.zeros(8, 1000, device="cuda")
        with pytest.raises(MoltError):
            s.helmholtz_rows_tc(0.01, a, torch.empty_like(a))
    with Solver(nx=1024, ny=8, bc="neumann", precision="fp32") as s:
        a = torch.zeros(8, 1024, device="cuda")
        with pytest.raises(MoltError):
            s.helmholtz_rows_tc(0.01, a, torch.empty_like(a))
