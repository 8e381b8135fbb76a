"""GPU: the TMA column kernels against the cp.async column kernels and the oracle.

Both kernel families evaluate the same fused multiply-adds in the same order (the TMA kernels
pair the two swept fields of a node in fma.rn.f32x2, which rounds each half exactly like fmaf),
so their outputs must agree bit for bit; the oracle bounds both to the FP32 sweep tolerance.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.helmholtz import helmholtz_inverse  # noqa: E402
from paper_1611_04214_gb300.inputs import paper_ic_2d, spacing, uniform_noise  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


def _tma_launches():
    from paper_1611_04214_gb300.molt import molt_column_tma_launches
    return molt_column_tma_launches()


def _columns(f, bc, M, c, tma, monkeypatch):
    from paper_1611_04214_gb300.molt import Solver
    monkeypatch.setenv("MOLT_COLS_TMA", "1" if tma else "0")
    n, nx = f.shape
    before = _tma_launches()
    with Solver(nx=nx, ny=n, bc=bc, quad_order=M, precision="fp32", eps=0.1) as s:
        fin = torch.tensor(f, dtype=torch.float32, device="cuda")
        out = torch.empty_like(fin)
        s.helmholtz_apply(1, c, fin, out)
        torch.cuda.synchronize()
        got = out.double().cpu().numpy()
    return got, _tma_launches() - before


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("n", [256, 300, 1000, 2049])
def test_tma_columns_bitwise_equal_and_match_oracle(bc, M, n, monkeypatch):
    # 256 = two full tiles; 300 and 2049 leave ragged last tiles (44 and 1 rows); 1000 spans 8.
    nx = 64
    h = spacing(n, 2 * np.pi, bc == "periodic")
    c = (h / 0.4) ** 2
    f = uniform_noise((n, nx), 1.0, seed=M * 7 + n, mean=1.0).astype(np.float32)
    got_tma, used = _columns(f, bc, M, c, True, monkeypatch)
    got_ref, unused = _columns(f, bc, M, c, False, monkeypatch)
    assert used == 2 and unused == 0, (used, unused)
    assert np.array_equal(got_tma, got_ref)
    ref = helmholtz_inverse(f.astype(np.float64), c, h, bc, M, axis=0)
    assert np.abs(got_tma - ref).max() / np.abs(ref).max() < 1e-6


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
@pytest.mark.parametrize("shape", [(288, 96), (300, 64)])
def test_tma_columns_in_2d_steps_bitwise(bc, shape, monkeypatch):
    # Passes 1 and 3 (two fields per node) and the rhs inverse run through the TMA kernels.
    from paper_1611_04214_gb300.molt import Solver
    ny, nx = shape
    u0 = paper_ic_2d(nx, ny, periodic=(bc == "periodic")).astype(np.float32)
    if bc == "dirichlet":
        u0[0, :] = u0[-1, :] = -1
        u0[:, 0] = u0[:, -1] = -1
    results = {}
    for tma in (True, False):
        monkeypatch.setenv("MOLT_COLS_TMA", "1" if tma else "0")
        before = _tma_launches()
        with Solver(nx=nx, ny=ny, bc=bc, quad_order=4, precision="fp32", eps=0.18, tol=1e-6, max_iter=60) as s:
            u = torch.tensor(u0, device="cuda")
            infos = [s.step(u, 0.01, "sdirk2", raise_on_nonconvergence=False) for _ in range(2)]
            torch.cuda.synchronize()
            results[tma] = (u.cpu().numpy(), [i.iters for i in infos], _tma_launches() - before)
    (a, ia, na), (b, ib, nb) = results[True], results[False]
    assert na > 0 and nb == 0, (na, nb)
    assert ia == ib
    assert np.array_equal(a, b)


@pytest.mark.parametrize("bc", ["periodic", "dirichlet"])
def test_block_order_does_not_change_2d_steps(bc, monkeypatch):
    # The alternating block orders of the 2D passes (lines and tile rows from the last one up in
    # passes 1-3) only reorder independent lines and tiles: the steps agree bit for bit with every
    # pass run from the first line down.  1024-node rows take the pipelined row kernel, 288-row
    # columns of 1024 lines the TMA column kernels.
    from paper_1611_04214_gb300.molt import Solver
    ny, nx = 288, 1024
    u0 = paper_ic_2d(nx, ny, periodic=(bc == "periodic")).astype(np.float32)
    if bc == "dirichlet":
        u0[0, :] = u0[-1, :] = -1
        u0[:, 0] = u0[:, -1] = -1
    results = {}
    for order in ("1", "0"):
        monkeypatch.setenv("MOLT_BLOCK_ORDER", order)
        with Solver(nx=nx, ny=ny, bc=bc, quad_order=4, precision="fp32", eps=0.18, tol=1e-6, max_iter=60) as s:
            u = torch.tensor(u0, device="cuda")
            infos = [s.step(u, 0.01, "sdirk2", raise_on_nonconvergence=False) for _ in range(2)]
            torch.cuda.synchronize()
            results[order] = (u.cpu().numpy(), [i.iters for i in infos])
    (a, ia), (b, ib) = results["1"], results["0"]
    assert ia == ib
    assert np.array_equal(a, b)
