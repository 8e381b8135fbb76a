"""GPU: batched instances (molt_batch_*) against the single-instance solver and the oracle.

For instances whose rows are shorter than 1024 nodes and whose columns are shorter than 256, the
single-instance solver runs the same general row / column block bodies, the same stopping rule
and the same pointwise kernels as the batched passes, so every instance of a batch must match a
single-instance run of the same problem bit for bit, iteration counts included.  Against the
oracle, every instance is held to 1e-6 of max|u + 1| (tests/_parity.py).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle.solver import OracleSolver, Problem  # noqa: E402
from paper_1611_04214_gb300.inputs import uniform_noise  # noqa: E402

from _parity import check_fp32  # noqa: E402

# converged cases whose contraction factor puts 1e-6 below the FP32 rounding floor (rho measured by
# the oracle on the same run)
BATCH_RHO_LIMITED = {
    "batch_instance4_64x24_neumann_be_2steps_converged",     # rho = 0.991
    "batch_instance4_64x24_dirichlet_be_2steps_converged",   # rho = 0.955
}


@pytest.fixture(scope="module", autouse=True)
def _library():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1611_04214_gb300 import build
    build.build_library()


# (nx, ny, Lx, Ly, eps, dt): square and factorization regimes, uneven sizes and aspect ratios
INSTANCES = [
    (40, 56, 2 * np.pi, 2 * np.pi, 0.10, 2e-3),
    (96, 72, 3.0, 2.0, 0.06, 1e-3),
    (48, 128, 2 * np.pi, 4.0, 0.15, 5e-3),
    (33, 40, 1.5, 1.9, 0.08, 8e-4),
    (64, 24, 2.0, 1.0, 0.05, 3e-3),      # tau >= eps^2: factorization regime
]


def _initial(bc, seed, nx, ny):
    u = uniform_noise((ny, nx), 0.05, seed=seed, mean=0.0)
    if bc == "dirichlet":
        u[0, :] = u[-1, :] = -1
        u[:, 0] = u[:, -1] = -1
    return u.astype(np.float32)


def _run_batch(bc, scheme, steps, mode="graph", tol=1e-6, max_iter=300):
    from paper_1611_04214_gb300.molt import Batch
    inst = [(nx, ny, Lx, Ly, eps) for (nx, ny, Lx, Ly, eps, _) in INSTANCES]
    dts = [dt for (*_, dt) in INSTANCES]
    with Batch(inst, bc=bc, quad_order=4, tol=tol, max_iter=max_iter) as b:
        b.set_execution(mode)
        u0 = [_initial(bc, 10 + i, nx, ny) for i, (nx, ny, *_rest) in enumerate(INSTANCES)]
        u = torch.tensor(b.pack(u0), device="cuda")
        infos = [b.step(u, dts, scheme, raise_on_nonconvergence=False) for _ in range(steps)]
        torch.cuda.synchronize()
        out = b.unpack(u.cpu().numpy())
    return u0, out, infos


def _run_single(bc, scheme, steps, i, u0, tol=1e-6, max_iter=300):
    from paper_1611_04214_gb300.molt import Solver
    nx, ny, Lx, Ly, eps, dt = INSTANCES[i]
    with Solver(nx=nx, ny=ny, Lx=Lx, Ly=Ly, bc=bc, eps=eps, quad_order=4, precision="fp32", tol=tol,
                max_iter=max_iter) as s:
        u = torch.tensor(u0, device="cuda")
        infos = [s.step(u, dt, scheme, raise_on_nonconvergence=False) for _ in range(steps)]
        torch.cuda.synchronize()
        return u.cpu().numpy(), [inf.iters[0] for inf in infos], [inf.status for inf in infos]


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
@pytest.mark.parametrize("scheme,steps", [("be", 2), ("bdf2", 3)])
def test_batch_equals_single_instance_bitwise(bc, scheme, steps):
    u0, out, infos = _run_batch(bc, scheme, steps)
    for i in range(len(INSTANCES)):
        ref, iters, status = _run_single(bc, scheme, steps, i, u0[i])
        assert [inf.iters[i] for inf in infos] == iters, (i, iters)
        assert [inf.instance_status[i] for inf in infos] == status, (i, status)
        assert np.array_equal(out[i], ref), (i, np.abs(out[i] - ref).max())


@pytest.mark.parametrize("bc", ["neumann", "dirichlet"])
def test_batch_graph_equals_host_loop(bc):
    _, a, ia = _run_batch(bc, "bdf2", 3, mode="graph")
    _, b, ib = _run_batch(bc, "bdf2", 3, mode="host_loop")
    assert [x.iters for x in ia] == [x.iters for x in ib]
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
def test_batch_matches_oracle_fixed_iterations(bc):
    # Every instance and the oracle run the same 8 fixed-point iterations per stage (the FP32 stop
    # rules never fire that early), so the difference is the FP32 rounding of the batched passes,
    # held to 1e-6 of max|u + 1|.
    u0, out, infos = _run_batch(bc, "be", 2, tol=1e-30, max_iter=8)
    for i in range(len(INSTANCES)):
        nx, ny, Lx, Ly, eps, dt = INSTANCES[i]
        o = OracleSolver(Problem(nx=nx, ny=ny, Lx=Lx, Ly=Ly, bc=bc, eps=eps, M=4, tol=1e-30, max_iter=8))
        u = u0[i].astype(np.float64)
        for k in range(2):
            u, info = o.step(u, dt, "be")
            assert infos[k].iters[i] == info.iters[0] == 8
        check_fp32(f"batch_instance{i}_{nx}x{ny}_{bc}_be_2steps_8it", out[i], u, np.abs(u + 1).max())


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
def test_batch_matches_oracle_converged(bc):
    # Converged steps (tolerance 1e-10, which FP32 replaces by its rounding floor) against the
    # oracle converged to 1e-11; instances whose iteration contracts slowly are rho-limited
    # (tests/_parity.py) and named in BATCH_RHO_LIMITED.
    u0, out, infos = _run_batch(bc, "be", 2, tol=1e-10, max_iter=3000)
    for i in (0, 3, 4):
        nx, ny, Lx, Ly, eps, dt = INSTANCES[i]
        prob = Problem(nx=nx, ny=ny, Lx=Lx, Ly=Ly, bc=bc, eps=eps, M=4, tol=1e-11, max_iter=3000)
        o = OracleSolver(prob)
        u = u0[i].astype(np.float64)
        rho = 0.0
        for _ in range(2):
            u, info = o.step(u, dt, "be")
            rho = max(rho, info.contraction)
        case = f"batch_instance{i}_{nx}x{ny}_{bc}_be_2steps_converged"
        check_fp32(case, out[i], u, np.abs(u + 1).max(), rho,
                   rho_limited_w=np.abs(u).max() if case in BATCH_RHO_LIMITED else None,
                   residuals=[float(inf.residual[i]) for inf in infos])


def test_batch_arguments_and_status():
    from paper_1611_04214_gb300.molt import Batch, MoltError, NotConverged
    with pytest.raises(MoltError):
        Batch([(2048, 64, 1.0, 1.0, 0.1)])
    with pytest.raises(MoltError):
        Batch([(64, 64, 1.0, 1.0, -0.1)])
    with Batch([(64, 48, 2.0, 2.0, 0.05), (40, 40, 2.0, 2.0, 0.1)], bc="neumann", tol=1e-12, max_iter=3) as b:
        u = torch.tensor(b.pack([_initial("neumann", 1, 64, 48), _initial("neumann", 2, 40, 40)]), device="cuda")
        with pytest.raises(MoltError):
            b.step(u, [1e-3, 1e-3], "sdirk3")
        with pytest.raises(MoltError):
            b.step(u, [1e-3, -1.0], "be")
        with pytest.raises(NotConverged):
            b.step(u, [1e-3, 1e-3], "be")
        info = b.step(u, [1e-3, 1e-3], "be", raise_on_nonconvergence=False)
        assert info.iters == [3, 3] and all(s != 0 for s in info.instance_status)


def test_batch_autotune_keeps_results_bitwise():
    # The schedule (one block per work item, or a persistent grid looping over the items) changes
    # which block runs an item, not what it computes: after autotuning, steps are bit-identical.
    from paper_1611_04214_gb300.molt import Batch
    inst = [(nx, ny, Lx, Ly, eps) for (nx, ny, Lx, Ly, eps, _) in INSTANCES]
    dts = [dt for (*_, dt) in INSTANCES]
    u0 = [_initial("neumann", 30 + i, nx, ny) for i, (nx, ny, *_rest) in enumerate(INSTANCES)]
    outs = []
    for tune in (None, "autotune", (16, 16), (304, 1216)):
        with Batch(inst, bc="neumann", quad_order=4, tol=1e-6, max_iter=300) as b:
            if tune == "autotune":
                sched = b.autotune(dts)
                assert all(len(r) == 4 for r in sched["ms_per_iteration"])
            elif tune is not None:
                b.set_schedule(*tune)
            u = torch.tensor(b.pack(u0), device="cuda")
            for _ in range(2):
                b.step(u, dts, "bdf2", raise_on_nonconvergence=False)
            outs.append(u.cpu().numpy())
    for o in outs[1:]:
        assert np.array_equal(outs[0], o)


@pytest.mark.parametrize("bc", ["periodic", "neumann", "dirichlet"])
@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("axis", [0, 1])
def test_batch_helmholtz_apply_matches_oracle(bc, M, axis):
    # One batched line inversion per instance (molt_batch_helmholtz_apply) against the oracle's
    # H_c of each instance, each with its own c (nu = h / sqrt(c) from 0.02 to 3); a second call
    # with other c reuses nothing.  Held to 1e-6 of the input's scale: the recurrences sum values of
    # the input's size, and on a Dirichlet line much shorter than the decay length 1/alpha (24
    # nodes at nu = 0.02: alpha L = 0.46) the output is the remainder of those sums after the
    # boundary correction, 60 times smaller than the input.
    from oracle.helmholtz import helmholtz_inverse
    from paper_1611_04214_gb300.inputs import spacing
    from paper_1611_04214_gb300.molt import Batch
    inst = [(nx, ny, Lx, Ly, eps) for (nx, ny, Lx, Ly, eps, _) in INSTANCES]
    with Batch(inst, bc=bc, quad_order=M, tol=1e-6, max_iter=10) as b:
        fields = [uniform_noise((ny, nx), 1.0, seed=30 + i, mean=1.0) for i, (nx, ny, *_r) in enumerate(inst)]
        fin = torch.tensor(b.pack(fields), device="cuda")
        fout = torch.empty_like(fin)
        for nus in ([0.02, 0.08, 0.27, 1.0, 3.0], [3.0, 1.0, 0.27, 0.08, 0.02]):
            cs = []
            for (nx, ny, Lx, Ly, _), nu in zip(inst, nus):
                n, L = (nx, Lx) if axis == 0 else (ny, Ly)
                cs.append((spacing(n, L, bc == "periodic") / nu) ** 2)
            b.helmholtz_apply(axis, cs, fin, fout)
            torch.cuda.synchronize()
            got = b.unpack(fout.cpu().numpy())
            for i, (nx, ny, Lx, Ly, _) in enumerate(inst):
                h = spacing(nx if axis == 0 else ny, Lx if axis == 0 else Ly, bc == "periodic")
                f = b.unpack(b.pack(fields))[i].astype(np.float64)
                ref = helmholtz_inverse(f, cs[i], h, bc, M, axis=1 if axis == 0 else 0)
                err = np.abs(got[i] - ref).max() / np.abs(f).max()
                assert err < 1e-6, (i, nus[i], err)


def test_batch_helmholtz_apply_then_step_reloads_stage_parameters():
    # A batched sweep overwrites a slot of the stage parameters; the next step must reload them and
    # give the same result as a batch that never swept.
    from paper_1611_04214_gb300.molt import Batch
    inst = [(nx, ny, Lx, Ly, eps) for (nx, ny, Lx, Ly, eps, _) in INSTANCES]
    dts = [dt for (*_, dt) in INSTANCES]
    outs = []
    for sweep_first in (False, True):
        with Batch(inst, bc="neumann", quad_order=4, tol=1e-6, max_iter=20) as b:
            u = torch.tensor(b.pack([_initial("neumann", i, nx, ny) for i, (nx, ny, *_r) in enumerate(inst)]),
                             device="cuda")
            b.step(u, dts, "be", raise_on_nonconvergence=False)
            if sweep_first:
                tmp = torch.empty_like(u)
                b.helmholtz_apply(0, [0.5] * len(inst), u, tmp)
                b.helmholtz_apply(1, [0.5] * len(inst), u, tmp)
            b.step(u, dts, "be", raise_on_nonconvergence=False)
            torch.cuda.synchronize()
            outs.append(u.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])
