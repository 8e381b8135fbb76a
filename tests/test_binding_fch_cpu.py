"""The sixth-order solvers' Python binding (``Fch1D``, ``Fch2D``) marshals its arguments into the
C ABI as declared: checked on the CPU against a stand-in library that records each call (no device
work; the real entry points are exercised by tests/test_gpu_fch*.py)."""
import ctypes

import pytest

from paper_1611_04214_gb300 import molt


class _FakeLib:
    def __init__(self, step_status=0):
        self.calls = []
        self.step_status = step_status

    def __getattr__(self, name):
        if not name.startswith("molt_fch"):
            raise AttributeError(name)

        def fn(*args):
            self.calls.append((name, args))
            if name.endswith("_create"):
                ctypes.cast(args[0], ctypes.POINTER(ctypes.c_void_p))[0] = 0x1234
                return 0
            if name.endswith("_step"):
                info = ctypes.cast(args[4], ctypes.POINTER(molt._StepInfo))[0]
                info.status, info.stages, info.total_iters, info.residual, info.tol_used = self.step_status, 1, 7, 1e-9, 1e-8
                info.iters[0] = 7
                return self.step_status
            if name.endswith("_launches"):
                return 42
            return 0
        return fn

    def molt_last_error(self, handle):
        return b"stand-in error"


class _FakeTensor:
    def __init__(self, shape, itemsize, cuda=True):
        self.shape, self.is_cuda = shape, cuda
        self.dtype = type("dt", (), {"itemsize": itemsize})()

    def is_floating_point(self):
        return True

    def is_contiguous(self):
        return True

    def data_ptr(self):
        return 0x5000


@pytest.fixture
def fake(monkeypatch):
    lib = _FakeLib()
    monkeypatch.setattr(molt, "_lib", lib)
    return lib


def test_fch1d_marshals_create_step_and_close(fake):
    s = molt.Fch1D(128, lines=4, L=2.0, bc="neumann", eps=0.2, eta=3.0, quad_order=4, tol=1e-9, max_iter=77,
                   precision="fp32")
    name, args = fake.calls[0]
    assert name == "molt_fch1d_create"
    assert args[1:6] == (128, 4, 2.0, molt.BC["neumann"], 3.0)
    p = ctypes.cast(args[6], ctypes.POINTER(molt._Params))[0]
    assert (p.eps, p.quad_order, p.precision, p.tol, p.max_iter) == (0.2, 4, molt.PRECISION["fp32"], 1e-9, 77)
    info = s.step(_FakeTensor((4, 128), 4), 0.05, stream=7)
    name, args = fake.calls[1]
    assert name == "molt_fch1d_step" and args[0].value == 0x1234 and args[1].value == 0x5000
    assert args[2] == 0.05 and args[3].value == 7
    assert info.iters == [7] and info.total_iters == 7
    assert s.kernel_launches() == 42
    with pytest.raises(ValueError):
        s.step(_FakeTensor((4, 128), 8), 0.05, stream=7)       # FP64 tensor for an FP32 solver
    with pytest.raises(ValueError):
        s.step(_FakeTensor((128, 4), 4), 0.05, stream=7)       # transposed shape
    s.close()
    assert fake.calls[-1][0] == "molt_fch1d_destroy"
    s.close()                                                  # idempotent
    assert sum(c[0] == "molt_fch1d_destroy" for c in fake.calls) == 1


def test_fch2d_marshals_create_and_reports_nonconvergence(fake):
    with molt.Fch2D(64, 48, Lx=1.0, Ly=1.5, bc="periodic", eps=0.18, eta=1.0, precision="fp64") as s:
        name, args = fake.calls[0]
        assert name == "molt_fch2d_create"
        assert args[1:7] == (64, 48, 1.0, 1.5, molt.BC["periodic"], 1.0)
        fake.step_status = molt.MOLT_ERR_NOT_CONVERGED
        u = _FakeTensor((48, 64), 8)
        assert s.step(u, 0.1, stream=3, raise_on_nonconvergence=False).status == molt.MOLT_ERR_NOT_CONVERGED
        with pytest.raises(molt.NotConverged):
            s.step(u, 0.1, stream=3)
        assert fake.calls[-1][0] == "molt_fch2d_step"
    assert fake.calls[-1][0] == "molt_fch2d_destroy"
