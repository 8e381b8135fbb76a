"""CPU-only checks of the C-ABI library: it builds, loads, exports every symbol the header
declares, and its host-side quadrature weights agree with the oracle's (no GPU calls)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1611_04214_gb300 import build as molt_build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    molt_build.build_library()
    from paper_1611_04214_gb300 import molt
    return molt.load_library()


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "molt.h")) as fh:
        text = fh.read()
    decl = re.compile(r"^\s*(?:molt_status|void|const char\s*\*|long long)\s+(molt_[a-z0-9_]+)\s*\(", re.M)
    return sorted(set(decl.findall(text)))


def test_header_symbols_exported(lib):
    from paper_1611_04214_gb300 import molt
    declared = _declared_symbols()
    assert declared, "no declarations parsed"
    assert sorted(molt.EXPORTS) == declared
    for name in declared:
        assert hasattr(lib, name), name


@pytest.mark.parametrize("M", [2, 4, 6])
@pytest.mark.parametrize("nu", [1e-3, 0.08, 0.27, 1.5, 2.5, 9.0])
def test_host_weights_match_oracle(lib, M, nu):
    # The library computes the weights from exponential moments (series / recursion); the oracle
    # integrates the definition by Gauss-Legendre quadrature.  Same Sec. 3.2 definition.
    from oracle.weights import local_weights
    from paper_1611_04214_gb300.molt import molt_quadrature_weights
    H = M // 2
    for offs in [list(range(-H, H + 1)), list(range(0, M + 1)), list(range(-M, 1)), list(range(-1, M))]:
        for side in ("L", "R"):
            got = np.array(molt_quadrature_weights(nu, M, offs, side))
            ref = local_weights(nu, tuple(offs), side)
            np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-15 * max(nu, 1.0))


def test_weights_reject_bad_arguments(lib):
    from paper_1611_04214_gb300.molt import MoltError, molt_quadrature_weights
    with pytest.raises(MoltError):
        molt_quadrature_weights(0.0, 4, [-2, -1, 0, 1, 2], "L")
    with pytest.raises(MoltError):
        molt_quadrature_weights(0.1, 3, [-1, 0, 1, 2], "L")


def test_grid_validation_host_only(lib):
    # molt_grid_create does no device work, so its argument checks run without a GPU.
    g = ctypes.c_void_p()
    assert lib.molt_grid_create(ctypes.byref(g), 2, 64, 48, 1.0, 1.0, 1) == 0
    lib.molt_grid_destroy(g)
    assert lib.molt_grid_create(ctypes.byref(g), 1, 64, 2, 1.0, 1.0, 0) == -1       # 1D needs ny = 1
    assert b"ny = 1" in lib.molt_last_error(None)
    assert lib.molt_grid_create(ctypes.byref(g), 2, 4, 48, 1.0, 1.0, 0) == -1       # too short
    assert lib.molt_grid_create(ctypes.byref(g), 2, 64, 48, -1.0, 1.0, 0) == -1     # bad length
    assert lib.molt_grid_create(ctypes.byref(g), 2, 64, 48, 1.0, 1.0, 7) == -1      # bad bc
    assert lib.molt_grid_create(ctypes.byref(g), 3, 64, 48, 1.0, 1.0, 0) == -1      # bad dim


def test_solver3d_validation_host_only(lib):
    # molt_solver3d_create checks its arguments before any device work.
    from paper_1611_04214_gb300 import molt
    h = ctypes.c_void_p()
    p32 = molt._Params(0.1, 4, molt.PRECISION["fp32"], 1e-8, 50)
    p64 = molt._Params(0.1, 4, molt.PRECISION["fp64"], 1e-8, 50)
    create = lib.molt_solver3d_create
    assert create(ctypes.byref(h), 32, 32, 32, 1.0, 1.0, 1.0, 2, ctypes.byref(p32)) == molt.MOLT_ERR_UNSUPPORTED
    assert b"periodic and Neumann" in lib.molt_last_error(None)
    assert create(ctypes.byref(h), 32, 32, 32, 1.0, 1.0, 1.0, 0, ctypes.byref(p64)) == molt.MOLT_ERR_UNSUPPORTED
    assert create(ctypes.byref(h), 2048, 32, 32, 1.0, 1.0, 1.0, 0, ctypes.byref(p32)) == -1    # nx > 1024
    assert create(ctypes.byref(h), 32, 32, 4, 1.0, 1.0, 1.0, 0, ctypes.byref(p32)) == -1       # nz < M + 2
    assert create(ctypes.byref(h), 32, 32, 32, 1.0, -1.0, 1.0, 0, ctypes.byref(p32)) == -1     # bad length
    assert create(ctypes.byref(h), 32, 32, 32, 1.0, 1.0, 1.0, 0, None) == -1                   # no params
    assert lib.molt_solver3d_step(None, None, 1e-3, 0, None, None) == -1
    assert lib.molt_solver3d_apply(None, 0, 1.0, None, None, None) == -1
    assert lib.molt_batch_helmholtz_apply(None, 0, None, None, None, None) == -1


def test_fch1d_validation_host_only(lib):
    # molt_fch1d_create checks its arguments before any device work.
    from paper_1611_04214_gb300 import molt
    h = ctypes.c_void_p()
    p = molt._Params(0.18, 6, molt.PRECISION["fp64"], 1e-10, 50)
    create = lib.molt_fch1d_create
    assert create(ctypes.byref(h), 128, 4, 6.28, 2, 1.0, ctypes.byref(p)) == molt.MOLT_ERR_UNSUPPORTED   # Dirichlet
    assert b"periodic and Neumann" in lib.molt_last_error(None)
    assert create(ctypes.byref(h), 7, 4, 6.28, 0, 1.0, ctypes.byref(p)) == -1               # nx < M + 2
    assert create(ctypes.byref(h), 1 << 20, 4, 6.28, 0, 1.0, ctypes.byref(p)) == -1         # beyond the row kernel
    assert create(ctypes.byref(h), 128, 0, 6.28, 0, 1.0, ctypes.byref(p)) == -1             # no lines
    assert create(ctypes.byref(h), 128, 4, 0.0, 0, 1.0, ctypes.byref(p)) == -1              # bad length
    assert create(ctypes.byref(h), 128, 4, 6.28, 0, float("nan"), ctypes.byref(p)) == -1    # eta
    assert create(ctypes.byref(h), 128, 4, 6.28, 0, 1.0, None) == -1
    assert lib.molt_fch1d_step(None, None, 0.05, None, None) == -1


def test_fch2d_validation_host_only(lib):
    # molt_fch2d_create checks its arguments before any device work.
    from paper_1611_04214_gb300 import molt
    h = ctypes.c_void_p()
    p = molt._Params(0.18, 6, molt.PRECISION["fp64"], 1e-10, 50)
    create = lib.molt_fch2d_create
    assert create(ctypes.byref(h), 128, 128, 6.28, 6.28, 2, 1.0, ctypes.byref(p)) == molt.MOLT_ERR_UNSUPPORTED
    assert b"periodic and Neumann" in lib.molt_last_error(None)
    assert create(ctypes.byref(h), 7, 128, 6.28, 6.28, 0, 1.0, ctypes.byref(p)) == -1          # nx < M + 2
    assert create(ctypes.byref(h), 128, 7, 6.28, 6.28, 0, 1.0, ctypes.byref(p)) == -1          # ny < M + 2
    assert create(ctypes.byref(h), 1 << 20, 128, 6.28, 6.28, 0, 1.0, ctypes.byref(p)) == -1    # beyond the rows
    assert create(ctypes.byref(h), 128, 128, 6.28, -1.0, 0, 1.0, ctypes.byref(p)) == -1        # bad length
    assert create(ctypes.byref(h), 128, 128, 6.28, 6.28, 0, float("inf"), ctypes.byref(p)) == -1
    assert create(ctypes.byref(h), 128, 128, 6.28, 6.28, 0, 1.0, None) == -1
    assert lib.molt_fch2d_step(None, None, 0.05, None, None) == -1


def test_missing_library_fails_loudly(tmp_path):
    from paper_1611_04214_gb300 import molt
    saved = molt._lib
    try:
        molt._lib = None
        with pytest.raises(ImportError):
            molt.load_library(str(tmp_path / "libmolt.so"))
    finally:
        molt._lib = saved


def _c_kind(decl: str):
    t = " ".join(decl.split())
    if t == "void":
        return None
    if "*" in t:
        return "p"
    if "double" in t:
        return "d"
    if "long long" in t:
        return "q"
    return "i"   # int, unsigned, enums


def _ctypes_kind(t):
    if t is None:
        return None
    if t in (ctypes.c_int, ctypes.c_uint):
        return "i"
    if t is ctypes.c_double:
        return "d"
    if t is ctypes.c_longlong:
        return "q"
    return "p"   # c_void_p, c_char_p, POINTER(...)


def test_binding_signatures_match_the_header():
    # Every entry point declared in include/molt.h has a ctypes signature in the binding with the same
    # number of arguments and the same kind (integer / double / 64-bit integer / pointer) per
    # argument and for the result.
    import re

    from paper_1611_04214_gb300 import molt
    text = open(os.path.join(ROOT, "include", "molt.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    decls = {}
    for m in re.finditer(r"([A-Za-z_][\w\s\*]*?)\b(molt_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        ret, name, params = m.group(1), m.group(2), m.group(3).strip()
        ret = ret.replace("extern", "").strip()
        kinds = []
        if params not in ("", "void"):
            for prm in params.split(","):
                prm = prm.strip()
                prm = re.sub(r"\b[A-Za-z_]\w*$", "", prm) if not prm.endswith("*") else prm
                kinds.append(_c_kind(prm))
        decls[name] = (kinds, _c_kind(ret))
    sig = molt.signatures()
    assert set(decls) == set(sig), (sorted(set(decls) ^ set(sig)))
    for name, (args, res) in sig.items():
        assert [_ctypes_kind(a) for a in args] == decls[name][0], name
        assert _ctypes_kind(res) == decls[name][1], name
