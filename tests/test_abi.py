"""The C ABI library builds, loads and exports every declared symbol; host-side
argument checks run before any CUDA call (no GPU needed)."""
import ctypes as C
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1510_02065_gb300 import build as B
from paper_1510_02065_gb300 import rlt2


@pytest.fixture(scope="module")
def L():
    B.build()
    return rlt2.lib()


def test_exports_every_header_symbol(L):
    names = rlt2.header_symbols()
    assert len(names) >= 14
    for name in names:
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", rlt2.LIB_PATH], capture_output=True,
                         text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    assert set(names) <= exported


def test_strerror_and_defaults(L):
    assert rlt2.rlt2_strerror(0) == "ok"
    assert "overflow" in rlt2.rlt2_strerror(rlt2.RLT2_E_OVERFLOW) or "int32" in rlt2.rlt2_strerror(-3)
    o = rlt2.rlt2_default_opts()
    assert o.use_graph == 1 and o.max_iters == 65536 and o.rlt1_only == 0
    assert rlt2.rlt2_row_stride(30) == 32 and rlt2.rlt2_row_stride(20) == 20
    assert rlt2.rlt2_row_stride(35) == 36 and rlt2.rlt2_row_stride(3) == 4


def _create_rc(L, F, D, N, Bl=None):
    F = np.ascontiguousarray(F, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    ctx = C.c_void_p()
    bl = None if Bl is None else np.ascontiguousarray(Bl, np.int32).ctypes.data_as(C.POINTER(C.c_int32))
    return L.rlt2_create(F.ctypes.data_as(C.POINTER(C.c_int32)), D.ctypes.data_as(C.POINTER(C.c_int32)),
                         N, bl, 0, None, C.byref(ctx))


def test_create_rejects_bad_input_before_cuda(L):
    Z = np.zeros((4, 4), np.int32)
    assert _create_rc(L, Z[:2, :2], Z[:2, :2], 2) == rlt2.RLT2_E_INVAL   # N < 3
    assert _create_rc(L, np.zeros((65, 65), np.int32), np.zeros((65, 65), np.int32), 65) == rlt2.RLT2_E_INVAL
    F = Z.copy()
    F[0, 1] = -1
    assert _create_rc(L, F, Z, 4) == rlt2.RLT2_E_INVAL                   # negative flow
    Bl = Z.copy()
    Bl[2, 2] = -5
    assert _create_rc(L, Z, Z, 4, Bl) == rlt2.RLT2_E_INVAL               # negative linear cost
    # U = sum F * max D beyond 2^29 - 1
    F = np.full((4, 4), 50000, np.int32)
    D = np.full((4, 4), 1000, np.int32)
    assert _create_rc(L, F, D, 4) == rlt2.RLT2_E_OVERFLOW
    assert L.rlt2_create(None, None, 5, None, 0, None, C.byref(C.c_void_p())) == rlt2.RLT2_E_INVAL


def test_guard_boundary(L):
    # U = 12 * f * d for a 4 x 4 all-off-diagonal instance: exactly at and just past the limit
    lim = rlt2.RLT2_LAP_MAX_ENTRY
    F = np.ones((4, 4), np.int32)
    np.fill_diagonal(F, 0)
    D = np.zeros((4, 4), np.int32)
    D[0, 1] = lim // 12 + 1        # 12 * that > lim
    assert _create_rc(L, F, D, 4) == rlt2.RLT2_E_OVERFLOW


def test_lap_batch_rejects_bad_arguments(L):
    assert rlt2.rlt2_lap_batch(0, 0, 1, 0) == rlt2.RLT2_E_INVAL     # n = 0
    assert rlt2.rlt2_lap_batch(0, 65, 1, 0) == rlt2.RLT2_E_INVAL    # n > 64
    assert rlt2.rlt2_lap_batch(0, 5, -1, 0) == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_lap_batch(0, 5, 3, 0) == rlt2.RLT2_E_INVAL     # null buffers
    assert rlt2.rlt2_lap_batch(0, 5, 0, 0) == rlt2.RLT2_OK          # empty batch


def test_binding_fails_loudly_without_library(tmp_path):
    code = ("import paper_1510_02065_gb300.rlt2 as r; r.LIB_PATH = %r; "
            "import sys\ntry:\n    r.lib()\nexcept ImportError as e:\n    print('raised', e); sys.exit(0)\n"
            "sys.exit(1)" % str(tmp_path / "missing.so"))
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", code], cwd=root, capture_output=True, text=True)
    assert r.returncode == 0 and "raised" in r.stdout, r.stdout + r.stderr


def _f64_create_rc(L, F, D, N, Bl=None, const=0.0):
    F = np.ascontiguousarray(F, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    ctx = C.c_void_p()
    bl = None if Bl is None else np.ascontiguousarray(Bl, np.float64).ctypes.data_as(C.POINTER(C.c_double))
    return L.rlt2_f64_create(F.ctypes.data_as(C.POINTER(C.c_int32)), D.ctypes.data_as(C.POINTER(C.c_int32)),
                             N, bl, const, None, C.byref(ctx))


def test_f64_create_rejects_bad_input_before_cuda(L):
    Z = np.zeros((4, 4), np.int32)
    assert _f64_create_rc(L, Z[:2, :2], Z[:2, :2], 2) == rlt2.RLT2_E_INVAL
    assert _f64_create_rc(L, np.zeros((65, 65), np.int32), np.zeros((65, 65), np.int32), 65) == rlt2.RLT2_E_INVAL
    F = Z.copy()
    F[1, 0] = -2
    assert _f64_create_rc(L, F, Z, 4) == rlt2.RLT2_E_INVAL
    Bl = np.zeros((4, 4))
    Bl[3, 1] = -0.5
    assert _f64_create_rc(L, Z, Z, 4, Bl) == rlt2.RLT2_E_INVAL
    Bl[3, 1] = np.nan
    assert _f64_create_rc(L, Z, Z, 4, Bl) == rlt2.RLT2_E_INVAL
    Bl[3, 1] = np.inf
    assert _f64_create_rc(L, Z, Z, 4, Bl) == rlt2.RLT2_E_INVAL
    assert _f64_create_rc(L, Z, Z, 4, None, float("nan")) == rlt2.RLT2_E_INVAL
    assert L.rlt2_f64_create(None, None, 5, None, 0.0, None, C.byref(C.c_void_p())) == rlt2.RLT2_E_INVAL


def test_f64_lap_batch_rejects_bad_arguments(L):
    assert rlt2.rlt2_f64_lap_batch(0, 0, 1, 0) == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_f64_lap_batch(0, 65, 1, 0) == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_f64_lap_batch(0, 5, -1, 0) == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_f64_lap_batch(0, 5, 3, 0) == rlt2.RLT2_E_INVAL
    assert rlt2.rlt2_f64_lap_batch(0, 5, 0, 0) == rlt2.RLT2_OK
