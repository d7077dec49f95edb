"""ctypes wrapper of the C oracle -- TEST INFRASTRUCTURE ONLY.

Only tests/, ``__graft_entry__.smoke()`` and bench.py's CPU-baseline leg may
import this module.  Every function mirrors one function of rlt2_oracle.c; the
state arrays are exposed as numpy views indexed by the paper's subscripts:
``b[i, j]``, ``c[i, j, k, n]``, ``d[i, j, k, n, p, q]``.
"""
from __future__ import annotations

import ctypes as C
import numpy as np

from .build import build

_lib = None
_i64p = C.POINTER(C.c_int64)
_i32p = C.POINTER(C.c_int32)


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.orc_lap.restype = C.c_int64
        L.orc_lap.argtypes = [C.c_int, _i64p, _i64p, _i64p, _i32p, _i64p, C.c_void_p]
        L.orc_lap_batch.restype = None
        L.orc_lap_batch.argtypes = [C.c_int, C.c_int, _i64p, _i64p, _i64p, _i64p, _i32p, _i64p]
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.c_int, _i32p, _i32p, _i64p, C.c_int64, C.c_int]
        L.orc_set_paired.restype = None
        L.orc_set_paired.argtypes = [C.c_void_p, C.c_int]
        L.orc_child.restype = C.c_void_p
        L.orc_child.argtypes = [C.c_void_p, C.c_int, C.c_int]
        L.orc_destroy.argtypes = [C.c_void_p]
        for name in ("orc_spread_B_to_C", "orc_spread_C_to_D", "orc_complementary_D",
                     "orc_concentrate_D_to_C", "orc_complementary_C", "orc_concentrate_C_to_B"):
            getattr(L, name).argtypes = [C.c_void_p]
            getattr(L, name).restype = None
        for name in ("orc_spread_C_to_D_range", "orc_complementary_D_range",
                     "orc_concentrate_D_to_C_range"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, C.c_int]
            getattr(L, name).restype = None
        L.orc_concentrate_B_to_LB.restype = C.c_int64
        L.orc_concentrate_B_to_LB.argtypes = [C.c_void_p]
        L.orc_iterate.restype = C.c_int64
        L.orc_iterate.argtypes = [C.c_void_p]
        L.orc_run.argtypes = [C.c_void_p, C.c_int, _i64p]
        L.orc_N.restype = C.c_int
        L.orc_N.argtypes = [C.c_void_p]
        L.orc_LB.restype = C.c_int64
        L.orc_LB.argtypes = [C.c_void_p]
        for name in ("orc_b", "orc_c", "orc_d"):
            getattr(L, name).restype = _i64p
            getattr(L, name).argtypes = [C.c_void_p]
        L.orc_work.argtypes = [C.c_void_p, _i64p]
        L.orc_add_LB.argtypes = [C.c_void_p, C.c_int64]
        L.orc_subproblem.restype = C.c_int
        L.orc_subproblem.argtypes = [C.c_int, _i32p, _i32p, C.c_int, _i32p, _i32p,
                                     _i32p, _i32p, _i64p, _i64p]
        # FP64 form (reading R14)
        _f64p = C.POINTER(C.c_double)
        L.orf_lap.restype = C.c_double
        L.orf_lap.argtypes = [C.c_int, _f64p, _f64p, _f64p, _i32p, _i64p, C.c_void_p]
        L.orf_lap_batch.restype = None
        L.orf_lap_batch.argtypes = [C.c_int, C.c_int, _f64p, _f64p, _f64p, _f64p, _i32p, _i64p]
        L.orf_create.restype = C.c_void_p
        L.orf_create.argtypes = [C.c_int, _i32p, _i32p, _f64p, C.c_double, C.c_int]
        L.orf_destroy.argtypes = [C.c_void_p]
        for name in ("orf_spread_B_to_C", "orf_spread_C_to_D", "orf_complementary_D",
                     "orf_concentrate_D_to_C", "orf_complementary_C", "orf_concentrate_C_to_B"):
            getattr(L, name).argtypes = [C.c_void_p]
            getattr(L, name).restype = None
        for name in ("orf_spread_C_to_D_range", "orf_complementary_D_range",
                     "orf_concentrate_D_to_C_range"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_int, C.c_int]
            getattr(L, name).restype = None
        L.orf_concentrate_B_to_LB.restype = C.c_double
        L.orf_concentrate_B_to_LB.argtypes = [C.c_void_p]
        L.orf_iterate.restype = C.c_double
        L.orf_iterate.argtypes = [C.c_void_p]
        L.orf_run.argtypes = [C.c_void_p, C.c_int, _f64p]
        L.orf_LB.restype = C.c_double
        L.orf_LB.argtypes = [C.c_void_p]
        L.orf_add_LB.argtypes = [C.c_void_p, C.c_double]
        for name in ("orf_b", "orf_c", "orf_d"):
            getattr(L, name).restype = _f64p
            getattr(L, name).argtypes = [C.c_void_p]
        L.orf_work.argtypes = [C.c_void_p, _i64p]
        _lib = L
    return _lib


def _p64(a):
    return a.ctypes.data_as(_i64p)


def _p32(a):
    return a.ctypes.data_as(_i32p)


def _pf(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lap(M):
    """Hungarian method on one n x n matrix -> (S, col_of_row, u, v, (steps, relaxations))."""
    M = np.ascontiguousarray(M, dtype=np.int64)
    n = M.shape[0]
    u = np.zeros(n, np.int64)
    v = np.zeros(n, np.int64)
    sig = np.zeros(n, np.int32)
    work = np.zeros(3, np.int64)
    S = lib().orc_lap(n, _p64(M), _p64(u), _p64(v), _p32(sig), _p64(work), None)
    return int(S), sig, u, v, (int(work[0]), int(work[1]))


def lap_batch(M):
    """Batch of count x n x n matrices -> (S[count], col_of_row, u, v, work[count,3])."""
    M = np.ascontiguousarray(M, dtype=np.int64)
    count, n, _ = M.shape
    S = np.zeros(count, np.int64)
    u = np.zeros((count, n), np.int64)
    v = np.zeros((count, n), np.int64)
    sig = np.zeros((count, n), np.int32)
    work = np.zeros((count, 3), np.int64)
    lib().orc_lap_batch(n, count, _p64(M), _p64(S), _p64(u), _p64(v), _p32(sig), _p64(work))
    return S, sig, u, v, work


def subproblem(F, D, fac, loc):
    """Residual instance of a node fixing fac[t] -> loc[t] -> (F', D', Blin, const)."""
    F = np.ascontiguousarray(F, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    fac = np.ascontiguousarray(fac, np.int32)
    loc = np.ascontiguousarray(loc, np.int32)
    N = F.shape[0]
    Np = N - len(fac)
    Fp = np.zeros((Np, Np), np.int32)
    Dp = np.zeros((Np, Np), np.int32)
    Bl = np.zeros((Np, Np), np.int64)
    cst = np.zeros(1, np.int64)
    lib().orc_subproblem(N, _p32(F), _p32(D), len(fac), _p32(fac), _p32(loc),
                         _p32(Fp), _p32(Dp), _p64(Bl), _p64(cst))
    return Fp, Dp, Bl, int(cst[0])


class State:
    """RLT2 dual-ascent state of the oracle (Algorithm 1)."""

    def __init__(self, F, D, B_lin=None, lb_const=0, rlt1_only=False, paired=False):
        F = np.ascontiguousarray(F, np.int32)
        D = np.ascontiguousarray(D, np.int32)
        self.N = N = F.shape[0]
        bl = None
        if B_lin is not None:
            self._bl = np.ascontiguousarray(B_lin, np.int64)
            bl = _p64(self._bl)
        self._h = lib().orc_create(N, _p32(F), _p32(D), bl, int(lb_const), int(rlt1_only))
        if not self._h:
            raise MemoryError("oracle state allocation failed (N=%d)" % N)
        self.rlt1_only = rlt1_only
        self.paired = paired
        if paired:
            lib().orc_set_paired(self._h, 1)

    def child(self, f, l):
        """Warm-started state of the node fixing facility f to location l."""
        h = lib().orc_child(self._h, int(f), int(l))
        if not h:
            raise ValueError("no child state (N too small or bad indices)")
        st = State.__new__(State)
        st._h = h
        st.N = self.N - 1
        st.rlt1_only = self.rlt1_only
        st.paired = self.paired
        return st

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- the seven operations of Algorithm 1
    def spread_B_to_C(self): lib().orc_spread_B_to_C(self._h)
    def spread_C_to_D(self): lib().orc_spread_C_to_D(self._h)
    def complementary_D(self): lib().orc_complementary_D(self._h)
    def concentrate_D_to_C(self): lib().orc_concentrate_D_to_C(self._h)
    def complementary_C(self): lib().orc_complementary_C(self._h)
    def concentrate_C_to_B(self): lib().orc_concentrate_C_to_B(self._h)
    def concentrate_B_to_LB(self): return int(lib().orc_concentrate_B_to_LB(self._h))

    def spread_C_to_D_range(self, lo, hi): lib().orc_spread_C_to_D_range(self._h, lo, hi)
    def complementary_D_range(self, lo, hi): lib().orc_complementary_D_range(self._h, lo, hi)
    def concentrate_D_to_C_range(self, lo, hi): lib().orc_concentrate_D_to_C_range(self._h, lo, hi)

    def iterate(self):
        return int(lib().orc_iterate(self._h))

    def iterate_threaded(self, threads):
        """One pass of Algorithm 1, the three operations over D split by
        facility (the oracle's _range functions) over `threads` host threads.
        ctypes releases the GIL during each call, and the ranges of one
        operation write disjoint entries (their own first facility, or for the
        complementary transfer the classes of their smallest facility), so the
        result is that of iterate(); the work counters are updated without
        synchronisation and may undercount.  For timing on all host cores."""
        from concurrent.futures import ThreadPoolExecutor
        assert not self.paired, "the paired spread writes into other facilities' tiles"
        N = self.N
        lib().orc_spread_B_to_C(self._h)
        if not self.rlt1_only:
            with ThreadPoolExecutor(max_workers=threads) as ex:
                for fn in (self.spread_C_to_D_range, self.complementary_D_range,
                           self.concentrate_D_to_C_range):
                    # one task per facility, the costliest (smallest i) first
                    list(ex.map(lambda i: fn(i, i + 1), range(N)))
        lib().orc_complementary_C(self._h)
        lib().orc_concentrate_C_to_B(self._h)
        self.add_LB(self.concentrate_B_to_LB())
        return self.LB

    def run(self, k):
        hist = np.zeros(k, np.int64)
        lib().orc_run(self._h, k, _p64(hist))
        return hist

    @property
    def LB(self):
        return int(lib().orc_LB(self._h))

    def add_LB(self, x):
        lib().orc_add_LB(self._h, int(x))

    @property
    def b(self):
        N = self.N
        return np.ctypeslib.as_array(lib().orc_b(self._h), shape=(N, N))

    @property
    def c(self):
        N = self.N
        return np.ctypeslib.as_array(lib().orc_c(self._h), shape=(N, N, N, N))

    @property
    def d(self):
        N = self.N
        if self.rlt1_only:
            return None
        return np.ctypeslib.as_array(lib().orc_d(self._h), shape=(N,) * 6)

    def work(self):
        w = np.zeros(4, np.int64)
        lib().orc_work(self._h, _p64(w))
        return dict(laps=int(w[0]), steps=int(w[1]), relaxations=int(w[2]), max_abs=int(w[3]))


# ------------------------------------------------------------ FP64 form (R14)

def lap_f64(M):
    """FP64 Hungarian method on one n x n matrix -> (S, col_of_row, u, v, (steps, relaxations))."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    n = M.shape[0]
    u = np.zeros(n)
    v = np.zeros(n)
    sig = np.zeros(n, np.int32)
    work = np.zeros(3, np.int64)
    S = lib().orf_lap(n, _pf(M), _pf(u), _pf(v), _p32(sig), _p64(work), None)
    return float(S), sig, u, v, (int(work[0]), int(work[1]))


def lap_batch_f64(M):
    """Batch of count x n x n double matrices -> (S[count], col_of_row, u, v, work[count,3])."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    count, n, _ = M.shape
    S = np.zeros(count)
    u = np.zeros((count, n))
    v = np.zeros((count, n))
    sig = np.zeros((count, n), np.int32)
    work = np.zeros((count, 3), np.int64)
    lib().orf_lap_batch(n, count, _pf(M), _pf(S), _pf(u), _pf(v), _p32(sig), _p64(work))
    return S, sig, u, v, work


class StateF64:
    """RLT2 dual-ascent state of the oracle in the FP64 form (reading R14)."""

    def __init__(self, F, D, B_lin=None, lb_const=0.0, rlt1_only=False):
        F = np.ascontiguousarray(F, np.int32)
        D = np.ascontiguousarray(D, np.int32)
        self.N = N = F.shape[0]
        bl = None
        if B_lin is not None:
            self._bl = np.ascontiguousarray(B_lin, np.float64)
            bl = _pf(self._bl)
        self._h = lib().orf_create(N, _p32(F), _p32(D), bl, float(lb_const), int(rlt1_only))
        if not self._h:
            raise MemoryError("oracle state allocation failed (N=%d)" % N)
        self.rlt1_only = rlt1_only

    def close(self):
        if self._h:
            lib().orf_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def spread_B_to_C(self): lib().orf_spread_B_to_C(self._h)
    def spread_C_to_D(self): lib().orf_spread_C_to_D(self._h)
    def complementary_D(self): lib().orf_complementary_D(self._h)
    def concentrate_D_to_C(self): lib().orf_concentrate_D_to_C(self._h)
    def complementary_C(self): lib().orf_complementary_C(self._h)
    def concentrate_C_to_B(self): lib().orf_concentrate_C_to_B(self._h)
    def concentrate_B_to_LB(self): return float(lib().orf_concentrate_B_to_LB(self._h))

    def spread_C_to_D_range(self, lo, hi): lib().orf_spread_C_to_D_range(self._h, lo, hi)
    def complementary_D_range(self, lo, hi): lib().orf_complementary_D_range(self._h, lo, hi)
    def concentrate_D_to_C_range(self, lo, hi): lib().orf_concentrate_D_to_C_range(self._h, lo, hi)

    def iterate(self):
        return float(lib().orf_iterate(self._h))

    def run(self, k):
        hist = np.zeros(k)
        lib().orf_run(self._h, k, _pf(hist))
        return hist

    @property
    def LB(self):
        return float(lib().orf_LB(self._h))

    def add_LB(self, x):
        lib().orf_add_LB(self._h, float(x))

    @property
    def b(self):
        N = self.N
        return np.ctypeslib.as_array(lib().orf_b(self._h), shape=(N, N))

    @property
    def c(self):
        N = self.N
        return np.ctypeslib.as_array(lib().orf_c(self._h), shape=(N, N, N, N))

    @property
    def d(self):
        N = self.N
        if self.rlt1_only:
            return None
        return np.ctypeslib.as_array(lib().orf_d(self._h), shape=(N,) * 6)

    def work(self):
        w = np.zeros(3, np.int64)
        lib().orf_work(self._h, _p64(w))
        return dict(laps=int(w[0]), steps=int(w[1]), relaxations=int(w[2]))
