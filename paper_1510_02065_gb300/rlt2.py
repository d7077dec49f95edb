"""Thin Python binding of the C ABI in include/rlt2.h (argument marshalling only).

Every function carries the name of the C entry point it calls.  Host arrays
are numpy; device buffers are passed as integer addresses (e.g. a torch CUDA
tensor's ``data_ptr()``) and streams as ``cudaStream_t`` integers (e.g.
``torch.cuda.current_stream().cuda_stream``).  All computation happens in
librlt2.so; there is no fallback: if the library is not built, importing the
binding's functions raises.
"""
from __future__ import annotations

import ctypes as C
import os
import re

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librlt2.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "rlt2.h")

RLT2_OK = 0
RLT2_E_INVAL = -1
RLT2_E_OOM = -2
RLT2_E_OVERFLOW = -3
RLT2_E_CUDA = -4
RLT2_E_TIMEOUT = -5
RLT2_E_STATE = -6
RLT2_E_INTERNAL = -7
RLT2_E_IO = -8
RLT2_STORE_TILES = 0
RLT2_STORE_CLASSES = 1
RLT2_STORE_PAIRS = 2
RLT2_MIN_N = 3
RLT2_MAX_N = 64
RLT2_LAP_MAX_ENTRY = 536870911


class Rlt2Error(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s failed: %s (%d)" % (where, rlt2_strerror(code), code))


class rlt2_node(C.Structure):
    _fields_ = [("k", C.c_int), ("fac", C.POINTER(C.c_int32)), ("loc", C.POINTER(C.c_int32))]


class rlt2_opts(C.Structure):
    _fields_ = [("rlt1_only", C.c_int), ("use_graph", C.c_int), ("profile", C.c_int),
                ("max_iters", C.c_int), ("ub", C.c_double), ("min_progress", C.c_double),
                ("stream", C.c_void_p), ("store", C.c_int), ("lanes", C.c_int),
                ("cta_warps", C.c_int)]


_lib = None
_i32p = C.POINTER(C.c_int32)
_i64p = C.POINTER(C.c_int64)
_dblp = C.POINTER(C.c_double)
_intp = C.POINTER(C.c_int)
_vp = C.c_void_p


def lib():
    """Load librlt2.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError("librlt2.so is not built (%s); run "
                          "`python -c 'import __graft_entry__ as g; g.build()'`" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    sig = {
        "rlt2_default_opts": (None, [C.POINTER(rlt2_opts)]),
        "rlt2_strerror": (C.c_char_p, [C.c_int]),
        "rlt2_create": (C.c_int, [_i32p, _i32p, C.c_int, _i32p, C.c_int64,
                                  C.POINTER(rlt2_opts), C.POINTER(_vp)]),
        "rlt2_destroy": (None, [_vp]),
        "rlt2_iterate": (C.c_int, [_vp, C.c_int]),
        "rlt2_bound": (C.c_int, [_vp, _dblp, _i64p, _intp]),
        "rlt2_bound_history": (C.c_int, [_vp, _i64p, C.c_int, _intp]),
        "rlt2_get_state": (C.c_int, [_vp, C.c_int, _i32p, C.c_size_t]),
        "rlt2_work": (C.c_int, [_vp, _i64p]),
        "rlt2_dlap_shape": (C.c_int, [_vp, _intp]),
        "rlt2_stage_times": (C.c_int, [_vp, _dblp, _intp]),
        "rlt2_reset_stage_times": (C.c_int, [_vp]),
        "rlt2_device_state": (_vp, [_vp, C.c_int]),
        "rlt2_row_stride": (C.c_int, [C.c_int]),
        "rlt2_lap_batch": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
        "rlt2_lap_batch_static": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
        "rlt2_lap_batch_auction": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp]),
        "rlt2_selftest_timeout": (C.c_int, [C.c_uint, _vp]),
        "rlt2_state_bytes": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int]),
        "rlt2_save": (C.c_int, [_vp, C.c_char_p]),
        "rlt2_child": (C.c_int, [_vp, C.c_int, C.c_int, C.POINTER(rlt2_opts), C.POINTER(_vp)]),
        "rlt2_load": (C.c_int, [C.c_char_p, C.POINTER(rlt2_opts), C.POINTER(_vp)]),
        "rlt2_group_create": (C.c_int, [C.POINTER(_vp), C.c_int, _vp, C.POINTER(_vp)]),
        "rlt2_group_iterate": (C.c_int, [_vp, C.c_int]),
        "rlt2_group_sync": (C.c_int, [_vp]),
        "rlt2_group_destroy": (None, [_vp]),
        "rlt2_subproblem": (C.c_int, [_i32p, _i32p, C.c_int, C.c_int, _i32p, _i32p, _i32p, _i32p,
                                      _i32p, _i64p]),
        "rlt2_batch_bound": (C.c_int, [_i32p, _i32p, C.c_int, C.POINTER(rlt2_node), C.c_int, C.c_int,
                                       C.POINTER(rlt2_opts), _i64p, _dblp, _intp]),
        "rlt2_f64_create": (C.c_int, [_i32p, _i32p, C.c_int, _dblp, C.c_double, C.POINTER(rlt2_opts),
                                      C.POINTER(_vp)]),
        "rlt2_f64_destroy": (None, [_vp]),
        "rlt2_f64_iterate": (C.c_int, [_vp, C.c_int]),
        "rlt2_f64_bound": (C.c_int, [_vp, _dblp, _intp]),
        "rlt2_f64_bound_history": (C.c_int, [_vp, _dblp, C.c_int, _intp]),
        "rlt2_f64_get_state": (C.c_int, [_vp, C.c_int, _dblp, C.c_size_t]),
        "rlt2_f64_device_state": (_vp, [_vp, C.c_int]),
        "rlt2_f64_work": (C.c_int, [_vp, _i64p]),
        "rlt2_f64_stage_times": (C.c_int, [_vp, _dblp, _intp]),
        "rlt2_f64_lap_batch": (C.c_int, [_vp, C.c_int, C.c_int, _vp, _vp, _vp, _vp, _vp, _vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def header_symbols():
    """Names of the functions include/rlt2.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rlt2_[a-z0-9_]+)\s*\(", text)))


def _chk(rc, where):
    if rc != RLT2_OK:
        raise Rlt2Error(rc, where)


def _p32(a):
    return a.ctypes.data_as(_i32p)


def _p64(a):
    return a.ctypes.data_as(_i64p)


# ---------------------------------------------------------------- C names

def rlt2_strerror(code: int) -> str:
    return lib().rlt2_strerror(int(code)).decode()


def rlt2_default_opts() -> rlt2_opts:
    o = rlt2_opts()
    lib().rlt2_default_opts(C.byref(o))
    return o


def rlt2_create(F, D, N=None, B_lin=None, lb_const=0, opts=None):
    """Returns a context handle (int).  F, D (and B_lin): host N x N int32."""
    F = np.ascontiguousarray(F, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    N = F.shape[0] if N is None else int(N)
    bl = None
    if B_lin is not None:
        B_lin = np.ascontiguousarray(B_lin, np.int32)
        bl = _p32(B_lin)
    ctx = _vp()
    rc = lib().rlt2_create(_p32(F), _p32(D), N, bl, int(lb_const),
                           C.byref(opts) if opts is not None else None, C.byref(ctx))
    _chk(rc, "rlt2_create")
    return ctx.value


def rlt2_destroy(ctx):
    lib().rlt2_destroy(_vp(ctx))


def rlt2_child(ctx, f, l, opts=None):
    out = _vp()
    _chk(lib().rlt2_child(_vp(ctx), int(f), int(l), C.byref(opts) if opts is not None else None, C.byref(out)),
         "rlt2_child")
    return out.value


def rlt2_save(ctx, path):
    _chk(lib().rlt2_save(_vp(ctx), os.fsencode(path)), "rlt2_save")


def rlt2_load(path, opts=None):
    out = _vp()
    _chk(lib().rlt2_load(os.fsencode(path), C.byref(opts) if opts is not None else None, C.byref(out)),
         "rlt2_load")
    return out.value


def rlt2_iterate(ctx, k: int):
    _chk(lib().rlt2_iterate(_vp(ctx), int(k)), "rlt2_iterate")


def rlt2_bound(ctx):
    """-> (LB as float, LB as exact int, passes completed)"""
    lb = C.c_double()
    ex = C.c_int64()
    it = C.c_int()
    _chk(lib().rlt2_bound(_vp(ctx), C.byref(lb), C.byref(ex), C.byref(it)), "rlt2_bound")
    return lb.value, ex.value, it.value


def rlt2_bound_history(ctx, cap: int):
    out = np.zeros(max(cap, 0), np.int64)
    cnt = C.c_int()
    _chk(lib().rlt2_bound_history(_vp(ctx), _p64(out), int(cap), C.byref(cnt)), "rlt2_bound_history")
    return out[:cnt.value]


def rlt2_get_state(ctx, level: int, N: int):
    counts = {0: N * N, 1: N * N * (N - 1) ** 2, 2: N * N * (N - 1) ** 2 * (N - 2) ** 2}
    out = np.empty(counts[level], np.int32)
    _chk(lib().rlt2_get_state(_vp(ctx), int(level), _p32(out), out.size), "rlt2_get_state")
    return out


def rlt2_dlap_shape(ctx):
    """(lanes per D->C LAP, warps per CTA, tuning passes still to come) of a context."""
    out = (C.c_int * 3)()
    _chk(lib().rlt2_dlap_shape(_vp(ctx), out), "rlt2_dlap_shape")
    return out[0], out[1], bool(out[2])


def rlt2_work(ctx):
    out = np.zeros(6, np.int64)
    _chk(lib().rlt2_work(_vp(ctx), _p64(out)), "rlt2_work")
    return dict(laps=int(out[0]), steps=int(out[1]), relaxations=int(out[2]),
                d_laps=int(out[3]), d_steps=int(out[4]), d_relaxations=int(out[5]))


def rlt2_stage_times(ctx):
    out = (C.c_double * 4)()
    n = C.c_int()
    _chk(lib().rlt2_stage_times(_vp(ctx), out, C.byref(n)), "rlt2_stage_times")
    return list(out), n.value


def rlt2_reset_stage_times(ctx):
    _chk(lib().rlt2_reset_stage_times(_vp(ctx)), "rlt2_reset_stage_times")


def rlt2_device_state(ctx, which: int) -> int:
    return lib().rlt2_device_state(_vp(ctx), int(which)) or 0


def rlt2_row_stride(N: int) -> int:
    return lib().rlt2_row_stride(int(N))


def rlt2_selftest_timeout(polls, stream=0) -> int:
    """Returns the C code (RLT2_E_TIMEOUT expected)."""
    return lib().rlt2_selftest_timeout(int(polls), _vp(stream or None))


def rlt2_lap_batch_auction(M_ptr, n, count, S_ptr, assign_ptr=0, work_ptr=0, stream=0):
    """Device addresses in, device addresses out (see rlt2.h).  Returns the C code."""
    return lib().rlt2_lap_batch_auction(_vp(M_ptr or None), int(n), int(count), _vp(S_ptr or None),
                                        _vp(assign_ptr or None), _vp(work_ptr or None), _vp(stream or None))


def rlt2_lap_batch(M_ptr, n, count, S_ptr, assign_ptr=0, u_ptr=0, v_ptr=0, work_ptr=0, stream=0):
    """Device addresses in, device addresses out (see rlt2.h).  Returns the C code."""
    return lib().rlt2_lap_batch(_vp(M_ptr or None), int(n), int(count), _vp(S_ptr or None),
                                _vp(assign_ptr or None), _vp(u_ptr or None), _vp(v_ptr or None),
                                _vp(work_ptr or None), _vp(stream or None))


def rlt2_lap_batch_static(M_ptr, n, count, S_ptr, assign_ptr=0, u_ptr=0, v_ptr=0, work_ptr=0,
                          stream=0):
    """rlt2_lap_batch without any device allocation by the library (for callers
    whose device memory all comes from their own allocator): its status block
    lives in a fixed per-GPU array; overlapping calls on one GPU race on it."""
    return lib().rlt2_lap_batch_static(_vp(M_ptr or None), int(n), int(count), _vp(S_ptr or None),
                                       _vp(assign_ptr or None), _vp(u_ptr or None),
                                       _vp(v_ptr or None), _vp(work_ptr or None),
                                       _vp(stream or None))


def rlt2_state_bytes(N, rlt1_only=False, max_iters=65536, store=RLT2_STORE_TILES) -> int:
    return int(lib().rlt2_state_bytes(int(N), int(rlt1_only), int(max_iters), int(store)))


def rlt2_group_create(ctxs, stream=0):
    arr = (_vp * len(ctxs))(*ctxs)
    out = _vp()
    _chk(lib().rlt2_group_create(arr, len(ctxs), _vp(stream or None), C.byref(out)), "rlt2_group_create")
    return out.value


def rlt2_group_iterate(group, k):
    _chk(lib().rlt2_group_iterate(_vp(group), int(k)), "rlt2_group_iterate")


def rlt2_group_sync(group):
    _chk(lib().rlt2_group_sync(_vp(group)), "rlt2_group_sync")


def rlt2_group_destroy(group):
    lib().rlt2_group_destroy(_vp(group))


def rlt2_subproblem(F, D, fac, loc):
    """Residual instance of a node fixing fac[t] -> loc[t] -> (Fp, Dp, Blin, lb_const)."""
    F = np.ascontiguousarray(F, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    fac = np.ascontiguousarray(fac, np.int32)
    loc = np.ascontiguousarray(loc, np.int32)
    N, k = F.shape[0], len(fac)
    Np = N - k
    Fp = np.zeros((Np, Np), np.int32)
    Dp = np.zeros((Np, Np), np.int32)
    Bl = np.zeros((Np, Np), np.int32)
    cst = C.c_int64()
    _chk(lib().rlt2_subproblem(_p32(F), _p32(D), N, k, _p32(fac), _p32(loc), _p32(Fp), _p32(Dp),
                               _p32(Bl), C.byref(cst)), "rlt2_subproblem")
    return Fp, Dp, Bl, cst.value


def rlt2_batch_bound(F, D, nodes, iters, stream=0, store=RLT2_STORE_TILES, lanes=0, return_lanes=False,
                     ub=0.0, cta_warps=0):
    """nodes: list of (fac, loc) arrays -> (LB per node as int64 array, device ms)
    [, D->C shapes used: ((lanes, CTA warps) for the nodes with N' > 16, the
    same for those with N' <= 16), (0, 0) where there are none]."""
    F = np.ascontiguousarray(F, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    keep = [(np.ascontiguousarray(f, np.int32), np.ascontiguousarray(l, np.int32)) for f, l in nodes]
    arr = (rlt2_node * len(keep))()
    for b, (f, l) in enumerate(keep):
        arr[b].k = len(f)
        arr[b].fac = _p32(f)
        arr[b].loc = _p32(l)
    o = rlt2_default_opts()
    o.stream = stream or None
    o.store = int(store)
    o.lanes = int(lanes)
    o.cta_warps = int(cta_warps)
    o.ub = float(ub)
    out = np.zeros(len(keep), np.int64)
    ms = C.c_double()
    used = (C.c_int * 4)()
    _chk(lib().rlt2_batch_bound(_p32(F), _p32(D), F.shape[0], arr, len(keep), int(iters), C.byref(o),
                                _p64(out), C.byref(ms), used), "rlt2_batch_bound")
    shapes = ((used[0], used[1]), (used[2], used[3]))
    return (out, ms.value, shapes) if return_lanes else (out, ms.value)


# ------------------------------------------------------------ convenience

class Context:
    """Owning wrapper of an rlt2_ctx (same calls, released on close/exit)."""

    def __init__(self, F, D, B_lin=None, lb_const=0, rlt1_only=False, use_graph=True,
                 profile=False, max_iters=65536, ub=0.0, min_progress=0.0, stream=0,
                 store=RLT2_STORE_TILES, lanes=0, cta_warps=0):
        o = self._opts(rlt1_only, use_graph, profile, max_iters, ub, min_progress, stream, store, lanes,
                       cta_warps)
        self.N = int(np.asarray(F).shape[0])
        self.ctx = rlt2_create(F, D, self.N, B_lin, lb_const, o)

    @staticmethod
    def _opts(rlt1_only=False, use_graph=True, profile=False, max_iters=65536, ub=0.0,
              min_progress=0.0, stream=0, store=RLT2_STORE_TILES, lanes=0, cta_warps=0):
        o = rlt2_default_opts()
        o.store = int(store)
        o.lanes = int(lanes)
        o.cta_warps = int(cta_warps)
        o.rlt1_only = int(rlt1_only)
        o.use_graph = int(use_graph)
        o.profile = int(profile)
        o.max_iters = int(max_iters)
        o.ub = float(ub)
        o.min_progress = float(min_progress)
        o.stream = stream or None
        return o

    @classmethod
    def load(cls, path, **kw):
        """A context resumed from a checkpoint written by save()."""
        self = cls.__new__(cls)
        self.ctx = rlt2_load(path, cls._opts(**kw))
        with open(path, "rb") as f:   # N: the int32 after the magic and the version
            self.N = int(np.frombuffer(f.read(16), np.int32)[3])
        return self

    def save(self, path):
        rlt2_save(self.ctx, path)

    def child(self, f, l, **kw):
        """Warm-started child fixing facility f to location l (indices of this context)."""
        ch = Context.__new__(Context)
        ch.ctx = rlt2_child(self.ctx, f, l, self._opts(**kw))
        ch.N = self.N - 1
        return ch

    def iterate(self, k=1):
        rlt2_iterate(self.ctx, k)

    def bound(self):
        return rlt2_bound(self.ctx)

    def history(self, cap=None):
        return rlt2_bound_history(self.ctx, cap if cap is not None else 65536)

    def state(self, level):
        return rlt2_get_state(self.ctx, level, self.N)

    def work(self):
        return rlt2_work(self.ctx)

    def dlap_shape(self):
        return rlt2_dlap_shape(self.ctx)

    def stage_times(self):
        return rlt2_stage_times(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            rlt2_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ FP64 form (rlt2_f64_*)

def _pd(a):
    return a.ctypes.data_as(_dblp)


def rlt2_f64_create(F, D, N=None, B_lin=None, lb_const=0.0, opts=None):
    F = np.ascontiguousarray(F, np.int32)
    D = np.ascontiguousarray(D, np.int32)
    N = int(F.shape[0]) if N is None else int(N)
    bl = None
    if B_lin is not None:
        B_lin = np.ascontiguousarray(B_lin, np.float64)
        bl = _pd(B_lin)
    out = _vp()
    _chk(lib().rlt2_f64_create(_p32(F), _p32(D), N, bl, float(lb_const),
                               C.byref(opts) if opts is not None else None, C.byref(out)),
         "rlt2_f64_create")
    return out


def rlt2_f64_destroy(ctx):
    lib().rlt2_f64_destroy(ctx)


def rlt2_f64_iterate(ctx, k: int):
    _chk(lib().rlt2_f64_iterate(ctx, int(k)), "rlt2_f64_iterate")


def rlt2_f64_bound(ctx):
    lb = C.c_double()
    it = C.c_int()
    _chk(lib().rlt2_f64_bound(ctx, C.byref(lb), C.byref(it)), "rlt2_f64_bound")
    return lb.value, it.value


def rlt2_f64_bound_history(ctx, cap: int):
    out = np.zeros(max(cap, 1))
    cnt = C.c_int()
    _chk(lib().rlt2_f64_bound_history(ctx, _pd(out), int(cap), C.byref(cnt)), "rlt2_f64_bound_history")
    return out[: cnt.value]


def rlt2_f64_get_state(ctx, level: int, N: int):
    m = N - 1
    count = {0: N * N, 1: N * N * m * m, 2: N * N * m * m * (N - 2) ** 2}[level]
    out = np.zeros(count)
    _chk(lib().rlt2_f64_get_state(ctx, int(level), _pd(out), count), "rlt2_f64_get_state")
    return out


def rlt2_f64_device_state(ctx, which: int) -> int:
    return lib().rlt2_f64_device_state(ctx, int(which)) or 0


def rlt2_f64_work(ctx):
    out = np.zeros(6, np.int64)
    _chk(lib().rlt2_f64_work(ctx, _p64(out)), "rlt2_f64_work")
    return out


def rlt2_f64_stage_times(ctx):
    out = np.zeros(4)
    n = C.c_int()
    _chk(lib().rlt2_f64_stage_times(ctx, _pd(out), C.byref(n)), "rlt2_f64_stage_times")
    return out, n.value


def rlt2_f64_lap_batch(M_ptr, n, count, S_ptr, assign_ptr=0, u_ptr=0, v_ptr=0, work_ptr=0, stream=0):
    """Device pointers (integers); returns the status code (0 = ok)."""
    return lib().rlt2_f64_lap_batch(M_ptr or None, int(n), int(count), S_ptr or None, assign_ptr or None,
                                    u_ptr or None, v_ptr or None, work_ptr or None, stream or None)


class ContextF64:
    """Owning wrapper of an rlt2_f64_ctx (the FP64 form)."""

    def __init__(self, F, D, B_lin=None, lb_const=0.0, rlt1_only=False, profile=False, max_iters=65536,
                 stream=0):
        o = Context._opts(rlt1_only=rlt1_only, profile=profile, max_iters=max_iters, stream=stream)
        self.N = int(np.asarray(F).shape[0])
        self.ctx = rlt2_f64_create(F, D, self.N, B_lin, lb_const, o)

    def iterate(self, k=1):
        rlt2_f64_iterate(self.ctx, k)

    def bound(self):
        return rlt2_f64_bound(self.ctx)

    def history(self, cap=None):
        return rlt2_f64_bound_history(self.ctx, cap if cap is not None else 65536)

    def state(self, level):
        return rlt2_f64_get_state(self.ctx, level, self.N)

    def work(self):
        return rlt2_f64_work(self.ctx)

    def stage_times(self):
        return rlt2_f64_stage_times(self.ctx)

    def close(self):
        if getattr(self, "ctx", None):
            rlt2_f64_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
