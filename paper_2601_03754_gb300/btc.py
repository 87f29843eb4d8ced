"""Thin ctypes binding of libbtc.so (include/btc.h), with the same entry-point names.

Argument marshalling only: every numerical step runs inside the library's CUDA
kernels. Device arrays are passed as torch CUDA tensors (their data_ptr()) or
as raw integer addresses; streams as torch.cuda.Stream or raw cudaStream_t
integers. If the library has not been built, loading raises an error: there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

F64, F32, MIXED_F32, MIXED_TF32, MIXED_BF16 = 0, 1, 2, 3, 4
DTYPES = {"f64": F64, "f32": F32, "mixed_f32": MIXED_F32}

OK, ERR_ARG, ERR_OOM, ERR_CUDA, ERR_NOT_SPD, ERR_TIMEOUT, ERR_NOT_FACTORED, ERR_UNSUPPORTED, ERR_NOT_CONVERGED = (
    0, -1, -2, -3, -4, -5, -6, -7, -8)

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libbtc.so")
_lib = None
_lock = threading.Lock()


class BtcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"btc error {code}: {msg}")
        self.code = code


class btc_plan_info(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n", ctypes.c_int), ("np", ctypes.c_int), ("levels", ctypes.c_int),
                ("dtype", ctypes.c_int), ("offdiag_blocks", ctypes.c_int64), ("fill_blocks", ctypes.c_int64),
                ("factor_flops", ctypes.c_double), ("seq_factor_flops", ctypes.c_double),
                ("critical_path_flops", ctypes.c_double), ("critical_path_formula", ctypes.c_double),
                ("solve_flops_per_rhs", ctypes.c_double), ("factor_bytes", ctypes.c_double),
                ("solve_bytes", ctypes.c_double), ("device_bytes", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_vp, _ip, _dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double)
_lp = ctypes.POINTER(ctypes.c_int64)

_SIGS = {
    "btc_describe": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(btc_plan_info)],
    "btc_schedule": [ctypes.c_int, _ip, _ip],
    "btc_schedule_items": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _lp, _ip, _lp, _ip, _ip, _ip],
    "btc_describe_order": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                           ctypes.POINTER(btc_plan_info), _ip, _ip],
    "btc_plan": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
    "btc_plan_query": [_vp, ctypes.POINTER(btc_plan_info)],
    "btc_plan_set_schedule": [_vp, ctypes.c_int],
    "btc_factor": [_vp, _vp, _vp],
    "btc_solve": [_vp, _vp, ctypes.c_int],
    "btc_solve_refined": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "btc_factor_solve": [_vp, _vp, _vp, _vp, ctypes.c_int],
    "btc_plan_set_timing": [_vp, ctypes.c_int],
    "btc_plan_set_autotune": [_vp, ctypes.c_int],
    "btc_plan_set_graphs": [_vp, ctypes.c_int],
    "btc_plan_tuning": [_vp, _ip, _ip, _ip],
    "btc_plan_tuning_interlaced": [_vp, _ip, _ip, _ip],
    "btc_plan_set_flow_config": [_vp, ctypes.c_int, ctypes.c_int],
    "btc_plan_flow_configs": [_vp, _ip, _ip, _ip],
    "btc_plan_timing": [_vp, _dp, _ip],
    "btc_schedule_interlaced": [ctypes.c_int, ctypes.c_int, _ip, _ip, _ip, _ip, _ip, _ip],
    "btc_factor_solve_refined": [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "btc_factor_solve_host": [_vp, _vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "btc_info": [_vp, _ip, _ip],
    "btc_get_factor": [_vp, _vp, _vp, _ip],
    "btc_residual": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _dp, _vp],
    "btc_residual_noalloc": [ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _dp, _vp],
    "btc_free": [_vp],
    "btc_plan_set_stream": [_vp, _vp],
    "btc_plan_set_variant": [_vp, ctypes.c_int],
    "btc_plan_set_trace": [_vp, _vp, _vp],
    "btc_solve_gmres_ir": [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_double, _ip, _ip,
                           _dp],
    "btc_plan_set_root_precision": [_vp, ctypes.c_int],
    "btc_plan_set_order": [_vp, ctypes.c_int, ctypes.c_int],
    "btc_plan_inject_stall": [_vp, ctypes.c_int, ctypes.c_int64],
    "btc_plan_set_phase_trace": [_vp, _vp],
    "btc_server_start": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int64, ctypes.c_int],
    "btc_server_submit": [_vp, _vp, ctypes.POINTER(ctypes.c_int64)],
    "btc_server_poll": [_vp, ctypes.c_int64, ctypes.c_int, _ip, _ip, _dp, _dp],
    "btc_server_stats": [_vp, _vp],
    "btc_server_stop": [_vp],
    "btc_server_prewarm": [_vp, ctypes.c_int, ctypes.c_int, ctypes.c_int],
    "btc_server_reset_stats": [_vp],
    "btc_server_footprint": [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_int64)],
    "btc_batch_plan": [ctypes.POINTER(_vp), ctypes.c_int, _ip, _ip, ctypes.c_int, _vp],
    "btc_batch_plan_orders": [ctypes.POINTER(_vp), ctypes.c_int, _ip, _ip, _ip, ctypes.c_int, _vp],
    "btc_batch_orders": [_vp, _ip],
    "btc_dispatch_orders": [ctypes.c_int, _ip, _ip, ctypes.c_int, _ip],
    "btc_batch_query": [_vp, _ip, _dp, ctypes.POINTER(ctypes.c_int64)],
    "btc_batch_factor": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "btc_batch_solve": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp)],
    "btc_batch_solve_refined": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.c_double, ctypes.c_int, _ip,
                                _dp],
    "btc_batch_info": [_vp, _ip, _ip, _ip],
    "btc_batch_free": [_vp],
    "btc_batch_factor_solve_refined": [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                       ctypes.POINTER(_vp), ctypes.c_double, ctypes.c_int, _ip, _dp],
    "btc_batch_set_autotune": [_vp, ctypes.c_int],
    "btc_batch_set_graphs": [_vp, ctypes.c_int],
    "btc_batch_tuning": [_vp, ctypes.c_int, _ip, _ip, _ip, _ip, _dp],
    "btc_arrow_plan": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
    "btc_arrow_factor": [_vp, _vp, _vp, _vp, _vp, ctypes.c_double, ctypes.c_int],
    "btc_arrow_solve": [_vp, _vp, _vp, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "btc_arrow_free": [_vp],
    "btc_banded_plan": [ctypes.POINTER(_vp), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, _vp],
    "btc_banded_inner": [_vp],
    "btc_banded_grouped": [_vp, _vp, _vp, _ip, _ip],
    "btc_banded_factor": [_vp, _vp],
    "btc_banded_solve_refined": [_vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "btc_banded_factor_solve_refined": [_vp, _vp, _vp, _vp, ctypes.c_int, ctypes.c_double, ctypes.c_int, _ip, _dp],
    "btc_banded_free": [_vp],
    "btc_last_error": [],
    "btc_version": [],
}


def header_symbols():
    """Names of the entry points declared in include/btc.h."""
    import re
    path = os.path.join(os.path.dirname(_HERE), "include", "btc.h")
    with open(path) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(btc_\w+)\s*\(", text, re.M)))


def load():
    """Load libbtc.so (built by build.build()); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} not found: run paper_2601_03754_gb300.build.build() first "
                                   "(there is no CPU fallback)")
            lib = ctypes.CDLL(LIB_PATH)
            for name, args in _SIGS.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_int
            lib.btc_last_error.restype = ctypes.c_char_p
            lib.btc_banded_inner.restype = ctypes.c_void_p
            _lib = lib
    return _lib


def _check(rc, allow=()):
    if rc != OK and rc not in allow:
        raise BtcError(rc, load().btc_last_error().decode())
    return rc


def _ptr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return s
    return s.cuda_stream


def btc_version():
    return load().btc_version()


def btc_describe(N, n, dtype=F64):
    info = btc_plan_info()
    _check(load().btc_describe(N, n, dtype, ctypes.byref(info)))
    return info.as_dict()


def btc_schedule(N):
    order = np.zeros(N, dtype=np.int32)
    levels = np.zeros(N, dtype=np.int32)
    _check(load().btc_schedule(N, order.ctypes.data_as(_ip), levels.ctypes.data_as(_ip)))
    return order, levels


def btc_describe_order(N, n, dtype=F64, order=0, chunks=1):
    """Host-only planner for either elimination order: (info dict, order, launch levels)."""
    info = btc_plan_info()
    o = np.zeros(N, dtype=np.int32)
    lv = np.zeros(N, dtype=np.int32)
    _check(load().btc_describe_order(N, n, dtype, order, chunks, ctypes.byref(info), o.ctypes.data_as(_ip),
                                     lv.ctypes.data_as(_ip)))
    return info.as_dict(), o, lv


def btc_schedule_items(N, order=0, chunks=1):
    """Host-only: (factor rows [F,14], solve rows [S,10], slot rows [K,3]) of a plan's work items, offsets
    in blocks."""
    L = load()
    nf, ns, nk = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(L.btc_schedule_items(N, order, chunks, None, ctypes.byref(nf), None, ctypes.byref(ns), None,
                                ctypes.byref(nk)))
    fr = np.zeros((max(nf.value, 1), 14), dtype=np.int64)
    sr = np.zeros((max(ns.value, 1), 10), dtype=np.int64)
    kr = np.zeros((max(nk.value, 1), 3), dtype=np.int32)
    _check(L.btc_schedule_items(N, order, chunks, fr.ctypes.data_as(_lp), ctypes.byref(nf),
                                sr.ctypes.data_as(_lp), ctypes.byref(ns), kr.ctypes.data_as(_ip),
                                ctypes.byref(nk)))
    return fr[:nf.value], sr[:ns.value], kr[:nk.value]


class Plan:
    """Owning handle of a btc_plan_t (released by free() or garbage collection)."""

    def __init__(self, N, n, dtype=F64, stream=None):
        h = _vp()
        _check(load().btc_plan(ctypes.byref(h), N, n, dtype, _stream(stream)))
        self.h = h
        self.N, self.n, self.dtype = N, n, dtype

    def free(self):
        if getattr(self, "h", None):
            load().btc_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def btc_plan(N, n, dtype=F64, stream=None):
    return Plan(N, n, dtype, stream)


SCHED_LEVELS, SCHED_FLOW = 0, 1


def btc_plan_set_schedule(plan, mode):
    return _check(load().btc_plan_set_schedule(plan.h, mode))


def btc_plan_query(plan):
    info = btc_plan_info()
    _check(load().btc_plan_query(plan.h, ctypes.byref(info)))
    return info.as_dict()


def btc_factor(plan, D, B):
    return _check(load().btc_factor(plan.h, _ptr(D), _ptr(B)))


def btc_solve(plan, rhs, nrhs):
    return _check(load().btc_solve(plan.h, _ptr(rhs), nrhs))


def btc_solve_refined(plan, b, x, nrhs, tol=1e-10, maxit=20, allow_not_converged=False):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    rc = _check(load().btc_solve_refined(plan.h, _ptr(b), _ptr(x), nrhs, tol, maxit, ctypes.byref(it),
                                         ctypes.byref(rel)), allow)
    return it.value, rel.value, rc


TIME_FACTOR, TIME_FACTOR_FORWARD, TIME_ROOT, TIME_SOLVE, TIME_SOLVE_TAIL, TIME_RESIDUAL = range(6)
TIMING_CLASSES = 6


def btc_plan_set_graphs(plan, enable=True):
    return _check(load().btc_plan_set_graphs(plan.h, int(bool(enable))))


def btc_plan_set_autotune(plan, enable=True):
    """enable: False/0 off, True/1 on, 2 = only a configuration remembered for the shape (no trials)."""
    return _check(load().btc_plan_set_autotune(plan.h, int(enable)))


def btc_plan_tuning(plan):
    """(register-budget cap, CTAs per SM, tuned) of the plan's persistent factorization."""
    a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().btc_plan_tuning(plan.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, bool(c.value)


def btc_plan_tuning_interlaced(plan):
    """(register-budget cap, CTAs per SM, tuned) of the plan's interlaced factor + forward launch."""
    a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
    _check(load().btc_plan_tuning_interlaced(plan.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, bool(c.value)


def btc_plan_set_flow_config(plan, resident_cap, ctas_per_sm=0):
    return _check(load().btc_plan_set_flow_config(plan.h, resident_cap, ctas_per_sm))


def btc_plan_flow_configs(plan):
    """[(register-budget cap, max CTAs per SM)] of the compiled persistent factor kernels."""
    caps = (ctypes.c_int * 8)()
    mx = (ctypes.c_int * 8)()
    n = ctypes.c_int(8)
    _check(load().btc_plan_flow_configs(plan.h, caps, mx, ctypes.byref(n)))
    return [(caps[i], mx[i]) for i in range(min(n.value, 8))]


def btc_plan_set_timing(plan, enable=True):
    return _check(load().btc_plan_set_timing(plan.h, int(bool(enable))))


def btc_plan_timing(plan):
    """Per kernel class: (summed device ms, launches) since the last call (synchronizes)."""
    ms = (ctypes.c_double * TIMING_CLASSES)()
    n = (ctypes.c_int * TIMING_CLASSES)()
    _check(load().btc_plan_timing(plan.h, ms, n))
    return [float(v) for v in ms], [int(v) for v in n]


def btc_schedule_interlaced(N, root_separate):
    """Entries of the interlaced factor + forward launch: (kind, node, level, deps[count, 6]), tail length."""
    import numpy as np
    lib = load()
    count = ctypes.c_int(0)
    _check(lib.btc_schedule_interlaced(N, int(root_separate), None, None, None, None, ctypes.byref(count), None))
    c = count.value
    kind, node, level = (np.zeros(max(c, 1), dtype=np.int32) for _ in range(3))
    deps = np.zeros(max(c, 1) * 6, dtype=np.int32)
    tail = ctypes.c_int(0)
    ip = lambda a: a.ctypes.data_as(_ip)
    _check(lib.btc_schedule_interlaced(N, int(root_separate), ip(kind), ip(node), ip(level), ip(deps),
                                       ctypes.byref(count), ctypes.byref(tail)))
    return kind[:c], node[:c], level[:c], deps[:6 * c].reshape(c, 6), tail.value


def btc_factor_solve(plan, D, B, rhs, nrhs):
    """Factor with the forward sweep interlaced, then the backward sweep; rhs is overwritten by x."""
    return _check(load().btc_factor_solve(plan.h, _ptr(D), _ptr(B), _ptr(rhs), nrhs))


def btc_factor_solve_refined(plan, D, B, b, x, nrhs, tol=1e-10, maxit=20, allow_not_converged=False):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    rc = _check(load().btc_factor_solve_refined(plan.h, _ptr(D), _ptr(B), _ptr(b), _ptr(x), nrhs, tol, maxit,
                                                ctypes.byref(it), ctypes.byref(rel)), allow)
    return it.value, rel.value, rc


def btc_factor_solve_host(plan, D, B, b, x, nrhs, tol=1e-10, maxit=20):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    rc = _check(load().btc_factor_solve_host(plan.h, _ptr(D), _ptr(B), _ptr(b), _ptr(x), nrhs, tol, maxit,
                                             ctypes.byref(it), ctypes.byref(rel)), (ERR_NOT_CONVERGED,))
    return it.value, rel.value, rc


def btc_solve_gmres_ir(plan, b, x, tol=1e-10, max_outer=20, restart=30, inner_tol=1e-6, allow_not_converged=False):
    """GMRES-IR on the plan's factor (one right-hand side): returns (outer steps, Arnoldi steps, relres, rc)."""
    o, i = ctypes.c_int(0), ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    rc = _check(load().btc_solve_gmres_ir(plan.h, _ptr(b), _ptr(x), tol, max_outer, restart, inner_tol,
                                          ctypes.byref(o), ctypes.byref(i), ctypes.byref(rel)), allow)
    return o.value, i.value, rel.value, rc


def btc_info(plan):
    blk = ctypes.c_int(0)
    col = ctypes.c_int(0)
    rc = load().btc_info(plan.h, ctypes.byref(blk), ctypes.byref(col))
    _check(rc, (ERR_NOT_SPD,))
    return rc, blk.value, col.value


def btc_get_factor(plan):
    """(Dhat [N,n,n], U [offdiag,n,n], pairs [offdiag,2]) as numpy arrays (host copies)."""
    q = btc_plan_query(plan)
    dt = np.float64 if plan.dtype == F64 else np.float32
    N, n, K = plan.N, plan.n, q["offdiag_blocks"]
    Dh = np.zeros((N, n, n), dtype=dt)
    U = np.zeros((max(K, 1), n, n), dtype=dt)
    pairs = np.zeros((max(K, 1), 2), dtype=np.int32)
    _check(load().btc_get_factor(plan.h, Dh.ctypes.data, U.ctypes.data, pairs.ctypes.data_as(_ip)))
    return Dh, U[:K], pairs[:K]


def btc_residual(N, n, nrhs, D, B, x, b, stream=None):
    out = (ctypes.c_double * 3)()
    _check(load().btc_residual(N, n, nrhs, _ptr(D), _ptr(B), _ptr(x), _ptr(b), out, _stream(stream)))
    return out[0], out[1], out[2]


def btc_residual_noalloc(N, n, nrhs, D, B, x, b, stream=None):
    """btc_residual with its scratch in a fixed device array (no device allocation)."""
    out = (ctypes.c_double * 3)()
    _check(load().btc_residual_noalloc(N, n, nrhs, _ptr(D), _ptr(B), _ptr(x), _ptr(b), out, _stream(stream)))
    return out[0], out[1], out[2]


def btc_free(plan):
    plan.free()
    return OK


def _ptr_array(xs):
    arr = (_vp * len(xs))()
    for i, x in enumerate(xs):
        arr[i] = _ptr(x)
    return arr


class Batch:
    """Owning handle of a btc_batch_t."""

    def __init__(self, Ns, ns, dtype=MIXED_F32, stream=None, chunks=None):
        Ns = np.ascontiguousarray(Ns, dtype=np.int32)
        ns = np.ascontiguousarray(ns, dtype=np.int32)
        h = _vp()
        if chunks is None:
            _check(load().btc_batch_plan(ctypes.byref(h), len(Ns), Ns.ctypes.data_as(_ip), ns.ctypes.data_as(_ip),
                                         dtype, _stream(stream)))
        else:
            ch = np.ascontiguousarray(chunks, dtype=np.int32)
            _check(load().btc_batch_plan_orders(ctypes.byref(h), len(Ns), Ns.ctypes.data_as(_ip),
                                                ns.ctypes.data_as(_ip), ch.ctypes.data_as(_ip), dtype,
                                                _stream(stream)))
        self.h = h
        self.count, self.dtype = len(Ns), dtype
        self.Ns, self.ns = Ns, ns

    def free(self):
        if getattr(self, "h", None):
            load().btc_batch_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def btc_batch_plan(Ns, ns, dtype=MIXED_F32, stream=None, chunks=None):
    """A batch plan; chunks (optional, per instance): 0 = nested dissection, c >= 1 = partition order."""
    return Batch(Ns, ns, dtype, stream, chunks)


def btc_batch_orders(batch):
    out = np.zeros(batch.count, dtype=np.int32)
    _check(load().btc_batch_orders(batch.h, out.ctypes.data_as(_ip)))
    return out


def btc_dispatch_orders(Ns, ns, dtype=MIXED_F32):
    """Host-only dispatch model: the per-instance chunk counts (0 = nested dissection) for a batch."""
    Ns = np.ascontiguousarray(Ns, dtype=np.int32)
    ns = np.ascontiguousarray(ns, dtype=np.int32)
    out = np.zeros(len(Ns), dtype=np.int32)
    _check(load().btc_dispatch_orders(len(Ns), Ns.ctypes.data_as(_ip), ns.ctypes.data_as(_ip), dtype,
                                      out.ctypes.data_as(_ip)))
    return out


def btc_batch_query(batch):
    g = ctypes.c_int(0)
    f = ctypes.c_double(0)
    d = ctypes.c_int64(0)
    _check(load().btc_batch_query(batch.h, ctypes.byref(g), ctypes.byref(f), ctypes.byref(d)))
    return {"groups": g.value, "factor_flops": f.value, "device_bytes": d.value}


def btc_batch_factor(batch, Ds, Bs):
    return _check(load().btc_batch_factor(batch.h, _ptr_array(Ds), _ptr_array(Bs)))


def btc_batch_solve(batch, bs, xs):
    return _check(load().btc_batch_solve(batch.h, _ptr_array(bs), _ptr_array(xs)))


def btc_batch_solve_refined(batch, bs, xs, tol=1e-10, maxit=30):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    rc = _check(load().btc_batch_solve_refined(batch.h, _ptr_array(bs), _ptr_array(xs), tol, maxit, ctypes.byref(it),
                                               ctypes.byref(rel)), (ERR_NOT_CONVERGED,))
    return it.value, rel.value, rc


def btc_batch_factor_solve_refined(batch, Ds, Bs, bs, xs, tol=1e-10, maxit=30):
    """Factor + FP64-refined solve of every instance (one captured graph once the tuning is settled)."""
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    rc = _check(load().btc_batch_factor_solve_refined(batch.h, _ptr_array(Ds), _ptr_array(Bs), _ptr_array(bs),
                                                      _ptr_array(xs), tol, maxit, ctypes.byref(it),
                                                      ctypes.byref(rel)), (ERR_NOT_CONVERGED,))
    return it.value, rel.value, rc


def btc_batch_set_autotune(batch, enable=True):
    return _check(load().btc_batch_set_autotune(batch.h, int(bool(enable))))


def btc_batch_set_graphs(batch, enable=True):
    return _check(load().btc_batch_set_graphs(batch.h, int(bool(enable))))


def btc_batch_tuning(batch, group):
    """(np, register-budget cap, CTAs per SM, tuned, tuned factor ms) of a group (launch order)."""
    v = [ctypes.c_int(0) for _ in range(4)]
    ms = ctypes.c_double(0.0)
    _check(load().btc_batch_tuning(batch.h, group, *[ctypes.byref(a) for a in v], ctypes.byref(ms)))
    return v[0].value, v[1].value, v[2].value, bool(v[3].value), ms.value


def btc_batch_info(batch):
    k = ctypes.c_int(0)
    blk = ctypes.c_int(0)
    col = ctypes.c_int(0)
    rc = load().btc_batch_info(batch.h, ctypes.byref(k), ctypes.byref(blk), ctypes.byref(col))
    _check(rc, (ERR_NOT_SPD,))
    return rc, k.value, blk.value, col.value


def btc_batch_free(batch):
    batch.free()
    return OK


def btc_plan_set_trace(plan, factor_trace, solve_trace):
    return _check(load().btc_plan_set_trace(plan.h, _ptr(factor_trace), _ptr(solve_trace)))


def btc_plan_set_phase_trace(plan, phase):
    """phase: device int64 tensor of 8 * N words (per-node phase stamps), or None to disable."""
    return _check(load().btc_plan_set_phase_trace(plan.h, _ptr(phase)))


VARIANT_HYBRID, VARIANT_RIGHT_LOOKING = 0, 1
ROOT_DOUBLE_FP32, ROOT_FP64 = 0, 1


def btc_plan_set_root_precision(plan, precision):
    """Top-separator Cholesky of the mixed paths in FP64 (ROOT_FP64, default) or double-FP32 (ROOT_DOUBLE_FP32)."""
    return _check(load().btc_plan_set_root_precision(plan.h, precision))


ORDER_ND, ORDER_PARTITION = 0, 1


def btc_plan_set_order(plan, order, chunks=1):
    """Elimination order: ORDER_ND (nested dissection, default) or ORDER_PARTITION with `chunks`
    chunks (Sec. 4.1, Alg. 4; chunks=1 is the natural order). Rebuilds the plan's schedules."""
    return _check(load().btc_plan_set_order(plan.h, order, chunks))


def btc_plan_inject_stall(plan, item, max_polls=4096):
    """Test hook: factor item `item` waits on a flag nothing sets, every wait gives up after max_polls
    polls (item=-1 restores the plan)."""
    return _check(load().btc_plan_inject_stall(plan.h, item, max_polls))


def btc_plan_set_variant(plan, variant):
    return _check(load().btc_plan_set_variant(plan.h, variant))


def btc_plan_set_stream(plan, stream):
    return _check(load().btc_plan_set_stream(plan.h, _stream(stream)))


class btc_request(ctypes.Structure):
    _fields_ = [("N", ctypes.c_int), ("n", ctypes.c_int), ("D", _vp), ("B", _vp), ("b", _vp), ("x", _vp),
                ("factor_id", ctypes.c_int64), ("tol", ctypes.c_double), ("maxit", ctypes.c_int)]


class btc_server_stats_t(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("evictions", ctypes.c_int64), ("cache_hits", ctypes.c_int64), ("cache_misses", ctypes.c_int64),
                ("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("mean_us", ctypes.c_double),
                ("solves_per_s", ctypes.c_double), ("device_bytes", ctypes.c_int64),
                ("p50_queue_us", ctypes.c_double), ("p99_queue_us", ctypes.c_double),
                ("p50_service_us", ctypes.c_double), ("p99_service_us", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class Server:
    """Owning handle of a btc_server_t (stopped by stop() or garbage collection)."""

    def __init__(self, dtype=MIXED_F32, slots=4, hbm_budget_bytes=8 << 30, cache_factors=True):
        h = _vp()
        _check(load().btc_server_start(ctypes.byref(h), dtype, slots, int(hbm_budget_bytes), int(cache_factors)))
        self.h = h

    def stop(self):
        if getattr(self, "h", None):
            load().btc_server_stop(self.h)
            self.h = None

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def btc_server_start(dtype=MIXED_F32, slots=4, hbm_budget_bytes=8 << 30, cache_factors=True):
    return Server(dtype, slots, hbm_budget_bytes, cache_factors)


def btc_server_submit(server, N, n, D, B, b, x, factor_id=-1, tol=1e-10, maxit=30):
    req = btc_request(N, n, _ptr(D), _ptr(B), _ptr(b), _ptr(x), factor_id, tol, maxit)
    t = ctypes.c_int64(0)
    _check(load().btc_server_submit(server.h, ctypes.byref(req), ctypes.byref(t)))
    return t.value


def btc_server_poll(server, ticket, wait=True):
    """None while queued/running (wait=False); else dict(status, iters, relres, latency_us)."""
    st = ctypes.c_int(0)
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0)
    lat = ctypes.c_double(0)
    rc = load().btc_server_poll(server.h, ticket, int(wait), ctypes.byref(st), ctypes.byref(it), ctypes.byref(rel),
                                ctypes.byref(lat))
    if rc == 1:
        return None
    _check(rc)
    return {"status": st.value, "iters": it.value, "relres": rel.value, "latency_us": lat.value}


def btc_server_stats(server):
    s = btc_server_stats_t()
    _check(load().btc_server_stats(server.h, ctypes.byref(s)))
    return s.as_dict()


def btc_server_prewarm(server, n, N_max, copies=1):
    """Build, tune and capture `copies` plans of every size bucket up to N_max for block size n."""
    return _check(load().btc_server_prewarm(server.h, n, N_max, copies))


def btc_server_footprint(dtype, N, n):
    """Device bytes a request of size (N, n) reserves in a server (its bucket plan and staging)."""
    b = ctypes.c_int64(0)
    _check(load().btc_server_footprint(dtype, N, n, ctypes.byref(b)))
    return b.value


def btc_server_reset_stats(server):
    return _check(load().btc_server_reset_stats(server.h))


def btc_server_stop(server):
    server.stop()
    return OK


class Arrow:
    """Owning handle of a btc_arrow_t (a bordered block-tridiagonal system)."""

    def __init__(self, N, n, m, dtype=MIXED_F32, stream=None):
        h = _vp()
        _check(load().btc_arrow_plan(ctypes.byref(h), N, n, m, dtype, _stream(stream)))
        self.h = h
        self.N, self.n, self.m, self.dtype = N, n, m, dtype

    def free(self):
        if getattr(self, "h", None):
            load().btc_arrow_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def btc_arrow_plan(N, n, m, dtype=MIXED_F32, stream=None):
    return Arrow(N, n, m, dtype, stream)


def btc_arrow_factor(arrow, D, B, C, A, tol=1e-12, maxit=30):
    return _check(load().btc_arrow_factor(arrow.h, _ptr(D), _ptr(B), _ptr(C), _ptr(A), tol, maxit))


def btc_arrow_solve(arrow, b, x, tol=1e-10, maxit=10, allow_not_converged=False):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    rc = _check(load().btc_arrow_solve(arrow.h, _ptr(b), _ptr(x), tol, maxit, ctypes.byref(it), ctypes.byref(rel)),
                allow)
    return it.value, rel.value, rc


def btc_arrow_free(arrow):
    arrow.free()
    return OK


class Banded:
    """Owning handle of a btc_banded_t (a block-banded system: Nb block rows of size b, lower block
    bandwidth w, solved as a block-tridiagonal system of w-row super-rows)."""

    def __init__(self, Nb, b, w, dtype=MIXED_F32, stream=None):
        h = _vp()
        _check(load().btc_banded_plan(ctypes.byref(h), Nb, b, w, dtype, _stream(stream)))
        self.h = h
        self.Nb, self.b, self.w, self.dtype = Nb, b, w, dtype
        self.N, self.n = -(-Nb // w), w * b
        inner = load().btc_banded_inner(h)
        self.inner = Plan.__new__(Plan)  # a view of the owned inner plan (never freed through it)
        self.inner.h, self.inner.N, self.inner.n, self.inner.dtype = _vp(inner), self.N, self.n, dtype
        self.inner.free = lambda: None

    def free(self):
        if getattr(self, "h", None):
            load().btc_banded_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def btc_banded_plan(Nb, b, w, dtype=MIXED_F32, stream=None):
    return Banded(Nb, b, w, dtype, stream)


def btc_banded_factor(band, A):
    return _check(load().btc_banded_factor(band.h, _ptr(A)), (ERR_NOT_SPD,))


def btc_banded_solve_refined(band, rhs, x, nrhs, tol=1e-10, maxit=20, allow_not_converged=False):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    rc = _check(load().btc_banded_solve_refined(band.h, _ptr(rhs), _ptr(x), nrhs, tol, maxit, ctypes.byref(it),
                                                ctypes.byref(rel)), allow)
    return it.value, rel.value, rc


def btc_banded_factor_solve_refined(band, A, rhs, x, nrhs, tol=1e-10, maxit=20, allow_not_converged=False):
    it = ctypes.c_int(0)
    rel = ctypes.c_double(0.0)
    allow = (ERR_NOT_CONVERGED,) if allow_not_converged else ()
    rc = _check(load().btc_banded_factor_solve_refined(band.h, _ptr(A), _ptr(rhs), _ptr(x), nrhs, tol, maxit,
                                                       ctypes.byref(it), ctypes.byref(rel)), allow)
    return it.value, rel.value, rc


def btc_banded_grouped(band):
    """Host copies (D' [N, n, n], B' [N-1, n, n]) of the grouped blocks of the last factor call."""
    D = np.zeros((band.N, band.n, band.n))
    B = np.zeros((max(band.N - 1, 0), band.n, band.n))
    _check(load().btc_banded_grouped(band.h, D.ctypes.data, B.ctypes.data if B.size else None, None, None))
    return D, B


def btc_banded_free(band):
    band.free()
    return OK
