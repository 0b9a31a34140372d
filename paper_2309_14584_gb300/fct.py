"""Thin Python binding of the C ABI in include/fct.h (argument marshalling only).

Every step of the transform runs inside libfct_gb300.so; this module converts
numpy arrays / torch tensors to pointers and status codes to exceptions.  There
is no fallback: if the library is missing, loading fails loudly.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FCT_OK = 0
FCT_ERR_INVALID_ARG = 1
FCT_ERR_RANK = 2
FCT_ERR_NOCONV = 3
FCT_ERR_TIMEOUT = 4
FCT_ERR_OOM = 5
FCT_ERR_NONFINITE = 6
FCT_ERR_CUDA = 7
FCT_ERR_NO_DEVICE = 8

FCT_FP64 = 0
FCT_MIXED = 1
FCT_GRID_EXTREMA = 0
FCT_GRID_FIRST_KIND = 1
FCT_PLAN_BUILD_AUTO = 0
FCT_PLAN_BUILD_HOST = 1
FCT_PLAN_BUILD_DEVICE = 2

FCT_FAMILY_POLY = 0
FCT_FAMILY_GAUSSCOS = 1
FCT_FAMILY_RATIONAL = 2
FCT_FAMILY_POLY_GAUSSCOS = 3
FCT_SAMPLE_FOLDED = 0x100


class fct_options(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int),
        ("tol", ctypes.c_double),
        ("max_iter", ctypes.c_int),
        ("inner_tol", ctypes.c_double),
        ("max_refine", ctypes.c_int),
        ("block_threads", ctypes.c_int),
        ("max_blocks", ctypes.c_int),
        ("coef_lanes", ctypes.c_int),
        ("timeout_s", ctypes.c_double),
        ("normal_matrix", ctypes.c_int),
        ("grid_kind", ctypes.c_int),
        ("entries_per_lane", ctypes.c_int),
        ("plan_build", ctypes.c_int),
        ("tensor_dct", ctypes.c_int),
        ("coef_split", ctypes.c_int),
        ("kappa_max", ctypes.c_double),
    ]


class fct_report(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int),
        ("iterations", ctypes.c_int),
        ("refinements", ctypes.c_int),
        ("reserved", ctypes.c_int),
        ("rel_normal_residual", ctypes.c_double),
        ("gamma0", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "reserved"}


class fct_plan_info(ctypes.Structure):
    _fields_ = [
        ("N", ctypes.c_int64),
        ("M", ctypes.c_int64),
        ("R", ctypes.c_int64),
        ("nnz", ctypes.c_int64),
        ("D", ctypes.c_int32),
        ("K", ctypes.c_int32),
        ("passes", ctypes.c_int32),
        ("grid_blocks", ctypes.c_int32),
        ("block_threads", ctypes.c_int32),
        ("coef_lanes", ctypes.c_int32),
        ("device_bytes", ctypes.c_int64),
        ("normal_nnz", ctypes.c_int64),
        ("tensor_dct_grids", ctypes.c_int64),
        ("coef_split", ctypes.c_int32),
        ("row_units", ctypes.c_int32),
        ("wide_rows", ctypes.c_int32),
        ("coef_chunks", ctypes.c_int32),
        ("entries_per_lane", ctypes.c_int32),
        ("kernel_variant", ctypes.c_int32),
        ("tensor_dct_flops", ctypes.c_int64),
        ("kappa_estimate", ctypes.c_double),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class FctError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


_P = ctypes.c_void_p
_lib = None

# (name, restype, argtypes) of every exported entry point of include/fct.h
SIGNATURES = [
    ("fct_default_options", None, [ctypes.POINTER(fct_options)]),
    ("fct_last_error", ctypes.c_char_p, []),
    ("fct_status_string", ctypes.c_char_p, [ctypes.c_int]),
    ("fct_plan_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int64, _P, ctypes.c_int, _P, _P,
                                       ctypes.POINTER(fct_options)]),
    ("fct_plan_get_info", ctypes.c_int, [_P, ctypes.POINTER(fct_plan_info)]),
    ("fct_grid_offsets", ctypes.c_int, [_P, _P]),
    ("fct_sample", ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int64, _P, _P]),
    ("fct_execute", ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(fct_report)]),
    ("fct_execute_host", ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(fct_report)]),
    ("fct_execute_batch", ctypes.c_int, [ctypes.c_int, _P, _P, _P, ctypes.c_int, _P, _P]),
    ("fct_batch_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, _P, _P, ctypes.c_int]),
    ("fct_batch_launch", ctypes.c_int, [_P, _P]),
    ("fct_batch_reports", ctypes.c_int, [_P, _P, _P]),
    ("fct_batch_destroy", ctypes.c_int, [_P]),
    ("fct_plan_last_report", ctypes.c_int, [_P, _P, ctypes.POINTER(fct_report)]),
    ("fct_execute_noalloc", ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(fct_report)]),
    ("fct_destroy", ctypes.c_int, [_P]),
    ("fct_plan_clone", ctypes.c_int, [ctypes.POINTER(_P), _P]),
    ("fct_evaluate", ctypes.c_int, [_P, _P, ctypes.c_int64, _P, _P, _P]),
    ("fct_plan_rhs", ctypes.c_int, [_P, _P, _P, _P, _P]),
    ("fct_plan_apply", ctypes.c_int, [_P, _P, _P, ctypes.c_int, _P, _P]),
    ("fct_plan_tables", ctypes.c_int, [_P, _P, _P, _P, _P, _P, _P]),
    ("fct_measure_team_barrier", ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.POINTER(ctypes.c_double)]),
    ("fct_plan_condition", ctypes.c_int, [_P, _P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                          ctypes.POINTER(ctypes.c_int), _P]),
    ("fct_server_create", ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_double]),
    ("fct_server_submit", ctypes.c_int, [_P, _P, _P, _P, ctypes.POINTER(ctypes.c_int64)]),
    ("fct_server_poll", ctypes.c_int, [_P, ctypes.c_int64, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(fct_report)]),
    ("fct_server_wait", ctypes.c_int, [_P, ctypes.c_int64, ctypes.c_double, ctypes.POINTER(fct_report)]),
    ("fct_server_destroy", ctypes.c_int, [_P]),
    ("fct_selftest_wait_timeout", ctypes.c_int, [ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                                 ctypes.POINTER(ctypes.c_double)]),
    ("fct_measure_l2", ctypes.c_int, [ctypes.c_int64, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                      ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]),
    ("fct_measure_fp64", ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    ("fct_alias_tables_host", ctypes.c_int, [ctypes.c_int, ctypes.c_int64, _P, ctypes.c_int, _P, _P, ctypes.c_int, _P,
                                             _P, _P, ctypes.POINTER(ctypes.c_int64)]),
]


def library_path() -> str:
    return _build.LIB


def lib() -> ctypes.CDLL:
    """Load libfct_gb300.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_2309_14584_gb300.build.build()")
        L = ctypes.CDLL(path)
        for name, res, args in SIGNATURES:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def status_string(status: int) -> str:
    return lib().fct_status_string(int(status)).decode()


def _check(status: int):
    if status != FCT_OK:
        raise FctError(status, lib().fct_last_error().decode())


def _ptr(x) -> int | None:
    """Address of a numpy array, a torch tensor or an int (None stays NULL)."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot take the address of {type(x)!r}")


def _stream(stream) -> int | None:
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def fct_default_options(**overrides) -> fct_options:
    o = fct_options()
    lib().fct_default_options(ctypes.byref(o))
    for k, v in overrides.items():
        if v is None:
            continue
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def fct_plan_create(support: np.ndarray, sizes: np.ndarray, nodes: np.ndarray | None = None,
                    options: fct_options | None = None) -> int:
    support = np.ascontiguousarray(support, dtype=np.uint16)
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    N, D = support.shape
    K = sizes.shape[0]
    if sizes.shape != (K, D):
        raise ValueError("sizes must be [K, D]")
    if nodes is not None:
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
        if nodes.shape != (K, D):
            raise ValueError("nodes must be [K, D]")
    h = _P()
    opt = options if options is not None else fct_default_options()
    _check(lib().fct_plan_create(ctypes.byref(h), D, N, _ptr(support), K, _ptr(sizes), _ptr(nodes),
                                 ctypes.byref(opt)))
    return h.value


def fct_plan_get_info(plan: int) -> dict:
    info = fct_plan_info()
    _check(lib().fct_plan_get_info(plan, ctypes.byref(info)))
    return info.as_dict()


def fct_grid_offsets(plan: int) -> np.ndarray:
    K = fct_plan_get_info(plan)["K"]
    off = np.zeros(K + 1, dtype=np.int64)
    _check(lib().fct_grid_offsets(plan, _ptr(off)))
    return off


def fct_sample(plan: int, family: int, params: np.ndarray, samples, stream=None):
    params = np.ascontiguousarray(params, dtype=np.float64)
    _check(lib().fct_sample(plan, family, _ptr(params), params.size, _ptr(samples), _stream(stream)))


def fct_execute(plan: int, samples, coeffs, stream=None, report: bool = True) -> dict | None:
    """Execute on device buffers.  With report=True waits and returns the report."""
    if report:
        rep = fct_report()
        st = lib().fct_execute(plan, _ptr(samples), _ptr(coeffs), _stream(stream), ctypes.byref(rep))
        if st not in (FCT_OK,):
            raise FctError(st, lib().fct_last_error().decode() + f" (report {rep.as_dict()})")
        return rep.as_dict()
    _check(lib().fct_execute(plan, _ptr(samples), _ptr(coeffs), _stream(stream), None))
    return None


def fct_execute_host(plan: int, samples_host, coeffs_host, stream=None) -> dict:
    rep = fct_report()
    st = lib().fct_execute_host(plan, _ptr(samples_host), _ptr(coeffs_host), _stream(stream), ctypes.byref(rep))
    if st != FCT_OK:
        raise FctError(st, lib().fct_last_error().decode() + f" (report {rep.as_dict()})")
    return rep.as_dict()


def fct_execute_batch(plans, samples, coeffs, team_blocks: int = 0, stream=None, report: bool = True):
    B = len(plans)
    hp = (_P * B)(*plans)
    hs = (_P * B)(*[_ptr(s) for s in samples])
    hc = (_P * B)(*[_ptr(c) for c in coeffs])
    if report:
        reps = (fct_report * B)()
        st = lib().fct_execute_batch(B, hp, hs, hc, team_blocks, _stream(stream), reps)
        if st != FCT_OK:
            raise FctError(st, lib().fct_last_error().decode())
        return [r.as_dict() for r in reps]
    _check(lib().fct_execute_batch(B, hp, hs, hc, team_blocks, _stream(stream), None))
    return None


def fct_batch_create(plans, samples, coeffs, team_blocks: int = 0) -> int:
    """A prepared batch (include/fct.h): the job table stays on the device, so
    fct_batch_launch needs nothing from the host and can be captured in a
    CUDA graph."""
    B = len(plans)
    hp = (_P * B)(*plans)
    hs = (_P * B)(*[_ptr(s) for s in samples])
    hc = (_P * B)(*[_ptr(c) for c in coeffs])
    out = _P()
    _check(lib().fct_batch_create(ctypes.byref(out), B, hp, hs, hc, team_blocks))
    return out.value


def fct_batch_launch(batch: int, stream=None):
    _check(lib().fct_batch_launch(batch, _stream(stream)))


def fct_batch_reports(batch: int, n: int, stream=None) -> list:
    reps = (fct_report * n)()
    st = lib().fct_batch_reports(batch, _stream(stream), reps)
    if st != FCT_OK:
        raise FctError(st, lib().fct_last_error().decode())
    return [r.as_dict() for r in reps]


def fct_batch_destroy(batch: int):
    _check(lib().fct_batch_destroy(batch))


def fct_execute_noalloc(plan: int, samples, coeffs, stream=None, report: bool = True) -> dict | None:
    """fct_execute with the solver workspace in the library's fixed device
    array (no device allocation; see include/fct.h)."""
    if report:
        rep = fct_report()
        st = lib().fct_execute_noalloc(plan, _ptr(samples), _ptr(coeffs), _stream(stream), ctypes.byref(rep))
        if st != FCT_OK:
            raise FctError(st, lib().fct_last_error().decode() + f" (report {rep.as_dict()})")
        return rep.as_dict()
    _check(lib().fct_execute_noalloc(plan, _ptr(samples), _ptr(coeffs), _stream(stream), None))
    return None


def fct_plan_last_report(plan: int, stream=None) -> dict:
    rep = fct_report()
    st = lib().fct_plan_last_report(plan, _stream(stream), ctypes.byref(rep))
    if st != FCT_OK:
        raise FctError(st, lib().fct_last_error().decode())
    return rep.as_dict()


def fct_selftest_wait_timeout(timeout_s: float = 0.2) -> tuple[int, float]:
    """(device status, seconds) of a wait that can only end by its limit."""
    st = ctypes.c_int()
    el = ctypes.c_double()
    _check(lib().fct_selftest_wait_timeout(timeout_s, ctypes.byref(st), ctypes.byref(el)))
    return st.value, el.value


def fct_plan_condition(plan: int, start, work, iterations: int = 200, stream=None) -> dict:
    """Lanczos estimate of kappa(A) from `iterations` CG iterations on
    A^T A z = start (device double[N]; work: device double[N] scratch)."""
    k, lo, hi = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    used = ctypes.c_int()
    _check(lib().fct_plan_condition(plan, _ptr(start), _ptr(work), iterations, ctypes.byref(k), ctypes.byref(lo),
                                    ctypes.byref(hi), ctypes.byref(used), _stream(stream)))
    return {"kappa": k.value, "lambda_min": lo.value, "lambda_max": hi.value, "iterations": used.value}


def fct_evaluate(plan: int, coeffs, points, values, stream=None):
    """values[p] = sum_m coeffs[m] prod_i T_{m_i}(points[p, i]) (device buffers)."""
    n = int(points.shape[0]) if hasattr(points, "shape") else 0
    _check(lib().fct_evaluate(plan, _ptr(coeffs), n, _ptr(points), _ptr(values), _stream(stream)))


def fct_measure_team_barrier(blocks: int, block_threads: int = 256, rounds: int = 2000) -> float:
    """Microseconds per crossing of the team barrier with no work in between."""
    us = ctypes.c_double()
    _check(lib().fct_measure_team_barrier(blocks, block_threads, rounds, ctypes.byref(us)))
    return us.value


def fct_measure_l2(bytes_: int = 32 << 20, passes: int = 200) -> dict:
    """L2 read bandwidth (GB/s) and random 8-byte gather rate of the current device."""
    r, g, s = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().fct_measure_l2(bytes_, passes, ctypes.byref(r), ctypes.byref(g), ctypes.byref(s)))
    return {"read_gbs": r.value, "gather_gloads_per_s": g.value, "gather_sector_gbs": s.value}


def fct_measure_fp64(iters: int = 1 << 16) -> float:
    """FP64 fma rate of the current device in TFLOP/s."""
    t = ctypes.c_double()
    _check(lib().fct_measure_fp64(iters, ctypes.byref(t)))
    return t.value


def fct_plan_apply(plan: int, x, y, transpose: bool = False, stream=None) -> np.ndarray:
    """y = A x (transpose False) or y = A^T x (True) on device buffers; returns
    each row's sample index (host int64[R])."""
    R = fct_plan_get_info(plan)["R"]
    bins = np.zeros(R, dtype=np.int64)
    _check(lib().fct_plan_apply(plan, _ptr(x), _ptr(y), 1 if transpose else 0, _ptr(bins), _stream(stream)))
    return bins


def fct_plan_tables(plan: int) -> dict:
    """The plan's alias tables copied to the host (rows in the internal
    order): rowptr int32[R+1], col int32[K N], wcsr f64[K N] (CSR), crow
    int32[K, N], wcm f64[K, N] (coefficient-major), bins int64[R]."""
    info = fct_plan_get_info(plan)
    R, K, N = info["R"], info["K"], info["N"]
    t = {"rowptr": np.zeros(R + 1, np.int32), "col": np.zeros(K * N, np.int32), "wcsr": np.zeros(K * N),
         "crow": np.zeros((K, N), np.int32), "wcm": np.zeros((K, N)), "bins": np.zeros(R, np.int64)}
    _check(lib().fct_plan_tables(plan, _ptr(t["rowptr"]), _ptr(t["col"]), _ptr(t["wcsr"]), _ptr(t["crow"]),
                                 _ptr(t["wcm"]), _ptr(t["bins"])))
    return t


def fct_plan_rhs(plan: int, samples, b, stream=None) -> np.ndarray:
    """b = F f at the nonempty bins into the device buffer b (double[R]);
    returns each row's sample index (host int64[R])."""
    R = fct_plan_get_info(plan)["R"]
    bins = np.zeros(R, dtype=np.int64)
    _check(lib().fct_plan_rhs(plan, _ptr(samples), _ptr(b), _ptr(bins), _stream(stream)))
    return bins


def fct_plan_clone(plan: int) -> int:
    h = _P()
    _check(lib().fct_plan_clone(ctypes.byref(h), plan))
    return h.value


def fct_server_create(block_threads: int = 0, team_blocks: int = 0, teams: int = 0,
                      idle_timeout_s: float = 0.05) -> int:
    h = _P()
    _check(lib().fct_server_create(ctypes.byref(h), block_threads, team_blocks, teams, idle_timeout_s))
    return h.value


def fct_server_submit(server: int, plan: int, samples, coeffs) -> int:
    t = ctypes.c_int64()
    _check(lib().fct_server_submit(server, plan, _ptr(samples), _ptr(coeffs), ctypes.byref(t)))
    return t.value


def fct_server_poll(server: int, ticket: int) -> dict | None:
    done = ctypes.c_int()
    rep = fct_report()
    _check(lib().fct_server_poll(server, ticket, ctypes.byref(done), ctypes.byref(rep)))
    return rep.as_dict() if done.value else None


def fct_server_wait(server: int, ticket: int, timeout_s: float = 60.0) -> dict:
    rep = fct_report()
    st = lib().fct_server_wait(server, ticket, timeout_s, ctypes.byref(rep))
    if st != FCT_OK:
        raise FctError(st, lib().fct_last_error().decode() + f" (report {rep.as_dict()})")
    return rep.as_dict()


def fct_server_destroy(server: int):
    if server:
        _check(lib().fct_server_destroy(server))


def fct_destroy(plan: int):
    if plan:
        _check(lib().fct_destroy(plan))


def fct_alias_tables_host(support: np.ndarray, sizes: np.ndarray, nodes: np.ndarray | None = None,
                          grid_kind: int = 0):
    """Host-only alias tables: (bin int32[K,N], crow int32[K,N], weight f64[K,N], R)."""
    support = np.ascontiguousarray(support, dtype=np.uint16)
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    N, D = support.shape
    K = sizes.shape[0]
    if nodes is not None:
        nodes = np.ascontiguousarray(nodes, dtype=np.float64)
    b = np.zeros((K, N), dtype=np.int32)
    c = np.zeros((K, N), dtype=np.int32)
    w = np.zeros((K, N), dtype=np.float64)
    R = ctypes.c_int64()
    _check(lib().fct_alias_tables_host(D, N, _ptr(support), K, _ptr(sizes), _ptr(nodes), grid_kind, _ptr(b), _ptr(c),
                                       _ptr(w), ctypes.byref(R)))
    return b, c, w, int(R.value)


class Plan:
    """Owning wrapper around a fct_plan handle."""

    def __init__(self, support, sizes, nodes=None, **options):
        self.support = np.ascontiguousarray(support, dtype=np.uint16)
        self.sizes = np.ascontiguousarray(sizes, dtype=np.int32)
        self.handle = fct_plan_create(self.support, self.sizes, nodes, fct_default_options(**options))
        self.info = fct_plan_get_info(self.handle)
        self.offsets = fct_grid_offsets(self.handle)

    @property
    def N(self):
        return self.info["N"]

    @property
    def M(self):
        return self.info["M"]

    def clone(self) -> "Plan":
        """Another handle on the same device tables with its own workspace."""
        c = Plan.__new__(Plan)
        c.support, c.sizes = self.support, self.sizes
        c.handle = fct_plan_clone(self.handle)
        c.info = fct_plan_get_info(c.handle)
        c.offsets = self.offsets
        return c

    def sample(self, family, params, samples, stream=None):
        fct_sample(self.handle, family, params, samples, stream)

    def execute(self, samples, coeffs, stream=None, report=True):
        return fct_execute(self.handle, samples, coeffs, stream, report)

    def evaluate(self, coeffs, points, values, stream=None):
        fct_evaluate(self.handle, coeffs, points, values, stream)

    def execute_host(self, samples_host, coeffs_host, stream=None):
        return fct_execute_host(self.handle, samples_host, coeffs_host, stream)

    def close(self):
        if getattr(self, "handle", None):
            fct_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
