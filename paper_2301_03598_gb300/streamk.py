"""Python binding of libstreamk (include/streamk.h).

The functions carry the C ABI's names and do argument marshalling only: torch
tensors are passed as their ``data_ptr()``, streams as their ``cuda_stream``
handle, names of dtypes/layouts/modes as the C enums.  Every step of the GEMM
runs in the library's CUDA kernels; there is no fallback, and loading fails
loudly when libstreamk.so has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

from .build import INCLUDE, LIB

SK_OK, SK_ERR_INVALID, SK_ERR_UNSUPPORTED, SK_ERR_CUDA, SK_ERR_TIMEOUT, SK_ERR_NOMEM, \
    SK_ERR_DEVICE, SK_ERR_BUSY = range(8)
DTYPES = {"f16": 0, "bf16": 1, "f32": 2, "e4m3": 3}
LAYOUTS = {"row": 0, "col": 1}
MODES = {"auto": 0, "dp": 1, "sk": 2, "hybrid": 3, "hybrid1": 4}
MODE_NAMES = {v: k for k, v in MODES.items()}
ATTRS = {
    "tile_n": 1, "grid": 2, "raster_group": 3, "timeout_ns": 4, "lda": 5, "ldb": 6, "ldc": 7,
    "debug_skip_signal": 8, "pdl": 9, "cluster_m": 10, "store": 11, "independent_inputs": 12,
    "stages": 13,
    "mode": 20, "tile_m": 21, "tile_k": 22, "tiles_m": 23,
    "tiles_n": 24, "tiles": 25, "iters_per_tile": 26, "sk_tiles": 27, "dp_tiles": 28,
    "workspace_bytes": 29, "num_sms": 30, "trace_ints": 31, "trace_cap": 32, "ctas": 33,
    "segments": 34,
}
GROUPED_ONLY_ATTRS = ("segments",)
TRACE_FIELDS = 9
TRACE_HEADER = 4
TRACE_RECORD = 16


class StreamKError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {sk_status_string(status)}")
        self.status = status


class sk_schedule_info(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("tile_m", ctypes.c_int32), ("tile_n", ctypes.c_int32),
                ("tile_k", ctypes.c_int32), ("tiles_m", ctypes.c_int32),
                ("tiles_n", ctypes.c_int32), ("tiles", ctypes.c_int64),
                ("iters_per_tile", ctypes.c_int32), ("grid", ctypes.c_int32),
                ("sk_tiles", ctypes.c_int64), ("dp_tiles", ctypes.c_int64),
                ("sk_iters", ctypes.c_int64), ("raster_group", ctypes.c_int32),
                ("max_segments", ctypes.c_int32), ("workspace_bytes", ctypes.c_int64),
                ("cluster_m", ctypes.c_int32), ("ctas", ctypes.c_int32)]

    def as_dict(self):
        d = {name: getattr(self, name) for name, _ in self._fields_}
        d["mode_name"] = MODE_NAMES.get(d["mode"], "?")
        return d


_lib = None


def lib() -> ctypes.CDLL:
    """The loaded libstreamk.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise ImportError(f"libstreamk.so is not built ({LIB}); run "
                          "`python -m paper_2301_03598_gb300.build`")
    L = ctypes.CDLL(LIB)
    i32, i64, vp, f32 = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p, ctypes.c_float
    L.sk_plan.argtypes = [ctypes.POINTER(vp), i64, i64, i64, i32, i32, i32, i32, i32, i32, i32,
                          i32]
    L.sk_gemm.argtypes = [vp, vp, vp, vp, f32, f32, vp]
    L.sk_gemm_traced.argtypes = [vp, vp, vp, vp, f32, f32, vp, i64, vp]
    L.sk_gemm_scaled.argtypes = [vp, vp, vp, vp, vp, vp, f32, f32, vp]
    L.sk_last_error.argtypes = [vp, ctypes.POINTER(i32)]
    L.sk_plan_destroy.argtypes = [vp]
    L.sk_plan_set.argtypes = [vp, i32, i64]
    L.sk_plan_get.argtypes = [vp, i32, ctypes.POINTER(i64)]
    L.sk_plan_attach_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    L.sk_plan_describe.argtypes = [i64, i64, i64, i32, i32, i32, i32, i32, i32,
                                   ctypes.POINTER(sk_schedule_info)]
    L.sk_model_coefficients.argtypes = [i32, i32, ctypes.POINTER(ctypes.c_double)]
    L.sk_model_time.argtypes = [ctypes.POINTER(sk_schedule_info), ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_double)]
    L.sk_grid_model.argtypes = [i64, i64, i64, i32, i32, i32, i32, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(i32)]
    L.sk_gemm_noalloc.argtypes = [i64, i64, i64, i32, i32, vp, i64, vp, i64, vp, i64, f32, f32,
                                  i32, vp, vp]
    vpp = ctypes.POINTER(vp)
    i64p = ctypes.POINTER(i64)
    f32p = ctypes.POINTER(f32)
    L.sk_grouped_plan.argtypes = [ctypes.POINTER(vp), i32, i64p, i64p, i64p, i32, i32, i32]
    L.sk_grouped_gemm.argtypes = [vp, vpp, vpp, vpp, f32p, f32p, vp]
    L.sk_grouped_gemm_traced.argtypes = [vp, vpp, vpp, vpp, f32p, f32p, vp, i64, vp]
    L.sk_grouped_gemm_scaled.argtypes = [vp, vpp, vpp, vpp, vpp, vpp, f32p, f32p, vp]
    L.sk_grouped_last_error.argtypes = [vp, ctypes.POINTER(i32)]
    L.sk_grouped_set.argtypes = [vp, i32, i64]
    L.sk_grouped_get.argtypes = [vp, i32, i64p]
    L.sk_grouped_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), i64, i64p]
    L.sk_grouped_destroy.argtypes = [vp]
    dblp = ctypes.POINTER(ctypes.c_double)
    L.sk_server_create.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, i64]
    L.sk_server_submit.argtypes = [vp, i64, i64, i64, vp, vp, vp, f32, f32,
                                   ctypes.POINTER(ctypes.c_uint64)]
    L.sk_server_submit_scaled.argtypes = [vp, i64, i64, i64, vp, vp, vp, vp, vp, f32, f32,
                                          ctypes.POINTER(ctypes.c_uint64)]
    L.sk_server_poll.argtypes = [vp, ctypes.c_uint64, ctypes.POINTER(i32), dblp]
    L.sk_server_wait.argtypes = [vp, ctypes.c_uint64, dblp]
    L.sk_server_stats.argtypes = [vp, i64p]
    L.sk_server_destroy.argtypes = [vp]
    L.sk_plan_autotune.argtypes = [vp, vp, vp, vp, i32, vp, dblp]
    L.sk_grouped_autotune.argtypes = [vp, vpp, vpp, vpp, i32, vp, dblp]
    L.sk_plan_autotune_scaled.argtypes = [vp, vp, vp, vp, vp, vp, i32, vp, dblp]
    L.sk_grouped_autotune_scaled.argtypes = [vp, vpp, vpp, vpp, vpp, vpp, i32, vp, dblp]
    L.sk_grouped_plan_describe.argtypes = [i32, i64p, i64p, i64p, i32, i32, i32, i32, i32, i64p,
                                           ctypes.POINTER(ctypes.c_int32), i64, i64p]
    L.sk_status_string.argtypes = [i32]
    L.sk_status_string.restype = ctypes.c_char_p
    for name in ("sk_plan", "sk_gemm", "sk_gemm_traced", "sk_last_error", "sk_plan_destroy",
                 "sk_plan_set", "sk_plan_get", "sk_plan_attach_workspace", "sk_plan_describe",
                 "sk_grid_model", "sk_model_coefficients", "sk_model_time", "sk_gemm_noalloc",
                 "sk_grouped_plan", "sk_grouped_gemm",
                 "sk_grouped_gemm_traced", "sk_grouped_last_error", "sk_grouped_set",
                 "sk_grouped_get", "sk_grouped_schedule", "sk_grouped_destroy",
                 "sk_grouped_plan_describe", "sk_plan_autotune", "sk_grouped_autotune",
                 "sk_gemm_scaled", "sk_grouped_gemm_scaled", "sk_plan_autotune_scaled",
                 "sk_grouped_autotune_scaled", "sk_server_submit_scaled",
                 "sk_server_create", "sk_server_submit", "sk_server_poll", "sk_server_wait",
                 "sk_server_stats", "sk_server_destroy"):
        getattr(L, name).restype = i32
    _lib = L
    return L


def header_functions():
    """Names of the functions include/*.h declares (for export checks)."""
    names = []
    for f in sorted(os.listdir(INCLUDE)):
        if f.endswith(".h"):
            text = open(os.path.join(INCLUDE, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[a-z_0-9]+\s*\*?\s*(sk_[a-z_0-9]+)\s*\(", text,
                                re.M)
    return names


def _code(table, v, what):
    if isinstance(v, int):
        return v
    try:
        return table[v]
    except KeyError:
        raise ValueError(f"unknown {what} {v!r}") from None


def _dtype_name(x):
    try:
        import torch
        m = {torch.float16: "f16", torch.bfloat16: "bf16", torch.float32: "f32",
             torch.float8_e4m3fn: "e4m3"}
        if x in m:
            return m[x]
    except ImportError:  # pragma: no cover
        pass
    return x


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> Optional[int]:
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _check(status, what):
    if status != SK_OK:
        raise StreamKError(status, what)


class Plan:
    """Owner of an sk_plan_t handle."""

    def __init__(self, handle: int, m: int, n: int, k: int, a_type: str, c_type: str):
        self.handle = handle
        self.m, self.n, self.k = m, n, k
        self.a_type, self.c_type = a_type, c_type

    def get(self, attr) -> int:
        return sk_plan_get(self, attr)

    def set(self, attr, value: int) -> None:
        sk_plan_set(self, attr, value)

    def info(self):
        return {name: self.get(name) for name in ATTRS if name not in GROUPED_ONLY_ATTRS}

    def destroy(self):
        if self.handle:
            lib().sk_plan_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.destroy()
        except Exception:
            pass


def sk_status_string(status: int) -> str:
    return lib().sk_status_string(status).decode()


def sk_plan(m: int, n: int, k: int, a_type="bf16", b_type=None, c_type="bf16",
            compute_type="f32", a_layout="row", b_layout="col", c_layout="row",
            mode="auto") -> Plan:
    a_type = _dtype_name(a_type)
    b_type = a_type if b_type is None else _dtype_name(b_type)
    c_type = _dtype_name(c_type)
    h = ctypes.c_void_p()
    st = lib().sk_plan(ctypes.byref(h), m, n, k, _code(DTYPES, a_type, "dtype"),
                       _code(DTYPES, b_type, "dtype"), _code(DTYPES, c_type, "dtype"),
                       _code(DTYPES, _dtype_name(compute_type), "dtype"),
                       _code(LAYOUTS, a_layout, "layout"), _code(LAYOUTS, b_layout, "layout"),
                       _code(LAYOUTS, c_layout, "layout"), _code(MODES, mode, "mode"))
    _check(st, "sk_plan")
    return Plan(h.value, m, n, k, a_type, c_type)


def sk_plan_destroy(plan: Plan) -> None:
    plan.destroy()


def sk_plan_set(plan: Plan, attr, value: int) -> None:
    _check(lib().sk_plan_set(plan.handle, _code(ATTRS, attr, "attr"), int(value)), "sk_plan_set")


def sk_plan_get(plan: Plan, attr) -> int:
    v = ctypes.c_int64()
    _check(lib().sk_plan_get(plan.handle, _code(ATTRS, attr, "attr"), ctypes.byref(v)),
           "sk_plan_get")
    return v.value


def sk_plan_attach_workspace(plan: Plan, ws, nbytes: int) -> None:
    """Attach caller memory as the plan's workspace.  The plan object keeps a
    reference to ``ws`` so the memory outlives every launch that uses it."""
    _check(lib().sk_plan_attach_workspace(plan.handle, _ptr(ws), nbytes),
           "sk_plan_attach_workspace")
    plan._workspace = ws


def sk_gemm(plan: Plan, A, B, C, alpha: float = 1.0, beta: float = 0.0, stream=None) -> None:
    """C = alpha * A @ B + beta * C (A row-major m x k, B column-major k x n,
    i.e. an n x k row-major tensor).  Asynchronous on ``stream``."""
    _check(lib().sk_gemm(plan.handle, _ptr(A), _ptr(B), _ptr(C), alpha, beta, _stream(stream)),
           "sk_gemm")


def sk_gemm_scaled(plan: Plan, A, B, scale_a, scale_b, C, alpha: float = 1.0, beta: float = 0.0,
                   stream=None) -> None:
    """Block-scaled E4M3 GEMM: C = alpha * sum over k-blocks of 128 of
    scale_a[i/128, kb] * scale_b[j/128, kb] * A_kb @ B_kb + beta * C, with
    scale_a FP32 [ceil(m/128), ceil(k/128)] and scale_b [ceil(n/128),
    ceil(k/128)] on the device."""
    _check(lib().sk_gemm_scaled(plan.handle, _ptr(A), _ptr(B), _ptr(scale_a), _ptr(scale_b),
                                _ptr(C), alpha, beta, _stream(stream)), "sk_gemm_scaled")


def sk_gemm_traced(plan: Plan, A, B, C, alpha: float, beta: float, trace, stream=None) -> None:
    n_ints = trace.numel() if hasattr(trace, "numel") else plan.get("trace_ints")
    _check(lib().sk_gemm_traced(plan.handle, _ptr(A), _ptr(B), _ptr(C), alpha, beta, _ptr(trace),
                                n_ints, _stream(stream)), "sk_gemm_traced")


def sk_gemm_noalloc(m: int, n: int, k: int, ab_type, c_type, A, lda: int, B, ldb: int, C,
                    ldc: int, alpha: float = 1.0, beta: float = 0.0, mode="auto",
                    device_status=None, stream=None) -> None:
    """The allocation-free GEMM (no plan; fixed scratch inside the library)."""
    _check(lib().sk_gemm_noalloc(m, n, k, _code(DTYPES, _dtype_name(ab_type), "dtype"),
                                 _code(DTYPES, _dtype_name(c_type), "dtype"), _ptr(A), lda,
                                 _ptr(B), ldb, _ptr(C), ldc, alpha, beta,
                                 _code(MODES, mode, "mode"), _ptr(device_status),
                                 _stream(stream)), "sk_gemm_noalloc")


def sk_last_error(plan: Plan):
    """(status, device_status) after waiting for the plan's last launch."""
    dev = ctypes.c_int(0)
    st = lib().sk_last_error(plan.handle, ctypes.byref(dev))
    return st, dev.value


def sk_plan_describe(m: int, n: int, k: int, mode="auto", tile_n: int = 0, grid: int = 0,
                     raster_group: int = 0, num_sms: int = 148, cluster_m: int = 0):
    info = sk_schedule_info()
    _check(lib().sk_plan_describe(m, n, k, _code(MODES, mode, "mode"), tile_n, grid,
                                  raster_group, cluster_m, num_sms, ctypes.byref(info)),
           "sk_plan_describe")
    return info.as_dict()


def sk_grid_model(m: int, n: int, k: int, bm: int, bn: int, bk: int, p: int, coef) -> int:
    c = (ctypes.c_double * 4)(*coef)
    g = ctypes.c_int(0)
    _check(lib().sk_grid_model(m, n, k, bm, bn, bk, p, c, ctypes.byref(g)), "sk_grid_model")
    return g.value


def sk_model_coefficients(tile_n: int, cluster_m: int):
    """The planner's six model terms (us) of one tile configuration."""
    c = (ctypes.c_double * 6)()
    _check(lib().sk_model_coefficients(tile_n, cluster_m, c), "sk_model_coefficients")
    return list(c)


def sk_model_time(m: int, n: int, k: int, mode="auto", tile_n: int = 0, grid: int = 0,
                  num_sms: int = 148, cluster_m: int = 0, coef=None):
    """Modelled time (us) of the schedule sk_plan_describe gives for these
    arguments, under `coef` (default: its configuration's built-in terms)."""
    info = sk_schedule_info()
    _check(lib().sk_plan_describe(m, n, k, _code(MODES, mode, "mode"), tile_n, grid, 0,
                                  cluster_m, num_sms, ctypes.byref(info)), "sk_plan_describe")
    if coef is None:
        coef = sk_model_coefficients(info.tile_n, info.cluster_m)
    c = (ctypes.c_double * 6)(*coef)
    us = ctypes.c_double(0.0)
    _check(lib().sk_model_time(ctypes.byref(info), c, ctypes.byref(us)), "sk_model_time")
    return us.value


def decode_trace(trace_host, grid: int, cap: int, with_times: bool = False):
    """Turn a copied-back trace buffer into records: tuples of the 9 schedule
    fields, or (fields, (t_acc, t_fix, t_done), t_cta_start) with ``with_times``
    (global-timer nanoseconds)."""
    vals = [int(v) for v in trace_host]
    stride = TRACE_HEADER + cap * TRACE_RECORD

    def u64(lo, hi):
        return (lo & 0xffffffff) | ((hi & 0xffffffff) << 32)

    out = []
    for x in range(grid):
        base = x * stride
        count = vals[base]
        t0 = u64(vals[base + 2], vals[base + 3])
        if count > cap:
            raise ValueError(f"CTA {x} recorded {count} segments, capacity {cap}")
        for r in range(count):
            o = base + TRACE_HEADER + r * TRACE_RECORD
            fields = tuple(vals[o:o + TRACE_FIELDS])
            if with_times:
                ts = tuple(u64(vals[o + 10 + 2 * i], vals[o + 11 + 2 * i]) for i in range(3))
                out.append((fields, ts, t0))
            else:
                out.append(fields)
    return out


# ---------------------------------------------------------------- grouped GEMM
class GroupedPlan:
    """Owner of an sk_grouped_t handle (Stream-K across a group of problems)."""

    def __init__(self, handle: int, shapes, a_type: str, c_type: str):
        self.handle = handle
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.a_type, self.c_type = a_type, c_type

    def get(self, attr) -> int:
        v = ctypes.c_int64()
        _check(lib().sk_grouped_get(self.handle, _code(ATTRS, attr, "attr"), ctypes.byref(v)),
               "sk_grouped_get")
        return v.value

    def set(self, attr, value: int) -> None:
        _check(lib().sk_grouped_set(self.handle, _code(ATTRS, attr, "attr"), int(value)),
               "sk_grouped_set")

    def info(self):
        names = ("mode", "tile_m", "tile_n", "tile_k", "grid", "ctas", "tiles", "sk_tiles",
                 "dp_tiles", "workspace_bytes", "num_sms", "trace_cap", "trace_ints", "segments",
                 "stages", "cluster_m")
        return {name: self.get(name) for name in names}

    def destroy(self):
        if self.handle:
            lib().sk_grouped_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()

    def __del__(self):  # pragma: no cover - interpreter shutdown order
        try:
            self.destroy()
        except Exception:
            pass


def sk_grouped_plan(shapes, ab_type="bf16", c_type="bf16", mode="auto") -> GroupedPlan:
    """shapes: a sequence of (m, n, k)."""
    cnt = len(shapes)
    arr = lambda j: (ctypes.c_int64 * cnt)(*[int(s[j]) for s in shapes])
    h = ctypes.c_void_p()
    ab = _dtype_name(ab_type)
    c = _dtype_name(c_type)
    _check(lib().sk_grouped_plan(ctypes.byref(h), cnt, arr(0), arr(1), arr(2),
                                 _code(DTYPES, ab, "dtype"), _code(DTYPES, c, "dtype"),
                                 _code(MODES, mode, "mode")), "sk_grouped_plan")
    return GroupedPlan(h.value, shapes, ab, c)


def _ptr_array(xs):
    return (ctypes.c_void_p * len(xs))(*[_ptr(x) for x in xs])


def _f32_array(xs):
    return None if xs is None else (ctypes.c_float * len(xs))(*[float(v) for v in xs])


def sk_grouped_gemm(plan: GroupedPlan, As, Bs, Cs, alpha=None, beta=None, stream=None) -> None:
    """C_i = alpha_i * A_i @ B_i + beta_i * C_i for every problem of the plan, in
    one launch (A_i m x k row-major, B_i an n x k row-major tensor)."""
    _check(lib().sk_grouped_gemm(plan.handle, _ptr_array(As), _ptr_array(Bs), _ptr_array(Cs),
                                 _f32_array(alpha), _f32_array(beta), _stream(stream)),
           "sk_grouped_gemm")


def sk_grouped_gemm_scaled(plan: GroupedPlan, As, Bs, SAs, SBs, Cs, alpha=None, beta=None,
                           stream=None) -> None:
    """sk_grouped_gemm for an E4M3 group, with every problem's block scales."""
    _check(lib().sk_grouped_gemm_scaled(plan.handle, _ptr_array(As), _ptr_array(Bs),
                                        _ptr_array(SAs), _ptr_array(SBs), _ptr_array(Cs),
                                        _f32_array(alpha), _f32_array(beta), _stream(stream)),
           "sk_grouped_gemm_scaled")


def sk_grouped_gemm_traced(plan: GroupedPlan, As, Bs, Cs, alpha, beta, trace, stream=None) -> None:
    _check(lib().sk_grouped_gemm_traced(plan.handle, _ptr_array(As), _ptr_array(Bs),
                                        _ptr_array(Cs), _f32_array(alpha), _f32_array(beta),
                                        _ptr(trace), trace.numel(), _stream(stream)),
           "sk_grouped_gemm_traced")


def sk_grouped_last_error(plan: GroupedPlan):
    dev = ctypes.c_int(0)
    st = lib().sk_grouped_last_error(plan.handle, ctypes.byref(dev))
    return st, dev.value


def sk_grouped_schedule(plan: GroupedPlan):
    """The plan's schedule as records (cta, problem, tile, tm, tn, kb0, kb1,
    role, peer_first, peer_last), CTA by CTA in processing order."""
    cnt = ctypes.c_int64(0)
    _check(lib().sk_grouped_schedule(plan.handle, None, 0, ctypes.byref(cnt)), "sk_grouped_schedule")
    buf = (ctypes.c_int32 * (10 * max(1, cnt.value)))()
    _check(lib().sk_grouped_schedule(plan.handle, buf, 10 * max(1, cnt.value), ctypes.byref(cnt)),
           "sk_grouped_schedule")
    vals = list(buf)
    return [tuple(vals[10 * i:10 * i + 10]) for i in range(cnt.value)]


def sk_grouped_destroy(plan: GroupedPlan) -> None:
    plan.destroy()


def sk_grouped_plan_describe(shapes, mode="auto", tile_n: int = 0, grid: int = 0,
                             num_sms: int = 148, cluster_m: int = 1):
    """Host-only grouped planning: (summary dict, records) without a device.
    cluster_m 0 lets the model choose single CTAs or CTA pairs (records and
    grid then count units)."""
    cnt = len(shapes)
    arr = lambda j: (ctypes.c_int64 * cnt)(*[int(s[j]) for s in shapes])
    m, n, k = arr(0), arr(1), arr(2)
    summary = (ctypes.c_int64 * 9)()
    nrec = ctypes.c_int64(0)
    _check(lib().sk_grouped_plan_describe(cnt, m, n, k, _code(MODES, mode, "mode"), tile_n, grid,
                                          num_sms, cluster_m, summary, None, 0,
                                          ctypes.byref(nrec)), "sk_grouped_plan_describe")
    buf = (ctypes.c_int32 * (10 * max(1, nrec.value)))()
    _check(lib().sk_grouped_plan_describe(cnt, m, n, k, _code(MODES, mode, "mode"), tile_n, grid,
                                          num_sms, cluster_m, summary, buf,
                                          10 * max(1, nrec.value), ctypes.byref(nrec)),
           "sk_grouped_plan_describe")
    keys = ("mode", "tile_n", "tile_k", "grid", "tiles", "sk_tiles", "workspace_bytes",
            "max_segments", "cluster_m")
    info = dict(zip(keys, list(summary)))
    info["mode_name"] = MODE_NAMES.get(info["mode"], "?")
    vals = list(buf)
    return info, [tuple(vals[10 * i:10 * i + 10]) for i in range(nrec.value)]


def sk_plan_autotune(plan: Plan, A, B, C, reps: int = 5, stream=None) -> float:
    """Time every configuration on these operands and keep the fastest (C is
    overwritten).  Returns the kept configuration's mean microseconds."""
    best = ctypes.c_double(0.0)
    _check(lib().sk_plan_autotune(plan.handle, _ptr(A), _ptr(B), _ptr(C), int(reps),
                                  _stream(stream), ctypes.byref(best)), "sk_plan_autotune")
    return best.value


def sk_plan_autotune_scaled(plan: Plan, A, B, scale_a, scale_b, C, reps: int = 5,
                            stream=None) -> float:
    best = ctypes.c_double(0.0)
    _check(lib().sk_plan_autotune_scaled(plan.handle, _ptr(A), _ptr(B), _ptr(scale_a),
                                         _ptr(scale_b), _ptr(C), int(reps), _stream(stream),
                                         ctypes.byref(best)), "sk_plan_autotune_scaled")
    return best.value


def sk_grouped_autotune_scaled(plan: GroupedPlan, As, Bs, SAs, SBs, Cs, reps: int = 3,
                               stream=None) -> float:
    best = ctypes.c_double(0.0)
    _check(lib().sk_grouped_autotune_scaled(plan.handle, _ptr_array(As), _ptr_array(Bs),
                                            _ptr_array(SAs), _ptr_array(SBs), _ptr_array(Cs),
                                            int(reps), _stream(stream), ctypes.byref(best)),
           "sk_grouped_autotune_scaled")
    return best.value


def sk_grouped_autotune(plan: GroupedPlan, As, Bs, Cs, reps: int = 3, stream=None) -> float:
    best = ctypes.c_double(0.0)
    _check(lib().sk_grouped_autotune(plan.handle, _ptr_array(As), _ptr_array(Bs), _ptr_array(Cs),
                                     int(reps), _stream(stream), ctypes.byref(best)),
           "sk_grouped_autotune")
    return best.value


# ---------------------------------------------------------------- serving loop
class Server:
    """Owner of an sk_server_t (continuous batching over grouped launches)."""

    def __init__(self, handle: int):
        self.handle = handle

    def submit(self, A, B, C, alpha: float = 1.0, beta: float = 0.0) -> int:
        """Queue C = alpha*A@B + beta*C (A m x k, B an n x k tensor, C m x n);
        returns the ticket.  The tensors must stay alive until it completes."""
        m, k = A.shape
        n = B.shape[0]
        t = ctypes.c_uint64(0)
        _check(lib().sk_server_submit(self.handle, m, n, k, _ptr(A), _ptr(B), _ptr(C), alpha, beta,
                                      ctypes.byref(t)), "sk_server_submit")
        return t.value

    def submit_scaled(self, A, B, scale_a, scale_b, C, alpha: float = 1.0,
                      beta: float = 0.0) -> int:
        """Queue a block-scaled E4M3 request (as sk_gemm_scaled)."""
        m, k = A.shape
        n = B.shape[0]
        t = ctypes.c_uint64(0)
        _check(lib().sk_server_submit_scaled(self.handle, m, n, k, _ptr(A), _ptr(B),
                                             _ptr(scale_a), _ptr(scale_b), _ptr(C), alpha, beta,
                                             ctypes.byref(t)), "sk_server_submit_scaled")
        return t.value

    def poll(self, ticket: int):
        """(done, status, latency_us)."""
        st = ctypes.c_int(0)
        lat = ctypes.c_double(0.0)
        rc = lib().sk_server_poll(self.handle, ticket, ctypes.byref(st), ctypes.byref(lat))
        return st.value == 2, rc, lat.value

    def wait(self, ticket: int):
        """Block until the request is done: (status, latency_us)."""
        lat = ctypes.c_double(0.0)
        rc = lib().sk_server_wait(self.handle, ticket, ctypes.byref(lat))
        return rc, lat.value

    def stats(self):
        v = (ctypes.c_int64 * 6)()
        _check(lib().sk_server_stats(self.handle, v), "sk_server_stats")
        return dict(zip(("submitted", "completed", "batches", "max_batch", "problems", "queued"),
                        list(v)))

    def destroy(self):
        if self.handle:
            lib().sk_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.destroy()


def sk_server_create(ab_type="bf16", c_type="bf16", max_batch: int = 64, slots: int = 2,
                     hbm_budget_bytes: int = 64 << 30) -> Server:
    h = ctypes.c_void_p()
    _check(lib().sk_server_create(ctypes.byref(h), _code(DTYPES, _dtype_name(ab_type), "dtype"),
                                  _code(DTYPES, _dtype_name(c_type), "dtype"), max_batch, slots,
                                  int(hbm_budget_bytes)), "sk_server_create")
    return Server(h.value)
