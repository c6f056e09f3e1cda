"""Thin ctypes binding of the C ABI in ``include/gbfft.h`` (same names).

Argument marshalling only: every step of the transform runs in the CUDA
kernels of ``libgbfft.so``.  There is no fallback: if the library is missing
or fails to load, every call raises :class:`GbfftError`.

Functions return plain Python values and raise :class:`GbfftError` carrying
the ``gbfft_status`` code on failure.  Device pointers may be given as ints
or as objects with a ``data_ptr()`` method (e.g. ``torch.Tensor``); streams
as ints (``cudaStream_t`` values), ``None`` (legacy default stream) or
objects with a ``cuda_stream`` attribute (``torch.cuda.Stream``).
"""
from __future__ import annotations

import ctypes
import os
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgbfft.so")

GBFFT_FORWARD = -1
GBFFT_INVERSE = +1
GBFFT_C2C_F32 = 0
GBFFT_C2C_F32_TC_FP16X2 = 1
GBFFT_C2C_F32_TC_BF16X2 = 2
GBFFT_C2C_F64 = 3

STATUS_NAMES = {
    0: "GBFFT_OK",
    1: "GBFFT_ERR_INVALID_ARG",
    2: "GBFFT_ERR_UNSUPPORTED_SIZE",
    3: "GBFFT_ERR_ALIGNMENT",
    4: "GBFFT_ERR_OVERLAP",
    5: "GBFFT_ERR_OOM",
    6: "GBFFT_ERR_BUDGET",
    7: "GBFFT_ERR_CUDA",
    8: "GBFFT_ERR_TIMEOUT",
    9: "GBFFT_ERR_DEVICE_STATUS",
    10: "GBFFT_ERR_NOT_FOUND",
}
globals().update({v: k for k, v in STATUS_NAMES.items()})

_c_i64 = ctypes.c_int64
_c_int = ctypes.c_int
_c_vp = ctypes.c_void_p
_c_size = ctypes.c_size_t
_c_i64p = ctypes.POINTER(ctypes.c_int64)
_c_intp = ctypes.POINTER(ctypes.c_int)
_c_sizep = ctypes.POINTER(ctypes.c_size_t)

# name -> (restype, argtypes); mirrors include/gbfft.h
PROTOTYPES = {
    "gbfft_status_string": (ctypes.c_char_p, [_c_int]),
    "gbfft_version": (_c_int, []),
    "gbfft_plan_create": (_c_int, [ctypes.POINTER(_c_vp), _c_i64, _c_i64, _c_int, _c_int]),
    "gbfft_plan_create_variant": (_c_int, [ctypes.POINTER(_c_vp), _c_i64, _c_i64, _c_int, _c_int, _c_int]),
    "gbfft_plan_create_twopass": (_c_int, [ctypes.POINTER(_c_vp), _c_i64, _c_i64, _c_int, _c_int, _c_i64]),
    "gbfft_plan_factors": (_c_int, [_c_vp, _c_i64p, _c_i64p]),
    "gbfft_execute": (_c_int, [_c_vp, _c_vp, _c_vp, _c_vp]),
    "gbfft_execute_host": (_c_int, [_c_vp, _c_vp, _c_vp, _c_vp]),
    "gbfft_destroy": (_c_int, [_c_vp]),
    "gbfft_plan_info": (_c_int, [_c_vp, _c_i64p, _c_i64p, _c_intp, _c_intp, _c_intp, _c_intp, _c_sizep]),
    "gbfft_num_variants": (_c_int, [_c_i64]),
    "gbfft_variant_info": (_c_int, [_c_i64, _c_int, _c_intp, _c_intp, _c_intp, _c_intp, _c_intp]),
    "gbfft_plan_device_status": (_c_int, [_c_vp]),
    "gbfft_variant_kind": (_c_int, [_c_i64, _c_int]),
    "gbfft_plan_grid_cap": (_c_int, [_c_vp]),
    "gbfft_autotune": (_c_int, [_c_i64, _c_i64, _c_int, _c_int, _c_int, _c_intp, _c_i64p,
                                ctypes.POINTER(ctypes.c_float)]),
    "gbfft_wisdom_lookup": (_c_int, [_c_i64, _c_int, _c_int, _c_intp, _c_i64p]),
    "gbfft_wisdom_export": (_c_int, [ctypes.c_char_p]),
    "gbfft_wisdom_import": (_c_int, [ctypes.c_char_p, _c_int]),
    "gbfft_wisdom_forget": (_c_int, []),
    "gbfft_execute_twopass_noalloc": (_c_int, [_c_i64, _c_i64, _c_int, _c_vp, _c_vp, _c_vp]),
    "gbfft_plan_ragged": (_c_int, [ctypes.POINTER(_c_vp), _c_i64p, _c_i64p, _c_i64, _c_int, _c_int]),
    "gbfft_execute_ragged": (_c_int, [_c_vp, _c_vp, _c_vp, _c_vp]),
    "gbfft_ragged_autotune": (_c_int, [_c_vp, _c_vp, _c_vp, _c_int, ctypes.POINTER(ctypes.c_float)]),
    "gbfft_ragged_num_items": (_c_i64, [_c_vp]),
    "gbfft_ragged_tile_split": (_c_int, [_c_vp, _c_i64]),
    "gbfft_ragged_queue_order": (_c_int, [_c_vp]),
    "gbfft_ragged_set_queue_order": (_c_int, [_c_vp, _c_int]),
    "gbfft_ragged_schedule": (_c_int, [_c_vp, _c_i64, _c_intp]),
    "gbfft_ragged_set_engine": (_c_int, [_c_vp, _c_i64, _c_int]),
    "gbfft_ragged_engine": (_c_int, [_c_vp, _c_i64]),
    "gbfft_plan_create_nd": (_c_int, [ctypes.POINTER(_c_vp), _c_int, _c_i64p, _c_i64, _c_int, _c_int]),
    "gbfft_plan_dims": (_c_int, [_c_vp, _c_intp, _c_i64p]),
    "gbfft_server_phases": (_c_int, [_c_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double)]),
    "gbfft_server_timing": (_c_int, [_c_vp, ctypes.c_uint64, ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_double)]),
    "gbfft_formula_check": (_c_int, [ctypes.c_char_p, _c_i64p, _c_intp, _c_int, _c_intp, _c_i64p, ctypes.c_char_p,
                                     ctypes.c_size_t]),
    "gbfft_plan_create_formula": (_c_int, [ctypes.POINTER(_c_vp), ctypes.c_char_p, _c_i64, _c_int, _c_int, _c_intp]),
    "gbfft_formula_form": (_c_int, [ctypes.c_char_p]),
    "gbfft_ragged_set_item_ready": (_c_int, [_c_vp, _c_i64, _c_int]),
    "gbfft_ragged_set_wait_limit": (_c_int, [_c_vp, _c_i64]),
    "gbfft_server_create": (_c_int, [ctypes.POINTER(_c_vp), _c_size, _c_int, _c_int]),
    "gbfft_server_prepare": (_c_int, [_c_vp, _c_i64, _c_int]),
    "gbfft_server_submit": (_c_int, [_c_vp, _c_i64, _c_i64, _c_int, _c_vp, _c_vp,
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "gbfft_server_poll": (_c_int, [_c_vp, ctypes.c_uint64, _c_intp, ctypes.POINTER(ctypes.c_double)]),
    "gbfft_server_wait": (_c_int, [_c_vp, ctypes.c_uint64, ctypes.c_double]),
    "gbfft_server_release": (_c_int, [_c_vp, ctypes.c_uint64]),
    "gbfft_server_replay": (_c_int, [_c_vp, _c_i64, _c_i64p, _c_i64p, _c_intp, ctypes.POINTER(_c_vp),
                                     ctypes.POINTER(_c_vp), ctypes.POINTER(ctypes.c_double),
                                     ctypes.POINTER(ctypes.c_uint64)]),
    "gbfft_server_stats": (_c_int, [_c_vp, ctypes.POINTER(ctypes.c_double)]),
    "gbfft_server_reset_stats": (_c_int, [_c_vp]),
    "gbfft_server_destroy": (_c_int, [_c_vp]),
}
GBFFT_SERVER_SERIAL = 1
GBFFT_SERVER_PHASES = 2
GBFFT_SERVER_PER_LENGTH = 4
GBFFT_SERVER_STAGED = 8
SERVER_PHASES = ("queued_s", "host_s", "device_wait_s", "h2d_s", "kernel_s", "d2h_s", "observe_s", "latency_s")
SERVER_STATS = ("completed", "p50_s", "p99_s", "max_s", "req_per_s", "gb_per_s", "groups",
                "max_inflight_requests", "max_arena_bytes", "window_s")


class GbfftError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = int(status)
        super().__init__(f"{where}: {STATUS_NAMES.get(self.status, self.status)}")


_lib = None
_lock = threading.Lock()


def lib() -> ctypes.CDLL:
    """Load ``libgbfft.so`` (built by ``paper_2207_06803_gb300.build``)."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise GbfftError(GBFFT_ERR_CUDA, f"{LIB_PATH} is missing; run the build first")
                handle = ctypes.CDLL(LIB_PATH)
                for name, (res, args) in PROTOTYPES.items():
                    fn = getattr(handle, name)
                    fn.restype = res
                    fn.argtypes = args
                _lib = handle
    return _lib


def _ptr(x) -> int:
    if x is None:
        return 0
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    return int(x)


def _stream(s) -> int:
    if s is None:
        return 0
    if hasattr(s, "cuda_stream"):
        return int(s.cuda_stream)
    return int(s)


def _check(rc: int, where: str) -> None:
    if rc != 0:
        raise GbfftError(rc, where)


def gbfft_status_string(status: int) -> str:
    return lib().gbfft_status_string(int(status)).decode()


def gbfft_version() -> int:
    return int(lib().gbfft_version())


def gbfft_plan_create(n: int, batch: int, direction: int = GBFFT_FORWARD, dtype: int = GBFFT_C2C_F32) -> int:
    h = _c_vp()
    _check(lib().gbfft_plan_create(ctypes.byref(h), n, batch, direction, dtype), "gbfft_plan_create")
    return int(h.value)


def gbfft_plan_create_variant(n: int, batch: int, direction: int, dtype: int, variant: int) -> int:
    h = _c_vp()
    _check(lib().gbfft_plan_create_variant(ctypes.byref(h), n, batch, direction, dtype, variant),
           "gbfft_plan_create_variant")
    return int(h.value)


def gbfft_plan_create_twopass(n: int, batch: int, direction: int = GBFFT_FORWARD, dtype: int = GBFFT_C2C_F32,
                              k_outer: int = 0) -> int:
    h = _c_vp()
    _check(lib().gbfft_plan_create_twopass(ctypes.byref(h), n, batch, direction, dtype, k_outer),
           "gbfft_plan_create_twopass")
    return int(h.value)


def gbfft_plan_factors(plan: int) -> tuple[int, int]:
    k, m = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().gbfft_plan_factors(plan, ctypes.byref(k), ctypes.byref(m)), "gbfft_plan_factors")
    return k.value, m.value


def gbfft_execute(plan: int, x_in, x_out, stream=None) -> None:
    _check(lib().gbfft_execute(plan, _ptr(x_in), _ptr(x_out), _stream(stream)), "gbfft_execute")


def gbfft_execute_host(plan: int, host_in, host_out, stream=None) -> None:
    """Host pointers (ints, or tensors/arrays exposing data_ptr()/ctypes.data)."""
    def hp(x):
        if hasattr(x, "ctypes"):
            return int(x.ctypes.data)
        return _ptr(x)
    _check(lib().gbfft_execute_host(plan, hp(host_in), hp(host_out), _stream(stream)), "gbfft_execute_host")


def gbfft_destroy(plan: int) -> None:
    _check(lib().gbfft_destroy(plan), "gbfft_destroy")


def gbfft_plan_info(plan: int) -> dict:
    n, batch = ctypes.c_int64(), ctypes.c_int64()
    direction, nst, variant = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    radices = (ctypes.c_int * 8)()
    ws = ctypes.c_size_t()
    _check(lib().gbfft_plan_info(plan, ctypes.byref(n), ctypes.byref(batch), ctypes.byref(direction),
                                 ctypes.byref(nst), radices, ctypes.byref(variant), ctypes.byref(ws)),
           "gbfft_plan_info")
    return {"n": n.value, "batch": batch.value, "direction": direction.value,
            "radices": list(radices[: nst.value]), "variant": variant.value, "workspace_bytes": ws.value}


def gbfft_num_variants(n: int) -> int:
    return int(lib().gbfft_num_variants(n))


def gbfft_variant_info(n: int, index: int) -> dict:
    nst, rows, tpb, smem = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    radices = (ctypes.c_int * 8)()
    _check(lib().gbfft_variant_info(n, index, ctypes.byref(nst), radices, ctypes.byref(rows),
                                    ctypes.byref(tpb), ctypes.byref(smem)), "gbfft_variant_info")
    return {"radices": list(radices[: nst.value]), "rows_per_cta": rows.value,
            "threads_per_cta": tpb.value, "smem_bytes": smem.value}


def gbfft_autotune(n: int, batch: int, direction: int = GBFFT_FORWARD, dtype: int = GBFFT_C2C_F32,
                   reps: int = 5) -> dict:
    v, k, ms = ctypes.c_int(), ctypes.c_int64(), ctypes.c_float()
    _check(lib().gbfft_autotune(n, batch, direction, dtype, reps, ctypes.byref(v), ctypes.byref(k), ctypes.byref(ms)),
           "gbfft_autotune")
    return {"variant": v.value, "k_outer": k.value, "ms": ms.value}


def gbfft_wisdom_lookup(n: int, dtype: int = GBFFT_C2C_F32, direction: int = GBFFT_FORWARD):
    """(variant, k_outer) recorded for (n, dtype, direction), or None."""
    v, k = ctypes.c_int(), ctypes.c_int64()
    rc = lib().gbfft_wisdom_lookup(n, dtype, direction, ctypes.byref(v), ctypes.byref(k))
    if rc == GBFFT_ERR_NOT_FOUND:
        return None
    _check(rc, "gbfft_wisdom_lookup")
    return v.value, k.value


def gbfft_wisdom_export(path: str) -> None:
    _check(lib().gbfft_wisdom_export(os.fsencode(path)), "gbfft_wisdom_export")


def gbfft_wisdom_import(path: str, require_same_gpu: bool = True) -> None:
    _check(lib().gbfft_wisdom_import(os.fsencode(path), 1 if require_same_gpu else 0), "gbfft_wisdom_import")


def gbfft_wisdom_forget() -> None:
    _check(lib().gbfft_wisdom_forget(), "gbfft_wisdom_forget")


def gbfft_plan_grid_cap(plan: int) -> int:
    return int(lib().gbfft_plan_grid_cap(plan))


def gbfft_variant_kind(n: int, index: int) -> int:
    return int(lib().gbfft_variant_kind(n, index))


def gbfft_plan_device_status(plan: int) -> int:
    return int(lib().gbfft_plan_device_status(plan))


def gbfft_execute_twopass_noalloc(n: int, batch: int, direction: int, x_in, x_out, stream=None) -> None:
    """Plan-free two-pass transform whose workspace and tables live in the
    library's static device array (see include/gbfft.h); allocates nothing."""
    _check(lib().gbfft_execute_twopass_noalloc(n, batch, direction, _ptr(x_in), _ptr(x_out), _stream(stream)),
           "gbfft_execute_twopass_noalloc")


def gbfft_plan_ragged(n, offsets, direction: int = GBFFT_FORWARD, dtype: int = GBFFT_C2C_F32) -> int:
    """n, offsets: sequences of int64 (lengths and starting complex elements)."""
    count = len(n)
    an = (ctypes.c_int64 * count)(*[int(v) for v in n])
    ao = (ctypes.c_int64 * count)(*[int(v) for v in offsets])
    h = _c_vp()
    _check(lib().gbfft_plan_ragged(ctypes.byref(h), an, ao, count, direction, dtype), "gbfft_plan_ragged")
    return int(h.value)


def gbfft_execute_ragged(plan: int, x_in, x_out, stream=None) -> None:
    _check(lib().gbfft_execute_ragged(plan, _ptr(x_in), _ptr(x_out), _stream(stream)), "gbfft_execute_ragged")


def gbfft_ragged_autotune(plan: int, x_in, x_out, reps: int = 5) -> float:
    ms = ctypes.c_float()
    _check(lib().gbfft_ragged_autotune(plan, _ptr(x_in), _ptr(x_out), reps, ctypes.byref(ms)),
           "gbfft_ragged_autotune")
    return float(ms.value)


def gbfft_ragged_num_items(plan: int) -> int:
    return int(lib().gbfft_ragged_num_items(plan))


def gbfft_ragged_tile_split(plan: int, n: int) -> int:
    return int(lib().gbfft_ragged_tile_split(plan, n))


def gbfft_plan_create_nd(dims, batch: int, direction: int = GBFFT_FORWARD, dtype: int = GBFFT_C2C_F32) -> int:
    d = (ctypes.c_int64 * max(3, len(dims)))(*[int(v) for v in dims])
    h = ctypes.c_void_p()
    _check(lib().gbfft_plan_create_nd(ctypes.byref(h), len(dims), d, batch, direction, dtype),
           "gbfft_plan_create_nd")
    return h.value


def gbfft_plan_dims(plan: int) -> list[int]:
    r = ctypes.c_int()
    d = (ctypes.c_int64 * 3)()
    _check(lib().gbfft_plan_dims(plan, ctypes.byref(r), d), "gbfft_plan_dims")
    return list(d[: r.value])


def gbfft_formula_check(formula: str) -> dict:
    """Check a Table I factorisation formula; {'n', 'k_outer', 'leaves'} or GbfftError (message in .args)."""
    n, k = ctypes.c_int64(), ctypes.c_int64()
    leaves = (ctypes.c_int * 64)()
    nl = ctypes.c_int()
    err = ctypes.create_string_buffer(256)
    rc = lib().gbfft_formula_check(formula.encode("utf-8"), ctypes.byref(n), leaves, 64, ctypes.byref(nl),
                                   ctypes.byref(k), err, 256)
    if rc != 0:
        raise GbfftError(rc, "gbfft_formula_check: " + err.value.decode("utf-8", "replace"))
    return {"n": n.value, "k_outer": k.value, "leaves": list(leaves[: min(nl.value, 64)])}


def gbfft_formula_form(formula: str) -> int:
    """0 Eq. 2 (or one DFT), 1 its transpose (DIF), 2 Pease's form, -1 rejected."""
    return int(lib().gbfft_formula_form(formula.encode("utf-8")))


def gbfft_plan_create_formula(formula: str, batch: int, direction: int = GBFFT_FORWARD,
                              dtype: int = GBFFT_C2C_F32) -> tuple[int, int]:
    """(plan handle, match level) for a factorisation formula."""
    h = ctypes.c_void_p()
    m = ctypes.c_int()
    _check(lib().gbfft_plan_create_formula(ctypes.byref(h), formula.encode("utf-8"), batch, direction, dtype,
                                           ctypes.byref(m)), "gbfft_plan_create_formula")
    return h.value, m.value


def gbfft_ragged_schedule(plan: int, n: int) -> list[int]:
    rad = (ctypes.c_int * 8)()
    ns = int(lib().gbfft_ragged_schedule(plan, n, rad))
    return list(rad[:max(ns, 0)])


def gbfft_ragged_set_engine(plan: int, n: int, compiled: int) -> None:
    _check(lib().gbfft_ragged_set_engine(plan, n, compiled), "gbfft_ragged_set_engine")


def gbfft_ragged_engine(plan: int, n: int) -> int:
    return int(lib().gbfft_ragged_engine(plan, n))


def gbfft_ragged_set_queue_order(plan: int, order: int) -> None:
    _check(lib().gbfft_ragged_set_queue_order(plan, order), "gbfft_ragged_set_queue_order")


def gbfft_ragged_queue_order(plan: int) -> int:
    return int(lib().gbfft_ragged_queue_order(plan))


def gbfft_ragged_set_item_ready(plan: int, item: int, ready: int) -> None:
    _check(lib().gbfft_ragged_set_item_ready(plan, item, ready), "gbfft_ragged_set_item_ready")


def gbfft_ragged_set_wait_limit(plan: int, nanoseconds: int) -> None:
    _check(lib().gbfft_ragged_set_wait_limit(plan, nanoseconds), "gbfft_ragged_set_wait_limit")


class RaggedPlan:
    """Owning wrapper of a ragged plan."""

    def __init__(self, n, offsets, direction: int = GBFFT_FORWARD, dtype: int = GBFFT_C2C_F32):
        self.handle = gbfft_plan_ragged(n, offsets, direction, dtype)

    def execute(self, x_in, x_out, stream=None) -> None:
        gbfft_execute_ragged(self.handle, x_in, x_out, stream)

    def autotune(self, x_in, x_out, reps: int = 5) -> float:
        return gbfft_ragged_autotune(self.handle, x_in, x_out, reps)

    def num_items(self) -> int:
        return gbfft_ragged_num_items(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            gbfft_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _hptr(x) -> int:
    if hasattr(x, "ctypes"):
        return int(x.ctypes.data)
    return _ptr(x)


def gbfft_server_create(mem_budget_bytes: int, n_streams: int = 4, flags: int = 0) -> int:
    h = _c_vp()
    _check(lib().gbfft_server_create(ctypes.byref(h), mem_budget_bytes, n_streams, flags), "gbfft_server_create")
    return int(h.value)


def gbfft_server_prepare(srv: int, n: int, direction: int = GBFFT_FORWARD) -> None:
    _check(lib().gbfft_server_prepare(srv, n, direction), "gbfft_server_prepare")


def gbfft_server_submit(srv: int, n: int, batch: int, direction: int, host_in, host_out) -> int:
    t = ctypes.c_uint64()
    _check(lib().gbfft_server_submit(srv, n, batch, direction, _hptr(host_in), _hptr(host_out), ctypes.byref(t)),
           "gbfft_server_submit")
    return int(t.value)


def gbfft_server_poll(srv: int, ticket: int) -> tuple[int, float]:
    done, lat = ctypes.c_int(), ctypes.c_double()
    _check(lib().gbfft_server_poll(srv, ticket, ctypes.byref(done), ctypes.byref(lat)), "gbfft_server_poll")
    return done.value, lat.value


def gbfft_server_phases(srv: int, ticket: int) -> dict:
    out = (ctypes.c_double * 8)()
    _check(lib().gbfft_server_phases(srv, ticket, out), "gbfft_server_phases")
    return dict(zip(SERVER_PHASES, list(out)))


def gbfft_server_timing(srv: int, ticket: int) -> tuple[float, float]:
    """(seconds queued before admission, total latency) of a finished request."""
    q, lat = ctypes.c_double(), ctypes.c_double()
    _check(lib().gbfft_server_timing(srv, ticket, ctypes.byref(q), ctypes.byref(lat)), "gbfft_server_timing")
    return q.value, lat.value


def gbfft_server_wait(srv: int, ticket: int, timeout_s: float = 60.0) -> None:
    _check(lib().gbfft_server_wait(srv, ticket, timeout_s), "gbfft_server_wait")


def gbfft_server_release(srv: int, ticket: int) -> None:
    _check(lib().gbfft_server_release(srv, ticket), "gbfft_server_release")


def gbfft_server_replay(srv: int, n, batch, direction, host_in, host_out, arrival_s) -> list[int]:
    cnt = len(n)
    an = (ctypes.c_int64 * cnt)(*[int(v) for v in n])
    ab = (ctypes.c_int64 * cnt)(*[int(v) for v in batch])
    ad = (ctypes.c_int * cnt)(*[int(v) for v in direction])
    ai = (_c_vp * cnt)(*[_hptr(v) for v in host_in])
    ao = (_c_vp * cnt)(*[_hptr(v) for v in host_out])
    at = (ctypes.c_double * cnt)(*[float(v) for v in arrival_s])
    tk = (ctypes.c_uint64 * cnt)()
    _check(lib().gbfft_server_replay(srv, cnt, an, ab, ad, ai, ao, at, tk), "gbfft_server_replay")
    return [int(v) for v in tk]


def gbfft_server_stats(srv: int) -> dict:
    out = (ctypes.c_double * 10)()
    _check(lib().gbfft_server_stats(srv, out), "gbfft_server_stats")
    return dict(zip(SERVER_STATS, list(out)))


def gbfft_server_reset_stats(srv: int) -> None:
    _check(lib().gbfft_server_reset_stats(srv), "gbfft_server_reset_stats")


def gbfft_server_destroy(srv: int) -> None:
    _check(lib().gbfft_server_destroy(srv), "gbfft_server_destroy")


class Server:
    """Continuous-batching FFT server (see include/gbfft.h); host or device buffers in/out."""

    def __init__(self, mem_budget_bytes: int = 4 << 30, n_streams: int = 4, serial: bool = False,
                 phases: bool = False, per_length: bool = False, staged: bool = False):
        flags = ((GBFFT_SERVER_SERIAL if serial else 0) | (GBFFT_SERVER_PHASES if phases else 0)
                 | (GBFFT_SERVER_PER_LENGTH if per_length else 0) | (GBFFT_SERVER_STAGED if staged else 0))
        self.handle = gbfft_server_create(mem_budget_bytes, n_streams, flags)

    def prepare(self, n: int, direction: int = GBFFT_FORWARD) -> None:
        gbfft_server_prepare(self.handle, n, direction)

    def submit(self, n: int, batch: int, direction: int, host_in, host_out) -> int:
        return gbfft_server_submit(self.handle, n, batch, direction, host_in, host_out)

    def poll(self, ticket: int) -> tuple[int, float]:
        return gbfft_server_poll(self.handle, ticket)

    def timing(self, ticket: int) -> tuple[float, float]:
        return gbfft_server_timing(self.handle, ticket)

    def phases(self, ticket: int) -> dict:
        return gbfft_server_phases(self.handle, ticket)

    def wait(self, ticket: int, timeout_s: float = 60.0) -> None:
        gbfft_server_wait(self.handle, ticket, timeout_s)

    def release(self, ticket: int) -> None:
        gbfft_server_release(self.handle, ticket)

    def replay(self, n, batch, direction, host_in, host_out, arrival_s) -> list[int]:
        return gbfft_server_replay(self.handle, n, batch, direction, host_in, host_out, arrival_s)

    def stats(self) -> dict:
        return gbfft_server_stats(self.handle)

    def reset_stats(self) -> None:
        gbfft_server_reset_stats(self.handle)

    def close(self) -> None:
        if getattr(self, "handle", None):
            lib().gbfft_server_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _prod(dims) -> int:
    out = 1
    for v in dims:
        out *= int(v)
    return out


class Plan:
    """Owning wrapper: ``with Plan(n, batch) as p: p.execute(x, y, stream)``; ``n`` may be a shape
    tuple (dims[0], ..., dims[rank-1]) for a multi-dimensional transform."""

    def __init__(self, n, batch: int, direction: int = GBFFT_FORWARD, dtype: int = GBFFT_C2C_F32,
                 variant: int | None = None, k_outer: int | None = None):
        if isinstance(n, (tuple, list)):
            self.handle = gbfft_plan_create_nd(n, batch, direction, dtype)
            self.n, self.batch, self.direction = _prod(n), batch, direction
            return
        if k_outer is not None:
            self.handle = gbfft_plan_create_twopass(n, batch, direction, dtype, k_outer)
        elif variant is None:
            self.handle = gbfft_plan_create(n, batch, direction, dtype)
        else:
            self.handle = gbfft_plan_create_variant(n, batch, direction, dtype, variant)
        self.n, self.batch, self.direction = n, batch, direction

    def execute(self, x_in, x_out, stream=None) -> None:
        gbfft_execute(self.handle, x_in, x_out, stream)

    def execute_host(self, host_in, host_out, stream=None) -> None:
        gbfft_execute_host(self.handle, host_in, host_out, stream)

    def info(self) -> dict:
        d = gbfft_plan_info(self.handle)
        d["k_outer"], d["m_inner"] = gbfft_plan_factors(self.handle)
        return d

    def close(self) -> None:
        if getattr(self, "handle", None):
            gbfft_destroy(self.handle)
            self.handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
