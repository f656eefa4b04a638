"""Python binding of libdmerge (include/dmerge.h): argument marshalling only.

The functions below carry the C ABI's names and forward to it through
ctypes; every step of the merge runs in the library's CUDA kernels.  Device
memory and streams come from PyTorch: pass tensors (their data pointers are
taken) and a torch.cuda.Stream (or None for the current stream).

There is no fallback: if libdmerge.so is missing or cannot be loaded,
``load()`` raises.  Build it with ``paper_1109_6885_gb300.build.build()``.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import threading

import numpy as np

from . import build as _build

_lib = None
_lock = threading.Lock()

(DM_OK, DM_EINVAL, DM_ENOMEM, DM_EUNSORTED, DM_ECODE, DM_ECUDA, DM_ETIMEOUT, DM_EBUSY,
 DM_ENOENT, DM_EINTERNAL) = range(10)
DM_FLAG_GENERIC_REENCODE = 0x1
DM_FLAG_X_SMEM = 0x2
DM_FLAG_X_GLOBAL = 0x4
DM_FLAG_TIMING = 0x8
DM_FLAG_SERIAL = 0x10
DM_FLAG_AUTOTUNE = 0x20
DM_FLAG_NO_GRAPH = 0x40
DM_STAGE_AUTO, DM_STAGE_SMEM, DM_STAGE_GLOBAL = 0, 1, 2
DM_WAIT_TEST_OFF = 0xFFFFFFFF
DM_SERVER_DIGEST = 0x1000
DM_X8_AUTO, DM_X8_OFF = 0, 1

EXPORTS = [
    "dm_create", "dm_destroy", "dm_reserve", "dm_arena_bytes", "dm_packed_bytes", "dm_bits_for",
    "dm_max_bits", "dm_scratch_bytes", "dm_merge_column", "dm_merge_table",
    "dm_table_scratch_bytes", "dm_merge_column_host", "dm_host_scratch_bytes", "dm_sort_delta",
    "dm_merge_dicts", "dm_reencode", "dm_sync_status", "dm_last_timing", "dm_timing_sum",
    "dm_launch_count", "dm_merge_dicts_noalloc", "dm_set_tuning", "dm_get_tuning", "dm_last_error",
    "dm_server_create", "dm_server_destroy", "dm_server_add_table", "dm_server_submit",
    "dm_server_drain", "dm_server_request_info", "dm_server_stats_get", "dm_server_table_version",
    "dm_sched_simulate", "dm_server_tune_cache",
    "dm_status_str",
    "dm_tune_key_of", "dm_tune_cache_create", "dm_tune_cache_destroy", "dm_tune_cache_put",
    "dm_tune_cache_get", "dm_tune_cache_size", "dm_tune_cache_generation", "dm_tune_cache_clear",
    "dm_tune_cache_save", "dm_tune_cache_load", "dm_set_tune_cache", "dm_get_tune_cache",
    "dm_tune_candidates", "dm_autotune_column", "dm_reencode_search", "dm_ingest_scratch_bytes",
    "dm_ingest_delta", "dm_set_wait_test", "dm_server_add_online_table", "dm_server_insert",
    "dm_server_pause", "dm_server_online_view", "dm_online_simulate", "dm_server_online_copy",
    "dm_column_digest", "dm_ingest_table_scratch_bytes", "dm_ingest_table",
]


class DmError(RuntimeError):
    def __init__(self, status: int, what: str):
        self.status = status
        name = _load().dm_status_str(status).decode() if _lib is not None else str(status)
        super().__init__(f"{what}: {name}")


class ColumnIn(ctypes.Structure):
    _fields_ = [
        ("value_bytes", ctypes.c_uint32),
        ("main_dict", ctypes.c_void_p),
        ("main_dict_len", ctypes.c_uint64),
        ("main_packed", ctypes.c_void_p),
        ("main_bits", ctypes.c_uint32),
        ("main_rows", ctypes.c_uint64),
        ("delta_dict", ctypes.c_void_p),
        ("delta_dict_len", ctypes.c_uint64),
        ("delta_codes", ctypes.c_void_p),
        ("delta_rows", ctypes.c_uint64),
    ]


class Tuning(ctypes.Structure):
    _fields_ = [
        ("reencode_warps", ctypes.c_uint32),
        ("reencode_stages", ctypes.c_uint32),
        ("reencode_obufs", ctypes.c_uint32),
        ("host_chunks", ctypes.c_uint32),
        ("table_branches", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 3),
    ]


class TuneKey(ctypes.Structure):
    _fields_ = [
        ("value_bytes", ctypes.c_uint32),
        ("main_bits", ctypes.c_uint32),
        ("max_bits", ctypes.c_uint32),
        ("log2_m", ctypes.c_uint32),
        ("log2_d", ctypes.c_uint32),
        ("log2_main_rows", ctypes.c_uint32),
        ("log2_delta_rows", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32),
    ]

    def as_tuple(self):
        return tuple(getattr(self, f) for f, _ in self._fields_[:-1])


class TuneChoice(ctypes.Structure):
    _fields_ = [
        ("reencode_warps", ctypes.c_uint32),
        ("reencode_stages", ctypes.c_uint32),
        ("reencode_obufs", ctypes.c_uint32),
        ("x_staging", ctypes.c_uint32),
        ("x8", ctypes.c_uint32),
        ("step1_blocks", ctypes.c_uint32),
        ("reserved", ctypes.c_uint32 * 2),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "reserved"}


class TuneReport(ctypes.Structure):
    _fields_ = [
        ("key", TuneKey),
        ("best", TuneChoice),
        ("best_ms", ctypes.c_float),
        ("default_ms", ctypes.c_float),
        ("candidates", ctypes.c_uint32),
        ("reps", ctypes.c_uint32),
    ]


class ServerConfig(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_uint32), ("scratch_budget", ctypes.c_uint64),
                ("flags", ctypes.c_uint32)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("table_id", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("submit_ns", ctypes.c_uint64), ("admit_ns", ctypes.c_uint64),
                ("done_ns", ctypes.c_uint64), ("footprint", ctypes.c_uint64),
                ("slot", ctypes.c_uint32), ("automatic", ctypes.c_uint32),
                ("version", ctypes.c_uint64), ("delta_rows", ctypes.c_uint64),
                ("digest", ctypes.c_uint64)]


class OnlineColumn(ctypes.Structure):
    _fields_ = [("value_bytes", ctypes.c_uint32), ("main_dict", ctypes.c_void_p),
                ("main_dict_len", ctypes.c_uint64), ("main_packed", ctypes.c_void_p),
                ("main_bits", ctypes.c_uint32)]


class IngestColumn(ctypes.Structure):
    """dm_ingest_column: one column of a table ingest."""
    _fields_ = [("value_bytes", ctypes.c_uint32), ("values", ctypes.c_void_p), ("dict_out", ctypes.c_void_p),
                ("codes_out", ctypes.c_void_p), ("d_dict_len", ctypes.c_void_p)]


class OnlineConfig(ctypes.Structure):
    _fields_ = [("main_rows", ctypes.c_uint64), ("rows_capacity", ctypes.c_uint64),
                ("delta_capacity", ctypes.c_uint64), ("trigger", ctypes.c_double)]


class InsertInfo(ctypes.Structure):
    _fields_ = [("delta", ctypes.c_uint32), ("first_row", ctypes.c_uint64),
                ("lands_in", ctypes.c_uint64), ("triggered", ctypes.c_uint32),
                ("request", ctypes.c_uint64)]


class OnlineView(ctypes.Structure):
    _fields_ = [("version", ctypes.c_uint64), ("main_dict", ctypes.c_void_p),
                ("main_dict_len", ctypes.c_uint64), ("main_packed", ctypes.c_void_p),
                ("main_bits", ctypes.c_uint32), ("main_rows", ctypes.c_uint64),
                ("delta_rows", ctypes.c_uint64)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("failed", ctypes.c_uint64), ("tuples", ctypes.c_uint64),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("first_submit_ns", ctypes.c_uint64), ("last_done_ns", ctypes.c_uint64),
                ("peak_scratch_bytes", ctypes.c_uint64), ("scratch_budget", ctypes.c_uint64),
                ("peak_concurrency", ctypes.c_uint32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class ColumnOut(ctypes.Structure):
    _fields_ = [
        ("new_dict", ctypes.c_void_p),
        ("new_packed", ctypes.c_void_p),
        ("x_main", ctypes.c_void_p),
        ("x_delta", ctypes.c_void_p),
        ("d_new_dict_len", ctypes.c_void_p),
        ("d_new_bits", ctypes.c_void_p),
    ]


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libdmerge.so (raises when it is absent)."""
    return _load()


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libdmerge.so not built ({path}); run "
                               "paper_1109_6885_gb300.build.build() — there is no CPU fallback")
        lib = ctypes.CDLL(path)
        vp, u32, u64, sz, i32 = (ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_size_t,
                                 ctypes.c_int)
        pin, pout = ctypes.POINTER(ColumnIn), ctypes.POINTER(ColumnOut)
        sig = {
            "dm_create": ([ctypes.POINTER(vp), i32, sz], i32),
            "dm_destroy": ([vp], None),
            "dm_reserve": ([vp, sz], i32),
            "dm_arena_bytes": ([vp], sz),
            "dm_packed_bytes": ([u64, u32], sz),
            "dm_bits_for": ([u64], u32),
            "dm_max_bits": ([pin], u32),
            "dm_scratch_bytes": ([pin, u32], sz),
            "dm_merge_column": ([vp, pin, pout, vp, u32], i32),
            "dm_merge_table": ([vp, pin, u32, pout, vp, u32], i32),
            "dm_table_scratch_bytes": ([pin, u32, u32], sz),
            "dm_merge_column_host": ([vp, pin, pout, vp, u32, ctypes.POINTER(u64),
                                      ctypes.POINTER(u32)], i32),
            "dm_host_scratch_bytes": ([pin, u32], sz),
            "dm_sort_delta": ([vp, u32, vp, u64, vp, vp, vp], i32),
            "dm_merge_dicts": ([vp, u32, vp, u64, vp, vp, u64, vp, vp, vp, vp, vp, vp], i32),
            "dm_reencode": ([vp, vp, u32, u64, vp, u64, vp, u64, vp, u64, vp, u32, vp, vp, u32],
                            i32),
            "dm_sync_status": ([vp, vp], i32),
            "dm_last_timing": ([vp, ctypes.POINTER(ctypes.c_float)], i32),
            "dm_timing_sum": ([vp, ctypes.POINTER(ctypes.c_float), ctypes.POINTER(u32)], i32),
            "dm_launch_count": ([vp], u64),
            "dm_status_str": ([i32], ctypes.c_char_p),
            "dm_set_tuning": ([vp, ctypes.POINTER(Tuning)], i32),
            "dm_last_error": ([vp], ctypes.c_char_p),
            "dm_server_create": ([ctypes.POINTER(vp), i32, ctypes.POINTER(ServerConfig)], i32),
            "dm_server_destroy": ([vp], None),
            "dm_server_add_table": ([vp, u32, pin, u32, pout], i32),
            "dm_server_submit": ([vp, u32, ctypes.POINTER(u64)], i32),
            "dm_server_drain": ([vp, u64], i32),
            "dm_server_request_info": ([vp, u64, ctypes.POINTER(RequestInfo)], i32),
            "dm_server_stats_get": ([vp, ctypes.POINTER(ServerStats)], i32),
            "dm_server_table_version": ([vp, u32], u64),
            "dm_sched_simulate": ([u64, u32, u32, vp, vp, u64, vp, vp, vp, vp, vp,
                                   ctypes.POINTER(u64), ctypes.POINTER(u32)], i32),
            "dm_get_tuning": ([vp, ctypes.POINTER(Tuning)], i32),
            "dm_merge_dicts_noalloc": ([u32, vp, u64, vp, vp, u64, vp, vp, vp, vp, vp, vp, vp],
                                       i32),
            "dm_server_tune_cache": ([vp], vp),
            "dm_tune_key_of": ([pin, ctypes.POINTER(TuneKey)], i32),
            "dm_tune_cache_create": ([ctypes.POINTER(vp)], i32),
            "dm_tune_cache_destroy": ([vp], None),
            "dm_tune_cache_put": ([vp, ctypes.POINTER(TuneKey), ctypes.POINTER(TuneChoice)], i32),
            "dm_tune_cache_get": ([vp, ctypes.POINTER(TuneKey), ctypes.POINTER(TuneChoice)], i32),
            "dm_tune_cache_size": ([vp], u64),
            "dm_tune_cache_generation": ([vp], u64),
            "dm_tune_cache_clear": ([vp], i32),
            "dm_tune_cache_save": ([vp, ctypes.c_char_p], i32),
            "dm_tune_cache_load": ([vp, ctypes.c_char_p], i32),
            "dm_set_tune_cache": ([vp, vp], i32),
            "dm_get_tune_cache": ([vp], vp),
            "dm_tune_candidates": ([vp, pin, ctypes.POINTER(TuneChoice), u32], u32),
            "dm_autotune_column": ([vp, pin, pout, vp, u32, u32, ctypes.POINTER(TuneReport)], i32),
            "dm_reencode_search": ([vp, pin, pout, vp], i32),
            "dm_ingest_scratch_bytes": ([u32, u64], sz),
            "dm_ingest_delta": ([vp, u32, vp, u64, vp, vp, vp, vp], i32),
            "dm_ingest_table_scratch_bytes": ([vp, u32, u64], sz),
            "dm_ingest_table": ([vp, vp, u32, u64, vp], i32),
            "dm_set_wait_test": ([vp, u32, u32], i32),
            "dm_server_add_online_table": ([vp, u32, u32, ctypes.POINTER(OnlineColumn),
                                            ctypes.POINTER(OnlineConfig)], i32),
            "dm_server_insert": ([vp, u32, u64, ctypes.POINTER(vp), ctypes.POINTER(InsertInfo)], i32),
            "dm_server_pause": ([vp, u32, i32], i32),
            "dm_server_online_view": ([vp, u32, u32, ctypes.POINTER(OnlineView)], i32),
            "dm_server_online_copy": ([vp, u32, u32, vp, sz, vp, sz, ctypes.POINTER(OnlineView)], i32),
            "dm_column_digest": ([pin, pout, u32, vp, vp], i32),
            "dm_online_simulate": ([u32, u32, vp, vp, vp, vp, u64, vp, vp, vp, vp, vp, vp, u64, vp, vp,
                                    vp, vp, vp, vp, ctypes.POINTER(u64)], i32),
        }
        for name, (args, res) in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = res
        _lib = lib
        return lib


def _check(rc: int, what: str, ctx=None):
    if rc != DM_OK:
        if rc == DM_ECUDA and ctx is not None and ctx.handle:
            what = f"{what} ({_load().dm_last_error(ctx.handle).decode()})"
        raise DmError(rc, what)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data if t.size else None
    return t.data_ptr() if t.numel() else None


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


# ------------------------------------------------------------------ thin wrappers

def dm_packed_bytes(rows: int, bits: int) -> int:
    return int(_load().dm_packed_bytes(rows, bits))


def dm_bits_for(n: int) -> int:
    return int(_load().dm_bits_for(n))


def dm_max_bits(cin: ColumnIn) -> int:
    return int(_load().dm_max_bits(ctypes.byref(cin)))


def dm_scratch_bytes(cin: ColumnIn, flags: int = 0) -> int:
    return int(_load().dm_scratch_bytes(ctypes.byref(cin), flags))


def dm_host_scratch_bytes(cin: ColumnIn, flags: int = 0) -> int:
    return int(_load().dm_host_scratch_bytes(ctypes.byref(cin), flags))


def dm_table_scratch_bytes(cins, flags: int = 0) -> int:
    arr = (ColumnIn * len(cins))(*cins)
    return int(_load().dm_table_scratch_bytes(arr, len(cins), flags))


def dm_tune_key_of(cin: ColumnIn) -> TuneKey:
    k = TuneKey()
    _check(_load().dm_tune_key_of(ctypes.byref(cin), ctypes.byref(k)), "dm_tune_key_of")
    return k


class TuneCache:
    """dm_tune_cache: launch choices per column class (host memory only).

    Created with no handle it owns a new cache; given one (a context's or a
    server's) it borrows it and `owner` keeps that owner alive."""

    def __init__(self, handle=None, owner=None):
        self._owned = handle is None
        self.owner = owner
        if handle is None:
            h = ctypes.c_void_p()
            _check(_load().dm_tune_cache_create(ctypes.byref(h)), "dm_tune_cache_create")
            self.handle = h
        else:
            self.handle = ctypes.c_void_p(handle)

    def close(self):
        if self._owned and self.handle:
            _load().dm_tune_cache_destroy(self.handle)
        self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def put(self, key: TuneKey, choice: TuneChoice):
        _check(_load().dm_tune_cache_put(self.handle, ctypes.byref(key), ctypes.byref(choice)),
               "dm_tune_cache_put")

    def get(self, key: TuneKey) -> TuneChoice | None:
        c = TuneChoice()
        rc = _load().dm_tune_cache_get(self.handle, ctypes.byref(key), ctypes.byref(c))
        if rc == DM_ENOENT:
            return None
        _check(rc, "dm_tune_cache_get")
        return c

    def __len__(self) -> int:
        return int(_load().dm_tune_cache_size(self.handle))

    @property
    def generation(self) -> int:
        return int(_load().dm_tune_cache_generation(self.handle))

    def clear(self):
        _check(_load().dm_tune_cache_clear(self.handle), "dm_tune_cache_clear")

    def save(self, path: str):
        _check(_load().dm_tune_cache_save(self.handle, os.fsencode(path)), "dm_tune_cache_save")

    def load(self, path: str):
        _check(_load().dm_tune_cache_load(self.handle, os.fsencode(path)), "dm_tune_cache_load")


class Context:
    """Owns a dm_ctx (device, scratch arena, status word, tune cache)."""

    def __init__(self, device: int = 0, arena_bytes: int = 0):
        self.handle = ctypes.c_void_p()
        _check(_load().dm_create(ctypes.byref(self.handle), device, arena_bytes), "dm_create")
        self.device = device

    def close(self):
        if self.handle:
            _load().dm_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reserve(self, nbytes: int):
        _check(_load().dm_reserve(self.handle, nbytes), "dm_reserve")

    @property
    def arena_bytes(self) -> int:
        return int(_load().dm_arena_bytes(self.handle))

    @property
    def launches(self) -> int:
        return int(_load().dm_launch_count(self.handle))

    def set_tuning(self, **kw):
        """Launch parameters (reencode_warps, reencode_stages, reencode_obufs,
        host_chunks; 0 = default)."""
        t = self.get_tuning()
        names = {f[0] for f in Tuning._fields_} - {"reserved"}
        for k, v in kw.items():
            if k not in names:
                raise TypeError(f"unknown tuning field {k!r}")
            setattr(t, k, int(v))
        _check(_load().dm_set_tuning(self.handle, ctypes.byref(t)), "dm_set_tuning")

    def get_tuning(self) -> Tuning:
        t = Tuning()
        _check(_load().dm_get_tuning(self.handle, ctypes.byref(t)), "dm_get_tuning")
        return t

    @property
    def tune_cache(self) -> TuneCache:
        """The cache this context looks launch choices up in."""
        h = _load().dm_get_tune_cache(self.handle)
        if not h:
            raise DmError(DM_EINVAL, "dm_get_tune_cache")
        return TuneCache(h, owner=self)

    def set_tune_cache(self, cache: TuneCache | None):
        """Share `cache` (kept alive by this context); None: the context's own."""
        _check(_load().dm_set_tune_cache(self.handle, cache.handle if cache else None),
               "dm_set_tune_cache")
        self._shared_cache = cache

    def tune_candidates(self, cin: ColumnIn) -> list[TuneChoice]:
        n = int(_load().dm_tune_candidates(self.handle, ctypes.byref(cin), None, 0))
        arr = (TuneChoice * n)()
        _load().dm_tune_candidates(self.handle, ctypes.byref(cin), arr, n)
        return list(arr)

    def sync_status(self, stream=None) -> int:
        return int(_load().dm_sync_status(self.handle, _stream(stream)))

    def set_wait_test(self, withhold_tile: int | None, spin_limit: int = 0):
        """Testing the bounded waits: merge tile `withhold_tile` of later Step 1
        launches withholds its look-back word and waits give up after
        `spin_limit` polls; None (and 0) restores normal merges."""
        t = DM_WAIT_TEST_OFF if withhold_tile is None else int(withhold_tile)
        _check(_load().dm_set_wait_test(self.handle, t, int(spin_limit)), "dm_set_wait_test")

    def last_timing(self):
        """ms of Step 1(a), 1(b)+2(a), the X_M directory, the Step 2(b) kernel and the
        whole last timed merge."""
        ms = (ctypes.c_float * 5)()
        _check(_load().dm_last_timing(self.handle, ms), "dm_last_timing")
        return list(ms)

    def timing_sum(self):
        """(summed ms per step as in last_timing, number of timed calls); resets."""
        ms = (ctypes.c_float * 5)()
        n = ctypes.c_uint32(0)
        _check(_load().dm_timing_sum(self.handle, ms, ctypes.byref(n)), "dm_timing_sum")
        return list(ms), int(n.value)


def dm_merge_column(ctx: Context, cin: ColumnIn, cout: ColumnOut, stream=None, flags: int = 0):
    _check(_load().dm_merge_column(ctx.handle, ctypes.byref(cin), ctypes.byref(cout),
                                   _stream(stream), flags), "dm_merge_column", ctx)


def dm_autotune_column(ctx: Context, cin: ColumnIn, cout: ColumnOut, stream=None, flags: int = 0,
                       reps: int = 0) -> TuneReport:
    rep = TuneReport()
    _check(_load().dm_autotune_column(ctx.handle, ctypes.byref(cin), ctypes.byref(cout),
                                      _stream(stream), flags, reps, ctypes.byref(rep)),
           "dm_autotune_column", ctx)
    return rep


def dm_reencode_search(ctx: Context, cin: ColumnIn, cout: ColumnOut, stream=None):
    _check(_load().dm_reencode_search(ctx.handle, ctypes.byref(cin), ctypes.byref(cout), _stream(stream)),
           "dm_reencode_search", ctx)


def dm_ingest_scratch_bytes(w: int, n: int) -> int:
    return int(_load().dm_ingest_scratch_bytes(w, n))


def dm_ingest_delta(ctx: Context, w: int, values, n: int, dict_out, codes_out, d_len, stream=None):
    """Appended values -> (D_dict in order of first arrival, codes); |D_dict| to the device scalar d_len."""
    need = dm_ingest_scratch_bytes(w, n)
    if need > ctx.arena_bytes:
        ctx.reserve(need)
    _check(_load().dm_ingest_delta(ctx.handle, w, _ptr(values), n, _ptr(dict_out), _ptr(codes_out), _ptr(d_len),
                                   _stream(stream)), "dm_ingest_delta", ctx)


def dm_ingest_table(ctx: Context, cols, n: int, stream=None):
    """n rows appended to a table: cols is a list of (w, values, dict_out,
    codes_out, d_len) per column, each ingested as dm_ingest_delta does, the
    columns side by side on the context's branches."""
    arr = (IngestColumn * max(len(cols), 1))()
    for k, (w, values, dict_out, codes_out, d_len) in enumerate(cols):
        arr[k] = IngestColumn(w, _ptr(values), _ptr(dict_out), _ptr(codes_out), _ptr(d_len))
    need = int(_load().dm_ingest_table_scratch_bytes(arr, len(cols), n))
    if need > ctx.arena_bytes:
        ctx.reserve(need)
    _check(_load().dm_ingest_table(ctx.handle, arr, len(cols), n, _stream(stream)), "dm_ingest_table", ctx)


def dm_merge_table(ctx: Context, cins, couts, stream=None, flags: int = 0):
    n = len(cins)
    ain = (ColumnIn * n)(*cins)
    aout = (ColumnOut * n)(*couts)
    _check(_load().dm_merge_table(ctx.handle, ain, n, aout, _stream(stream), flags),
           "dm_merge_table", ctx)


def dm_merge_column_host(ctx: Context, cin: ColumnIn, cout: ColumnOut, stream=None,
                         flags: int = 0):
    u = ctypes.c_uint64(0)
    b = ctypes.c_uint32(0)
    _check(_load().dm_merge_column_host(ctx.handle, ctypes.byref(cin), ctypes.byref(cout),
                                        _stream(stream), flags, ctypes.byref(u), ctypes.byref(b)),
           "dm_merge_column_host")
    return int(u.value), int(b.value)


def dm_sort_delta(ctx: Context, w: int, delta_dict, d: int, ud_out, perm_out, stream=None):
    _check(_load().dm_sort_delta(ctx.handle, w, _ptr(delta_dict), d, _ptr(ud_out), _ptr(perm_out),
                                 _stream(stream)), "dm_sort_delta")


def dm_merge_dicts(ctx: Context, w: int, main_dict, m: int, ud, perm, d: int, new_dict, x_main,
                   x_delta, d_u, d_bits, stream=None):
    _check(_load().dm_merge_dicts(ctx.handle, w, _ptr(main_dict), m, _ptr(ud), _ptr(perm), d,
                                  _ptr(new_dict), _ptr(x_main), _ptr(x_delta), _ptr(d_u),
                                  _ptr(d_bits), _stream(stream)), "dm_merge_dicts")


def dm_merge_dicts_noalloc(w: int, main_dict, m: int, ud, perm, d: int, new_dict, x_main,
                           x_delta, d_u, d_bits, d_status=None, stream=None):
    """Step 1(b) + 2(a) with scratch in the library's static device memory
    (no context, no allocation); m + d <= DM_NOALLOC_MAX_ENTRIES."""
    _check(_load().dm_merge_dicts_noalloc(w, _ptr(main_dict), m, _ptr(ud), _ptr(perm), d,
                                          _ptr(new_dict), _ptr(x_main), _ptr(x_delta), _ptr(d_u),
                                          _ptr(d_bits), _ptr(d_status), _stream(stream)),
           "dm_merge_dicts_noalloc")


DM_NOALLOC_MAX_ENTRIES = 1 << 24


def dm_reencode(ctx: Context, main_packed, main_bits: int, n_main: int, delta_codes, n_delta: int,
                x_main, m: int, x_delta, d: int, d_bits, max_bits: int, out_packed, stream=None,
                flags: int = 0):
    _check(_load().dm_reencode(ctx.handle, _ptr(main_packed), main_bits, n_main, _ptr(delta_codes),
                               n_delta, _ptr(x_main), m, _ptr(x_delta), d, _ptr(d_bits), max_bits,
                               _ptr(out_packed), _stream(stream), flags), "dm_reencode")


# ------------------------------------------------------------------ tensor helpers

_SIGNED = {np.dtype(np.uint32): np.int32, np.dtype(np.uint64): np.int64}


def to_device(a: np.ndarray, device="cuda"):
    """numpy (unsigned) array -> torch tensor on the device (same bytes)."""
    import torch
    a = np.ascontiguousarray(a)
    sa = a.view(_SIGNED.get(a.dtype, a.dtype))
    if sa.size == 0:
        return torch.empty(sa.shape, dtype=torch.from_numpy(sa[:0].copy()).dtype, device=device)
    return torch.from_numpy(sa).to(device)


def to_host(t, dtype) -> np.ndarray:
    """torch tensor -> numpy array reinterpreted as `dtype` (unsigned)."""
    return t.detach().cpu().numpy().view(dtype)


def key_tensor_empty(n: int, w: int, device="cuda"):
    import torch
    if w == 4:
        return torch.empty(n, dtype=torch.int32, device=device)
    if w == 8:
        return torch.empty(n, dtype=torch.int64, device=device)
    return torch.empty((n, 2), dtype=torch.int64, device=device)


def key_np_dtype(w: int):
    return np.uint32 if w == 4 else np.uint64


@dataclasses.dataclass
class DeviceColumn:
    """A column's inputs resident in device memory (torch tensors)."""
    w: int
    main_dict: object
    m: int
    main_packed: object
    main_bits: int
    n_main: int
    delta_dict: object
    d: int
    delta_codes: object
    n_delta: int

    def cin(self) -> ColumnIn:
        return ColumnIn(self.w, _ptr(self.main_dict), self.m, _ptr(self.main_packed),
                        self.main_bits, self.n_main, _ptr(self.delta_dict), self.d,
                        _ptr(self.delta_codes), self.n_delta)

    @staticmethod
    def from_numpy(w, main_dict, main_packed, main_bits, n_main, delta_dict, delta_codes,
                   device="cuda"):
        return DeviceColumn(w, to_device(main_dict, device), int(main_dict.shape[0]),
                            to_device(main_packed, device), int(main_bits), int(n_main),
                            to_device(delta_dict, device), int(delta_dict.shape[0]),
                            to_device(delta_codes, device), int(delta_codes.size))


@dataclasses.dataclass
class DeviceResult:
    """Output buffers of one column merge (torch tensors, device)."""
    new_dict: object
    new_packed: object
    x_main: object
    x_delta: object
    scalars: object       # int64[2]: |U'| then E'_C (low 32 bits)

    def cout(self) -> ColumnOut:
        base = self.scalars.data_ptr()
        return ColumnOut(_ptr(self.new_dict), _ptr(self.new_packed), _ptr(self.x_main),
                         _ptr(self.x_delta), base, base + 8)

    def u_bits(self):
        s = self.scalars.cpu().numpy()
        return int(s[0]), int(s[1] & 0xFFFFFFFF)


def alloc_result(col: DeviceColumn, device="cuda", with_x: bool = True) -> DeviceResult:
    import torch
    maxb = dm_bits_for(col.m + col.d)
    nbytes = dm_packed_bytes(col.n_main + col.n_delta, maxb)
    return DeviceResult(
        key_tensor_empty(col.m + col.d, col.w, device),
        torch.empty(max(nbytes // 4, 0), dtype=torch.int32, device=device),
        torch.empty(col.m, dtype=torch.int32, device=device) if with_x else None,
        torch.empty(col.d, dtype=torch.int32, device=device) if with_x else None,
        torch.zeros(2, dtype=torch.int64, device=device),
    )


def merge_column(ctx: Context, col: DeviceColumn, res: DeviceResult | None = None, stream=None,
                 flags: int = 0) -> DeviceResult:
    """dm_merge_column on a DeviceColumn; grows the arena when needed."""
    cin = col.cin()
    need = dm_scratch_bytes(cin, flags)
    if need > ctx.arena_bytes:
        ctx.reserve(need)
    if res is None:
        res = alloc_result(col)
    dm_merge_column(ctx, cin, res.cout(), stream, flags)
    return res


def fetch(res: DeviceResult, w: int, n_out: int):
    """Copy a merge result back: (U', X_M, X_D, packed words, E'_C, |U'|)."""
    u, b = res.u_bits()
    kd = key_np_dtype(w)
    new_dict = to_host(res.new_dict[:u], kd)
    nwords = dm_packed_bytes(n_out, b) // 4
    packed = to_host(res.new_packed[:nwords], np.uint32)
    xm = to_host(res.x_main, np.uint32) if res.x_main is not None else None
    xd = to_host(res.x_delta, np.uint32) if res.x_delta is not None else None
    return new_dict, xm, xd, packed, b, u


def dm_column_digest(cin: ColumnIn, cout: ColumnOut, col_index: int, d_digest, stream=None):
    """Add the checksum of a merged column's outputs to the device word d_digest."""
    _check(_load().dm_column_digest(ctypes.byref(cin), ctypes.byref(cout), col_index, _ptr(d_digest),
                                    _stream(stream)), "dm_column_digest")


def column_digests(cins, couts, stream=None):
    """One checksum per column (host ints), from dm_column_digest."""
    import torch
    acc = torch.zeros(max(len(cins), 1), dtype=torch.int64, device="cuda")
    for j, (ci, co) in enumerate(zip(cins, couts)):
        dm_column_digest(ci, co, j, acc[j:j + 1], stream)
    return [int(x) & (2**64 - 1) for x in acc[:len(cins)].cpu().tolist()]


# ------------------------------------------------------------------ served merges

class Server:
    """dm_server: resident tables, merge requests admitted with continuous batching."""

    def __init__(self, device: int = 0, slots: int = 4, scratch_budget: int = 1 << 30,
                 flags: int = 0):
        self.handle = ctypes.c_void_p()
        cfg = ServerConfig(slots, scratch_budget, flags)
        _check(_load().dm_server_create(ctypes.byref(self.handle), device, ctypes.byref(cfg)),
               "dm_server_create")

    def close(self):
        if self.handle:
            _load().dm_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_table(self, table_id: int, cins, couts):
        n = len(cins)
        _check(_load().dm_server_add_table(self.handle, table_id, (ColumnIn * n)(*cins), n,
                                           (ColumnOut * n)(*couts)), "dm_server_add_table")

    def submit(self, table_id: int) -> int:
        rid = ctypes.c_uint64(0)
        _check(_load().dm_server_submit(self.handle, table_id, ctypes.byref(rid)),
               "dm_server_submit")
        return int(rid.value)

    def drain(self, timeout_ms: int = 600_000):
        _check(_load().dm_server_drain(self.handle, timeout_ms), "dm_server_drain")

    def info(self, request_id: int) -> RequestInfo:
        r = RequestInfo()
        _check(_load().dm_server_request_info(self.handle, request_id, ctypes.byref(r)),
               "dm_server_request_info")
        return r

    def stats(self) -> ServerStats:
        st = ServerStats()
        _check(_load().dm_server_stats_get(self.handle, ctypes.byref(st)), "dm_server_stats_get")
        return st

    def version(self, table_id: int) -> int:
        return int(_load().dm_server_table_version(self.handle, table_id))

    def add_online_table(self, table_id: int, cols, main_rows: int, rows_capacity: int,
                         delta_capacity: int, trigger: float = 0.0):
        """Register a server-owned online table; cols: OnlineColumn structures."""
        n = len(cols)
        cfg = OnlineConfig(main_rows, rows_capacity, delta_capacity, float(trigger))
        _check(_load().dm_server_add_online_table(self.handle, table_id, n, (OnlineColumn * n)(*cols),
                                                  ctypes.byref(cfg)), "dm_server_add_online_table")

    def insert(self, table_id: int, nrows: int, values) -> InsertInfo:
        """Append nrows rows; values: one tensor (device) or array per column."""
        ptrs = (ctypes.c_void_p * max(len(values), 1))(*[_ptr(v) for v in values])
        info = InsertInfo()
        _check(_load().dm_server_insert(self.handle, table_id, nrows, ptrs, ctypes.byref(info)),
               "dm_server_insert")
        return info

    def pause(self, table_id: int, paused: bool = True):
        _check(_load().dm_server_pause(self.handle, table_id, 1 if paused else 0), "dm_server_pause")

    def resume(self, table_id: int):
        self.pause(table_id, False)

    def online_view(self, table_id: int, col: int) -> OnlineView:
        v = OnlineView()
        _check(_load().dm_server_online_view(self.handle, table_id, col, ctypes.byref(v)),
               "dm_server_online_view")
        return v

    def online_copy(self, table_id: int, col: int, w: int):
        """The committed version of a column, copied to host memory:
        (version, U_M keys, packed words, E_C, N_M)."""
        v = self.online_view(table_id, col)
        for _ in range(8):
            kd = key_np_dtype(w)
            keys = np.zeros((v.main_dict_len, 2) if w == 16 else v.main_dict_len, kd)
            words = np.zeros(dm_packed_bytes(v.main_rows, 32) // 4 + 4, np.uint32)
            got = OnlineView()
            rc = _load().dm_server_online_copy(self.handle, table_id, col, _ptr(keys), keys.nbytes,
                                               _ptr(words), words.nbytes, ctypes.byref(got))
            if rc == DM_OK and got.main_dict_len == v.main_dict_len:
                nw = dm_packed_bytes(got.main_rows, got.main_bits) // 4
                return int(got.version), keys, words[:nw].copy(), int(got.main_bits), int(got.main_rows)
            if rc not in (DM_OK, DM_EINVAL):
                _check(rc, "dm_server_online_copy")
            v = self.online_view(table_id, col)   # a commit came in between: size again
        raise DmError(DM_EBUSY, "dm_server_online_copy")

    @property
    def tune_cache(self) -> TuneCache:
        """The cache every slot looks its launch choices up in."""
        h = _load().dm_server_tune_cache(self.handle)
        if not h:
            raise DmError(DM_EINVAL, "dm_server_tune_cache")
        return TuneCache(h, owner=self)


def dm_sched_simulate(pool_bytes: int, slots: int, footprint, service_ns, req_table, arrival_ns):
    """The server's admission rules on a fake clock (no GPU): returns
    (admit_ns, done_ns, slot, peak_bytes, peak_running)."""
    fp = np.ascontiguousarray(footprint, np.uint64)
    sv = np.ascontiguousarray(service_ns, np.uint64)
    rt = np.ascontiguousarray(req_table, np.uint32)
    ar = np.ascontiguousarray(arrival_ns, np.uint64)
    n = rt.size
    admit = np.zeros(n, np.uint64)
    done = np.zeros(n, np.uint64)
    slot = np.zeros(n, np.uint32)
    pb = ctypes.c_uint64(0)
    pr = ctypes.c_uint32(0)
    _check(_load().dm_sched_simulate(pool_bytes, slots, fp.size, _ptr(fp), _ptr(sv), n, _ptr(rt),
                                     _ptr(ar), _ptr(admit), _ptr(done), _ptr(slot),
                                     ctypes.byref(pb), ctypes.byref(pr)), "dm_sched_simulate")
    return admit, done, slot, int(pb.value), int(pr.value)


def dm_online_simulate(slots: int, main_rows, delta_capacity, trigger, service_ns, ev_kind, ev_table,
                       ev_rows, ev_ns, max_merges: int = 4096):
    """The online-table rules on a fake clock (no GPU).  Events: kind 0 insert
    (ev_rows rows), 1 merge request, 2 pause, 3 resume.  Returns a dict with,
    per event, 'lands_in' (the version an insert was told) and 'version' (the
    version whose merge took it), and per merge in admission order 'table',
    'admit_ns', 'done_ns', 'rows', 'version', 'automatic'."""
    mr = np.ascontiguousarray(main_rows, np.uint64)
    dc = np.ascontiguousarray(delta_capacity, np.uint64)
    tg = np.ascontiguousarray(trigger, np.float64)
    sv = np.ascontiguousarray(service_ns, np.uint64)
    ek = np.ascontiguousarray(ev_kind, np.uint32)
    et = np.ascontiguousarray(ev_table, np.uint32)
    er = np.ascontiguousarray(ev_rows, np.uint64)
    en = np.ascontiguousarray(ev_ns, np.uint64)
    n = ek.size
    lands = np.zeros(max(n, 1), np.uint64)
    ver = np.zeros(max(n, 1), np.uint64)
    mt = np.zeros(max_merges, np.uint32)
    ma = np.zeros(max_merges, np.uint64)
    md = np.zeros(max_merges, np.uint64)
    mrw = np.zeros(max_merges, np.uint64)
    mv = np.zeros(max_merges, np.uint64)
    mau = np.zeros(max_merges, np.uint32)
    nm = ctypes.c_uint64(0)
    _check(_load().dm_online_simulate(slots, mr.size, _ptr(mr), _ptr(dc), _ptr(tg), _ptr(sv), n, _ptr(ek),
                                      _ptr(et), _ptr(er), _ptr(en), _ptr(lands), _ptr(ver), max_merges,
                                      _ptr(mt), _ptr(ma), _ptr(md), _ptr(mrw), _ptr(mv), _ptr(mau),
                                      ctypes.byref(nm)), "dm_online_simulate")
    k = min(int(nm.value), max_merges)
    return {"lands_in": lands[:n], "version": ver[:n], "table": mt[:k], "admit_ns": ma[:k],
            "done_ns": md[:k], "rows": mrw[:k], "version_of_merge": mv[:k], "automatic": mau[:k],
            "merges": int(nm.value)}
