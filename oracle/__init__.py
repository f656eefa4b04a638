"""TEST INFRASTRUCTURE: Python face of the CPU oracle (dmerge_oracle.cpp).

The oracle is the plain single-threaded statement of the per-column merge of
Section 5 of the paper (Steps 1(a), 1(b), 2(a), 2(b) with the Section 5.3
translation tables, plus the Section 5.2 binary-search route as a second
path).  Only tests, the smoke check and the benchmark's CPU-baseline leg may
import this module; the CUDA library never does, and the two share no code.

Functions take and return numpy arrays.  Keys: (n,) uint32 for 4-byte
values, (n,) uint64 for 8-byte values, (n, 2) uint64 rows (hi, lo) for
16-byte values.  Packed vectors are uint32 word arrays (LSB-first stream).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmerge_oracle.cpp")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, BAD_ARG, UNSORTED, BAD_CODE = 0, 1, 2, 3


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with code {code}")
        self.code = code


def build_native(force: bool = False) -> str:
    """Compile the oracle with g++ (-O2, single thread, no GPU)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_native())
        u64, u32, i32, vp = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_void_p
        pu64, pu32 = ctypes.POINTER(u64), ctypes.POINTER(u32)
        lib.oracle_packed_words.argtypes = [u64, u32]
        lib.oracle_packed_words.restype = u64
        lib.oracle_new_width.argtypes = [u64]
        lib.oracle_new_width.restype = u32
        lib.oracle_sort_delta.argtypes = [u32, vp, u64, vp, vp]
        lib.oracle_sort_delta.restype = i32
        lib.oracle_merge_dicts.argtypes = [u32, vp, u64, vp, vp, u64, vp, vp, vp, pu64]
        lib.oracle_merge_dicts.restype = i32
        lib.oracle_reencode.argtypes = [vp, u32, u64, vp, u64, vp, u64, vp, u64, u32, vp]
        lib.oracle_reencode.restype = i32
        lib.oracle_validate.argtypes = [u32, vp, u64, vp, u32, u64, u64, vp, u64]
        lib.oracle_validate.restype = i32
        lib.oracle_merge_column.argtypes = [u32, vp, u64, vp, u32, u64, vp, u64, vp, u64, vp, vp,
                                            vp, vp, pu64, pu32]
        lib.oracle_merge_column.restype = i32
        lib.oracle_naive_reencode.argtypes = [u32, vp, u64, vp, u32, u64, vp, u64, vp, u64, vp, u64,
                                              u32, vp]
        lib.oracle_naive_reencode.restype = i32
        lib.oracle_ingest_delta.argtypes = [u32, vp, u64, vp, vp, pu64]
        lib.oracle_ingest_delta.restype = i32
        _lib = lib
        return lib


def _p(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _keys(a: np.ndarray, w: int) -> np.ndarray:
    dt = np.uint32 if w == 4 else np.uint64
    a = np.ascontiguousarray(a, dtype=dt)
    if w == 16 and (a.ndim != 2 or a.shape[1] != 2):
        raise ValueError("16-byte keys are (n, 2) uint64 rows (hi, lo)")
    return a


def _empty_keys(n: int, w: int) -> np.ndarray:
    if w == 16:
        return np.zeros((n, 2), np.uint64)
    return np.zeros(n, np.uint32 if w == 4 else np.uint64)


def packed_words(n: int, b: int) -> int:
    return int(_load().oracle_packed_words(n, b))


def new_width(u: int) -> int:
    """Step 2(a), Eq. 4."""
    return int(_load().oracle_new_width(u))


def ingest_delta(w: int, values: np.ndarray):
    """Delta ingest (Section 4): (D_dict in order of first arrival, one code per tuple)."""
    v = _keys(values, w)
    n = v.shape[0]
    dd = _empty_keys(n, w)
    codes = np.zeros(n, np.uint32)
    d = ctypes.c_uint64(0)
    rc = _load().oracle_ingest_delta(w, _p(v), n, _p(dd), _p(codes), ctypes.byref(d))
    if rc:
        raise OracleError(rc, "ingest_delta")
    return dd[:d.value], codes


def sort_delta(w: int, delta_dict: np.ndarray):
    """Step 1(a): (U_D, perm) with perm[j] the insertion code of U_D[j]."""
    dd = _keys(delta_dict, w)
    d = dd.shape[0]
    ud = _empty_keys(d, w)
    perm = np.zeros(d, np.uint32)
    rc = _load().oracle_sort_delta(w, _p(dd), d, _p(ud), _p(perm))
    if rc:
        raise OracleError(rc, "sort_delta")
    return ud, perm


def merge_dicts(w: int, main_dict: np.ndarray, ud: np.ndarray, perm: np.ndarray):
    """Step 1(b): (U', X_M, X_D) with X_D indexed by insertion code."""
    um = _keys(main_dict, w)
    ud = _keys(ud, w)
    perm = np.ascontiguousarray(perm, np.uint32)
    m, d = um.shape[0], ud.shape[0]
    unew = _empty_keys(m + d, w)
    xm = np.zeros(m, np.uint32)
    xd = np.zeros(d, np.uint32)
    u = ctypes.c_uint64(0)
    rc = _load().oracle_merge_dicts(w, _p(um), m, _p(ud), _p(perm), d, _p(unew), _p(xm), _p(xd),
                                    ctypes.byref(u))
    if rc:
        raise OracleError(rc, "merge_dicts")
    return unew[: u.value].copy(), xm, xd


def reencode(main_packed: np.ndarray, b: int, n_main: int, delta_codes: np.ndarray,
             xm: np.ndarray, xd: np.ndarray, b_new: int) -> np.ndarray:
    """Step 2(b), Eq. 11: the new packed vector of N_M + N_D codes at b_new bits."""
    mw = np.ascontiguousarray(main_packed, np.uint32)
    dc = np.ascontiguousarray(delta_codes, np.uint32)
    xm = np.ascontiguousarray(xm, np.uint32)
    xd = np.ascontiguousarray(xd, np.uint32)
    out = np.zeros(packed_words(n_main + dc.size, b_new), np.uint32)
    rc = _load().oracle_reencode(_p(mw), b, n_main, _p(dc), dc.size, _p(xm), xm.size, _p(xd),
                                 xd.size, b_new, _p(out))
    if rc:
        raise OracleError(rc, "reencode")
    return out


def validate(w, main_dict, main_packed, b, n_main, d, delta_codes) -> int:
    um = _keys(main_dict, w)
    mw = np.ascontiguousarray(main_packed, np.uint32)
    dc = np.ascontiguousarray(delta_codes, np.uint32)
    return int(_load().oracle_validate(w, _p(um), um.shape[0], _p(mw), b, n_main, d, _p(dc),
                                       dc.size))


@dataclasses.dataclass
class MergeResult:
    new_dict: np.ndarray     # U'
    x_main: np.ndarray       # X_M
    x_delta: np.ndarray      # X_D (by insertion code)
    new_packed: np.ndarray   # M' (uint32 words)
    new_bits: int            # E'_C
    u: int                   # |U'|


def merge_column(w: int, main_dict, main_packed, b: int, n_main: int, delta_dict,
                 delta_codes) -> MergeResult:
    """All of Section 5 for one column; raises OracleError on invalid input."""
    um = _keys(main_dict, w)
    dd = _keys(delta_dict, w)
    mw = np.ascontiguousarray(main_packed, np.uint32)
    dc = np.ascontiguousarray(delta_codes, np.uint32)
    m, d = um.shape[0], dd.shape[0]
    unew = _empty_keys(m + d, w)
    xm = np.zeros(m, np.uint32)
    xd = np.zeros(d, np.uint32)
    out = np.zeros(packed_words(n_main + dc.size, new_width(m + d)), np.uint32)
    u = ctypes.c_uint64(0)
    bn = ctypes.c_uint32(0)
    rc = _load().oracle_merge_column(w, _p(um), m, _p(mw), b, n_main, _p(dd), d, _p(dc), dc.size,
                                     _p(unew), _p(xm), _p(xd), _p(out), ctypes.byref(u),
                                     ctypes.byref(bn))
    if rc:
        raise OracleError(rc, "merge_column")
    nw = packed_words(n_main + dc.size, bn.value)
    return MergeResult(unew[: u.value].copy(), xm, xd, out[:nw].copy(), int(bn.value),
                       int(u.value))


def naive_reencode(w, main_dict, main_packed, b, n_main, delta_dict, delta_codes, new_dict,
                   b_new) -> np.ndarray:
    """Step 2(b) by the Section 5.2 route (decode, then binary search in U')."""
    um = _keys(main_dict, w)
    dd = _keys(delta_dict, w)
    un = _keys(new_dict, w)
    mw = np.ascontiguousarray(main_packed, np.uint32)
    dc = np.ascontiguousarray(delta_codes, np.uint32)
    out = np.zeros(packed_words(n_main + dc.size, b_new), np.uint32)
    rc = _load().oracle_naive_reencode(w, _p(um), um.shape[0], _p(mw), b, n_main, _p(dd),
                                       dd.shape[0], _p(dc), dc.size, _p(un), un.shape[0], b_new,
                                       _p(out))
    if rc:
        raise OracleError(rc, "naive_reencode")
    return out


def merge_synth_column(col) -> MergeResult:
    """Oracle merge of a synth.Column."""
    return merge_column(col.w, col.main_dict, col.main_packed, col.main_bits, col.n_main,
                        col.delta_dict, col.delta_codes)
