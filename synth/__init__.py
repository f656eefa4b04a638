"""Seeded synthetic inputs for the delta-to-main merge.

Builds the inputs of one column merge (Section 5: main dictionary U_M, the
bit-packed main vector M, the delta partition D) with the shapes of the
paper's experiments (Section 7: uniform random values, value lengths 4-16
bytes, unique fractions 0.1%-100%).  Nothing here performs a merge step;
the CUDA library and the CPU oracle both consume these arrays.

The heavy loops run in the small C library ``dmgen.c`` next to this file,
compiled on first use (or by ``build_native``).
"""
from __future__ import annotations

import ctypes
import dataclasses
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dmgen.c")
_LIB_PATH = os.path.join(_HERE, "libdmgen.so")
_lock = threading.Lock()
_lib = None

KEY_DTYPE = {4: np.uint32, 8: np.uint64, 16: np.uint64}


def build_native(force: bool = False) -> str:
    """Compile dmgen.c into libdmgen.so beside it (plain C, no GPU)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC,
                           "-lpthread", "-lm"])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build_native())
        u64, u32, i32, dbl, vp = (ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_void_p)
        lib.synth_subseed.argtypes = [u64, u64]
        lib.synth_subseed.restype = u64
        lib.synth_dict.argtypes = [u64, u32, u64, vp]
        lib.synth_dict.restype = i32
        lib.synth_codes.argtypes = [u64, u64, u64, i32, dbl, vp, i32]
        lib.synth_codes.restype = i32
        lib.synth_packed_words.argtypes = [u64, u32]
        lib.synth_packed_words.restype = u64
        lib.synth_pack.argtypes = [vp, u64, u32, vp, i32]
        lib.synth_pack.restype = i32
        lib.synth_delta.argtypes = [u64, u64, u32, vp, u64, u64, dbl, u64, i32, dbl, vp,
                                    ctypes.POINTER(u64), vp]
        lib.synth_delta.restype = i32
        _lib = lib
        return lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data if a.size else 0


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def bits_for(n: int) -> int:
    """Smallest b with 2**b >= n (0 for n <= 1): the width of codes 0..n-1."""
    return 0 if n <= 1 else int(n - 1).bit_length()


def subseed(seed: int, tag: int) -> int:
    return int(_load().synth_subseed(seed & (2**64 - 1), tag & (2**64 - 1)))


def key_array(n: int, w: int) -> np.ndarray:
    """Empty key array: (n,) uint32 / uint64, or (n, 2) uint64 as (hi, lo)."""
    if w == 16:
        return np.zeros((n, 2), dtype=np.uint64)
    return np.zeros(n, dtype=KEY_DTYPE[w])


def dictionary(seed: int, w: int, m: int) -> np.ndarray:
    """m sorted distinct keys of width w bytes (stratified uniform)."""
    out = key_array(m, w)
    rc = _load().synth_dict(seed, w, m, _ptr(out))
    if rc != 0:
        raise ValueError(f"cannot draw {m} distinct {w}-byte keys")
    return out


def codes(seed: int, m: int, n: int, dist: str = "uniform", s: float = 1.0) -> np.ndarray:
    """n codes over a dictionary of m entries, uniform or Zipf(s) over ranks."""
    out = np.zeros(n, dtype=np.uint32)
    if n == 0:
        return out
    rc = _load().synth_codes(seed, m, n, 1 if dist == "zipf" else 0, float(s), _ptr(out),
                             _threads())
    if rc != 0:
        raise ValueError("code generation failed")
    return out


def packed_words(n: int, b: int) -> int:
    """32-bit words in an LSB-first stream of n codes at b bits, padded to 16 bytes."""
    return ((n * b + 127) // 128) * 4


def pack(codes_: np.ndarray, b: int) -> np.ndarray:
    """Pack uint32 codes LSB-first at b bits into little-endian 32-bit words."""
    codes_ = np.ascontiguousarray(codes_, dtype=np.uint32)
    out = np.zeros(packed_words(codes_.size, b), dtype=np.uint32)
    rc = _load().synth_pack(_ptr(codes_), codes_.size, b, _ptr(out), _threads())
    if rc != 0:
        raise ValueError("bad width")
    return out


def delta(seed: int, code_seed: int, w: int, main_dict: np.ndarray, n_delta: int, f_new: float,
          pool: int, dist: str = "uniform", s: float = 1.0):
    """Delta partition: (insertion-order dictionary, uint32 row codes)."""
    m = main_dict.shape[0]
    ddict = key_array(n_delta, w)
    dcodes = np.zeros(n_delta, dtype=np.uint32)
    d = ctypes.c_uint64(0)
    main_dict = np.ascontiguousarray(main_dict)
    rc = _load().synth_delta(seed, code_seed, w, _ptr(main_dict), m, n_delta, float(f_new),
                             int(pool), 1 if dist == "zipf" else 0, float(s), _ptr(ddict),
                             ctypes.byref(d), _ptr(dcodes))
    if rc != 0:
        raise ValueError(f"delta generation failed ({rc})")
    return ddict[: d.value].copy(), dcodes


@dataclasses.dataclass
class ColumnSpec:
    """Shape of one column merge input (symbols as in the paper's Table 1).

    n_main  N_M, main rows        m      |U_M|, main dictionary entries
    w       E, value bytes         b      E_C, main code width (None: minimal)
    n_delta N_D, delta rows        f_new  fraction of delta rows carrying new values
    pool    number of distinct new values (None: max(1, round(m/N_M * f_new * N_D));
            0: every fresh row its own new value)
    """
    n_main: int
    m: int
    w: int = 8
    n_delta: int = 0
    f_new: float = 0.3
    dist: str = "uniform"
    zipf_s: float = 1.0
    pool: int | None = None
    b: int | None = None
    seed: int = 0x11096885

    def pool_size(self) -> int:
        if self.pool is not None:
            return self.pool
        lam = self.m / self.n_main if self.n_main else 1.0
        return max(1, round(lam * self.f_new * self.n_delta))


@dataclasses.dataclass
class Column:
    spec: ColumnSpec
    main_dict: np.ndarray      # U_M, sorted, distinct
    main_codes: np.ndarray     # uint32 codes (unpacked, for checks)
    main_bits: int             # E_C
    main_packed: np.ndarray    # uint32 words, LSB-first stream
    delta_dict: np.ndarray     # insertion-order distinct delta values
    delta_codes: np.ndarray    # uint32 row codes into delta_dict

    @property
    def w(self) -> int:
        return self.spec.w

    @property
    def n_main(self) -> int:
        return int(self.main_codes.size)

    @property
    def n_delta(self) -> int:
        return int(self.delta_codes.size)


def make_column(spec: ColumnSpec) -> Column:
    s_dict = subseed(spec.seed, 1)
    s_codes = subseed(spec.seed, 2)
    s_delta = subseed(spec.seed, 3)
    main_dict = dictionary(s_dict, spec.w, spec.m)
    b = bits_for(spec.m) if spec.b is None else spec.b
    if spec.n_main and spec.m == 0:
        raise ValueError("main rows need a non-empty dictionary")
    mc = codes(s_codes, spec.m, spec.n_main, spec.dist, spec.zipf_s) if spec.n_main else \
        np.zeros(0, np.uint32)
    ddict, dcodes = delta(s_delta, s_codes, spec.w, main_dict, spec.n_delta, spec.f_new,
                          spec.pool_size(), spec.dist, spec.zipf_s)
    return Column(spec, main_dict, mc, b, pack(mc, b), ddict, dcodes)


def column_seed(config: int, column: int) -> int:
    """Seed of column `column` of workload `config`."""
    return subseed(0x11096885 ^ (config << 32), column)
