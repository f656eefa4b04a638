"""Brute-force statements of the merge's result, for tiny inputs.

Written from the definitions alone, sharing nothing with the oracle's code:
the packed format is read and written one bit at a time; the merged
dictionary is the sorted Python set of Eq. 3 (union of the two
dictionaries); every new code is the position of the row's value in it
(Section 5.2: "the index of the corresponding uncompressed value in the new
dictionary"); the width is Eq. 4 written as a bit length.
"""
from __future__ import annotations

import numpy as np


def key_list(arr: np.ndarray, w: int) -> list:
    """Keys as Python ints (16-byte keys as hi * 2**64 + lo, i.e. hi first)."""
    if w == 16:
        return [int(h) << 64 | int(l) for h, l in np.asarray(arr).reshape(-1, 2)]
    return [int(v) for v in np.asarray(arr).reshape(-1)]


def key_array(values: list, w: int) -> np.ndarray:
    if w == 16:
        out = np.zeros((len(values), 2), np.uint64)
        for i, v in enumerate(values):
            out[i, 0] = v >> 64
            out[i, 1] = v & (2**64 - 1)
        return out
    return np.array(values, dtype=np.uint32 if w == 4 else np.uint64)


def width(n: int) -> int:
    """Eq. 4 as a bit length: codes 0..n-1 need (n-1).bit_length() bits."""
    return max(0, (n - 1)).bit_length() if n > 0 else 0


def unpack_bits(words: np.ndarray, n: int, b: int) -> list:
    """Code i is stream bits i*b .. i*b+b-1, stream bit k = bit k%32 of word k//32."""
    ws = [int(x) for x in np.asarray(words, np.uint32)]
    out = []
    for i in range(n):
        c = 0
        for t in range(b):
            k = i * b + t
            c |= ((ws[k // 32] >> (k % 32)) & 1) << t
        out.append(c)
    return out


def pack_bits(codes: list, b: int) -> np.ndarray:
    nbits = len(codes) * b
    nwords = ((nbits + 127) // 128) * 4
    ws = [0] * nwords
    for i, c in enumerate(codes):
        for t in range(b):
            if (c >> t) & 1:
                k = i * b + t
                ws[k // 32] |= 1 << (k % 32)
    return np.array(ws, dtype=np.uint32)


def merge(w: int, main_dict, main_codes: list, delta_dict, delta_codes: list):
    """(U', X_M, X_D, new codes, b', packed words) by set + index lookup."""
    um = key_list(main_dict, w)
    dd = key_list(delta_dict, w)
    new = sorted(set(um) | set(dd))
    pos = {v: k for k, v in enumerate(new)}
    xm = [pos[v] for v in um]
    xd = [pos[v] for v in dd]
    codes = [pos[um[c]] for c in main_codes] + [pos[dd[c]] for c in delta_codes]
    bn = width(len(new))
    return new, xm, xd, codes, bn, pack_bits(codes, bn)
