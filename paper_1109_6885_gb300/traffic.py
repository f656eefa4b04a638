"""Memory-traffic arithmetic of the merge.

Two parts:

* the paper's CPU traffic model, Section 6.1 (Eq. 8-14), the parallel
  overhead of Section 6.2.1 (Eq. 15), the update-rate formulas (Eq. 1 and
  the worked Eq. 16) and the projections of Section 7.4 (Eq. 17, Eq. 18 and
  the 6.6 / 14.2 cycles-per-tuple figures).  These are quoted as context and
  pinned by tests against the numbers the paper prints.
* the algorithmic bytes of the GPU path, the numerator of every roofline
  fraction this project reports: the bytes a perfect implementation must
  move (each input read once, each output written once), without the
  write-allocate read the CPU model counts in Eq. 14.

Symbols follow the paper's Table 1: E value bytes, N_M / N_D rows,
E_C / E'_C code widths in bits, L the cache-line size.
"""
from __future__ import annotations


# ------------------------------------------------------------------ paper model

def eq1_update_rate(n_delta: float, t_update_s: float, t_merge_s: float) -> float:
    """Eq. 1: updates per second = N_D / (T_U + T_M)."""
    return n_delta / (t_update_s + t_merge_s)


def eq8_step1a_bytes(E: float, UD: float, ND: float, L: float = 64) -> float:
    """Eq. 8: tree traversal (3E read + E written per value) and tuple rewrite."""
    return 4 * E * UD + (2 * L + 4) * ND


def eq9_step1b_read_bytes(E, UM, UD, Unew, ECnew, XM, XD, include_unew: bool = True) -> float:
    """Eq. 9 as printed; include_unew=False drops the E*|U'| read term (see
    step1b_model_cpt: the Section 7.4 figure of 6.6 cpt holds only without it)."""
    read = E * (UM + UD + (Unew if include_unew else 0))
    return read + ECnew * (XM + XD) / 8


def eq10_step1b_write_bytes(E, Unew, ECnew, XM, XD) -> float:
    """Eq. 10: write U' and the packed translation tables."""
    return E * Unew + ECnew * (XM + XD) / 8


def eq12_gather_bytes(L, NM, ND) -> float:
    """Eq. 12: one cache line per translation-table lookup (tables not cached)."""
    return L * (NM + ND)


def eq13_stream_read_bytes(EC, NM, ND) -> float:
    """Eq. 13: stream the packed main and delta codes in."""
    return EC * (NM + ND) / 8


def eq14_stream_write_bytes(ECnew, NM, ND) -> float:
    """Eq. 14: write the merged vector, counted twice (write-allocate read)."""
    return 2 * ECnew * (NM + ND) / 8


def eq15_parallel_extra_bytes(E, UM, UD, Unew) -> float:
    """Eq. 15: second read of both dictionaries plus a second write of U'."""
    return E * (UM + UD) + 2 * E * Unew


def eq16_update_rate(n_delta, n_main, n_cols, cycles_per_tuple, hz) -> float:
    """Eq. 16: updates/s from an update cost in cycles per tuple per column."""
    return n_delta * hz / (cycles_per_tuple * (n_main + n_delta) * n_cols)


def eq17_step1a_cpt(E=8, UD=1_000_000, ND=1_000_000, NM=100_000_000, L=64,
                    stream_bpc=7.0, random_bpc=5.0) -> float:
    """Eq. 17: Step 1(a) at 100% unique, streaming part at 7 B/cycle, random part at 5."""
    return (4 * E * UD / stream_bpc + (2 * L + 4) * ND / random_bpc) / (NM + ND)


def step1b_model_cpt(E=8, UM=100_000_000, UD=1_000_000, ECnew=27, stream_bpc=7.0,
                     include_unew_read: bool = False) -> float:
    """Section 7.4: Step 1(b) cost from Eq. 9 + Eq. 10 + Eq. 15 at 7 B/cycle."""
    Unew = UM + UD
    total = (eq9_step1b_read_bytes(E, UM, UD, Unew, ECnew, UM, UD, include_unew_read)
             + eq10_step1b_write_bytes(E, Unew, ECnew, UM, UD)
             + eq15_parallel_extra_bytes(E, UM, UD, Unew))
    return total / stream_bpc / (UM + UD)


def step2_model_cpt(EC=27, ECnew=27, NM=100_000_000, ND=1_000_000, L=64, stream_bpc=7.0,
                    random_bpc=5.0) -> float:
    """Section 7.4: Step 2(b) from Eq. 12 (random) and Eq. 13 + Eq. 14 (streaming)."""
    n = NM + ND
    return (eq12_gather_bytes(L, NM, ND) / random_bpc
            + (eq13_stream_read_bytes(EC, NM, ND) + eq14_stream_write_bytes(ECnew, NM, ND))
            / stream_bpc) / n


def eq18_step2_cached_cpt(EC=19.9, ECnew=19.9, ops=4.0, threads=6, stream_bpc=7.0) -> float:
    """Eq. 18: Step 2 with cached tables: compute part plus streaming part."""
    return ops / threads + (EC / 8 + 2 * ECnew / 8) / stream_bpc


# ------------------------------------------------------------------ GPU algorithmic bytes

def step1_bytes(w: int, m: int, d: int, u: int) -> int:
    """Steps 1(a)+1(b): read both dictionaries once, write U' and 32-bit X_M, X_D."""
    return w * (m + d) + w * u + 4 * (m + d)


def step2_bytes(b: int, b_new: int, n_main: int, n_delta: int, m: int, d: int) -> int:
    """Step 2(b): read the packed main and the 32-bit delta codes, read X_M and
    X_D once, write the merged packed vector once."""
    return (b * n_main + 7) // 8 + 4 * n_delta + 4 * (m + d) + (b_new * (n_main + n_delta) + 7) // 8


def column_bytes(w, m, d, u, b, b_new, n_main, n_delta) -> int:
    return step1_bytes(w, m, d, u) + step2_bytes(b, b_new, n_main, n_delta, m, d)
