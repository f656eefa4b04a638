"""Online tables on the GPU: inserts during a merge land in the next version.

Section 3 of the paper: the merge works on a copy of the table while rows
inserted meanwhile collect in a second delta; the commit swaps the merged
main in, and the second delta becomes the delta the next merge takes.
Section 4: a merge is triggered once N_D exceeds a fraction of N_M.

A server-owned online table is merged while rows are inserted into it; each
committed version, copied back, must equal the oracle's merge of the
previous version with exactly the rows its merge took: the delta as the
paper keeps it, the inserted values in arrival order (D_dict = those
values, row r coded r; repeated values are tolerated, Eq. 3).  Versions are
checked byte for byte (dictionary and packed codes).
"""
import time

import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm

pytestmark = pytest.mark.gpu


class Chain:
    """The oracle's versions of one column: main 0, then one merge per batch."""

    def __init__(self, col):
        self.w = col.w
        self.dict, self.packed, self.bits, self.rows = col.main_dict, col.main_packed, col.main_bits, col.n_main

    def merge(self, values):
        n = values.shape[0]
        r = oracle.merge_column(self.w, self.dict, self.packed, self.bits, self.rows, values,
                                np.arange(n, dtype=np.uint32))
        self.dict, self.packed, self.bits, self.rows = r.new_dict, r.new_packed, r.new_bits, self.rows + n


def batch(col, n, seed, frac_new=0.3):
    """n inserted values of a column: mostly values already in it (with the
    main's code distribution), the rest new, in arrival order."""
    rng = np.random.default_rng(seed)
    src = col.main_dict[col.main_codes[rng.integers(0, col.n_main, n)]]
    fresh = synth.dictionary(synth.subseed(seed, 9), col.w, max(1, n // 7))
    pick = rng.random(n) < frac_new
    src[pick] = fresh[rng.integers(0, fresh.shape[0], int(pick.sum()))]
    return np.ascontiguousarray(src)


def online_table(srv, tid, cols, rows_capacity, delta_capacity, trigger=0.0):
    keep = []
    specs = []
    for c in cols:
        d = dm.to_device(c.main_dict)
        p = dm.to_device(c.main_packed)
        keep += [d, p]
        specs.append(dm.OnlineColumn(c.w, d.data_ptr(), c.main_dict.shape[0], p.data_ptr(), c.main_bits))
    srv.add_online_table(tid, specs, cols[0].n_main, rows_capacity, delta_capacity, trigger)
    return keep


def check_version(srv, tid, chains, version):
    for j, ch in enumerate(chains):
        v, keys, words, bits, rows = srv.online_copy(tid, j, ch.w)
        assert v == version
        assert rows == ch.rows and bits == ch.bits, (j, rows, ch.rows, bits, ch.bits)
        assert np.array_equal(keys, ch.dict), j
        assert np.array_equal(words, ch.packed), j


def wait_admitted(srv, rid, timeout=30.0):
    t0 = time.perf_counter()
    while srv.info(rid).admit_ns == 0 and srv.info(rid).status < 0:
        assert time.perf_counter() - t0 < timeout


def make_cols(n_main, seed):
    out = []
    for j, (w, m) in enumerate([(8, 400_000), (16, 60_000), (4, 3_000)]):
        spec = synth.ColumnSpec(n_main=n_main, m=m, w=w, n_delta=1, f_new=0.0, dist="zipf", zipf_s=1.0,
                                seed=synth.column_seed(61 + seed, j))
        out.append(synth.make_column(spec))
    return out


def test_rows_inserted_during_a_merge_land_in_the_next_version():
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    n_main = 100_000_000
    cols = make_cols(n_main, 0)
    chains = [Chain(c) for c in cols]
    srv = dm.Server(0, slots=2, scratch_budget=8 << 30)
    keep = online_table(srv, 7, cols, rows_capacity=n_main + 1_200_000, delta_capacity=300_000)
    check_version(srv, 7, chains, 0)

    mid_merge = 0
    for k in range(3):
        va, vb = 2 * k + 1, 2 * k + 2                  # the versions of this pass's two merges
        a = [batch(c, 300_000, 100 * k + j) for j, c in enumerate(cols)]
        b = [batch(c, 50_000, 100 * k + 50 + j) for j, c in enumerate(cols)]
        adev, bdev = [dm.to_device(x) for x in a], [dm.to_device(x) for x in b]
        torch.cuda.synchronize()
        info = srv.insert(7, 300_000, adev)
        assert info.lands_in == va
        rid = srv.submit(7)
        wait_admitted(srv, rid)
        # the merge has frozen batch a; b goes to the second delta
        info_b = srv.insert(7, 50_000, bdev)
        mid_merge += srv.info(rid).status < 0
        assert info_b.lands_in == vb
        srv.drain()
        assert srv.info(rid).status == dm.DM_OK and srv.info(rid).version == va
        assert srv.info(rid).delta_rows == 300_000
        for ch, x in zip(chains, a):
            ch.merge(x)
        check_version(srv, 7, chains, va)              # holds a, not b
        assert srv.online_view(7, 0).delta_rows == 50_000
        # the next merge takes b and nothing else
        rid2 = srv.submit(7)
        srv.drain()
        assert srv.info(rid2).status == dm.DM_OK and srv.info(rid2).delta_rows == 50_000
        for ch, x in zip(chains, b):
            ch.merge(x)
        check_version(srv, 7, chains, vb)
        assert srv.online_view(7, 0).delta_rows == 0
    assert mid_merge >= 1, "the second batch never arrived while the merge was on the GPU"
    srv.close()
    del keep


def test_trigger_requests_merges_and_pause_holds_them():
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    n_main = 2_000_000
    cols = make_cols(n_main, 1)
    chains = [Chain(c) for c in cols]
    srv = dm.Server(0, slots=1, scratch_budget=4 << 30)
    keep = online_table(srv, 3, cols, rows_capacity=n_main + 400_000, delta_capacity=100_000, trigger=0.01)
    srv.pause(3)
    # 20,000 rows pass the trigger (k N_M = 20,000) only with the third batch
    batches = [[batch(c, 8_000, 7 * i + j) for j, c in enumerate(cols)] for i in range(3)]
    infos = [srv.insert(3, 8_000, [dm.to_device(x) for x in bt]) for bt in batches]
    assert [i.triggered for i in infos] == [0, 0, 1]
    time.sleep(0.2)
    assert srv.version(3) == 0, "a paused table merged"
    srv.resume(3)
    srv.drain()
    assert srv.version(3) == 1
    rid = infos[2].request
    assert srv.info(rid).automatic == 1 and srv.info(rid).delta_rows == 24_000
    for ch, j in zip(chains, range(3)):
        ch.merge(np.concatenate([bt[j] for bt in batches]))
    check_version(srv, 3, chains, 1)
    srv.close()
    del keep


def test_insert_past_the_delta_capacity_is_refused_whole():
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    cols = make_cols(500_000, 2)
    chains = [Chain(c) for c in cols]
    srv = dm.Server(0, slots=1, scratch_budget=1 << 30)
    keep = online_table(srv, 1, cols, rows_capacity=600_000, delta_capacity=10_000)
    a = [batch(c, 9_000, 300 + j) for j, c in enumerate(cols)]
    srv.insert(1, 9_000, [dm.to_device(x) for x in a])
    with pytest.raises(dm.DmError) as e:
        srv.insert(1, 2_000, [dm.to_device(batch(c, 2_000, 400 + j)) for j, c in enumerate(cols)])
    assert e.value.status == dm.DM_EBUSY
    srv.submit(1)
    srv.drain()
    for ch, x in zip(chains, a):
        ch.merge(x)
    check_version(srv, 1, chains, 1)
    srv.close()
    del keep
