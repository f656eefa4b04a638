"""Served merges (dm_server): continuous batching on the GPU.

A table's merge result is the same when it runs alone and when it runs in a
burst of concurrent requests over many tables (bit-exact: integer work);
every table's result matches the oracle; the scratch held at once never
exceeds the budget; merges did overlap; each completed merge commits one new
version of its table.
"""
import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm

pytestmark = pytest.mark.gpu


def make_tables(ntables, seed):
    rng = np.random.default_rng(seed)
    tables = []
    for t in range(ntables):
        ncols = int(rng.integers(2, 6))
        n_main = int(np.exp(rng.uniform(np.log(100_000), np.log(1_500_000))))
        n_delta = max(1, int(n_main * np.exp(rng.uniform(np.log(0.001), np.log(0.1)))))
        cols, dcols, res = [], [], []
        for j in range(ncols):
            m = int(np.exp(rng.uniform(np.log(2), np.log(n_main))))
            spec = synth.ColumnSpec(n_main=n_main, m=m, w=int(rng.choice([4, 8, 16])),
                                    n_delta=n_delta, f_new=float(rng.uniform(0, 0.5)),
                                    dist="zipf", zipf_s=0.8,
                                    seed=synth.column_seed(5 + 100 * seed + t, j))
            col = synth.make_column(spec)
            dc = dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits,
                                            col.n_main, col.delta_dict, col.delta_codes)
            cols.append(col)
            dcols.append(dc)
            res.append(dm.alloc_result(dc))
        tables.append((cols, dcols, res))
    return tables


def snapshot(cols, res):
    return [dm.fetch(r, c.w, c.n_main + c.n_delta) for c, r in zip(cols, res)]


def check_oracle(cols, snap):
    for col, (new_dict, xm, xd, packed, b, u) in zip(cols, snap):
        ref = oracle.merge_synth_column(col)
        assert u == ref.u and b == ref.new_bits
        assert np.array_equal(new_dict, ref.new_dict)
        assert np.array_equal(packed, ref.new_packed)
        assert np.array_equal(xm, ref.x_main) and np.array_equal(xd, ref.x_delta)


def same(a, b):
    for x, y in zip(a, b):
        for p, q in zip(x, y):
            if isinstance(p, np.ndarray):
                assert np.array_equal(p, q)
            else:
                assert p == q


def test_served_results_same_alone_and_in_mix():
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    tables = make_tables(6, seed=1)
    footprints = [dm.dm_table_scratch_bytes([d.cin() for d in t[1]]) for t in tables]
    budget = int(2.5 * max(footprints))
    srv = dm.Server(0, slots=3, scratch_budget=budget)
    for tid, (cols, dcols, res) in enumerate(tables):
        srv.add_table(tid, [d.cin() for d in dcols], [r.cout() for r in res])

    # alone
    srv.submit(2)
    srv.drain()
    torch.cuda.synchronize()
    alone = snapshot(tables[2][0], tables[2][2])
    check_oracle(tables[2][0], alone)

    # in a burst over every table, five rounds
    rids = [srv.submit(tid) for _ in range(5) for tid in range(len(tables))]
    srv.drain()
    torch.cuda.synchronize()
    st = srv.stats()
    assert st.failed == 0 and st.completed == 1 + len(rids)
    assert st.peak_scratch_bytes <= budget
    assert st.peak_concurrency >= 2, "no merges overlapped"
    for rid in rids:
        info = srv.info(rid)
        assert info.status == dm.DM_OK
        assert info.submit_ns <= info.admit_ns <= info.done_ns
    same(snapshot(tables[2][0], tables[2][2]), alone)
    for cols, dcols, res in tables:
        check_oracle(cols, snapshot(cols, res))
    assert srv.version(2) == 6 and srv.version(0) == 5
    srv.close()


def test_server_rejects_a_table_larger_than_the_budget():
    from paper_1109_6885_gb300 import build
    build.build()
    cols, dcols, res = make_tables(1, seed=2)[0]
    srv = dm.Server(0, slots=1, scratch_budget=4096)
    with pytest.raises(dm.DmError) as e:
        srv.add_table(0, [d.cin() for d in dcols], [r.cout() for r in res])
    assert e.value.status == dm.DM_ENOMEM
    srv.close()


def test_request_digests_equal_solo_runs_and_change_with_the_result():
    """DM_SERVER_DIGEST: each request's checksum equals that of its table
    merged alone, and a column whose result differs has a different one."""
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    tables = make_tables(5, seed=3)
    footprints = [dm.dm_table_scratch_bytes([d.cin() for d in t[1]]) for t in tables]
    srv = dm.Server(0, slots=3, scratch_budget=int(2.5 * max(footprints)), flags=dm.DM_SERVER_DIGEST)
    for tid, (cols, dcols, res) in enumerate(tables):
        srv.add_table(tid, [d.cin() for d in dcols], [r.cout() for r in res])
    solo = []
    for tid in range(len(tables)):
        rid = srv.submit(tid)
        srv.drain()
        solo.append(srv.info(rid).digest)
    rids = [(tid, srv.submit(tid)) for _ in range(4) for tid in range(len(tables))]
    srv.drain()
    for tid, rid in rids:
        assert srv.info(rid).digest == solo[tid]
    assert len(set(solo)) == len(solo)
    # the same checksum from dm_column_digest, and a flipped output word changes it
    cols, dcols, res = tables[0]
    cins, couts = [d.cin() for d in dcols], [r.cout() for r in res]
    torch.cuda.synchronize()
    per_col = dm.column_digests(cins, couts)
    assert sum(per_col) % 2**64 == solo[0]
    res[0].new_packed[0] ^= 1
    assert dm.column_digests(cins, couts)[0] != per_col[0]
    srv.close()
