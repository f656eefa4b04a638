"""Bit-exact parity at the full shapes of the batched table and served workloads.

`table-300x50M-mixed` is 300 columns sharing 50,000,000 main rows and
500,000 delta rows, per column a dictionary size log-uniform in [2, 5e7], a
value width from {4, 8, 16} bytes, Zipf(0.8) codes and a new-value fraction
uniform in [0, 0.5] (the column data repeats every 30 columns, each column
still merged on its own into its own outputs).  The whole table goes through
dm_merge_table as the bench times it: one CUDA graph over eight branches,
with the capped Step 1 grids that send the large dictionaries to the split
form, then a replay of the recorded graph, then per-column plain launches
(DM_FLAG_SERIAL).  After each, every column's U', X_M, X_D, |U'|, E'_C and
packed bytes must equal the oracle's merge of its data.  The served
workload's test is described in its own docstring below.
"""
from __future__ import annotations

import concurrent.futures
import gc

import numpy as np
import pytest

import bench
import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm

pytestmark = pytest.mark.gpu


def _pool_map(fn, items, workers=16):
    # the generator and the oracle are C libraries called through ctypes,
    # which releases the interpreter lock: threads run them in parallel
    with concurrent.futures.ThreadPoolExecutor(max_workers=workers) as ex:
        return list(ex.map(fn, items))


class DeviceRef:
    """The oracle's merge of one column, on the device for fast comparison."""

    def __init__(self, ref):
        self.u, self.b = ref.u, ref.new_bits
        self.new_dict = dm.to_device(ref.new_dict)
        self.x_main = dm.to_device(ref.x_main)
        self.x_delta = dm.to_device(ref.x_delta)
        self.packed = dm.to_device(ref.new_packed)


def assert_same(res, ref: DeviceRef, n_out: int, what: str):
    import torch
    u, b = res.u_bits()
    assert (u, b) == (ref.u, ref.b), (what, u, ref.u, b, ref.b)
    nwords = dm.dm_packed_bytes(n_out, b) // 4
    assert torch.equal(res.new_dict[:u], ref.new_dict), what
    assert torch.equal(res.x_main, ref.x_main), what
    assert torch.equal(res.x_delta, ref.x_delta), what
    assert torch.equal(res.new_packed[:nwords], ref.packed), what


def poison(res):
    for t in (res.new_dict, res.new_packed, res.x_main, res.x_delta):
        t.fill_(-1)
    res.scalars.fill_(-1)


def test_table_300x50M_bit_exact_batched_replayed_and_serial():
    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    gc.collect()
    torch.cuda.empty_cache()
    name = "table-300x50M-mixed"
    specs = bench.table_specs(name)
    nsrc = bench.TABLES[name]["distinct"]
    assert len(specs) == 300 and nsrc == 30
    cols = _pool_map(synth.make_column, specs[:nsrc])
    refs = _pool_map(oracle.merge_synth_column, cols)
    srcs = [dm.DeviceColumn.from_numpy(c.w, c.main_dict, c.main_packed, c.main_bits, c.n_main,
                                       c.delta_dict, c.delta_codes) for c in cols]
    drefs = [DeviceRef(r) for r in refs]
    del refs
    dcols = [srcs[j % nsrc] for j in range(len(specs))]
    res = [dm.alloc_result(d) for d in dcols]
    cins = [d.cin() for d in dcols]
    couts = [r.cout() for r in res]
    ctx = dm.Context(0)
    ctx.reserve(max(dm.dm_table_scratch_bytes(cins, 0),
                    dm.dm_table_scratch_bytes(cins, dm.DM_FLAG_SERIAL)))
    n_out = [c.n_main + c.n_delta for c in cols]
    # the large dictionaries do take the capped split Step 1 in the batched form
    assert max(c.main_dict.shape[0] for c in cols) > 10_000_000

    def check(what):
        torch.cuda.synchronize()
        assert ctx.sync_status() == dm.DM_OK, what
        for j, r in enumerate(res):
            assert_same(r, drefs[j % nsrc], n_out[j % nsrc], f"{what}: column {j}")

    for what, flags in [("batched graph (recorded)", 0), ("batched graph (replayed)", 0),
                        ("per-column plain launches", dm.DM_FLAG_SERIAL)]:
        for r in res:
            poison(r)
        dm.dm_merge_table(ctx, cins, couts, None, flags)
        check(what)
    ctx.close()
    del res, dcols, srcs, drefs
    gc.collect()
    torch.cuda.empty_cache()


def test_served_64_tables_each_request_equals_its_solo_run_and_a_sample_the_oracle():
    """`serve-64tables-poisson20`: 64 resident tables of 20-200 columns, main
    rows log-uniform in [1e5, 2e8], delta 0.1-10% of main, a 150 GB admission
    budget and Poisson arrivals at 20 requests/s (each table's columns repeat
    two distinct column data sets, inputs and outputs, as in the bench).
    Every table is merged alone first; then 200 seeded Poisson requests are
    served with continuous batching.  Each request's output checksum must
    equal its table's solo checksum, and ten tables (the largest among them)
    must equal the oracle byte for byte, after the solo runs and again after
    the mix."""
    import time

    import torch

    from paper_1109_6885_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    gc.collect()
    torch.cuda.empty_cache()
    cfg = bench.SERVES["serve-64tables-poisson20"]
    tables, dev, specs = bench.serve_tables(dm, cfg, 0)
    assert len(tables) == 64
    first = np.cumsum([0] + [len(sps) for _, sps in specs])   # first distinct column of each table
    tuples = [sum(ci.main_rows + ci.delta_rows for ci in cins) for cins, _ in tables]
    rng = np.random.default_rng(20)
    sample = sorted({int(np.argmax(tuples))} | set(int(t) for t in rng.choice(64, 12, replace=False)))[:10]
    if int(np.argmax(tuples)) not in sample:
        sample[-1] = int(np.argmax(tuples))
    host = {}
    for t in sample:
        host[t] = _pool_map(synth.make_column, specs[t][1])
    refs = {t: _pool_map(oracle.merge_synth_column, host[t]) for t in sample}

    def check_sample(what):
        torch.cuda.synchronize()
        for t in sample:
            for k, (col, ref) in enumerate(zip(host[t], refs[t])):
                _, res = dev[first[t] + k]
                new_dict, _, _, packed, b, u = dm.fetch(res, col.w, col.n_main + col.n_delta)
                assert (u, b) == (ref.u, ref.new_bits), (what, t, k)
                assert np.array_equal(new_dict, ref.new_dict), (what, t, k)
                assert np.array_equal(packed, ref.new_packed), (what, t, k)

    srv = dm.Server(0, slots=cfg["slots"], scratch_budget=cfg["budget"], flags=dm.DM_SERVER_DIGEST)
    for t, (cins, couts) in enumerate(tables):
        srv.add_table(t, cins, couts)
    solo = []
    for t in range(64):
        rid = srv.submit(t)
        srv.drain()
        info = srv.info(rid)
        assert info.status == dm.DM_OK and info.digest != 0
        solo.append(info.digest)
    check_sample("solo")

    nreq = 200
    tabs = rng.integers(0, 64, nreq)
    gaps = rng.exponential(1.0 / cfg["rate"], nreq)
    due = time.perf_counter()
    rids = []
    for t, g in zip(tabs, gaps):
        due += g
        while time.perf_counter() < due:
            time.sleep(0.0005)
        rids.append((int(t), srv.submit(int(t))))
    srv.drain()
    st = srv.stats()
    assert st.failed == 0
    assert st.peak_scratch_bytes <= cfg["budget"]
    assert st.peak_concurrency >= 2, "no requests overlapped"
    for t, rid in rids:
        info = srv.info(rid)
        assert info.status == dm.DM_OK
        assert info.digest == solo[t], (rid, t)
    check_sample("after the mix")
    srv.close()
    del tables, dev
    gc.collect()
    torch.cuda.empty_cache()
