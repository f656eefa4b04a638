"""Bit-exact parity at the full shape of the batched table workload.

`table-300x50M-mixed` is 300 columns sharing 50,000,000 main rows and
500,000 delta rows, per column a dictionary size log-uniform in [2, 5e7], a
value width from {4, 8, 16} bytes, Zipf(0.8) codes and a new-value fraction
uniform in [0, 0.5] (the column data repeats every 30 columns, each column
still merged on its own into its own outputs).  The whole table goes through
dm_merge_table as the bench times it: one CUDA graph over eight branches,
with the capped Step 1 grids that send the large dictionaries to the split
form, then a replay of the recorded graph, then per-column plain launches
(DM_FLAG_SERIAL).  After each, every column's U', X_M, X_D, |U'|, E'_C and
packed bytes must equal the oracle's merge of its data.
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
