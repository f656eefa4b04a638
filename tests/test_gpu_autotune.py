"""The autotuner on the GPU: every candidate launch choice, forced through the
tune cache, gives the oracle's bytes; a tuned column, a tuned table and a
server sharing one cache all stay exact; tuning happens once per class."""
import numpy as np
import pytest

import oracle
import synth
from paper_1109_6885_gb300 import dmerge as dm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def built():
    import torch
    assert torch.cuda.is_available()
    from paper_1109_6885_gb300 import build
    build.build()


def _device_column(col):
    return dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits, col.n_main,
                                      col.delta_dict, col.delta_codes)


class DeviceRef:
    """The oracle's result of a column, on the device, for fast repeated checks."""

    def __init__(self, col):
        import torch
        ref = oracle.merge_synth_column(col)
        self.u, self.b = ref.u, ref.new_bits
        self.new_dict = dm.to_device(ref.new_dict) if ref.u else None
        self.packed = dm.to_device(ref.new_packed) if ref.new_packed.size else None
        self.xm = dm.to_device(ref.x_main) if ref.x_main.size else None
        self.xd = dm.to_device(ref.x_delta) if ref.x_delta.size else None
        self.torch = torch

    def check(self, res, w):
        torch = self.torch
        u, b = res.u_bits()
        assert (u, b) == (self.u, self.b)
        if self.new_dict is not None:
            got = res.new_dict[:u]
            assert torch.equal(got.reshape(-1).view(torch.uint8),
                               self.new_dict.reshape(-1).view(torch.uint8))
        if self.packed is not None:
            n = self.packed.numel()
            assert torch.equal(res.new_packed[:n].view(torch.int32), self.packed.view(torch.int32))
        if self.xm is not None:
            assert torch.equal(res.x_main.view(torch.int32), self.xm.view(torch.int32))
        if self.xd is not None:
            assert torch.equal(res.x_delta.view(torch.int32), self.xd.view(torch.int32))


def _fill_junk(res):
    import torch
    for t in (res.new_dict, res.new_packed, res.x_main, res.x_delta):
        if t is not None and t.numel():
            t.view(torch.uint8).fill_(0xA5)
    res.scalars.fill_(-1)


FORCED_CASES = {
    # X_M in a shared-memory table (m <= 16384) or the global gather
    "small-dict": dict(n_main=300_007, m=5_000, w=4, n_delta=3_001, f_new=0.4, dist="zipf", zipf_s=0.8),
    # directory of X_M's steps (m above the table) from 2^20 main rows
    "directory": dict(n_main=1_500_003, m=100_000, w=8, n_delta=15_001, f_new=0.3, dist="zipf", zipf_s=1.0),
    "wide-keys": dict(n_main=1_100_001, m=60_000, w=16, n_delta=40_000, f_new=0.5, dist="uniform"),
    # byte table for crowded directory buckets (above 11 * 2^20 main codes)
    "byte-table": dict(n_main=10_000_000, m=12_000_000, w=8, n_delta=1_000_000, f_new=0.5, dist="zipf",
                       zipf_s=0.8),
    "delta-only": dict(n_main=0, m=0, w=8, n_delta=200_003, f_new=1.0, dist="uniform"),
}


@pytest.mark.parametrize("case", list(FORCED_CASES))
def test_every_candidate_choice_is_exact(built, case):
    import torch
    spec = synth.ColumnSpec(seed=synth.column_seed(9, len(case)), **FORCED_CASES[case])
    col = synth.make_column(spec)
    ref = DeviceRef(col)
    ctx = dm.Context(0, 0)
    dcol = _device_column(col)
    cin = dcol.cin()
    ctx.reserve(dm.dm_scratch_bytes(cin))
    res = dm.alloc_result(dcol)
    cands = ctx.tune_candidates(cin)
    n_stage = 1 if col.n_main == 0 else 2
    n_x8 = 2 if case == "byte-table" else 1
    assert len(cands) == n_stage * n_x8 * 7 * 3
    key = dm.dm_tune_key_of(cin)
    cache = ctx.tune_cache
    for c in cands:
        cache.put(key, c)
        _fill_junk(res)
        dm.dm_merge_column(ctx, cin, res.cout())
        torch.cuda.synchronize()
        assert ctx.sync_status() == dm.DM_OK, c.as_dict()
        ref.check(res, col.w)
    ctx.close()


def test_autotune_column(built):
    import torch
    spec = synth.ColumnSpec(seed=synth.column_seed(9, 100), **FORCED_CASES["directory"])
    col = synth.make_column(spec)
    ref = DeviceRef(col)
    ctx = dm.Context(0, 0)
    dcol = _device_column(col)
    cin = dcol.cin()
    ctx.reserve(dm.dm_scratch_bytes(cin))
    res = dm.alloc_result(dcol)
    _fill_junk(res)
    rep = dm.dm_autotune_column(ctx, cin, res.cout(), reps=3)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    ref.check(res, col.w)
    assert rep.key.as_tuple() == dm.dm_tune_key_of(cin).as_tuple()
    assert rep.reps == 3
    # the default, then each axis's values other than the best so far:
    # 2 stagings + 6 more launch shapes + 2 more Step 1 grids
    assert rep.candidates == 11
    assert 0 < rep.best_ms <= rep.default_ms
    assert ctx.tune_cache.get(rep.key).as_dict() == rep.best.as_dict()
    cands = [c.as_dict() for c in ctx.tune_candidates(cin)]
    for f in rep.best.as_dict():
        assert rep.best.as_dict()[f] in {c[f] for c in cands} | {0}
    # later merges use the stored choice and stay exact
    _fill_junk(res)
    dm.dm_merge_column(ctx, cin, res.cout())
    torch.cuda.synchronize()
    ref.check(res, col.w)
    ctx.close()


def test_merge_column_autotune_flag_tunes_once(built):
    import torch
    spec = synth.ColumnSpec(seed=synth.column_seed(9, 101), **FORCED_CASES["small-dict"])
    col = synth.make_column(spec)
    ref = DeviceRef(col)
    ctx = dm.Context(0, 0)
    dcol = _device_column(col)
    cin = dcol.cin()
    ctx.reserve(dm.dm_scratch_bytes(cin))
    res = dm.alloc_result(dcol)
    assert len(ctx.tune_cache) == 0
    dm.dm_merge_column(ctx, cin, res.cout(), flags=dm.DM_FLAG_AUTOTUNE)
    torch.cuda.synchronize()
    ref.check(res, col.w)
    assert len(ctx.tune_cache) == 1
    gen, launches = ctx.tune_cache.generation, ctx.launches
    _fill_junk(res)
    dm.dm_merge_column(ctx, cin, res.cout(), flags=dm.DM_FLAG_AUTOTUNE)
    torch.cuda.synchronize()
    ref.check(res, col.w)
    assert ctx.tune_cache.generation == gen
    assert ctx.launches - launches <= 3      # one merge, no tuning merges
    ctx.close()


def _uneven_table(seed, ncols, n_main, n_delta, max_m):
    rng = np.random.default_rng(seed)
    cols = []
    for j in range(ncols):
        m = int(np.exp(rng.uniform(np.log(2), np.log(max_m))))
        spec = synth.ColumnSpec(n_main=n_main, m=m, w=int(rng.choice([4, 8, 16])), n_delta=n_delta,
                                f_new=float(rng.uniform(0, 0.5)), dist="zipf", zipf_s=0.8,
                                seed=synth.column_seed(40 + seed, j))
        cols.append(synth.make_column(spec))
    return cols


def test_merge_table_autotune(built):
    import torch
    cols = _uneven_table(1, 10, 400_003, 4_001, 400_000)
    refs = [DeviceRef(c) for c in cols]
    dcols = [_device_column(c) for c in cols]
    results = [dm.alloc_result(d) for d in dcols]
    cins = [d.cin() for d in dcols]
    couts = [r.cout() for r in results]
    ctx = dm.Context(0, 0)
    ctx.reserve(dm.dm_table_scratch_bytes(cins))
    for r in results:
        _fill_junk(r)
    dm.dm_merge_table(ctx, cins, couts, flags=dm.DM_FLAG_AUTOTUNE)
    torch.cuda.synchronize()
    assert ctx.sync_status() == dm.DM_OK
    for ref, r, c in zip(refs, results, cols):
        ref.check(r, c.w)
    classes = {dm.dm_tune_key_of(ci).as_tuple() for ci in cins}
    assert len(ctx.tune_cache) == len(classes)
    # replays: no more tuning, one graph launch each, same bytes
    gen = ctx.tune_cache.generation
    for r in results:
        _fill_junk(r)
    l0 = ctx.launches
    dm.dm_merge_table(ctx, cins, couts, flags=dm.DM_FLAG_AUTOTUNE)
    l1 = ctx.launches
    dm.dm_merge_table(ctx, cins, couts)
    l2 = ctx.launches
    torch.cuda.synchronize()
    assert ctx.tune_cache.generation == gen
    assert l1 - l0 == l2 - l1
    for ref, r, c in zip(refs, results, cols):
        ref.check(r, c.w)
    # serial form under the tuned choices
    for r in results:
        _fill_junk(r)
    dm.dm_merge_table(ctx, cins, couts, flags=dm.DM_FLAG_SERIAL)
    torch.cuda.synchronize()
    for ref, r, c in zip(refs, results, cols):
        ref.check(r, c.w)
    ctx.close()


def test_saved_cache_drives_another_context(built, tmp_path):
    import torch
    spec = synth.ColumnSpec(seed=synth.column_seed(9, 102), **FORCED_CASES["wide-keys"])
    col = synth.make_column(spec)
    ref = DeviceRef(col)
    dcol = _device_column(col)
    cin = dcol.cin()
    res = dm.alloc_result(dcol)
    a = dm.Context(0, dm.dm_scratch_bytes(cin))
    rep = dm.dm_autotune_column(a, cin, res.cout(), reps=2)
    path = str(tmp_path / "tune.json")
    a.tune_cache.save(path)
    a.close()
    shared = dm.TuneCache()
    shared.load(path)
    b = dm.Context(0, dm.dm_scratch_bytes(cin))
    b.set_tune_cache(shared)
    assert b.tune_cache.get(rep.key).as_dict() == rep.best.as_dict()
    _fill_junk(res)
    dm.dm_merge_column(b, cin, res.cout(), flags=dm.DM_FLAG_AUTOTUNE)   # found: no tuning
    torch.cuda.synchronize()
    ref.check(res, col.w)
    assert len(shared) == 1
    b.set_tune_cache(None)
    assert len(b.tune_cache) == 0
    b.close()


def test_server_slots_share_one_cache(built):
    import torch
    cols = _uneven_table(2, 4, 300_001, 3_001, 300_000)
    refs = [DeviceRef(c) for c in cols]
    dcols = [_device_column(c) for c in cols]
    results = [dm.alloc_result(d) for d in dcols]
    cins = [d.cin() for d in dcols]
    budget = 2 * dm.dm_table_scratch_bytes(cins)
    srv = dm.Server(0, slots=2, scratch_budget=budget, flags=dm.DM_FLAG_AUTOTUNE)
    srv.add_table(0, cins, [r.cout() for r in results])
    srv.submit(0)
    srv.drain()
    torch.cuda.synchronize()
    for ref, r, c in zip(refs, results, cols):
        ref.check(r, c.w)
    classes = {dm.dm_tune_key_of(ci).as_tuple() for ci in cins}
    assert len(srv.tune_cache) == len(classes)
    gen = srv.tune_cache.generation
    for r in results:
        _fill_junk(r)
    srv.submit(0)
    srv.drain()
    torch.cuda.synchronize()
    assert srv.tune_cache.generation == gen
    for ref, r, c in zip(refs, results, cols):
        ref.check(r, c.w)
    srv.close()


# Step 1 under a capped grid: the merge (and, for a large delta dictionary,
# the sort) leave the cooperative kernel for kernels that take tiles from a
# counter.  Delta dictionaries of ~200k uniform keys partition on their top
# byte; ~750k+ keys overflow its buckets and take the byte-by-byte passes.
SPLIT_CASES = {
    "msd": dict(n_main=2_000_003, m=300_000, n_delta=400_001, f_new=0.5, dist="zipf", zipf_s=0.8),
    "lsd": dict(n_main=1_000_003, m=1_000_000, n_delta=1_500_001, f_new=0.5, dist="uniform"),
}


@pytest.mark.parametrize("w", [4, 8, 16])
@pytest.mark.parametrize("case", list(SPLIT_CASES))
def test_capped_step1_split_forms(built, w, case):
    import torch
    spec = synth.ColumnSpec(w=w, seed=synth.column_seed(11, w + len(case)), **SPLIT_CASES[case])
    col = synth.make_column(spec)
    if case == "lsd":
        assert col.delta_dict.shape[0] > 256 * 2048   # the top byte's buckets overflow
    ref = DeviceRef(col)
    ctx = dm.Context(0, 0)
    dcol = _device_column(col)
    cin = dcol.cin()
    ctx.reserve(dm.dm_scratch_bytes(cin))
    res = dm.alloc_result(dcol)
    key = dm.dm_tune_key_of(cin)
    for blocks in (1, 8, 38):
        ctx.tune_cache.put(key, choice_of(step1_blocks=blocks))
        for _ in range(2):
            _fill_junk(res)
            dm.dm_merge_column(ctx, cin, res.cout())
            torch.cuda.synchronize()
            assert ctx.sync_status() == dm.DM_OK, blocks
            ref.check(res, col.w)
    ctx.close()


def choice_of(**kw):
    c = dm.TuneChoice()
    for k, v in kw.items():
        setattr(c, k, v)
    return c
