"""The merge server's admission rules on a fake clock (CPU only).

Checks what continuous batching under an HBM budget promises: admitted
footprints never exceed the pool, a table serves one merge at a time, no
more merges run than there are slots, a request blocked by a busy table does
not hold back others, and every request finishes.
"""
import numpy as np
import pytest

from paper_1109_6885_gb300 import build
from paper_1109_6885_gb300 import dmerge as dm


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    dm.load()


def check_schedule(pool, slots, fp, sv, rt, ar, admit, done, slot, peak_bytes, peak_running):
    n = len(rt)
    assert np.all(admit >= ar)
    assert np.all(done == admit + sv[rt])
    assert peak_bytes <= pool and peak_running <= slots
    # replay the intervals: bytes and merges in flight at every event
    events = sorted([(int(admit[i]), 1, i) for i in range(n)] + [(int(done[i]), 0, i) for i in range(n)])
    used = running = 0
    for _, kind, i in events:
        if kind:
            used += int(fp[rt[i]])
            running += 1
            assert used <= pool, "footprints over the budget"
            assert running <= slots
        else:
            used -= int(fp[rt[i]])
            running -= 1
    # one merge per table at a time; one merge per slot at a time
    for key in (rt, slot):
        for k in np.unique(key):
            idx = np.nonzero(key == k)[0]
            iv = sorted((int(admit[i]), int(done[i])) for i in idx)
            assert all(a1 >= d0 for (_, d0), (a1, _) in zip(iv, iv[1:]))


def test_unbounded_resources_admit_on_arrival():
    fp = np.array([100, 200, 300], np.uint64)
    sv = np.array([1000, 2000, 3000], np.uint64)
    rt = np.array([0, 1, 2], np.uint32)
    ar = np.array([0, 10, 20], np.uint64)
    admit, done, slot, pb, pr = dm.dm_sched_simulate(1 << 30, 8, fp, sv, rt, ar)
    assert np.array_equal(admit, ar)
    assert pr == 3


def test_budget_limits_inflight_bytes():
    fp = np.array([600, 600, 600, 600], np.uint64) * 256
    sv = np.array([1000, 1000, 1000, 1000], np.uint64)
    rt = np.array([0, 1, 2, 3], np.uint32)
    ar = np.zeros(4, np.uint64)
    pool = 1300 * 256                                   # room for two at a time
    admit, done, slot, pb, pr = dm.dm_sched_simulate(pool, 8, fp, sv, rt, ar)
    check_schedule(pool, 8, fp, sv, rt, ar, admit, done, slot, pb, pr)
    assert pr == 2 and sorted(admit.tolist()) == [0, 0, 1000, 1000]


def test_busy_table_does_not_block_others():
    fp = np.array([256, 256], np.uint64)
    sv = np.array([5000, 100], np.uint64)
    rt = np.array([0, 0, 1], np.uint32)                 # the second table-0 request must wait
    ar = np.array([0, 1, 2], np.uint64)
    admit, done, slot, pb, pr = dm.dm_sched_simulate(1 << 20, 4, fp, sv, rt, ar)
    assert admit[1] == done[0]                          # waited for its table
    assert admit[2] == 2                                # the later request passed it


def test_slots_bound_concurrency():
    fp = np.full(6, 256, np.uint64)
    sv = np.full(6, 1000, np.uint64)
    rt = np.arange(6, dtype=np.uint32)
    ar = np.zeros(6, np.uint64)
    admit, done, slot, pb, pr = dm.dm_sched_simulate(1 << 20, 2, fp, sv, rt, ar)
    check_schedule(1 << 20, 2, fp, sv, rt, ar, admit, done, slot, pb, pr)
    assert pr == 2 and sorted(admit.tolist()) == [0, 0, 1000, 1000, 2000, 2000]


@pytest.mark.parametrize("seed", range(5))
def test_poisson_trace_fake_clock(seed):
    """Poisson arrivals (seeded exponential gaps) over 64 tables under a budget."""
    rng = np.random.default_rng(seed)
    ntab, nreq = 64, 2000
    fp = (rng.integers(1, 64, ntab) * (1 << 20)).astype(np.uint64)
    sv = rng.integers(1_000_000, 80_000_000, ntab).astype(np.uint64)      # 1-80 ms
    rt = rng.integers(0, ntab, nreq).astype(np.uint32)
    ar = np.cumsum(rng.exponential(50e6, nreq)).astype(np.uint64)          # mean 20 req/s
    pool, slots = 150 << 20, 4
    admit, done, slot, pb, pr = dm.dm_sched_simulate(pool, slots, fp, sv, rt, ar)
    check_schedule(pool, slots, fp, sv, rt, ar, admit, done, slot, pb, pr)
    assert np.all(done > 0)


def test_footprint_larger_than_pool_is_refused():
    with pytest.raises(dm.DmError) as e:
        dm.dm_sched_simulate(1000, 2, np.array([5000], np.uint64), np.array([1], np.uint64),
                             np.array([0], np.uint32), np.array([0], np.uint64))
    assert e.value.status == dm.DM_ENOMEM
