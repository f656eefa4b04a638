"""The online-table rules of the merge server on a fake clock (CPU only).

Section 3 of the paper: a merge works on a copy of the table while incoming
rows go to a second delta, which becomes the delta when the merge commits;
a scheduler may pause and resume merges.  Section 4: a merge is triggered
once N_D exceeds a fraction k of N_M.  These tests drive the scheduler core
the server runs (dm_online_simulate) with inserts, requests, pauses and
resumes and check what those rules fix: every accepted row lands in exactly
one committed version, the version the insert was told; rows inserted while
a merge runs land in the next version; versions never go back in insert
order; the trigger fires at the first crossing of k N_M; a paused table
merges nothing until it is resumed; a full delta rejects rows whole.
"""
import numpy as np
import pytest

from paper_1109_6885_gb300 import build
from paper_1109_6885_gb300 import dmerge as dm

MS = 1_000_000
INSERT, SUBMIT, PAUSE, RESUME = 0, 1, 2, 3


@pytest.fixture(scope="module", autouse=True)
def lib():
    build.build()
    dm.load()


def steady_inserts(table, rows, every_ns, count, t0=0):
    return [(t0 + i * every_ns, INSERT, table, rows) for i in range(count)]


def run(events, main_rows, delta_cap, trigger, service_ns, slots=1):
    events = sorted(events, key=lambda e: e[0])
    ns = [e[0] for e in events]
    kind = [e[1] for e in events]
    table = [e[2] for e in events]
    rows = [e[3] for e in events]
    r = dm.dm_online_simulate(slots, main_rows, delta_cap, trigger, service_ns, kind, table, rows, ns)
    return events, r


def check_invariants(events, r, main_rows0, trigger):
    ntab = len(main_rows0)
    ins = [i for i, e in enumerate(events) if e[1] == INSERT]
    accepted = [i for i in ins if r["version"][i] > 0]
    # every accepted row lands where the insert said; rows still in a delta
    # when the run ends were told the version after the table's last one
    last = {t: max([int(v) for k, v in enumerate(r["version_of_merge"]) if r["table"][k] == t] + [0])
            for t in range(ntab)}
    for i in ins:
        if not r["lands_in"][i]:
            continue
        if r["version"][i]:
            assert r["version"][i] == r["lands_in"][i], (i, events[i])
        else:
            assert r["lands_in"][i] == last[events[i][2]] + 1, (i, events[i])
    # a merge of version v took exactly the rows of the inserts that landed in v
    for k in range(r["merges"]):
        t, v = int(r["table"][k]), int(r["version_of_merge"][k])
        took = sum(events[i][3] for i in accepted if events[i][2] == t and r["version"][i] == v)
        if v:
            assert took == int(r["rows"][k]), (k, took, r["rows"][k])
        else:
            assert int(r["rows"][k]) == 0
    for t in range(ntab):
        mine = [k for k in range(r["merges"]) if r["table"][k] == t and r["version_of_merge"][k]]
        vers = [int(r["version_of_merge"][k]) for k in mine]
        assert vers == list(range(1, len(vers) + 1)), vers
        # one merge of a table at a time
        for a, b in zip(mine, mine[1:]):
            assert r["admit_ns"][b] >= r["done_ns"][a]
        # versions never go back in insert order, and rows inserted while a
        # merge of version v runs land in version v + 1
        got = [(events[i][0], int(r["version"][i])) for i in accepted if events[i][2] == t]
        assert all(a[1] <= b[1] for a, b in zip(got, got[1:]))
        for k in mine:
            a, d, v = r["admit_ns"][k], r["done_ns"][k], int(r["version_of_merge"][k])
            for i in accepted:
                if events[i][2] == t and a < events[i][0] < d:
                    assert r["version"][i] == v + 1, (events[i], v)
        # automatic merges: the delta had passed k * N_M when they started
        n_m = main_rows0[t]
        for k in mine:
            if r["automatic"][k]:
                assert r["rows"][k] > trigger[t] * n_m, (k, r["rows"][k], n_m)
            n_m += int(r["rows"][k])


def test_trigger_fires_at_the_first_crossing_and_inserts_during_a_merge_land_next():
    main_rows, k = [1000], [0.1]
    ev = steady_inserts(0, 10, 1 * MS, 60)
    events, r = run(ev, main_rows, [10**6], k, [5 * MS])
    check_invariants(events, r, main_rows, k)
    assert r["merges"] >= 3
    # the first merge starts with the insert that takes the delta past 100 rows
    assert r["admit_ns"][0] == 10 * MS and r["rows"][0] == 110 and r["automatic"][0] == 1
    # inserts at 11..14 ms arrive during it: version 2; the one at 15 ms comes
    # right after its commit, into the same (now primary) delta: version 2 too
    for t_ms in range(11, 16):
        i = t_ms
        assert events[i][0] == t_ms * MS and r["version"][i] == 2


def test_paused_table_merges_nothing_until_resumed():
    main_rows, k = [1000], [0.1]
    ev = steady_inserts(0, 10, 1 * MS, 40) + [(0, PAUSE, 0, 0), (30 * MS + 1, RESUME, 0, 0)]
    events, r = run(ev, main_rows, [10**6], k, [5 * MS])
    check_invariants(events, r, main_rows, k)
    # the trigger queued a merge at 10 ms; it starts only at the resume, with
    # every row inserted until then
    assert r["admit_ns"][0] == 30 * MS + 1
    assert r["rows"][0] == 31 * 10
    ins_ms = [e[0] for e in events if e[1] == INSERT]
    assert all(v == 1 for t, v in zip(ins_ms, r["version"][[i for i, e in enumerate(events) if e[1] == INSERT]])
               if t <= 30 * MS)


def test_full_delta_rejects_rows_whole_and_manual_merges_empty_it():
    main_rows = [500]
    ev = steady_inserts(0, 30, 1 * MS, 5)                 # 150 rows into a 100-row delta
    ev += [(10 * MS, SUBMIT, 0, 0)]                       # merge what fits
    ev += steady_inserts(0, 30, 1 * MS, 3, t0=20 * MS)     # room again after the commit
    ev += [(30 * MS, SUBMIT, 0, 0)]
    events, r = run(ev, main_rows, [100], [0.0], [2 * MS])
    check_invariants(events, r, main_rows, [0.0])
    ins = [i for i, e in enumerate(events) if e[1] == INSERT]
    got = [int(r["version"][i]) for i in ins]
    assert got == [1, 1, 1, 0, 0, 2, 2, 2]
    assert list(r["rows"][:2]) == [90, 90]
    assert not r["automatic"].any()


def test_a_request_with_an_empty_delta_commits_nothing():
    events, r = run([(1 * MS, SUBMIT, 0, 0)] + steady_inserts(0, 5, 1 * MS, 2, t0=2 * MS) +
                    [(5 * MS, SUBMIT, 0, 0)], [100], [1000], [0.0], [1 * MS])
    assert r["merges"] == 2
    assert r["rows"][0] == 0 and r["version_of_merge"][0] == 0
    assert r["rows"][1] == 10 and r["version_of_merge"][1] == 1


def test_tables_share_one_slot_and_keep_their_own_versions():
    main_rows, k = [1000, 4000], [0.05, 0.05]
    rng = np.random.default_rng(7)
    ev = []
    for t in (0, 1):
        times = np.sort(rng.integers(0, 200 * MS, 300))
        ev += [(int(x), INSERT, t, int(rng.integers(1, 20))) for x in times]
    events, r = run(ev, main_rows, [10**6, 10**6], k, [4 * MS, 9 * MS], slots=1)
    check_invariants(events, r, main_rows, k)
    # one slot: no two merges overlap
    order = np.argsort(r["admit_ns"])
    for a, b in zip(order, order[1:]):
        assert r["admit_ns"][b] >= r["done_ns"][a]
    assert sum(1 for t in r["table"] if t == 0) >= 2 and sum(1 for t in r["table"] if t == 1) >= 2
