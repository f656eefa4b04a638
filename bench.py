#!/usr/bin/env python3
"""Benchmark of the GB300 delta-to-main merge.

One step = one whole column merge (Steps 1(a), 1(b), 2(a), 2(b) of Section 5)
of one synthetic column through dm_merge_column, with inputs resident in HBM.
Default workload: 100,000,000 main rows of 8-byte values over a 1,000,000-entry
dictionary (1% unique), Zipf(1.0) codes at 20 bits; 1,000,000 delta rows with
30% new values.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
  python bench.py --impl reference ...   # the CPU oracle, as the reference arm

Multi-GPU (torchrun): every rank merges its own column (independent problems,
weak scaling); only the timing is reduced across ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from paper_1109_6885_gb300 import shard, traffic  # noqa: E402

METRIC = "merged tuples/s per column"
UNIT = "tuples/s"

WORKLOADS = {
    # 100M-row column, 8-byte values, 1% unique, Zipf(1.0) codes, 1M-row delta, 30% new
    "column-100M-u64-zipf1-delta1M": dict(n_main=100_000_000, m=1_000_000, w=8, n_delta=1_000_000,
                                          f_new=0.3, dist="zipf", zipf_s=1.0),
    # the same with 16-byte keys
    "column-100M-k16-zipf1-delta1M": dict(n_main=100_000_000, m=1_000_000, w=16,
                                          n_delta=1_000_000, f_new=0.3, dist="zipf", zipf_s=1.0),
    # the literal reading of "30% new values": every fresh delta row brings its
    # own new value (300,000 of them), so U' grows to 1.3M entries at 21 bits
    "column-100M-u64-zipf1-delta1M-300knew": dict(n_main=100_000_000, m=1_000_000, w=8,
                                                  n_delta=1_000_000, f_new=0.3, dist="zipf",
                                                  zipf_s=1.0, pool=0),
    # a narrow column: 50M rows over 8 distinct 4-byte values (3 bits), 1% delta
    "column-50M-u32-3bit-delta500k": dict(n_main=50_000_000, m=8, w=4, n_delta=500_000, f_new=0.3,
                                          dist="zipf", zipf_s=0.8),
    # the same shape at 40% of the rows (for profiler captures: a few GB on the device)
    "column-40M-u64-zipf1-delta400k": dict(n_main=40_000_000, m=400_000, w=8, n_delta=400_000,
                                           f_new=0.3, dist="zipf", zipf_s=1.0),
    # Figure 9's largest main partition: 1B rows of 8-byte values, 1% unique
    # (10M values, 24 bits), delta 1% of main (host generation takes minutes)
    "column-1B-u64-uniq1pct-delta1pct": dict(n_main=1_000_000_000, m=10_000_000, w=8, n_delta=10_000_000,
                                             f_new=0.3, dist="uniform"),
    # Figure 8's 100%-unique corner: 100M rows over 100M uint64 values (27
    # bits), delta 1% of main; X_M (400 MB) is larger than L2
    "column-100M-u64-uniq100pct-delta1pct": dict(n_main=100_000_000, m=100_000_000, w=8, n_delta=1_000_000,
                                                 f_new=0.3, dist="uniform"),
    # 1M-row column over 100k uniform uint64 values at 17 bits, 10k-row delta, half new
    "column-1M-u64-delta10k": dict(n_main=1_000_000, m=100_000, w=8, n_delta=10_000, f_new=0.5,
                                   dist="uniform", pool=0),
}
# tables: columns sharing the row counts; per column the dictionary size is
# log-uniform in [2, max_m], the value width drawn from {4, 8, 16} bytes,
# codes Zipf(0.8), the delta's new-value fraction uniform in [0, 0.5]
TABLES = {
    "table-64x8M-mixed": dict(ncols=64, n_main=8_000_000, n_delta=80_000, max_m=8_000_000),
    # 300 columns whose data repeats every 30 (each column is still merged on
    # its own, into its own outputs): host generation of 300 distinct 50M-row
    # columns would take longer than the run
    "table-300x50M-mixed": dict(ncols=300, n_main=50_000_000, n_delta=500_000, max_m=50_000_000,
                                distinct=30),
    # the shape of the sales-document table of Section 2's example: 33M rows,
    # 230 columns, a 750,000-row delta (column data repeating every 23)
    "table-230x33M-vbap": dict(ncols=230, n_main=33_000_000, n_delta=750_000, max_m=33_000_000,
                               distinct=23),
}
# served merges: resident tables of 20-60 columns, main rows log-uniform in
# [100k, 4M], delta 0.1-10% of main; Poisson arrivals at `rate` requests/s
SERVES = {
    "serve-16tables-poisson20": dict(ntables=16, cols=(20, 60), rows=(100_000, 4_000_000), rate=20.0,
                                     requests=200, slots=4, budget=16 << 30),
    "serve-16tables-burst": dict(ntables=16, cols=(20, 60), rows=(100_000, 4_000_000), rate=0.0,
                                 requests=200, slots=4, budget=16 << 30),
    # the served configuration's shape: 64 tables of 20-200 columns, main rows
    # log-uniform in [100k, 200M], delta 0.1-10%, Poisson 20 requests/s, 150 GB
    # admission budget.  Distinct data for all ~7,000 columns would need about
    # 0.5 TB, beyond HBM, so a table's columns repeat `distinct` column data
    # sets (inputs and outputs; repeats write identical bytes)
    "serve-64tables-poisson20": dict(ntables=64, cols=(20, 200), rows=(100_000, 200_000_000), rate=20.0,
                                     requests=400, slots=4, budget=150 << 30, distinct=2),
}
# the single-column sweep: main 100M rows, unique fraction x value width x
# delta size, 30% of the delta new, uniform codes, minimal widths (each point
# timed as its own column; --sweep-deltas picks the delta sizes)
SWEEPS = {
    "sweep-100M": dict(n_main=100_000_000, unique=(1e-5, 1e-3, 0.1, 1.0), widths=(4, 8, 16),
                       deltas=(0.001, 0.01, 0.1), f_new=0.3),
}
DEFAULT_WORKLOAD = "column-100M-u64-zipf1-delta1M"
L2_BYTES = 129 * 2**20


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=20)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--workload", default=DEFAULT_WORKLOAD,
                   choices=sorted(WORKLOADS) + sorted(TABLES) + sorted(SERVES) + sorted(SWEEPS))
    p.add_argument("--sweep-deltas", default="0.01",
                   help="sweep workloads: comma-separated delta sizes as fractions of main (default 0.01)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-clocks", action="store_true")
    p.add_argument("--ingest", action="store_true",
                   help="column and table workloads: also time delta ingest (Section 4) of the workload's delta "
                        "rows and report the update rate N_D / (T_U + T_M)")
    p.add_argument("--unopt", action="store_true",
                   help="column workloads: also time Step 2(b) by binary search in U' (Section 5.2) against the "
                        "translation tables")
    p.add_argument("--no-autotune", action="store_true",
                   help="table workloads: run on the library defaults instead of tuned launch choices")
    p.add_argument("--serve-slots", default=None,
                   help="served workloads: comma-separated slot counts, each timed on the same arrivals "
                        "(the first is the line's value; default: the workload's)")
    p.add_argument("--serve-flags", type=int, default=None,
                   help="served workloads: dm_merge_table flags of the served arm (default: the workload's)")
    p.add_argument("--tune-cache", default=None,
                   help="table workloads: load tuned choices from this JSON file first, save them after")
    p.add_argument("--verify", action="store_true",
                   help="table and served workloads: after the timed regions, check with device checksums "
                        "that every column's result is the same in every form (batched and plain; every served "
                        "request and the same table merged alone)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def make_column(name: str, rank: int):
    spec = synth.ColumnSpec(**WORKLOADS[name], seed=synth.column_seed(2, rank))
    return synth.make_column(spec)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, enabled: bool):
        self.proc = None
        self.path = None
        if not enabled:
            return
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def wait_ready(self, timeout: float = 1.0):
        """Wait for the first sample (or the timeout): nvidia-smi's start-up
        stalls the GPU for about a millisecond, which must not land in a
        timed region."""
        if self.proc is None:
            return
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < timeout:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        time.sleep(0.05)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def strip_comments(text: str) -> str:
    """C/C++ source without its comments, whitespace runs collapsed to one
    space (string and character literals kept as they are)."""
    out, i, n = [], 0, len(text)
    while i < n:
        ch = text[i]
        if ch in "\"'":
            j = i + 1
            while j < n and text[j] != ch:
                j += 2 if text[j] == "\\" else 1
            out.append(text[i:j + 1])
            i = j + 1
        elif text.startswith("//", i):
            j = text.find("\n", i)
            i = n if j < 0 else j
        elif text.startswith("/*", i):
            j = text.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        else:
            out.append(ch)
            i += 1
    return " ".join("".join(out).split())


def sources_digest(paths) -> str:
    """sha256 over source files with their comments removed, so that a record
    taken on a kernel stays valid across comment edits but not code edits."""
    import hashlib
    h = hashlib.sha256()
    for f in paths:
        with open(os.path.join(ROOT, f), encoding="utf-8") as fh:
            h.update(strip_comments(fh.read()).encode())
        h.update(b"\0")
    return h.hexdigest()


def recorded_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of `kernel` on `workload` from the
    committed ncu record under profiles/, or None when there is none or the
    kernel's sources (comments aside) changed since it was taken."""
    path = os.path.join(ROOT, "profiles", f"{kernel}_{workload}.traffic.json")
    try:
        rec = json.load(open(path))[kernel]
    except (OSError, ValueError, KeyError):
        return None
    try:
        digest = sources_digest(rec["sources"])
    except OSError:
        return None
    if digest != rec.get("sources_sha256") or rec.get("workload") != workload:
        return None
    return int(rec["dram_bytes_read"]) + int(rec["dram_bytes_write"])


def host_cpu():
    """The host's CPU model and logical core count (the oracle uses one of them)."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            k, _, v = line.partition(":")
            if k.strip() == "Model name" and v.strip():
                model = v.strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if model is None:
        try:
            for line in open("/proc/cpuinfo"):
                k, _, v = line.partition(":")
                if k.strip() in ("model name", "Model", "Hardware") and v.strip():
                    model = v.strip()
                    break
        except OSError:
            pass
    import platform
    return {"nproc": os.cpu_count(), "model": model or platform.machine()}


def cpu_oracle_rate(col, budget_s: float = 20.0):
    """The oracle as it stands, one host core: tuples/s over whole-column merges."""
    import oracle
    n = col.n_main + col.n_delta
    done, t0 = 0, time.perf_counter()
    while True:
        oracle.merge_synth_column(col)
        done += 1
        el = time.perf_counter() - t0
        if el > budget_s / 2 or done >= 3:
            break
    return n * done / el, done, el


def cpu_oracle_columns_rate(cols, budget_s: float = 25.0):
    """The oracle as it stands, one host core, over whole-column merges of
    `cols` in order until the budget is spent (at least one): tuple-columns/s,
    columns merged, seconds."""
    import oracle
    done, tuples, el = 0, 0, 0.0
    for col in cols:   # a generator may build each column here, outside the timing
        t0 = time.perf_counter()
        oracle.merge_synth_column(col)
        el += time.perf_counter() - t0
        done += 1
        tuples += col.n_main + col.n_delta
        if el > budget_s:
            break
    return tuples / el, done, el


def sample_column(col, rows: int):
    """The first `rows` main rows with the whole dictionaries and delta."""
    if rows >= col.n_main:
        return col
    codes = col.main_codes[:rows]
    spec = synth.ColumnSpec(**{**col.spec.__dict__, "n_main": rows})
    return synth.Column(spec, col.main_dict, codes, col.main_bits, synth.pack(codes, col.main_bits),
                        col.delta_dict, col.delta_codes)


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build_native()
    col = make_column(args.workload, 0)
    rows = col.n_main
    samp = sample_column(col, rows)
    n = samp.n_main + samp.n_delta
    for _ in range(args.warmup):
        oracle.merge_synth_column(samp)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.merge_synth_column(samp)
    el = time.perf_counter() - t0
    value = n * args.steps / el
    desc = (f"the whole workload per step: {rows:,} main rows, {col.n_delta:,} delta rows, "
            "one host thread")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": f"u{8 * col.w}" if col.w < 16 else "u128", "data": "synthetic",
        "config": {"workload": args.workload, "sample": desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": desc, "host": host_cpu()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_gpu(args):
    import torch

    from paper_1109_6885_gb300 import build
    from paper_1109_6885_gb300 import dmerge as dm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    dm.load()

    col = make_column(args.workload, rank)
    m, d, w = col.main_dict.shape[0], col.delta_dict.shape[0], col.w
    n_tuples = col.n_main + col.n_delta
    ctx = dm.Context(local)
    dcol = dm.DeviceColumn.from_numpy(w, col.main_dict, col.main_packed, col.main_bits, col.n_main,
                                      col.delta_dict, col.delta_codes)
    res = dm.alloc_result(dcol)
    ctx.reserve(dm.dm_scratch_bytes(dcol.cin()))
    cin, cout = dcol.cin(), res.cout()
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    # clock samples run from before the warm-up to after the timed region
    sampler = ClockSampler(local, not args.no_clocks)
    sampler.wait_ready()
    # warm-up with both timed loops' flags (the first call with per-kernel
    # events creates the context's event ring; also checks the result once
    # against the status word)
    for k in range(max(args.warmup, 3)):
        dm.dm_merge_column(ctx, cin, cout, stream, dm.DM_FLAG_TIMING if k % 2 else 0)
    torch.cuda.synchronize()
    st = ctx.sync_status()
    if st != dm.DM_OK:
        raise RuntimeError(f"device status {st} after warm-up")
    u, b_new = res.u_bits()

    # a column whose packed streams fit in L2 is timed cold: a write larger
    # than L2 between merges, outside each merge's events
    stream_bytes = dm.dm_packed_bytes(col.n_main, col.main_bits) + dm.dm_packed_bytes(n_tuples, b_new)
    flush = (torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
             if stream_bytes < L2_BYTES else None)

    def back_to_back():
        # K whole merges, one CUDA event per step on the launching stream
        # (per-kernel events would add gaps between the kernels)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        barrier()
        torch.cuda.synchronize()
        ev[0].record(stream)
        for k in range(args.steps):
            dm.dm_merge_column(ctx, cin, cout, stream)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        barrier()
        return [ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps)], ev[0].elapsed_time(ev[args.steps])

    def flushed():
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        barrier()
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            dm.dm_merge_column(ctx, cin, cout, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        barrier()
        per = [a.elapsed_time(b) for a, b in ev]
        return per, sum(per)

    launches0 = ctx.launches
    per_step, total_ms = back_to_back() if flush is None else flushed()
    launches = ctx.launches - launches0
    warm = None
    if flush is not None:
        wper, wtot = back_to_back()
        warm = {"value": shard.aggregate_rate(n_tuples * args.steps, wtot / 1e3, "cuda"),
                "ms_per_step": wtot / args.steps, "form": "the same merges back to back, inputs warm in L2"}
    # a second timed region of K merges with events around every kernel:
    # the per-kernel durations behind the roofline
    ctx.timing_sum()
    barrier()
    torch.cuda.synchronize()
    for k in range(args.steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        dm.dm_merge_column(ctx, cin, cout, stream, dm.DM_FLAG_TIMING)
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    phase_ms, calls = ctx.timing_sum()
    # every rank merged its own column: all ranks' tuples over the slowest rank's time
    value = shard.aggregate_rate(n_tuples * args.steps, total_ms / 1e3, "cuda")
    total_ms = 1e3 * shard.max_over_ranks(total_ms / 1e3, "cuda")

    # roofline of the dominant kernel (Step 2(b) re-encode), bytes it must move
    reencode_ms = phase_ms[3] / max(calls, 1)

    ingest = None
    if args.ingest:
        # delta ingest of the workload's delta rows in arrival order: the
        # insertion-order dictionary and codes the merge reads
        vals = dcol.delta_dict[dcol.delta_codes.long()]
        nd = col.n_delta
        igd = dm.key_tensor_empty(max(nd, 1), w)
        igc = torch.empty(max(nd, 1), dtype=torch.int32, device=f"cuda:{local}")
        igl = torch.zeros(1, dtype=torch.int64, device=f"cuda:{local}")
        dm.dm_ingest_delta(ctx, w, vals, nd, igd, igc, igl, stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        for k in range(args.steps):
            if flush is not None:
                flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            dm.dm_ingest_delta(ctx, w, vals, nd, igd, igc, igl, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ims = sorted(a.elapsed_time(b) for a, b in ev)[args.steps // 2]
        dl = int(igl.item())
        same = dl == dcol.d and bool(torch.equal(igd[:dl], dcol.delta_dict)) and \
            bool(torch.equal(igc[:nd], dcol.delta_codes))
        # the update rate of Eq. 1 / Eq. 16: the delta's rows over the time
        # to insert them (T_U, the ingest) plus the time to merge them (T_M)
        merge_ms = total_ms / args.steps
        ingest = {"rows": nd, "ms": ims, "rows_per_s": nd / (ims / 1e3), "dict": dl,
                  "same_as_the_workload_delta": same, "status": ctx.sync_status(),
                  "update_rate": {"updates_per_s": nd / ((ims + merge_ms) / 1e3), "t_u_ms": ims,
                                  "t_m_ms": merge_ms, "definition": "N_D / (T_U + T_M), Eq. 1 and Eq. 16, "
                                                                     "one column"}}

    unopt = None
    if args.unopt:
        # Step 2(b) by the unoptimised route on the same merged column: the
        # value of each tuple looked up in U' (Eq. 5) instead of X_M / X_D
        nwords = dm.dm_packed_bytes(n_tuples, b_new) // 4
        want = res.new_packed[:nwords].clone()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(args.steps)]
        dm.dm_reencode_search(ctx, cin, cout, stream)
        for k in range(args.steps):
            if flush is not None:
                flush.fill_(k & 0xFF)
            ev[k][0].record(stream)
            dm.dm_reencode_search(ctx, cin, cout, stream)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        ums = sorted(a.elapsed_time(b) for a, b in ev)[args.steps // 2]
        unopt = {"ms_per_reencode": ums, "opt_reencode_ms": reencode_ms, "tables_speedup": ums / reencode_ms,
                 "same_bytes": bool(torch.equal(want, res.new_packed[:nwords])),
                 "status": ctx.sync_status()}
    step2 = traffic.step2_bytes(col.main_bits, b_new, col.n_main, col.n_delta, m, d)
    peak, peak_kind = measured_peaks()
    achieved = step2 / (reencode_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic("reencode_kernel", args.workload),
                "kernel": "reencode_kernel<b>",
                "algorithmic_bytes": step2, "peak_source": peak_kind,
                "kernel_timing": "events around each kernel, a second timed pass of the same K merges",
                "phase_ms_avg": {
                    "step1_kernel": (phase_ms[0] + phase_ms[1] + phase_ms[2]) / max(calls, 1),
                    "reencode_2b_kernel": reencode_ms,
                    "whole": phase_ms[4] / max(calls, 1)}}
    step1 = traffic.step1_bytes(w, m, d, u)

    # end to end: host buffers through dm_merge_column_host (pinned memory)
    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(dm, ctx, col, m, d, w, u, b_new, args, world, barrier)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        rate, reps, el = cpu_oracle_rate(col)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{reps} whole-column merge(s) of this workload, {el:.1f} s, one thread",
               "host": host_cpu()}

    if rank == 0:
        ps = sorted(per_step)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(args.warmup, 3), "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": f"u{8 * w}" if w < 16 else "u128", "data": "synthetic",
            "config": {
                "workload": args.workload, "n_main": col.n_main, "dict_main": m, "value_bytes": w,
                "bits_in": col.main_bits, "n_delta": col.n_delta, "dict_delta": d, "dict_new": u,
                "bits_out": b_new, "code_dist": col.spec.dist, "zipf_s": col.spec.zipf_s,
                "f_new": col.spec.f_new, "l2": (
                    f"inputs larger than L2: each step streams {stream_bytes / 1e6:.0f} MB"
                    f" of packed codes against a {L2_BYTES / 2**20:.0f} MiB L2" if flush is None else
                    f"L2 flushed between steps (a {2 * L2_BYTES / 2**20:.0f} MiB write outside each step's"
                    f" events); each step streams {stream_bytes / 1e6:.1f} MB of packed codes"),
                "parallelism": f"{world} independent column(s), one per GPU",
                "algorithmic_bytes_per_step": step1 + step2,
            },
            "latency_ms": {"p50": ps[len(ps) // 2], "p99": ps[min(len(ps) - 1, int(0.99 * len(ps)))],
                           "min": ps[0], "max": ps[-1]},
            "roofline": roofline,
            **({"warm": warm} if warm else {}),
            **({"unopt": unopt} if unopt else {}),
            **({"ingest": ingest} if ingest else {}),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": launches,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def run_e2e(dm, ctx, col, m, d, w, u, b_new, args, world, barrier):
    import torch
    kd = dm.key_np_dtype(w)

    def pinned(a):
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int64 if a.dtype == np.uint64 else np.int32)
                             if a.size else np.zeros(1, np.int32)).pin_memory()
        return t

    h_md, h_mp = pinned(col.main_dict), pinned(col.main_packed)
    h_dd, h_dc = pinned(col.delta_dict), pinned(col.delta_codes)
    n_out = col.n_main + col.n_delta
    h_new = torch.empty(max((m + d) * (w // 4), 1), dtype=torch.int32).pin_memory()
    h_packed = torch.empty(max(dm.dm_packed_bytes(n_out, dm.dm_bits_for(m + d)) // 4, 1),
                           dtype=torch.int32).pin_memory()
    cin = dm.ColumnIn(w, h_md.data_ptr(), m, h_mp.data_ptr(), col.main_bits, col.n_main,
                      h_dd.data_ptr(), d, h_dc.data_ptr(), col.n_delta)
    cout = dm.ColumnOut(h_new.data_ptr(), h_packed.data_ptr(), None, None, None, None)
    ctx.reserve(dm.dm_host_scratch_bytes(cin))
    stream = torch.cuda.current_stream()
    for _ in range(3):
        dm.dm_merge_column_host(ctx, cin, cout, stream)
    steps = args.steps
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        uu, bb = dm.dm_merge_column_host(ctx, cin, cout, stream)
    torch.cuda.synchronize()
    barrier()
    el = shard.max_over_ranks(time.perf_counter() - t0, "cuda")
    assert (uu, bb) == (u, b_new)
    h2d = m * w + col.main_packed.nbytes + d * w + col.delta_codes.nbytes
    d2h = u * w + dm.dm_packed_bytes(n_out, b_new) + 16
    return {"value": world * n_out * steps / el, "unit": UNIT, "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * el / steps,
            "path": "dm_merge_column_host: pinned host inputs -> device, merge, results -> host"}


def table_specs(name: str):
    """Column specs of a table, the same on every rank: dictionary sizes
    log-uniform in [2, max_m], widths from {4, 8, 16}, Zipf(0.8) codes, new
    fractions uniform in [0, 0.5].  With `distinct`, column j repeats the data
    of column j mod distinct."""
    t = TABLES[name]
    rng = np.random.default_rng(0x11096885)
    specs = []
    for j in range(t.get("distinct", t["ncols"])):
        m = int(np.exp(rng.uniform(np.log(2), np.log(t["max_m"]))))
        w = int(rng.choice([4, 8, 16]))
        specs.append(synth.ColumnSpec(n_main=t["n_main"], m=m, w=w, n_delta=t["n_delta"],
                                      f_new=float(rng.uniform(0, 0.5)), dist="zipf", zipf_s=0.8,
                                      seed=synth.column_seed(4, j)))
    return [specs[j % len(specs)] for j in range(t["ncols"])]


def make_table(name: str, rank: int = 0):
    """The table's distinct columns, generated on the host."""
    specs = table_specs(name)
    return [synth.make_column(s) for s in specs[:TABLES[name].get("distinct", len(specs))]]


def run_table(args):
    """Table merges: one batched graph launch vs per-column plain launches."""
    import torch

    from paper_1109_6885_gb300 import build
    from paper_1109_6885_gb300 import dmerge as dm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    build.build()
    dm.load()
    # the table's columns are shared out over the ranks, longest first by the
    # bytes their merges move (strong scaling: the table is fixed)
    specs = table_specs(args.workload)
    nsrc = TABLES[args.workload].get("distinct", len(specs))
    costs = [shard.column_cost(sp.w, sp.m, sp.n_delta, synth.bits_for(sp.m), sp.n_main, sp.n_delta)
             for sp in specs]
    mine = shard.plan_columns(costs, world)[rank]
    srcs = {}
    for j in mine:
        k = j % nsrc
        if k not in srcs:
            c = synth.make_column(specs[k])
            srcs[k] = (c, dm.DeviceColumn.from_numpy(c.w, c.main_dict, c.main_packed, c.main_bits, c.n_main,
                                                     c.delta_dict, c.delta_codes))
    cols = [srcs[j % nsrc][0] for j in mine]
    dcols = [srcs[j % nsrc][1] for j in mine]
    ctx = dm.Context(local)
    res = [dm.alloc_result(d, with_x=False) for d in dcols]
    cins = [d.cin() for d in dcols]
    couts = [r.cout() for r in res]
    ctx.reserve(max(dm.dm_table_scratch_bytes(cins, 0), dm.dm_table_scratch_bytes(cins, dm.DM_FLAG_SERIAL)))
    stream = torch.cuda.current_stream()
    tuples = sum(c.n_main + c.n_delta for c in cols)

    def timed(flags):
        for _ in range(max(args.warmup, 3)):
            dm.dm_merge_table(ctx, cins, couts, stream, flags)
        torch.cuda.synchronize()
        if ctx.sync_status() != dm.DM_OK:
            raise RuntimeError("device status after warm-up")
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev[0].record(stream)
        for k in range(args.steps):
            dm.dm_merge_table(ctx, cins, couts, stream, flags)
            ev[k + 1].record(stream)
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        per = sorted(ev[k].elapsed_time(ev[k + 1]) for k in range(args.steps))
        total = ev[0].elapsed_time(ev[args.steps])
        rate = shard.aggregate_rate(tuples * args.steps, total / 1e3, "cuda")
        return 1e3 * shard.max_over_ranks(total / 1e3, "cuda"), per, rate

    # autotuning: the batched form on library defaults first, then every
    # column class tuned (outside the timed regions), then both forms on the
    # tuned choices
    tune = None
    if not args.no_autotune:
        t_default, _, _ = timed(0)
        cache = ctx.tune_cache
        if args.tune_cache and os.path.exists(args.tune_cache):
            cache.load(args.tune_cache)
        n0 = len(cache)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dm.dm_merge_table(ctx, cins, couts, stream, dm.DM_FLAG_AUTOTUNE)
        torch.cuda.synchronize()
        tune_s = time.perf_counter() - t0
        if args.tune_cache:
            cache.save(args.tune_cache)
        classes = {dm.dm_tune_key_of(ci).as_tuple() for ci in cins}
        tune = {"classes": len(classes), "tuned_now": len(cache) - n0, "tuning_s": tune_s,
                "defaults_ms_per_step": t_default / args.steps}
    launches0 = ctx.launches
    sampler = ClockSampler(local, not args.no_clocks)
    sampler.wait_ready()
    t_batched, per_b, rate_b = timed(0)
    clocks = sampler.stop()
    launches = (ctx.launches - launches0) // (args.steps + max(args.warmup, 3))
    t_serial, per_s, rate_s = timed(dm.DM_FLAG_SERIAL)
    verify = None
    if args.verify:
        # the last merge of each form left its results in the outputs
        dm.dm_merge_table(ctx, cins, couts, stream, 0)
        batched = dm.column_digests(cins, couts, stream)
        dm.dm_merge_table(ctx, cins, couts, stream, dm.DM_FLAG_SERIAL)
        serial = dm.column_digests(cins, couts, stream)
        torch.cuda.synchronize()
        verify = {"columns": len(cins), "batched_equals_plain": batched == serial,
                  "mismatched_columns": [j for j, (a, b) in enumerate(zip(batched, serial)) if a != b][:10],
                  "status": ctx.sync_status(), "check": "dm_column_digest of U', E'_C and the packed codes"}
    if tune is not None:
        tune["speedup_vs_defaults"] = tune["defaults_ms_per_step"] / (t_batched / args.steps)
    update = None
    if args.ingest:
        # Eq. 16's update rate for the table: its N_D delta rows over the time
        # to insert them into every column (T_U: one table ingest, the
        # columns side by side) plus the batched merge (T_M)
        n_d = TABLES[args.workload]["n_delta"]
        vals = {}
        ig_cols = []
        for j in mine:
            k = j % nsrc
            d = srcs[k][1]
            assert int(d.n_delta) == n_d
            if k not in vals:
                vals[k] = d.delta_dict[d.delta_codes.long()]
            igd = dm.key_tensor_empty(max(n_d, 1), d.w)
            igc = torch.empty(max(n_d, 1), dtype=torch.int32, device=f"cuda:{local}")
            igl = torch.zeros(1, dtype=torch.int64, device=f"cuda:{local}")
            ig_cols.append((d.w, vals[k], igd, igc, igl))
        dm.dm_ingest_table(ctx, ig_cols, n_d, stream)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
        for a_, b_ in ev:
            a_.record(stream)
            dm.dm_ingest_table(ctx, ig_cols, n_d, stream)
            b_.record(stream)
        torch.cuda.synchronize()
        t_u = sorted(a_.elapsed_time(b_) for a_, b_ in ev)[2]
        # each distinct column's ingest reproduces its delta partition
        same, seen = True, set()
        for j, (w_, _, igd, igc, igl) in zip(mine, ig_cols):
            k = j % nsrc
            if k in seen:
                continue
            seen.add(k)
            d = srcs[k][1]
            dl = int(igl.item())
            same = same and dl == d.d and bool(torch.equal(igd[:dl], d.delta_dict)) and \
                bool(torch.equal(igc[:n_d], d.delta_codes))
        t_m = t_batched / args.steps
        update = {"updates_per_s": n_d / ((t_u + t_m) / 1e3), "t_u_ms": t_u, "t_m_ms": t_m, "columns": len(mine),
                  "ingest": "dm_ingest_table: the table's columns side by side on the context's branches",
                  "same_as_the_workload_deltas": same, "status": ctx.sync_status(),
                  "definition": "N_D / (T_U + T_M), Eq. 16: T_U the table's delta ingest, T_M the batched merge"}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # every distinct column data set once: the table repeats each of them
        # equally often, so the oracle's rate over them is its rate on the table
        distinct = [srcs[k][0] for k in sorted(srcs)]
        rate, ncols_done, el = cpu_oracle_columns_rate(distinct)
        cpu = {"value": rate, "unit": "tuple-columns/s", "cores": 1, "kind": "oracle",
               "sample": f"{ncols_done} of the table's {len(distinct)} distinct columns merged once each "
                         f"({el:.1f} s, one thread); the {len(specs)} columns repeat them equally often, "
                         "so the rate is extrapolated to the table unchanged",
               "host": host_cpu()}
    step2 = 0
    for c, r in zip(cols, res):
        u, b = r.u_bits()
        step2 += traffic.step2_bytes(c.main_bits, b, c.n_main, c.n_delta, c.main_dict.shape[0],
                                     c.delta_dict.shape[0])
    pct = lambda v, q: v[min(len(v) - 1, int(q * len(v)))]
    if rank == 0:
        peak, peak_kind = measured_peaks()
        line = {
            "metric": "merged tuple-columns/s per table", "value": rate_b,
            "unit": "tuple-columns/s", "n_gpus": world, "steps": args.steps, "warmup": max(args.warmup, 3),
            "ms_per_step": t_batched / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "mixed u32/u64/u128", "data": "synthetic",
            "config": {"workload": args.workload, **TABLES[args.workload],
                       "form": "one CUDA-graph launch per table (8 branches)",
                       "launch_choices": "autotuned per column class" if tune else "library defaults",
                       "parallelism": f"the table's {len(specs)} columns shared over {world} GPU(s), longest first",
                       "l2": "inputs larger than L2"},
            "latency_ms": {"p50": pct(per_b, 0.5), "p99": pct(per_b, 0.99)},
            "serial": {"value": rate_s, "ms_per_step": t_serial / args.steps,
                       "latency_ms": {"p50": pct(per_s, 0.5), "p99": pct(per_s, 0.99)},
                       "form": "per-column plain launches, one stream"},
            "speedup_vs_serial": t_serial / t_batched,
            "step2_bytes_per_table": step2,
            "table_hbm_gbs_effective": step2 / (t_batched / args.steps / 1e3) / 1e9, "hbm_peak_gbs": peak,
            "gpu_launches": launches, "clocks": clocks,
        }
        if tune is not None:
            line["autotune"] = tune
        if verify is not None:
            line["verify"] = verify
        if update is not None:
            line["update_rate"] = update
        line["cpu_baseline"] = cpu
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def serve_specs(cfg, rank: int = 0):
    """The served workload's tables: per table (ncols, distinct column specs),
    drawn in a fixed order from one seeded generator (the same on every
    call).  Column j of a table repeats distinct column j mod len(specs)."""
    rng = np.random.default_rng(0x5E7E + rank)
    out = []
    for t in range(cfg["ntables"]):
        ncols = int(rng.integers(cfg["cols"][0], cfg["cols"][1] + 1))
        n_main = int(np.exp(rng.uniform(np.log(cfg["rows"][0]), np.log(cfg["rows"][1]))))
        n_delta = max(1, int(n_main * np.exp(rng.uniform(np.log(0.001), np.log(0.1)))))
        nsrc = min(ncols, cfg.get("distinct", ncols))
        specs = []
        for j in range(ncols):
            m = int(np.exp(rng.uniform(np.log(2), np.log(n_main))))
            spec = synth.ColumnSpec(n_main=n_main, m=m, w=int(rng.choice([4, 8, 16])), n_delta=n_delta,
                                    f_new=float(rng.uniform(0, 0.5)), dist="zipf", zipf_s=0.8,
                                    seed=synth.column_seed(5 + 1000 * rank + t, j))
            if j < nsrc:
                specs.append(spec)
        out.append((ncols, specs))
    return out


def serve_tables(dm, cfg, rank: int = 0):
    """The served workload's tables resident on the device: a list of
    (cins, couts) per table (repeated columns share inputs and outputs), the
    device buffers to keep alive as (DeviceColumn, DeviceResult) per distinct
    column, and the specs.  Columns are generated on the host by a thread
    pool (the generator is C code that releases the interpreter lock)."""
    import concurrent.futures
    specs = serve_specs(cfg, rank)
    flat = [sp for _, sps in specs for sp in sps]
    dev = []
    with concurrent.futures.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        for k in range(0, len(flat), 16):
            for c in ex.map(synth.make_column, flat[k:k + 16]):
                d = dm.DeviceColumn.from_numpy(c.w, c.main_dict, c.main_packed, c.main_bits, c.n_main,
                                               c.delta_dict, c.delta_codes)
                dev.append((d, dm.alloc_result(d, with_x=False)))
                del c
    tables, pos = [], 0
    for ncols, sps in specs:
        mine = dev[pos:pos + len(sps)]
        pos += len(sps)
        cins = [mine[j % len(sps)][0].cin() for j in range(ncols)]
        couts = [mine[j % len(sps)][1].cout() for j in range(ncols)]
        tables.append((cins, couts))
    return tables, dev, specs


def serve_verify(dm, tables, cfg, slots, flags, tabs, gaps, device):
    """Every served request's result equals its table merged alone: the
    server's per-request checksums (DM_SERVER_DIGEST) of each table merged
    by itself, then of the same arrivals served together."""
    srv = dm.Server(device, slots=slots, scratch_budget=cfg["budget"], flags=flags | dm.DM_SERVER_DIGEST)
    for t, (cins, couts) in enumerate(tables):
        srv.add_table(t, cins, couts)
    solo = []
    for t in range(len(tables)):
        rid = srv.submit(t)
        srv.drain()
        solo.append(srv.info(rid).digest)
    t0 = time.perf_counter()
    due = t0
    rids = []
    for t, g in zip(tabs, gaps):
        due += g
        while time.perf_counter() < due:
            time.sleep(0.0005)
        rids.append((int(t), srv.submit(int(t))))
    srv.drain()
    bad = [(rid, t) for t, rid in rids if srv.info(rid).status != dm.DM_OK or srv.info(rid).digest != solo[t]]
    st = srv.stats()
    srv.close()
    return {"requests": len(rids), "tables": len(tables), "mismatches": len(bad), "first_mismatches": bad[:5],
            "peak_concurrency": st.peak_concurrency,
            "check": "DM_SERVER_DIGEST per request against the table merged alone"}


def run_serve(args):
    """Served merges: Poisson (or burst) arrivals of table merges, continuous
    batching; the same arrivals again through a plain arm (one table at a
    time, per-column plain launches)."""
    import torch

    from paper_1109_6885_gb300 import build
    from paper_1109_6885_gb300 import dmerge as dm

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    build.build()
    dm.load()
    cfg = SERVES[args.workload]
    tables, keep, specs = serve_tables(dm, cfg, rank)
    rng = np.random.default_rng(0x5E7E + rank + 1)
    table_tuples = [int(sum(ci.main_rows + ci.delta_rows for ci in c)) for c, _ in tables]
    nreq = max(args.steps * 10, cfg["requests"])
    tabs = rng.integers(0, cfg["ntables"], nreq)
    gaps = rng.exponential(1.0 / cfg["rate"], nreq) if cfg["rate"] > 0 else np.zeros(nreq)

    def arm(slots, flags, clocks_on):
        srv = dm.Server(local, slots=slots, scratch_budget=cfg["budget"], flags=flags)
        for t, (cins, couts) in enumerate(tables):
            srv.add_table(t, cins, couts)
        # warm-up: one merge of every table (records their graphs)
        for t in range(cfg["ntables"]):
            srv.submit(t)
        srv.drain()
        base = srv.stats()
        sampler = ClockSampler(local, clocks_on)
        sampler.wait_ready()
        t0 = time.perf_counter()
        due = t0
        for t, g in zip(tabs, gaps):
            due += g
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                time.sleep(min(due - now, 0.002))
            srv.submit(int(t))
        srv.drain()
        wall = time.perf_counter() - t0
        clocks = sampler.stop()
        st = srv.stats()
        # latency over the timed requests only
        lat, per = [], []
        for rid in range(base.submitted, st.submitted):
            info = srv.info(rid)
            lat.append((info.done_ns - info.submit_ns) / 1e6)
            per.append((lat[-1], int(info.table_id), (info.admit_ns - info.submit_ns) / 1e6))
        lat.sort()
        per.sort(reverse=True)
        slowest = [{"table": t, "tuples": table_tuples[t], "ms": round(ms, 3), "queued_ms": round(q, 3)}
                   for ms, t, q in per[:5]]
        out = {"value": (st.tuples - base.tuples) / wall, "wall_s": wall,
               "latency_ms": {"p50": lat[len(lat) // 2], "p99": lat[min(len(lat) - 1, int(0.99 * len(lat)))],
                              "max": lat[-1]},
               "failed": st.failed - base.failed, "peak_concurrency": st.peak_concurrency,
               "peak_scratch_bytes": st.peak_scratch_bytes, "scratch_budget": st.scratch_budget,
               "clocks": clocks, "slowest": slowest}
        srv.close()
        return out

    served_flags = cfg.get("flags", 0) if args.serve_flags is None else args.serve_flags
    slot_counts = [int(x) for x in args.serve_slots.split(",")] if args.serve_slots else [cfg["slots"]]
    served = arm(slot_counts[0], served_flags, not args.no_clocks)
    sweep = []
    for k in slot_counts[1:]:
        r = arm(k, served_flags, False)
        sweep.append({"slots": k, "value": r["value"], "latency_ms": r["latency_ms"], "failed": r["failed"],
                      "peak_concurrency": r["peak_concurrency"]})
    plain = arm(1, dm.DM_FLAG_SERIAL, False)
    verify = serve_verify(dm, tables, cfg, slot_counts[0], served_flags, tabs, gaps, local) if args.verify else None
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # a seeded sample of the tables' distinct column data sets, each
        # generated on the host and merged once by the oracle
        flat = [sp for _, sps in specs for sp in sps]
        pick = np.random.default_rng(0xC0DE).permutation(len(flat))[:48]
        rate, ncols_done, el = cpu_oracle_columns_rate((synth.make_column(flat[i]) for i in pick), budget_s=15.0)
        cpu = {"value": rate, "unit": "tuple-columns/s", "cores": 1, "kind": "oracle",
               "sample": f"{ncols_done} seeded columns of the {len(flat)} distinct column data sets, merged once "
                         f"each ({el:.1f} s of merging, one thread); rate over those columns, extrapolated to "
                         "the served mix",
               "host": host_cpu()}
    if rank == 0:
        line = {
            "metric": "served merged tuple-columns/s; p50/p99 merge latency", "value": served["value"],
            "unit": "tuple-columns/s", "n_gpus": world, "steps": nreq, "warmup": cfg["ntables"],
            "ms_per_step": 1e3 * served["wall_s"] / nreq, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "mixed u32/u64/u128", "data": "synthetic",
            "config": {"workload": args.workload, **{k: v for k, v in cfg.items()},
                       "columns": sum(len(c) for c, _ in tables),
                       "tuples_per_merge_mean": float(np.mean([sum(ci.main_rows + ci.delta_rows for ci in c)
                                                               for c, _ in tables]))},
            "latency_ms": served["latency_ms"], "requests": nreq, "failed": served["failed"],
            "peak_concurrency": served["peak_concurrency"], "peak_scratch_bytes": served["peak_scratch_bytes"],
            "scratch_budget": served["scratch_budget"], "clocks": served["clocks"],
            "slots": slot_counts[0], "served_flags": served_flags, "slowest": served["slowest"],
            "plain": {"form": "one table at a time, per-column plain launches, same arrivals",
                      "value": plain["value"], "latency_ms": plain["latency_ms"], "failed": plain["failed"],
                      "slowest": plain["slowest"]},
            **({"slots_sweep": sweep} if sweep else {}),
            **({"verify": verify} if verify else {}),
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)


def time_column(dm, ctx, dcol, res, steps, warmup, flush):
    """Median-free per-kernel timing of `steps` merges of one resident column
    (L2 flushed before each when `flush` is given): (ms per merge from one
    event per step, Step 1 ms, Step 2(b) ms, device status)."""
    import torch
    cin, cout = dcol.cin(), res.cout()
    for k in range(max(warmup, 3)):
        dm.dm_merge_column(ctx, cin, cout, None, dm.DM_FLAG_TIMING if k % 2 else 0)
    torch.cuda.synchronize()
    ctx.timing_sum()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        ev[k][0].record()
        dm.dm_merge_column(ctx, cin, cout)
        ev[k][1].record()
    for k in range(steps):
        if flush is not None:
            flush.fill_(k & 0xFF)
        dm.dm_merge_column(ctx, cin, cout, None, dm.DM_FLAG_TIMING)
    torch.cuda.synchronize()
    ms, calls = ctx.timing_sum()
    whole = sum(a.elapsed_time(b) for a, b in ev) / steps
    return whole, (ms[0] + ms[1] + ms[2]) / max(calls, 1), ms[3] / max(calls, 1), ctx.sync_status()


def run_sweep(args):
    """The single-column sweep (unique fraction x value width x delta size):
    one JSON line with every point's merged tuples/s, the re-encode's
    fraction of measured HBM bandwidth and the Step 1 / Step 2(b) split."""
    import torch

    from paper_1109_6885_gb300 import build
    from paper_1109_6885_gb300 import dmerge as dm

    rank, world, local = dist_env()
    if rank != 0:
        return
    torch.cuda.set_device(local)
    build.build()
    dm.load()
    cfg = SWEEPS[args.workload]
    deltas = [float(x) for x in args.sweep_deltas.split(",")]
    peak, peak_kind = measured_peaks()
    flush = torch.empty(2 * L2_BYTES, dtype=torch.uint8, device=f"cuda:{local}")
    points = []
    sampler = ClockSampler(local, not args.no_clocks)
    sampler.wait_ready()
    for j, (lam, w, fd) in enumerate([(l, w, f) for l in cfg["unique"] for w in cfg["widths"] for f in deltas]):
        n_main = cfg["n_main"]
        m = max(1, int(round(lam * n_main)))
        if w == 4 and m > 2**31:
            continue
        spec = synth.ColumnSpec(n_main=n_main, m=m, w=w, n_delta=int(fd * n_main), f_new=cfg["f_new"],
                                dist="uniform", seed=synth.column_seed(3, j))
        col = synth.make_column(spec)
        ctx = dm.Context(local)
        dcol = dm.DeviceColumn.from_numpy(col.w, col.main_dict, col.main_packed, col.main_bits, col.n_main,
                                          col.delta_dict, col.delta_codes)
        res = dm.alloc_result(dcol, with_x=False)
        ctx.reserve(dm.dm_scratch_bytes(dcol.cin()))
        whole, s1, s2, st = time_column(dm, ctx, dcol, res, args.steps, args.warmup, flush)
        u, b_new = res.u_bits()
        d = col.delta_dict.shape[0]
        step2 = traffic.step2_bytes(col.main_bits, b_new, col.n_main, col.n_delta, m, d)
        n = col.n_main + col.n_delta
        points.append({"unique": lam, "value_bytes": w, "delta": fd, "dict_main": m, "dict_delta": d,
                       "dict_new": u, "bits_in": col.main_bits, "bits_out": b_new,
                       "tuples_per_s": n / (whole / 1e3), "ms_per_merge": whole, "step1_ms": s1,
                       "reencode_ms": s2, "reencode_frac_of_hbm": step2 / (s2 / 1e3) / 1e9 / peak,
                       "status": st})
        ctx.close()
        del dcol, res, col
        torch.cuda.empty_cache()
    clocks = sampler.stop()
    line = {"metric": "merged tuples/s per column (sweep)", "value": min(p["tuples_per_s"] for p in points),
            "unit": "tuples/s", "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/u64/u128",
            "data": "synthetic", "config": {"workload": args.workload, **{k: v for k, v in cfg.items()},
                                            "deltas": deltas, "l2": "L2 flushed before every merge"},
            "peak_gbs": peak, "peak_source": peak_kind, "points": points, "clocks": clocks}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload in SWEEPS:
        run_sweep(args)
    elif args.workload in TABLES:
        run_table(args)
    elif args.workload in SERVES:
        run_serve(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
