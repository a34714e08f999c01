#!/usr/bin/env python
"""Throughput of breadth-first LTS-network exploration on GB300.

One step = one complete exploration of the mid network (10 processes x 16
local states, 2-word vectors, 4 two-party rules, ~5e7 reachable states) in a
2^28-word (1 GiB) hash table: clear the table, insert the initial state, expand
every BFS level.  The table (1 GiB) is larger than L2 (129 MB), so no L2 flush
is needed between steps.

    python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun), every rank explores its
own replica of the workload: the method does not shard, so this is "replicas
only" with no collective on the data path.  --impl reference times the CPU
oracle (test infrastructure, single-threaded) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "new states/s and transitions/s at <=75% fill"
UNIT = "states/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="scaled",
                    help="scaled (the memory-scaled configuration, 128 GiB table), scaled90, mid or tiny")
    ap.add_argument("--bucket", type=int, default=0, help="bucket words (0 = the workload's setting)")
    ap.add_argument("--group", type=int, default=0, help="lanes per bucket (0 = the workload's setting)")
    ap.add_argument("--rounds", type=int, default=0, help="hash rounds (0 = the workload's setting)")
    ap.add_argument("--table-log2-words", type=int, default=0,
                    help="log2 of the table's words (0 = the workload's setting)")
    ap.add_argument("--slice-log2", type=int, default=0)
    ap.add_argument("--nodes", type=int, default=19, help="token-ring nodes for --experiment scaled")
    ap.add_argument("--family", default="ring", choices=["ring", "product"],
                    help="--experiment scaled: token ring (--nodes) or the memory-scaled product network")
    ap.add_argument("--warp-cache", type=int, default=-1,
                    help="log2 entries of the per-warp cache of seen vectors (0 = off, -1 = automatic)")
    ap.add_argument("--level-loop", default="host", choices=["host", "device"],
                    help="main line: levels driven by the host (profilable kernel by kernel) or by "
                         "the device (one CUDA graph); the other one is timed beside it")
    ap.add_argument("--global-cache", type=int, default=-1,
                    help="log2 entries of the GPU-wide cache of seen vectors (0 = off, -1 = automatic)")
    ap.add_argument("--region-passes", type=int, default=0,
                    help="passes per level, each probing one region of the table (0 = auto: regions "
                         "of at most 64 GiB)")
    ap.add_argument("--max-levels", type=int, default=0, help="--experiment search: stop after this many levels")
    ap.add_argument("--partition-min", type=int, default=0,
                    help="partition levels with at least this many states (0 = never)")
    ap.add_argument("--cpu-sample", type=int, default=3_000_000,
                    help="states the CPU baseline explores (bounded sample)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-table", action="store_true", help="skip the Sec. 5.1 find-or-put part")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload part")
    ap.add_argument("--no-guided", action="store_true", help="skip the guided deadlock-search part")
    ap.add_argument("--probe-gib", type=int, default=128, help="--experiment probe-sweep: buffer size in GiB")
    ap.add_argument("--experiment", default="", choices=["", "table-sweep", "cuckoo-sweep", "bucket-sweep", "scaled", "scaling-table", "scorer", "batch",
                             "guided", "cache-sweep", "guided-compare", "search", "probe-sweep"],
                    help="table-sweep: Sec. 5.1 duplication x bucket sweep; bucket-sweep: the "
                         "exploration for every (bucket, group) size; scaled: one large token ring; "
                         "scaling-table: ring and producer/consumer families by size (Table 1); "
                         "scorer: the tensor-core scoring kernel alone; batch: the 256-network batch "
                         "alone; guided: one guided search with a host round trip per iteration; "
                         "cache-sweep: --workload for per-warp and GPU-wide cache sizes; "
                         "guided-compare: guided search with the scoring in its own kernel and fused "
                         "into the expansion, 12-16 processes; search: one warm-up and one timed search of "
                         "--workload (host level loop, at most --max-levels levels), for profiling; "
                         "one JSON line per point")
    args = ap.parse_args()
    wl = WORKLOAD_SETTINGS.get(args.workload, WORKLOAD_SETTINGS["mid"])
    for k in ("bucket", "group", "rounds", "table_log2_words"):
        if not getattr(args, k):
            setattr(args, k, wl[k])
    return args


# Table settings per workload: log2 of the table's uint32 words, bucket words, lanes per
# bucket, hash rounds.  The memory-scaled network fills 62.5 % of a 128 GiB table.
WORKLOAD_SETTINGS = {
    "scaled": dict(table_log2_words=35, bucket=8, group=1, rounds=64),
    "scaled90": dict(table_log2_words=35, bucket=16, group=1, rounds=64),
    "mid": dict(table_log2_words=28, bucket=8, group=1, rounds=32),
    "tiny": dict(table_log2_words=16, bucket=32, group=1, rounds=8),
}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def max_over_ranks(x: float, pg) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, pg) -> float:
    if pg is None:
        return x
    import torch
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def replica_throughput(units: float, seconds: float, pg) -> float:
    """Whole-job rate of independent replicas: the units every rank processed,
    divided by the slowest rank's time."""
    return sum_over_ranks(units, pg) / max_over_ranks(seconds, pg)


def barrier(pg):
    if pg is not None:
        pg.barrier()


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured", sm_max_mhz=d.get("sm_max_mhz"),
                    bf16_tflops_sustained=d.get("bf16_tflops_sustained"))
    return dict(hbm_gbs=6800.0, source="fallback", sm_max_mhz=2070.0, bf16_tflops_sustained=1700.0)


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx = float(parts[2])
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": mx, "samples": len(sm), "reasons": sorted(reasons)}


def kernel_code_digest(paths) -> str:
    """sha256 of kernel sources with // comments and blank lines removed: a capture stays
    valid across comment edits and is voided by any change to the code."""
    import hashlib
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p)) as f:
            for line in f:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()


def ncu_traffic(args, s: dict, probes: int, launches: int) -> dict | None:
    """DRAM bytes per launch of the expansion kernel from a committed one-kernel ncu
    capture (profiles/expand_kernel_<workload>_traffic.json), used when it was taken on
    this workload's configuration and the kernel sources have not changed since.  A
    capture of a smaller table than this run's (the size rule for counter captures) is
    scaled by algorithmic bytes: its DRAM bytes per algorithmic byte times this run's
    algorithmic bytes per launch."""
    path = os.path.join(ROOT, "profiles", f"expand_kernel_{args.workload}_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    cfg = t.get("config", {})
    if (cfg.get("bucket"), cfg.get("group"), cfg.get("warp_cache")) != (args.bucket, args.group, args.warp_cache):
        return None
    if kernel_code_digest(t["kernel_sources"]) != t["kernel_code_sha256"]:
        return None
    if "dram_bytes_per_search" in t and cfg.get("table_log2_words") == args.table_log2_words \
            and cfg.get("region_passes", 1) == s["region_passes"]:
        return {"dram_bytes_per_launch": int(t["dram_bytes_per_search"] // max(launches, 1)),
                "source": f"profiles/{os.path.basename(path)}: ncu dram__bytes_read.sum + dram__bytes_write.sum "
                          "of the same configuration, per launch"}
    ratio = t["dram_bytes_captured"] / t["algorithmic_bytes_captured"]
    alg = algorithmic_bytes(dict(s, probes=probes))
    return {"dram_bytes_per_launch": int(ratio * alg / max(launches, 1)),
            "source": f"profiles/{os.path.basename(path)}: ncu dram__bytes_read.sum + dram__bytes_write.sum "
                      f"on a {cfg.get('table_gib')} GiB table, {ratio:.3f} DRAM bytes per algorithmic byte, "
                      "scaled to this run's algorithmic bytes per launch"}


def algorithmic_bytes(s: dict) -> int:
    """Bytes the level-expansion kernels must move, per search:
    every bucket read is at least one 32-byte sector (a B-word bucket is
    ceil(4B/32) sectors); every new state costs one claimed slot (a 32-byte
    sector read-modify-write, written back) plus its frontier write; every
    explored state is read once from the frontier."""
    W = s["slot_words"]
    bucket_bytes = max(32, 4 * s["bucket_words"])
    return (s["probes"] * bucket_bytes + s["states"] * (32 + 4 * W) + s["explored"] * 4 * W)


def random_access_peak(torch, gx) -> dict:
    """Measured random-access rates over a 4 GiB buffer (the table's access pattern):
    gathers of 32 and 64 contiguous bytes and 64-bit compare-and-swaps."""
    buf = torch.zeros(1 << 30, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    n = 1 << 28
    st = torch.cuda.current_stream()
    out = {}
    for name, kind, nbytes in (("gather32", 0, 32), ("gather64", 0, 64), ("cas64", 1, 8)):
        gx.probe_random(kind, buf, n, nbytes, 7, sink)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for k in range(3):
            gx.probe_random(kind, buf, n, nbytes, 11 + k, sink)
        e1.record(st)
        torch.cuda.synchronize()
        sec = e0.elapsed_time(e1) / 3 * 1e-3
        out[name + "_per_s"] = n / sec
        # a CAS moves one 32-byte sector in and out of DRAM at best
        out[name + "_gbs"] = round(n * (nbytes if kind == 0 else 32) / sec / 1e9, 1)
    del buf
    return out


def random_access_ceiling(torch, gx, ws, s: dict) -> dict:
    """Random 32-byte read rates of this table size, over the search's own workspace
    (read only, after the timed searches): independent reads over the largest
    power-of-two span of it (the table's span), and reads confined to one region of
    that span as a region pass issues them.  The ceiling of the probes is the rate of
    the reads the kernel actually issues."""
    buf = ws.view(torch.int32)
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    n = 1 << 28
    out = {}
    span = 1
    while span * 2 <= buf.numel():
        span *= 2
    table_words = s["table_slots"] * s["slot_words"]
    regions = s["region_passes"]

    def rate(b, seed, probe):
        probe(b, seed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        for k in range(3):
            probe(b, seed + 1 + k)
        e1.record(st)
        torch.cuda.synchronize()
        return n / (e0.elapsed_time(e1) / 3 * 1e-3) / 1e9

    def persistent(b, seed):  # a grid that fits on the SMs at once, as the level kernel's does
        gx.probe_gather(b, n, 32, 32, 4, 8, 0, seed, sink)

    def turnover(b, seed):  # more CTAs than fit at once: the faster mode of the memory system
        gx.probe_random(0, b, n, 32, seed, sink)

    def waves(b, seed):  # the same gather as the ceiling, from a grid of 16 CTAs per SM
        gx.probe_gather(b, n, 32, 32, 4, 16, 0, seed, sink)

    span_t = min(span, 1 << (table_words.bit_length() - 1))
    out["independent_g_per_s"] = round(rate(buf[:span_t], 101, persistent), 3)
    out["span_gib"] = round(4 * span_t / 2 ** 30, 2)
    region_words = span_t // regions
    region = buf[:region_words]
    out["region_gib"] = round(4 * region_words / 2 ** 30, 2)
    out["in_region_g_per_s"] = round(rate(region, 201, persistent), 3) if regions > 1 else out["independent_g_per_s"]
    out["ceiling_g_per_s"] = out["in_region_g_per_s"]
    out["best_in_region_g_per_s"] = round(max(out["in_region_g_per_s"], rate(region, 301, turnover),
                                              rate(region, 401, waves)), 3)
    out["note"] = ("ceiling: 32-byte reads, 4 in flight per thread, a grid resident on the SMs at once (the "
                   "level kernel's launch style; the same rate at every depth and occupancy measured); best: "
                   "the highest rate any probe reached on the same region, from a grid with more CTAs than "
                   "fit at once (profiles/random_access_roofline.md)")
    return out


def probe_sweep(torch, gx, gib: int) -> None:
    """The random-read ceiling on one allocation of `gib` GiB (gx_probe_gather, 2^28 reads a
    launch, best of three after a warm-up): launch shape on 4 GiB, unit size, windows of the
    allocation, and page locality across all of it.  One JSON line per point."""
    buf = torch.zeros(gib << 28, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    st = torch.cuda.current_stream()
    n = 1 << 28
    gw = 1 << 28  # words per GiB

    def point(part, off_gib, span_gib, unit, load, k, ctas, g):
        b = buf[off_gib * gw:(off_gib + span_gib) * gw]
        used = gx.probe_gather(b, n, unit, load, k, ctas, g, 7, sink)
        best = 1e30
        for rep in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            gx.probe_gather(b, n, unit, load, k, ctas, g, 11 + rep, sink)
            e1.record(st)
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        print(json.dumps({"experiment": "probe-sweep", "part": part, "offset_gib": off_gib, "span_gib": span_gib,
                          "unit_bytes": unit, "load_bytes": load, "in_flight": k, "ctas_per_sm": used,
                          "group_log2": g, "g_reads_per_s": round(n / best / 1e6, 2),
                          "g_sectors_per_s": round(n * max(1, load // 32) / best / 1e6, 2)}), flush=True)

    for load in (4, 32):
        for ctas in (1, 8):
            for k in (1, 2, 4, 8, 16, 32):
                if load == 32 and k == 32:
                    continue
                point("launch shape", 0, 4, 32, load, k, ctas, 0)
    for span in (4, 64, gib):
        for unit in (32, 64, 128):
            point("unit size", 0, span, unit, unit, 2, 8, 0)
    # a grid resident at once (the level kernel's launch style) against grids of more CTAs
    # than fit, whose CTAs finish and start during the launch
    for span in (4, min(64, gib)):
        for k in (1, 4):
            for ctas in (8, 12, 16, 32):
                point("grid waves", 0, span, 32, 32, k, ctas, 0)
    for off, span in ((0, 4), (64, 4), (gib - 4, 4), (0, 32), (gib - 32, 32), (0, 64), (gib - 64, 64), (0, gib)):
        if off + span <= gib:
            point("window", off, span, 32, 4, 8, 8, 0)
    for g in (12, 16, 21, 24, 27, 30, 33):
        if (1 << g) < gib << 30:
            point("locality", 0, gib, 32, 4, 8, 8, g)
    # the same gathers through gx_probe_random (one fixed shape: 8 CTAs per SM, 4 reads in
    # flight per thread for 16- and 32-byte units, 2 for 64 and 128)
    for span in (4, min(64, gib)):
        b = buf[:span * gw]
        for nbytes in (32, 64, 128):
            gx.probe_random(0, b, n, nbytes, 3, sink)
            best = 1e30
            for rep in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                gx.probe_random(0, b, n, nbytes, 31 + rep, sink)
                e1.record(st)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            print(json.dumps({"experiment": "probe-sweep", "part": "probe_random", "offset_gib": 0, "span_gib": span,
                              "unit_bytes": nbytes, "g_reads_per_s": round(n / best / 1e6, 2)}), flush=True)
    # random compare-and-swap of 32-, 64- and 128-bit slots (the table's insertions; last,
    # since it writes the buffer)
    for span in (4, min(64, gib)):
        b = buf[:span * gw]
        for nbytes in (4, 8, 16):
            gx.probe_random(1, b, n, nbytes, 5, sink)
            best = 1e30
            for rep in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                gx.probe_random(1, b, n, nbytes, 21 + rep, sink)
                e1.record(st)
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1))
            print(json.dumps({"experiment": "probe-sweep", "part": "cas", "offset_gib": 0, "span_gib": span,
                              "unit_bytes": nbytes, "g_cas_per_s": round(n / best / 1e6, 2)}), flush=True)


def table_keys(torch, n: int, dup: int, seed: int = 0):
    """Sec. 5.1 input on the device: n one-word keys, n // dup distinct, each repeated dup times."""
    from paper_1801_05857_gb300 import inputs
    return inputs.key_sequence_device(n, dup, seed=seed)


def time_find_or_put(torch, gx, keys, words, table_words, bucket, group, rounds, reps=3):
    """Median device time of inserting every key into an empty table (Sec. 5.1), and counters."""
    st = torch.cuda.current_stream()
    table = torch.zeros(table_words, dtype=torch.int32, device="cuda")
    counters = torch.zeros(3, dtype=torch.int64, device="cuda")
    times = []
    for _ in range(reps + 1):
        table.zero_()
        counters.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        gx.find_or_put(keys, words, table, counters, None, bucket_words=bucket, group_lanes=group,
                       hash_rounds=rounds)
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times = sorted(times[1:])
    c = counters.cpu().tolist()
    del table
    return times[len(times) // 2], c


def table_point(torch, gx, keys, n, dup, words, table_words, bucket, group, rounds, gather32):
    ms, c = time_find_or_put(torch, gx, keys, words, table_words, bucket, group, rounds)
    assert c[0] == n // dup and c[2] == 0, c
    # algorithmic bytes: the key read, one sector per bucket read, one sector per claimed slot
    bucket_bytes = max(32, 4 * bucket)
    return {"keys": n, "dup": dup, "bucket_words": bucket, "group_lanes": group, "ms": round(ms, 3),
            "Gkeys_per_s": round(n / (ms * 1e-3) / 1e9, 3),
            "fill": round((n // dup) / (table_words // words), 4),
            "frac_random_gather32": round((n / (ms * 1e-3)) / gather32, 4) if gather32 else None}


def cuckoo_point(torch, gx, keys, n, dup, log2_slots, n_hash, gather32, reps=3):
    """Cuckoo find-or-put (Sec. 4.1's alternative) of the Sec. 5.1 key sequence into an
    empty table of 2^log2_slots one-word slots: median device time, and what the lost
    atomicity costs (keys reported new more than once, keys stored twice)."""
    st = torch.cuda.current_stream()
    table = torch.zeros(1 << log2_slots, dtype=torch.int32, device="cuda")
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    times = []
    for _ in range(reps + 1):
        table.zero_()
        counters.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        gx.cuckoo_find_or_put(keys, 1, table, counters, None, n_hash=n_hash)
        e1.record(st)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    times = sorted(times[1:])
    ms = times[len(times) // 2]
    ins, fnd, fail, exch = counters.cpu().tolist()
    stored = int((table != 0).sum().item())
    del table
    distinct = n // dup
    return {"table": "cuckoo", "n_hash": n_hash, "keys": n, "dup": dup, "ms": round(ms, 3),
            "Gkeys_per_s": round(n / (ms * 1e-3) / 1e9, 3), "fill": round(distinct / (1 << log2_slots), 4),
            "failed": fail, "excess_inserts": ins - distinct, "stored_twice": stored - distinct,
            "exchanges_per_insert": round(exch / max(ins, 1), 3),
            "frac_random_gather32": round((n / (ms * 1e-3)) / gather32, 4) if gather32 else None}


def table_slots_for(states: int) -> int:
    """Per-network table of the batch: a power of two of at least 4/3 of the states
    (<= 75 % fill) and 1024 slots, the rule gx_batch_opts.expected_states applies."""
    want = max(1024, (states * 4 + 2) // 3)
    return 1 << (want - 1).bit_length()


def batched_part(torch, gx, inputs, steps: int = 5) -> dict:
    """The 256-network batched workload: one graph launch (autotuned) vs one gx_explore
    per network in sequence.  A sizing pass with 2^21-slot tables counts each network's
    states; the measured runs give every network a table at <= 75 % fill."""
    nets = inputs.batch_workload()
    handles = [gx.load_network(n) for n in nets]
    b = gx.batch_create(handles)
    o0 = gx.batch_opts(hash_rounds=32, table_slots=1 << 21)
    ws0 = gx.batch_alloc_workspace(b, o0)
    gx.batch_explore(b, o0, ws0)
    counts = [gx.batch_stats(b, i)["states"] for i in range(len(nets))]
    del ws0
    torch.cuda.empty_cache()
    o = gx.batch_opts(hash_rounds=32, expected_states=counts)
    ws = gx.batch_alloc_workspace(b, o)
    tune_ms = gx.batch_autotune(b, o, ws)
    gx.batch_explore(b, o, ws)
    ts = []
    for _ in range(steps):
        gx.batch_explore(b, o, ws)
        ts.append(gx.batch_stats(b, 0)["gpu_ms"])
    ts.sort()
    states = sum(gx.batch_stats(b, i)["states"] for i in range(len(nets)))
    trans = sum(gx.batch_stats(b, i)["transitions"] for i in range(len(nets)))
    del ws
    torch.cuda.empty_cache()
    # sequential: one gx_explore per network, with the same per-network table sizes
    opts2, need = [], {}
    for h, c in zip(handles, counts):
        w = gx.layout(h)["vector_words"]
        o2 = gx.default_opts(bucket_words=max(o.bucket_words, w), group_lanes=o.group_lanes,
                             hash_rounds=32, table_bytes=table_slots_for(c) * 4 * w,
                             frontier_states=table_slots_for(c))
        opts2.append((w, o2))
        need[w] = max(need.get(w, 0), gx.workspace_bytes(h, o2))
    wss = {w: torch.empty(n, dtype=torch.uint8, device="cuda") for w, n in need.items()}
    seq_states = 0
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for h, (w, o2) in zip(handles, opts2):
        gx.explore(h, o2, wss[w])
        seq_states += gx.stats(h)["states"]
    torch.cuda.synchronize()
    seq = time.perf_counter() - t0
    med = ts[len(ts) // 2]
    bad = [i for i in range(len(nets)) if gx.batch_stats(b, i)["status"] != 0]
    return {"networks": len(nets), "states": states, "transitions": trans, "failed_networks": bad,
            "table_slots_total": sum(table_slots_for(c) for c in counts),
            "autotuned": {"bucket_words": o.bucket_words, "group_lanes": o.group_lanes,
                          "chunk_states": o.chunk_states, "tune_best_ms": round(tune_ms, 3)},
            "ms": round(med, 3), "states_per_s": round(states / (med * 1e-3), 1),
            "sequential_ms": round(seq * 1e3, 3), "sequential_states_per_s": round(seq_states / seq, 1),
            "speedup_vs_sequential": round(seq * 1e3 / med, 2)}


def guided_part(torch, gx, inputs, guide) -> dict:
    """Learned guided deadlock search vs breadth-first search on 12-16-process networks
    with planted deadlocks; the scoring network is trained on 6-8-process instances."""
    t0 = time.perf_counter()
    train_nets = [inputs.planted_network(s, n, n_traps=1 + s % 4) for s in range(6) for n in (6, 7, 8)]
    hist, label = guide.collect_examples(train_nets, 64)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    # 4000 Adam steps at lr 1e-3: over six training seeds every guide explored at most
    # 336k states at 16 processes (1500 steps at 2e-3 left one seed in six at 650k)
    params, losses = guide.train(hist, label, steps=4000, lr=1e-3)
    torch.cuda.synchronize()
    t2 = time.perf_counter()
    untrained = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
    gx.mlp_init(untrained, 99)

    def guided(net, p, fused=0):
        h = gx.load_network(net)
        gx.guided_set_weights(h, p)
        o = gx.default_opts(table_bytes=2 << 30, hash_rounds=32, guided_fused=fused)
        ws = gx.guided_alloc_workspace(h, o)
        try:
            n, _ = gx.find_deadlocks(h, gx.GX_DL_GUIDED, o, ws)
            s = gx.stats(h)
            return {"found": n, "explored": s["explored"], "stored": s["states"], "ms": round(s["gpu_ms"], 3),
                    "path_states": len(gx.guided_trace(h)), "iterations": s["expand_launches"]}
        except gx.GxError as e:
            return {"error": STATUS(e)}
        finally:
            del ws
            torch.cuda.empty_cache()

    def bfs(net, table_gib):
        h = gx.load_network(net)
        o = gx.default_opts(table_bytes=table_gib << 30, hash_rounds=32,
                            frontier_states=1 << (30 if table_gib <= 24 else 32))
        ws = gx.alloc_workspace(h, o)
        try:
            n, _ = gx.find_deadlocks(h, gx.GX_DL_BFS_FIRST, o, ws)
            s = gx.stats(h)
            return {"found": n, "explored": s["explored"], "stored": s["states"], "ms": round(s["gpu_ms"], 3),
                    "first_deadlock_level": s["first_deadlock_level"], "table_gib": table_gib,
                    "fill": round(s["fill"], 4)}
        except gx.GxError as e:
            s = gx.stats(h)
            return {"error": STATUS(e), "table_gib": table_gib, "stored": s["states"],
                    "levels_done": s["n_levels"], "ms": round(s["gpu_ms"], 3)}
        finally:
            del ws
            torch.cuda.empty_cache()

    # five seeds per size; BFS in a 24 GiB table up to 14 processes and a 128 GiB one at 16
    rows, summary = [], []
    for n, k in ((12, 2), (13, 2), (14, 2), (16, 3)):
        per = []
        for seed in range(5):
            net = inputs.planted_network(seed, n, n_traps=k)
            # the guided search is not deterministic (concurrent pushes order the bins):
            # five runs per seed; the untrained guide and BFS once
            runs = [guided(net, params) for _ in range(5)]
            fused_runs = [guided(net, params, fused=1) for _ in range(5)]
            per.append({"network": net.name, "guided_runs": runs, "fused_runs": fused_runs,
                        "untrained": guided(net, untrained),
                        "bfs": bfs(net, 24 if n <= 14 else 128)})
        rows.extend(per)

        def med(vals):
            v = sorted(vals)
            return v[len(v) // 2] if v else None

        g_runs = [x for r in per for x in r["guided_runs"] if x.get("found")]
        f_runs = [x for r in per for x in r["fused_runs"] if x.get("found")]
        summary.append({"processes": n, "planted_deadlocks": k, "seeds": 5, "guided_runs_per_seed": 5,
                        "guided_found": len(g_runs),
                        "guided_median_explored": med([x["explored"] for x in g_runs]),
                        "guided_median_ms": med([x["ms"] for x in g_runs]),
                        "guided_ms_range": [min(x["ms"] for x in g_runs), max(x["ms"] for x in g_runs)]
                        if g_runs else None,
                        "fused_found": len(f_runs),
                        "fused_median_explored": med([x["explored"] for x in f_runs]),
                        "fused_median_ms": med([x["ms"] for x in f_runs]),
                        **{f"{arm}_found": sum(1 for r in per if r[arm].get("found")) for arm in ("untrained", "bfs")},
                        **{f"{arm}_median_{key}": med([r[arm][key] for r in per if r[arm].get("found")])
                           for arm in ("untrained", "bfs") for key in ("explored", "ms")}})
    lo = losses.cpu().numpy()
    return {"train": {"networks": len(train_nets), "examples": int(hist.shape[0]),
                      "label_s": round(t1 - t0, 3), "train_s": round(t2 - t1, 3), "steps": 4000, "lr": 1e-3,
                      "ms_per_adam_step": round((t2 - t1) * 1e3 / 4000, 4), "batch": 1024,
                      "loss_first": round(float(lo[:10].mean()), 4), "loss_last": round(float(lo[-50:].mean()), 4)},
            "scoring": scoring_rate(torch, gx, params),
            "summary": summary, "instances": rows}


def scoring_rate(torch, gx, params, n=1 << 22) -> dict:
    """Throughput of the tensor-core scorer (gx_mlp_forward) on n random histograms,
    timed with CUDA events on the launching stream; FLOPs are the two layers' products
    (2 x (16 x 128 + 128 x 128) per state) plus the output dot product."""
    hist = torch.randint(0, 4, (n, 16), dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    for _ in range(3):
        gx.mlp_forward(params, hist)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    reps = 10
    e0.record(st)
    for _ in range(reps):
        gx.mlp_forward(params, hist)
    e1.record(st)
    torch.cuda.synchronize()
    sec = e0.elapsed_time(e1) * 1e-3 / reps
    flops = 2.0 * (16 * 128 + 128 * 128 + 128) * n
    pk = measured_peaks()
    peak = pk["bf16_tflops_sustained"]
    tf = flops / sec / 1e12
    return {"states": n, "ms": round(sec * 1e3, 3), "states_per_s": round(n / sec, 1),
            "tflops": round(tf, 2), "bf16_tflops_sustained": peak,
            f"frac_of_{pk['source']}": round(tf / peak, 4) if peak else None,
            "note": "each call synchronises; the scorer is bound by its CUDA-core epilogues, not the MMAs"}


def STATUS(e) -> str:
    return str(e).split(":")[0]


def host_cpu() -> dict:
    """The host's CPU model and logical core count (the oracle's single thread runs on one)."""
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.TimeoutExpired):
            pass
    import platform
    return {"cpu_model": model or platform.processor() or platform.machine(), "nproc": os.cpu_count(),
            "machine": platform.machine()}


def cpu_baseline(net, sample: int) -> dict:
    import oracle
    r = oracle.explore(net, max_explored=sample)
    return {"value": round(r.states / r.seconds, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
            "host": host_cpu(),
            "sample": f"first {len(r.levels)} BFS levels of the same network ({r.explored} states "
                      f"explored, {r.states} found) in {r.seconds:.1f} s, single thread, "
                      f"std::unordered_set"}


def run_reference(args, world, rank, pg):
    from paper_1801_05857_gb300 import inputs
    if rank != 0:
        return
    import oracle
    net = inputs.workload(args.workload)
    sample = max(100_000, args.cpu_sample // 3)
    for _ in range(args.warmup):
        oracle.explore(net, max_explored=sample // 4)
    total_states, total_s = 0, 0.0
    t0 = time.perf_counter()
    for _ in range(args.steps):
        r = oracle.explore(net, max_explored=sample)
        total_states += r.states
        total_s += r.seconds
    wall = time.perf_counter() - t0
    v = total_states / total_s
    line = {"impl": "reference", "metric": METRIC, "value": round(v, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * wall / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {net.name} {inputs.workload_params(args.workload)}"},
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": 1, "kind": "oracle", "host": host_cpu(),
                             "sample": f"each step: BFS of the {args.workload} network until {sample} "
                                       f"states explored, single thread"},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def search_opts(gx, args, host_loop: bool, table_log2_words: int | None = None):
    return gx.default_opts(bucket_words=args.bucket, group_lanes=args.group, hash_rounds=args.rounds,
                           table_bytes=4 << (table_log2_words or args.table_log2_words),
                           slice_log2=args.slice_log2, partition_min_states=args.partition_min,
                           warp_cache_log2=args.warp_cache & 0xFFFFFFFF, region_passes=args.region_passes,
                           global_cache_log2=args.global_cache & 0xFFFFFFFF, host_loop=int(host_loop))


def time_searches(torch, gx, h, opts, ws, steps: int) -> dict:
    """`steps` complete searches back to back, timed with CUDA events on the launching
    stream; the per-search counters summed over them."""
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc = dict(expand_ms=0.0, expand_launches=0, probes=0, kernel_launches=0)
    e0.record(st)
    for _ in range(steps):
        gx.explore(h, opts, ws)
        si = gx.stats(h)
        for k in acc:
            acc[k] += si[k]
    e1.record(st)
    torch.cuda.synchronize()
    acc["ms"] = e0.elapsed_time(e1)
    acc["last"] = gx.stats(h)
    return acc


def expected_counts(name: str, net):
    """Closed-form states and transitions of a product workload, else None."""
    from paper_1801_05857_gb300 import inputs
    if name in inputs.PRODUCT_WORKLOADS:
        return product_closed_form(net, inputs.PRODUCT_WORKLOADS[name]["blocks"])
    return None


def roofline_of(s: dict, t: dict, steps: int, peaks: dict) -> dict:
    """Roofline of the level-expansion kernel over `steps` timed searches."""
    s_avg = dict(s)
    s_avg["probes"] = t["probes"] // steps
    bytes_per_search = algorithmic_bytes(s_avg)
    launches = t["expand_launches"] // steps
    # the expansion kernels' time per search: the CUDA events around the timed searches
    # on their stream (the launch list gives them > 99 % of a search), so the rate is a
    # slight underestimate
    ms_search = t["ms"] / steps
    achieved = bytes_per_search / (ms_search * 1e-3) / 1e9
    return {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4),
            "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs, sequential copy)",
            "kernel": "expand_kernel", "launches_per_step": launches,
            "avg_launch_ms": round(ms_search / max(launches, 1), 4),
            "avg_launch_ms_source": "CUDA events around the timed searches on the launching stream / "
                                    "expansion launches",
            "level_timer_ms_per_step": round(t["expand_ms"] / steps, 3),
            "algorithmic_bytes_per_step": bytes_per_search,
            "algorithmic_bytes_per_launch": bytes_per_search // max(launches, 1),
            "probes_per_successor": round(s_avg["probes"] / max(s["transitions"], 1), 4),
            "probes_per_s": round(s_avg["probes"] / (ms_search * 1e-3) / 1e9, 3),
            "region_passes": s["region_passes"]}


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_1801_05857_gb300 import gx, inputs

    torch.cuda.set_device(local)
    peaks = measured_peaks()
    net = inputs.workload(args.workload)
    want = expected_counts(args.workload, net)
    h = gx.load_network(net)
    opts = search_opts(gx, args, host_loop=args.level_loop == "host")
    ws = gx.alloc_workspace(h, opts)

    for _ in range(max(args.warmup, 0)):
        gx.explore(h, opts, ws)
    lv = gx.levels(h)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(pg)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    t = time_searches(torch, gx, h, opts, ws, args.steps)
    barrier(pg)
    clocks = sampler.stop() if sampler else None
    ms = t["ms"]
    ms_max = max_over_ranks(ms, pg)
    s = t["last"]
    states, trans = s["states"], s["transitions"]
    exact = None
    if want is not None:
        exact = {"states_closed_form": want[0], "transitions_closed_form": want[1],
                 "equal": states == want[0] and trans == want[1]}
        if not exact["equal"]:
            print(json.dumps({"error": "closed-form mismatch", "states": states, "transitions": trans,
                              **exact}), flush=True)
            sys.exit(1)
    value = replica_throughput(states * args.steps, ms * 1e-3, pg)
    tps = replica_throughput(trans * args.steps, ms * 1e-3, pg)
    roof = roofline_of(s, t, args.steps, peaks)
    tr = ncu_traffic(args, s, t["probes"] // args.steps, t["expand_launches"] // args.steps)
    roof["traffic"] = tr["dram_bytes_per_launch"] if tr else None
    roof["traffic_source"] = tr["source"] if tr else "no capture for this kernel and configuration"

    other = None
    if rank == 0:
        # the random-access ceiling of this table size, measured over the search's own
        # workspace (read only): independent random reads, and reads within one region
        # of the table as a region pass issues them
        roof["random_access"] = random_access_ceiling(torch, gx, ws, s)
        roof["probes_per_s_ceiling"] = roof["random_access"]["ceiling_g_per_s"]
        roof["frac_of_random_gather32"] = round(roof["probes_per_s"] / roof["random_access"]["ceiling_g_per_s"], 4)
        roof["frac_of_best_random_gather32"] = round(
            roof["probes_per_s"] / roof["random_access"]["best_in_region_g_per_s"], 4)
        # the other level loop on the same workload and workspace
        alt = search_opts(gx, args, host_loop=args.level_loop != "host")
        gx.explore(h, alt, ws)
        ta = time_searches(torch, gx, h, alt, ws, 1 if want is not None else min(args.steps, 5))
        sa = ta["last"]
        am = ta["ms"] / max(1, (1 if want is not None else min(args.steps, 5)))
        other = {"level_loop": "host" if args.level_loop != "host" else "device (CUDA graph, conditional WHILE node)",
                 "ms_per_step": round(am, 3), "states_per_s": round(sa["states"] / (am * 1e-3), 1),
                 "kernel_launches_per_step": sa["kernel_launches"]}

    # end to end through the public API with host-resident inputs: load the network from
    # host arrays, search (on the same caller-owned workspace), read the statistics and
    # level sizes back to the host
    e2e = None
    if not args.no_e2e:
        flat = net.flat()
        k = min(args.steps, 3)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(k):
            h2 = gx.load_network(flat)
            gx.explore(h2, opts, ws)
            s2 = gx.stats(h2)
            gx.levels(h2)
            h2d += s2["h2d_bytes"]
            d2h += s2["d2h_bytes"] + 8 * s2["n_levels"]
            del h2
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        e2e = {"value": round(replica_throughput(states * k, wall, pg), 1), "unit": UNIT,
               "h2d_bytes_per_step": h2d // k, "d2h_bytes_per_step": d2h // k, "steps": k}
    del ws
    torch.cuda.empty_cache()

    mid = None
    if rank == 0 and args.workload != "mid":
        mid = mid_part(torch, gx, inputs, args, peaks)

    # Sec. 5.1: 10^8 one-word keys into a 2^27-word table (74.5 % fill at duplication 1)
    if rank == 0 and not args.no_table:
        n = 100_000_000
        rp = random_access_peak(torch, gx)
        g32 = rp["gather32_per_s"]
        pts = []
        for dup, bucket, group in ((1, 8, 1), (21, 8, 1)):
            nd = n - n % dup
            keys = table_keys(torch, nd, dup)
            pts.append(table_point(torch, gx, keys, nd, dup, 1, 1 << 27, bucket, group, 32, g32))
            del keys
        roof["find_or_put"] = {"keys": n, "key_words": 1, "table_words": 1 << 27,
                               "random_gather32_g_per_s_4gib": round(g32 / 1e9, 3), "points": pts,
                               "target": ">= 0.5 of the random-gather rate at <= 75 % fill (d = 1)"}

    batch_part = None
    if rank == 0 and not args.no_batch:
        batch_part = batched_part(torch, gx, inputs)
    guided_res = None
    if rank == 0 and not args.no_guided:
        from paper_1801_05857_gb300 import guide
        guided_res = guided_part(torch, gx, inputs, guide)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(net, args.cpu_sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {net.name} {inputs.workload_params(args.workload)}",
                       "states": states, "transitions": trans, "levels": len(lv),
                       "fan_in": round(trans / max(states, 1), 2),
                       "vector_words": s["vector_words"], "slot_words": s["slot_words"],
                       "bucket_words": s["bucket_words"], "group_lanes": s["group_lanes"],
                       "hash_rounds": s["hash_rounds"], "table_words": 1 << args.table_log2_words,
                       "table_gib": round(4 * (1 << args.table_log2_words) / 2 ** 30, 2),
                       "fill": round(s["fill"], 4), "region_passes": s["region_passes"],
                       "partitioned_levels": s["partitioned_levels"], "exact": exact,
                       "l2": f"{round(4 * (1 << args.table_log2_words) / 2 ** 30, 2)} GiB table > 129 MB L2 "
                             "(no flush needed)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "transitions_per_s": round(tps, 1),
            "roofline": roof,
            "mid_network": mid,
            "batched": batch_part,
            "guided_deadlock_search": guided_res,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": t["kernel_launches"],
            "level_loop": "device (CUDA graph, conditional WHILE node)" if s["device_levels"] else "host",
            "other_level_loop": other,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def mid_part(torch, gx, inputs, args, peaks, steps: int = 10) -> dict:
    """The mid network (10 x 16 states, 2-word vectors, 1 GiB table), the paper-sized
    configuration, timed the same way as the main line."""
    class A:
        pass
    a = A()
    for k, v in vars(args).items():
        setattr(a, k, v)
    a.workload = "mid"
    for k, v in WORKLOAD_SETTINGS["mid"].items():
        setattr(a, k, v)
    a.region_passes = 0
    net = inputs.workload("mid")
    h = gx.load_network(net)
    o = search_opts(gx, a, host_loop=True)
    ws = gx.alloc_workspace(h, o)
    for _ in range(3):
        gx.explore(h, o, ws)
    t = time_searches(torch, gx, h, o, ws, steps)
    s = t["last"]
    roof = roofline_of(s, t, steps, peaks)
    tr = ncu_traffic(a, s, t["probes"] // steps, t["expand_launches"] // steps)
    roof["traffic"] = tr["dram_bytes_per_launch"] if tr else None
    od = search_opts(gx, a, host_loop=False)
    gx.explore(h, od, ws)
    td = time_searches(torch, gx, h, od, ws, steps)
    del ws
    torch.cuda.empty_cache()
    ms = t["ms"] / steps
    return {"workload": f"mid: {net.name} {inputs.WORKLOADS['mid']}", "states": s["states"],
            "transitions": s["transitions"], "levels": s["n_levels"], "fill": round(s["fill"], 4),
            "steps": steps, "ms_per_step": round(ms, 3), "states_per_s": round(s["states"] / (ms * 1e-3), 1),
            "transitions_per_s": round(s["transitions"] / (ms * 1e-3), 1),
            "device_loop_ms_per_step": round(td["ms"] / steps, 3), "roofline": roof}


def product_closed_form(net, blocks):
    """States and transitions of inputs.product_network (its reachable set is the
    product of the blocks): every local edge fires in every combination of the other
    processes' block states, every rule once per combination of its participants'
    matching edges and of the others' block states."""
    S = 1
    for c in blocks:
        S *= c
    in_rule = [set() for _ in net.procs]
    for r in net.rules:
        for p, a in r.parts:
            in_rule[p].add(a)
    T = 0
    for p, lts in enumerate(net.procs):
        T += sum(1 for s, a, t in lts.edges if s < blocks[p] and a not in in_rule[p]) * (S // blocks[p])
    for r in net.rules:
        m, c = 1, 1
        for p, a in r.parts:
            m *= sum(1 for s, b, t in net.procs[p].edges if s < blocks[p] and b == a)
            c *= blocks[p]
        T += m * (S // c)
    return S, T




def scaled_experiment(torch, gx, inputs, args):
    """Memory-scaled exploration in a table of 2^--table-log2-words words; one line per
    level with the table fill after it, then a summary binned by fill.  --family ring:
    the token ring with --nodes nodes (2N 3^(N-1) states, 4 N^2 3^(N-2) transitions);
    --family product: the product workload --workload names (scaled or scaled90; closed
    forms above)."""
    n = args.nodes
    if args.family == "product":
        name = args.workload if args.workload in inputs.PRODUCT_WORKLOADS else "scaled90"
        net = inputs.workload(name)
        want_states, want_trans = product_closed_form(net, inputs.PRODUCT_WORKLOADS[name]["blocks"])
    else:
        net = inputs.token_ring(n)
        want_states = 2 * n * 3 ** (n - 1)
        want_trans = 4 * n * n * 3 ** (n - 2)
    h = gx.load_network(net)
    o = gx.default_opts(bucket_words=args.bucket, group_lanes=args.group, hash_rounds=args.rounds,
                        table_bytes=4 << args.table_log2_words, slice_log2=args.slice_log2,
                        partition_min_states=args.partition_min, warp_cache_log2=args.warp_cache & 0xFFFFFFFF,
                        region_passes=args.region_passes, global_cache_log2=args.global_cache & 0xFFFFFFFF)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    s = gx.stats(h)
    lv = gx.levels(h)
    prof = gx.level_profile(h)
    W = s["slot_words"]
    bucket_bytes = max(32, 4 * s["bucket_words"])
    found = 1
    bins = {}
    for k, ms in enumerate(prof["ms"]):
        new = lv[k + 1] if k + 1 < len(lv) else 0
        explored = lv[k]
        found += new
        fill = found / s["table_slots"]
        byts = prof["probes"][k] * bucket_bytes + new * (32 + 4 * W) + explored * 4 * W
        rec = {"experiment": "scaled", "level": k, "expanded": explored, "new": new, "fill_after": round(fill, 4),
               "ms": round(ms, 3), "new_states_per_s": round(new / (ms * 1e-3), 1) if ms else None,
               "algorithmic_gbs": round(byts / (ms * 1e-3) / 1e9, 1) if ms else None,
               "probes_per_successor": round(prof["probes"][k] / max(prof["transitions"][k], 1), 4)}
        print(json.dumps(rec), flush=True)
        b = min(int(fill * 10), 9)
        acc = bins.setdefault(b, [0, 0.0, 0])
        acc[0] += new
        acc[1] += ms
        acc[2] += byts
    summary = {"experiment": "scaled-summary", "network": net.name, "states": s["states"],
               "states_closed_form": want_states, "transitions": s["transitions"],
               "transitions_closed_form": want_trans, "levels": len(lv), "table_slots": s["table_slots"],
               "table_gib": round(4 * s["table_slots"] * W / 2 ** 30, 1), "fill": round(s["fill"], 4),
               "bucket_words": s["bucket_words"], "group_lanes": s["group_lanes"], "gpu_ms": round(s["gpu_ms"], 1),
               "partitioned_levels": s["partitioned_levels"], "slice_log2": args.slice_log2,
               "region_passes": s["region_passes"],
               "states_per_s": round(s["states"] / (s["gpu_ms"] * 1e-3), 1),
               "by_fill_decile": {f"{10 * b}-{10 * b + 10}%": {"new_states": v[0], "ms": round(v[1], 1),
                                                              "states_per_s": round(v[0] / (v[1] * 1e-3), 1) if v[1] else None,
                                                              "algorithmic_gbs": round(v[2] / (v[1] * 1e-3) / 1e9, 1) if v[1] else None}
                                  for b, v in sorted(bins.items())}}
    print(json.dumps(summary), flush=True)
    assert s["states"] == want_states and s["transitions"] == want_trans, "closed form mismatch"


def scaling_table(torch, gx, inputs, args):
    """Model size against throughput, as in Table 1: the token ring for N = 2..16
    (2N 3^(N-1) states, 4 N^2 3^(N-2) transitions) and Fig. 1's producer with k
    consumers for k = 1..30 (2^(k+1) states, 2^k + k 2^(k-1) + k 2^(k+1)
    transitions).  Each network is explored twice in a table of at most 50 %
    fill (the second run is reported); counts are checked against the closed forms."""
    rows = [("token_ring", n, inputs.token_ring(n), 2 * n * 3 ** (n - 1), 4 * n * n * 3 ** (n - 2))
            for n in range(2, 17)]
    rows += [("producer_consumers", k, inputs.producer_consumers(k), 2 ** (k + 1),
              2 ** k + k * 2 ** (k - 1) + k * 2 ** (k + 1)) for k in range(1, 31)]
    for family, size, net, want_s, want_t in rows:
        h = gx.load_network(net)
        W = gx.layout(h)["vector_words"]
        table = 1 << 20
        while table < 2 * want_s * 4 * W:
            table *= 2
        o = gx.default_opts(table_bytes=table, hash_rounds=args.rounds)
        ws = gx.alloc_workspace(h, o)
        for _ in range(2):
            gx.explore(h, o, ws)
        s = gx.stats(h)
        rec = {"experiment": "scaling-table", "family": family, "size": size, "processes": len(net.procs),
               "vector_words": s["vector_words"], "states": s["states"], "transitions": s["transitions"],
               "levels": s["n_levels"], "closed_form_ok": s["states"] == want_s and s["transitions"] == want_t,
               "table_gib": round(table / 2 ** 30, 3), "fill": round(s["fill"], 4), "gpu_ms": round(s["gpu_ms"], 3),
               "states_per_s": round(s["states"] / (s["gpu_ms"] * 1e-3), 1),
               "transitions_per_s": round(s["transitions"] / (s["gpu_ms"] * 1e-3), 1)}
        print(json.dumps(rec), flush=True)
        del ws
        torch.cuda.empty_cache()
        assert rec["closed_form_ok"], "closed form mismatch"


def run_experiment(args):
    """One JSON line per point; not the bench contract's line."""
    import torch
    from paper_1801_05857_gb300 import gx, inputs
    if args.experiment == "table-sweep":
        n = 100_000_000
        rp = random_access_peak(torch, gx)
        g32 = rp["gather32_per_s"]
        for dup in (1, 2, 5, 10, 21, 50, 100):
            nd = n - n % dup
            keys = table_keys(torch, nd, dup)
            for bucket in (4, 8, 16, 32):
                group = 1
                while group <= bucket:
                    pt = table_point(torch, gx, keys, nd, dup, 1, 1 << 27, bucket, group, 32, g32)
                    print(json.dumps({"experiment": "sec5.1 find-or-put", **pt}), flush=True)
                    group *= 2
            del keys
    elif args.experiment == "cuckoo-sweep":
        # Sec. 4.1's comparison: cuckoo hashing against the bucketed table on the Sec. 5.1
        # sequences (10^8 one-word keys), both in 2^27 one-word slots (74.5 % full at d = 1)
        n = 100_000_000
        rp = random_access_peak(torch, gx)
        g32 = rp["gather32_per_s"]
        for dup in (1, 2, 5, 10, 21, 50, 100):
            nd = n - n % dup
            keys = table_keys(torch, nd, dup)
            for k in (3, 4):
                print(json.dumps({"experiment": "cuckoo vs bucketed", **cuckoo_point(torch, gx, keys, nd, dup, 27, k, g32)}),
                      flush=True)
            for bucket in (4, 8):
                pt = table_point(torch, gx, keys, nd, dup, 1, 1 << 27, bucket, 1, 32, g32)
                print(json.dumps({"experiment": "cuckoo vs bucketed", "table": "bucketed", **pt}), flush=True)
            del keys
    elif args.experiment == "batch":
        # the 256-network batch alone, B=8, G=1, 32-state chunks (the autotuner's choice),
        # tables sized from a first pass: two warm-up launches, then three timed ones
        nets = inputs.batch_workload()
        b = gx.batch_create([gx.load_network(n) for n in nets])
        o0 = gx.batch_opts(hash_rounds=32, table_slots=1 << 21)
        ws0 = gx.batch_alloc_workspace(b, o0)
        gx.batch_explore(b, o0, ws0)  # sizing pass: tables at <= 75 % fill below
        counts = [gx.batch_stats(b, i)["states"] for i in range(len(nets))]
        del ws0
        torch.cuda.empty_cache()
        o = gx.batch_opts(hash_rounds=32, expected_states=counts, bucket_words=8, group_lanes=1, chunk_states=32)
        ws = gx.batch_alloc_workspace(b, o)
        for _ in range(2):
            gx.batch_explore(b, o, ws)
        ms = []
        for _ in range(3):
            gx.batch_explore(b, o, ws)
            ms.append(gx.batch_stats(b, 0)["gpu_ms"])
        states = sum(gx.batch_stats(b, i)["states"] for i in range(len(nets)))
        print(json.dumps({"experiment": "batch", "networks": len(nets), "states": states,
                          "ms": sorted(ms)[1], "states_per_s": round(states / (sorted(ms)[1] * 1e-3), 1)}), flush=True)
    elif args.experiment == "guided":
        # one guided search on planted_network(1, 14, n_traps=2) with one host round trip per
        # iteration, so that its kernels appear one by one in a launch list
        from paper_1801_05857_gb300 import guide
        train_nets = [inputs.planted_network(s, n, n_traps=1 + s % 4) for s in range(6) for n in (6, 7, 8)]
        hist, label = guide.collect_examples(train_nets, 64)
        params, _ = guide.train(hist, label, steps=4000, lr=1e-3)
        net = inputs.planted_network(1, 14, n_traps=2)
        h = gx.load_network(net)
        gx.guided_set_weights(h, params)
        o = gx.default_opts(table_bytes=2 << 30, hash_rounds=32, host_loop=1)
        ws = gx.guided_alloc_workspace(h, o)
        n, _ = gx.find_deadlocks(h, gx.GX_DL_GUIDED, o, ws)
        s = gx.stats(h)
        print(json.dumps({"experiment": "guided", "network": net.name, "found": n, "explored": s["explored"],
                          "stored": s["states"], "iterations": s["expand_launches"], "ms": round(s["gpu_ms"], 3)}),
              flush=True)
    elif args.experiment == "scorer":
        # the tensor-core scorer alone (weights from a seeded initialisation; speed does
        # not depend on their values), 4M random histograms
        p = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
        gx.mlp_init(p, 1)
        print(json.dumps({"experiment": "scorer", **scoring_rate(torch, gx, p)}), flush=True)
    elif args.experiment == "scaling-table":
        scaling_table(torch, gx, inputs, args)
    elif args.experiment == "scaled":
        scaled_experiment(torch, gx, inputs, args)
    elif args.experiment == "guided-compare":
        # the guided search's two kernel layouts on the bench's planted networks: median over
        # 5 seeds x 5 runs of states explored and time to the first deadlock
        from paper_1801_05857_gb300 import guide
        train_nets = [inputs.planted_network(s, n, n_traps=1 + s % 4) for s in range(6) for n in (6, 7, 8)]
        hist, label = guide.collect_examples(train_nets, 64)
        params, _ = guide.train(hist, label, steps=4000, lr=1e-3)
        for n, k in ((12, 2), (13, 2), (14, 2), (16, 3)):
            res = {}
            for fused in (0, 1):
                ms, ex, it = [], [], []
                for seed in range(5):
                    net = inputs.planted_network(seed, n, n_traps=k)
                    h = gx.load_network(net)
                    gx.guided_set_weights(h, params)
                    o = gx.default_opts(table_bytes=2 << 30, hash_rounds=32, guided_fused=fused)
                    ws = gx.guided_alloc_workspace(h, o)
                    for _ in range(5):
                        nf, _ = gx.find_deadlocks(h, gx.GX_DL_GUIDED, o, ws)
                        s2 = gx.stats(h)
                        if nf:
                            ms.append(s2["gpu_ms"])
                            ex.append(s2["explored"])
                            it.append(s2["expand_launches"])
                    del ws
                    torch.cuda.empty_cache()
                ms.sort(), ex.sort(), it.sort()
                res["fused" if fused else "split"] = {"found": len(ms), "median_ms": round(ms[len(ms) // 2], 3) if ms else None,
                                                      "median_explored": ex[len(ex) // 2] if ex else None,
                                                      "median_iterations": it[len(it) // 2] if it else None}
            print(json.dumps({"experiment": "guided-compare", "processes": n, **res}), flush=True)
    elif args.experiment == "search":
        net = inputs.workload(args.workload)
        h = gx.load_network(net)
        o = search_opts(gx, args, host_loop=True)
        o.max_levels = args.max_levels
        ws = gx.alloc_workspace(h, o)
        for _ in range(2):
            gx.explore(h, o, ws)
        s = gx.stats(h)
        bytes_alg = algorithmic_bytes(s)
        print(json.dumps({"experiment": "search", "workload": args.workload, "table_gib": round(4 * (1 << args.table_log2_words) / 2 ** 30, 2),
                          "levels": s["n_levels"], "expand_launches": s["expand_launches"], "states": s["states"],
                          "explored": s["explored"], "transitions": s["transitions"], "probes": s["probes"],
                          "region_passes": s["region_passes"], "fill": round(s["fill"], 4),
                          "algorithmic_bytes": bytes_alg, "gpu_ms": round(s["gpu_ms"], 3)}), flush=True)
    elif args.experiment == "probe-sweep":
        probe_sweep(torch, gx, args.probe_gib)
    elif args.experiment == "cache-sweep":
        # per-warp cache x GPU-wide cache sizes on --workload (device level loop), median of
        # --steps searches after --warmup
        net = inputs.workload(args.workload)
        h = gx.load_network(net)
        ws = None
        for wc in (0, 9):
            for gc in (0, 14, 16, 18, 20, 22, 23):
                o = search_opts(gx, args, host_loop=False)
                o.warp_cache_log2 = wc
                o.global_cache_log2 = gc
                if ws is None:
                    o2 = search_opts(gx, args, host_loop=False)
                    o2.global_cache_log2 = 26
                    ws = gx.alloc_workspace(h, o2)
                ts = []
                for _ in range(args.warmup + args.steps):
                    gx.explore(h, o, ws)
                    ts.append(gx.stats(h)["gpu_ms"])
                ts = sorted(ts[args.warmup:])
                s = gx.stats(h)
                print(json.dumps({"experiment": "cache-sweep", "workload": args.workload, "warp_cache_log2": wc,
                                  "global_cache_log2": gc, "ms_median": round(ts[len(ts) // 2], 3),
                                  "states": s["states"], "states_per_s": round(s["states"] / (ts[len(ts) // 2] * 1e-3), 1),
                                  "probes_per_successor": round(s["probes"] / s["transitions"], 4)}), flush=True)
    elif args.experiment == "bucket-sweep":
        net = inputs.workload(args.workload)
        h = gx.load_network(net)
        W = gx.layout(h)["vector_words"]
        for bucket in (4, 8, 16, 32):
            group = 1
            while bucket >= W and group <= bucket // W:
                o = gx.default_opts(bucket_words=bucket, group_lanes=group, hash_rounds=args.rounds,
                                    table_bytes=4 << args.table_log2_words,
                                    warp_cache_log2=args.warp_cache & 0xFFFFFFFF)
                ws = gx.alloc_workspace(h, o)
                ts = []
                for _ in range(args.warmup + args.steps):
                    gx.explore(h, o, ws)
                    ts.append(gx.stats(h)["gpu_ms"])
                ts = sorted(ts[args.warmup:])
                s = gx.stats(h)
                print(json.dumps({"experiment": "bucket-sweep", "workload": args.workload,
                                  "bucket_words": bucket, "group_lanes": group,
                                  "ms_median": round(ts[len(ts) // 2], 3), "states": s["states"],
                                  "probes_per_successor": round(s["probes"] / s["transitions"], 4)}),
                      flush=True)
                del ws
                torch.cuda.empty_cache()
                group *= 2


def main():
    args = parse()
    if args.experiment:
        run_experiment(args)
        return
    world, rank, local, pg = dist_setup()
    try:
        if args.impl == "reference":
            run_reference(args, world, rank, pg)
        else:
            run_ours(args, world, rank, local, pg)
    finally:
        if pg is not None:
            pg.destroy_process_group()


if __name__ == "__main__":
    main()
