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
    ap.add_argument("--workload", default="mid")
    ap.add_argument("--bucket", type=int, default=8)
    ap.add_argument("--group", type=int, default=0)
    ap.add_argument("--rounds", type=int, default=32)
    ap.add_argument("--table-log2-words", type=int, default=28)
    ap.add_argument("--cpu-sample", type=int, default=3_000_000,
                    help="states the CPU baseline explores (bounded sample)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    return ap.parse_args()


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


def barrier(pg):
    if pg is not None:
        pg.barrier()


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), source="measured", sm_max_mhz=d.get("sm_max_mhz"))
    return dict(hbm_gbs=6800.0, source="fallback", sm_max_mhz=2070.0)


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


def cpu_baseline(net, sample: int) -> dict:
    import oracle
    r = oracle.explore(net, max_explored=sample)
    return {"value": round(r.states / r.seconds, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
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
            "config": {"workload": f"{args.workload} network {inputs.WORKLOADS[args.workload]}"},
            "cpu_baseline": {"value": round(v, 1), "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"each step: BFS of the {args.workload} network until {sample} "
                                       f"states explored, single thread"},
            "e2e": {"value": round(v, 1), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_ours(args, world, rank, local, pg):
    import torch
    from paper_1801_05857_gb300 import gx, inputs

    torch.cuda.set_device(local)
    net = inputs.workload(args.workload)
    h = gx.load_network(net)
    table_bytes = 4 << args.table_log2_words
    opts = gx.default_opts(bucket_words=args.bucket, group_lanes=args.group, hash_rounds=args.rounds,
                           table_bytes=table_bytes)
    ws = gx.alloc_workspace(h, opts)
    st = torch.cuda.current_stream()

    for _ in range(max(args.warmup, 0)):
        gx.explore(h, opts, ws)
    s = gx.stats(h)
    lv = gx.levels(h)

    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier(pg)
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    expand_ms, launches, probes = 0.0, 0, 0
    for _ in range(args.steps):
        gx.explore(h, opts, ws)
        si = gx.stats(h)
        expand_ms += si["expand_ms"]
        launches += si["expand_launches"]
        probes += si["probes"]
    e1.record(st)
    torch.cuda.synchronize()
    barrier(pg)
    clocks = sampler.stop() if sampler else None
    ms = e0.elapsed_time(e1)
    ms_max = max_over_ranks(ms, pg)
    s = gx.stats(h)
    states, trans = s["states"], s["transitions"]
    value = world * states * args.steps / (ms_max * 1e-3)
    tps = world * trans * args.steps / (ms_max * 1e-3)

    # roofline of the dominant kernel (level expansion)
    peaks = measured_peaks()
    s_avg = dict(s)
    s_avg["probes"] = probes // args.steps
    bytes_per_search = algorithmic_bytes(s_avg)
    exp_ms_per_search = expand_ms / args.steps
    achieved = bytes_per_search / (exp_ms_per_search * 1e-3) / 1e9
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": round(achieved / peaks["hbm_gbs"], 4), "traffic": None,
            "peak_source": peaks["source"] + " (MEASURED_PEAKS.json hbm_gbs, sequential copy)",
            "kernel": "expand_kernel", "launches_per_step": launches // args.steps,
            "avg_launch_ms": round(expand_ms / max(launches, 1), 4),
            "algorithmic_bytes_per_step": bytes_per_search,
            "probes_per_successor": round(s_avg["probes"] / max(trans, 1), 4)}
    if rank == 0:
        rp = random_access_peak(torch, gx)
        roof["random_access"] = {k: (round(v / 1e9, 3) if k.endswith("_per_s") else v)
                                 for k, v in rp.items()}
        roof["random_access_unit"] = "G accesses/s, GB/s"
        roof["probes_per_s"] = round(s_avg["probes"] / (exp_ms_per_search * 1e-3) / 1e9, 3)

    # end to end through the public API with host-resident inputs: load the network
    # description from host arrays, explore with a library-allocated workspace, read the
    # results back to the host
    e2e = None
    if not args.no_e2e:
        flat = net.flat()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h2d = d2h = 0
        for _ in range(args.steps):
            h2 = gx.load_network(flat)
            gx.explore(h2, opts, None)
            s2 = gx.stats(h2)
            gx.levels(h2)
            h2d += s2["h2d_bytes"]
            d2h += s2["d2h_bytes"] + 8 * s2["n_levels"]
            del h2
        torch.cuda.synchronize()
        wall = max_over_ranks(time.perf_counter() - t0, pg)
        e2e = {"value": round(world * states * args.steps / wall, 1), "unit": UNIT,
               "h2d_bytes_per_step": h2d // args.steps, "d2h_bytes_per_step": d2h // args.steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(net, args.cpu_sample)

    if rank == 0:
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload} network {inputs.WORKLOADS[args.workload]}",
                       "states": states, "transitions": trans, "levels": len(lv),
                       "vector_words": s["vector_words"], "bucket_words": s["bucket_words"],
                       "group_lanes": s["group_lanes"], "hash_rounds": s["hash_rounds"],
                       "table_words": 1 << args.table_log2_words, "fill": round(s["fill"], 4),
                       "l2": "1 GiB table > 129 MB L2 (no flush needed)",
                       "parallelism": "replicas" if world > 1 else "single"},
            "transitions_per_s": round(tps, 1),
            "roofline": roof,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": args.steps * (1 + launches // args.steps),
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)


def main():
    args = parse()
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
