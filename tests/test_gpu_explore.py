"""Parity of the CUDA exploration path with the CPU oracle (through the C ABI).

Bit-exact on: reachable-state count, transition count, every BFS level size,
deadlock count and order-free deadlock digest, and the digest of the whole
reachable set read back from the hash table.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_1801_05857_gb300 import gx, inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def run_gpu(net, **opts):
    import torch
    h = gx.load_network(net)
    o = gx.default_opts(**opts)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    torch.cuda.synchronize()
    return h, gx.stats(h), gx.levels(h), ws


def assert_parity(net, check_set=True, **opts):
    r = oracle.explore(net, deadlocks_cap=1 << 14)
    h, s, lv, ws = run_gpu(net, **opts)
    assert s["status"] == 0 and s["complete"] == 1
    assert s["states"] == r.states
    assert s["transitions"] == r.transitions
    assert lv == r.levels
    assert s["explored"] == r.explored
    assert s["deadlock_count"] == r.deadlock_count
    assert s["deadlock_sum"] == r.deadlock_sum
    assert s["deadlock_xor"] == r.deadlock_xor
    if check_set:
        c, ssum, sxor = gx.set_digest(h, ws)
        assert (c, ssum, sxor) == (r.states, r.set_sum, r.set_xor)
    if 0 < r.deadlock_count <= 1024:
        got = {tuple(x) for x in gx.deadlocks(h)}
        assert got == {tuple(x) for x in r.deadlocks}
    return s


def test_fig1(cuda):
    s = assert_parity(inputs.producer_consumers(), table_bytes=1 << 16)
    assert s["states"] == 8 and s["transitions"] == 24


@pytest.mark.parametrize("n_nodes", list(range(2, 13)))
def test_token_ring(cuda, n_nodes):
    s = assert_parity(inputs.token_ring(n_nodes), table_bytes=1 << 26)
    assert s["vector_words"] == (1 if n_nodes <= 10 else 2)


@pytest.mark.parametrize("seed", range(10))
def test_tiny_config(cuda, seed):
    # 4 processes x 8 states, out-degree 1-3 over 6 labels, 2 two-party rules; 2^16-word table, B=32
    net = inputs.random_network(seed, 4, 8, 1, 3, 6, n_sync=2, parties=2)
    assert_parity(net, table_bytes=4 << 16, bucket_words=32)


def _nets_by_width():
    return {
        1: inputs.random_network(7, 6, 8, 1, 3, 8, n_sync=2, parties=2),
        2: inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4),
        4: inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4),
    }


@pytest.mark.parametrize("W", [1, 2, 4])
def test_every_bucket_and_group_size(cuda, W):
    net = _nets_by_width()[W]
    r = oracle.explore(net)
    assert 1000 < r.states < 5_000_000
    for B in (4, 8, 16, 32):
        if B < W:
            continue
        G = 1
        while G <= B // W and G <= 32:
            h, s, lv, ws = run_gpu(net, bucket_words=B, group_lanes=G, hash_rounds=32,
                                   table_bytes=1 << 26)
            assert s["slot_words"] == W
            assert (s["states"], s["transitions"], lv) == (r.states, r.transitions, r.levels), (B, G)
            assert (s["deadlock_count"], s["deadlock_sum"]) == (r.deadlock_count, r.deadlock_sum)
            G *= 2


@pytest.mark.parametrize("net", [
    inputs.random_network(s, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4) for s in range(3)] + [
    inputs.random_network(0, 20, 16, 1, 3, 20, n_sync=8, parties=3, cluster=2)], ids=lambda n: n.name)
def test_three_party_four_words(cuda, net):
    s = assert_parity(net, table_bytes=1 << 26)
    assert s["slot_words"] == 4


@pytest.mark.parametrize("seed", range(8))
def test_deadlock_networks(cuda, seed):
    net = inputs.random_network(seed, 8, 8, 0, 2, 10, n_sync=4, parties=2)
    assert_parity(net, table_bytes=1 << 22)
    net = inputs.random_network(seed, 4, 5, 0, 2, 6, n_sync=2, parties=2)
    assert_parity(net, table_bytes=1 << 22)


def test_bfs_first_deadlock_mode(cuda):
    checked = 0
    for seed in range(30):
        net = inputs.random_network(seed, 4, 5, 0, 2, 6, n_sync=2, parties=2)
        r = oracle.explore(net, stop_at_first_deadlock=True)
        if r.deadlock_count == 0:
            continue
        h = gx.load_network(net)
        o = gx.default_opts(table_bytes=1 << 22)
        ws = gx.alloc_workspace(h, o)
        n, states = gx.find_deadlocks(h, gx.GX_DL_BFS_FIRST, o, ws)
        s = gx.stats(h)
        assert n == r.deadlock_count
        assert s["first_deadlock_level"] == r.first_deadlock_level
        assert gx.levels(h) == r.levels
        assert s["explored"] == r.explored and s["transitions"] == r.transitions
        assert {tuple(x) for x in states} == {tuple(x) for x in r.deadlocks}
        # every reported state is a reachable deadlock: no successor in the oracle
        for x in states:
            assert len(oracle.successors(net, x)) == 0
        checked += 1
    assert checked >= 3


def test_table_full_is_reported(cuda):
    h = gx.load_network(inputs.token_ring(8))
    o = gx.default_opts(table_bytes=4096, bucket_words=8)
    ws = gx.alloc_workspace(h, o)
    with pytest.raises(gx.GxError) as e:
        gx.explore(h, o, ws)
    assert e.value.status == gx.GX_ERR_TABLE_FULL
    s = gx.stats(h)
    assert s["complete"] == 0 and s["status"] == gx.GX_ERR_TABLE_FULL


def test_frontier_overflow_is_reported(cuda):
    h = gx.load_network(inputs.token_ring(9))
    o = gx.default_opts(table_bytes=1 << 24, frontier_states=64)
    ws = gx.alloc_workspace(h, o)
    with pytest.raises(gx.GxError) as e:
        gx.explore(h, o, ws)
    assert e.value.status == gx.GX_ERR_FRONTIER_OVERFLOW


def test_workspace_too_small_and_library_allocation(cuda):
    import torch
    net = inputs.token_ring(6)
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 20)
    small = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(gx.GxError) as e:
        gx.explore(h, o, small)
    assert e.value.status == gx.GX_ERR_OOM
    gx.explore(h, o, None)  # library-owned workspace
    assert gx.stats(h)["states"] == 2 * 6 * 3 ** 5


def test_repeated_runs_identical(cuda):
    net = inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4)
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 26)
    ws = gx.alloc_workspace(h, o)
    out = []
    for _ in range(3):
        gx.explore(h, o, ws)
        s = gx.stats(h)
        out.append((s["states"], s["transitions"], tuple(gx.levels(h)), gx.set_digest(h, ws)))
    assert out[0] == out[1] == out[2]


def _golden_case(name):
    path = os.path.join(GOLDEN, name)
    if not os.path.exists(path):
        pytest.skip(f"{name} not generated")
    with open(path) as f:
        return json.load(f)


@pytest.mark.parametrize("bucket", [32, 16, 8, 4])
def test_mid_config_against_stored_oracle(cuda, bucket):
    """Mid network (10 x 16 states, 2-word vectors, 12 labels with 4 two-party rules),
    2^28-word table; expected values written by tests/golden/make_golden.py (oracle only)."""
    g = _golden_case("mid_network.json")
    net = inputs.random_network(**g["generator"])
    h, s, lv, ws = run_gpu(net, table_bytes=4 << 28, bucket_words=bucket, hash_rounds=32)
    assert s["states"] == g["states"]
    assert s["transitions"] == g["transitions"]
    assert lv == g["levels"]
    assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"]) == (
        g["deadlock_count"], g["deadlock_sum"], g["deadlock_xor"])
    assert gx.set_digest(h, ws) == (g["states"], g["set_sum"], g["set_xor"])
    assert s["fill"] <= 0.75


def test_large_irregular_network_with_the_global_cache(cuda):
    """The same 1.08e8-state network (16 fields of 4 bits: a 64-bit cache key) with
    the GPU-wide cache (2^23 entries) and two region passes: exact against the stored
    oracle values, with fewer bucket reads than without the cache."""
    g = _golden_case("large3_network.json")
    net = inputs.random_network(**g["generator"])
    runs = {}
    for log2 in (0, 23):
        h, s, lv, ws = run_gpu(net, table_bytes=4 << 30, bucket_words=16, hash_rounds=32, region_passes=2,
                               global_cache_log2=log2, warp_cache_log2=0)
        assert s["global_cache_entries"] == (1 << log2 if log2 else 0)
        assert (s["states"], s["transitions"], lv) == (g["states"], g["transitions"], g["levels"])
        assert gx.set_digest(h, ws) == (g["states"], g["set_sum"], g["set_xor"])
        runs[log2] = s["probes"]
        del ws
    assert runs[23] < runs[0]


def _part_nets():
    return [inputs.token_ring(11),
            inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4),
            inputs.random_network(7, 6, 8, 1, 3, 8, n_sync=2, parties=2),
            inputs.random_network(6, 8, 8, 0, 2, 10, n_sync=4, parties=2)]


@pytest.mark.parametrize("net", _part_nets(), ids=lambda n: n.name)
@pytest.mark.parametrize("slices,buf", [(1, 0), (3, 40000), (6, 0), (4, 20000)])
def test_partitioned_path(cuda, net, slices, buf):
    """Every level through the count / scatter / slice-ordered probe passes; a small
    successor buffer splits levels into several batches."""
    s = assert_parity(net, table_bytes=1 << 25, slice_log2=slices, successor_buffer=buf,
                      partition_min_states=1)
    assert s["partitioned_levels"] > 0


def test_partitioned_buffer_too_small_falls_back(cuda):
    """A level whose CTA ranges produce more successors than the buffer holds is
    expanded by the direct kernel instead; results stay exact."""
    s = assert_parity(inputs.token_ring(10), table_bytes=1 << 22, slice_log2=2, successor_buffer=1,
                      partition_min_states=1)
    assert s["partitioned_levels"] < s["n_levels"] - 1  # only levels with one successor fit


@pytest.mark.parametrize("cache_log2", [4, 9, 11])
@pytest.mark.parametrize("net", [inputs.token_ring(10), inputs.token_ring(12),
                                 inputs.random_network(7, 6, 8, 1, 3, 8, n_sync=2, parties=2),
                                 inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4),
                                 inputs.random_network(6, 8, 8, 0, 2, 10, n_sync=4, parties=2)],
                         ids=lambda n: n.name)
def test_warp_cache_keeps_results_exact(cuda, net, cache_log2):
    """The per-warp cache of seen vectors only skips lookups; every count stays exact
    (a 16-entry cache is overwritten all the time, a 4096-entry one rarely)."""
    for B, G in ((8, 1), (16, 2)):
        assert_parity(net, table_bytes=1 << 27, bucket_words=B, group_lanes=G, hash_rounds=32,
                      warp_cache_log2=cache_log2)


def test_warp_cache_too_large_is_rejected(cuda):
    h = gx.load_network(inputs.token_ring(12))
    o = gx.default_opts(table_bytes=1 << 27, warp_cache_log2=12)
    with pytest.raises(gx.GxError) as e:
        gx.explore(h, o, gx.alloc_workspace(h, o))
    assert e.value.status == gx.GX_ERR_INVALID and "shared memory" in e.value.message


@pytest.mark.parametrize("host_loop", [1, 0])
def test_mid_config_in_the_benchmark_configuration(cuda, host_loop):
    """The mid network exactly as bench.py times it (2^28-word table, B=8, G=1, 2^9-entry
    warp caches, 32 hash-constant sets; the host level loop of its main line, and the
    device loop it times beside it) against the stored oracle values."""
    g = _golden_case("mid_network.json")
    net = inputs.random_network(**g["generator"])
    h, s, lv, ws = run_gpu(net, table_bytes=4 << 28, bucket_words=8, group_lanes=1, hash_rounds=32,
                           warp_cache_log2=9, host_loop=host_loop)
    assert (s["states"], s["transitions"], lv) == (g["states"], g["transitions"], g["levels"])
    assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"]) == (
        g["deadlock_count"], g["deadlock_sum"], g["deadlock_xor"])
    assert gx.set_digest(h, ws) == (g["states"], g["set_sum"], g["set_xor"])
    assert s["device_levels"] == (0 if host_loop else s["n_levels"])


@pytest.mark.parametrize("k", [1, 2, 7, 16, 22])
def test_producer_consumers_family(cuda, k):
    """Fig. 1 with k consumers: 2^(k+1) states and 2^k + k 2^(k-1) + k 2^(k+1)
    transitions (closed form; pinned against the oracle up to k = 10)."""
    net = inputs.producer_consumers(k)
    if k <= 10:
        s = assert_parity(net, table_bytes=1 << 24)
    else:
        _, s, _, _ = run_gpu(net, table_bytes=1 << 27)
    assert s["states"] == 2 ** (k + 1)
    assert s["transitions"] == 2 ** k + k * 2 ** (k - 1) + k * 2 ** (k + 1)
    assert s["deadlock_count"] == 0 and s["complete"] == 1


def _chain(n):
    """One process walking a path of n local states: n BFS levels, the last state a deadlock."""
    return inputs.Network(1, [inputs.LTS(n, 0, [(i, 0, i + 1) for i in range(n - 1)])], [],
                          name=f"chain_{n}")


@pytest.mark.parametrize("n", [4095, 4096, 4097, 6000])
def test_device_loop_hands_over_to_the_host_after_4096_levels(cuda, n):
    """The device-driven level loop records 4096 levels at most; the host loop
    carries on from there with the same results."""
    s = assert_parity(_chain(n), table_bytes=1 << 20)
    assert s["n_levels"] == n and s["first_deadlock_level"] == n - 1
    assert s["device_levels"] == min(n, 4095)
    assert len(gx.level_profile(run_gpu(_chain(n), table_bytes=1 << 20)[0])["ms"]) == n


@pytest.mark.parametrize("net", [inputs.token_ring(7), inputs.random_network(6, 8, 8, 0, 2, 10, n_sync=4, parties=2),
                                 inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4)],
                         ids=lambda n: n.name)
def test_host_and_device_level_loops_agree(cuda, net):
    h1, s1, lv1, _ = run_gpu(net, table_bytes=1 << 24)
    h2, s2, lv2, _ = run_gpu(net, table_bytes=1 << 24, host_loop=1)
    assert s1["device_levels"] == s1["n_levels"] and s2["device_levels"] == 0
    assert lv1 == lv2
    # bucket reads are not compared: warp-cache hits depend on which warp takes which state
    for k in ("states", "transitions", "explored", "deadlock_count", "deadlock_sum", "deadlock_xor",
              "first_deadlock_level", "complete"):
        assert s1[k] == s2[k], k
    p1, p2 = gx.level_profile(h1), gx.level_profile(h2)
    assert p1["transitions"] == p2["transitions"] and len(p1["ms"]) == len(p2["ms"])
    assert s1["kernel_launches"] == 2 + 2 * s1["expand_launches"]
    assert s2["kernel_launches"] == 1 + s2["expand_launches"]


def test_device_loop_max_levels_and_repeated_graph_launches(cuda):
    """max_levels stops the device loop; the cached graph is rebuilt when the
    options change and reused when they do not."""
    net = inputs.token_ring(8)
    r = oracle.explore(net)
    for lim in (1, 5, 20):
        _, s, lv, _ = run_gpu(net, table_bytes=1 << 22, max_levels=lim)
        assert s["explored"] == sum(r.levels[:lim]) and lv == r.levels[:lim + 1]
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 22)
    ws = gx.alloc_workspace(h, o)
    for _ in range(3):
        gx.explore(h, o, ws)
        assert gx.stats(h)["states"] == r.states


def _product_closed_form(net, blocks):
    from test_oracle import product_closed_form
    return product_closed_form(net, blocks)


@pytest.mark.parametrize("seed,n,ns,blocks", [
    (0, 8, 16, [2, 3, 2, 3, 2, 2, 3, 2]),              # 1 word
    (1, 16, 16, [2] * 12 + [3] * 4),                   # 3 words -> 4-word slots, 3.3e5 states
    (2, 20, 16, [2] * 16 + [3, 3, 4, 4]),              # 4-word slots, 9.4e6 states
    (3, 16, 64, [3] * 10 + [2] * 6)])                  # 6 bits a process, 4-word slots, 3.8e6 states
def test_product_family_against_closed_forms(cuda, seed, n, ns, blocks):
    """The memory-scaled family (3-party rules on 10 % of the labels): states and
    transitions equal the closed forms pinned on the oracle; the first
    instance is also checked level by level against the oracle."""
    net = inputs.product_network(seed, n, ns, blocks)
    S, T = _product_closed_form(net, blocks)
    if S < 10 ** 5:
        s = assert_parity(net, table_bytes=1 << 24)
    else:
        _, s, _, _ = run_gpu(net, table_bytes=1 << 30, bucket_words=32, hash_rounds=32)
    assert (s["states"], s["transitions"], s["deadlock_count"], s["complete"]) == (S, T, 0, 1)


def test_memory_scaled_network_in_a_128_gib_table(cuda):
    """The bench's main workload in its configuration: 5.37e9 states in 2^33 4-word slots
    (128 GiB), 8-word buckets, one lane per bucket, 64 hash rounds, two region passes with
    the queued kernel, and every hash round after the first inside round 0's 64 GiB span
    (the only table size at which that rule changes the probe sequence).  States and
    transitions equal the product family's closed forms, the level sizes add up to them,
    and the table holds each state once."""
    import torch
    free, _ = torch.cuda.mem_get_info()
    if free < (170 << 30):
        pytest.skip("needs 170 GiB of free device memory")
    blocks = inputs.workload_params("scaled")["blocks"]
    net = inputs.workload("scaled")
    S, T = _product_closed_form(net, blocks)
    h, s, lv, ws = run_gpu(net, table_bytes=4 << 35, bucket_words=8, group_lanes=1, hash_rounds=64)
    assert s["region_passes"] == 2 and s["complete"] == 1 and s["slot_words"] == 4
    assert (s["states"], s["transitions"]) == (S, T)
    assert sum(lv) == S
    count = gx.set_digest(h, ws)[0]
    del ws
    torch.cuda.empty_cache()  # hand the 160 GiB back before the next test
    assert count == S


@pytest.mark.parametrize("passes", [2, 4, 16])
@pytest.mark.parametrize("host_loop", [1, 0])
@pytest.mark.parametrize("net", [inputs.token_ring(11), inputs.workload("tiny"),
                                 inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4),
                                 inputs.random_network(6, 8, 8, 0, 2, 10, n_sync=4, parties=2)],
                         ids=lambda n: n.name)
def test_region_passes_are_exact(cuda, net, passes, host_loop):
    """Region passes (each level expanded once per table region, a pass probing only
    the successors whose first bucket is in its region) give the oracle's results
    bit for bit: counts, levels, deadlock and set digests, in both level loops."""
    s = assert_parity(net, table_bytes=1 << 25, region_passes=passes, host_loop=host_loop)
    assert s["region_passes"] == passes
    assert s["expand_launches"] == passes * (s["n_levels"])


def test_region_passes_with_full_buckets_and_the_safety_check(cuda):
    """At high fill a vector's later hash rounds leave its region; the safety check
    and the transition count are taken in the first pass only."""
    net = inputs.token_ring(9)
    r = oracle.explore(net, watch=(3, 4))
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 19, hash_rounds=64, bucket_words=4, region_passes=8,
                        watch=1, watch_proc=3, watch_state=4)
    gx.explore(h, o, gx.alloc_workspace(h, o))
    s = gx.stats(h)
    assert s["fill"] > 0.8
    assert (s["states"], s["transitions"], gx.levels(h)) == (r.states, r.transitions, r.levels)
    assert (s["violation_count"], s["violation_sum"], s["violation_xor"], s["first_violation_level"]) == \
        (r.violation_count, r.violation_sum, r.violation_xor, r.first_violation_level)


def test_region_passes_are_validated(cuda):
    h = gx.load_network(inputs.token_ring(5))
    for bad in (3, 32):
        with pytest.raises(gx.GxError) as e:
            gx.explore(h, gx.default_opts(table_bytes=1 << 20, region_passes=bad), None)
        assert e.value.status == gx.GX_ERR_INVALID
    o = gx.default_opts(table_bytes=1 << 20)
    gx.explore(h, o, None)
    assert gx.stats(h)["region_passes"] == 1  # auto: tables up to 64 GiB take one pass


@pytest.mark.parametrize("log2", [0, 4, 12, 20])
@pytest.mark.parametrize("host_loop", [1, 0])
@pytest.mark.parametrize("net", [inputs.token_ring(11), inputs.workload("tiny"),
                                 inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4),
                                 inputs.random_network(6, 8, 8, 0, 2, 10, n_sync=4, parties=2)],
                         ids=lambda n: n.name)
def test_global_cache_keeps_results_exact(cuda, net, log2, host_loop):
    """The GPU-wide cache of seen vectors (2^0 entries: every vector fights for one;
    2^20: the default) only skips probes of vectors already in the table, so the
    results equal the oracle's; with it on, fewer buckets are read."""
    s = assert_parity(net, table_bytes=1 << 25, global_cache_log2=log2, host_loop=host_loop, warp_cache_log2=0)
    assert s["global_cache_entries"] == (1 << log2 if log2 else 0)


@pytest.mark.parametrize("passes", [2, 4])
@pytest.mark.parametrize("net", [inputs.token_ring(11), inputs.workload("tiny"),
                                 inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4)],
                         ids=lambda n: n.name)
def test_global_cache_with_region_passes(cuda, net, passes):
    """1- and 2-word vectors with the GPU-wide cache and region passes together (the
    queued kernel filters by region first, then by the cache; every pass reads the cache
    that earlier passes filled): exact against the oracle."""
    s = assert_parity(net, table_bytes=1 << 25, bucket_words=8, group_lanes=1, region_passes=passes,
                      global_cache_log2=20, warp_cache_log2=0)
    assert s["region_passes"] == passes and s["global_cache_entries"] == 1 << 20


def test_global_cache_reads_fewer_buckets_and_ignores_wide_4_word_vectors(cuda):
    """Fewer bucket reads with the cache; 4-word vectors whose fields take more than
    64 bits (13 processes x 6 bits) have no 64-bit key and run without it."""
    net = inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4)
    base = assert_parity(net, table_bytes=1 << 25, global_cache_log2=0, warp_cache_log2=0)
    with_cache = assert_parity(net, table_bytes=1 << 25, global_cache_log2=20, warp_cache_log2=0)
    assert with_cache["probes"] < 0.8 * base["probes"]
    s4 = assert_parity(inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4),
                       table_bytes=1 << 25, global_cache_log2=20)
    assert s4["slot_words"] == 4 and s4["global_cache_entries"] == 0


@pytest.mark.parametrize("log2", [4, 12, 20])
@pytest.mark.parametrize("bucket,group", [(16, 1), (32, 8)])
@pytest.mark.parametrize("net", [
    inputs.random_network(1, 15, 16, 1, 3, 16, n_sync=8, parties=3, cluster=4),   # 60 field bits
    inputs.product_network(1, 16, 16, [2] * 12 + [3] * 4)],                        # 64 field bits
    ids=lambda n: n.name)
def test_global_cache_keeps_4_word_results_exact(cuda, net, log2, bucket, group):
    """4-word vectors (3 words of fields) whose fields fit 64 bits use the GPU-wide
    cache with their field bits packed into one key; with one lane per bucket and
    with 8 lanes per 32-word bucket, the results equal the oracle's."""
    s = assert_parity(net, table_bytes=1 << 25, bucket_words=bucket, group_lanes=group,
                      global_cache_log2=log2, warp_cache_log2=0)
    assert s["slot_words"] == 4 and s["group_lanes"] == group
    assert s["global_cache_entries"] == 1 << log2


@pytest.mark.parametrize("bucket", [4, 8])
@pytest.mark.parametrize("passes", [2, 4])
@pytest.mark.parametrize("caches", [dict(), dict(warp_cache_log2=0), dict(global_cache_log2=20, warp_cache_log2=0),
                                    dict(global_cache_log2=12, warp_cache_log2=4)], ids=["auto", "none", "global", "both"])
def test_queued_four_word_kernel_is_exact(cuda, bucket, passes, caches):
    """The level kernel with the per-warp successor queue for 4-word slots (one lane per
    bucket of 4 or 8 words, region passes), with and without the caches of seen
    vectors: every count, level and digest equals the oracle's and the closed forms."""
    blocks = [2] * 12 + [3] * 4
    net = inputs.product_network(1, 16, 16, blocks)
    S, T = _product_closed_form(net, blocks)
    s = assert_parity(net, table_bytes=1 << 25, bucket_words=bucket, group_lanes=1, hash_rounds=32,
                      region_passes=passes, **caches)
    assert (s["states"], s["transitions"], s["slot_words"], s["region_passes"]) == (S, T, 4, passes)


@pytest.mark.parametrize("host_loop", [1, 0])
def test_queued_four_word_kernel_with_deadlocks_and_full_buckets(cuda, host_loop):
    """A 4-word network with deadlocks in a table filled to 86 % (many vectors go
    past their first bucket) through the queued kernel: exact."""
    net = inputs.random_network(2, 12, [1000] * 12, 0, 2, 14, n_sync=5, parties=2)  # 224,532 states, 888 deadlocks
    r = oracle.explore(net)
    assert r.deadlock_count > 0
    table = 1 << 12
    while table * 9 // 10 < r.states * 16:
        table *= 2
    s = assert_parity(net, table_bytes=table, bucket_words=8, group_lanes=1, hash_rounds=64, region_passes=2,
                      host_loop=host_loop)
    assert s["slot_words"] == 4 and s["fill"] > 0.8


def test_global_cache_never_holds_the_all_zero_key(cuda):
    """The vector whose fields are all 0 packs to key 0, the value of an empty entry,
    so it is never cached.  Here it is reachable (the product family reaches every
    combination of block states from any start) but not the initial state: a hit on
    an empty entry would drop it from the set."""
    net = inputs.product_network(1, 16, 16, [2] * 12 + [3] * 4)
    for p in net.procs:
        p.initial = 1
    S, T = _product_closed_form(net, [2] * 12 + [3] * 4)
    s = assert_parity(net, table_bytes=1 << 25, global_cache_log2=20, warp_cache_log2=0)
    assert (s["states"], s["transitions"]) == (S, T)
    assert s["global_cache_entries"] == 1 << 20


def test_global_cache_is_cleared_between_searches(cuda):
    """Two different networks explored one after the other in the same workspace:
    entries left by the first are not hits in the second."""
    import torch
    a = inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4)
    b = inputs.random_network(2, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4)
    o = gx.default_opts(table_bytes=1 << 25, global_cache_log2=16)
    ha, hb = gx.load_network(a), gx.load_network(b)
    ws = gx.alloc_workspace(ha, o)
    assert gx.workspace_bytes(hb, o) <= ws.numel()
    for h, net in ((ha, a), (hb, b), (ha, a)):
        gx.explore(h, o, ws)
        torch.cuda.synchronize()
        r = oracle.explore(net)
        s = gx.stats(h)
        assert (s["states"], s["transitions"], gx.levels(h)) == (r.states, r.transitions, r.levels)


@pytest.mark.parametrize("bucket,group,passes", [(16, 0, 1), (8, 0, 2), (32, 0, 4), (8, 1, 1), (8, 1, 2), (4, 1, 4)])
def test_large_irregular_network_against_stored_oracle(cuda, bucket, group, passes):
    """16 processes x 16 local states (3-word vectors in 4-word slots), 3-party rules
    on 10 % of the labels that shape the reachable set (1.08e8 states, 3.5 times as
    many as without the rule edges): states, transitions, every level, the deadlock
    digest and the digest of the whole set equal the oracle's, written by
    tests/golden/make_golden.py; with one, two and four region passes, one lane per
    slot (group 0: the default) or one lane per bucket (with region passes, 4- and
    8-word buckets of 4-word slots run the level kernel with the successor queue)."""
    g = _golden_case("large3_network.json")
    net = inputs.random_network(**g["generator"])
    h, s, lv, ws = run_gpu(net, table_bytes=4 << 30, bucket_words=bucket, group_lanes=group, hash_rounds=32,
                           region_passes=passes)
    assert s["slot_words"] == 4 and s["region_passes"] == passes
    assert s["group_lanes"] == (group or bucket // 4)
    assert (s["states"], s["transitions"]) == (g["states"], g["transitions"])
    assert lv == g["levels"]
    assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"]) == (
        g["deadlock_count"], g["deadlock_sum"], g["deadlock_xor"])
    assert gx.set_digest(h, ws) == (g["states"], g["set_sum"], g["set_xor"])
    assert s["fill"] <= 0.75


def test_large_irregular_network_with_the_global_cache(cuda):
    """The same 1.08e8-state network (16 fields of 4 bits: a 64-bit cache key) with
    the GPU-wide cache (2^23 entries) and two region passes: exact against the stored
    oracle values, with fewer bucket reads than without the cache."""
    g = _golden_case("large3_network.json")
    net = inputs.random_network(**g["generator"])
    runs = {}
    for log2 in (0, 23):
        h, s, lv, ws = run_gpu(net, table_bytes=4 << 30, bucket_words=16, hash_rounds=32, region_passes=2,
                               global_cache_log2=log2, warp_cache_log2=0)
        assert s["global_cache_entries"] == (1 << log2 if log2 else 0)
        assert (s["states"], s["transitions"], lv) == (g["states"], g["transitions"], g["levels"])
        assert gx.set_digest(h, ws) == (g["states"], g["set_sum"], g["set_xor"])
        runs[log2] = s["probes"]
        del ws
    assert runs[23] < runs[0]


@pytest.mark.parametrize("host_loop", [1, 0])
def test_global_cache_with_multi_lane_groups_on_the_mid_network(cuda, host_loop):
    """The GPU-wide cache forced on with 16 lanes per 32-word bucket on the mid network
    (62M states): one lane of each group reads the cache and the group takes its
    answer, so a concurrent write by another warp cannot split the group before
    find-or-put's group-wide votes.  Exact against the stored oracle values."""
    g = _golden_case("mid_network.json")
    net = inputs.random_network(**g["generator"])
    h, s, lv, ws = run_gpu(net, table_bytes=4 << 28, bucket_words=32, hash_rounds=32, global_cache_log2=23,
                           host_loop=host_loop)
    assert s["group_lanes"] == 16 and s["global_cache_entries"] == 1 << 23
    assert (s["states"], s["transitions"], lv) == (g["states"], g["transitions"], g["levels"])
    assert gx.set_digest(h, ws) == (g["states"], g["set_sum"], g["set_xor"])
