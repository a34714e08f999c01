"""gx_explore_noalloc, the exploration entry point that allocates nothing.

It serves callers that cannot allocate device memory: a host framework that has
reserved the GPU's memory for its own pool, or a latency-critical caller that must
not pay cudaFree's device-wide synchronisation.  It runs on a static scratch array
inside the library, which keeps the previous call's contents, so two calls in a
row must both give exactly what the oracle gives, and what gx_explore gives on the
same network and options.  This file is collected last on purpose.
"""
import pytest

import oracle
from paper_1801_05857_gb300 import gx, inputs

pytestmark = pytest.mark.gpu

FIELDS = ("states", "explored", "transitions", "n_levels", "deadlock_count", "deadlock_sum",
          "deadlock_xor", "first_deadlock_level", "table_slots", "complete", "status")


def _nets():
    return [
        inputs.workload("tiny"),                                                # 1-word vectors
        inputs.token_ring(11),                                                  # 2-word vectors
        inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4),  # 4-word
        inputs.random_network(1, 15, 16, 1, 3, 16, n_sync=8, parties=3, cluster=4),  # 4-word, 60 bits
        inputs.random_network(6, 4, 5, 0, 2, 6, n_sync=2, parties=2),           # has deadlocks
    ]


def _oracle_fields(r):
    return {"states": r.states, "explored": r.explored, "transitions": r.transitions,
            "n_levels": len(r.levels), "deadlock_count": r.deadlock_count,
            "deadlock_sum": r.deadlock_sum, "deadlock_xor": r.deadlock_xor,
            "first_deadlock_level": r.first_deadlock_level, "complete": int(r.complete)}


@pytest.mark.parametrize("cache", [9, 0], ids=["caches", "no_caches"])
@pytest.mark.parametrize("net", _nets(), ids=lambda n: n.name)
def test_noalloc_matches_oracle_and_explore_on_two_calls_in_a_row(cuda, net, cache):
    import torch
    r = oracle.explore(net)
    want_oracle = _oracle_fields(r)
    h = gx.load_network(net)
    opts = gx.default_opts(table_bytes=32 << 20, bucket_words=8, warp_cache_log2=cache,
                           global_cache_log2=20 if cache else 0)  # the GPU-wide cache is opt-in
    ws = gx.alloc_workspace(h, opts)
    gx.explore(h, opts, ws)
    want = gx.stats(h)
    for _ in range(2):
        got, levels = gx.explore_noalloc(h, opts)
        torch.cuda.synchronize()
        assert {k: got[k] for k in want_oracle} == want_oracle
        assert levels == r.levels
        assert {k: got[k] for k in FIELDS} == {k: want[k] for k in FIELDS}


@pytest.mark.parametrize("stop", [0, 1])
def test_noalloc_safety_check_matches_oracle(cuda, stop):
    """The watched property (node 3 of the token ring holding the token, local
    state 4) is counted and digested as by the oracle, with its first level; with
    stop_at_first_violation the search ends after that level."""
    net = inputs.token_ring(8)
    r = oracle.explore(net, watch=(3, 4), stop_at_first_violation=bool(stop))
    h = gx.load_network(net)
    opts = gx.default_opts(table_bytes=16 << 20, watch=1, watch_proc=3, watch_state=4,
                           stop_at_first_violation=stop)
    for _ in range(2):
        got, levels = gx.explore_noalloc(h, opts)
        assert (got["violation_count"], got["violation_sum"], got["violation_xor"],
                got["first_violation_level"]) == (r.violation_count, r.violation_sum, r.violation_xor,
                                                  r.first_violation_level)
        assert levels == r.levels and got["states"] == r.states
        assert got["transitions"] == r.transitions


@pytest.mark.parametrize("bucket", [4, 8])
@pytest.mark.parametrize("passes", [2, 4])
@pytest.mark.parametrize("net", [
    inputs.random_network(1, 15, 16, 1, 3, 16, n_sync=8, parties=3, cluster=4),   # 4-word, 60 field bits
    inputs.random_network(2, 12, [1000] * 12, 0, 2, 14, n_sync=5, parties=2)],    # 4-word, deadlocks
    ids=lambda n: n.name)
def test_noalloc_region_passes_with_one_lane_per_bucket(cuda, net, bucket, passes):
    """4-word slots in 4- or 8-word buckets, one lane per bucket, with region passes: the
    entry point runs the level kernel with the successor queue, as gx_explore does; twice
    in a row, exact against the oracle."""
    import torch
    r = oracle.explore(net)
    h = gx.load_network(net)
    opts = gx.default_opts(table_bytes=32 << 20, bucket_words=bucket, group_lanes=1, hash_rounds=32,
                           region_passes=passes)
    for _ in range(2):
        got, levels = gx.explore_noalloc(h, opts)
        torch.cuda.synchronize()
        assert {k: got[k] for k in _oracle_fields(r)} == _oracle_fields(r)
        assert levels == r.levels
        assert got["region_passes"] == passes and got["slot_words"] == 4


def test_noalloc_rejects_what_it_cannot_do(cuda):
    h = gx.load_network(inputs.token_ring(6))
    with pytest.raises(gx.GxError) as e:
        gx.explore_noalloc(h, gx.default_opts(table_bytes=1 << 30))
    assert e.value.status == gx.GX_ERR_INVALID
    assert "static array" in e.value.message
    with pytest.raises(gx.GxError) as e:
        gx.explore_noalloc(h, gx.default_opts(table_bytes=1 << 20, partition_min_states=1024))
    assert e.value.status == gx.GX_ERR_INVALID and "partition" in e.value.message
    with pytest.raises(gx.GxError) as e:
        gx.explore_noalloc(h, gx.default_opts(table_bytes=1 << 20, watch=1, watch_proc=6, watch_state=0))
    assert e.value.status == gx.GX_ERR_INVALID
    # still usable afterwards
    s, lv = gx.explore_noalloc(h, gx.default_opts(table_bytes=1 << 20))
    assert s["states"] == 2 * 6 * 3 ** 5 and sum(lv) == s["states"]
