"""Batched exploration (one graph launch for many networks) against the oracle."""
import json
import os

import pytest

import oracle
from paper_1801_05857_gb300 import gx, inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _mixed():
    return [inputs.token_ring(5), inputs.token_ring(11), inputs.producer_consumers(),
            inputs.workload("tiny"),
            inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4),
            inputs.random_network(6, 4, 5, 0, 2, 6, n_sync=2, parties=2),
            inputs.random_network(1, 10, 16, 1, 3, 12, n_sync=4, parties=2, cluster=4),
            inputs.random_network(7, 6, 8, 1, 3, 8, n_sync=2, parties=2)]


def _check_net(b, i, r):
    s = gx.batch_stats(b, i)
    assert s["complete"] == 1, i
    assert (s["states"], s["transitions"]) == (r.states, r.transitions), i
    assert gx.batch_levels(b, i) == r.levels, i
    assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"]) == (
        r.deadlock_count, r.deadlock_sum, r.deadlock_xor), i
    assert s["first_deadlock_level"] == r.first_deadlock_level, i
    assert s["explored"] == r.explored, i


@pytest.mark.parametrize("bucket,group,chunk", [(8, 1, 32), (4, 1, 64), (16, 2, 128), (32, 4, 32)])
def test_mixed_batch_matches_oracle(cuda, bucket, group, chunk):
    nets = _mixed()
    want = [oracle.explore(n) for n in nets]
    b = gx.batch_create(nets)
    # the batch pads every network to 4-word slots (its widest), so buckets hold few
    # slots: tables at most half full and 64 hash rounds
    o = gx.batch_opts(bucket_words=bucket, group_lanes=group, chunk_states=chunk, hash_rounds=64,
                      expected_states=[2 * r.states for r in want])
    ws = gx.batch_alloc_workspace(b, o)
    for _ in range(2):  # the cached graph is relaunched: every run starts from scratch
        gx.batch_explore(b, o, ws)
        for i, r in enumerate(want):
            _check_net(b, i, r)


@pytest.mark.parametrize("wide", [gx.BATCH_WIDE_OFF, 1 << 20])
def test_lane_and_warp_layouts_alone_match_oracle(cuda, wide):
    """Every iteration with one state per lane (wide path off), or every iteration with
    one state per warp and successors by index (a factor no iteration exceeds)."""
    nets = _mixed()
    want = [oracle.explore(n) for n in nets]
    b = gx.batch_create(nets)
    o = gx.batch_opts(hash_rounds=64, expected_states=[2 * r.states for r in want], wide_factor=wide)
    ws = gx.batch_alloc_workspace(b, o)
    gx.batch_explore(b, o, ws)
    for i, r in enumerate(want):
        _check_net(b, i, r)


def test_autotune_picks_a_working_configuration(cuda):
    nets = _mixed()
    want = [oracle.explore(n) for n in nets]
    b = gx.batch_create(nets)
    o = gx.batch_opts(hash_rounds=64, table_slots=1 << 22)
    ws = gx.batch_alloc_workspace(b, o)
    ms = gx.batch_autotune(b, o, ws)
    assert ms > 0 and o.bucket_words in (4, 8, 16, 32) and o.chunk_states in (32, 64, 128)
    gx.batch_explore(b, o, ws)
    for i, r in enumerate(want):
        _check_net(b, i, r)


def test_levels_cap_overflow_is_reported(cuda):
    b = gx.batch_create([inputs.token_ring(6)])
    o = gx.batch_opts(levels_cap=4, table_slots=1 << 14)
    ws = gx.batch_alloc_workspace(b, o)
    with pytest.raises(gx.GxError) as e:
        gx.batch_explore(b, o, ws)
    assert e.value.status == gx.GX_ERR_OOM


def test_batched_workload_against_stored_oracle(cuda):
    """The 256-network batched workload (4-10 processes x 8-32 states, 10^3..10^6
    states each), expected values written by tests/golden/make_golden.py batch."""
    path = os.path.join(GOLDEN, "batch_networks.json")
    if not os.path.exists(path):
        pytest.skip("batch_networks.json not generated")
    g = json.load(open(path))
    nets = [inputs.random_network(**x["generator"]) for x in g["networks"]]
    b = gx.batch_create(nets)
    o = gx.batch_opts(hash_rounds=32, expected_states=[x["states"] for x in g["networks"]])
    ws = gx.batch_alloc_workspace(b, o)
    gx.batch_explore(b, o, ws)
    for i, x in enumerate(g["networks"]):
        s = gx.batch_stats(b, i)
        assert (s["states"], s["transitions"]) == (x["states"], x["transitions"]), i
        assert gx.batch_levels(b, i) == x["levels"], i
        assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"]) == (
            x["deadlock_count"], x["deadlock_sum"], x["deadlock_xor"]), i
