"""gx_explore_noalloc, the exploration entry point that allocates nothing.

It serves callers that cannot allocate device memory: a host framework that has
reserved the GPU's memory for its own pool, or a latency-critical caller that must
not pay cudaFree's device-wide synchronisation.  It runs on a static scratch array
inside the library, which keeps the previous call's contents, so two calls in a
row must both give exactly what gx_explore gives on the same network and options.
This file is collected last on purpose.
"""
import pytest

from paper_1801_05857_gb300 import gx, inputs

pytestmark = pytest.mark.gpu

FIELDS = ("states", "explored", "transitions", "n_levels", "deadlock_count", "deadlock_sum",
          "deadlock_xor", "first_deadlock_level", "table_slots", "complete", "status")


def _nets():
    return [
        inputs.workload("tiny"),                                                # 1-word vectors
        inputs.token_ring(11),                                                  # 2-word vectors
        inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4),  # 4-word
        inputs.random_network(6, 4, 5, 0, 2, 6, n_sync=2, parties=2),           # has deadlocks
    ]


@pytest.mark.parametrize("net", _nets(), ids=lambda n: n.name)
def test_noalloc_matches_explore_on_two_calls_in_a_row(cuda, net):
    import torch
    h = gx.load_network(net)
    opts = gx.default_opts(table_bytes=32 << 20, bucket_words=8)
    ws = gx.alloc_workspace(h, opts)
    gx.explore(h, opts, ws)
    want = gx.stats(h)
    want_levels = gx.levels(h)
    for _ in range(2):
        got, levels = gx.explore_noalloc(h, opts)
        torch.cuda.synchronize()
        assert {k: got[k] for k in FIELDS} == {k: want[k] for k in FIELDS}
        assert levels == want_levels


def test_noalloc_rejects_sizes_beyond_its_scratch(cuda):
    h = gx.load_network(inputs.token_ring(6))
    with pytest.raises(gx.GxError) as e:
        gx.explore_noalloc(h, gx.default_opts(table_bytes=1 << 30))
    assert e.value.status == gx.GX_ERR_INVALID
    assert "static array" in e.value.message
    # still usable afterwards
    s, lv = gx.explore_noalloc(h, gx.default_opts(table_bytes=1 << 20))
    assert s["states"] == 2 * 6 * 3 ** 5 and sum(lv) == s["states"]
