"""Failure detection without a GPU fault: a bounded device wait that runs out
reaches the host as GX_ERR_SPIN_LIMIT, and the context stays usable.  The wait
is on an mbarrier that nothing arrives on, so it always runs out; it is bounded
by its poll limit, so it never hangs."""
import pytest

import oracle
from paper_1801_05857_gb300 import gx, inputs


def test_wait_selftest_rejects_bad_limits():
    # host-side validation (stream 0 given, so no CUDA runtime is asked)
    for bad in (0, (1 << 22) + 1):
        with pytest.raises(gx.GxError) as e:
            gx.wait_selftest(bad, stream=0)
        assert e.value.status == gx.GX_ERR_INVALID


@pytest.mark.gpu
def test_wait_that_runs_out_is_reported_and_the_context_stays_usable(cuda):
    import torch
    for limit in (1, 1000, 100000):
        with pytest.raises(gx.GxError) as e:
            gx.wait_selftest(limit)
        assert e.value.status == gx.GX_ERR_SPIN_LIMIT and str(limit) in e.value.message
    # the same context then explores a network exactly
    net = inputs.token_ring(8)
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 22)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    torch.cuda.synchronize()
    s, r = gx.stats(h), oracle.explore(net)
    assert (s["states"], s["transitions"], s["status"]) == (r.states, r.transitions, 0)
