"""Safety checking (Sec. 3: the negation of a safety property is one more
automaton of the network; a state in which that automaton is in its error
state violates the property), GPU against the oracle through the C ABI.

Bit-exact on: the violation count, its order-free digest, the level of the
first violation, the violating states themselves, and, when the search stops
at the first violating level, the levels explored and that level's violations.
"""
import numpy as np
import pytest

import oracle
from paper_1801_05857_gb300 import gx, inputs

pytestmark = pytest.mark.gpu


def _gpu(net, watch, stop=False, **opts):
    import torch
    h = gx.load_network(net)
    o = gx.default_opts(watch=1, watch_proc=watch[0], watch_state=watch[1],
                        stop_at_first_violation=int(stop), **opts)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    torch.cuda.synchronize()
    return h, gx.stats(h), gx.levels(h)


def _check(net, watch, stop=False, **opts):
    r = oracle.explore(net, watch=watch, stop_at_first_violation=stop, violations_cap=1 << 14)
    h, s, lv = _gpu(net, watch, stop, **opts)
    assert s["status"] == 0
    assert s["violation_count"] == r.violation_count
    assert s["violation_sum"] == r.violation_sum
    assert s["violation_xor"] == r.violation_xor
    assert s["first_violation_level"] == r.first_violation_level
    assert s["explored"] == r.explored
    assert lv == r.levels
    if 0 < r.violation_count <= 1024:
        got = {tuple(x) for x in gx.violations(h)}
        assert got == {tuple(x) for x in r.violations}
        assert all(x[watch[0]] == watch[1] for x in got)
    return s, r


def _watches(net, k, seed):
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(k):
        p = int(rng.integers(0, len(net.procs)))
        out.append((p, int(rng.integers(0, net.procs[p].n_states))))
    return out


def _nets():
    return [inputs.producer_consumers(), inputs.token_ring(6), inputs.token_ring(11),
            inputs.random_network(3, 4, 8, 1, 3, 6, n_sync=2, parties=2),
            inputs.random_network(6, 8, 8, 0, 2, 10, n_sync=4, parties=2),
            inputs.random_network(1, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4)]


@pytest.mark.parametrize("net", _nets(), ids=lambda n: n.name)
@pytest.mark.parametrize("stop", [False, True])
def test_violations_match_oracle(cuda, net, stop):
    for i, w in enumerate(_watches(net, 4, len(net.procs))):
        _check(net, w, stop, table_bytes=1 << 26)


def test_token_ring_first_violation_depth(cuda):
    """Node k of an 8-node ring first holds the token in h1 after 1 + 4k steps,
    in 3^7 states overall; stopping there leaves exactly one violating state."""
    net = inputs.token_ring(8)
    for k in (0, 3, 7):
        s, _ = _check(net, (k, 4), table_bytes=1 << 24)
        assert (s["violation_count"], s["first_violation_level"]) == (3 ** 7, 1 + 4 * k)
        s, _ = _check(net, (k, 4), stop=True, table_bytes=1 << 24)
        assert s["violation_count"] == 1 and s["complete"] == 0


@pytest.mark.parametrize("net", [inputs.token_ring(11),
                                 inputs.random_network(0, 13, 64, 1, 3, 16, n_sync=8, parties=3, cluster=4)],
                         ids=lambda n: n.name)
def test_violations_on_the_partitioned_path(cuda, net):
    for w in _watches(net, 3, 5):
        s, _ = _check(net, w, table_bytes=1 << 25, slice_log2=3, partition_min_states=1)
        assert s["partitioned_levels"] > 0


def test_every_bucket_size_and_no_cache(cuda):
    net = inputs.random_network(6, 8, 8, 0, 2, 10, n_sync=4, parties=2)
    w = _watches(net, 1, 9)[0]
    for B in (4, 8, 16, 32):
        _check(net, w, table_bytes=1 << 24, bucket_words=B, group_lanes=1)
    _check(net, w, table_bytes=1 << 24, warp_cache_log2=0)


def test_violation_cap_keeps_the_count(cuda):
    net = inputs.token_ring(7)
    h, s, _ = _gpu(net, (2, 4), violation_cap=5, table_bytes=1 << 24)
    assert s["violation_count"] == 3 ** 6
    v = gx.violations(h)
    assert len(v) == 5 and (v[:, 2] == 4).all()


def test_invalid_watch_is_rejected(cuda):
    net = inputs.token_ring(4)
    for bad in (dict(watch_proc=4, watch_state=0), dict(watch_proc=1, watch_state=5)):
        h = gx.load_network(net)
        with pytest.raises(gx.GxError) as e:
            gx.workspace_bytes(h, gx.default_opts(watch=1, **bad))
        assert e.value.status == gx.GX_ERR_INVALID


def test_guided_search_rejects_a_watch(cuda):
    import torch
    net = inputs.planted_network(0, 6)
    h = gx.load_network(net)
    p = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
    gx.mlp_init(p, 1)
    gx.guided_set_weights(h, p)
    o = gx.default_opts(table_bytes=1 << 24, watch=1, watch_proc=0, watch_state=1)
    ws = gx.guided_alloc_workspace(h, o)
    with pytest.raises(gx.GxError) as e:
        gx.find_deadlocks(h, gx.GX_DL_GUIDED, o, ws)
    assert e.value.status == gx.GX_ERR_INVALID
