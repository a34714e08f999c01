"""Degenerate and extreme networks, GPU against the oracle through the C ABI.

* a single state without transitions (the initial state is a deadlock at level 0);
* a single state with a self-loop (one transition, no deadlock);
* rules that can never fire (a participant without any matching edge);
* duplicate edges (transitions count with multiplicity);
* a 16-party rule (the most participants the encoding allows);
* 124 processes of 2 states each: 124 one-bit fields fill all four 31-bit words.
Each runs in both level loops and, all six together, as one batched exploration.
The counts are also closed forms worked out by hand (CLOSED_FORM), which pin the
oracle on the CPU.
"""
import pytest

import oracle
from paper_1801_05857_gb300 import gx, inputs

LTS, Rule, Network = inputs.LTS, inputs.Rule, inputs.Network


def _nets():
    nets = [Network(1, [LTS(1, 0, [])], [], name="one_state_deadlock"),
            Network(1, [LTS(1, 0, [(0, 0, 0)])], [], name="one_state_self_loop")]
    # label 1 is a rule label of both processes, but process 1 has no edge with it
    nets.append(Network(3, [LTS(3, 0, [(0, 0, 1), (1, 1, 2), (2, 0, 0)]), LTS(2, 0, [(0, 2, 1), (1, 2, 0)])],
                        [Rule([(0, 1), (1, 1)], 1)], name="dead_rule"))
    # the same edge three times in one process, and twice inside a rule
    nets.append(Network(3, [LTS(2, 0, [(0, 0, 1), (0, 0, 1), (0, 0, 1), (1, 1, 0), (1, 1, 0)]),
                            LTS(2, 0, [(0, 1, 1), (1, 2, 0)])],
                        [Rule([(0, 1), (1, 1)], 1)], name="duplicate_edges"))
    # 16 processes that all step together once, then each may move on alone
    procs = [LTS(3, 0, [(0, 0, 1), (1, 1, 2)]) for _ in range(16)]
    nets.append(Network(2, procs, [Rule([(p, 0) for p in range(16)], 0)], name="sixteen_party_rule"))
    # 124 one-bit processes: only the first three move, the rest stay in state 0
    procs = [LTS(2, 0, [(0, 0, 1), (1, 0, 0)]) for _ in range(3)] + [LTS(2, 0, []) for _ in range(121)]
    nets.append(Network(1, procs, [], name="widest_vector"))
    return nets


# (states, transitions, deadlocks, first deadlock level), counted by hand:
# dead_rule: process 0 stops in state 1, process 1 alternates, 2 x 2 states, 2 + 2 + 1 + 1 moves;
# duplicate_edges: (0,0) has 3 moves, (1,0) 2 x 1 joint moves, (0,1) 3 + 1, (1,1) 1;
# sixteen_party_rule: one joint step, then 2^16 independent choices, 16 x 2^15 single moves;
# widest_vector: 2^3 states, 3 moves each.
CLOSED_FORM = {"one_state_deadlock": (1, 0, 1, 0), "one_state_self_loop": (1, 1, 0, -1),
               "dead_rule": (4, 6, 0, -1), "duplicate_edges": (4, 10, 0, -1),
               "sixteen_party_rule": (1 + 2 ** 16, 1 + 16 * 2 ** 15, 1, 17),
               "widest_vector": (8, 24, 0, -1)}


@pytest.mark.parametrize("net", _nets(), ids=lambda n: n.name)
def test_oracle_closed_forms(net):
    r = oracle.explore(net)
    assert (r.states, r.transitions, r.deadlock_count, r.first_deadlock_level) == CLOSED_FORM[net.name]
    assert r.complete and sum(r.levels) == r.states


@pytest.mark.gpu
@pytest.mark.parametrize("host_loop", [0, 1])
@pytest.mark.parametrize("net", _nets(), ids=lambda n: n.name)
def test_degenerate_network(cuda, net, host_loop):
    import torch
    r = oracle.explore(net)
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 22, host_loop=host_loop)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    torch.cuda.synchronize()
    s = gx.stats(h)
    assert (s["states"], s["transitions"], gx.levels(h)) == (r.states, r.transitions, r.levels)
    assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"]) == (
        r.deadlock_count, r.deadlock_sum, r.deadlock_xor)
    assert s["first_deadlock_level"] == r.first_deadlock_level and s["complete"] == 1
    assert gx.set_digest(h, ws) == (r.states, r.set_sum, r.set_xor)
    if net.name == "widest_vector":
        assert s["vector_words"] == 4


@pytest.mark.gpu
def test_degenerate_networks_batched(cuda):
    nets = _nets()
    want = [oracle.explore(n) for n in nets]
    b = gx.batch_create(nets)
    o = gx.batch_opts(hash_rounds=64, expected_states=[2 * r.states for r in want])
    ws = gx.batch_alloc_workspace(b, o)
    gx.batch_explore(b, o, ws)
    for i, r in enumerate(want):
        s = gx.batch_stats(b, i)
        assert s["complete"] == 1 and gx.batch_levels(b, i) == r.levels, nets[i].name
        assert (s["states"], s["transitions"], s["explored"]) == (r.states, r.transitions, r.explored)
        assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"], s["first_deadlock_level"]) == (
            r.deadlock_count, r.deadlock_sum, r.deadlock_xor, r.first_deadlock_level), nets[i].name


@pytest.mark.gpu
@pytest.mark.parametrize("net", _nets(), ids=lambda n: n.name)
def test_degenerate_networks_guided_and_first_deadlock(cuda, net):
    """The guided search (untrained weights) either ends exhaustive with the oracle's
    counts or returns a deadlock whose path replays; the BFS first-deadlock mode stops
    on the oracle's first deadlock level."""
    import torch
    r = oracle.explore(net)
    params = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
    gx.mlp_init(params, 3)
    h = gx.load_network(net)
    gx.guided_set_weights(h, params)
    o = gx.default_opts(table_bytes=1 << 22, hash_rounds=32)
    n, found = gx.find_deadlocks(h, gx.GX_DL_GUIDED, o, gx.guided_alloc_workspace(h, o))
    s = gx.stats(h)
    if r.deadlock_count == 0:
        assert n == 0 and s["complete"] == 1
        assert (s["states"], s["transitions"]) == (r.states, r.transitions)
    else:
        assert n == 1
        trace = gx.guided_trace(h)
        assert list(trace[0]) == [p.initial for p in net.procs]
        for a, b in zip(trace[:-1], trace[1:]):
            assert tuple(b) in {tuple(x) for x in oracle.successors(net, a)}
        assert len(oracle.successors(net, trace[-1])) == 0 and list(found[0]) == list(trace[-1])
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 22)
    n, found = gx.find_deadlocks(h, gx.GX_DL_BFS_FIRST, o, gx.alloc_workspace(h, o))
    s = gx.stats(h)
    assert s["first_deadlock_level"] == r.first_deadlock_level
    assert (n > 0) == (r.deadlock_count > 0)
    for x in found[:n]:
        assert len(oracle.successors(net, x)) == 0
