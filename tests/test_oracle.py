"""Pins of the CPU oracle against what the paper and the mathematics fix.

* Fig. 1's network has 8 states and 24 transitions (Sec. 3).
* Our token ring reproduces every Token Ring count of Table 1 (Sec. 5.2) and
  the transition count derived below.
* Without rules the product's reachable set, transitions, BFS level sizes and
  deadlocks have closed forms in per-process quantities.
* On tiny networks with rules, the oracle agrees with a brute force that
  writes the product as a sum of Kronecker products over the whole product
  space (oracle/product_matrix.py) -- a different formulation of the same
  semantics, not a second copy of the successor enumeration.
* The state digest's mixer is splitmix64, whose first output from seed 0 is
  the published value 0xE220A8397B1DCDAF.
"""
import json
import os
from collections import deque
from itertools import product

import numpy as np
import pytest

import oracle
from oracle import product_matrix as pm
from paper_1801_05857_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def test_splitmix64_published_first_output():
    # splitmix64 seeded with 0 first returns 0xE220A8397B1DCDAF (Steele, Lea & Flood 2014;
    # the reference sequence of the algorithm).  The oracle's digest of the one-process
    # state (0,) is exactly that first output.
    assert oracle.state_digest([0]) == 0xE220A8397B1DCDAF
    assert inputs.SplitMix64(0).next() == 0xE220A8397B1DCDAF


def test_fig1_counts():
    g = golden("fig1_producer_consumers.json")
    r = oracle.explore(inputs.producer_consumers())
    assert r.states == g["states"]
    assert r.transitions == g["transitions"]
    assert r.deadlock_count == 0 and r.complete
    assert sum(r.levels) == r.states


def test_fig1_readings_that_the_counts_exclude():
    """The two other readings of Sec. 3 give other counts: letting rule labels also
    fire alone gives 36 transitions, and counting distinct (s, a, t) edges gives 22.
    The oracle's reading is the only one that yields the published 24."""
    net = inputs.producer_consumers()
    t = pm.transition_matrix(net).toarray()
    r = oracle.explore(net)
    reach = pm.explore(net)["reachable"]
    states = pm.states_of(net, reach)
    # rule labels firing alone as well (the reachable set stays all 8 states): count the
    # rule-labelled edges enabled in each state as extra single-process moves
    extra = 0
    for st in states:
        for p in range(net.n_procs):
            rl = {a for rule in net.rules for (q, a) in rule.parts if q == p}
            extra += sum(1 for (s, lab, d) in net.procs[p].edges if s == st[p] and lab in rl)
    assert r.transitions + extra == 36
    # distinct (source, target) pairs: two consumers' 'work' self-loops in the same global
    # state are one edge (s, work, s) when edges are not counted with multiplicity
    distinct = set()
    for st in states:
        for succ in oracle.successors(net, st):
            distinct.add((tuple(st), tuple(succ)))
    assert len(distinct) == 22
    assert int(t[np.ix_(reach, reach)].sum()) == 24


@pytest.mark.parametrize("n_nodes", list(range(2, 12)))
def test_token_ring_table1(n_nodes):
    g = golden("token_ring_table1.json")
    r = oracle.explore(inputs.token_ring(n_nodes))
    assert r.states == g["states"][str(n_nodes)]
    # Derivation: a global state is (token holder k, holder state h0|h1, the other
    # N-1 nodes each in i0|i1|i2), all reachable: 2N 3^(N-1) states.  Enabled moves:
    # each non-holder not at i2 steps (2/3 of them on average), the holder in h0 steps,
    # the holder in h1 passes the token iff its right neighbour is at i2.  Summing,
    # T = N * (4(N-1) 3^(N-2) + 3^(N-1) + 3^(N-2)) = 4 N^2 3^(N-2).
    assert r.transitions == 4 * n_nodes * n_nodes * 3 ** (n_nodes - 2)
    assert r.deadlock_count == 0 and r.complete
    assert sum(r.levels) == r.states


def _local_facts(lts):
    """Per-process BFS: depth of every reachable local state."""
    depth = {lts.initial: 0}
    q = deque([lts.initial])
    adj = {}
    for (s, a, t) in lts.edges:
        adj.setdefault(s, []).append(t)
    while q:
        s = q.popleft()
        for t in adj.get(s, []):
            if t not in depth:
                depth[t] = depth[s] + 1
                q.append(t)
    deg = {s: len(adj.get(s, [])) for s in depth}
    return depth, deg


@pytest.mark.parametrize("seed", range(6))
def test_no_sync_closed_forms(seed):
    net = inputs.no_sync_network(seed, n_procs=5, n_states=6, deg_lo=0, deg_hi=3)
    facts = [_local_facts(p) for p in net.procs]
    sizes = [len(d) for d, _ in facts]
    states = int(np.prod(sizes))
    trans = 0
    for p, (d, deg) in enumerate(facts):
        trans += sum(deg.values()) * int(np.prod([sizes[q] for q in range(len(sizes)) if q != p]))
    poly = np.array([1], dtype=object)
    for d, _ in facts:
        pp = np.zeros(max(d.values()) + 1, dtype=object)
        for s, k in d.items():
            pp[k] += 1
        poly = np.convolve(poly, pp)
    sinks = [[s for s, k in deg.items() if k == 0] for _, deg in facts]
    dead = list(product(*sinks))
    r = oracle.explore(net)
    assert r.states == states
    assert r.transitions == trans
    assert r.levels == [int(x) for x in poly]
    assert r.deadlock_count == len(dead)
    hs = [oracle.state_digest(list(s)) for s in dead]
    assert r.deadlock_sum == sum(hs) % (1 << 64)
    x = 0
    for h in hs:
        x ^= h
    assert r.deadlock_xor == x
    # digest of the whole reachable set: the product of the local reachable sets
    allh = [oracle.state_digest(list(s)) for s in product(*[sorted(d) for d, _ in facts])]
    assert r.set_sum == sum(allh) % (1 << 64)


def _tiny_sync_networks():
    nets = [inputs.producer_consumers(), inputs.token_ring(3), inputs.token_ring(4)]
    for seed in range(8):
        nets.append(inputs.random_network(seed, 4, 5, 0, 3, 6, n_sync=2, parties=2))
    for seed in range(4):
        nets.append(inputs.random_network(100 + seed, 4, 4, 1, 3, 5, n_sync=2, parties=3))
    nets.append(inputs.random_network(0, 4, 8, 1, 3, 6, n_sync=2, parties=2))  # tiny config shape
    return nets


@pytest.mark.parametrize("net", _tiny_sync_networks(), ids=lambda n: n.name)
def test_oracle_matches_kronecker_brute_force(net):
    bf = pm.explore(net)
    r = oracle.explore(net, deadlocks_cap=1 << 16)
    states, dist = oracle.deadlock_distances(net)
    assert r.states == len(bf["reachable"])
    got = {pm.index_of(net, s) for s in states}
    assert got == set(int(i) for i in bf["reachable"])
    assert r.levels == bf["levels"]
    assert r.transitions == bf["transitions"]
    assert r.deadlock_count == len(bf["deadlocks"])
    assert {pm.index_of(net, s) for s in r.deadlocks} == set(int(i) for i in bf["deadlocks"])
    assert (dist == 0).sum() == len(bf["deadlocks"])


@pytest.mark.parametrize("seed", range(4))
def test_deadlock_distances_are_backward_bfs(seed):
    net = inputs.random_network(seed, 4, 5, 0, 2, 6, n_sync=2, parties=2)
    states, dist = oracle.deadlock_distances(net)
    idx = {tuple(s): i for i, s in enumerate(states)}
    inf = np.iinfo(np.uint32).max
    for i, s in enumerate(states):
        succ = oracle.successors(net, s)
        if len(succ) == 0:
            assert dist[i] == 0
            continue
        best = min(int(dist[idx[tuple(t)]]) for t in succ)
        assert dist[i] == (inf if best == inf else best + 1)


def test_stop_at_first_deadlock_finishes_that_level():
    for seed in range(20):
        net = inputs.random_network(seed, 4, 5, 0, 2, 6, n_sync=2, parties=2)
        full = oracle.explore(net)
        if full.deadlock_count == 0:
            continue
        first = oracle.explore(net, stop_at_first_deadlock=True)
        k = first.first_deadlock_level
        assert k == full.first_deadlock_level
        assert first.levels[:k + 1] == full.levels[:k + 1]
        assert first.explored == sum(full.levels[:k + 1])
        # every deadlock of level k is found, and only those: the brute force's
        # deadlocks whose BFS depth (matrix-step distance) is k
        bf = pm.explore(net)
        t = pm.transition_matrix(net).transpose().tocsr()
        depth = {}
        front = {pm.index_of(net, [p.initial for p in net.procs])}
        d = 0
        while front:
            for i in front:
                depth[i] = d
            nxt = set()
            for i in front:
                v = np.zeros(t.shape[0], dtype=np.int64)
                v[i] = 1
                nxt |= set(np.flatnonzero(t @ v).tolist())
            front = nxt - set(depth)
            d += 1
        want = {int(i) for i in bf["deadlocks"] if depth[int(i)] == k}
        assert {pm.index_of(net, s) for s in first.deadlocks} == want
        assert first.deadlock_count == len(want)
        return
    pytest.fail("no seed produced a deadlock")


def test_key_sequence_duplication():
    for d in (1, 2, 5, 21):
        keys = inputs.key_sequence(2100, d, words=1, seed=3)
        u, c = np.unique(keys[:, 0], return_counts=True)
        assert len(u) == 2100 // d and (c == d).all()
        assert (keys != 0).all() and ((keys >> 31) == 0).all()
    k4 = inputs.key_sequence(1000, 4, words=4, seed=1)
    u = np.unique(k4, axis=0)
    assert len(u) == 250 and ((k4 >> 31) == 0).all()


def test_device_key_sequence_has_the_same_keys():
    pytest.importorskip("torch")
    for d in (1, 7, 21):
        a = inputs.key_sequence_device(2100, d, seed=5, device="cpu").numpy().view(np.uint32)
        b = inputs.key_sequence(2100, d, words=1, seed=5)[:, 0]
        assert sorted(a.tolist()) == sorted(b.tolist())


def test_mlp_oracle_gradient_matches_finite_differences():
    """Pins oracle/mlp.py's backward pass: central differences in float64 on the
    unrounded network agree with the analytic gradient."""
    from oracle import mlp
    rng = np.random.default_rng(0)
    p = (rng.standard_normal(mlp.NPARAM) * 0.2).astype(np.float32)
    hist = rng.integers(0, 5, size=(12, 16))
    hist[:, 0] += 1  # no empty row
    label = rng.random(12)
    _, g = mlp.loss_and_grad(p, hist, label, bf16=False)
    pd = p.astype(np.float64)

    def loss_at(q):
        W1, b1, W2, b2, w3, b3 = mlp.unpack(q.astype(np.float32))  # layout only
        x = hist / hist.sum(axis=1, keepdims=True)
        a1 = x @ q[:mlp.H * mlp.IN].reshape(mlp.H, mlp.IN).T + q[mlp.H * mlp.IN:mlp.H * mlp.IN + mlp.H]
        o = mlp.H * mlp.IN + mlp.H
        W2q = q[o:o + mlp.H * mlp.H].reshape(mlp.H, mlp.H); o += mlp.H * mlp.H
        b2q = q[o:o + mlp.H]; o += mlp.H
        w3q = q[o:o + mlp.H]; o += mlp.H
        y = np.maximum(np.maximum(a1, 0) @ W2q.T + b2q, 0) @ w3q + q[o]
        return np.mean((y - label) ** 2)

    idx = np.concatenate([rng.choice(mlp.H * mlp.IN, 20, replace=False),
                          mlp.H * mlp.IN + mlp.H + rng.choice(mlp.H * mlp.H, 30, replace=False),
                          [mlp.NPARAM - 1], mlp.NPARAM - 1 - mlp.H + rng.choice(mlp.H, 10, replace=False)])
    for i in idx:
        e = np.zeros_like(pd)
        e[i] = 1e-6
        fd = (loss_at(pd + e) - loss_at(pd - e)) / 2e-6
        assert abs(fd - g[i]) <= 1e-5 + 1e-4 * abs(g[i]), (i, fd, g[i])


def test_bf16_rounding_definition():
    """bfloat16 keeps the upper 16 bits of binary32, rounding to nearest, ties to even."""
    from oracle import mlp
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, -2.5, 3.140625], dtype=np.float32)
    r = mlp.bf16_round(x)
    assert r[0] == 1.0
    assert r[1] == 1.0                      # halfway: tie to even (mantissa ...0)
    assert r[2] == np.float32(1.0 + 4 * 2 ** -8)  # halfway: tie to even (rounds up)
    assert r[3] == 1.0
    assert r[4] == -2.5 and r[5] == np.float32(3.140625)
    assert ((r.view(np.uint32) & 0xFFFF) == 0).all()


def test_mlp_oracle_rounds_the_hidden_layer_input_to_bf16():
    """Closed-form case: W1 = 0 and b1 = 1 + 2^-8 (a bfloat16 tie) make every
    hidden unit 1 + 2^-8 before rounding.  W2 = I (first unit only), w3 = e0,
    b2 = b3 = 0 pass the first unit to the output, so y is 1 exactly when the
    second layer sees the rounded value (tie to even), and 1 + 2^-8 without
    rounding.  A hidden unit of 1 + 3 * 2^-8 rounds up to 1 + 2^-6 instead."""
    from oracle import mlp
    for pre, want in ((1 + 2 ** -8, 1.0), (1 + 3 * 2 ** -8, 1 + 2 ** -6)):
        p = np.zeros(mlp.NPARAM, dtype=np.float32)
        o = mlp.H * mlp.IN
        p[o:o + mlp.H] = pre                              # b1
        o += mlp.H
        p[o] = 1.0                                        # W2[0, 0]
        o += mlp.H * mlp.H + mlp.H
        p[o] = 1.0                                        # w3[0]
        hist = np.array([[3] + [0] * 15, [0] * 15 + [16]])
        assert (mlp.forward(p, hist) == want).all()
        assert (mlp.forward(p, hist, bf16=False) == np.float64(np.float32(pre))).all()


def test_mlp_oracle_features_are_bf16_fractions_of_processes():
    """Closed-form case: W1 picks input 0 into hidden unit 0 (weight 1), W2 and
    w3 pass hidden unit 0 to the output, all biases 0, so y = x0.  x0 is the
    fraction of processes in local state 0, rounded to bfloat16 from its
    binary32 value: 1/3 -> 0.333984375 and 2/3 -> 0.66796875 (round up past
    the halfway point), 1/4 and 1 exact, 0 for an empty row."""
    from oracle import mlp
    p = np.zeros(mlp.NPARAM, dtype=np.float32)
    p[0] = 1.0                                            # W1[0, 0]
    o = mlp.H * mlp.IN + mlp.H
    p[o] = 1.0                                            # W2[0, 0]
    p[o + mlp.H * mlp.H + mlp.H] = 1.0                    # w3[0]
    rows = np.zeros((5, 16), dtype=np.int64)
    rows[0, :2] = (1, 2)
    rows[1, :2] = (2, 1)
    rows[2, :2] = (3, 9)
    rows[3, 0] = 16
    y = mlp.forward(p, rows)
    assert y.tolist() == [0.333984375, 0.66796875, 0.25, 1.0, 0.0]


def _mlp_params(W1=None, b1=None, W2=None, b2=None, w3=None, b3=0.0):
    from oracle import mlp
    H, IN = mlp.H, mlp.IN
    parts = [np.zeros((H, IN)) if W1 is None else W1, np.zeros(H) if b1 is None else b1,
             np.zeros((H, H)) if W2 is None else W2, np.zeros(H) if b2 is None else b2,
             np.zeros(H) if w3 is None else w3, [b3]]
    return np.concatenate([np.ravel(np.asarray(a, dtype=np.float64)) for a in parts]).astype(np.float32)


def test_mlp_reference_features_are_exact_fractions():
    """Closed form: W1 picks input k into hidden unit 0, W2 and w3 pass unit 0
    to the output, so y = x_k = hist_k / n exactly in float64 (1/3, 5/7, 2/9),
    where the kernels' model rounds x to bfloat16 (0.333984375 for 1/3)."""
    from oracle import mlp
    for k, row, want in ((0, {0: 1, 1: 2}, 1 / 3), (3, {3: 5, 7: 2}, 5 / 7), (15, {15: 2, 2: 7}, 2 / 9)):
        W1 = np.zeros((mlp.H, mlp.IN))
        W1[0, k] = 1.0
        W2 = np.zeros((mlp.H, mlp.H))
        W2[0, 0] = 1.0
        w3 = np.zeros(mlp.H)
        w3[0] = 1.0
        h = np.zeros((2, 16), dtype=np.int64)
        for i, c in row.items():
            h[0, i] = c
        y, h2 = mlp.forward_reference(_mlp_params(W1, W2=W2, w3=w3), h)
        assert y[0] == want and y[1] == 0.0          # an all-zero row has x = 0
        assert h2[0, 0] == want and (h2[0, 1:] == 0).all()


def test_mlp_reference_rounds_weights_only():
    """Closed form: weights are bfloat16, nothing else.  A weight of 1 + 2^-9
    (a tie) acts as 1, and 1 + 3 * 2^-9 as 1 + 2^-7 (tie to even), while a bias
    or a hidden unit of 1 + 2^-9 passes unrounded: with W1 = 0, b1 = 1 + 2^-9,
    W2[0, 0] = w, w3[0] = 1, y = (1 + 2^-9) w."""
    from oracle import mlp
    for w, eff in ((1 + 2 ** -9, 1.0), (1 + 3 * 2 ** -9, 1 + 2 ** -7), (-0.5, -0.5)):
        W2 = np.zeros((mlp.H, mlp.H))
        W2[0, 0] = w
        b1 = np.zeros(mlp.H)
        b1[0] = 1 + 2 ** -9
        w3 = np.zeros(mlp.H)
        w3[0] = 1.0
        y, _ = mlp.forward_reference(_mlp_params(b1=b1, W2=W2, w3=w3), np.eye(16, dtype=np.int64)[:3])
        want = max((1 + 2 ** -9) * eff, 0.0)         # the second layer's ReLU
        assert (y == want).all()


def test_mlp_reference_layers_in_order_with_relu_and_biases():
    """Closed form over all three layers with every unit in use: W1 = c * ones
    (each hidden unit gets c * sum(x) = c, as the fractions sum to 1) plus b1_j,
    so h1_j = relu(c + b1_j); W2 = ones / 128 makes every h2 unit the mean of h1
    plus b2_j, through a ReLU; y = sum_j w3_j h2_j + b3.  Half of the b1 and b2
    entries are negative enough to be cut by the ReLUs, which a dropped ReLU,
    a sign error, a transposed W2 (it is not symmetric once row 0 is scaled) or
    a lost bias would change."""
    from oracle import mlp
    H = mlp.H
    c = 0.5
    b1 = np.where(np.arange(H) % 2 == 0, 0.25, -1.0)   # even units 0.75, odd units cut to 0
    W2 = np.full((H, H), 1.0 / H)
    W2[0] *= 2.0                                        # row 0 (unit 0) doubles its input
    b2 = np.where(np.arange(H) % 4 == 1, -2.0, 0.125)   # units 1, 5, 9, ... cut to 0
    w3 = (np.arange(H) - 64) / 64.0                     # multiples of 1/64: exact in bfloat16
    p = _mlp_params(np.full((H, mlp.IN), c), b1, W2, b2, w3, b3=0.375)
    h = np.array([[4] + [0] * 14 + [12], [1] * 16], dtype=np.int64)
    mean_h1 = (H // 2) * 0.75 / H                       # = 0.375
    h2 = np.array([max((2.0 if j == 0 else 1.0) * mean_h1 + b2[j], 0.0) for j in range(H)])
    want = float(np.dot(w3, h2) + 0.375)
    y, got_h2 = mlp.forward_reference(p, h)
    assert np.allclose(got_h2, h2[None, :], rtol=0, atol=1e-15)
    assert np.allclose(y, want, rtol=0, atol=1e-14)
    assert np.allclose(mlp.output_scale(p, got_h2),
                       np.dot(np.abs(w3), h2) + 0.375, rtol=0, atol=1e-14)


def test_mlp_kernel_model_stays_within_the_reference_tolerance():
    """The kernels' arithmetic model (x and h1 rounded to bfloat16) differs from
    the reference only by those two roundings, 2^-9 relative each, so on seeded
    weights and histograms its outputs stay within 1e-2 of the output scale;
    the largest deviation is a few 1e-3."""
    from oracle import mlp
    rng = np.random.default_rng(5)
    H, IN = mlp.H, mlp.IN
    p = _mlp_params(rng.uniform(-0.25, 0.25, (H, IN)), rng.uniform(-0.1, 0.1, H),
                    rng.uniform(-H ** -0.5, H ** -0.5, (H, H)), rng.uniform(-0.1, 0.1, H),
                    rng.uniform(-H ** -0.5, H ** -0.5, H), 0.2)
    hist = rng.multinomial(14, np.ones(16) / 16, size=4000)
    y, h2 = mlp.forward_reference(p, hist)
    dev = np.abs(mlp.forward(p, hist) - y) / mlp.output_scale(p, h2)
    assert dev.max() < 1e-2
    assert dev.max() > 1e-5  # the two forms do differ: the model rounds


@pytest.mark.parametrize("seed", range(4))
def test_safety_watch_closed_forms_without_rules(seed):
    """Independent processes: the states with process p in local state s are
    every combination of the other processes' reachable local states, so
    there are prod_{q != p} |R_q| violations (0 if s is unreachable in p's
    LTS).  Their digest is the digest of that product set.  The first one is
    at p's local BFS depth of s, where the only violating state has every
    other process still in its initial state."""
    net = inputs.no_sync_network(seed, n_procs=4, n_states=6, deg_lo=0, deg_hi=3)
    facts = [_local_facts(pr) for pr in net.procs]
    for p in range(4):
        for s in range(6):
            d = facts[p][0]
            r = oracle.explore(net, watch=(p, s))
            if s not in d:
                assert (r.violation_count, r.first_violation_level) == (0, -1)
                continue
            others = [sorted(facts[q][0]) for q in range(4) if q != p]
            combos = [c[:p] + (s,) + c[p:] for c in product(*others)]
            assert r.violation_count == len(combos)
            hs = [oracle.state_digest(list(c)) for c in combos]
            assert r.violation_sum == sum(hs) % (1 << 64)
            x = 0
            for h in hs:
                x ^= h
            assert r.violation_xor == x
            assert r.first_violation_level == d[s]
            r1 = oracle.explore(net, watch=(p, s), stop_at_first_violation=True)
            init = [pr.initial for pr in net.procs]
            init[p] = s
            assert r1.violation_count == 1 and r1.violations[0].tolist() == init
            # levels 0..depth are explored (the next one is built, not expanded)
            assert r1.explored == sum(r.levels[:d[s] + 1])
            assert r1.levels[:d[s] + 1] == r.levels[:d[s] + 1]


@pytest.mark.parametrize("n_nodes", [2, 3, 4, 5, 6])
def test_safety_watch_token_ring_closed_forms(n_nodes):
    """Token ring (Sec. 5.2), watching node k in h1 (local state 4).  The token
    holder is unique, so node k holds it in h1 in 3^(N-1) states (every other
    node in i0, i1 or i2).  The shortest path there takes 1 + 4k steps: node 0
    goes h0 -> h1, then each node j = 1..k makes two idle steps, receives the
    token, and goes h0 -> h1.  At that depth exactly one state violates."""
    net = inputs.token_ring(n_nodes)
    for k in range(n_nodes):
        r = oracle.explore(net, watch=(k, 4))
        assert r.violation_count == 3 ** (n_nodes - 1)
        assert r.first_violation_level == 1 + 4 * k
        r1 = oracle.explore(net, watch=(k, 4), stop_at_first_violation=True)
        assert r1.violation_count == 1
        assert r1.violations[0, k] == 4


@pytest.mark.parametrize("k", range(1, 11))
def test_producer_consumers_family_closed_forms(k):
    """Fig. 1 with k consumers.  Every combination of local states is
    reachable (2^(k+1) states).  Counting enabled transitions per state:
    gen_work in the 2^k states with the producer in p0; send/rec with consumer
    i in the 2^(k-1) states with the producer in p1 and consumer i in c0, for
    each i; work and tau of consumer i in the 2^k states with consumer i in
    c1.  No state is a deadlock."""
    r = oracle.explore(inputs.producer_consumers(k))
    assert r.states == 2 ** (k + 1)
    assert r.transitions == 2 ** k + k * 2 ** (k - 1) + k * 2 ** (k + 1)
    assert r.deadlock_count == 0
    if k == 2:
        assert (r.states, r.transitions) == (8, 24)


def product_closed_form(net, blocks):
    """States and transitions of inputs.product_network: the reachable set is the
    product of the blocks, so a process's local edge fires in every combination
    of the others' block states, and a rule fires once per combination of its
    participants' matching edges times every combination of the rest."""
    S = int(np.prod(blocks))
    in_rule = [set() for _ in net.procs]
    for r in net.rules:
        for p, a in r.parts:
            in_rule[p].add(a)
    T = 0
    for p, lts in enumerate(net.procs):
        local = sum(1 for s, a, t in lts.edges if s < blocks[p] and a not in in_rule[p])
        T += local * (S // blocks[p])
    for r in net.rules:
        m, c = 1, 1
        for p, a in r.parts:
            m *= sum(1 for s, b, t in net.procs[p].edges if s < blocks[p] and b == a)
            c *= blocks[p]
        T += m * (S // c)
    return S, T


@pytest.mark.parametrize("seed,n,ns,blocks,parties", [
    (0, 6, 8, [2, 3, 2, 3, 2, 2], 3), (1, 8, 16, [2, 3, 2, 3, 2, 2, 3, 2], 3),
    (2, 7, 16, [4, 1, 3, 2, 2, 3, 2], 2), (3, 9, 6, 2, 3), (4, 5, 64, [5, 4, 3, 6, 2], 3)])
def test_product_family_closed_forms(seed, n, ns, blocks, parties):
    net = inputs.product_network(seed, n, ns, blocks, parties=parties)
    b = blocks if isinstance(blocks, list) else [blocks] * n
    S, T = product_closed_form(net, b)
    r = oracle.explore(net)
    assert (r.states, r.transitions, r.deadlock_count) == (S, T, 0)
    assert any(len(rule.parts) == parties for rule in net.rules)


def test_planted_networks_have_exactly_the_planted_deadlocks():
    """The guided-search generator: a global state is a deadlock exactly when every
    process sits in a trap, so there are n_traps deadlocks (process 0 owns the traps,
    the others have one).  Each process needs two local moves to reach a trap (into
    its pre-trap state, which the initial state enters directly, then the fail edge),
    so the first deadlock is at BFS depth 2n exactly."""
    for seed in range(3):
        for n in (3, 4, 5):
            for k in (1, 2, 3):
                net = inputs.planted_network(seed, n, n_traps=k)
                r = oracle.explore(net, deadlocks_cap=64)
                assert r.deadlock_count == k and r.first_deadlock_level == 2 * n
                ns0 = net.procs[0].n_states
                assert sorted(int(d[0]) for d in r.deadlocks) == list(range(ns0 - k, ns0))
                for d in r.deadlocks:
                    assert all(int(d[p]) == net.procs[p].n_states - 1 for p in range(1, n))
