"""Learned guidance for deadlock search, against the oracle.

* Distance labels computed on the GPU equal the oracle's backward BFS.
* The MLP's forward pass and gradient match a float64 reference.
* Training lowers the loss.
* Guided search reports a deadlock with a path the oracle replays step by
  step, explores fewer states than breadth-first search, and is exhaustive
  when there is no deadlock.
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1801_05857_gb300 import guide, gx, inputs

pytestmark = pytest.mark.gpu

MAX_DIST = 64


def _hist(states):
    return np.stack([np.bincount(s, minlength=16)[:16] for s in states]).astype(np.int64)


@pytest.mark.parametrize("net", [inputs.planted_network(s, n, n_traps=k) for s, n, k in
                                 ((0, 6, 1), (1, 6, 4), (2, 7, 2), (3, 8, 3))] +
                         [inputs.random_network(6, 4, 5, 0, 2, 6, n_sync=2, parties=2),
                          inputs.token_ring(6)], ids=lambda n: n.name)
def test_labels_equal_oracle_backward_bfs(cuda, net):
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=1 << 24, hash_rounds=32)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    hist, label = gx.training_set(h, ws, MAX_DIST)
    states, dist = oracle.deadlock_distances(net)
    want = sorted(zip(map(tuple, _hist(states)),
                      [min(int(d), MAX_DIST) for d in dist]))
    got = sorted(zip(map(tuple, hist.cpu().numpy().astype(np.int64)),
                     [int(round(float(x) * MAX_DIST)) for x in label.cpu().numpy()]))
    assert got == want


def test_mlp_forward_and_gradient_match_float64(cuda):
    import torch
    p = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
    gx.mlp_init(p, 3)
    rng = np.random.default_rng(1)
    hist_np = rng.integers(0, 9, size=(1000, 16)).astype(np.uint8)
    label_np = rng.random(1000).astype(np.float32)
    hist = torch.from_numpy(hist_np).cuda()
    label = torch.from_numpy(label_np).cuda()
    pn = p.cpu().numpy()
    y = gx.mlp_forward(p, hist).cpu().numpy()
    yr = omlp.forward(pn, hist_np)
    assert np.max(np.abs(y - yr) / np.maximum(np.abs(yr), 1e-3)) < 1e-2
    assert np.max(np.abs(y - yr)) < 1e-4
    g, loss = gx.mlp_grad(p, hist, label)
    lr_, gr = omlp.loss_and_grad(pn, hist_np, label_np)
    g = g.cpu().numpy()
    assert abs(float(loss.item()) - lr_) <= 1e-4 * lr_ + 1e-7
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr)) + 1e-7


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 256 * 128 + 300])
def test_tensor_core_gradient_tiles_match_float64(cuda, n):
    """The gradient on the tensor cores, one 128-example tile per product: a single
    example, ragged tails, and more tiles than CTAs (256 at most), so that a CTA
    accumulates several tiles in TMEM.  Against the float64 gradient of the kernels'
    arithmetic model within 1e-3 of its largest entry; the loss within 1e-4."""
    import torch
    p = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
    gx.mlp_init(p, 11)
    rng = np.random.default_rng(n)
    hist_np = rng.multinomial(10, np.ones(16) / 16, size=n).astype(np.uint8)
    label_np = rng.random(n).astype(np.float32)
    g, loss = gx.mlp_grad(p, torch.from_numpy(hist_np).cuda(), torch.from_numpy(label_np).cuda())
    lr_, gr = omlp.loss_and_grad(p.cpu().numpy(), hist_np, label_np)
    g = g.cpu().numpy()
    assert np.isfinite(g).all()
    assert abs(float(loss.item()) - lr_) <= 1e-4 * lr_ + 1e-7
    assert np.max(np.abs(g - gr)) <= 1e-3 * np.max(np.abs(gr)) + 1e-7


@pytest.mark.parametrize("n", [1, 127, 128, 129, 4099, 152 * 4 * 128 * 2 + 77])
def test_tensor_core_forward_tiles_match_float64(cuda, n):
    """gx_mlp_forward scores 128 states per tile on the tensor cores; ragged
    tails, a single state, and more tiles than CTAs (each CTA loops) must all
    equal the float64 network with BF16 operands.  Rows 0 and 1 are the
    extreme inputs: every process in local state 15, and all 16 processes in
    state 0."""
    import torch
    p = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
    gx.mlp_init(p, 7)
    rng = np.random.default_rng(n)
    hist_np = rng.multinomial(12, np.ones(16) / 16, size=n).astype(np.uint8)
    hist_np[0] = 0
    hist_np[0, 15] = 16
    if n > 1:
        hist_np[1] = 0
        hist_np[1, 0] = 16
    y = gx.mlp_forward(p, torch.from_numpy(hist_np).cuda()).cpu().numpy()
    pick = np.unique(np.concatenate([np.arange(min(n, 300)), rng.integers(0, n, 700), [n - 1]]))
    assert np.isfinite(y).all()
    _check_scores(p.cpu().numpy(), hist_np[pick], y[pick])


def _check_scores(pn, hist_np, y):
    """Scores against the FP64 reference (the network's definition: BF16 weights,
    float64 features, activations and sums) within 1e-2 of each output's scale
    (sum_j |w3_j| h2_j + |b3|), element by element; and against the kernels'
    arithmetic model (x and h1 also rounded to BF16) within 1e-4 absolute, the
    tighter check of where they round."""
    yr, h2 = omlp.forward_reference(pn, hist_np)
    rel = np.abs(y - yr) / omlp.output_scale(pn, h2)
    assert rel.max() <= 1e-2, (rel.argmax(), y[rel.argmax()], yr[rel.argmax()])
    assert np.max(np.abs(y - omlp.forward(pn, hist_np))) < 1e-4


@pytest.mark.parametrize("n", [1, 127, 128, 129, 4099, 152 * 4 * 128 * 2 + 77])
def test_trained_scores_match_float64_reference(cuda, trained_params, n):
    """The same tile sizes with a trained guide, whose outputs are distance
    estimates in [0, 1] rather than near-zero sums of cancelling terms: every
    score is also within 1e-2 of the reference relative to the score itself
    wherever the score is at least 0.05 in size."""
    import torch
    rng = np.random.default_rng(100 + n)
    k = rng.integers(6, 17, size=n)
    hist_np = np.stack([np.bincount(rng.integers(0, 16, kk), minlength=16) for kk in k]).astype(np.uint8)
    y = gx.mlp_forward(trained_params, torch.from_numpy(hist_np).cuda()).cpu().numpy()
    pn = trained_params.cpu().numpy()
    _check_scores(pn, hist_np, y)
    yr, _ = omlp.forward_reference(pn, hist_np)
    big = np.abs(yr) >= 0.05
    assert big.any() or n == 1
    assert np.max(np.abs(y[big] - yr[big]) / np.abs(yr[big])) <= 1e-2


@pytest.fixture(scope="module")
def trained_params(cuda):
    params, _ = _trained(600)
    return params


def _trained(steps=600):
    nets = [inputs.planted_network(s, n, n_traps=1 + s % 4) for s in range(6) for n in (6, 7, 8)]
    hist, label = guide.collect_examples(nets, MAX_DIST)
    params, losses = guide.train(hist, label, steps=steps)
    return params, losses.cpu().numpy()


def test_training_lowers_the_loss(cuda):
    """The histogram features cannot tell which states have lost every path to a
    deadlock (that depends on the instance's local graphs), so the loss has a floor;
    training still has to halve it."""
    _, losses = _trained(400)
    assert losses[-50:].mean() < 0.5 * losses[:10].mean()


def _replay(net, trace):
    init = [p.initial for p in net.procs]
    assert list(trace[0]) == init
    for a, b in zip(trace[:-1], trace[1:]):
        succ = {tuple(x) for x in oracle.successors(net, a)}
        assert tuple(b) in succ
    assert len(oracle.successors(net, trace[-1])) == 0


def _guided(net, params, table_bytes=1 << 27, **kw):
    h = gx.load_network(net)
    gx.guided_set_weights(h, params)
    o = gx.default_opts(table_bytes=table_bytes, hash_rounds=32, **kw)
    ws = gx.guided_alloc_workspace(h, o)
    n, found = gx.find_deadlocks(h, gx.GX_DL_GUIDED, o, ws)
    return h, n, found, gx.stats(h)


def _bfs_first(net):
    h = gx.load_network(net)
    o = gx.default_opts(table_bytes=4 << 30, hash_rounds=32, frontier_states=1 << 27)
    ws = gx.alloc_workspace(h, o)
    n, found = gx.find_deadlocks(h, gx.GX_DL_BFS_FIRST, o, ws)
    return n, gx.stats(h)


@pytest.mark.parametrize("fused", [0, 1], ids=["split", "fused"])
@pytest.mark.parametrize("seed,n_procs,k", [(10, 9, 1), (11, 10, 3), (12, 12, 2)])
def test_guided_search_finds_a_replayable_deadlock_faster_than_bfs(cuda, seed, n_procs, k, fused):
    params, _ = _trained()
    net = inputs.planted_network(seed, n_procs, n_traps=k)
    h, n, found, s = _guided(net, params, guided_fused=fused)
    assert n == 1 and s["deadlock_count"] == 1
    trace = gx.guided_trace(h)
    _replay(net, trace)
    assert list(found[0]) == list(trace[-1])
    nb, sb = _bfs_first(net)
    assert nb >= 1
    assert s["explored"] < sb["explored"]


def test_trained_network_beats_untrained(cuda):
    import torch
    params, _ = _trained()
    untrained = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device="cuda")
    gx.mlp_init(untrained, 99)
    net = inputs.planted_network(21, 11, n_traps=2)
    _, n1, _, s1 = _guided(net, params, table_bytes=1 << 29)
    _, n2, _, s2 = _guided(net, untrained, table_bytes=1 << 29)
    assert n1 == 1 and n2 == 1
    assert s1["explored"] < s2["explored"]


@pytest.mark.parametrize("fused", [0, 1], ids=["split", "fused"])
def test_guided_search_without_deadlock_is_exhaustive(cuda, fused):
    params, _ = _trained(100)
    net = inputs.token_ring(8)
    h, n, found, s = _guided(net, params, guided_batch=256, guided_fused=fused)
    assert n == 0 and s["complete"] == 1 and s["deadlock_count"] == 0
    r = oracle.explore(net)
    assert s["states"] == r.states and s["explored"] == r.states
    assert s["transitions"] == r.transitions


@pytest.mark.parametrize("fused", [0, 1], ids=["split", "fused"])
@pytest.mark.parametrize("host_loop", [0, 1])
def test_device_and_host_iteration_loops(cuda, host_loop, fused):
    """The guided search runs as one graph (device loop) or one host round trip
    per iteration, with the scoring in its own kernel or inside the expansion;
    each finds a replayable deadlock, and each is exhaustive on a network
    without one."""
    params, _ = _trained(200)
    net = inputs.planted_network(10, 9, n_traps=1)
    h, n, found, s = _guided(net, params, host_loop=host_loop, guided_fused=fused)
    assert n == 1 and s["deadlock_count"] == 1
    trace = gx.guided_trace(h)
    _replay(net, trace)
    assert list(found[0]) == list(trace[-1])
    ring = inputs.token_ring(7)
    _, n2, _, s2 = _guided(ring, params, host_loop=host_loop, guided_batch=512, guided_fused=fused)
    r = oracle.explore(ring)
    assert n2 == 0 and s2["complete"] == 1 and (s2["states"], s2["transitions"]) == (r.states, r.transitions)


def test_path_longer_than_the_batch_buffer(cuda):
    """With 16-state batches the deadlock's path (2n + 1 states deep) no longer fits
    the buffer the device walk uses, and the host walks it entry by entry."""
    params, _ = _trained(200)
    net = inputs.planted_network(3, 10, n_traps=1)
    h, n, found, s = _guided(net, params, guided_batch=16)
    assert n == 1
    trace = gx.guided_trace(h)
    assert len(trace) > 16
    _replay(net, trace)


def test_training_and_gradients_are_deterministic(cuda):
    """Examples sorted by content, partial gradients per CTA summed in a fixed
    order: exploring, labelling and training twice from scratch gives
    bit-identical examples and weights, and a gradient does not depend on
    scheduling."""
    import torch
    nets = [inputs.planted_network(s, n, n_traps=1 + s % 4) for s in range(2) for n in (6, 7)]
    hist, label = guide.collect_examples(nets, MAX_DIST)
    hist2, label2 = guide.collect_examples(nets, MAX_DIST)
    assert torch.equal(hist, hist2) and torch.equal(label, label2)
    # one network's examples ascend as (the 16 histogram bytes as 4 words, label bits)
    h = gx.load_network(nets[0])
    o = gx.default_opts(table_bytes=1 << 26, bucket_words=8, group_lanes=1, hash_rounds=32)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    h1, l1 = gx.training_set(h, ws, MAX_DIST)
    words = h1.contiguous().view(torch.int32).view(-1, 4).cpu().numpy().view(np.uint32).astype(np.uint64)
    bits = l1.cpu().numpy().view(np.uint32).astype(np.uint64)
    rows = list(zip(*[words[:, c].tolist() for c in range(4)], bits.tolist()))
    assert len(rows) > 1000 and all(rows[i] <= rows[i + 1] for i in range(len(rows) - 1))
    p1, l1 = guide.train(hist, label, steps=200)
    p2, l2 = guide.train(hist2, label2, steps=200)
    assert torch.equal(p1, p2) and torch.equal(l1, l2)
    g1, s1 = gx.mlp_grad(p1, hist, label)
    g2, s2 = gx.mlp_grad(p1, hist, label)
    assert torch.equal(g1, g2) and torch.equal(s1, s2)
