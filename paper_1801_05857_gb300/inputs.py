"""Seeded synthetic inputs: networks of LTSs and key sequences.

This module only *draws* inputs. It holds none of the exploration arithmetic
(no successor generation, no packing, no hashing of states), so the CPU oracle
and the CUDA path can both be fed from it without sharing any of the method.

A network (Sec. 3, Fig. 1) is a list of process LTSs -- each a set of local
states, an initial state and labelled edges -- plus synchronisation rules.  A
rule lists (process, label) participants; those participants move together,
and a label that a process uses in some rule never fires alone in that
process.  Every other (process, label) pair interleaves.

Randomness comes from a splitmix64 stream (Steele, Lea & Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014), written out in plain
Python integers so that the same seed gives the same network on any machine.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

M64 = (1 << 64) - 1


class SplitMix64:
    """splitmix64 generator: state += golden gamma, then the two-multiply finaliser."""

    def __init__(self, seed: int):
        self.state = seed & M64

    def next(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & M64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        return z ^ (z >> 31)

    def below(self, n: int) -> int:
        """Uniform-ish integer in [0, n) (modulo bias < n / 2^64)."""
        return self.next() % n

    def between(self, lo: int, hi: int) -> int:
        """Integer in [lo, hi] inclusive."""
        return lo + self.below(hi - lo + 1)

    def sample(self, n: int, k: int) -> list[int]:
        """k distinct values from range(n), partial Fisher-Yates."""
        pool = list(range(n))
        for i in range(k):
            j = i + self.below(n - i)
            pool[i], pool[j] = pool[j], pool[i]
        return pool[:k]


def substream(seed: int, *path: int) -> SplitMix64:
    """Independent stream for (seed, path...): each component is folded through one draw."""
    g = SplitMix64(seed)
    s = g.next()
    for p in path:
        s = SplitMix64(s ^ ((p + 1) * 0xD1B54A32D192ED03 & M64)).next()
    return SplitMix64(s)


@dataclass
class LTS:
    n_states: int
    initial: int
    edges: list  # list of (src, label, dst)


@dataclass
class Rule:
    parts: list  # list of (proc, label); processes are distinct
    result: int = 0


@dataclass
class Network:
    n_labels: int
    procs: list
    rules: list = field(default_factory=list)
    name: str = ""

    @property
    def n_procs(self) -> int:
        return len(self.procs)

    def flat(self) -> dict:
        """Plain arrays for marshalling across a C boundary.

        edges[e] = (src, label, dst) with process p's edges in
        edges[edge_off[p]:edge_off[p+1]]; rule r's participants are
        rule_parts[rule_off[r]:rule_off[r+1]] as (proc, label) rows.
        """
        n = self.n_procs
        n_states = np.array([p.n_states for p in self.procs], dtype=np.uint32)
        initial = np.array([p.initial for p in self.procs], dtype=np.uint32)
        edge_off = np.zeros(n + 1, dtype=np.uint32)
        rows = []
        for i, p in enumerate(self.procs):
            rows.extend(p.edges)
            edge_off[i + 1] = edge_off[i] + len(p.edges)
        edges = np.array(rows, dtype=np.uint32).reshape(-1, 3)
        rule_off = np.zeros(len(self.rules) + 1, dtype=np.uint32)
        parts = []
        for r, rule in enumerate(self.rules):
            parts.extend(rule.parts)
            rule_off[r + 1] = rule_off[r] + len(rule.parts)
        rule_parts = np.array(parts, dtype=np.uint32).reshape(-1, 2)
        rule_result = np.array([r.result for r in self.rules], dtype=np.uint32)
        return dict(n_procs=n, n_labels=self.n_labels, n_states=n_states, initial=initial,
                    edge_off=edge_off, edges=np.ascontiguousarray(edges),
                    rule_off=rule_off, rule_parts=np.ascontiguousarray(rule_parts),
                    rule_result=rule_result)


# --------------------------------------------------------------------------------------------
# Hand-written networks
# --------------------------------------------------------------------------------------------

def producer_consumers(n_consumers: int = 2) -> Network:
    """The producer / consumers network of Fig. 1 (two consumers there).

    Labels: 0 gen_work, 1 send, 2 rec, 3 work, 4 tau, 5 trans.
    Producer: p0 -gen_work-> p1, p1 -send-> p0.
    Consumer: c0 -rec-> c1, c1 -work-> c1, c1 -tau-> c0.
    Rules: one per consumer i, send (producer) * rec (consumer i) -> trans.
    With k consumers every combination of local states is reachable:
    2^(k+1) states and 2^k + k 2^(k-1) + k 2^(k+1) transitions (8 and 24 for
    k = 2, the counts the paper gives for Fig. 1).
    """
    producer = LTS(2, 0, [(0, 0, 1), (1, 1, 0)])
    consumer = lambda: LTS(2, 0, [(0, 2, 1), (1, 3, 1), (1, 4, 0)])
    rules = [Rule([(0, 1), (i, 2)], 5) for i in range(1, n_consumers + 1)]
    name = "fig1_producer_consumers" if n_consumers == 2 else f"producer_consumers_{n_consumers}"
    return Network(6, [producer] + [consumer() for _ in range(n_consumers)], rules, name=name)


def token_ring(n_nodes: int) -> Network:
    """A ring of n nodes passing one token forward (Sec. 5.2 describes the model only in words).

    Each node has two communication transitions (receive from the left
    neighbour, send to the right one) and three internal transitions:
      idle states i0 -> i1 -> i2 (two internal steps),
      i2 -recv-> h0 (token arrives), h0 -> h1 (internal), h1 -send-> i0.
    Local state numbering: i0=0, i1=1, i2=2, h0=3, h1=4 (3 bits per node).
    Node 0 starts holding the token in h0, all others in i0.
    Label 2k+0 is node k's internal step label, one 'pass_k' label per link
    k -> k+1 is shared by node k (send) and node k+1 (recv) through a 2-party rule.
    """
    assert n_nodes >= 2
    tau = 0
    procs = []
    for k in range(n_nodes):
        send = 1 + k                      # link k -> k+1
        recv = 1 + (k - 1) % n_nodes      # link k-1 -> k
        edges = [(0, tau, 1), (1, tau, 2), (3, tau, 4), (2, recv, 3), (4, send, 0)]
        procs.append(LTS(5, 3 if k == 0 else 0, edges))
    rules = [Rule([(k, 1 + k), ((k + 1) % n_nodes, 1 + k)], 1 + k) for k in range(n_nodes)]
    return Network(1 + n_nodes, procs, rules, name=f"token_ring_{n_nodes}")


# --------------------------------------------------------------------------------------------
# Random networks
# --------------------------------------------------------------------------------------------

def random_lts(rng: SplitMix64, n_states: int, deg_lo: int, deg_hi: int, labels: list,
               initial: int = 0, cluster: int = 0, free_labels=()) -> LTS:
    """Each state gets U{deg_lo..deg_hi} distinct (label, dst) edges, label uniform over `labels`.

    With cluster > 0 the states form consecutive blocks of `cluster` states;
    an edge stays inside its source's block unless its label is in
    `free_labels`, in which case its destination is uniform over all states.
    """
    edges = []
    for s in range(n_states):
        d = rng.between(deg_lo, deg_hi)
        seen = set()
        while len(seen) < d:
            a = labels[rng.below(len(labels))]
            if cluster and a not in free_labels:
                base = (s // cluster) * cluster
                t = base + rng.below(min(cluster, n_states - base))
            else:
                t = rng.below(n_states)
            if (a, t) not in seen:
                seen.add((a, t))
                edges.append((s, a, t))
    return LTS(n_states, initial, edges)


def random_network(seed: int, n_procs: int, n_states, deg_lo: int = 1, deg_hi: int = 3,
                   n_labels: int = 6, n_sync: int = 2, parties: int = 2,
                   sync_weight: float = 1.0, cluster: int = 0, name: str = "") -> Network:
    """Random network in the style of the paper's benchmark models.

    * n_states: int or a list with one entry per process.
    * Labels 0..n_sync-1 synchronise: label a gets one rule over `parties`
      distinct processes chosen once (a fixed rendezvous group); the others
      are local.
    * cluster > 0: local edges stay inside blocks of `cluster` consecutive
      states and only synchronised edges lead out of a block, so rules gate
      how far each process can wander (this is what keeps the product small
      enough to enumerate).
    * sync_weight scales how often a process picks, for an edge, one of the
      sync labels it takes part in, relative to a local label (1.0 = uniform
      over all labels it may use).  A process only draws labels that are
      local or that it shares through a rule.
    """
    sizes = list(n_states) if isinstance(n_states, (list, tuple)) else [n_states] * n_procs
    top = substream(seed, 0)
    rules = []
    member = [[] for _ in range(n_procs)]
    for a in range(n_sync):
        ps = sorted(top.sample(n_procs, parties))
        rules.append(Rule([(p, a) for p in ps], a))
        for p in ps:
            member[p].append(a)
    local = list(range(n_sync, n_labels))
    procs = []
    for p in range(n_procs):
        rng = substream(seed, 1, p)
        mine = member[p]
        if sync_weight == 1.0 or not mine:
            pool = local + mine
        else:
            # integer weights: repeat labels so the draw stays a plain uniform pick
            w_sync = max(1, int(round(sync_weight * 4)))
            pool = local * 4 + mine * w_sync
        procs.append(random_lts(rng, sizes[p], deg_lo, deg_hi, pool, cluster=cluster,
                                free_labels=set(mine)))
    return Network(n_labels, procs, rules, name=name or f"random_s{seed}_n{n_procs}")


def product_network(seed: int, n_procs: int, n_states: int, blocks, n_labels: int = 30,
                    sync_frac: float = 0.1, parties: int = 3, deg_lo: int = 1, deg_hi: int = 3,
                    name: str = "") -> Network:
    """Memory-scaled family whose reachable set is a product (counts in closed form).

    * blocks: int or one entry per process: process p reaches local states
      0..blocks[p]-1 (its block) and no other; the remaining states up to
      n_states exist only to widen the vector (bits = ceil(log2 n_states)).
    * round(sync_frac * n_labels) labels synchronise, each as one rule over
      `parties` distinct processes; the other labels are local.
    * Every block state has a local edge to the next block state (a cycle, so
      the block is reachable and no state is a deadlock) plus
      U{deg_lo-1..deg_hi-1} more edges inside the block, labelled with a local
      label or one of the process's rule labels.  States outside the block
      only have edges among themselves.
    Every combination of block states is then reachable by local moves, and
    rule edges never leave the blocks, so the state space is the product of
    the blocks.
    """
    sizes = list(blocks) if isinstance(blocks, (list, tuple)) else [blocks] * n_procs
    assert all(1 <= c <= n_states for c in sizes)
    top = substream(seed, 0)
    n_sync = max(1, int(round(sync_frac * n_labels)))
    rules, member = [], [[] for _ in range(n_procs)]
    for a in range(n_sync):
        ps = sorted(top.sample(n_procs, parties))
        rules.append(Rule([(p, a) for p in ps], a))
        for p in ps:
            member[p].append(a)
    local = list(range(n_sync, n_labels))
    procs = []
    for p in range(n_procs):
        rng = substream(seed, 4, p)
        c = sizes[p]
        pool = local + member[p]
        edges = []
        for lo, hi in ((0, c), (c, n_states)):
            for st in range(lo, hi):
                seen = set()
                if lo == 0:  # the block's cycle
                    a = local[rng.below(len(local))]
                    t = lo + (st - lo + 1) % (hi - lo)
                    seen.add((a, t))
                    edges.append((st, a, t))
                extra = rng.between(deg_lo, deg_hi) - (1 if lo == 0 else 0)
                while len(seen) < extra + (1 if lo == 0 else 0):
                    a = pool[rng.below(len(pool))]
                    t = lo + rng.below(hi - lo)
                    if (a, t) not in seen:
                        seen.add((a, t))
                        edges.append((st, a, t))
        procs.append(LTS(n_states, 0, edges))
    return Network(n_labels, procs, rules, name=name or f"product_s{seed}_n{n_procs}")


def planted_network(seed: int, n_procs: int, n_traps: int = 1, n_states: int = 16,
                    deg_lo: int = 1, deg_hi: int = 3, cluster: int = 3, sync_frac: float = 0.3,
                    risk_edges: int = 2, name: str = "") -> Network:
    """Network with planted deadlocks (the guided-search workload).

    Per process: states 0..n_states-3 form a random LTS as in random_network
    (local edges inside blocks of `cluster` states, some two-party rules), and
    every one of them keeps at least one local edge, so no process is ever
    blocked there.  State n_states-2 ("pre-trap") is entered by `risk_edges`
    local edges from states of the initial block (always including the initial
    state 0) and leaves by a local edge
    back to state 0 or by a local "fail" edge into the trap state n_states-1,
    which has no outgoing edge.  Process 0 has n_traps trap states (the last
    n_traps indices; the pre-trap is the index before them) with a fail edge
    into each.  A global state is a deadlock exactly when every process sits in
    a trap state, so the network has exactly n_traps deadlocks, all reachable.
    """
    top = substream(seed, 0)
    n_labels = 4 * n_procs
    n_sync = max(1, int(round(sync_frac * n_labels)))
    # labels: [0, n_sync) rule labels, then per process: a local pool, risk, back, fail
    rules, member = [], [[] for _ in range(n_procs)]
    for a in range(n_sync):
        ps = sorted(top.sample(n_procs, 2))
        rules.append(Rule([(p, a) for p in ps], a))
        for p in ps:
            member[p].append(a)
    locals_ = list(range(n_sync, n_labels))
    procs = []
    for p in range(n_procs):
        rng = substream(seed, 3, p)
        traps = n_traps if p == 0 else 1
        pre = n_states - 1 - traps
        normal = pre  # states 0..pre-1
        pool = locals_ + member[p]
        edges = []
        for s in range(normal):
            d = rng.between(deg_lo, deg_hi)
            seen = set()
            # one guaranteed local edge, inside the block
            base = (s // cluster) * cluster
            t = base + rng.below(min(cluster, normal - base))
            a = locals_[rng.below(len(locals_))]
            seen.add((a, t))
            edges.append((s, a, t))
            while len(seen) < d:
                a = pool[rng.below(len(pool))]
                if a in member[p]:
                    t = rng.below(normal)
                else:
                    t = base + rng.below(min(cluster, normal - base))
                if (a, t) not in seen:
                    seen.add((a, t))
                    edges.append((s, a, t))
        risk, back, fail = locals_[0], locals_[1], locals_[2]
        for s in sorted({0} | set(rng.below(min(cluster, normal)) for _ in range(risk_edges - 1))):
            edges.append((s, risk, pre))
        edges.append((pre, back, 0))
        for k in range(traps):
            edges.append((pre, fail, pre + 1 + k))
        procs.append(LTS(n_states, 0, edges))
    return Network(n_labels, procs, rules, name=name or f"planted_s{seed}_n{n_procs}_k{n_traps}")


def no_sync_network(seed: int, n_procs: int, n_states: int, deg_lo: int = 0, deg_hi: int = 2,
                    n_labels: int = 4) -> Network:
    """Random network without rules; deg_lo = 0 allows local sink states (deadlocks)."""
    procs = []
    for p in range(n_procs):
        rng = substream(seed, 2, p)
        procs.append(random_lts(rng, n_states, deg_lo, deg_hi, list(range(n_labels))))
    return Network(n_labels, procs, [], name=f"nosync_s{seed}_n{n_procs}")


# --------------------------------------------------------------------------------------------
# Named workloads (generator arguments)
# --------------------------------------------------------------------------------------------

WORKLOADS = {
    # 4 processes x 8 local states (3 bits, one word), out-degree 1-3 over 6 labels,
    # 2 labels as two-party rules between fixed pairs; 2^16-word table, 32-word buckets
    "tiny": dict(seed=0, n_procs=4, n_states=8, deg_lo=1, deg_hi=3, n_labels=6, n_sync=2,
                 parties=2, name="tiny_s0"),
    # 10 processes x 16 local states (4 bits, 40 bits -> 2 words), out-degree 1-3,
    # 12 labels of which 4 (30 %) are two-party rules; local edges stay in blocks of 8
    # states; 2^28-word table
    "mid": dict(seed=11, n_procs=10, n_states=16, deg_lo=1, deg_hi=3, n_labels=12, n_sync=4,
                parties=2, cluster=8, name="mid_s11"),
}


# Memory-scaled workloads: product networks (every combination of block states is
# reachable, so states and transitions are closed forms at any size).
PRODUCT_WORKLOADS = {
    # 16 processes x 16 local states (4 bits each: 3 words, padded to 4-word slots),
    # 3-party rules on 3 of 30 labels (10 %), out-degree 1-2 inside blocks of 4 local
    # states (one of 5): 4^15 * 5 = 5.37e9 states, 62.5 % of a 2^33-slot (128 GiB) table
    "scaled": dict(seed=7, n_procs=16, n_states=16, blocks=[4] * 15 + [5], deg_lo=1, deg_hi=2,
                   name="scaled_s7_n16"),
    # the same family taken to 90 % fill: 20 processes, out-degree 1-3, blocks of 3
    # (one of 4, one of 5): 7.75e9 states in 2^33 slots
    "scaled90": dict(seed=7, n_procs=20, n_states=16, blocks=[3] * 18 + [4, 5], name="scaled90_s7_n20"),
}


def workload(name: str) -> Network:
    if name in PRODUCT_WORKLOADS:
        return product_network(**PRODUCT_WORKLOADS[name])
    return random_network(**WORKLOADS[name])


def workload_params(name: str) -> dict:
    return dict(PRODUCT_WORKLOADS[name]) if name in PRODUCT_WORKLOADS else dict(WORKLOADS[name])


def batch_params(seed: int) -> dict:
    """Generator arguments of one network of the batched workload: 4-10 processes
    x 8-32 local states, out-degree 1-3, about half the processes in two-party
    rules, local edges in blocks of 4-8 states."""
    r = substream(seed, 77)
    n = r.between(4, 10)
    ns = r.between(8, 32)
    cl = r.between(4, 8)
    nl = 2 * n + r.between(0, 4)
    nsync = max(1, min(nl - 1, n // 2 + 1 + r.between(0, 3)))
    return dict(seed=1000 + seed, n_procs=n, n_states=ns, deg_lo=1, deg_hi=3, n_labels=nl,
                n_sync=nsync, parties=2, cluster=cl, name=f"batch_{seed}")


# Seeds of batch_params whose networks have 10^3..10^6 reachable states, chosen by
# tests/golden/make_golden.py (it runs the oracle on candidate seeds in order and keeps
# those in range); the batched workload is the first 256 of them.
BATCH_SEEDS = [
    0, 1, 2, 3, 4, 6, 7, 8, 11, 13, 15, 19, 21, 22, 23, 24,
    28, 29, 30, 31, 32, 33, 35, 36, 37, 38, 42, 44, 45, 47, 48, 49,
    51, 52, 53, 54, 55, 56, 58, 60, 61, 63, 66, 67, 69, 70, 71, 72,
    73, 74, 75, 76, 79, 80, 82, 83, 84, 85, 87, 88, 89, 90, 91, 92,
    94, 97, 100, 101, 102, 103, 104, 105, 110, 111, 112, 113, 114, 116, 117, 118,
    120, 126, 127, 128, 129, 130, 131, 134, 136, 137, 138, 139, 140, 141, 142, 144,
    149, 150, 151, 152, 155, 156, 157, 159, 160, 161, 162, 164, 165, 166, 169, 170,
    171, 173, 174, 176, 178, 180, 181, 182, 185, 186, 189, 191, 192, 193, 194, 197,
    198, 200, 201, 202, 205, 207, 208, 210, 211, 213, 214, 215, 216, 217, 219, 220,
    221, 224, 228, 230, 232, 234, 235, 238, 239, 240, 241, 243, 244, 247, 248, 249,
    250, 251, 252, 253, 254, 255, 256, 257, 260, 264, 265, 267, 268, 271, 272, 273,
    276, 279, 282, 283, 284, 285, 286, 289, 290, 291, 292, 294, 296, 297, 298, 299,
    300, 301, 303, 304, 305, 306, 307, 312, 313, 315, 316, 317, 318, 320, 321, 322,
    325, 327, 328, 329, 330, 331, 332, 333, 335, 336, 337, 338, 339, 340, 343, 344,
    345, 347, 349, 350, 351, 352, 353, 355, 356, 357, 358, 359, 361, 362, 363, 365,
    366, 367, 369, 371, 373, 374, 376, 377, 379, 380, 381, 382, 383, 384, 387, 389,
]


def batch_workload(count: int = 256) -> list:
    return [random_network(**batch_params(s)) for s in BATCH_SEEDS[:count]]


# --------------------------------------------------------------------------------------------
# Key sequences for the isolated hash-table experiment (Sec. 5.1)
# --------------------------------------------------------------------------------------------

def _mix31(i: np.ndarray, seed: int) -> np.ndarray:
    """Bijection on [0, 2^31): odd multiply and xor-shifts, each invertible mod 2^31."""
    m = np.uint64((1 << 31) - 1)
    x = (i.astype(np.uint64) + np.uint64(seed & 0x7FFFFFFF)) & m
    for mul in (0x2C1B3C6D, 0x297A2D39, 0x7FEB352D):
        x = (x * np.uint64(mul | 1)) & m
        x ^= x >> np.uint64(15)
    return x


def key_sequence(n: int, duplication: int, words: int = 1, seed: int = 0) -> np.ndarray:
    """n keys of `words` uint32 each, n // duplication distinct ones, each repeated
    `duplication` times, in a seeded random order (the paper's Sec. 5.1 input).

    Keys are nonzero and keep bit 31 of every word clear.  Distinctness comes
    from a bijection of the unique index in word 0, so no duplicates can
    arise by chance.  Returns a (n, words) uint32 array (n must be a multiple
    of duplication).
    """
    assert n % duplication == 0
    u = n // duplication
    idx = np.arange(u, dtype=np.uint64)
    w0 = _mix31(idx, seed)
    # the bijection sends exactly one index to 0; give that key the image of u instead,
    # which no index below u can have
    w0 = np.where(w0 == 0, _mix31(np.array([u], dtype=np.uint64), seed)[0], w0)
    cols = [w0.astype(np.uint32)]
    for k in range(1, words):
        cols.append(_mix31(idx, seed * 7919 + 104729 * k).astype(np.uint32))
    uniq = np.stack(cols, axis=1)
    order = np.random.Generator(np.random.PCG64(seed)).permutation(n) % u
    return np.ascontiguousarray(uniq[order])


def key_sequence_device(n: int, duplication: int, seed: int = 0, device="cuda"):
    """The same distinct keys as key_sequence(words=1), generated on a torch device.

    The order comes from torch.randperm with a seeded generator instead of
    numpy's PCG64, so it differs from key_sequence's order; the multiset of keys
    is identical.  Returns an int32 tensor of n keys (bit patterns of uint32).
    """
    import torch
    assert n % duplication == 0
    u = n // duplication
    m = (1 << 31) - 1

    def mix31(i):
        x = (i + (seed & 0x7FFFFFFF)) & m
        for mul in (0x2C1B3C6D, 0x297A2D39, 0x7FEB352D):
            x = (x * (mul | 1)) & m
            x = x ^ (x >> 15)
        return x

    w0 = mix31(torch.arange(u, dtype=torch.int64, device=device))
    w0 = torch.where(w0 == 0, mix31(torch.tensor([u], dtype=torch.int64, device=device)), w0)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    order = torch.randperm(n, generator=g, device=device) % u
    return w0[order].to(torch.int32)
