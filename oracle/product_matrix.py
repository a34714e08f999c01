"""Brute-force pin for the BFS oracle -- TEST INFRASTRUCTURE ONLY.

The synchronous product of a network of LTSs (Sec. 3, Fig. 1) written as a
matrix over the full product space, independently of any successor
enumeration:

    T = sum_p  I (x) .. (x) L_p (x) .. (x) I   +   sum_r  (x)_q X_{r,q}

where (x) is the Kronecker product, L_p[s, t] counts process p's edges s -> t
whose label is not one of p's rule labels, and for rule r, X_{r,q} counts
q's edges s -> t carrying q's label in r (X_{r,q} = I for q outside r).
T[u, v] is then the number of global transitions from u to v, with
multiplicity.  BFS levels are the successive frontiers f_{k+1} =
(T^T f_k > 0) minus everything seen, reachability is their union, and a
deadlock is a reachable state whose row of T sums to zero.

Global index: process 0 is the most significant digit (the order np.kron and
scipy.sparse.kron use).  Only for tiny networks (product space up to ~10^6).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def _counts(n_states, edges, keep):
    m = sp.lil_matrix((n_states, n_states), dtype=np.int64)
    for (s, a, t) in edges:
        if keep(a):
            m[s, t] += 1
    return m.tocsr()


def transition_matrix(net) -> sp.csr_matrix:
    n = net.n_procs
    sizes = [p.n_states for p in net.procs]
    rule_labels = [set() for _ in range(n)]
    for rule in net.rules:
        for (p, a) in rule.parts:
            rule_labels[p].add(a)
    eye = [sp.identity(m, dtype=np.int64, format="csr") for m in sizes]
    total = None

    def kron_all(factors):
        out = factors[0]
        for f in factors[1:]:
            out = sp.kron(out, f, format="csr")
        return out

    for p in range(n):
        lp = _counts(sizes[p], net.procs[p].edges, lambda a, p=p: a not in rule_labels[p])
        term = kron_all([lp if q == p else eye[q] for q in range(n)])
        total = term if total is None else total + term
    for rule in net.rules:
        lab = dict(rule.parts)
        factors = []
        for q in range(n):
            if q in lab:
                factors.append(_counts(sizes[q], net.procs[q].edges, lambda a, want=lab[q]: a == want))
            else:
                factors.append(eye[q])
        total = total + kron_all(factors)
    return total.tocsr()


def index_of(net, local_states) -> int:
    idx = 0
    for p, s in enumerate(local_states):
        idx = idx * net.procs[p].n_states + int(s)
    return idx


def states_of(net, indices: np.ndarray) -> np.ndarray:
    """Decode global indices into an (k, n_procs) array of local states."""
    idx = np.asarray(indices, dtype=np.int64).copy()
    out = np.zeros((idx.size, net.n_procs), dtype=np.uint32)
    for p in range(net.n_procs - 1, -1, -1):
        m = net.procs[p].n_states
        out[:, p] = idx % m
        idx //= m
    return out


def explore(net):
    """Reachable set, BFS level sizes, transition count and deadlock set by matrix steps."""
    t = transition_matrix(net)
    size = t.shape[0]
    tt = t.transpose().tocsr()
    seen = np.zeros(size, dtype=bool)
    init = index_of(net, [p.initial for p in net.procs])
    frontier = np.zeros(size, dtype=bool)
    frontier[init] = True
    seen[init] = True
    levels = []
    while frontier.any():
        levels.append(int(frontier.sum()))
        reach = (tt @ frontier.astype(np.int64)) > 0
        frontier = reach & ~seen
        seen |= frontier
    out_deg = np.asarray(t.sum(axis=1)).ravel()
    reachable = np.flatnonzero(seen)
    dead = reachable[out_deg[reachable] == 0]
    return dict(reachable=reachable, levels=levels,
                transitions=int(out_deg[reachable].sum()), deadlocks=dead)
