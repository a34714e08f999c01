"""CPU oracle for the exploration path -- TEST INFRASTRUCTURE ONLY.

Only tests/, the smoke check and the bench's CPU-baseline leg may import this
package.  It shares no code with the CUDA path (see bfs_oracle.cpp for what it
computes and which passages of the paper it follows):

* ``explore``      -- plain BFS over the synchronous product (C++, std::unordered_set)
* ``successors``   -- the successor multiset of one global state
* ``state_digest`` -- the order-free digest of one global state
* ``deadlock_distances`` -- backward-BFS distance of every reachable state to a deadlock
* ``product_matrix`` -- brute force: the product's transition-count matrix as a
  sum of Kronecker products, and BFS levels by matrix-vector steps (tiny networks)
* ``mlp``          -- FP64 forward and gradient of the guided search's scoring network
* ``cuckoo``       -- sequential cuckoo hashing, the table Sec. 4.1 compares with its own
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with the host C++ compiler (plain -O2, no architecture flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-shared", "-fPIC", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class OracleResult(ctypes.Structure):
    _fields_ = [(n, ctypes.c_uint64) for n in (
        "states", "explored", "transitions", "n_levels", "deadlock_count", "deadlock_sum",
        "deadlock_xor", "set_sum", "set_xor")] + [
        ("first_deadlock_level", ctypes.c_int64), ("complete", ctypes.c_uint64),
        ("seconds", ctypes.c_double), ("violation_count", ctypes.c_uint64),
        ("violation_sum", ctypes.c_uint64), ("violation_xor", ctypes.c_uint64),
        ("first_violation_level", ctypes.c_int64)]


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.POINTER
        u32p = P(ctypes.c_uint32)
        net_args = [ctypes.c_uint32, ctypes.c_uint32, u32p, u32p, u32p, u32p,
                    ctypes.c_uint32, u32p, u32p]
        lib.oracle_explore.argtypes = net_args + [
            ctypes.c_uint32, ctypes.c_uint64, P(OracleResult), P(ctypes.c_uint64),
            ctypes.c_uint32, u32p, ctypes.c_uint32,
            ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint32, u32p, ctypes.c_uint32]
        lib.oracle_explore.restype = ctypes.c_int
        lib.oracle_state_digest.argtypes = [ctypes.c_uint32, u32p]
        lib.oracle_state_digest.restype = ctypes.c_uint64
        lib.oracle_successors.argtypes = net_args + [u32p, u32p, ctypes.c_uint64]
        lib.oracle_successors.restype = ctypes.c_int64
        lib.oracle_deadlock_distances.argtypes = net_args + [u32p, u32p, ctypes.c_uint64]
        lib.oracle_deadlock_distances.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _u32(a):
    a = np.ascontiguousarray(a, dtype=np.uint32)
    if a.size == 0:
        a = np.zeros(1, dtype=np.uint32)
    return a


def _net_args(net):
    f = net.flat() if hasattr(net, "flat") else net
    keep = [_u32(f["n_states"]), _u32(f["initial"]), _u32(f["edge_off"]), _u32(f["edges"]),
            _u32(f["rule_off"]), _u32(f["rule_parts"])]
    ptr = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))
    args = [f["n_procs"], f["n_labels"], ptr(keep[0]), ptr(keep[1]), ptr(keep[2]), ptr(keep[3]),
            len(f["rule_off"]) - 1, ptr(keep[4]), ptr(keep[5])]
    return f, args, keep


@dataclass
class Exploration:
    states: int
    explored: int
    transitions: int
    levels: list
    deadlock_count: int
    deadlock_sum: int
    deadlock_xor: int
    set_sum: int
    set_xor: int
    first_deadlock_level: int
    complete: bool
    seconds: float
    deadlocks: np.ndarray  # (min(count, cap), n_procs) local states
    violation_count: int = 0
    violation_sum: int = 0
    violation_xor: int = 0
    first_violation_level: int = -1
    violations: np.ndarray = None  # (min(count, cap), n_procs) local states


def explore(net, stop_at_first_deadlock: bool = False, max_explored: int = 0,
            levels_cap: int = 1 << 16, deadlocks_cap: int = 4096, watch=None,
            stop_at_first_violation: bool = False, violations_cap: int = 4096) -> Exploration:
    """Breadth-first exploration; watch = (process, local state) turns on the
    safety check (that local state is the error state of the property automaton)."""
    lib = _load()
    f, args, keep = _net_args(net)
    res = OracleResult()
    levels = np.zeros(levels_cap, dtype=np.uint64)
    dl = np.zeros((deadlocks_cap, f["n_procs"]), dtype=np.uint32)
    vi = np.zeros((violations_cap, f["n_procs"]), dtype=np.uint32)
    wp, ws = (0xFFFFFFFF, 0) if watch is None else watch
    u32p = ctypes.POINTER(ctypes.c_uint32)
    rc = lib.oracle_explore(*args, int(bool(stop_at_first_deadlock)), int(max_explored),
                            ctypes.byref(res), levels.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                            levels_cap, dl.ctypes.data_as(u32p), deadlocks_cap,
                            int(wp), int(ws), int(bool(stop_at_first_violation)), vi.ctypes.data_as(u32p),
                            violations_cap)
    if rc != 0:
        raise ValueError("oracle: invalid network")
    n_lv = int(res.n_levels)
    return Exploration(int(res.states), int(res.explored), int(res.transitions),
                       [int(x) for x in levels[:min(n_lv, levels_cap)]], int(res.deadlock_count),
                       int(res.deadlock_sum), int(res.deadlock_xor), int(res.set_sum),
                       int(res.set_xor), int(res.first_deadlock_level), bool(res.complete),
                       float(res.seconds), dl[:min(int(res.deadlock_count), deadlocks_cap)].copy(),
                       int(res.violation_count), int(res.violation_sum), int(res.violation_xor),
                       int(res.first_violation_level), vi[:min(int(res.violation_count), violations_cap)].copy())


def state_digest(local_states) -> int:
    lib = _load()
    a = _u32(local_states)
    return int(lib.oracle_state_digest(len(local_states), a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))))


def successors(net, state, cap: int = 1 << 16) -> np.ndarray:
    """Successor multiset of one global state, as an (m, n_procs) array in the oracle's order."""
    lib = _load()
    f, args, keep = _net_args(net)
    st = _u32(state)
    out = np.zeros((cap, f["n_procs"]), dtype=np.uint32)
    m = lib.oracle_successors(*args, st.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                              out.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cap)
    if m < 0:
        raise ValueError("oracle: invalid network or state")
    if m > cap:
        raise ValueError("oracle: successor buffer too small")
    return out[:m].copy()


def deadlock_distances(net, cap: int = 1 << 22):
    """(states, dist): every reachable state (BFS order) and its backward distance to a deadlock."""
    lib = _load()
    f, args, keep = _net_args(net)
    states = np.zeros((cap, f["n_procs"]), dtype=np.uint32)
    dist = np.zeros(cap, dtype=np.uint32)
    m = lib.oracle_deadlock_distances(*args, states.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                                      dist.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)), cap)
    if m == -2:
        raise ValueError("oracle: reachable set larger than cap")
    if m < 0:
        raise ValueError("oracle: invalid network")
    return states[:m].copy(), dist[:m].copy()
