"""Thin ctypes binding of the gx C ABI (include/gx.h).

Every function marshals arguments and calls the entry point of the same name;
all exploration work runs in the CUDA library.  PyTorch only provides device
memory (workspaces, key and table buffers) and the current CUDA stream.  If
libgx.so is missing, import of this module still succeeds but every call
raises: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from . import build as _build

P = ctypes.POINTER
u32, u64, i64 = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int64

GX_OK, GX_ERR_INVALID, GX_ERR_OOM, GX_ERR_TABLE_FULL = 0, 1, 2, 3
GX_ERR_FRONTIER_OVERFLOW, GX_ERR_SPIN_LIMIT, GX_ERR_CUDA, GX_ERR_STATE = 4, 5, 6, 7
GX_DL_BFS_FIRST, GX_DL_BFS_ALL, GX_DL_GUIDED = 0, 1, 2
STATUS_NAMES = {0: "GX_OK", 1: "GX_ERR_INVALID", 2: "GX_ERR_OOM", 3: "GX_ERR_TABLE_FULL",
                4: "GX_ERR_FRONTIER_OVERFLOW", 5: "GX_ERR_SPIN_LIMIT", 6: "GX_ERR_CUDA",
                7: "GX_ERR_STATE"}


class GxError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status
        self.message = message


class gx_lts(ctypes.Structure):
    _fields_ = [("n_states", u32), ("n_edges", u32), ("initial", u32),
                ("src", P(u32)), ("label", P(u32)), ("dst", P(u32))]


class gx_rule(ctypes.Structure):
    _fields_ = [("n_parts", u32), ("proc", P(u32)), ("label", P(u32)), ("result_label", u32)]


class gx_net_desc(ctypes.Structure):
    _fields_ = [("n_procs", u32), ("n_labels", u32), ("procs", P(gx_lts)),
                ("n_rules", u32), ("rules", P(gx_rule))]


class gx_explore_opts(ctypes.Structure):
    _fields_ = [("bucket_words", u32), ("group_lanes", u32), ("hash_rounds", u32),
                ("stop_at_first_deadlock", u32), ("max_levels", u32), ("deadlock_cap", u32),
                ("ctas_per_sm", u32), ("guided_batch", u32), ("table_bytes", u64),
                ("frontier_states", u64), ("successor_buffer", u64), ("slice_log2", u32),
                ("partition_min_states", u32), ("guided_bins", u32), ("warp_cache_log2", u32),
                ("guided_scale", ctypes.c_float), ("watch", u32), ("watch_proc", u32),
                ("watch_state", u32), ("stop_at_first_violation", u32), ("violation_cap", u32),
                ("host_loop", u32), ("region_passes", u32), ("global_cache_log2", u32),
                ("guided_fused", u32)]


MLP_IN, MLP_HIDDEN = 16, 128
MLP_PARAMS = MLP_HIDDEN * MLP_IN + MLP_HIDDEN + MLP_HIDDEN * MLP_HIDDEN + MLP_HIDDEN + MLP_HIDDEN + 1


MLP_GRAD_CTAS = 256  # GX_MLP_GRAD_CTAS
BATCH_WIDE_OFF = 0xFFFFFFFF  # GX_BATCH_WIDE_OFF


def mlp_state_bytes(batch: int) -> int:
    """GX_MLP_STATE_BYTES(batch)."""
    return 4 * ((3 + MLP_GRAD_CTAS) * MLP_PARAMS + MLP_GRAD_CTAS + 2) + 8 * batch


class gx_stats_t(ctypes.Structure):
    _fields_ = [("states", u64), ("explored", u64), ("transitions", u64), ("n_levels", u64),
                ("deadlock_count", u64), ("deadlock_sum", u64), ("deadlock_xor", u64),
                ("first_deadlock_level", i64), ("table_slots", u64),
                ("vector_words", u32), ("slot_words", u32), ("bucket_words", u32),
                ("group_lanes", u32), ("hash_rounds", u32), ("complete", u32), ("status", u32),
                ("region_passes", u32), ("fill", ctypes.c_double), ("gpu_ms", ctypes.c_double),
                ("expand_ms", ctypes.c_double), ("expand_launches", u64), ("probes", u64),
                ("h2d_bytes", u64), ("d2h_bytes", u64), ("partitioned_levels", u64),
                ("violation_count", u64), ("violation_sum", u64), ("violation_xor", u64),
                ("first_violation_level", ctypes.c_int64), ("kernel_launches", u64),
                ("device_levels", u64), ("global_cache_entries", u64)]


class gx_batch_opts(ctypes.Structure):
    _fields_ = [("bucket_words", u32), ("group_lanes", u32), ("hash_rounds", u32),
                ("chunk_states", u32), ("table_slots", u64), ("expected_states", P(u64)),
                ("levels_cap", u32), ("wide_factor", u32)]


_lib = None


def lib_path() -> str:
    return _build.LIB


def lib(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libgx.so (building it first if asked and the toolkit is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise GxError(GX_ERR_INVALID, f"CUDA library {path} is not built; run "
                      "python -m paper_1801_05857_gb300.build")
    L = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    sig = {
        "gx_load_network": ([P(gx_net_desc), P(vp)], ctypes.c_int),
        "gx_free": ([vp], None),
        "gx_load_exp": ([ctypes.c_char_p, u32, P(ctypes.c_char_p), P(ctypes.c_char_p), P(vp)], ctypes.c_int),
        "gx_label_name": ([vp, u32, ctypes.c_char_p, u32, P(u32)], ctypes.c_int),
        "gx_network_counts": ([vp, P(u32), P(u32), P(u32), P(u64)], ctypes.c_int),
        "gx_last_error": ([], ctypes.c_char_p),
        "gx_layout": ([vp, P(u32), P(u32), P(u32), P(u32)], ctypes.c_int),
        "gx_default_opts": ([P(gx_explore_opts)], ctypes.c_int),
        "gx_workspace_bytes": ([vp, P(gx_explore_opts), P(u64)], ctypes.c_int),
        "gx_explore": ([vp, P(gx_explore_opts), vp, u64, vp], ctypes.c_int),
        "gx_find_deadlocks": ([vp, P(gx_explore_opts), u32, vp, u64, vp, P(u32), u32, P(u64)],
                              ctypes.c_int),
        "gx_stats": ([vp, P(gx_stats_t)], ctypes.c_int),
        "gx_levels": ([vp, P(u64), u32, P(u32)], ctypes.c_int),
        "gx_deadlocks": ([vp, P(u32), u32, P(u32)], ctypes.c_int),
        "gx_violations": ([vp, P(u32), u32, P(u32)], ctypes.c_int),
        "gx_level_profile": ([vp, P(ctypes.c_double), P(u64), P(u64), u32, P(u32)], ctypes.c_int),
        "gx_set_digest": ([vp, vp, u64, vp, P(u64), P(u64), P(u64)], ctypes.c_int),
        "gx_find_or_put": ([vp, u64, u32, u32, u32, u32, vp, u64, vp, vp, vp], ctypes.c_int),
        "gx_cuckoo_find_or_put": ([vp, u64, u32, u32, u32, vp, vp, u64, vp, vp, vp], ctypes.c_int),
        "gx_wait_selftest": ([u32, vp], ctypes.c_int),
        "gx_probe_random": ([u32, vp, u64, u64, u32, u64, vp, vp], ctypes.c_int),
        "gx_probe_gather": ([vp, u64, u64, u32, u32, u32, u32, u32, u64, vp, vp, P(u32)], ctypes.c_int),
        "gx_explore_noalloc": ([vp, P(gx_explore_opts), vp, P(gx_stats_t), P(u64), u32, P(u32)],
                               ctypes.c_int),
        "gx_training_set": ([vp, vp, u64, vp, vp, u32, vp, vp, u64, P(u64)], ctypes.c_int),
        "gx_mlp_init": ([vp, u64, vp], ctypes.c_int),
        "gx_mlp_forward": ([vp, vp, u64, vp, vp], ctypes.c_int),
        "gx_mlp_grad": ([vp, vp, vp, u64, vp, vp, vp], ctypes.c_int),
        "gx_mlp_train": ([vp, vp, vp, vp, u64, u32, u32, ctypes.c_float, u64, vp, vp], ctypes.c_int),
        "gx_guided_set_weights": ([vp, vp], ctypes.c_int),
        "gx_guided_workspace_bytes": ([vp, P(gx_explore_opts), P(u64)], ctypes.c_int),
        "gx_guided_trace": ([vp, P(u32), u32, P(u32)], ctypes.c_int),
        "gx_batch_create": ([P(vp), u32, P(vp)], ctypes.c_int),
        "gx_batch_free": ([vp], None),
        "gx_batch_workspace_bytes": ([vp, P(gx_batch_opts), P(u64)], ctypes.c_int),
        "gx_batch_explore": ([vp, P(gx_batch_opts), vp, u64, vp], ctypes.c_int),
        "gx_batch_stats": ([vp, u32, P(gx_stats_t)], ctypes.c_int),
        "gx_batch_levels": ([vp, u32, P(u64), u32, P(u32)], ctypes.c_int),
        "gx_batch_autotune": ([vp, P(gx_batch_opts), vp, u64, vp, P(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    _lib = L
    return L


def header_symbols() -> list:
    """Entry points declared in include/gx.h."""
    hdr = os.path.join(_build.INCLUDE, "gx.h")
    txt = open(hdr).read()
    return sorted(set(re.findall(r"^\s*(?:gx_status|void|const char\*)\s+(gx_\w+)\s*\(", txt, re.M)))


def _check(st: int):
    if st != GX_OK:
        raise GxError(st, lib().gx_last_error().decode())


def _ptr(t) -> int | None:
    """Device pointer of a torch tensor (or None)."""
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# --------------------------------------------------------------------------------------------
# networks
# --------------------------------------------------------------------------------------------

class Net:
    """Owner of a gx_net handle (gx_free on deletion)."""

    def __init__(self, handle: int, n_procs: int):
        self.handle = handle
        self.n_procs = n_procs

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.gx_free(self.handle)
            self.handle = None


def load_network(net) -> Net:
    """gx_load_network from an inputs.Network (or its flat() dict)."""
    f = net.flat() if hasattr(net, "flat") else net
    n = int(f["n_procs"])
    edges = np.ascontiguousarray(f["edges"], dtype=np.uint32).reshape(-1, 3)
    keep = []
    procs = (gx_lts * n)()
    for p in range(n):
        e0, e1 = int(f["edge_off"][p]), int(f["edge_off"][p + 1])
        cols = [np.ascontiguousarray(edges[e0:e1, k]) for k in range(3)]
        keep.extend(cols)
        procs[p].n_states = int(f["n_states"][p])
        procs[p].n_edges = e1 - e0
        procs[p].initial = int(f["initial"][p])
        procs[p].src, procs[p].label, procs[p].dst = [c.ctypes.data_as(P(u32)) for c in cols]
    n_rules = len(f["rule_off"]) - 1
    rules = (gx_rule * max(n_rules, 1))()
    parts = np.ascontiguousarray(f["rule_parts"], dtype=np.uint32).reshape(-1, 2)
    for r in range(n_rules):
        j0, j1 = int(f["rule_off"][r]), int(f["rule_off"][r + 1])
        pc = np.ascontiguousarray(parts[j0:j1, 0])
        lc = np.ascontiguousarray(parts[j0:j1, 1])
        keep.extend([pc, lc])
        rules[r].n_parts = j1 - j0
        rules[r].proc = pc.ctypes.data_as(P(u32))
        rules[r].label = lc.ctypes.data_as(P(u32))
        rules[r].result_label = int(f["rule_result"][r]) if len(f["rule_result"]) else 0
    desc = gx_net_desc(n, int(f["n_labels"]), procs, n_rules, rules)
    h = ctypes.c_void_p()
    _check(lib().gx_load_network(ctypes.byref(desc), ctypes.byref(h)))
    return Net(h.value, n)


def load_exp(exp_text: str, files: dict) -> Net:
    """gx_load_exp: an EXP.OPEN composition and the .aut texts it names
    (files: name as written in the composition -> contents)."""
    names = list(files)
    n = len(names)
    cn = (ctypes.c_char_p * max(n, 1))(*[x.encode() for x in names])
    ct = (ctypes.c_char_p * max(n, 1))(*[files[x].encode() for x in names])
    h = ctypes.c_void_p()
    _check(lib().gx_load_exp(exp_text.encode(), n, cn, ct, ctypes.byref(h)))
    np_ = u32()
    _check(lib().gx_network_counts(h.value, ctypes.byref(np_), None, None, None))
    return Net(h.value, int(np_.value))


def load_exp_file(path: str) -> Net:
    """A composition file and the .aut files it names, read relative to its directory
    (every quoted name in the composition that is an existing file is passed on)."""
    import os
    import re
    with open(path) as f:
        text = f.read()
    base = os.path.dirname(os.path.abspath(path))
    files = {}
    for name in re.findall(r'"([^"\n]+)"', text):
        full = os.path.join(base, name)
        if name not in files and os.path.isfile(full):
            with open(full) as g:
                files[name] = g.read()
    return load_exp(text, files)


def label_name(net: Net, label: int) -> str:
    n = u32()
    _check(lib().gx_label_name(net.handle, label, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(int(n.value) + 1)
    _check(lib().gx_label_name(net.handle, label, buf, len(buf), ctypes.byref(n)))
    return buf.value.decode()


def network_counts(net: Net) -> dict:
    a, b, c, d = u32(), u32(), u32(), u64()
    _check(lib().gx_network_counts(net.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c), ctypes.byref(d)))
    return dict(n_procs=int(a.value), n_labels=int(b.value), n_rules=int(c.value), n_edges=int(d.value))


def layout(net: Net) -> dict:
    w = u32()
    n = net.n_procs
    fw, fo, fb = (np.zeros(n, dtype=np.uint32) for _ in range(3))
    _check(lib().gx_layout(net.handle, ctypes.byref(w), fw.ctypes.data_as(P(u32)),
                           fo.ctypes.data_as(P(u32)), fb.ctypes.data_as(P(u32))))
    return dict(vector_words=int(w.value), field_word=fw, field_offset=fo, field_bits=fb)


def default_opts(**kw) -> gx_explore_opts:
    o = gx_explore_opts()
    _check(lib().gx_default_opts(ctypes.byref(o)))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, float(v) if k == "guided_scale" else int(v))
    return o


def workspace_bytes(net: Net, opts: gx_explore_opts | None = None) -> int:
    n = u64()
    _check(lib().gx_workspace_bytes(net.handle, ctypes.byref(opts) if opts else None, ctypes.byref(n)))
    return int(n.value)


def alloc_workspace(net: Net, opts: gx_explore_opts | None = None, device="cuda"):
    """A torch uint8 device buffer of gx_workspace_bytes() bytes."""
    import torch
    return torch.empty(workspace_bytes(net, opts), dtype=torch.uint8, device=device)


def explore(net: Net, opts: gx_explore_opts | None = None, workspace=None, stream=None) -> int:
    """gx_explore; returns the status (GX_OK) or raises GxError."""
    nbytes = workspace.numel() if workspace is not None else 0
    _check(lib().gx_explore(net.handle, ctypes.byref(opts) if opts else None, _ptr(workspace),
                            nbytes, _stream(stream)))
    return GX_OK


def find_deadlocks(net: Net, mode: int, opts: gx_explore_opts | None = None, workspace=None,
                   stream=None, cap: int = 1024):
    """gx_find_deadlocks; returns (n_found, (k, n_procs) array of reported states)."""
    out = np.zeros((max(cap, 1), net.n_procs), dtype=np.uint32)
    nf = u64()
    nbytes = workspace.numel() if workspace is not None else 0
    _check(lib().gx_find_deadlocks(net.handle, ctypes.byref(opts) if opts else None, mode,
                                   _ptr(workspace), nbytes, _stream(stream),
                                   out.ctypes.data_as(P(u32)), cap, ctypes.byref(nf)))
    k = min(int(nf.value), cap)
    return int(nf.value), out[:k].copy()


def stats(net: Net) -> dict:
    s = gx_stats_t()
    _check(lib().gx_stats(net.handle, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in gx_stats_t._fields_ }


def levels(net: Net) -> list:
    n = u32()
    _check(lib().gx_levels(net.handle, None, 0, ctypes.byref(n)))
    out = np.zeros(max(int(n.value), 1), dtype=np.uint64)
    _check(lib().gx_levels(net.handle, out.ctypes.data_as(P(u64)), int(n.value), ctypes.byref(n)))
    return [int(x) for x in out[:int(n.value)]]


def level_profile(net: Net) -> dict:
    """gx_level_profile: per expanded level, device ms, buckets read and successors."""
    n = u32()
    _check(lib().gx_level_profile(net.handle, None, None, None, 0, ctypes.byref(n)))
    k = int(n.value)
    ms = np.zeros(max(k, 1), dtype=np.float64)
    pr = np.zeros(max(k, 1), dtype=np.uint64)
    tr = np.zeros(max(k, 1), dtype=np.uint64)
    _check(lib().gx_level_profile(net.handle, ms.ctypes.data_as(P(ctypes.c_double)), pr.ctypes.data_as(P(u64)),
                                  tr.ctypes.data_as(P(u64)), k, ctypes.byref(n)))
    return dict(ms=ms[:k].tolist(), probes=[int(x) for x in pr[:k]], transitions=[int(x) for x in tr[:k]])


def deadlocks(net: Net, cap: int = 1 << 20) -> np.ndarray:
    out = np.zeros((cap, net.n_procs), dtype=np.uint32)
    n = u32()
    _check(lib().gx_deadlocks(net.handle, out.ctypes.data_as(P(u32)), cap, ctypes.byref(n)))
    return out[:int(n.value)].copy()


def violations(net: Net, cap: int = 1 << 20) -> np.ndarray:
    """Violating states of the last search with opts.watch (n_procs local states each)."""
    out = np.zeros((cap, net.n_procs), dtype=np.uint32)
    n = u32()
    _check(lib().gx_violations(net.handle, out.ctypes.data_as(P(u32)), cap, ctypes.byref(n)))
    return out[:int(n.value)].copy()


def set_digest(net: Net, workspace, stream=None):
    c, s, x = u64(), u64(), u64()
    _check(lib().gx_set_digest(net.handle, _ptr(workspace), workspace.numel(), _stream(stream),
                               ctypes.byref(c), ctypes.byref(s), ctypes.byref(x)))
    return int(c.value), int(s.value), int(x.value)


def explore_noalloc(net: Net, opts: gx_explore_opts | None = None, stream=None,
                    levels_cap: int = 1 << 16):
    """gx_explore_noalloc: the search on the library's static scratch array (for
    callers that cannot allocate device memory).  Returns (stats dict, level sizes)."""
    s = gx_stats_t()
    lv = np.zeros(max(levels_cap, 1), dtype=np.uint64)
    n = u32()
    _check(lib().gx_explore_noalloc(net.handle, ctypes.byref(opts) if opts else None,
                                    _stream(stream), ctypes.byref(s), lv.ctypes.data_as(P(u64)),
                                    levels_cap, ctypes.byref(n)))
    stats_d = {name: getattr(s, name) for name, _ in gx_stats_t._fields_ }
    return stats_d, [int(x) for x in lv[:min(int(n.value), levels_cap)]]


# --------------------------------------------------------------------------------------------
# learned guidance
# --------------------------------------------------------------------------------------------

def training_set(net: Net, workspace, max_dist: int, stream=None):
    """gx_training_set after a gx_explore on net: (hist uint8 (n, 16), label float32 (n,)) tensors."""
    import torch
    s = stats(net)
    dist = torch.empty(s["table_slots"], dtype=torch.int32, device=workspace.device)
    cap = s["states"]
    hist = torch.empty((max(cap, 1), 16), dtype=torch.uint8, device=workspace.device)
    label = torch.empty(max(cap, 1), dtype=torch.float32, device=workspace.device)
    n = u64()
    _check(lib().gx_training_set(net.handle, _ptr(workspace), workspace.numel(), _stream(stream), _ptr(dist),
                                 max_dist, _ptr(hist), _ptr(label), cap, ctypes.byref(n)))
    k = min(int(n.value), cap)
    return hist[:k], label[:k]


def mlp_init(params, seed: int, stream=None) -> None:
    _check(lib().gx_mlp_init(_ptr(params), seed, _stream(stream)))


def mlp_forward(params, hist, stream=None):
    import torch
    out = torch.empty(hist.shape[0], dtype=torch.float32, device=hist.device)
    _check(lib().gx_mlp_forward(_ptr(params), _ptr(hist), hist.shape[0], _ptr(out), _stream(stream)))
    return out


def mlp_grad(params, hist, label, stream=None):
    import torch
    g = torch.empty(MLP_PARAMS, dtype=torch.float32, device=hist.device)
    loss = torch.empty(1, dtype=torch.float32, device=hist.device)
    _check(lib().gx_mlp_grad(_ptr(params), _ptr(hist), _ptr(label), hist.shape[0], _ptr(g), _ptr(loss),
                             _stream(stream)))
    return g, loss


def mlp_train(params, hist, label, batch: int, steps: int, lr: float, seed: int, stream=None):
    """gx_mlp_train; returns the per-step mini-batch losses (torch tensor)."""
    import torch
    state = torch.empty(mlp_state_bytes(batch), dtype=torch.uint8, device=hist.device)
    loss = torch.empty(steps, dtype=torch.float32, device=hist.device)
    _check(lib().gx_mlp_train(_ptr(params), _ptr(state), _ptr(hist), _ptr(label), hist.shape[0], batch, steps,
                              lr, seed, _ptr(loss), _stream(stream)))
    return loss


def guided_set_weights(net: Net, params) -> None:
    _check(lib().gx_guided_set_weights(net.handle, _ptr(params)))
    net._guided_params = params  # keep the device buffer alive with the handle


def guided_workspace_bytes(net: Net, opts: gx_explore_opts | None = None) -> int:
    n = u64()
    _check(lib().gx_guided_workspace_bytes(net.handle, ctypes.byref(opts) if opts else None, ctypes.byref(n)))
    return int(n.value)


def guided_alloc_workspace(net: Net, opts: gx_explore_opts | None = None, device="cuda"):
    import torch
    return torch.empty(guided_workspace_bytes(net, opts), dtype=torch.uint8, device=device)


def guided_trace(net: Net) -> np.ndarray:
    n = u32()
    _check(lib().gx_guided_trace(net.handle, None, 0, ctypes.byref(n)))
    out = np.zeros((max(int(n.value), 1), net.n_procs), dtype=np.uint32)
    _check(lib().gx_guided_trace(net.handle, out.ctypes.data_as(P(u32)), int(n.value), ctypes.byref(n)))
    return out[:int(n.value)].copy()


# --------------------------------------------------------------------------------------------
# batched exploration
# --------------------------------------------------------------------------------------------

class Batch:
    """Owner of a gx_batch handle (gx_batch_free on deletion)."""

    def __init__(self, handle: int, n: int):
        self.handle = handle
        self.n = n

    def __del__(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.gx_batch_free(self.handle)
            self.handle = None


def batch_create(nets) -> Batch:
    """gx_batch_create from a list of Net handles (or inputs.Network objects)."""
    handles = [n if isinstance(n, Net) else load_network(n) for n in nets]
    arr = (ctypes.c_void_p * len(handles))(*[h.handle for h in handles])
    h = ctypes.c_void_p()
    _check(lib().gx_batch_create(arr, len(handles), ctypes.byref(h)))
    return Batch(h.value, len(handles))


def batch_opts(expected_states=None, **kw) -> gx_batch_opts:
    o = gx_batch_opts()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise TypeError(f"unknown option {k}")
        setattr(o, k, int(v))
    if expected_states is not None:
        arr = np.ascontiguousarray(expected_states, dtype=np.uint64)
        o._keep = arr
        o.expected_states = arr.ctypes.data_as(P(u64))
    return o


def batch_workspace_bytes(b: Batch, opts: gx_batch_opts | None = None) -> int:
    n = u64()
    _check(lib().gx_batch_workspace_bytes(b.handle, ctypes.byref(opts) if opts else None, ctypes.byref(n)))
    return int(n.value)


def batch_alloc_workspace(b: Batch, opts: gx_batch_opts | None = None, device="cuda"):
    import torch
    return torch.empty(batch_workspace_bytes(b, opts), dtype=torch.uint8, device=device)


def batch_explore(b: Batch, opts: gx_batch_opts | None, workspace, stream=None) -> None:
    _check(lib().gx_batch_explore(b.handle, ctypes.byref(opts) if opts else None, _ptr(workspace),
                                  workspace.numel(), _stream(stream)))


def batch_stats(b: Batch, i: int) -> dict:
    s = gx_stats_t()
    _check(lib().gx_batch_stats(b.handle, i, ctypes.byref(s)))
    return {name: getattr(s, name) for name, _ in gx_stats_t._fields_ }


def batch_levels(b: Batch, i: int) -> list:
    n = u32()
    _check(lib().gx_batch_levels(b.handle, i, None, 0, ctypes.byref(n)))
    out = np.zeros(max(int(n.value), 1), dtype=np.uint64)
    _check(lib().gx_batch_levels(b.handle, i, out.ctypes.data_as(P(u64)), int(n.value), ctypes.byref(n)))
    return [int(x) for x in out[:int(n.value)]]


def batch_autotune(b: Batch, opts: gx_batch_opts, workspace, stream=None) -> float:
    """gx_batch_autotune: updates opts in place, returns the best batch time (ms)."""
    ms = ctypes.c_double()
    _check(lib().gx_batch_autotune(b.handle, ctypes.byref(opts), _ptr(workspace), workspace.numel(),
                                   _stream(stream), ctypes.byref(ms)))
    return float(ms.value)


# --------------------------------------------------------------------------------------------
# isolated table experiment and probes
# --------------------------------------------------------------------------------------------

def find_or_put(keys, key_words: int, table, counters, result=None, bucket_words: int = 8,
                group_lanes: int = 0, hash_rounds: int = 0, stream=None) -> None:
    """gx_find_or_put on torch device tensors (keys: uint32/int32 with n*key_words
    elements; table: 32-bit, zeroed by the caller; counters: 3 x 64-bit)."""
    n = keys.numel() // key_words
    _check(lib().gx_find_or_put(_ptr(keys), n, key_words, bucket_words, group_lanes, hash_rounds,
                                _ptr(table), table.numel(), _ptr(result), _ptr(counters),
                                _stream(stream)))


def cuckoo_find_or_put(keys, key_words: int, table, counters, result=None, n_hash: int = 0,
                       max_chain: int = 0, muls=None, stream=None) -> None:
    """gx_cuckoo_find_or_put on torch device tensors (keys: 32-bit with n*key_words
    elements; table: 32-bit with slots*key_words elements, zeroed by the caller;
    counters: 4 x 64-bit); muls: host sequence of odd multipliers, or None."""
    n = keys.numel() // key_words
    m = None
    if muls is not None:
        m = np.ascontiguousarray(np.asarray(muls, dtype=np.uint64))
    _check(lib().gx_cuckoo_find_or_put(_ptr(keys), n, key_words, n_hash, max_chain,
                                       None if m is None else m.ctypes.data, _ptr(table),
                                       table.numel() // key_words, _ptr(result), _ptr(counters),
                                       _stream(stream)))


def wait_selftest(spin_limit: int, stream=None) -> None:
    """gx_wait_selftest: raises GxError(GX_ERR_SPIN_LIMIT) when the bounded wait gave up."""
    _check(lib().gx_wait_selftest(spin_limit, _stream(stream)))


def probe_random(kind: int, buffer, n: int, nbytes: int, seed: int, sink, stream=None) -> None:
    _check(lib().gx_probe_random(kind, _ptr(buffer), buffer.numel(), n, nbytes, seed, _ptr(sink),
                                 _stream(stream)))


def probe_gather(buffer, n: int, unit_bytes: int, load_bytes: int, in_flight: int, ctas_per_sm: int,
                 group_log2: int, seed: int, sink, stream=None) -> int:
    """Random gathers over `buffer` (an int32 device tensor, or a slice of one) with the given
    launch shape and locality; returns the CTAs per SM launched."""
    used = ctypes.c_uint32(0)
    _check(lib().gx_probe_gather(_ptr(buffer), buffer.numel(), n, unit_bytes, load_bytes, in_flight,
                                 ctas_per_sm, group_log2, seed, _ptr(sink), _stream(stream),
                                 ctypes.byref(used)))
    return used.value
