"""Training the scoring network of the guided deadlock search.

Each step runs in the CUDA library: every training network is explored
(gx_explore), its states are labelled with their distance to the nearest
deadlock (gx_training_set), and the network is trained on the union of the
examples with Adam (gx_mlp_train).  This module only sequences those calls and
concatenates device tensors.
"""
from __future__ import annotations

from . import gx


def collect_examples(nets, max_dist: int = 64, table_bytes: int = 1 << 26, stream=None):
    """(hist uint8 (n, 16), label float32 (n,)) device tensors over all networks."""
    import torch
    hs, ls = [], []
    for net in nets:
        h = gx.load_network(net)
        o = gx.default_opts(table_bytes=table_bytes, bucket_words=8, group_lanes=1, hash_rounds=32)
        ws = gx.alloc_workspace(h, o)
        gx.explore(h, o, ws, stream)
        hist, label = gx.training_set(h, ws, max_dist, stream)
        hs.append(hist.clone())
        ls.append(label.clone())
        del ws
    return torch.cat(hs), torch.cat(ls)


def train(hist, label, steps: int = 2000, batch: int = 1024, lr: float = 2e-3, seed: int = 1,
          stream=None):
    """A freshly initialised network trained on the examples: (params, per-step losses)."""
    import torch
    params = torch.empty(gx.MLP_PARAMS, dtype=torch.float32, device=hist.device)
    gx.mlp_init(params, seed, stream)
    losses = gx.mlp_train(params, hist, label, batch, steps, lr, seed + 1, stream)
    return params, losses
