"""Write the stored oracle results used by the GPU parity tests and the bench.

    python tests/golden/make_golden.py mid        # ~5 min, ~6 GB host RAM
    python tests/golden/make_golden.py large3     # irregular, 4-word, 3-party; see LARGE3

Every value written here comes from the CPU oracle (oracle/) run on a network
drawn by paper_1801_05857_gb300.inputs; nothing comes from the CUDA path.
"""
import json
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1801_05857_gb300 import inputs  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# Mid network: inputs.WORKLOADS["mid"] (10 x 16 states, 2-word vectors, 4 two-party rules)
MID = inputs.WORKLOADS["mid"]

# Irregular memory-scaled-shape network: 16 processes x 16 local states (3 words, in 4-word
# slots), 3 of 30 labels as 3-party rules (10 %), out-degree 1-2, local edges inside blocks
# of 5 states and rule edges weighted 6:1 so that the rules fire: 1.08e8 states, 3.5 times
# as many as the same network without its rule edges (the reachable set is no product of
# the blocks).  ~12 GB of host RAM.
LARGE3 = dict(seed=6, n_procs=16, n_states=16, deg_lo=1, deg_hi=2, n_labels=30, n_sync=3, parties=3,
              cluster=5, sync_weight=6.0, name="large3_s6_n16")


def write(name: str, gen: dict) -> None:
    net = inputs.random_network(**gen)
    r = oracle.explore(net, deadlocks_cap=1 << 12)
    assert r.complete
    out = dict(generator=gen, states=r.states, transitions=r.transitions, levels=r.levels,
               deadlock_count=r.deadlock_count, deadlock_sum=r.deadlock_sum,
               deadlock_xor=r.deadlock_xor, set_sum=r.set_sum, set_xor=r.set_xor,
               oracle_seconds=round(r.seconds, 2),
               note="written by tests/golden/make_golden.py from oracle.explore")
    with open(os.path.join(HERE, name), "w") as f:
        json.dump(out, f, indent=1)
    print(name, r.states, r.transitions, len(r.levels), round(r.seconds, 1), "s")


def write_batch(count: int = 256, lo: int = 1_000, hi: int = 1_000_000) -> None:
    """Select the batched workload: candidate seeds of inputs.batch_params in order, kept
    when the oracle finds lo..hi reachable states; store every kept network's results."""
    kept = []
    seed = 0
    while len(kept) < count:
        gen = inputs.batch_params(seed)
        r = oracle.explore(inputs.random_network(**gen), max_explored=hi + 1, deadlocks_cap=16)
        if r.complete and lo <= r.states <= hi:
            kept.append(dict(batch_seed=seed, generator=gen, states=r.states, transitions=r.transitions,
                             levels=r.levels, deadlock_count=r.deadlock_count,
                             deadlock_sum=r.deadlock_sum, deadlock_xor=r.deadlock_xor,
                             set_sum=r.set_sum, set_xor=r.set_xor))
            print(len(kept), seed, r.states, flush=True)
        seed += 1
    with open(os.path.join(HERE, "batch_networks.json"), "w") as f:
        json.dump(dict(note="written by tests/golden/make_golden.py batch from oracle.explore",
                       seeds=[k["batch_seed"] for k in kept], networks=kept), f)
    print("BATCH_SEEDS =", [k["batch_seed"] for k in kept])


if __name__ == "__main__":
    which = sys.argv[1:] or ["mid"]
    if "mid" in which:
        write("mid_network.json", MID)
    if "large3" in which:
        write("large3_network.json", LARGE3)
    if "batch" in which:
        write_batch()
