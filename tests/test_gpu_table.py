"""The find-or-put hash table on its own (Sec. 4.1, Sec. 5.1), through the C ABI.

Oracle: set semantics.  For a key sequence with n // d distinct keys each
repeated d times (the Sec. 5.1 input), exactly one occurrence of each
distinct key reports "inserted", all others "found", and the table ends up
holding exactly the distinct keys.
"""
import numpy as np
import pytest

from paper_1801_05857_gb300 import gx, inputs

pytestmark = pytest.mark.gpu

TAG = np.uint32(0x80000000)


def _run(keys_np, W, B, G, table_words, rounds=0):
    import torch
    keys = torch.from_numpy(keys_np.view(np.int32).reshape(-1)).cuda()
    table = torch.zeros(table_words, dtype=torch.int32, device="cuda")
    counters = torch.zeros(3, dtype=torch.int64, device="cuda")
    result = torch.zeros(len(keys_np), dtype=torch.uint8, device="cuda")
    gx.find_or_put(keys, W, table, counters, result, bucket_words=B, group_lanes=G, hash_rounds=rounds)
    torch.cuda.synchronize()
    return (table.cpu().numpy().view(np.uint32), counters.cpu().numpy(), result.cpu().numpy())


def _table_keys(table, W):
    slots = table.reshape(-1, W)
    occ = (slots & TAG).astype(bool).all(axis=1)
    return slots[occ] & ~TAG, slots[~occ]


def _configs():
    out = []
    for W in (1, 2, 4):
        for B in (4, 8, 16, 32):
            if B < W:
                continue
            G = 1
            while G <= B // W and G <= 32:
                out.append((W, B, G))
                G *= 2
    return out


@pytest.mark.parametrize("W,B,G", _configs())
def test_set_semantics(cuda, W, B, G):
    n, d = 1 << 16, 4
    keys = inputs.key_sequence(n, d, words=W, seed=11)
    table, counters, result = _run(keys, W, B, G, table_words=1 << 18, rounds=32)
    u = n // d
    assert counters.tolist() == [u, n - u, 0]
    stored, empty = _table_keys(table, W)
    assert len(stored) == u
    assert (empty == 0).all()  # no half-written slot is left behind
    assert {tuple(r) for r in stored} == {tuple(r) for r in np.unique(keys, axis=0)}
    # exactly one inserting occurrence per distinct key
    ins = keys[result == 1]
    assert len(ins) == u and len({tuple(r) for r in ins}) == u
    assert set(np.unique(result).tolist()) <= {0, 1}


@pytest.mark.parametrize("d", [1, 2, 5, 10, 21, 50, 100])
def test_duplication_sweep_counts(cuda, d):
    """Sec. 5.1: a sequence with duplication d has n / d distinct keys."""
    n = 100 * 2100
    keys = inputs.key_sequence(n, d, words=1, seed=d)
    for B, G in ((32, 32), (4, 4), (4, 1)):
        table, counters, _ = _run(keys, 1, B, G, table_words=1 << 20, rounds=16)
        assert counters.tolist() == [n // d, n - n // d, 0]


def test_second_pass_finds_everything(cuda):
    import torch
    keys_np = inputs.key_sequence(1 << 15, 1, words=2, seed=5)
    keys = torch.from_numpy(keys_np.view(np.int32).reshape(-1)).cuda()
    table = torch.zeros(1 << 18, dtype=torch.int32, device="cuda")
    c = torch.zeros(3, dtype=torch.int64, device="cuda")
    gx.find_or_put(keys, 2, table, c, bucket_words=8)
    gx.find_or_put(keys, 2, table, c, bucket_words=8)
    torch.cuda.synchronize()
    assert c.cpu().tolist() == [1 << 15, 1 << 15, 0]


def test_fig4_partial_match_then_first_free_slot(cuda):
    """Fig. 4: inserting (8, 2, 1) into a bucket whose first two slots hold other
    vectors, one of which matches it in one word: not found, stored in the third
    slot.  Three-word vectors use 4-word slots here (32-word bucket = 8 slots); both
    buckets of a 2-bucket table are prepared the same way, so wherever the vector
    hashes, the same situation arises."""
    import torch
    W, B = 4, 32
    table = np.zeros(2 * B, dtype=np.uint32)
    occupants = [(8, 5, 7, 0), (3, 2, 9, 0)]   # second word of the second one matches
    for b in range(2):
        for j, v in enumerate(occupants):
            table[b * B + j * W: b * B + (j + 1) * W] = np.array(v, dtype=np.uint32) | TAG
    t = torch.from_numpy(table.view(np.int32)).cuda()
    key = np.array([[8, 2, 1, 0]], dtype=np.uint32)
    k = torch.from_numpy(key.view(np.int32).reshape(-1)).cuda()
    c = torch.zeros(3, dtype=torch.int64, device="cuda")
    for G in (1, 2, 4, 8):
        t2 = t.clone()
        c.zero_()
        gx.find_or_put(k, W, t2, c, bucket_words=B, group_lanes=G, hash_rounds=1)
        torch.cuda.synchronize()
        out = t2.cpu().numpy().view(np.uint32).reshape(2, B // W, W)
        assert c.cpu().tolist() == [1, 0, 0]
        hit = [(b, j) for b in range(2) for j in range(B // W)
               if tuple(out[b, j]) == tuple((key[0] | TAG).tolist())]
        assert len(hit) == 1 and hit[0][1] == 2, (G, hit)
        # nothing else moved
        ref = table.reshape(2, B // W, W).copy()
        ref[hit[0][0], 2] = key[0] | TAG
        assert (out == ref).all()


def test_full_table_reports_failure(cuda):
    """Sec. 4.1: when every hash-constant set leads to a full bucket the insertion
    reports failure.  Two one-slot buckets hold at most two distinct keys."""
    keys = np.array([[1, 1, 1, 1], [2, 2, 2, 2], [3, 3, 3, 3]], dtype=np.uint32)
    table, counters, result = _run(keys, 4, 4, 1, table_words=8, rounds=8)
    assert counters.tolist()[0] <= 2 and counters.tolist()[2] >= 1
    assert counters.sum() == 3
    assert (result == 2).sum() == counters.tolist()[2]


def test_probe_kernels_run(cuda):
    import torch
    buf = torch.zeros(1 << 22, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    for nbytes in (16, 32, 64, 128):
        gx.probe_random(0, buf, 1 << 16, nbytes, 1, sink)
    for nbytes in (4, 8, 16):
        gx.probe_random(1, buf, 1 << 16, nbytes, 2, sink)
    torch.cuda.synchronize()
    assert int((buf != 0).sum().item()) > 0
