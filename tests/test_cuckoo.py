"""Cuckoo hashing, the table Sec. 4.1 compares with its own.

CPU: the oracle (oracle/cuckoo.py) against hand-worked eviction chains, the
published first splitmix64 output, and invariants of sequential insertion.
GPU (through the C ABI): one key per call is the sequential algorithm, so the
table equals the oracle's word for word; with all keys at once the stored set
equals the input set, every key sits at one of its positions, and the counters
add up; the excess of "inserted" over distinct keys is the lost atomicity of
find-or-put that Sec. 4.1 holds against cuckoo hashing.
"""
import numpy as np
import pytest

from oracle import cuckoo
from paper_1801_05857_gb300 import gx, inputs


def _muls(seed, k):
    g = inputs.SplitMix64(seed)
    return [g.next() | 1 for _ in range(k)]


def test_splitmix64_output_published_value():
    assert cuckoo.splitmix64_output(0) == 0xE220A8397B1DCDAF


def test_hand_worked_eviction_chain():
    # 4 slots, 2 positions per key, chosen by hand
    P = {"A": (0, 1), "B": (0, 2), "C": (0, 3), "D": (1, 0)}
    keys = {k: i + 1 for i, k in enumerate("ABCD")}
    name = {v: k for k, v in keys.items()}
    pos = lambda x, i: P[name[x]][i]
    seq = [keys[c] for c in "ABCAD"]
    # A -> 0; B evicts A to 1; C evicts B to 2; A found; D evicts A from 1, A (at its
    # position 1) goes back to its position 0 and evicts C, which moves on to 3
    t, res, cnt = cuckoo.insert_sequential(seq, 4, 2, 8, pos)
    assert [name.get(x, "-") for x in t] == ["A", "D", "B", "C"]
    assert res == [1, 1, 1, 0, 1] and cnt == (4, 1, 0, 1 + 2 + 2 + 3)
    # at most 2 writes: D's chain ends carrying C, which is dropped
    t, res, cnt = cuckoo.insert_sequential(seq, 4, 2, 2, pos)
    assert [name.get(x, "-") for x in t] == ["A", "D", "B", "-"]
    assert res == [1, 1, 1, 0, 2] and cnt == (3, 1, 1, 1 + 2 + 2 + 2)


def test_sequential_insertion_invariants():
    log2 = 10
    muls = _muls(5, 4)
    pos = cuckoo.multiply_shift_positions(muls, log2)
    keys = [cuckoo.slot_value([int(x)]) for x in inputs.key_sequence(700 * 2, 2, seed=3)[:, 0]]
    t, res, cnt = cuckoo.insert_sequential(keys, 1 << log2, 4, 500, pos)
    assert cnt[2] == 0 and cnt[0] == len(set(keys)) and cnt[1] == len(keys) - len(set(keys))
    stored = [x for x in t if x]
    assert sorted(stored) == sorted(set(keys))
    for s, x in enumerate(t):
        if x:
            assert s in {pos(x, i) for i in range(4)}
    arr = cuckoo.multiply_shift_positions_array(stored[:50], muls, log2)
    assert [[int(p) for p in row] for row in arr] == [[pos(x, i) for i in range(4)] for x in stored[:50]]


def _np_table(table, key_words):
    a = table.cpu().numpy().view(np.uint32).astype(np.uint64)
    if key_words == 2:
        a = a.reshape(-1, 2)
        a = a[:, 0] | (a[:, 1] << np.uint64(32))
    return a


def _values(keys_np):
    v = keys_np.astype(np.uint64) | np.uint64(1 << 31)
    if keys_np.shape[1] == 2:
        return v[:, 0] | (v[:, 1] << np.uint64(32))
    return v[:, 0]


def _at_own_position(tab, muls, log2):
    idx = np.nonzero(tab)[0]
    p = cuckoo.multiply_shift_positions_array(tab[idx], muls, log2)
    return bool((p == idx[:, None].astype(np.uint64)).any(axis=1).all())


@pytest.mark.gpu
@pytest.mark.parametrize("key_words,k,n,dup,chain", [(1, 4, 400, 2, 128), (2, 3, 300, 3, 128),
                                                     (1, 2, 200, 1, 128), (1, 2, 470, 1, 2),
                                                     (2, 8, 480, 2, 64)])
def test_one_key_per_call_equals_the_sequential_oracle(cuda, key_words, k, n, dup, chain):
    import torch
    log2 = 9
    muls = _muls(11 + k, k)
    keys_np = inputs.key_sequence(n - n % dup, dup, words=key_words, seed=k)
    keys = torch.from_numpy(keys_np.view(np.int32).reshape(-1)).cuda()
    table = torch.zeros((1 << log2) * key_words, dtype=torch.int32, device="cuda")
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    result = torch.zeros(len(keys_np), dtype=torch.uint8, device="cuda")
    for i in range(len(keys_np)):
        gx.cuckoo_find_or_put(keys[i * key_words:(i + 1) * key_words], key_words, table, counters,
                              result[i:i + 1], n_hash=k, max_chain=chain, muls=muls)
    vals = [int(x) for x in _values(keys_np)]
    t, res, cnt = cuckoo.insert_sequential(vals, 1 << log2, k, chain,
                                           cuckoo.multiply_shift_positions(muls, log2))
    assert [int(x) for x in _np_table(table, key_words)] == t
    assert result.cpu().tolist() == res
    assert tuple(counters.cpu().tolist()) == cnt
    if chain == 2:
        assert cnt[2] > 0  # the short chain did drop keys


@pytest.mark.gpu
@pytest.mark.parametrize("key_words", [1, 2])
@pytest.mark.parametrize("dup", [1, 2, 10, 100])
def test_concurrent_insertion_keeps_the_set(cuda, key_words, dup):
    import torch
    n, log2, k = 1 << 20, 21, 4
    n -= n % dup
    muls = _muls(dup, k)
    keys_np = inputs.key_sequence(n, dup, words=key_words, seed=dup)
    keys = torch.from_numpy(keys_np.view(np.int32).reshape(-1)).cuda()
    table = torch.zeros((1 << log2) * key_words, dtype=torch.int32, device="cuda")
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    result = torch.empty(n, dtype=torch.uint8, device="cuda")
    gx.cuckoo_find_or_put(keys, key_words, table, counters, result, n_hash=k, muls=muls)
    ins, fnd, fail, exch = counters.cpu().tolist()
    distinct = n // dup
    tab = _np_table(table, key_words)
    stored = tab[tab != 0]
    want = np.unique(_values(keys_np))
    assert fail == 0 and ins + fnd == n
    assert np.array_equal(np.unique(stored), want)
    assert distinct <= len(stored) <= ins and exch >= ins
    r = result.cpu().numpy()
    assert (r == 1).sum() == ins and (r == 0).sum() == fnd
    if dup == 1:  # no key is ever looked up while another thread moves it
        assert ins == n and len(stored) == n
    assert _at_own_position(tab, muls, log2)
    # a second pass finds every key and moves nothing
    before = table.clone()
    counters.zero_()
    gx.cuckoo_find_or_put(keys, key_words, table, counters, None, n_hash=k, muls=muls)
    assert counters.cpu().tolist() == [0, n, 0, 0]
    assert torch.equal(before, table)


@pytest.mark.gpu
def test_default_multipliers_and_a_full_table(cuda):
    import torch
    keys_np = inputs.key_sequence(1 << 12, 1, seed=1)
    keys = torch.from_numpy(keys_np.view(np.int32).reshape(-1)).cuda()
    table = torch.zeros(1 << 12, dtype=torch.int32, device="cuda")
    counters = torch.zeros(4, dtype=torch.int64, device="cuda")
    gx.cuckoo_find_or_put(keys[:1 << 11], 1, table, counters)
    assert counters.cpu().tolist()[:3] == [1 << 11, 0, 0]
    # 4096 keys into 4096 slots: chains run out and keys are dropped, never more
    # than the failures reported
    table.zero_()
    counters.zero_()
    gx.cuckoo_find_or_put(keys, 1, table, counters, n_hash=2, max_chain=16)
    ins, fnd, fail, _ = counters.cpu().tolist()
    tab = _np_table(table, 1)
    stored = np.unique(tab[tab != 0])
    assert fail > 0 and ins + fnd + fail == len(keys_np)
    assert len(np.setdiff1d(_values(keys_np), stored)) <= fail
    assert np.isin(stored, _values(keys_np)).all()


def test_invalid_arguments_are_rejected():
    # host-side validation (stream 0 given, so no CUDA runtime is asked): nothing reaches a device
    class Fake:
        def __init__(self, n):
            self.n = n

        def numel(self):
            return self.n

        def data_ptr(self):
            return 256

    t = Fake(1024)
    for kw, msg in ((dict(n_hash=1), "n_hash"), (dict(n_hash=9), "n_hash"), (dict(max_chain=5000), "max_chain"),
                    (dict(muls=[3, 4, 5, 7]), "odd")):
        with pytest.raises(gx.GxError) as e:
            gx.cuckoo_find_or_put(Fake(4), 1, t, Fake(4), stream=0, **kw)
        assert e.value.status == gx.GX_ERR_INVALID and msg in e.value.message
    with pytest.raises(gx.GxError) as e:
        gx.cuckoo_find_or_put(Fake(4), 4, t, Fake(4), stream=0)
    assert "key_words" in e.value.message
    with pytest.raises(gx.GxError) as e:
        gx.cuckoo_find_or_put(Fake(4), 1, Fake(1000), Fake(4), stream=0)
    assert "power of two" in e.value.message
