"""Sequential cuckoo hashing -- TEST INFRASTRUCTURE ONLY.

The alternative hash table Sec. 4.1 weighs against its own: cuckoo hashing
(Pagh & Rodler 2004) as Alcantara et al. run it on a GPU.  Every key has
n_hash candidate slots.  To insert a key it is put in its first slot; a key
that was there is evicted and goes to its next candidate slot, evicting in
turn, until a slot was empty.  This module runs that algorithm one key at a
time on plain Python integers, in the order the keys are given:

1. a key is present when one of its n_hash positions holds it (result 0);
2. otherwise it is written to position 0 (result 1).  Whatever sat there is
   carried on: a key y taken from slot p sat at its position j, the first j
   with pos_j(y) = p, and is written next to position (j + 1) mod n_hash.
   The chain stops at an empty slot, or at a slot that already holds the
   carried key.  After max_chain writes the key still carried is dropped
   (result 2).

Positions are a function argument, so a hand-made position table pins the
eviction order.  ``multiply_shift_positions`` is the hash the GPU table uses,
restated from its definition: pos_i(x) = (mix(x) * m_i mod 2^64) >> (64 - b)
for 2^b slots, with mix the splitmix64 output function (Steele, Lea & Flood
2014) and x the stored (tagged) slot value.
"""
from __future__ import annotations

M64 = (1 << 64) - 1
TAG = 1 << 31


def splitmix64_output(x: int) -> int:
    """The value splitmix64 returns from state x: (x + golden gamma) through its
    two xor-shift-multiply rounds and a final xor-shift."""
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def slot_value(key_words) -> int:
    """The stored value of a key: every word tagged with bit 31; a 2-word key is
    word 0 | word 1 << 32."""
    v = 0
    for i, w in enumerate(key_words):
        v |= (int(w) | TAG) << (32 * i)
    return v


def multiply_shift_positions(muls, log2_slots: int):
    """pos(x, i) for the table's hash: multiply-shift over splitmix64."""
    def pos(x: int, i: int) -> int:
        return ((splitmix64_output(x) * muls[i]) & M64) >> (64 - log2_slots)
    return pos


def insert_sequential(keys, n_slots: int, n_hash: int, max_chain: int, pos, table=None):
    """Insert the slot values `keys` one after another.  Returns (table, results,
    counters): table a list of n_slots values (0 = empty), results one of
    0/1/2 per key, counters (inserted, found, failed, writes)."""
    t = [0] * n_slots if table is None else table
    results = []
    inserted = found = failed = writes = 0
    for key in keys:
        if any(t[pos(key, i)] == key for i in range(n_hash)):
            results.append(0)
            found += 1
            continue
        r = 1
        x, p, n = key, pos(key, 0), 0
        while True:
            if n == max_chain:
                r = 2          # x is dropped
                break
            old, t[p] = t[p], x
            n += 1
            if old == 0:
                break
            if old == x:
                if n == 1:
                    r = 0      # only a concurrent insertion can reach this
                break
            x = old
            j = next((i for i in range(n_hash) if pos(old, i) == p), n_hash - 1)
            p = pos(old, (j + 1) % n_hash)
        writes += n
        results.append(r)
        inserted += r == 1
        found += r == 0
        failed += r == 2
    return t, results, (inserted, found, failed, writes)


def multiply_shift_positions_array(values, muls, log2_slots: int):
    """All n_hash positions of many slot values at once (numpy, uint64 arithmetic
    wrapping mod 2^64): an (len(values), len(muls)) array of slot indices."""
    import numpy as np
    z = np.asarray(values, dtype=np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    z = z ^ (z >> np.uint64(31))
    m = np.asarray(muls, dtype=np.uint64)
    return (z[:, None] * m[None, :]) >> np.uint64(64 - log2_slots)
