"""gx_probe_gather, the random-read probe the table's roofline is measured with.

It has no counterpart in the paper: these tests check that it reads what its
header says (the unit positions, the words of each unit, the locality blocks)
by recomputing its checksum on the host, with splitmix64's output function
(Steele, Lea & Flood 2014) written from its published definition.
"""
import pytest

from paper_1801_05857_gb300 import gx

pytestmark = pytest.mark.gpu

M64 = (1 << 64) - 1


def mix64(x: int) -> int:
    z = (x + 0x9E3779B97F4A7C15) & M64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return z ^ (z >> 31)


def expected_checksum(words: int, n: int, unit_bytes: int, load_bytes: int, k: int, group_log2: int,
                      seed: int) -> int:
    """XOR of every word read, for a buffer whose word i holds i."""
    uw = unit_bytes // 4
    units = 1
    while units * 2 * uw <= words:
        units *= 2
    mask = units - 1
    gbits = group_log2 - (unit_bytes.bit_length() - 1) if group_log2 else 0
    inner = (1 << gbits) - 1
    acc = 0
    for i in range(n):
        r = mix64((seed + i) & M64)
        if gbits:
            block = mix64((~seed & M64) ^ (i // (32 * k))) & mask & ~inner
            u = block | (r & inner)
        else:
            u = r & mask
        for w in range(load_bytes // 4):
            acc ^= u * uw + w
    return acc


@pytest.mark.parametrize("unit,load,k", [(32, 4, 1), (32, 32, 4), (64, 64, 2), (64, 4, 8),
                                         (128, 128, 1), (128, 128, 4), (128, 4, 16)])
@pytest.mark.parametrize("group_log2", [0, 12])
@pytest.mark.parametrize("ctas", [2, 24])
def test_probe_gather_reads_the_documented_positions(cuda, unit, load, k, group_log2, ctas):
    import torch
    words = 1 << 20
    buf = torch.arange(words, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    n, seed = 5000, 12345
    used = gx.probe_gather(buf, n, unit, load, k, ctas, group_log2, seed, sink)
    torch.cuda.synchronize()
    assert (1 <= used <= 2) if ctas <= 8 else used == ctas
    assert int(sink.item()) == expected_checksum(words, n, unit, load, k, group_log2, seed)


def test_probe_gather_rejects_shapes_it_does_not_build(cuda):
    import torch
    buf = torch.zeros(1 << 16, dtype=torch.int32, device="cuda")
    sink = torch.zeros(1, dtype=torch.int64, device="cuda")
    for args in ((48, 48, 1, 1, 0), (128, 128, 8, 1, 0), (32, 16, 1, 1, 0), (64, 64, 32, 1, 0),
                 (32, 32, 3, 1, 0), (32, 32, 1, 33, 0), (32, 32, 1, 0, 0), (128, 128, 1, 1, 6)):
        unit, load, k, ctas, g = args
        with pytest.raises(gx.GxError):
            gx.probe_gather(buf, 100, unit, load, k, ctas, g, 1, sink)
