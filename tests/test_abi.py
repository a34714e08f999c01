"""The C-ABI library: loads, exports every declared entry point, and validates
networks on the host (no GPU needed for any call here)."""
import numpy as np
import pytest

from paper_1801_05857_gb300 import gx, inputs


def test_library_exports_every_declared_symbol():
    L = gx.lib()
    declared = gx.header_symbols()
    assert len(declared) >= 14
    missing = [s for s in declared if not hasattr(L, s)]
    assert not missing, missing


def test_layout_token_ring_word_boundary():
    """Sec. 5.2: the token ring's vector exceeds 32 bits from 11 nodes on (3 bits a node)."""
    for n, words in ((2, 1), (10, 1), (11, 2), (20, 2), (21, 4)):
        lay = gx.layout(gx.load_network(inputs.token_ring(n)))
        assert lay["vector_words"] == words, n
        assert (lay["field_bits"] == 3).all()
        # no field straddles a word and bit 31 stays free
        assert ((lay["field_offset"] + lay["field_bits"]) <= 31).all()


def test_layout_bits_per_process():
    net = inputs.random_network(0, 5, 16, n_labels=6, n_sync=2)
    net.procs[1].n_states = 2
    net.procs[1].edges = [(0, 3, 1), (1, 3, 0)]
    net.procs[2].n_states = 1
    net.procs[2].edges = []
    net.procs[2].initial = 0
    net.procs[3].n_states = 17
    lay = gx.layout(gx.load_network(net))
    assert lay["field_bits"].tolist() == [4, 1, 1, 5, 4]


def _bad(mut):
    net = inputs.producer_consumers()
    mut(net)
    with pytest.raises(gx.GxError) as e:
        gx.load_network(net)
    assert e.value.status == gx.GX_ERR_INVALID
    return e.value.message


def test_invalid_networks_are_rejected():
    assert "label" in _bad(lambda n: n.procs[0].edges.append((0, 17, 1)))
    assert "state" in _bad(lambda n: n.procs[1].edges.append((5, 0, 1)))
    assert "initial" in _bad(lambda n: setattr(n.procs[2], "initial", 9))
    assert "twice" in _bad(lambda n: n.rules.append(inputs.Rule([(1, 2), (1, 3)], 5)))
    assert "process" in _bad(lambda n: n.rules.append(inputs.Rule([(7, 2)], 5)))

    def too_wide(n):
        n.procs.extend([inputs.LTS(1 << 20, 0, []) for _ in range(7)])
    assert "words" in _bad(too_wide)

    def too_many_successors(n):  # 16 processes x 4 parallel edges: 4^16 = 2^32 combinations
        n.procs.extend([inputs.LTS(2, 0, [(0, 0, 1)] * 4) for _ in range(16)])
        n.rules.append(inputs.Rule([(p, 0) for p in range(len(n.procs) - 16, len(n.procs))], 0))
    assert "2^32" in _bad(too_many_successors)


def test_workspace_and_option_validation():
    h = gx.load_network(inputs.token_ring(12))          # 2-word vectors
    assert gx.workspace_bytes(h, gx.default_opts(table_bytes=1 << 20)) > (1 << 20)
    for bad in (dict(bucket_words=12), dict(bucket_words=8, group_lanes=3),
                dict(bucket_words=8, group_lanes=8), dict(hash_rounds=65)):
        with pytest.raises(gx.GxError) as e:
            gx.workspace_bytes(h, gx.default_opts(**bad))
        assert e.value.status == gx.GX_ERR_INVALID
    h4 = gx.load_network(inputs.token_ring(21))         # 4-word vectors
    with pytest.raises(gx.GxError):
        gx.workspace_bytes(h4, gx.default_opts(bucket_words=4, group_lanes=2))
    assert gx.workspace_bytes(h4, gx.default_opts(bucket_words=4, group_lanes=1)) > 0


def test_stats_before_search_is_a_state_error():
    h = gx.load_network(inputs.token_ring(3))
    with pytest.raises(gx.GxError) as e:
        gx.stats(h)
    assert e.value.status == gx.GX_ERR_STATE


def test_default_opts_values():
    o = gx.default_opts()
    assert (o.bucket_words, o.hash_rounds, o.deadlock_cap) == (8, 8, 1024)
    # both caches of seen vectors automatic; region passes automatic; scoring in its own kernel
    assert (o.warp_cache_log2, o.global_cache_log2, o.region_passes, o.guided_fused) == (0xFFFFFFFF, 0xFFFFFFFF, 0, 0)


def test_binding_constants_match_the_header():
    import re
    import os
    from paper_1801_05857_gb300 import build
    txt = open(os.path.join(build.INCLUDE, "gx.h")).read()
    assert int(re.search(r"#define GX_MLP_GRAD_CTAS (\d+)", txt).group(1)) == gx.MLP_GRAD_CTAS
    assert int(re.search(r"#define GX_MLP_IN (\d+)", txt).group(1)) == gx.MLP_IN
    assert int(re.search(r"#define GX_MLP_HIDDEN (\d+)", txt).group(1)) == gx.MLP_HIDDEN
    assert int(re.search(r"#define GX_BATCH_WIDE_OFF (0x[0-9A-Fa-f]+)u", txt).group(1), 16) == gx.BATCH_WIDE_OFF


def test_limits_at_their_boundaries():
    LTS, Rule, Network = inputs.LTS, inputs.Rule, inputs.Network
    # 124 one-bit processes fill four 31-bit words exactly; one more does not fit
    ok = Network(1, [LTS(2, 0, [(0, 0, 1)]) for _ in range(124)], [])
    assert gx.layout(gx.load_network(ok))["vector_words"] == 4
    with pytest.raises(gx.GxError) as e:
        gx.load_network(Network(1, [LTS(2, 0, [(0, 0, 1)]) for _ in range(125)], []))
    assert e.value.status == gx.GX_ERR_INVALID and "124" in e.value.message
    # a rule may have 16 participants, not 17
    procs = [LTS(2, 0, [(0, 0, 1)]) for _ in range(17)]
    gx.load_network(Network(1, procs, [Rule([(p, 0) for p in range(16)], 0)]))
    with pytest.raises(gx.GxError) as e:
        gx.load_network(Network(1, procs, [Rule([(p, 0) for p in range(17)], 0)]))
    assert e.value.status == gx.GX_ERR_INVALID and "16" in e.value.message
