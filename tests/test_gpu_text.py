"""Networks read from the paper's input format (gx_load_exp) explore exactly
like the same networks given as arrays: GPU against the oracle."""
import os

import pytest

import oracle
from paper_1801_05857_gb300 import gx, inputs
from test_text import FIG1, to_text

pytestmark = pytest.mark.gpu


def _explore(h, **kw):
    import torch
    o = gx.default_opts(**kw)
    ws = gx.alloc_workspace(h, o)
    gx.explore(h, o, ws)
    torch.cuda.synchronize()
    return gx.stats(h), gx.levels(h)


def test_fig1_text_has_8_states_and_24_transitions(cuda):
    s, lv = _explore(gx.load_exp_file(os.path.join(FIG1, "fig1.exp")), table_bytes=1 << 16)
    assert (s["states"], s["transitions"], s["complete"]) == (8, 24, 1)
    r = oracle.explore(inputs.producer_consumers())
    assert lv == r.levels


@pytest.mark.parametrize("net", [inputs.token_ring(9)] +
                         [inputs.random_network(s, 6, 8, 0, 3, 10, n_sync=3, parties=2 + s % 2)
                          for s in range(6)], ids=lambda n: n.name)
def test_text_networks_match_the_oracle(cuda, net):
    exp, files = to_text(net)
    s, lv = _explore(gx.load_exp(exp, files), table_bytes=1 << 24)
    r = oracle.explore(net)
    assert (s["states"], s["transitions"], lv) == (r.states, r.transitions, r.levels)
    assert (s["deadlock_count"], s["deadlock_sum"], s["deadlock_xor"]) == \
        (r.deadlock_count, r.deadlock_sum, r.deadlock_xor)
