"""The text front end (gx_load_exp): the paper's input format of Sec. 3 /
Fig. 1, parsed on the host.  No GPU is needed for anything here."""
import os

import numpy as np
import pytest

from paper_1801_05857_gb300 import gx, inputs

FIG1 = os.path.join(os.path.dirname(__file__), "golden", "fig1")


def to_text(net):
    """An inputs.Network as an EXP.OPEN composition plus one .aut file per process."""
    files = {}
    for p, lts in enumerate(net.procs):
        lines = [f"des ({lts.initial}, {len(lts.edges)}, {lts.n_states})"]
        lines += [f'({s}, "a{a}", {t})' for s, a, t in lts.edges]
        files[f"p{p}.aut"] = "\n".join(lines) + "\n"
    vecs = []
    for r in net.rules:
        entry = ["_"] * len(net.procs)
        for p, a in r.parts:
            entry[p] = f"a{a}"
        vecs.append(" * ".join(entry) + f" -> r{r.result}")
    using = ("using\n    " + ",\n    ".join(vecs) + "\n") if vecs else ""
    procs = " || ".join(f'"p{p}.aut"' for p in range(len(net.procs)))
    return f"par {using}in\n    {procs}\nend par\n", files


def test_fig1_from_the_paper_format():
    h = gx.load_exp_file(os.path.join(FIG1, "fig1.exp"))
    c = gx.network_counts(h)
    assert c == dict(n_procs=3, n_labels=6, n_rules=2, n_edges=8)
    names = {gx.label_name(h, i) for i in range(c["n_labels"])}
    assert names == {"gen_work", "send", "rec", "work", "tau", "trans"}
    assert gx.layout(h)["field_bits"].tolist() == [1, 1, 1]


@pytest.mark.parametrize("net", [inputs.token_ring(5), inputs.producer_consumers()] +
                         [inputs.random_network(s, 6, 8, 1, 3, 10, n_sync=3, parties=2 + s % 2)
                          for s in range(6)], ids=lambda n: n.name)
def test_round_trip_keeps_the_network(net):
    exp, files = to_text(net)
    a = gx.load_exp(exp, files)
    b = gx.load_network(net)
    ca, cb = gx.network_counts(a), gx.network_counts(b)
    assert (ca["n_procs"], ca["n_rules"], ca["n_edges"]) == (cb["n_procs"], cb["n_rules"], cb["n_edges"])
    la, lb = gx.layout(a), gx.layout(b)
    assert la["vector_words"] == lb["vector_words"]
    for k in ("field_word", "field_offset", "field_bits"):
        assert (la[k] == lb[k]).all()


def test_same_file_for_several_processes_and_comments():
    exp = '(* two copies *) par using "go" * "go" -> sync (* end *) in "a.aut" || "a.aut" end par'
    h = gx.load_exp(exp, {"a.aut": 'des (0, 2, 2)\n(0, "go", 1)\n(1, i, 0)\n'})
    assert gx.network_counts(h) == dict(n_procs=2, n_labels=3, n_rules=1, n_edges=4)
    assert gx.label_name(h, 1) == "i"


def test_interleaving_only_composition():
    h = gx.load_exp('par in "a.aut" || "a.aut" || "a.aut" end par', {"a.aut": "des (1, 1, 3)\n(1, x, 2)\n"})
    c = gx.network_counts(h)
    assert (c["n_procs"], c["n_rules"]) == (3, 0)


A = 'des (0, 1, 2)\n(0, "x", 1)\n'


@pytest.mark.parametrize("exp,files,needle", [
    ('par using x * -> y in "a.aut" || "a.aut" end par', {"a.aut": A}, "label or '_'"),
    ('par using x * x * x -> y in "a.aut" || "a.aut" end par', {"a.aut": A}, "3 entries for 2"),
    ('par using _ * _ -> y in "a.aut" || "a.aut" end par', {"a.aut": A}, "without participants"),
    ('par in "a.aut" || "b.aut" end par', {"a.aut": A}, '"b.aut"'),
    ('par in "a.aut" end', {"a.aut": A}, "'par' after 'end'"),
    ('par in "a.aut" end par extra', {"a.aut": A}, "after 'end par'"),
    ('par (* open in "a.aut" end par', {"a.aut": A}, "unterminated comment"),
    ('par in "a.aut" end par', {"a.aut": 'des (0, 2, 2)\n(0, "x", 1)\n'}, "transition 1 of 2"),
    ('par in "a.aut" end par', {"a.aut": 'des (0, 1, 2)\n(0, "x", 2)\n'}, "state out of range"),
    ('par in "a.aut" end par', {"a.aut": 'des (2, 0, 2)\n'}, "initial state"),
    ('par in "a.aut" end par', {"a.aut": 'des (0, 1, 2)\n(0, "x", 1)\n(1, "y", 0)\n'}, "text after"),
    ('par in "a.aut" end par', {"a.aut": 'dez (0, 0, 1)\n'}, "expected 'des"),
])
def test_syntax_errors_name_the_place(exp, files, needle):
    with pytest.raises(gx.GxError) as e:
        gx.load_exp(exp, files)
    assert e.value.status == gx.GX_ERR_INVALID
    assert needle in e.value.message
    if needle != '"b.aut"':  # a missing file is named, not placed
        assert "line" in e.value.message
