"""The DIMACS / hybrid-format reader (Appendix A): grammar, type identifiers,
CARD normalisation, the simplifier's reductions, a round trip, and the
appendix's own worked example (tests/golden/appendix_a_example.txt, parsed
verbatim). The other inputs are written here for these checks."""
import numpy as np
import pytest

from oracle import fe_oracle as O
from paper_2606_06641_gb300 import dimacs, synth

CNF = """c a plain CNF over 5 variables
p cnf 5 3
1 -2 0
-3 4 5
0
2 -5 0
"""

HYBRID = """* hybrid constraints, every identifier spelling
p cnf 8 14
h 1 2 -3 0             c a clause with the prefix
x 2 3 4 0
h xor -1 5 6 0
n 1 2 3 4 0
h nae 5 -6 7 0
a 1 2 3 0
amo 4 5 6 7 8 0
e 6 7 8 0
h eo 1 -8 0
k 2 1 2 3 4 0
h ek 3 2 3 4 5 6 0
d >=3 1 2 3 4 5 0
card >= 2 4 5 6 0
h card 3 1 2 3 4 0
"""

CARD_FORMS = """p cnf 6 6
card >3 1 2 3 4 5 0
card <=1 1 2 3 0
card -2 2 3 4 5 0
card <4 1 2 3 4 5 6 0
card > 0 1 2 3 0
card <= 2 4 5 6 0
"""


def test_plain_cnf_with_a_constraint_across_lines():
    p = dimacs.parse(CNF)
    assert p.declared == (5, 3) and p.inst.n == 5 and p.inst.m == 3
    assert list(p.inst.ctype) == [synth.OR] * 3
    assert [list(p.inst.constraint(c)) for c in range(3)] == [[1, -2], [-3, 4, 5], [2, -5]]


def test_every_type_identifier():
    p = dimacs.parse(HYBRID, simplify=False)
    want = [synth.OR, synth.XOR, synth.XOR, synth.NAE, synth.NAE, synth.AMO, synth.AMO, synth.EO,
            synth.EO, synth.EK, synth.EK, synth.CARD, synth.CARD, synth.CARD]
    assert list(p.inst.ctype) == want
    assert list(p.inst.constraint(0)) == [1, 2, -3]   # the trailing comment is ignored
    assert p.inst.param[9] == 2 and p.inst.param[10] == 3
    assert [(int(p.inst.op[c]), int(p.inst.param[c])) for c in (11, 12, 13)] == [
        (synth.GE, 3), (synth.GE, 2), (synth.GE, 3)]
    assert all(int(p.inst.parity[c]) == 1 for c in (1, 2))   # XOR: an odd number true


def test_card_normalisation():
    p = dimacs.parse(CARD_FORMS, simplify=False)
    got = [(int(p.inst.op[c]), int(p.inst.param[c])) for c in range(p.inst.m)]
    # > 3 -> >= 4; <= 1 -> < 2; -2 -> < 2; < 4 stays; > 0 -> >= 1; <= 2 -> < 3
    assert got == [(synth.GE, 4), (synth.LT, 2), (synth.LT, 2), (synth.LT, 4), (synth.GE, 1), (synth.LT, 3)]
    # the normalised forms have the meaning of the written operators
    written = [lambda t: t > 3, lambda t: t <= 1, lambda t: t < 2, lambda t: t < 4, lambda t: t > 0,
               lambda t: t <= 2]
    for c, holds in enumerate(written):
        k = int(p.inst.lengths[c])
        f = O.truth_table(O.T_CARD, k, int(p.inst.op[c]), int(p.inst.param[c]))
        assert [f[t] < 0 for t in range(k + 1)] == [holds(t) for t in range(k + 1)]


def test_simplifier_reductions():
    text = """p cnf 6 9
card >=0 1 2 0
a 3 0
card >=1 1 -2 0
k 1 1 2 3 0
4 0
e -5 0
k 2 5 6 0
k 0 1 2 0
card >= 1 6 0
"""
    with pytest.raises(dimacs.Unsatisfiable):
        dimacs.parse(text)   # 5 False (unit EO) but EK 2 over {5, 6} forces 5 True
    ok = text.replace("e -5 0", "e 5 0").replace("k 0 1 2 0", "k 0 3 4 0")
    with pytest.raises(dimacs.Unsatisfiable):
        dimacs.parse(ok)     # 4 True (unit clause) but EK 0 over {3, 4} forces 4 False
    ok = ok.replace("k 0 3 4 0", "k 0 3 1 0")
    p = dimacs.parse(ok)
    assert p.dropped == 2                                  # CARD >= 0 and the one-literal AMO
    assert list(p.inst.ctype[:2]) == [synth.OR, synth.EO]  # CARD >= 1 -> OR, EK 1 -> EO
    assert p.units == {4: True, 5: True, 6: True, 3: False, 1: False}


def test_round_trip_through_the_writer():
    p = dimacs.parse(HYBRID, simplify=False)
    q = dimacs.parse(dimacs.format_instance(p.inst), simplify=False)
    for name in ("ctype", "op", "param", "parity", "lit_off", "lits"):
        np.testing.assert_array_equal(getattr(p.inst, name), getattr(q.inst, name))
    r = synth.mixed_small(3)
    r.parity[:] = 1   # the format has odd parity only
    q = dimacs.parse(dimacs.format_instance(r), simplify=False, n_vars=r.n)
    for name in ("ctype", "lit_off", "lits"):
        np.testing.assert_array_equal(getattr(r, name), getattr(q.inst, name))
    cards = r.ctype == synth.CARD
    np.testing.assert_array_equal(r.op[cards], q.inst.op[cards])
    np.testing.assert_array_equal(r.param[cards], q.inst.param[cards])


@pytest.mark.parametrize("text", [
    "p cnf 3 1\n1 2 3\n",            # not terminated
    "p cnf 2 1\n1 3 0\n",            # variable beyond the declared count
    "p cnf 3 1\nx 0\n",              # no literals
    "p cnf 3 1\nd 1 2 0\n".replace("d 1", "d foo 1"),
    "p cnf 3 1\ncard 0 1 2 0\n",     # a plain threshold must be nonzero
    "p cnf 3 1\nek -1 1 2 0\n",
    "p cnf x 1\n1 0\n",
])
def test_malformed_input_is_rejected(text):
    with pytest.raises(dimacs.ParseError):
        dimacs.parse(text)


def _appendix_blocks():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "appendix_a_example.txt")
    with open(path) as fh:
        blocks = fh.read().split("\n\n")
    # keep the blocks that hold more than comment lines ('c' as the first token)
    return [b for b in blocks if any(ln.split() and ln.split()[0] != "c" for ln in b.splitlines())]


def test_appendix_example_blocks_parse_verbatim():
    """The appendix's worked example (inline 'c' comments after the
    terminating 0, the 'h' prefix, 'h d >=2', plain and signed CARD
    thresholds) parses block by block into the constraints it describes, and
    each constraint's truth table is the one the appendix states."""
    cnf, hybrid, cards = [dimacs.parse(b, simplify=False) for b in _appendix_blocks()]
    assert cnf.declared == (4, 2) and [list(cnf.inst.constraint(c)) for c in range(2)] == [[1, -2, 3], [-1, 4]]
    assert list(cnf.inst.ctype) == [synth.OR, synth.OR]
    assert hybrid.declared == (6, 7)
    assert list(hybrid.inst.ctype) == [synth.OR, synth.XOR, synth.NAE, synth.AMO, synth.EO, synth.EK, synth.CARD]
    assert [list(hybrid.inst.constraint(c)) for c in range(7)] == [[1, -2, 3], [1, 2, 3], [1, 2, 3], [1, 2, 3],
                                                                   [4, 5, 6], [1, 2, 3], [1, 2, 3]]
    assert int(hybrid.inst.param[5]) == 2 and (int(hybrid.inst.op[6]), int(hybrid.inst.param[6])) == (O.OP_GE, 2)
    assert cards.declared is None and cards.inst.m == 4
    # the semantics records list the examples in the same order (the CNF
    # block's clauses share the first record's OR table)
    recs = []
    with open(__file__.replace("test_dimacs.py", "golden/appendix_a_semantics.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                recs.append([int(v) for v in line.split()[5:]])
    got = [O.truth_table(int(p.inst.ctype[c]), int(np.diff(p.inst.lit_off)[c]), int(p.inst.op[c]),
                         int(p.inst.param[c]), int(p.inst.parity[c])).tolist()
           for p in (hybrid, cards) for c in range(p.inst.m)]
    assert got == recs
