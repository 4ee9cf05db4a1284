"""Reader for standard DIMACS CNF and the hybrid DIMACS-like format of the
paper's Appendix A (input-format specification, grammar and type table).

A file is a sequence of lines: comments start with ``c`` or ``*``, the problem
line is ``p cnf <n_vars> <n_constraints>``, and a constraint is an optional
``h`` prefix, an optional type identifier and its literals, terminated by the
literal ``0`` (tokens after the terminating ``0`` on the same line are a
comment). Type identifiers (Appendix A, type table):

  (none)            OR   disjunction
  ``x``/``xor``     XOR  an odd number of literals true
  ``n``/``nae``     NAE  not all literals equal
  ``a``/``amo``     AMO  at most one literal true
  ``e``/``eo``      EO   exactly one literal true
  ``k``/``ek`` r    EK   exactly r literals true
  ``d``/``card`` T  CARD threshold T, where T is ``>=r``, ``>r``, ``<=r``,
                    ``<r`` (operator and number in one token or two) or a
                    plain signed integer: r > 0 means ``>= r``, r < 0 means
                    ``< |r|``.

CARD is normalised to ``>= r`` or ``< r`` (``> r`` -> ``>= r+1``, ``<= r`` ->
``< r+1``), the two forms the kernels' truth tables take.

``parse(text, simplify=True)`` returns a :class:`Parsed` with the instance and
the unit assignments the simplifier found. The simplifier applies the
appendix's reductions that need no propagation: CARD ``>= 0`` (and ``< r``
with r > k) and single-literal AMO are dropped as always true, CARD ``>= 1``
becomes OR and EK 1 becomes EO; single-literal OR and EO, CARD/EK with r = k
and EK 0 become unit assignments, which are kept as constraints too (so the
instance alone is still equivalent to the file) and reported in ``units``;
two units that disagree raise :class:`Unsatisfiable`.
"""
from __future__ import annotations

import re
from dataclasses import dataclass, field
from typing import Dict, List, Optional, Tuple

from . import synth

__all__ = ["Parsed", "ParseError", "Unsatisfiable", "parse", "parse_file", "format_instance"]


class ParseError(ValueError):
    pass


class Unsatisfiable(ValueError):
    pass


@dataclass
class Parsed:
    inst: synth.Instance
    units: Dict[int, bool] = field(default_factory=dict)   # variable (1-based) -> True/False
    dropped: int = 0                                      # constraints removed as always true
    declared: Optional[Tuple[int, int]] = None            # the problem line's (n, m)


_TYPES = {"x": synth.XOR, "xor": synth.XOR, "n": synth.NAE, "nae": synth.NAE, "a": synth.AMO,
          "amo": synth.AMO, "e": synth.EO, "eo": synth.EO}
_INT = re.compile(r"^-?[0-9]+$")
_CARD_OP = re.compile(r"^(>=|<=|>|<)(-?[0-9]+)?$")


def _card_threshold(tokens: List[str], pos: int, where: str) -> Tuple[int, int, int]:
    """(op, r, next position) for the CARD threshold starting at tokens[pos]."""
    if pos >= len(tokens):
        raise ParseError(f"{where}: CARD without a threshold")
    tok = tokens[pos]
    m = _CARD_OP.match(tok)
    if m:
        op, num = m.group(1), m.group(2)
        pos += 1
        if num is None:
            if pos >= len(tokens) or not _INT.match(tokens[pos]):
                raise ParseError(f"{where}: CARD operator {op} without a number")
            num = tokens[pos]
            pos += 1
        r = int(num)
        if r < 0:
            raise ParseError(f"{where}: CARD {op} needs a non-negative number")
        if op == ">=":
            return synth.GE, r, pos
        if op == ">":
            return synth.GE, r + 1, pos
        if op == "<":
            return synth.LT, r, pos
        return synth.LT, r + 1, pos   # <= r  ->  < r + 1
    if _INT.match(tok):
        r = int(tok)
        if r == 0:
            raise ParseError(f"{where}: a plain CARD threshold must be nonzero")
        return (synth.GE, r, pos + 1) if r > 0 else (synth.LT, -r, pos + 1)
    raise ParseError(f"{where}: bad CARD threshold {tok!r}")


def _constraint(tokens: List[str], where: str):
    """(ctype, op, param, parity, literals) of one constraint's tokens (without the final 0)."""
    pos = 0
    if pos < len(tokens) and tokens[pos] == "h":
        pos += 1
    if pos >= len(tokens):
        raise ParseError(f"{where}: empty constraint")
    head = tokens[pos].lower()
    ctype, op, param, parity = synth.OR, synth.GE, 0, 1
    if head in _TYPES:
        ctype = _TYPES[head]
        pos += 1
    elif head in ("k", "ek"):
        ctype = synth.EK
        pos += 1
        if pos >= len(tokens) or not _INT.match(tokens[pos]):
            raise ParseError(f"{where}: EK without its count")
        param = int(tokens[pos])
        if param < 0:
            raise ParseError(f"{where}: EK count must be non-negative")
        pos += 1
    elif head in ("d", "card"):
        ctype = synth.CARD
        op, param, pos = _card_threshold(tokens, pos + 1, where)
    lits = []
    for tok in tokens[pos:]:
        if not _INT.match(tok):
            raise ParseError(f"{where}: bad literal {tok!r}")
        v = int(tok)
        if v == 0:
            raise ParseError(f"{where}: literal 0 inside a constraint")
        lits.append(v)
    if not lits:
        raise ParseError(f"{where}: constraint without literals")
    return ctype, op, param, parity, lits


def _is_comment(first: str) -> bool:
    """A line whose first token is ``c`` (or starts with ``c`` and is not the
    ``card`` identifier) or starts with ``*`` is a comment."""
    return first.startswith("*") or (first[0] == "c" and first.lower() != "card")


def parse(text: str, simplify: bool = True, n_vars: Optional[int] = None) -> Parsed:
    declared = None
    records = []
    pending: List[str] = []
    pending_line = 0
    for lineno, raw in enumerate(text.splitlines(), 1):
        line = raw.strip()
        if not line:
            continue
        toks = line.split()
        if _is_comment(toks[0]):
            continue
        if not pending and toks[0] == "p":
            if len(toks) != 4 or toks[1] != "cnf" or not (_INT.match(toks[2]) and _INT.match(toks[3])):
                raise ParseError(f"line {lineno}: bad problem line")
            declared = (int(toks[2]), int(toks[3]))
            continue
        if not pending:
            pending_line = lineno
        for i, tok in enumerate(toks):
            if tok == "0" and not (pending and pending[-1] in ("k", "ek", "d", "card", ">=", ">", "<=", "<")):
                records.append(_constraint(pending, f"line {pending_line}"))
                pending = []
                # the rest of the line after a terminating 0 is a comment
                break
            pending.append(tok)
    if pending:
        raise ParseError(f"line {pending_line}: constraint not terminated by 0")
    n = n_vars if n_vars is not None else (declared[0] if declared else 0)
    n = max([n] + [abs(v) for rec in records for v in rec[4]])
    if declared and n > declared[0]:
        raise ParseError(f"a literal uses variable {n} beyond the declared {declared[0]}")

    units: Dict[int, bool] = {}
    dropped = 0

    def unit(v: int, val: bool):
        if units.get(v, val) != val:
            raise Unsatisfiable(f"variable {v} is forced both True and False")
        units[v] = val

    b = synth._Builder(n)
    for ctype, op, param, parity, lits in records:
        k = len(lits)
        if simplify:
            if ctype == synth.CARD and ((op == synth.GE and param <= 0) or (op == synth.LT and param > k)):
                dropped += 1
                continue
            if ctype == synth.AMO and k == 1:
                dropped += 1
                continue
            if ctype == synth.CARD and op == synth.GE and param == 1:
                ctype = synth.OR
            if ctype == synth.EK and param == 1:
                ctype = synth.EO
            if ctype in (synth.OR, synth.EO) and k == 1:
                unit(abs(lits[0]), lits[0] > 0)
            if (ctype == synth.EK or (ctype == synth.CARD and op == synth.GE)) and param == k:
                for v in lits:
                    unit(abs(v), v > 0)
            if ctype == synth.EK and param == 0:
                for v in lits:
                    unit(abs(v), v < 0)
        b.add(ctype, lits, op, param, parity)
    return Parsed(b.build(), units, dropped, declared)


def parse_file(path: str, simplify: bool = True) -> Parsed:
    with open(path) as fh:
        return parse(fh.read(), simplify=simplify)


_NAMES = {synth.XOR: "x", synth.NAE: "nae", synth.AMO: "amo", synth.EO: "eo"}


def format_instance(inst: synth.Instance) -> str:
    """The instance in the hybrid format (CARD as >=r or <r)."""
    out = [f"p cnf {inst.n} {inst.m}"]
    for c in range(inst.m):
        lits = " ".join(str(int(v)) for v in inst.constraint(c))
        t = int(inst.ctype[c])
        if t == synth.OR:
            out.append(f"h {lits} 0")
        elif t == synth.EK:
            out.append(f"h ek {int(inst.param[c])} {lits} 0")
        elif t == synth.CARD:
            op = ">=" if int(inst.op[c]) == synth.GE else "<"
            out.append(f"h card {op}{int(inst.param[c])} {lits} 0")
        elif t == synth.XOR and int(inst.parity[c]) == 0:
            raise ValueError("the hybrid format has no even-parity XOR")
        else:
            out.append(f"h {_NAMES[t]} {lits} 0")
    return "\n".join(out) + "\n"
