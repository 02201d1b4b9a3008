"""Readers of external constraint sets: DIMACS CNF and OPB.

The library evaluates symmetric pseudo-Boolean constraints (Sec. 2.2): a
predicate on the number t of true literals of a constraint.  A CNF clause is
the disjunction t >= 1.  An OPB linear constraint sum_i a_i l_i REL k is
symmetric when every coefficient is +1 or -1; a term -l_i is rewritten as
~l_i - 1 (so the right-hand side grows by one), and REL >= / = / <= becomes
at-least-k, exactly-k or at-most-k on the rewritten literals.  Other
coefficients are rejected: such a constraint is not a function of t alone.

Literal convention of the C interface: lit_sign +1 for a positive literal
(true when its variable is true), -1 for a negated one.  Variables are
numbered from 0 (DIMACS and OPB number them from 1).

The readers return a ConstraintSet, which api.Problem accepts directly.
"""
from __future__ import annotations

import os
import re
from dataclasses import dataclass, field
from typing import List, Optional, Tuple

import numpy as np

# constraint types of the C interface (include/cls.h)
CLS_OR, CLS_CARD_GE, CLS_CARD_LE, CLS_EK = 0, 2, 3, 6


@dataclass
class ConstraintSet:
    n: int
    offsets: np.ndarray
    lit_var: np.ndarray
    lit_sign: np.ndarray
    ctype: np.ndarray
    k: np.ndarray
    weight: np.ndarray
    spectra: Optional[np.ndarray] = None
    fixed: Optional[np.ndarray] = None
    fixed_val: Optional[np.ndarray] = None
    name: str = ""
    # lines dropped as always true (tautological clauses, trivially satisfied
    # linear constraints), for the caller's information
    dropped: int = 0
    notes: List[str] = field(default_factory=list)

    @property
    def m(self) -> int:
        return int(len(self.offsets) - 1)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])


def _text(src: str) -> str:
    if "\n" not in src and os.path.exists(src):
        with open(src) as f:
            return f.read()
    return src


def _pack(n, rows, name, dropped, notes) -> ConstraintSet:
    offsets = np.zeros(len(rows) + 1, dtype=np.int32)
    for c, (_, _, lits) in enumerate(rows):
        offsets[c + 1] = offsets[c] + len(lits)
    lit_var = np.array([v for _, _, lits in rows for v, _ in lits], dtype=np.int32)
    lit_sign = np.array([s for _, _, lits in rows for _, s in lits], dtype=np.int8)
    ctype = np.array([t for t, _, _ in rows], dtype=np.int32)
    k = np.array([kk for _, kk, _ in rows], dtype=np.int32)
    return ConstraintSet(n=int(n), offsets=offsets, lit_var=lit_var, lit_sign=lit_sign,
                         ctype=ctype, k=k, weight=np.ones(len(rows), dtype=np.float32),
                         name=name, dropped=dropped, notes=notes)


def read_dimacs(src: str, name: str = "") -> ConstraintSet:
    """DIMACS CNF ("p cnf n m", clauses of nonzero integers ended by 0; lines
    starting with c are comments; a line starting with % ends the file, as
    in collections that append "%" and a stray "0").  Repeated literals in a clause are merged;
    a clause holding a variable and its negation is always true and dropped.
    An empty clause raises ValueError (no assignment satisfies it)."""
    text = _text(src)
    n = None
    declared = None
    rows: List[Tuple[int, int, List[Tuple[int, int]]]] = []
    cur: List[int] = []
    dropped = 0

    def close(cl: List[int]):
        nonlocal dropped
        seen = {}
        for lit in cl:
            v, s = abs(lit) - 1, (1 if lit > 0 else -1)
            if v in seen and seen[v] != s:
                dropped += 1
                return
            seen[v] = s
        if not seen:
            raise ValueError("empty clause: the formula is unsatisfiable")
        rows.append((CLS_OR, 0, sorted(seen.items())))

    for line in text.splitlines():
        line = line.strip()
        if line.startswith("%"):      # end marker of some benchmark collections
            break
        if not line or line[0] == "c":
            continue
        if line[0] == "p":
            parts = line.split()
            if len(parts) < 4 or parts[1] != "cnf":
                raise ValueError(f"bad problem line: {line!r}")
            n, declared = int(parts[2]), int(parts[3])
            continue
        if n is None:
            raise ValueError("clause before the problem line")
        for tok in line.split():
            lit = int(tok)
            if lit == 0:
                close(cur)
                cur = []
            else:
                if abs(lit) > n:
                    raise ValueError(f"literal {lit} beyond {n} variables")
                cur.append(lit)
    if cur:
        close(cur)
    if n is None:
        raise ValueError("no problem line")
    notes = []
    if declared is not None and declared != len(rows) + dropped:
        notes.append(f"problem line declares {declared} clauses, file holds {len(rows) + dropped}")
    return _pack(n, rows, name or "dimacs", dropped, notes)


_TERM = re.compile(r"([+-]?\d+)\s+(~?)x(\d+)")


def read_opb(src: str, name: str = "") -> ConstraintSet:
    """OPB linear constraints with coefficients +1 / -1 ("+1 x1 -1 ~x2 >= 1 ;",
    relations >=, = and <=; lines starting with * are comments; an objective
    line "min:" / "max:" is ignored, since the solver targets satisfaction).
    The number of variables is the largest index seen, or the header's
    "#variable= n" if larger.  A constraint that always holds is dropped;
    one that never holds raises ValueError."""
    text = _text(src)
    n_decl = 0
    rows: List[Tuple[int, int, List[Tuple[int, int]]]] = []
    dropped = 0
    notes = []
    vmax = 0
    for raw in text.split(";"):
        for line in raw.splitlines():
            if line.strip().startswith("*"):
                m = re.search(r"#variable=\s*(\d+)", line)
                if m:
                    n_decl = max(n_decl, int(m.group(1)))
        body = " ".join(l for l in raw.splitlines() if not l.strip().startswith("*")).strip()
        if not body:
            continue
        if body.startswith(("min:", "max:")):
            notes.append("objective line ignored")
            continue
        m = re.match(r"^(.*?)(>=|<=|=)\s*([+-]?\d+)\s*$", body)
        if not m:
            raise ValueError(f"bad constraint: {body!r}")
        lhs, rel, rhs = m.group(1), m.group(2), int(m.group(3))
        terms = _TERM.findall(lhs)
        if not terms or _TERM.sub("", lhs).strip():
            raise ValueError(f"bad left-hand side: {lhs!r}")
        lits = {}
        k = rhs
        for coef, neg, idx in terms:
            a, v = int(coef), int(idx) - 1
            if a not in (1, -1):
                raise ValueError(f"coefficient {a}: not a symmetric constraint")
            if v < 0:
                raise ValueError("variables are numbered from 1")
            vmax = max(vmax, v + 1)
            s = -1 if neg else 1
            if a == -1:               # -l = ~l - 1
                s, k = -s, k + 1
            if v in lits:
                if lits[v] == s:
                    raise ValueError(f"x{v + 1} twice with the same sign: coefficient 2")
                del lits[v]           # l + ~l = 1
                k -= 1
                continue
            lits[v] = s
        L = len(lits)
        if rel == ">=":
            always, never, t = k <= 0, k > L, CLS_CARD_GE
        elif rel == "<=":
            always, never, t = k >= L, k < 0, CLS_CARD_LE
        else:
            always, never, t = False, k < 0 or k > L, CLS_EK
        if never:
            raise ValueError(f"constraint {body!r} can never hold")
        if always or L == 0:
            dropped += 1
            continue
        rows.append((t, k, sorted(lits.items())))
    return _pack(max(vmax, n_decl), rows, name or "opb", dropped, notes)
