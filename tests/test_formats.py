"""DIMACS CNF and OPB readers (host logic, no GPU).

Two kinds of check: the arrays a small hand-written file turns into, field
by field; and, on random files over few variables, the meaning -- for every
one of the 2^n assignments the number of constraints the oracle finds
satisfied (its Sec. 2.3 score on the parsed constraint set) equals the
number a direct evaluation of the file's own clauses or linear inequalities
finds (plus the always-true lines the reader dropped).  The texts are
written here or generated from a seed; none comes from a benchmark suite."""

import numpy as np
import pytest

from oracle import cls as O
from paper_2606_06656_b300 import binding as B
from paper_2606_06656_b300.formats import (CLS_CARD_GE, CLS_CARD_LE, CLS_EK, CLS_OR,
                                           read_dimacs, read_opb)


def all_assignments(n):
    """X[v, r] for every assignment r (bit v of r set = variable v True,
    which the library encodes as x < 0)."""
    R = 1 << n
    bits = (np.arange(R)[None, :] >> np.arange(n)[:, None]) & 1
    return np.where(bits == 1, -1.0, 1.0).astype(np.float32), bits.astype(bool)


# ---------------------------------------------------------------------------
# DIMACS
# ---------------------------------------------------------------------------

CNF = """c a small formula
c over four variables
p cnf 4 5
1 -2 3 0
-1 4 0
2 2 -3 0
c a tautology follows
1 -1 4 0
-4
 -3 0
"""


def test_dimacs_arrays():
    s = read_dimacs(CNF)
    assert s.n == 4 and s.m == 4 and s.dropped == 1
    assert s.offsets.tolist() == [0, 3, 5, 7, 9]
    assert s.lit_var.tolist() == [0, 1, 2, 0, 3, 1, 2, 2, 3]
    assert s.lit_sign.tolist() == [1, -1, 1, -1, 1, 1, -1, -1, -1]
    assert s.ctype.tolist() == [CLS_OR] * 4
    assert s.weight.tolist() == [1.0] * 4
    assert s.notes == []            # 4 kept + 1 dropped = the declared 5
    rc, msg = B.cls_problem_check(s)
    assert rc == 0, msg


def test_dimacs_errors_and_notes():
    with pytest.raises(ValueError, match="empty clause"):
        read_dimacs("p cnf 2 2\n1 2 0\n0\n")
    with pytest.raises(ValueError, match="beyond"):
        read_dimacs("p cnf 2 1\n1 3 0\n")
    with pytest.raises(ValueError, match="problem line"):
        read_dimacs("1 2 0\n")
    with pytest.raises(ValueError, match="bad problem line"):
        read_dimacs("p wcnf 2 1\n1 2 0\n")
    s = read_dimacs("p cnf 3 4\n1 2 0\n-3 0\n")   # last clause without its 0
    assert s.m == 2 and len(s.notes) == 1
    s = read_dimacs("p cnf 3 1\n1 2 3")
    assert s.offsets.tolist() == [0, 3]
    s = read_dimacs("p cnf 3 2\n1 -2 0\n2 3 0\n%\n0\n\n")   # end marker
    assert s.m == 2 and s.notes == []


def test_dimacs_reads_a_file(tmp_path):
    f = tmp_path / "f.cnf"
    f.write_text(CNF)
    a, b = read_dimacs(str(f)), read_dimacs(CNF)
    assert a.lit_var.tolist() == b.lit_var.tolist()


def random_cnf(rng, n, m, kmax):
    lines = [f"p cnf {n} {m}"]
    clauses = []
    for _ in range(m):
        k = int(rng.integers(1, kmax + 1))
        cl = [int(v + 1) * int(rng.choice([-1, 1])) for v in rng.integers(0, n, size=k)]
        clauses.append(cl)
        lines.append(" ".join(map(str, cl)) + " 0")
    return "\n".join(lines) + "\n", clauses


@pytest.mark.parametrize("seed", range(6))
def test_dimacs_meaning_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = 8
    text, clauses = random_cnf(rng, n, 30, 5)
    s = read_dimacs(text)
    X, truth = all_assignments(n)
    nsat, _, _ = O.score(s, X)
    direct = np.zeros(X.shape[1], dtype=np.int64)
    for cl in clauses:
        direct += np.any([truth[l - 1] if l > 0 else ~truth[-l - 1] for l in cl], axis=0)
    assert (nsat + s.dropped == direct).all()


# ---------------------------------------------------------------------------
# OPB
# ---------------------------------------------------------------------------

OPB = """* #variable= 6 #constraint= 6
* a made-up example
min: +1 x1 +1 x2 ;
+1 x1 +1 x2 +1 ~x3 >= 2 ;
-1 x1 -1 x4 >= -1 ;
+1 x2 +1 x5 +1 x6 = 1;
+1 x1 -1 x1 +1 x2 <= 0 ;
+1 x3 +1 ~x3 +1 x4 >= 1 ;
+1 x5
 +1 x6 <= 2 ;
"""


def test_opb_arrays():
    s = read_opb(OPB)
    assert s.n == 6 and s.m == 4 and s.dropped == 2
    assert s.notes == ["objective line ignored"]
    assert s.offsets.tolist() == [0, 3, 5, 8, 9]
    # x1 + x2 + ~x3 >= 2
    assert s.lit_var[:3].tolist() == [0, 1, 2] and s.lit_sign[:3].tolist() == [1, 1, -1]
    assert s.ctype[0] == CLS_CARD_GE and s.k[0] == 2
    # -x1 - x4 >= -1  ->  ~x1 + ~x4 >= 1
    assert s.lit_var[3:5].tolist() == [0, 3] and s.lit_sign[3:5].tolist() == [-1, -1]
    assert s.ctype[1] == CLS_CARD_GE and s.k[1] == 1
    # x2 + x5 + x6 = 1
    assert s.ctype[2] == CLS_EK and s.k[2] == 1
    # x1 - x1 + x2 <= 0  ->  x1 + ~x1 + x2 <= 1  ->  x2 <= 0
    assert s.lit_var[8:].tolist() == [1] and s.lit_sign[8:].tolist() == [1]
    assert s.ctype[3] == CLS_CARD_LE and s.k[3] == 0
    # x3 + ~x3 + x4 >= 1 is always true; x5 + x6 <= 2 too
    rc, msg = B.cls_problem_check(s)
    assert rc == 0, msg


def test_opb_errors():
    with pytest.raises(ValueError, match="coefficient 2"):
        read_opb("+2 x1 +1 x2 >= 1 ;")
    with pytest.raises(ValueError, match="coefficient 2"):
        read_opb("+1 x1 +1 x1 >= 1 ;")
    with pytest.raises(ValueError, match="never hold"):
        read_opb("+1 x1 +1 x2 >= 3 ;")
    with pytest.raises(ValueError, match="never hold"):
        read_opb("+1 x1 +1 ~x1 = 0 ;")
    with pytest.raises(ValueError, match="bad"):
        read_opb("+1 x1 +1 y2 >= 1 ;")
    with pytest.raises(ValueError, match="bad constraint"):
        read_opb("+1 x1 +1 x2 ;")


def random_opb(rng, n, m):
    lines = [f"* #variable= {n} #constraint= {m}"]
    cons = []
    for _ in range(m):
        L = int(rng.integers(1, 7))
        terms = []
        for v in rng.integers(0, n, size=L):
            terms.append((int(rng.choice([-1, 1])), bool(rng.integers(0, 2)), int(v)))
        # no same variable with the same literal twice (that would be a
        # coefficient 2 after merging)
        seen, kept = set(), []
        for a, neg, v in terms:
            key = (v, neg if a == 1 else not neg)
            if key in seen:
                continue
            seen.add(key)
            kept.append((a, neg, v))
        rel = str(rng.choice([">=", "<=", "="]))
        lo = sum(min(a, 0) for a, _, _ in kept)
        hi = sum(max(a, 0) for a, _, _ in kept)
        k = int(rng.integers(lo - 1, hi + 2))
        cons.append((kept, rel, k))
        body = " ".join(f"{a:+d} {'~' if neg else ''}x{v + 1}" for a, neg, v in kept)
        lines.append(f"{body} {rel} {k} ;")
    return "\n".join(lines) + "\n", cons


def linear_holds(cons, truth):
    kept, rel, k = cons
    lhs = np.zeros(truth.shape[1], dtype=np.int64)
    for a, neg, v in kept:
        lhs += a * (~truth[v] if neg else truth[v])
    return {">=": lhs >= k, "<=": lhs <= k, "=": lhs == k}[rel]


@pytest.mark.parametrize("seed", range(8))
def test_opb_meaning_brute_force(seed):
    rng = np.random.default_rng(100 + seed)
    n = 7
    X, truth = all_assignments(n)
    kept_cons, text_lines = [], [f"* #variable= {n}"]
    text, cons = random_opb(rng, n, 40)
    # keep the constraints that can hold somewhere (the reader raises on
    # the others); check that it does raise on them
    for c, line in zip(cons, text.splitlines()[1:]):
        if linear_holds(c, truth).any():
            kept_cons.append(c)
            text_lines.append(line)
        else:
            with pytest.raises(ValueError, match="never hold"):
                read_opb(line)
    s = read_opb("\n".join(text_lines))
    assert s.n == n
    nsat, _, _ = O.score(s, X)
    direct = sum(linear_holds(c, truth).astype(np.int64) for c in kept_cons)
    assert (nsat + s.dropped == direct).all()
    # a dropped line holds for every assignment
    assert s.m + s.dropped == len(kept_cons)


def test_readers_feed_problem_check():
    rng = np.random.default_rng(7)
    text, _ = random_cnf(rng, 50, 200, 4)
    rc, msg = B.cls_problem_check(read_dimacs(text))
    assert rc == 0, msg
    text, _ = random_opb(rng, 30, 60)
    lines = [l for l in text.splitlines()[1:]]
    good = []
    for l in lines:
        try:
            read_opb(l)
            good.append(l)
        except ValueError:
            pass
    rc, msg = B.cls_problem_check(read_opb("\n".join(good)))
    assert rc == 0, msg


def test_solver_format_detection(tmp_path):
    """The command-line solver reads a file as DIMACS when its first
    non-comment line is the problem line, as OPB otherwise."""
    from paper_2606_06656_b300.solve import read_any
    f = tmp_path / "a.cnf"
    f.write_text("c comment\n\np cnf 3 1\n1 -2 3 0\n")
    inst, kind = read_any(str(f))
    assert kind == "dimacs" and inst.m == 1
    g = tmp_path / "b.opb"
    g.write_text("* #variable= 3 #constraint= 1\n+1 x1 +1 x2 +1 x3 >= 2 ;\n")
    inst, kind = read_any(str(g))
    assert kind == "opb" and inst.m == 1 and inst.k.tolist() == [2]
