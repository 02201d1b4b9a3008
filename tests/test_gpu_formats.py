"""Constraint sets read from DIMACS CNF and OPB text, run through the CUDA
path and compared with the FP64 oracle on the same parsed set: FE within
1e-4 per constraint, gradient within 1e-4 of its norm per restart, counts
bit-exact (the tolerances of the parity suite).  The texts are generated
here from a seed: a random 3-SAT formula, and linear constraints with +1 / -1
coefficients long enough to reach the DFT, power-sum and corner passes."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cls as ocls
from paper_2606_06656_b300.formats import read_dimacs, read_opb

pytestmark = pytest.mark.gpu


def cnf_text(rng, n, m):
    lines = [f"p cnf {n} {m}"]
    for _ in range(m):
        v = rng.choice(n, size=3, replace=False) + 1
        s = rng.choice([-1, 1], size=3)
        lines.append(" ".join(str(int(a * b)) for a, b in zip(v, s)) + " 0")
    return "\n".join(lines) + "\n"


def opb_text(rng, n, m, lens):
    lines = [f"* #variable= {n} #constraint= {m}"]
    for _ in range(m):
        L = int(rng.integers(*lens))
        v = rng.choice(n, size=L, replace=False) + 1
        a = rng.choice([-1, 1], size=L)
        neg = rng.random(L) < 0.3
        rel = str(rng.choice([">=", "<=", "="]))
        # the right-hand side leaves the constraint satisfiable and not trivial
        lo, hi = int((a < 0).sum()) * -1, int((a > 0).sum())
        k = int(rng.integers(lo + 1, hi))
        body = " ".join(f"{int(c):+d} {'~' if g else ''}x{int(x)}" for c, g, x in zip(a, neg, v))
        lines.append(f"{body} {rel} {k} ;")
    return "\n".join(lines) + "\n"


def check(inst, X):
    from paper_2606_06656_b300 import Problem
    p = Problem(inst)
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    obj, grad, fe = p.eval(x, obj=True, grad=True, fe_con=True)
    nsat, _, bits = p.round_score(x)
    torch.cuda.synchronize()
    oobj, ograd, ofe = ocls.objective_grad(inst, X.astype(np.float64))
    assert np.max(np.abs(fe.cpu().numpy() - ofe)) <= 1e-4
    g = grad.cpu().numpy()
    assert (np.linalg.norm(g - ograd, axis=0)
            <= 1e-4 * np.linalg.norm(ograd, axis=0) + 1e-30).all()
    assert np.max(np.abs(obj.cpu().numpy() - oobj)) <= 1e-4 * max(1.0, inst.m)
    onsat, _, _ = ocls.score(inst, X)
    assert np.array_equal(nsat.cpu().numpy(), onsat)


def test_dimacs_3sat_parity():
    rng = np.random.default_rng(21)
    inst = read_dimacs(cnf_text(rng, 400, 1700))
    assert inst.m == 1700
    check(inst, W.uniform_points(inst.n, 77, seed=4))


@pytest.mark.parametrize("lens", [(2, 30), (30, 140), (140, 400)])
def test_opb_cardinality_parity(lens):
    rng = np.random.default_rng(lens[0])
    inst = read_opb(opb_text(rng, 500, 60, lens))
    assert inst.m + inst.dropped == 60
    check(inst, W.uniform_points(inst.n, 45, seed=5))


def test_solve_cli_finds_a_model(tmp_path, capsys):
    """The command-line solver on a planted 3-SAT file (clause/variable
    ratio 3, well below the threshold): it reports SATISFIABLE and the
    printed model satisfies every clause of the file."""
    from paper_2606_06656_b300.solve import main
    rng = np.random.default_rng(8)
    n, m = 200, 600
    plant = rng.random(n) < 0.5
    clauses = []
    while len(clauses) < m:
        v = rng.choice(n, size=3, replace=False)
        s = rng.choice([-1, 1], size=3)
        if any(plant[a] == (b > 0) for a, b in zip(v, s)):
            clauses.append([int((a + 1) * b) for a, b in zip(v, s)])
    f = tmp_path / "planted.cnf"
    f.write_text(f"p cnf {n} {m}\n" + "".join(" ".join(map(str, c)) + " 0\n" for c in clauses))
    rc = main([str(f), "--restarts", "256", "--steps", "500"])
    out = capsys.readouterr().out
    assert rc == 10 and "s SATISFIABLE" in out, out
    vline = [l for l in out.splitlines() if l.startswith("v ")][0]
    lits = [int(t) for t in vline.split()[1:]]
    assert lits[-1] == 0 and len(lits) == n + 1
    true = {abs(l) for l in lits[:-1] if l > 0}
    for c in clauses:
        assert any((abs(l) in true) == (l > 0) for l in c), c


def test_solve_cli_opb_with_weighting(tmp_path, capsys):
    """The solver with adaptive weighting on a planted OPB file (clauses
    written as linear constraints, at-most and exactly constraints that the
    plant satisfies): SATISFIABLE, and the printed model satisfies every
    linear constraint of the file, evaluated here directly."""
    from paper_2606_06656_b300.solve import main
    rng = np.random.default_rng(12)
    n = 120
    plant = rng.random(n) < 0.5
    lines, cons = [f"* #variable= {n} #constraint= 300"], []
    while len(cons) < 300:
        L = int(rng.integers(3, 9))
        v = rng.choice(n, size=L, replace=False)
        a = rng.choice([-1, 1], size=L)
        lhs = int(sum(c * int(plant[x]) for c, x in zip(a, v)))
        rel = str(rng.choice([">=", "<=", "="]))
        k = lhs - int(rng.integers(0, 2)) if rel == ">=" else (
            lhs + int(rng.integers(0, 2)) if rel == "<=" else lhs)
        lo, hi = int((a < 0).sum()) * -1, int((a > 0).sum())
        if (rel == ">=" and k <= lo) or (rel == "<=" and k >= hi):
            continue                                   # always true: skip
        cons.append((a, v, rel, k))
        lines.append(" ".join(f"{int(c):+d} x{int(x) + 1}" for c, x in zip(a, v))
                     + f" {rel} {k} ;")
    f = tmp_path / "planted.opb"
    f.write_text("\n".join(lines) + "\n")
    rc = main([str(f), "--restarts", "512", "--steps", "1500", "--reweight", "1.0"])
    out = capsys.readouterr().out
    assert rc == 10 and "s SATISFIABLE" in out, out
    vline = [l for l in out.splitlines() if l.startswith("v ")][0]
    val = {}
    for tok in vline.split()[1:]:
        val[int(tok.lstrip("-x"))] = not tok.startswith("-")
    for a, v, rel, k in cons:
        lhs = sum(int(c) * int(val[int(x) + 1]) for c, x in zip(a, v))
        assert {">=": lhs >= k, "<=": lhs <= k, "=": lhs == k}[rel]
