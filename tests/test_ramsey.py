"""Ramsey balanced-colouring instances (Sec. 3.1), CPU pins.

The generator's structure is checked by direct counting here (edges,
colour degrees of the plant), independently of the oracle; then the
oracle's satisfied counts at the plant and at single-edge changes of it
are checked against what the combinatorics fixes; and the paper's remark
that the redundant encoding equals 2*EO - 1 on the edge constraints (so it
doubles their gradient) is checked at the objective level: the redundant
instance's objective and gradient exceed the plain one's by exactly the
EO part's (minus 1 per edge)."""
import numpy as np
import pytest

import workloads as W
from oracle import cls as O


def colours_of(inst, x):
    """(E, C) bool: edge e has colour i at the corner x (True = -1)."""
    V, C = inst.meta["V"], inst.meta["C"]
    E = V * (V - 1) // 2
    return (np.asarray(x) < 0).reshape(E, C)


@pytest.mark.parametrize("V,C", [(16, 3), (16, 5), (10, 3), (8, 7)])
def test_generator_structure_and_plant(V, C):
    for red in (False, True):
        inst = W.ramsey_balanced(V, C, redundant=red)
        E = V * (V - 1) // 2
        assert inst.n == E * C
        assert inst.m == E + V * C + (2 * E if red else 0)
        L = np.diff(inst.offsets)
        assert (L[:E] == C).all() and (L[E:E + V * C] == V - 1).all()
        assert (inst.ctype[:E] == W.TYPE_EO).all()
        assert (inst.ctype[E:E + V * C] == W.TYPE_CARD_GE).all()
        assert (inst.k[E:E + V * C] == -(-(V - 1) // C)).all()
        # every variable is in one EO and in two balance constraints
        assert np.bincount(inst.lit_var, minlength=inst.n).tolist() == \
            [3 + (2 if red else 0)] * inst.n
        # the plant, counted directly: one colour per edge, (V-1)/C edges of
        # each colour at every vertex
        col = colours_of(inst, inst.plant)
        assert (col.sum(axis=1) == 1).all()
        edges = [(u, v) for u in range(V) for v in range(u + 1, V)]
        deg = np.zeros((V, C), dtype=int)
        for e, (u, v) in enumerate(edges):
            c = int(np.argmax(col[e]))
            deg[u, c] += 1
            deg[v, c] += 1
        assert (deg == (V - 1) // C).all()
        nsat, _, _ = O.score(inst, inst.plant.astype(np.float32)[:, None])
        assert nsat[0] == inst.m


def test_no_plant_when_unbalanceable():
    assert W.ramsey_balanced(16, 4).plant is None     # 4 does not divide 15
    assert W.ramsey_balanced(9, 4).plant is None      # odd V: no perfect matchings
    inst = W.ramsey_balanced(16, 4)
    assert (inst.k[120:] == 4).all()                  # ceil(15/4): 16 > 15 edges needed


@pytest.mark.parametrize("red", [False, True])
def test_single_edge_changes(red):
    """Recolouring one edge (still one colour): its two endpoints each lose
    one edge of the old colour (degree 4 < 5) -- exactly two balance
    constraints fail.  Giving an edge a second colour: its EO fails (and, in
    the redundant encoding, the at-most-one part too); balance still holds.
    Removing an edge's colour: EO fails (and the OR part), and both
    endpoints miss one edge of that colour."""
    inst = W.ramsey_balanced(16, 3, redundant=red)
    m, C = inst.m, 3
    base = inst.plant.astype(np.float32)
    col = colours_of(inst, base)
    cases = []
    for e in (0, 17, 119):
        c = int(np.argmax(col[e]))
        x = base.copy()
        x[e * C + c], x[e * C + (c + 1) % C] = 1.0, -1.0
        cases.append((x, m - 2))
        x = base.copy()
        x[e * C + (c + 1) % C] = -1.0
        cases.append((x, m - (2 if red else 1)))
        x = base.copy()
        x[e * C + c] = 1.0
        cases.append((x, m - (4 if red else 3)))
    X = np.stack([x for x, _ in cases], axis=1)
    nsat, _, _ = O.score(inst, X)
    assert nsat.tolist() == [w for _, w in cases]


def test_redundant_encoding_doubles_the_edge_gradient():
    """Sec. 3.1: CARD>=2(not x) + OR(x) = EO(x) - 1 on three literals, so the
    redundant instance's objective is the plain one's plus sum_e (FE_EO,e - 1)
    and its gradient the plain one's plus the EO part's gradient."""
    plain = W.ramsey_balanced(16, 3)
    red = W.ramsey_balanced(16, 3, redundant=True)
    E = 120
    eo_only = W.build(plain.n, [(W.TYPE_EO, 0, plain.lit_var[3 * e:3 * e + 3],
                                 plain.lit_sign[3 * e:3 * e + 3]) for e in range(E)])
    X = W.uniform_points(plain.n, 6, seed=3).astype(np.float64)
    op, gp, _ = O.objective_grad(plain, X)
    orr, gr, _ = O.objective_grad(red, X)
    oe, ge, _ = O.objective_grad(eo_only, X)
    assert np.allclose(orr, op + oe - E, atol=1e-10)
    assert np.allclose(gr, gp + ge, atol=1e-12)
    # the edge constraints' own gradient doubles
    red_edges = W.build(red.n, [(int(red.ctype[c]), int(red.k[c]),
                                 red.lit_var[red.offsets[c]:red.offsets[c + 1]],
                                 red.lit_sign[red.offsets[c]:red.offsets[c + 1]])
                                for c in list(range(E)) + list(range(E + 48, red.m))])
    _, gre, _ = O.objective_grad(red_edges, X)
    assert np.allclose(gre, 2 * ge, atol=1e-12)
