"""Oracle of the adaptive constraint weighting (Sec. 3.1), pinned on CPU.

The statistics are plain definitions, so they are pinned to closed forms
written out here: the clause (OR) and parity (XOR) expansions of Appendix A,
whose partials are products of the other literals' factors, give the
gradient norms directly; the violation counts are pinned to a direct count
over explicit corner points and to the invariant sum_c unsat = sum_r
(m - nsat).  The update rule is pinned to a small example worked by hand and
to its special cases (eta = 0, no violations, the w_max cap)."""
import numpy as np
import pytest

import workloads as W
from oracle import cls as O


def or_partials(Y):
    """OR over literals y (True = -1): FE = 2 prod (1+y)/2 - 1, so
    dFE/dy_i = prod_{j != i} (1+y_j)/2."""
    a = (1.0 + Y) / 2.0
    return np.stack([np.prod(np.delete(a, i, axis=0), axis=0) for i in range(len(Y))])


def xor_partials(Y):
    """XOR (t odd): FE = -prod y, so dFE/dy_i = -prod_{j != i} y_j."""
    return np.stack([-np.prod(np.delete(Y, i, axis=0), axis=0) for i in range(len(Y))])


@pytest.mark.parametrize("L", [1, 2, 3, 7, 12])
def test_gnorm_closed_forms(L):
    rng = np.random.default_rng(L)
    n, R = 3 * L, 9
    rows, parts = [], []
    for ct in (W.TYPE_OR, W.TYPE_XOR):
        v = rng.choice(n, size=L, replace=False).astype(np.int32)
        s = np.where(rng.random(L) < 0.5, -1, 1).astype(np.int8)
        rows.append((ct, 0, v, s))
    inst = W.build(n, rows, weights=np.array([2.5, 0.5], np.float32))
    X = W.uniform_points(n, R, seed=L)
    gnorm, unsat, has_fe = O.constraint_stats(inst, X)
    for c, (ct, _, v, s) in enumerate(rows):
        Y = s[:, None].astype(np.float64) * X[v].astype(np.float64)
        G = or_partials(Y) if ct == W.TYPE_OR else xor_partials(Y)
        want = np.sqrt((G ** 2).sum(axis=0)).sum()
        assert np.isclose(gnorm[c], want, rtol=1e-12, atol=1e-300)
    assert has_fe.all()


def test_unsat_counts_direct():
    """Corners drawn at random; the violation count of every constraint
    counted here from the truth values and each type's predicate."""
    rng = np.random.default_rng(2)
    types = [W.TYPE_OR, W.TYPE_XOR, W.TYPE_CARD_GE, W.TYPE_CARD_LE, W.TYPE_NAE,
             W.TYPE_EO, W.TYPE_EK, W.TYPE_AMO]
    inst = W.random_constraint_set(rng, 30, 80, types, (1, 12), weights="random")
    X = W.corner_points(inst.n, 50, seed=3)
    _, unsat, _ = O.constraint_stats(inst, X)
    true = X < 0
    for c in range(inst.m):
        a, b = inst.offsets[c], inst.offsets[c + 1]
        lt = true[inst.lit_var[a:b]] ^ (inst.lit_sign[a:b] < 0)[:, None]
        t = lt.sum(axis=0)
        L, k, ct = b - a, int(inst.k[c]), int(inst.ctype[c])
        holds = {W.TYPE_OR: t >= 1, W.TYPE_XOR: t % 2 == 1, W.TYPE_CARD_GE: t >= k,
                 W.TYPE_CARD_LE: t <= k, W.TYPE_NAE: (t > 0) & (t < L), W.TYPE_EO: t == 1,
                 W.TYPE_EK: t == k, W.TYPE_AMO: t <= 1}[ct]
        assert unsat[c] == int((~holds).sum()), c
    nsat, _, _ = O.score(inst, X)
    assert unsat.sum() == (inst.m - nsat).sum()


def test_constant_and_zero_weight_constraints_have_no_norm():
    """A constraint that always holds (CARD_GE 0) has a constant expansion;
    a weight of 0 hides the partials; with pinned variables folded in, a
    clause with a true pinned literal is constant too."""
    v = np.arange(4, dtype=np.int32)
    s = np.ones(4, np.int8)
    inst = W.build(6, [(W.TYPE_CARD_GE, 0, v, s), (W.TYPE_OR, 0, v, s),
                       (W.TYPE_OR, 0, np.array([3, 4, 5], np.int32), np.ones(3, np.int8))],
                   weights=np.array([1.0, 0.0, 1.0], np.float32))
    X = W.uniform_points(6, 5, seed=1)
    g, _, has_fe = O.constraint_stats(inst, X)
    assert g[0] == 0.0 and not has_fe[0]
    assert g[1] == 0.0 and has_fe[1]
    assert g[2] > 0.0 and has_fe[2]
    pinned = W.Instance(**{**inst.__dict__})
    pinned.fixed = np.array([0, 0, 0, 1, 0, 0], np.uint8)
    pinned.fixed_val = np.array([0, 0, 0, -1, 0, 0], np.float32)     # x3 True
    X[3] = -1.0
    g2, _, has2 = O.constraint_stats(pinned, X, free_only=True)
    assert not has2[2] and g2[2] == 0.0
    # without folding, the pinned literal's partial counts
    g3, _, has3 = O.constraint_stats(pinned, X, free_only=False)
    assert has3[2] and g3[2] > 0.0


def test_reweight_worked_example():
    """R = 4; g = gnorm/R = (1, 0.1, 0, 2) with the last constraint without
    FE work, so gbar = (1 + 0.1 + 0)/3 = 0.3666...; kappa = 4:
      c0: 4 > gbar -> rho = gbar/1 = 0.3666...;  u = 2/4
      c1: 0.4 > gbar -> rho = gbar/0.1 = 3.666...; u = 4/4
      c2: 0 <= gbar -> rho = 4;  u = 1/4
      c3: 8 > gbar -> rho = gbar/2;  u = 0
    eta = 1, w = (1, 1, 2, 1), w_max = 3:
      (1 + 0.5*0.36667, min(3, 1 + 3.6667), 2*(1 + 0.25*4), 1) = (1.18333, 3, 4 -> 3, 1)."""
    w = np.array([1, 1, 2, 1], np.float32)
    gnorm = np.array([4.0, 0.4, 0.0, 8.0])
    unsat = np.array([2, 4, 1, 0])
    has_fe = np.array([True, True, True, False])
    out = O.reweight(w, gnorm, unsat, has_fe, 4, 1.0, 4.0, 3.0)
    gbar = 1.1 / 3
    assert np.allclose(out, [1 + 0.5 * gbar, 3.0, 3.0, 1.0], rtol=1e-7)
    # without the cap
    out = O.reweight(w, gnorm, unsat, has_fe, 4, 1.0, 4.0, 100.0)
    assert np.allclose(out, [1 + 0.5 * gbar, 1 + gbar / 0.1, 4.0, 1.0], rtol=1e-7)
    # eta = 0 and no violations leave the weights alone
    assert np.array_equal(O.reweight(w, gnorm, unsat, has_fe, 4, 0.0, 4.0, 100.0), w)
    assert np.array_equal(O.reweight(w, gnorm, 0 * unsat, has_fe, 4, 2.0, 4.0, 100.0), w)


def test_reweight_on_ramsey_boosts_the_violated_balance_constraints():
    """At corners of the redundant Ramsey encoding where every edge
    constraint holds and some balance constraints fail, only the failing
    balance constraints gain weight."""
    inst = W.ramsey_balanced(16, 3, redundant=True)
    base = inst.plant.astype(np.float32)
    C = 3
    cols = []
    for e in (0, 30, 77):
        x = base.copy()
        c = int(np.argmax(base[e * C:(e + 1) * C] < 0))
        x[e * C + c], x[e * C + (c + 1) % C] = 1.0, -1.0
        cols.append(x)
    X = np.stack(cols, axis=1) * np.float32(0.999)   # just inside the corners
    g, u, has = O.constraint_stats(inst, X)
    wn = O.reweight(inst.weight, g, u, has, X.shape[1], 0.5, 4.0, 10.0)
    changed = np.nonzero(wn != inst.weight)[0]
    assert len(changed) > 0
    assert ((changed >= 120) & (changed < 168)).all()      # balance rows only
    assert (u[changed] > 0).all()
