"""Adaptive constraint weighting on the CUDA path vs the oracle.

cls_constraint_stats after cls_eval: gnorm within 1e-4 relative per
constraint plus an FP32 floor (the partials it reads carry the FE kernels'
absolute error, a few L*u per DFT literal), unsat bit-exact at the same
rounded point.  cls_reweight: the new weights within 5e-4 relative (the
update is smooth in the statistics; each ratio carries two statistics'
errors).  cls_set_weights: objective, gradient and wsat as with weights
given at creation.  Graphs recorded with all weights 1 are refused after a
weight change."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cls as ocls

pytestmark = pytest.mark.gpu

TYPES = [W.TYPE_OR, W.TYPE_XOR, W.TYPE_CARD_GE, W.TYPE_CARD_LE, W.TYPE_NAE, W.TYPE_EO,
         W.TYPE_EK, W.TYPE_AMO, W.TYPE_SPECTRUM]


def gpu_stats(p, X):
    from paper_2606_06656_b300 import binding as B
    R = X.shape[1]
    x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
    p.eval(x, obj=False, grad=True)
    nsat, _, bits = p.round_score(x)
    # round_score overwrites nothing the statistics read (partials stay)
    g = torch.empty(p.m, dtype=torch.float64, device="cuda")
    u = torch.empty(p.m, dtype=torch.int32, device="cuda")
    B.cls_constraint_stats(p.handle, R, bits, p.workspace(R), g, u)
    torch.cuda.synchronize()
    return g.cpu().numpy(), u.cpu().numpy()


def floor_of(inst, R):
    """Per constraint: R * sqrt(L) * 4 L u (FP32 partial floor per literal)."""
    L = np.diff(inst.offsets).astype(np.float64)
    return R * np.sqrt(L) * 4.0 * L * 2.0 ** -24


@pytest.mark.parametrize("R", [1, 33, 100])
@pytest.mark.parametrize("kind", ["uniform", "mixed"])
def test_stats_match_oracle(R, kind):
    from paper_2606_06656_b300 import Problem
    rng = np.random.default_rng(R)
    inst = W.random_constraint_set(rng, 150, 260, TYPES, (1, 90), weights="random")
    X = (W.uniform_points if kind == "uniform" else W.mixed_points)(inst.n, R, seed=R)
    p = Problem(inst)
    g, u = gpu_stats(p, X)
    og, ou, _ = ocls.constraint_stats(inst, X)
    assert np.array_equal(u, ou)
    tol = 1e-4 * og + floor_of(inst, R) + 1e-30
    bad = np.nonzero(np.abs(g - og) > tol)[0]
    assert len(bad) == 0, (bad[:5], g[bad[:5]], og[bad[:5]])


def test_stats_long_constraints_and_weights_cancel():
    """Constraints up to 700 literals (series, corner and dense DFT passes);
    gnorm does not depend on the weights."""
    from paper_2606_06656_b300 import Problem
    rng = np.random.default_rng(9)
    inst = W.random_constraint_set(rng, 800, 40, TYPES, (60, 700), weights="random")
    X = W.uniform_points(inst.n, 70, seed=2)
    g, u = gpu_stats(Problem(inst), X)
    og, ou, _ = ocls.constraint_stats(inst, X)
    assert np.array_equal(u, ou)
    assert (np.abs(g - og) <= 1e-4 * og + floor_of(inst, 70) + 1e-30).all()
    ones = W.Instance(**{**inst.__dict__})
    ones.weight = np.ones(inst.m, np.float32)
    g1, _ = gpu_stats(Problem(ones), X)
    assert np.allclose(g1, g, rtol=1e-5, atol=1e-30)


@pytest.mark.parametrize("simplify", [False, True])
def test_stats_with_pinned_variables(simplify):
    from paper_2606_06656_b300 import Problem
    inst = W.partial_assignment(W.mixed_pb(n=600, n_or=1500, n_xor=150, n_card=40,
                                           card_len=(10, 200), seed=4), 0.5)
    X = ocls.init_uniform(inst.n, 45, 5, fixed=inst.fixed, fixed_val=inst.fixed_val)
    g, u = gpu_stats(Problem(inst, simplify_fixed=simplify), X)
    og, ou, _ = ocls.constraint_stats(inst, X, free_only=simplify)
    assert np.array_equal(u, ou)
    assert (np.abs(g - og) <= 1e-4 * og + floor_of(inst, 45) + 1e-30).all()


def test_reweight_matches_oracle_and_takes_effect():
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    rng = np.random.default_rng(4)
    inst = W.random_constraint_set(rng, 200, 400, TYPES, (1, 80), weights="random")
    R = 64
    X = W.uniform_points(inst.n, R, seed=8)
    p = Problem(inst)
    x = torch.from_numpy(X).cuda()
    p.eval(x, obj=False, grad=True)
    nsat, _, bits = p.round_score(x)
    g = torch.empty(p.m, dtype=torch.float64, device="cuda")
    u = torch.empty(p.m, dtype=torch.int32, device="cuda")
    w = torch.empty(p.m, dtype=torch.float32, device="cuda")
    B.cls_constraint_stats(p.handle, R, bits, p.workspace(R), g, u)
    B.cls_reweight(p.handle, R, g, u, 0.7, 4.0, 5.0, w)
    torch.cuda.synchronize()
    og, ou, has = ocls.constraint_stats(inst, X)
    ow = ocls.reweight(inst.weight, og, ou, has, R, 0.7, 4.0, 5.0)
    assert np.allclose(w.cpu().numpy(), ow, rtol=5e-4, atol=0)
    assert (ow != inst.weight).any()
    # the problem now evaluates with the new weights (the oracle's own)
    new = W.Instance(**{**inst.__dict__})
    new.weight = ow
    X2 = W.uniform_points(inst.n, 40, seed=11)
    x2 = torch.from_numpy(X2).cuda()
    obj, grad, _ = p.eval(x2)
    ns, wsat, _ = p.round_score(x2)
    oobj, ograd, _ = ocls.objective_grad(new, X2.astype(np.float64))
    onsat, owsat, _ = ocls.score(new, X2)
    # the weights differ from the oracle's by <= 5e-4 relative, so the
    # objective by <= 5e-4 sum |w| (|FE| <= 1) on top of the FE tolerance,
    # and the gradient by <= 5e-4 sum_c w_c ||grad FE_c|| per restart
    wsum = float(np.abs(ow).sum())
    assert np.max(np.abs(obj.cpu().numpy() - oobj)) <= 6e-4 * wsum
    pull = np.array([float(ow @ ocls.constraint_stats(new, X2[:, r:r + 1])[0])
                     for r in range(X2.shape[1])])
    gn = np.linalg.norm(ograd, axis=0)
    assert (np.linalg.norm(grad.cpu().numpy() - ograd, axis=0)
            <= 1e-4 * gn + 5e-4 * pull + 1e-30).all()
    assert np.array_equal(ns.cpu().numpy(), onsat)
    assert np.allclose(wsat.cpu().numpy(), owsat, rtol=1e-3)
    # retuning reads the device weights back: results do not change
    before = p.eval(x2)[0].cpu().numpy()
    B.cls_tuning_set(p.handle, B.cls_tuning_get(p.handle))
    after = p.eval(x2)[0].cpu().numpy()
    assert np.array_equal(before, after)


def test_set_weights_equals_weights_at_creation():
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    rng = np.random.default_rng(6)
    inst = W.random_constraint_set(rng, 120, 300, TYPES, (1, 40), weights="ones")
    wts = rng.uniform(0.2, 3.0, inst.m).astype(np.float32)
    wts[::7] = 0.0
    other = W.Instance(**{**inst.__dict__})
    other.weight = wts
    X = W.uniform_points(inst.n, 50, seed=3)
    x = torch.from_numpy(X).cuda()
    p = Problem(inst)
    B.cls_set_weights(p.handle, torch.from_numpy(wts).cuda())
    q = Problem(other)
    a, b = p.eval(x), q.eval(x)
    sa, sb = p.round_score(x), q.round_score(x)
    torch.cuda.synchronize()
    assert np.array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
    assert np.array_equal(a[1].cpu().numpy(), b[1].cpu().numpy())
    assert np.array_equal(sa[1].cpu().numpy(), sb[1].cpu().numpy())


def test_graph_recorded_with_unit_weights_is_refused_after_a_change():
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    from paper_2606_06656_b300._lib import ClsError
    inst = W.random_ksat(n=60, m=250)
    R = 64
    p = Problem(inst)
    x = p.init_uniform(R, 1)
    ws = p.workspace(R)
    nsat = torch.empty(R, dtype=torch.int32, device="cuda")
    wsat = torch.empty(R, dtype=torch.float64, device="cuda")
    bits = torch.empty((inst.n, 2), dtype=torch.int32, device="cuda")
    g = B.cls_graph_create(p.handle, R, x, 0.1, 2, bits, nsat, wsat, ws)
    B.cls_graph_launch(g)
    B.cls_set_weights(p.handle, torch.full((inst.m,), 2.0, device="cuda"))
    with pytest.raises(ClsError):
        B.cls_graph_launch(g)
    B.cls_graph_destroy(g)
    g = B.cls_graph_create(p.handle, R, x, 0.1, 2, bits, nsat, wsat, ws)
    B.cls_graph_launch(g)
    torch.cuda.synchronize()
    assert np.allclose(wsat.cpu().numpy(), 2.0 * nsat.cpu().numpy())
    B.cls_graph_destroy(g)


def test_weighting_argument_checks_and_empty_set():
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300 import binding as B
    from paper_2606_06656_b300._lib import ClsError
    inst = W.random_ksat(n=40, m=100)
    p = Problem(inst)
    R = 40
    x = p.init_uniform(R, 2)
    p.eval(x, obj=False)
    _, _, bits = p.round_score(x)
    g, u = p.constraint_stats(bits, R)
    w = torch.empty(p.m, dtype=torch.float32, device="cuda")
    for eta, kappa, w_max in [(-1.0, 4.0, 10.0), (1.0, 0.0, 10.0), (1.0, 4.0, float("inf")),
                              (float("nan"), 4.0, 10.0), (1.0, 4.0, 0.0)]:
        with pytest.raises(ClsError):
            B.cls_reweight(p.handle, R, g, u, eta, kappa, w_max, w)
    with pytest.raises(ClsError):
        B.cls_reweight(p.handle, 0, g, u, 1.0, 4.0, 10.0, w)
    with pytest.raises(ClsError):
        B.cls_constraint_stats(p.handle, 0, bits, p.workspace(R), g, u)
    with pytest.raises(ClsError):                      # workspace of another R
        B.cls_constraint_stats(p.handle, 4 * R, bits, p.workspace(R), g, u)
    with pytest.raises(ValueError):
        p.set_weights(torch.ones(p.m + 1, device="cuda"))
    # eta = 0 leaves the weights (and the unit-weight results) alone
    w1 = p.reweight(g, u, R, 0.0)
    assert torch.equal(w1, torch.ones_like(w1))
    # a constraint set without constraints: nothing to do, no error
    empty = W.build(5, [])
    q = Problem(empty)
    xq = q.init_uniform(8, 1)
    q.eval(xq, obj=False)
    _, _, bq = q.round_score(xq)
    g0, u0 = q.constraint_stats(bq, 8)
    assert g0.numel() == 0 and u0.numel() == 0
    q.reweight(g0, u0, 8, 1.0)
