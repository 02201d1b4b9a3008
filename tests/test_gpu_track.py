"""Per-restart tracking, refill and histogram kernels against the oracle
(bit-exact), on seeded synthetic counts, states and points."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cls as ocls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2606_06656_b300 import Problem
    return Problem


def small_inst(seed=0, n=70, fixed=False):
    inst = W.random_ksat(n=n, m=300, seed=seed)
    if fixed:
        inst = W.partial_assignment(W.mixed_pb(n=n, n_or=200, n_xor=20, n_card=4,
                                               card_len=(10, 30), seed=seed), 0.3, seed=seed)
    return inst


@pytest.mark.parametrize("R", [1, 33, 300])
def test_track_step_matches_oracle(P, R):
    from paper_2606_06656_b300 import binding as B
    inst = small_inst()
    p = P(inst)
    rng = np.random.default_rng(R)
    trk = torch.empty((4, R), dtype=torch.int32, device="cuda")
    B.cls_track_reset(p.handle, R, trk)
    S = ocls.track_reset(R)
    for step in range(12):
        nsat = rng.integers(inst.m - 6, inst.m + 1, R).astype(np.int32)
        B.cls_track_step(p.handle, R, torch.from_numpy(nsat).cuda(), step, trk)
        S = ocls.track_step(S, nsat, step, inst.m)
    torch.cuda.synchronize()
    assert np.array_equal(trk.cpu().numpy(), S.astype(np.int32))


@pytest.mark.parametrize("R,fixed", [(5, False), (257, False), (64, True)])
def test_refill_matches_oracle(P, R, fixed):
    from paper_2606_06656_b300 import binding as B
    inst = small_inst(seed=1, fixed=fixed)
    p = P(inst)
    rng = np.random.default_rng(7)
    X = W.uniform_points(inst.n, R, seed=2)
    if fixed:
        f = inst.fixed.astype(bool)
        X[f] = inst.fixed_val[f][:, None]
    S = ocls.track_reset(R)
    S[0] = rng.integers(0, inst.m, R)
    S[1] = rng.integers(0, 50, R)
    S[2] = rng.integers(0, 40, R)
    S[3] = np.where(rng.random(R) < 0.3, rng.integers(0, 50, R), -1)
    x = torch.from_numpy(X.copy()).cuda()
    trk = torch.from_numpy(S.astype(np.int32)).cuda()
    cnt = torch.full((1,), 3, dtype=torch.int32, device="cuda")
    B.cls_refill(p.handle, R, x, trk, 20, 99, 0, 4, cnt)
    X1, S1, c1 = ocls.refill(X, S, 20, 99, 4, fixed=inst.fixed, fixed_val=inst.fixed_val)
    torch.cuda.synchronize()
    assert np.array_equal(x.cpu().numpy(), X1)          # bit-exact points
    assert np.array_equal(trk.cpu().numpy(), S1.astype(np.int32))
    assert int(cnt.item()) == 3 + c1


def test_refill_redraws_every_due_restart(P):
    """A restart refilled at generation g gets values that differ from the
    first draw and lie in [-1, 1); R = 0 and bad arguments."""
    from paper_2606_06656_b300 import binding as B
    from paper_2606_06656_b300._lib import ClsError
    inst = small_inst(seed=2)
    p = P(inst)
    R = 40
    x = p.init_uniform(R, seed=5)
    x0 = x.clone()
    trk = torch.empty((4, R), dtype=torch.int32, device="cuda")
    B.cls_track_reset(p.handle, R, trk)
    trk[2] = 100
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    B.cls_refill(p.handle, R, x, trk, 1, 5, 0, 1, cnt)
    torch.cuda.synchronize()
    assert int(cnt.item()) == R
    assert bool((x != x0).all()) and bool((x >= -1).all()) and bool((x < 1).all())
    B.cls_refill(p.handle, 0, None, None, 1, 5, 0, 1, None)
    with pytest.raises(ClsError):
        B.cls_refill(p.handle, R, x, trk, 0, 5, 0, 1, cnt)        # patience 0
    with pytest.raises(ClsError):
        B.cls_refill(p.handle, R, x, trk, 3, 5, 0, 0, cnt)        # generation 0
    with pytest.raises(ClsError):
        B.cls_track_step(p.handle, R, None, 0, trk)


@pytest.mark.parametrize("R", [1, 100, 1000])
def test_unsat_histogram_matches_oracle(P, R):
    from paper_2606_06656_b300 import binding as B
    inst = small_inst(seed=3)
    p = P(inst)
    rng = np.random.default_rng(R)
    nsat = rng.integers(0, inst.m + 1, R).astype(np.int32)
    hist = torch.full((inst.m + 1,), 7, dtype=torch.int32, device="cuda")
    B.cls_unsat_histogram(p.handle, R, torch.from_numpy(nsat).cuda(), hist)
    torch.cuda.synchronize()
    assert np.array_equal(hist.cpu().numpy(), ocls.unsat_histogram(nsat, inst.m).astype(np.int32))


@pytest.mark.parametrize("n,R", [(70, 1), (70, 33), (200, 300), (4500, 64)])
def test_movement_and_convergence_match_oracle(P, n, R):
    """Bit-exact: movement of a real step (clamped coordinates, pinned ones
    that never move) and of synthetic pairs with +-0, equal values and
    extremes; the convergence record over several steps.  n = 4500 spans
    several 64-variable chunks per restart."""
    from paper_2606_06656_b300 import binding as B
    inst = W.random_ksat(n=n, m=4 * n, seed=n)
    p = P(inst)
    x = p.init_uniform(R, seed=3)
    md = torch.empty(R, dtype=torch.float32, device="cuda")
    conv = torch.full((R,), -1, dtype=torch.int32, device="cuda")
    oconv = -np.ones(R, np.int64)
    for step in range(4):
        xp = x.clone()
        p.step(x, 0.3 if step < 2 else 1e-6, 1)
        B.cls_movement(p.handle, R, xp, x, md)
        B.cls_track_converged(p.handle, R, md, 1e-4, step, conv)
        torch.cuda.synchronize()
        want = ocls.movement(xp.cpu().numpy(), x.cpu().numpy())
        assert np.array_equal(md.cpu().numpy(), want)
        oconv = ocls.track_converged(oconv, want, 1e-4, step)
        assert np.array_equal(conv.cpu().numpy(), oconv)
    rng = np.random.default_rng(R)
    A = rng.uniform(-1, 1, (n, R)).astype(np.float32)
    Bm = A.copy()
    Bm[rng.random((n, R)) < 0.3] *= -1
    Bm[0] = np.where(A[0] == 0, np.float32(-0.0), A[0])
    Bm[-1, :] = np.float32(1.0)
    B.cls_movement(p.handle, R, torch.from_numpy(A).cuda(), torch.from_numpy(Bm).cuda(), md)
    torch.cuda.synchronize()
    assert np.array_equal(md.cpu().numpy(), ocls.movement(A, Bm))
