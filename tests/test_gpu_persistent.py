"""The step loop as one persistent cooperative launch (cls_step_persistent)
against the multi-launch step (cls_step), and the bounded grid barrier.

Both paths run the same per-item arithmetic (Eq. 1's expansion and gradient
for short closed forms, the projected step, the rounding, the counts) and sum
in the same orders, so x, the bitsets and the counts agree bit for bit; one
step is tied to the oracle through cls_step's own parity tests.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cls as ocls

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_2606_06656_b300 import Problem
    assert torch.cuda.is_available()
    return Problem


def _both(p, X0, lr, steps):
    x1 = torch.from_numpy(X0.copy()).cuda()
    x2 = torch.from_numpy(X0.copy()).cuda()
    a = p.step(x1, lr, n_steps=steps)
    b = p.step_persistent(x2, lr, n_steps=steps)
    torch.cuda.synchronize()
    return x1, a, x2, b


def _same(x1, a, x2, b):
    assert torch.equal(x1.view(torch.int32), x2.view(torch.int32))
    for u, v in zip(a, b):
        assert torch.equal(u, v)


CASES = [
    ("3sat_ragged", lambda: W.random_ksat(n=3000, m=12780, seed=5), 1000, 7),
    ("5sat", lambda: W.redundant_5sat(n=2000, m=12000, seed=6), 64, 5),
    ("or_xor_short", lambda: W.mixed_pb(n=1500, n_or=5000, n_xor=600, xor_len=(3, 16),
                                        n_card=0, seed=7), 200, 4),
    ("one_restart", lambda: W.random_ksat(n=50, m=213, seed=8), 1, 9),
    # tiles that fit in shared memory (x, every partial row and the bitset of
    # 32 restarts within 200 KB): one CTA per tile runs the loop
    ("tile_3sat_c1", lambda: W.random_ksat(n=100, m=426, seed=11), 64, 200),
    ("tile_3sat_ragged", lambda: W.random_ksat(n=100, m=426, seed=12), 50, 30),
    ("tile_3sat_many_tiles", lambda: W.random_ksat(n=100, m=426, seed=13), 2000, 12),
    # many restarts of few-row variables: cls_step's accumulate takes four
    # restart tiles per warp (a ragged last group of tiles and restarts)
    ("tile_3sat_wide", lambda: W.random_ksat(n=100, m=426, seed=16), 20003, 4),
    ("tile_or_xor_nae_weighted",
     lambda: W.random_constraint_set(np.random.default_rng(14), 150, 150,
                                     [W.TYPE_OR, W.TYPE_XOR, W.TYPE_NAE], (1, 16),
                                     weights="random"), 96, 25),
]


@pytest.mark.parametrize("name,make,R,steps", CASES, ids=[c[0] for c in CASES])
def test_persistent_equals_step(P, name, make, R, steps):
    inst = make()
    p = P(inst)
    X0 = W.uniform_points(inst.n, R, seed=3)
    _same(*_both(p, X0, 0.1, steps))


@pytest.mark.parametrize("simplify", [False, True])
def test_persistent_partial_assignment(P, simplify):
    inst = W.partial_assignment(W.redundant_5sat(n=2000, m=9000, seed=9), 0.5)
    p = P(inst, simplify_fixed=simplify)
    X0 = ocls.init_uniform(inst.n, 160, 4)
    X0[inst.fixed != 0] = inst.fixed_val[inst.fixed != 0][:, None]
    x1, a, x2, b = _both(p, X0, 0.2, 6)
    _same(x1, a, x2, b)
    # one persistent step against the oracle: counts exact on its own x
    x = torch.from_numpy(X0.copy()).cuda()
    nsat, _, _ = p.step_persistent(x, 0.2, n_steps=1)
    on, _, _ = ocls.score(inst, x.cpu().numpy())
    assert np.array_equal(nsat.cpu().numpy(), on)


@pytest.mark.parametrize("simplify", [False, True])
def test_tile_loop_partial_assignment(P, simplify):
    """Pinned variables in the one-CTA-per-tile loop (they never move; with
    CLS_SIMPLIFY_FIXED their literals leave the FE work)."""
    inst = W.partial_assignment(W.planted_ksat(n=120, m=400, seed=15), 0.5)
    p = P(inst, simplify_fixed=simplify)
    X0 = ocls.init_uniform(inst.n, 70, 5)
    X0[inst.fixed != 0] = inst.fixed_val[inst.fixed != 0][:, None]
    _same(*_both(p, X0, 0.2, 15))


def test_persistent_rejects_long_constraints(P):
    inst = W.mixed_pb(n=400, n_or=800, n_xor=50, n_card=10, card_len=(20, 60), seed=10)
    p = P(inst)
    x = torch.from_numpy(W.uniform_points(inst.n, 32, seed=1)).cuda()
    with pytest.raises(RuntimeError, match="closed-form"):
        p.step_persistent(x, 0.1, 2)


def test_persistent_covers_only_short_closed_forms(P):
    """Closed forms of up to 16 literals run in the persistent loop; one of
    17-24 literals (its own thread class in cls_step) is rejected."""
    rng = np.random.default_rng(12)
    n = 300
    def xor_rows(L, count):
        return [(W.TYPE_XOR, 0, rng.choice(n, L, replace=False).astype(np.int32),
                 np.where(rng.random(L) < 0.5, -1, 1).astype(np.int8)) for _ in range(count)]
    ok = P(W.build(n, xor_rows(16, 40)))
    x = torch.from_numpy(W.uniform_points(n, 32, seed=3)).cuda()
    ok.step_persistent(x, 0.1, 2)
    bad = P(W.build(n, xor_rows(16, 40) + xor_rows(20, 5)))
    with pytest.raises(RuntimeError, match="closed-form"):
        bad.step_persistent(x, 0.1, 2)


def test_persistent_zero_steps_leaves_x(P):
    inst = W.random_ksat(n=100, m=426, seed=11)
    p = P(inst)
    X0 = W.uniform_points(inst.n, 40, seed=2)
    x = torch.from_numpy(X0.copy()).cuda()
    p.step_persistent(x, 0.1, 0, score=False, bits=False)
    assert np.array_equal(x.cpu().numpy(), X0)


def test_grid_barrier_passes_and_times_out():
    """The persistent loop's barrier: all rounds pass when every block
    arrives; when the release count can never be reached, every block stops
    waiting after its poll limit, raises the flag and returns (no hang), and
    the context stays usable."""
    from paper_2606_06656_b300 import binding as B
    scratch = torch.zeros(16, dtype=torch.uint8, device="cuda")
    assert B.cls_grid_barrier_check(200, 0, 1 << 20, scratch) == (0, 200)
    assert B.cls_grid_barrier_check(3, 1, 1 << 12, scratch) == (1, 0)
    assert B.cls_grid_barrier_check(5, 0, 1 << 20, scratch) == (0, 5)
    y = torch.arange(10, device="cuda").sum().item()
    assert y == 45
