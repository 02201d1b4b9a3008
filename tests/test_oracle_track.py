"""Pins of the oracle's per-restart tracking, refill and histogram
definitions (Sec. 3.3's convergence profiles), CPU only."""
import numpy as np

from oracle import cls as O


def test_track_step_hand_trace():
    """A hand-worked trace of two restarts over five steps (m = 3)."""
    S = O.track_reset(2)
    assert S.tolist() == [[-1, -1], [-1, -1], [0, 0], [-1, -1]]
    seq = [(1, 2), (1, 3), (2, 3), (2, 1), (3, 3)]
    for step, nsat in enumerate(seq):
        S = O.track_step(S, nsat, step, 3)
    # restart 0: 1 (step 0), no gain, 2 (step 2), no gain, 3 (step 4, solved)
    # restart 1: 2 (step 0), 3 (step 1, solved), then three steps without gain
    assert S[:, 0].tolist() == [3, 4, 0, 4]
    assert S[:, 1].tolist() == [3, 1, 3, 1]


def test_refill_generation_zero_is_the_first_draw():
    """The refill draw with generation 0 is exactly init_uniform's draw (the
    counter layout: restart, quad, generation, 0), so generation g >= 1
    continues the same Philox stream family."""
    n, R, seed = 11, 5, 77
    X0 = O.init_uniform(n, R, seed)
    S = O.track_reset(R)
    S[2] = 9                                    # every restart stuck
    X1, S1, cnt = O.refill(np.zeros((n, R), np.float32), S, 5, seed, 0)
    assert cnt == R and np.array_equal(X1, X0)
    assert (S1[0] == -1).all() and (S1[2] == 0).all()


def test_refill_selects_stuck_unsolved_and_keeps_pins():
    n, R, seed = 9, 6, 3
    X = O.init_uniform(n, R, seed)
    S = O.track_reset(R)
    S[0] = [5, 5, 5, 5, 5, 5]
    S[2] = [0, 4, 5, 9, 9, 2]                   # patience 5: restarts 2, 3, 4
    S[3] = [-1, -1, -1, -1, 7, -1]              # 4 is solved: kept
    fixed = np.zeros(n, np.uint8)
    fixed[[0, 5]] = 1
    X1, S1, cnt = O.refill(X, S, 5, seed, 2, fixed=fixed, fixed_val=np.zeros(n, np.float32))
    assert cnt == 2
    moved = [r for r in range(R) if not np.array_equal(X1[:, r], X[:, r])]
    assert moved == [2, 3]
    assert np.array_equal(X1[[0, 5]], X[[0, 5]])   # pinned variables untouched
    assert S1[0].tolist() == [5, 5, -1, -1, 5, 5] and S1[2].tolist() == [0, 4, 0, 0, 9, 2]
    # a new generation gives new values, in [-1, 1)
    assert (np.abs(X1[1:5, 2:4] - X[1:5, 2:4]) > 0).all()
    assert (X1 >= -1).all() and (X1 < 1).all()


def test_unsat_histogram_counts():
    nsat = np.array([5, 3, 5, 0, 4])
    h = O.unsat_histogram(nsat, 5)
    assert h.tolist() == [2, 1, 1, 0, 0, 1] and h.sum() == 5


def test_movement_and_convergence_definitions():
    """movement = the largest coordinate change of a restart: zero for no
    change; for a projected step it is the step size |fl(lr g)| where no
    bound is hit, and the distance to the bound where one is.  The
    convergence record takes the first step at or below tol and keeps it."""
    rng = np.random.default_rng(4)
    X = rng.uniform(-0.5, 0.5, (30, 7)).astype(np.float32)
    assert (O.movement(X, X) == 0).all()
    G = rng.normal(size=(30, 7)).astype(np.float32) * 0.1
    Xn = O.pgd_step(X, G, 0.5)                        # |0.5 g| < 0.5: no clamp here
    t = np.abs(np.float32(0.5) * G)
    inside = np.abs(X.astype(np.float64) - 0.5 * G) < 0.99
    want = np.where(inside, t, np.abs(Xn - X)).max(axis=0)
    assert np.allclose(O.movement(X, Xn), want, rtol=1e-6, atol=0)
    # a coordinate pushed past the bound moves only to the bound
    Y = np.array([[0.9, -0.2]], np.float32)
    Yn = O.pgd_step(Y, np.array([[-1.0, 0.0]], np.float32), 1.0)
    assert O.movement(Y, Yn).tolist() == [np.float32(1.0) - np.float32(0.9), 0.0]
    conv = -np.ones(4, np.int64)
    conv = O.track_converged(conv, np.array([0.5, 1e-5, 0.0, 2e-4], np.float32), 1e-4, 3)
    assert conv.tolist() == [-1, 3, 3, -1]
    conv = O.track_converged(conv, np.array([1e-6, 1e-6, 1.0, 1e-4], np.float32), 1e-4, 4)
    assert conv.tolist() == [4, 3, 3, 4]
