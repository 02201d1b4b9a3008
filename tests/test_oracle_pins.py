"""Pins for the CPU oracle against what the paper and the mathematics fix.

Each test ties the oracle to a route other than itself: enumeration of the
2^L corners (Eq. 1's definition), exact rationals from Eq. 3, the Appendix A
closed forms, identities stated in Sec. 3.1.1, exact multilinear finite
differences, harmonicity (Sec. 2.3), integer brute force for scoring, and
numpy's own Philox4x64 for the initialiser.
"""
import itertools
import os
from fractions import Fraction
from math import comb

import numpy as np
import pytest

import workloads as W
from oracle import cls as ocls
from oracle import exact as oex
from oracle import fe as ofe
from oracle import spectra as osp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TYPES_K = [(osp.OR, 0), (osp.XOR, 0), (osp.NAE, 0), (osp.EO, 0), (osp.AMO, 0)]


def all_specs(L):
    """(type, k) pairs covering every type and every threshold for length L."""
    out = list(TYPES_K)
    for k in range(L + 1):
        out += [(osp.CARD_GE, k), (osp.CARD_LE, k), (osp.EK, k)]
    return out


def rng_points(rng, L, npts):
    pts = [rng.uniform(-1, 1, L) for _ in range(npts)]
    pts.append(np.zeros(L))
    pts.append(np.where(rng.random(L) < 0.5, -1.0, 1.0))
    return pts


# --- FE: DP vs the definition (Eq. 1) ------------------------------------
@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 7, 9])
def test_dp_matches_bruteforce_and_exact_fd(L):
    rng = np.random.default_rng(L)
    for ct, k in all_specs(L):
        sp = osp.spectrum(ct, L, k)
        for y in rng_points(rng, L, 3):
            fe, g = ofe.fe_grad_dp(sp, y[:, None])
            assert abs(fe[0] - ofe.fe_bruteforce(sp, y)) < 1e-12
            for i in range(L):
                yp, ym = y.copy(), y.copy()
                yp[i], ym[i] = 1.0, -1.0
                fd = 0.5 * (ofe.fe_bruteforce(sp, yp) - ofe.fe_bruteforce(sp, ym))
                assert abs(g[i, 0] - fd) < 1e-12, (ct, k, L, i)


def test_random_spectrum_dp_matches_bruteforce():
    rng = np.random.default_rng(7)
    for L in range(1, 9):
        for _ in range(4):
            sp = np.where(rng.random(L + 1) < 0.5, -1, 1)
            y = rng.uniform(-1, 1, L)
            fe, _ = ofe.fe_grad_dp(sp, y[:, None])
            assert abs(fe[0] - ofe.fe_bruteforce(sp, y)) < 1e-12


@pytest.mark.parametrize("L", [1, 4, 10])
def test_corners_are_exact_for_all_corners(L):
    for ct, k in all_specs(L):
        sp = osp.spectrum(ct, L, k)
        corners = np.array(list(itertools.product((-1.0, 1.0), repeat=L))).T
        fe, _ = ofe.fe_grad_dp(sp, corners)
        t = (corners == -1.0).sum(axis=0)
        assert np.array_equal(fe, sp[t].astype(np.float64))


@pytest.mark.parametrize("L", [33, 64, 300])
def test_random_corners_long(L):
    rng = np.random.default_rng(L)
    Y = np.where(rng.random((L, 16)) < 0.5, -1.0, 1.0)
    t = (Y == -1.0).sum(axis=0)
    for ct, k in [(osp.CARD_GE, L // 2), (osp.CARD_LE, L // 3), (osp.EK, t[0]),
                  (osp.NAE, 0), (osp.XOR, 0), (osp.EO, 0), (osp.AMO, 0)]:
        sp = osp.spectrum(ct, L, int(k))
        fe, _ = ofe.fe_grad_dp(sp, Y)
        assert np.max(np.abs(fe - sp[t])) < 1e-12


# --- coefficients: brute-force Walsh vs Eq. 3 vs Appendix A ---------------
@pytest.mark.parametrize("L", [1, 2, 3, 4, 5, 6])
def test_walsh_bruteforce_equals_eq3(L):
    for ct, k in all_specs(L):
        sp = osp.spectrum(ct, L, k)
        wal = ofe.walsh_coefficients_bruteforce(sp, L)
        eq3 = oex.wfcoef(sp)
        for S, v in wal.items():
            assert abs(v - float(eq3[len(S)])) < 1e-12, (ct, k, L, S)


def _eq3(name, n, k=0):
    ct = {"OR": osp.OR, "EO": osp.EO, "AMO": osp.AMO, "NAE": osp.NAE,
          "XOR": osp.XOR, "CARD_GE": osp.CARD_GE, "EK": osp.EK}[name]
    return oex.wfcoef(osp.spectrum(ct, n, k))


@pytest.mark.parametrize("n", list(range(1, 13)))
def test_appendix_a_closed_forms_equal_eq3(n):
    for name in ["OR", "EO", "NAE", "XOR"]:
        assert oex.closed_form(name, n) == _eq3(name, n), name
    if n >= 2:
        assert oex.closed_form("AMO", n) == _eq3("AMO", n)
        # the constant term as printed disagrees (reading documented)
        assert oex.closed_form("AMO", n, amo_as_printed=True)[0] != _eq3("AMO", n)[0]
        # ... while the printed |S| != 0 terms agree
        assert oex.closed_form("AMO", n, amo_as_printed=True)[1:] == _eq3("AMO", n)[1:]
    for k in range(1, n + 1):
        assert oex.closed_form("CARD_GE", n, k) == _eq3("CARD_GE", n, k), k
    for k in range(1, n):
        assert oex.closed_form("EK", n, k) == _eq3("EK", n, k), k


def test_golden_appendix_a_constants():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "appendix_a_constant_terms.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) >= 10
    for name, n, k, num, den, _src in rows:
        n, k, want = int(n), int(k), Fraction(int(num), int(den))
        if name == "AMO_PRINTED":
            assert oex.closed_form("AMO", n, amo_as_printed=True)[0] == want
            assert _eq3("AMO", n)[0] != want
            continue
        assert _eq3(name, n, k)[0] == want, (name, n, k)
        # and FE at y = 0 from the DP is that constant
        ct = {"OR": osp.OR, "EO": osp.EO, "AMO": osp.AMO, "NAE": osp.NAE,
              "XOR": osp.XOR, "CARD_GE": osp.CARD_GE, "EK": osp.EK}[name]
        fe, _ = ofe.fe_grad_dp(osp.spectrum(ct, n, k), np.zeros((n, 1)))
        assert abs(fe[0] - float(want)) < 1e-15


@pytest.mark.parametrize("L", [3, 8, 17, 40])
def test_eq3_exact_rationals_match_dp(L):
    rng = np.random.default_rng(100 + L)
    for ct, k in [(osp.OR, 0), (osp.XOR, 0), (osp.NAE, 0), (osp.EO, 0), (osp.AMO, 0),
                  (osp.CARD_GE, L // 2), (osp.CARD_LE, L // 3), (osp.EK, L // 2)]:
        sp = osp.spectrum(ct, L, k)
        coeffs = oex.wfcoef(sp)
        yq = [Fraction(int(v), 64) for v in rng.integers(-64, 65, size=L)]
        exact = oex.fe_exact(coeffs, yq)
        fe, _ = ofe.fe_grad_dp(sp, np.array([float(v) for v in yq])[:, None])
        assert abs(fe[0] - float(exact)) < 1e-12


def test_gradient_at_zero_is_degree_one_coefficient():
    for L in [2, 3, 6, 11]:
        for ct, k in all_specs(L):
            sp = osp.spectrum(ct, L, k)
            _, g = ofe.fe_grad_dp(sp, np.zeros((L, 1)))
            assert np.allclose(g[:, 0], float(oex.wfcoef(sp)[1]), atol=1e-15)
        # closed forms quoted: OR 2^(1-L), EO (2-L)/2^(L-1), CARD C(L-1,k-1)/2^(L-1)
        _, g = ofe.fe_grad_dp(osp.spectrum(osp.OR, L), np.zeros((L, 1)))
        assert abs(g[0, 0] - 2.0 ** (1 - L)) < 1e-15
        _, g = ofe.fe_grad_dp(osp.spectrum(osp.EO, L), np.zeros((L, 1)))
        assert abs(g[0, 0] - (2 - L) / 2.0 ** (L - 1)) < 1e-15
        k = max(1, L // 2)
        _, g = ofe.fe_grad_dp(osp.spectrum(osp.CARD_GE, L, k), np.zeros((L, 1)))
        assert abs(g[0, 0] - comb(L - 1, k - 1) / 2.0 ** (L - 1)) < 1e-15


# --- closed-form special cases and identities ----------------------------
def test_textbook_closed_forms():
    rng = np.random.default_rng(3)
    for L in [1, 2, 5, 12, 30]:
        Y = rng.uniform(-1, 1, (L, 8))
        a, b = (1 + Y) / 2, (1 - Y) / 2
        fe, g = ofe.fe_grad_dp(osp.spectrum(osp.OR, L), Y)
        # clause violation indicator prod (1 + s_i x_i)/2 = prod alpha (True -> -1)
        assert np.allclose(fe, 2 * a.prod(0) - 1, atol=1e-13)
        fe, _ = ofe.fe_grad_dp(osp.spectrum(osp.XOR, L), Y)
        assert np.allclose(fe, Y.prod(0), atol=1e-13)
        fe, _ = ofe.fe_grad_dp(osp.spectrum(osp.NAE, L), Y)
        assert np.allclose(fe, 2 * (a.prod(0) + b.prod(0)) - 1, atol=1e-13)
    # clause closed form at corners: violated exactly when all literals false
    x = np.array([1.0, 1.0, 1.0])
    fe, _ = ofe.fe_grad_dp(osp.spectrum(osp.OR, 3), x[:, None])
    assert fe[0] == 1.0


def test_redundant_encoding_identity_sec_3_1_1():
    """CARD>=2(not x) + OR(x) = EO(x) - 1 in 3 variables, everywhere."""
    rng = np.random.default_rng(11)
    Y = rng.uniform(-1, 1, (3, 50))
    c2, gc = ofe.fe_grad_dp(osp.spectrum(osp.CARD_GE, 3, 2), -Y)
    o, go = ofe.fe_grad_dp(osp.spectrum(osp.OR, 3), Y)
    e, ge = ofe.fe_grad_dp(osp.spectrum(osp.EO, 3), Y)
    assert np.allclose(c2 + o, e - 1, atol=1e-13)
    assert np.allclose(-gc + go, ge, atol=1e-13)   # chain rule on -y
    # general L: AMO + OR = EO - 1
    for L in [2, 5, 9]:
        Y = rng.uniform(-1, 1, (L, 20))
        am, _ = ofe.fe_grad_dp(osp.spectrum(osp.AMO, L), Y)
        o, _ = ofe.fe_grad_dp(osp.spectrum(osp.OR, L), Y)
        e, _ = ofe.fe_grad_dp(osp.spectrum(osp.EO, L), Y)
        assert np.allclose(am + o, e - 1, atol=1e-13)


def test_eo_plateau_at_all_true_corner_sec_3_1_1():
    for L in range(3, 12):
        _, g = ofe.fe_grad_dp(osp.spectrum(osp.EO, L), -np.ones((L, 1)))
        assert np.all(g == 0.0)
    _, g = ofe.fe_grad_dp(osp.spectrum(osp.EO, 2), -np.ones((2, 1)))
    assert np.all(g != 0.0)


def test_harmonic_multilinear_sec_2_3():
    rng = np.random.default_rng(5)
    for L in [3, 10, 25, 40]:
        for ct, k in [(osp.CARD_GE, L // 2), (osp.EK, L // 3), (osp.AMO, 0), (osp.NAE, 0)]:
            sp = osp.spectrum(ct, L, k)
            y = rng.uniform(-1, 1, L)
            fe0, g0 = ofe.fe_grad_dp(sp, y[:, None])
            for i in rng.choice(L, size=min(L, 5), replace=False):
                ys = np.repeat(y[:, None], 3, axis=1)
                ys[i] = [-1.0, 0.0, 1.0]
                f, _ = ofe.fe_grad_dp(sp, ys)
                assert abs(f[1] - 0.5 * (f[0] + f[2])) < 1e-13      # affine in y_i
                assert abs(g0[i, 0] - 0.5 * (f[2] - f[0])) < 1e-13  # exact FD


def test_bounds_and_complement():
    rng = np.random.default_rng(9)
    for L in [1, 7, 50, 120]:
        Y = rng.uniform(-1, 1, (L, 12))
        for k in sorted({0, 1, L // 2, L}):
            fe, g = ofe.fe_grad_dp(osp.spectrum(osp.CARD_GE, L, k), Y)
            fe2, g2 = ofe.fe_grad_dp(osp.spectrum(osp.CARD_LE, L, L - k), -Y)
            assert np.allclose(fe, fe2, atol=1e-13)
            assert np.allclose(g, -g2, atol=1e-13)
            assert np.all(np.abs(fe) <= 1 + 1e-14) and np.all(np.abs(g) <= 1 + 1e-14)


def test_permutation_invariance():
    rng = np.random.default_rng(13)
    L = 20
    sp = osp.spectrum(osp.EK, L, 7)
    Y = rng.uniform(-1, 1, (L, 4))
    p = rng.permutation(L)
    f1, g1 = ofe.fe_grad_dp(sp, Y)
    f2, g2 = ofe.fe_grad_dp(sp, Y[p])
    assert np.allclose(f1, f2, atol=1e-14)
    assert np.allclose(g1[p], g2, atol=1e-14)


# --- problem level -------------------------------------------------------
def _small_instance(seed=1, n=12, m=15, weights="random"):
    rng = np.random.default_rng(seed)
    types = [W.TYPE_OR, W.TYPE_XOR, W.TYPE_CARD_GE, W.TYPE_CARD_LE, W.TYPE_NAE,
             W.TYPE_EO, W.TYPE_EK, W.TYPE_AMO, W.TYPE_SPECTRUM]
    return W.random_constraint_set(rng, n, m, types, (1, 7), weights=weights)


def test_objective_gradient_exact_fd():
    inst = _small_instance()
    X = W.uniform_points(inst.n, 5, seed=2).astype(np.float64)
    obj, grad, fe_con = ocls.objective_grad(inst, X)
    assert np.allclose(obj, (inst.weight[:, None] * fe_con).sum(0))
    for v in range(inst.n):
        Xp, Xm = X.copy(), X.copy()
        Xp[v], Xm[v] = 1.0, -1.0
        fd = 0.5 * (ocls.objective_grad(inst, Xp)[0] - ocls.objective_grad(inst, Xm)[0])
        assert np.allclose(grad[v], fd, atol=1e-12)


def test_objective_bruteforce_small():
    inst = _small_instance(seed=4, n=8, m=6)
    X = W.uniform_points(inst.n, 3, seed=5).astype(np.float64)
    _, _, fe_con = ocls.objective_grad(inst, X)
    sps = osp.instance_spectra(inst)
    for c in range(inst.m):
        a, b = inst.offsets[c], inst.offsets[c + 1]
        for r in range(3):
            y = inst.lit_sign[a:b] * X[inst.lit_var[a:b], r]
            assert abs(fe_con[c, r] - ofe.fe_bruteforce(sps[c], y)) < 1e-12


def test_score_bruteforce_and_fe_identity():
    inst = _small_instance(seed=6, n=10, m=40, weights="ones")
    X = W.mixed_points(inst.n, 37, seed=8)
    nsat, wsat, sat = ocls.score(inst, X)
    Xr = np.where(X < 0, -1.0, 1.0)   # sign(X), True -> -1
    for r in range(X.shape[1]):
        cnt = 0
        for c in range(inst.m):
            a, b = inst.offsets[c], inst.offsets[c + 1]
            t = sum(1 for e in range(a, b) if inst.lit_sign[e] * Xr[inst.lit_var[e], r] == -1)
            cnt += W._holds(int(inst.ctype[c]), b - a, int(inst.k[c]), t,
                            osp.instance_spectra(inst)[c] if inst.ctype[c] == W.TYPE_SPECTRUM else None)
        assert cnt == nsat[r]
    # Sec. 2.3: sum_c FE_c(sign X) = m - 2 nsat (= -m iff all satisfied)
    _, _, fe_con = ocls.objective_grad(inst, Xr)
    assert np.allclose(fe_con.sum(0), inst.m - 2 * nsat, atol=1e-12)
    assert np.allclose(wsat, nsat)


def test_planted_instances_are_satisfied_by_plant():
    for inst in [W.mixed_pb(n=300, n_or=400, n_xor=60, n_card=20, card_len=(10, 120), seed=3),
                 W.redundant_5sat(n=200, m=900, redundancy=0.1, red_len=(20, 60), seed=4),
                 W.planted_ksat(n=450, seed=5)]:
        z = inst.plant.astype(np.float32)[:, None]
        nsat, _, _ = ocls.score(inst, z)
        assert nsat[0] == inst.m


def test_rounding_edge_cases():
    x = np.array([[-1.0], [1.0], [0.0], [-0.0], [np.nan], [-1e-38], [1e-45], [-np.inf]],
                 dtype=np.float32)
    assert ocls.round_true(x)[:, 0].tolist() == [True, False, False, False, False, True,
                                                 False, True]


def test_pgd_step_two_roundings_exact():
    rng = np.random.default_rng(21)
    X = rng.uniform(-1, 1, (64, 8)).astype(np.float32)
    G = (rng.standard_normal((64, 8)) * 3).astype(np.float32)
    lr = 0.1
    Xn = ocls.pgd_step(X, G, lr)
    lr32 = Fraction(float(np.float32(lr)))
    for (v, r) in [(i, j) for i in range(64) for j in range(8)]:
        t = np.float32(float(lr32 * Fraction(float(G[v, r]))))     # one rounding
        want = np.float32(float(Fraction(float(X[v, r])) - Fraction(float(t))))
        want = min(max(want, np.float32(-1)), np.float32(1))
        assert Xn[v, r] == want
    fixed = np.zeros(64, np.uint8)
    fixed[::3] = 1
    Xf = ocls.pgd_step(X, G, lr, fixed)
    assert np.array_equal(Xf[::3], X[::3])
    assert np.all(np.abs(Xf) <= 1)


def test_pack_bits():
    rng = np.random.default_rng(2)
    for R in [1, 31, 32, 33, 70]:
        B = rng.random((5, R)) < 0.5
        w = ocls.pack_bits(B)
        for v in range(5):
            for r in range(R):
                assert bool((int(w[v, r // 32]) >> (r % 32)) & 1) == B[v, r]


# --- Philox initialiser vs numpy's implementation ------------------------
def test_philox4x64_matches_numpy():
    for key in ([0, 0], [42, 0], [2 ** 63 + 5, 7]):
        for c0 in (0, 1, 1000, 2 ** 40):
            bg = np.random.Philox(key=np.array(key, dtype=np.uint64),
                                  counter=np.array([c0, 0, 0, 0], dtype=np.uint64))
            ref = [int(v) for v in bg.random_raw(4)]
            # numpy advances the counter before producing a block
            assert list(ocls.philox4x64((c0 + 1, 0, 0, 0), key)) == ref


def test_init_uniform_range_and_fixed():
    X = ocls.init_uniform(9, 40, seed=42)
    assert X.dtype == np.float32 and np.all(X >= -1) and np.all(X < 1)
    assert abs(float(X.mean())) < 0.2
    X2 = ocls.init_uniform(9, 20, seed=42, r_offset=20)
    assert np.array_equal(X[:, 20:], X2)      # keyed by global restart id
    fixed = np.zeros(9, np.uint8)
    fixed[[1, 4]] = 1
    fv = np.zeros(9, np.float32)
    fv[1], fv[4] = -1.0, 1.0
    X3 = ocls.init_uniform(9, 5, seed=1, fixed=fixed, fixed_val=fv)
    assert np.all(X3[1] == -1.0) and np.all(X3[4] == 1.0)
