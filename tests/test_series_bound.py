"""Host logic of the power-sum pass, pinned to the mathematics (no GPU).

For a constraint of L literals the GPU evaluates the low roots j = 1..js of
the Fourier form (Sec. 2.3) through Chebyshev expansions of every factor
alpha + beta w^j = h (1 + q y) on [-1, 1]: log F = C + sum E_{k-1} T_k / k,
dlog F / dy = sum E_k U_k, E_k = -2 r^(k+1), |r| = tan(phi/2).
cls_series_range(L, K) is the host's choice of js.  These tests check it
against exact complex logarithms computed here in FP64: at every root
j <= js the K-term expansions of log F_j and of d log F_j / dy are within
2^-24 (the log summed over L literals) at the points of [-1, 1] where the
Chebyshev polynomials peak; and the bound fails near js + 1 (the range is
tight)."""
import numpy as np
import pytest

from paper_2606_06656_b300 import binding as B

EPS = 2.0 ** -24


def factor(L, j, y):
    """alpha + beta w^j at y (alpha = (1 + y)/2, beta = (1 - y)/2)."""
    w = np.exp(2j * np.pi * j / (L + 1))
    return (1 + y) / 2 + (1 - y) / 2 * w


def cheb_T(k, y):
    return np.cos(k * np.arccos(np.clip(y, -1.0, 1.0)))


def cheb_U(k, y):
    if abs(y) == 1.0:
        return (k + 1) * (np.sign(y) ** k)
    th = np.arccos(y)
    return np.sin((k + 1) * th) / np.sin(th)


def truncation_errors(L, j, K, y):
    """|log F(y) - K-term Chebyshev series| and the relative error of the
    K-term derivative series, from exact FP64 complex arithmetic."""
    w = np.exp(2j * np.pi * j / (L + 1))
    h = (1 + w) / 2
    q = (1 - w) / (1 + w)
    r = -q / (1 + np.sqrt(1 - q * q))
    C = np.log(h) - np.log(1 + r * r)
    log_series = C + sum(-2 * r ** k * cheb_T(k, y) / k for k in range(1, K + 1))
    err_log = abs(np.log(np.exp(np.log(factor(L, j, y)) - log_series)))
    der_series = sum(-2 * r ** (k + 1) * cheb_U(k, y) for k in range(K))
    exact_der = ((1 - w) / 2) / factor(L, j, y)
    err_der = abs(der_series - exact_der) / abs(exact_der)
    return err_log, err_der


WORST = [1.0, -1.0, 0.0, 0.5, -0.5]   # |T_k| = 1 and |U_k| = k + 1 at the ends


@pytest.mark.parametrize("L", [64, 100, 129, 150, 220, 300, 511, 1024])
@pytest.mark.parametrize("K", [18, 26])
def test_series_range_within_bound(L, K):
    js = B.cls_series_range(L, K)
    assert 0 <= js <= 96 and 2 * js < L + 1
    for j in range(1, js + 1):
        for y in WORST:
            el, ed = truncation_errors(L, j, K, y)
            assert L * el <= EPS, (L, K, j, y, L * el)
            assert ed <= EPS, (L, K, j, y, ed)


@pytest.mark.parametrize("L", [64, 100, 150, 300])
@pytest.mark.parametrize("K", [18, 26])
def test_series_range_is_tight(L, K):
    """The root after the range breaks the bound at a worst point (the
    range is not chosen conservatively short), unless the cap stops it."""
    js = B.cls_series_range(L, K)
    j = js + 1
    if js >= 96 or 2 * j >= L + 1:
        pytest.skip("range capped")
    worst = max(max(L * el, ed) for el, ed in
                (truncation_errors(L, j, K, y) for y in WORST))
    # the host bound is a geometric-tail upper bound: the exact error at the
    # next root is within a small factor of 2^-24
    assert worst > EPS / 8, (L, K, js, worst)


def test_series_expansion_matches_exact_factor():
    """At random points and roots in range, the Chebyshev expansions
    reproduce log F_j and its derivative (the identities the GPU pass
    evaluates)."""
    rng = np.random.default_rng(3)
    for L in (80, 200, 300):
        js = B.cls_series_range(L, 26)
        for _ in range(50):
            j = int(rng.integers(1, js + 1))
            y = float(rng.uniform(-1, 1))
            el, ed = truncation_errors(L, j, 26, y)
            assert el <= EPS and ed <= EPS


def test_series_range_rejects_bad_arguments():
    from paper_2606_06656_b300._lib import ClsError
    with pytest.raises(ClsError):
        B.cls_series_range(0, 16)
    with pytest.raises(ClsError):
        B.cls_series_range(100, 0)
    # more terms never shrink the range; longer constraints never widen it
    # at a fixed angle (the log bound carries the factor L)
    for L in (64, 128, 256):
        assert B.cls_series_range(L, 26) >= B.cls_series_range(L, 18)
