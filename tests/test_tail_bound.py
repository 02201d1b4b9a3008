"""The root cutoff of the DFT kernels (kernels.cuh, tail_roots) drops the
roots j with B(s_j) >= ln(2J / 2^-24), s_j = sin^2(pi j/(L+1)),

    B(s) = 1/2 sum_{m=1..4} s^m (A_m - a_max^m) / m,   A_m = sum_i a_i^m,

a_i = 1 - y_i^2.  The bound behind it: |alpha + beta w^j|^2 = 1 - a s_j, and
-ln(1 - x) >= x + x^2/2 + x^3/3 + x^4/4, so every product of all or
all-but-one factors has modulus at most exp(-B(s_j)); the DFT coefficients
of a +-1 spectrum (Sec. 2.3; pairs weighted 2) and their derivative versions
have modulus at most 2.  This checks the resulting claim directly, in FP64
and with a plain DFT written here: the dropped terms add at most 2^-24 to
the expansion and to every partial derivative.  The points include the
regimes the bound is sharp in: many literals at +-1 with the rest spread
(the middle of a run), one literal at 0 among corners (the all-but-one
product), and near-corner values."""
import numpy as np
import pytest

EPS = 2.0 ** -24


def first_dropped(L, y):
    """Smallest root number whose terms the bound drops (J + 1 if none)."""
    J = (L + 1) // 2
    T = np.log(2 * J) + 24 * np.log(2)
    a = 1.0 - y * y
    amax = a.max() if len(a) else 0.0
    Ab = [max(0.0, (a ** m).sum() - amax ** m) for m in range(1, 5)]
    for j in range(1, J + 1):
        s = np.sin(np.pi * j / (L + 1)) ** 2
        if 0.5 * sum(s ** m * Ab[m - 1] / m for m in range(1, 5)) >= T:
            return j
    return J + 1


def first_dropped_linear(L, y):
    """The first version's bound (m = 1 only, a_max <= 1)."""
    J = (L + 1) // 2
    T = np.log(2 * J) + 24 * np.log(2)
    S = np.sum((1 - y * y) / 4)
    for j in range(1, J + 1):
        if 2 * np.sin(np.pi * j / (L + 1)) ** 2 * (S - 0.25) >= T:
            return j
    return J + 1


def dft_terms(sp, y):
    """Per root j = 1..J: Re(b'_j G_j) and Re(c'_j prod_{l != i} F_lj)."""
    L = len(y)
    N = L + 1
    J = N // 2
    a, b = (1 + y) / 2, (1 - y) / 2
    fe, gr = [], []
    for j in range(1, J + 1):
        w = np.exp(2j * np.pi * j / N)
        bj = (sp * np.exp(-2j * np.pi * j * np.arange(N) / N)).sum() / N
        bj *= 1.0 if 2 * j == N else 2.0
        F = a + b * w
        fe.append((bj * np.prod(F)).real)
        cj = bj * (1 - w) / 2
        gr.append(np.array([(cj * np.prod(np.delete(F, i))).real for i in range(L)]))
    return np.array(fe), np.array(gr)


def points(kind, L, rng):
    if kind == "uniform":
        return rng.uniform(-1, 1, L)
    if kind == "narrow":
        return rng.uniform(-0.3, 0.3, L)
    if kind == "half_corners":       # the middle of a run: half at +-1, the rest spread
        y = rng.uniform(-1, 1, L)
        c = rng.random(L) < 0.5
        y[c] = np.sign(y[c])
        return y
    if kind == "near_corners":       # |y| in [0.9, 1)
        return rng.choice([-1.0, 1.0], L) * rng.uniform(0.9, 1.0, L)
    if kind == "one_at_zero":        # corners, a few near-corner values, one literal at 0
        y = rng.choice([-1.0, 1.0], L)
        k = rng.choice(L, L // 3, replace=False)
        y[k] *= rng.uniform(0.5, 1.0, len(k))
        y[k[0]] = 0.0
        return y
    raise ValueError(kind)


@pytest.mark.parametrize("L,k,kind", [(60, 20, "uniform"), (120, 7, "uniform"),
                                      (200, 100, "uniform"), (200, 100, "narrow"),
                                      (150, 75, "half_corners"), (240, 100, "half_corners"),
                                      (120, 60, "near_corners"), (180, 90, "one_at_zero"),
                                      (90, 45, "narrow")])
def test_dropped_roots_below_eps(L, k, kind):
    rng = np.random.default_rng(L + k)
    sp = np.array([-1.0 if t >= k else 1.0 for t in range(L + 1)])
    for trial in range(3):
        y = points(kind, L, rng)
        j0 = first_dropped(L, y)
        assert j0 <= first_dropped_linear(L, y)      # never looser than m = 1 alone
        fe, gr = dft_terms(sp, y)
        tail_fe = np.abs(fe[j0 - 1:].sum()) if j0 <= len(fe) else 0.0
        tail_gr = np.abs(gr[j0 - 1:].sum(0)).max() if j0 <= len(fe) else 0.0
        assert tail_fe <= EPS and tail_gr <= EPS, (j0, len(fe), tail_fe, tail_gr)
        if kind == "uniform" and L >= 120:
            assert j0 <= len(fe)       # long constraints at uniform points: roots are dropped


def test_sharper_than_linear_bound_mid_run():
    """In the middle of a run (two thirds of the literals at +-1, the rest
    spread over [-1, 1]) the four-term bound keeps fewer roots than the m = 1
    bound; the roots it saves are the high ones, the most expensive to
    evaluate."""
    rng = np.random.default_rng(3)
    L = 300
    kept4 = kept1 = 0
    for _ in range(20):
        y = rng.uniform(-1, 1, L)
        c = rng.random(L) < 2 / 3
        y[c] = np.sign(y[c])
        kept4 += first_dropped(L, y) - 1
        kept1 += first_dropped_linear(L, y) - 1
    assert kept4 < 0.85 * kept1, (kept4, kept1)   # 0.83 here
