"""The root cutoff of the factored DFT kernel (kernels_fr.cu) drops the
roots j with 2 sin^2(pi j/(L+1)) (S - 1/4) >= ln(2J / 2^-24), S = sum_i
(1 - y_i^2)/4.  The bound behind it: |alpha + beta w^j|^2 = 1 - 2 alpha beta
(1 - cos theta_j), so every product of all or all-but-one factors has modulus
at most exp(-(S - 1/4)(1 - cos theta_j)), and the DFT coefficients of a +-1
spectrum (Sec. 2.3; pairs weighted 2) and their derivative versions have
modulus at most 2.  This checks the resulting claim directly, in FP64 and
with a plain DFT written here: the dropped terms add at most 2^-24 to the
expansion and to every partial derivative."""
import numpy as np
import pytest

EPS = 2.0 ** -24


def cutoff(L, S):
    J = (L + 1) // 2
    T = np.log(2 * J) + 24 * np.log(2)
    if S - 0.25 <= 0:
        return J
    q = T / (2 * (S - 0.25))
    if q >= 1:
        return J
    return min(J, int(np.ceil(np.arcsin(np.sqrt(q)) * (L + 1) / np.pi)) + 1)


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


@pytest.mark.parametrize("L,k,spread", [(60, 20, 1.0), (120, 7, 1.0), (200, 100, 1.0),
                                        (200, 100, 0.6), (90, 45, 0.3)])
def test_dropped_roots_below_eps(L, k, spread):
    rng = np.random.default_rng(L + k)
    for trial in range(3):
        y = rng.uniform(-spread, spread, L)
        sp = np.array([-1.0 if t >= k else 1.0 for t in range(L + 1)])
        S = np.sum((1 - y * y) / 4)
        jc = cutoff(L, S)
        fe, gr = dft_terms(sp, y)
        J = len(fe)
        tail_fe = np.abs(fe[jc:].sum()) if jc < J else 0.0
        tail_gr = np.abs(gr[jc:].sum(0)).max() if jc < J else 0.0
        assert tail_fe <= EPS and tail_gr <= EPS, (jc, J, tail_fe, tail_gr)
        if spread == 1.0 and L >= 120:
            assert jc < J          # long constraints at uniform points: roots are dropped
