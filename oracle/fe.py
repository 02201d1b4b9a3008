"""Walsh-Fourier expansion of one symmetric constraint -- oracle, test-only.

Literal values: y_i = s_i * x_{v_i} in [-1, 1], True -> -1 (Sec. 2.1).

Two routes to the same polynomial:

* `fe_bruteforce` / `walsh_coefficients_bruteforce` -- the definition.
  FE is the multilinear polynomial of Eq. 1 whose value at every corner
  b in {-1,1}^L is sp_{t(b)}; its coefficients are the Walsh-Fourier
  coefficients f^(S) = 2^-L sum_b f(b) prod_{i in S} b_i.  Exponential in L
  (L <= 14 in tests).

* `fe_grad_dp` -- the same polynomial evaluated in O(L^2) per point.  A
  multilinear polynomial equals the expectation of its corner values under
  independent coordinates with P[b_i = -1] = (1 - y_i)/2 (each factor
  (1 + b_i y_i)/2 is that probability).  So with
  alpha_i = (1 + y_i)/2 = P[literal i false] and
  beta_i  = (1 - y_i)/2 = P[literal i true],
  FE(y) = sum_t sp_t P(T = t), T = number of true literals, a
  Poisson-binomial count.  Forward DP over literals gives P(T = t).
  The gradient is the paper's discrete derivative (Sec. 2.1, text under
  Eq. 3: d_t = (sp_t - sp_{t+1})/2) averaged over the other literals:
  dFE/dy_i = sum_t d_t P(T_{-i} = t), T_{-i} = # true literals other than i.
  With prefix distributions P_{i-1} (literals 1..i-1) and the reverse
  recurrence D_L(a) = d_a, D_{i-1}(a) = alpha_i D_i(a) + beta_i D_i(a+1)
  (D_i(a) = E[d_{a + # true among literals i+1..L}]) it is
  dFE/dy_i = sum_a P_{i-1}(a) D_i(a).
  Every step is a convex combination, so for spectra whose d has one sign
  (OR, CARD) the partials carry relative FP64 accuracy even when tiny.
"""
import itertools
import numpy as np


def fe_bruteforce(sp, y):
    """Multilinear extension by enumeration of all 2^L corners (Eq. 1).
    sp: length L+1; y: length L. Returns FE(y) as float."""
    sp = np.asarray(sp, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    L = len(y)
    tot = 0.0
    for b in itertools.product((-1.0, 1.0), repeat=L):
        b = np.array(b)
        t = int((b == -1.0).sum())
        tot += sp[t] * np.prod((1.0 + b * y) / 2.0)
    return float(tot)


def walsh_coefficients_bruteforce(sp, L):
    """f^(S) for every subset S (as a dict frozenset -> value), from the
    corner values f(b) = sp_{t(b)} (Eq. 1)."""
    sp = np.asarray(sp, dtype=np.float64)
    corners = list(itertools.product((-1.0, 1.0), repeat=L))
    vals = [sp[sum(1 for v in b if v == -1.0)] for b in corners]
    out = {}
    for size in range(L + 1):
        for S in itertools.combinations(range(L), size):
            acc = 0.0
            for b, f in zip(corners, vals):
                p = 1.0
                for i in S:
                    p *= b[i]
                acc += f * p
            out[frozenset(S)] = acc / 2 ** L
    return out


def fe_from_walsh(coeffs, y):
    """Evaluate Eq. 1 given the coefficient dictionary."""
    tot = 0.0
    for S, f in coeffs.items():
        p = 1.0
        for i in S:
            p *= y[i]
        tot += f * p
    return tot


def fe_grad_dp(sp, Y):
    """FE and gradient for a batch of points.

    sp: length L+1 spectrum; Y: array (L, R) of literal values.
    Returns (fe[R], grad[L, R]) in float64, grad[i] = dFE/dy_i.
    """
    sp = np.asarray(sp, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    if Y.ndim == 1:
        Y = Y[:, None]
    L, R = Y.shape
    alpha = (1.0 + Y) / 2.0
    beta = (1.0 - Y) / 2.0
    # forward: prefix distributions P_i, i = 0..L (P_i has support 0..i)
    P = np.zeros((L + 1, L + 1, R))
    P[0, 0] = 1.0
    for i in range(1, L + 1):
        P[i] = alpha[i - 1] * P[i - 1]
        P[i, 1:] += beta[i - 1] * P[i - 1, :-1]
    fe = (sp[:, None] * P[L]).sum(axis=0)
    # reverse recurrence on the discrete derivative d_t, t = 0..L-1
    d = 0.5 * (sp[:-1] - sp[1:])
    D = np.zeros((L + 1, R))
    D[:L] = d[:, None]                    # D_L(a) = d_a
    grad = np.zeros((L, R))
    for i in range(L, 0, -1):
        # dFE/dy_i = sum_{a=0}^{i-1} P_{i-1}(a) D_i(a)
        grad[i - 1] = (P[i - 1, :i] * D[:i]).sum(axis=0)
        # D_{i-1}(a) = alpha_i D_i(a) + beta_i D_i(a+1), a = 0..i-2
        D[:i - 1] = alpha[i - 1] * D[:i - 1] + beta[i - 1] * D[1:i]
        D[i - 1:] = 0.0
    return fe, grad
