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
  Poisson-binomial count.  Forward DP over literals gives P(T = t); a reverse
  adjoint A_{i-1}(t) = alpha_i A_i(t) + beta_i A_i(t+1), A_L = sp, gives
  dFE/dy_i = 1/2 sum_t P_{i-1}(t) (A_i(t) - A_i(t+1)).
  All quantities are convex combinations, so FP64 is accurate to ~L*1e-16.
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
    # reverse adjoint: A_i(t) = E[sp_{t + #true among literals i+1..L}]
    A = np.repeat(sp[:, None], R, axis=1).astype(np.float64)  # A_L
    A_ext = np.zeros((L + 2, R))
    grad = np.zeros((L, R))
    for i in range(L, 0, -1):
        A_ext[:L + 1] = A
        A_ext[L + 1] = 0.0
        # dFE/dy_i = 1/2 sum_t P_{i-1}(t) (A_i(t) - A_i(t+1)), t = 0..i-1
        grad[i - 1] = 0.5 * (P[i - 1, :i] * (A_ext[:i] - A_ext[1:i + 1])).sum(axis=0)
        # A_{i-1}(t) = alpha_i A_i(t) + beta_i A_i(t+1)
        A = alpha[i - 1] * A_ext[:L + 1] + beta[i - 1] * A_ext[1:L + 2]
    return fe, grad
