"""Exact-rational Fourier coefficients -- oracle, test-only.

* `wfcoef` -- Eq. 3 (Sec. 2.1): the symmetric-constraint coefficient formula
      f^_0 = 2^-L sum_i C(L,i) sp_i
      f^_d = [rho^(d-1)] g(rho) / (C(L-1, d-1) 2^(L-1)),  d >= 1
      g(rho) = sum_{i=0}^{L-1} d_i C(L-1,i) (1+rho)^(L-i-1) (1-rho)^i
  (the paper writes n for the constraint length; here it is L).
* `closed_form` -- the per-type closed forms of Appendix A, transcribed as
  printed, with two readings where the printed text cannot be right:
  the AMO constant term is printed as 1 - (n-1)/2^(n-1); Eq. 3 gives
  1 - (n+1)/2^(n-1) (n = 2, a NAND: the mean of its corner values is -1/2,
  the printed form gives +1/2), so `closed_form(..., amo_as_printed=False)`
  uses Eq. 3's value; and the EK polynomial's "(1-p)" is read as (1-rho).
* `esp` -- elementary symmetric polynomials e_d(y) (Eq. 2, index bound read
  as j_i <= n), so FE(y) = sum_d f^_d e_d(y) (Eq. 1 with f^ depending on |S|
  only).
"""
from fractions import Fraction
from math import comb


def _poly_mul(a, b):
    out = [Fraction(0)] * (len(a) + len(b) - 1)
    for i, x in enumerate(a):
        if x == 0:
            continue
        for j, y in enumerate(b):
            out[i + j] += x * y
    return out


def _poly_pow(p, e):
    out = [Fraction(1)]
    for _ in range(e):
        out = _poly_mul(out, p)
    return out


def wfcoef(sp):
    """Eq. 3: coefficients f^_d, d = 0..L, as Fractions."""
    sp = [int(v) for v in sp]
    L = len(sp) - 1
    f0 = Fraction(sum(comb(L, i) * sp[i] for i in range(L + 1)), 2 ** L)
    out = [f0]
    if L == 0:
        return out
    g = [Fraction(0)] * L
    for i in range(L):
        d_i = Fraction(sp[i] - sp[i + 1], 2)
        if d_i == 0:
            continue
        term = _poly_mul(_poly_pow([Fraction(1), Fraction(1)], L - i - 1),
                         _poly_pow([Fraction(1), Fraction(-1)], i))
        for e, cf in enumerate(term):
            g[e] += d_i * comb(L - 1, i) * cf
    for d in range(1, L + 1):
        out.append(g[d - 1] / (comb(L - 1, d - 1) * 2 ** (L - 1)))
    return out


def closed_form(name, n, k=None, amo_as_printed=False):
    """Appendix A closed forms; returns f^_d, d = 0..n, as Fractions."""
    h = Fraction(1, 2 ** (n - 1))
    if name == "OR":
        return [h - 1] + [h] * n
    if name == "EO":
        return [1 - n * h] + [(2 * d - n) * h for d in range(1, n + 1)]
    if name == "AMO":
        c0 = 1 - (n - 1) * h if amo_as_printed else 1 - (n + 1) * h
        return [c0] + [(2 * d - n - 1) * h for d in range(1, n + 1)]
    if name == "NAE":
        q = Fraction(1, 2 ** (n - 2)) if n >= 2 else Fraction(2 ** (2 - n))
        return [q - 1] + [q if d % 2 == 0 else Fraction(0) for d in range(1, n + 1)]
    if name == "XOR":
        return [Fraction(0)] * n + [Fraction(1)]
    if name == "CARD_GE":
        c0 = 1 - Fraction(sum(comb(n, i) for i in range(k, n + 1)), 2 ** (n - 1))
        gp = _poly_mul(_poly_pow([Fraction(1), Fraction(1)], n - k),
                       _poly_pow([Fraction(1), Fraction(-1)], k - 1))
        return [c0] + [comb(n - 1, k - 1) * gp[d - 1] / (comb(n - 1, d - 1) * 2 ** (n - 1))
                       for d in range(1, n + 1)]
    if name == "EK":   # valid for 1 <= k <= n-1 (exponents of the printed g)
        c0 = 1 - Fraction(comb(n, k), 2 ** (n - 1))
        lin = [Fraction(2 * k - n), Fraction(n)]
        gp = _poly_mul(lin, _poly_mul(_poly_pow([Fraction(1), Fraction(1)], n - k - 1),
                                      _poly_pow([Fraction(1), Fraction(-1)], k - 1)))
        gp = [Fraction(comb(n, k), n) * v for v in gp]
        return [c0] + [gp[d - 1] / (comb(n - 1, d - 1) * 2 ** (n - 1)) for d in range(1, n + 1)]
    raise ValueError(name)


def esp(y):
    """e_d(y) for d = 0..len(y): coefficients of prod_i (1 + y_i z)."""
    e = [Fraction(1)]
    for yi in y:
        yi = Fraction(yi)
        new = e + [Fraction(0)]
        for d in range(len(e), 0, -1):
            new[d] += yi * e[d - 1]
        e = new
    return e


def fe_exact(coeffs, y):
    """FE(y) = sum_d f^_d e_d(y), exact for rational y."""
    e = esp(y)
    return sum(c * v for c, v in zip(coeffs, e))
