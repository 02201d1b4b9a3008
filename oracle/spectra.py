"""Truth tables (spectra) of symmetric constraints -- oracle, test-only.

Sec. 2.1 (text under Eq. 3): sp_i = -1 if the constraint is true when i of
its literals are true, +1 otherwise; d_i = (sp_i - sp_{i+1}) / 2 is the
discrete derivative of the spectrum.  The predicates follow the PB forms of
Table 2 (Appendix B) and the constraint list of Sec. 2.2; at-most-k
(CARD_LE) is the complement form t <= k.
"""
import numpy as np

OR, XOR, CARD_GE, CARD_LE, NAE, EO, EK, AMO, SPECTRUM = range(9)


def holds(ctype: int, L: int, k: int, t: int, spec=None) -> bool:
    """Does a constraint of this type hold with t of its L literals true?"""
    if ctype == OR:        # sum x >= 1
        return t >= 1
    if ctype == XOR:       # sum x == 1 (mod 2)
        return t % 2 == 1
    if ctype == CARD_GE:   # sum x >= k
        return t >= k
    if ctype == CARD_LE:   # sum x <= k
        return t <= k
    if ctype == NAE:       # 0 < sum x < L
        return 0 < t < L
    if ctype == EO:        # sum x == 1
        return t == 1
    if ctype == EK:        # sum x == k
        return t == k
    if ctype == AMO:       # sum x <= 1
        return t <= 1
    if ctype == SPECTRUM:  # explicit table
        return int(spec[t]) == -1
    raise ValueError(f"unknown constraint type {ctype}")


def spectrum(ctype: int, L: int, k: int = 0, spec=None) -> np.ndarray:
    """sp_t for t = 0..L (Eq. 3): -1 where the constraint holds, else +1."""
    return np.array([-1 if holds(ctype, L, k, t, spec) else 1 for t in range(L + 1)],
                    dtype=np.int64)


def discrete_derivative(sp) -> np.ndarray:
    """d_t = (sp_t - sp_{t+1}) / 2 for t = 0..L-1 (Sec. 2.1, under Eq. 3)."""
    sp = np.asarray(sp, dtype=np.float64)
    return 0.5 * (sp[:-1] - sp[1:])


def instance_spectra(inst):
    """List of per-constraint spectra of an instance (workloads.Instance)."""
    out, soff = [], 0
    L = np.diff(inst.offsets)
    for c in range(inst.m):
        spec = None
        if int(inst.ctype[c]) == SPECTRUM:
            spec = inst.spectra[soff:soff + L[c] + 1]
            soff += L[c] + 1
        out.append(spectrum(int(inst.ctype[c]), int(L[c]), int(inst.k[c]), spec))
    return out
