"""Seeded synthetic constraint sets shaped like the paper's workloads.

This module is the only code shared by the CUDA path's tests/bench and the
CPU oracle.  It draws instances (literal index/sign arrays, offsets, constraint
type and threshold, weights) and starting points; it contains none of the
method's arithmetic (no Walsh-Fourier expansion, gradient, step or score).

Instance format (all numpy, constraint-major):
  n            number of variables
  offsets      int32[m+1], literals of constraint c are offsets[c]..offsets[c+1]-1
  lit_var      int32[nnz], 0-based variable index of each literal
  lit_sign     int8[nnz],  +1 positive literal, -1 negated literal
  ctype        int32[m],   one of the TYPE_* codes below
  k            int32[m],   threshold for CARD_GE / CARD_LE / EK (0..L), else 0
  weight       float32[m]
  spectra      int8 array or None: concatenated L+1 entries (+-1) for every
               TYPE_SPECTRUM constraint, in constraint order
  fixed        uint8[n] or None: 1 = variable pinned (partial assignment)
  fixed_val    float32[n] or None: pinned value (+-1) where fixed
  plant        int8[n] or None: the planted satisfying assignment (+-1)

Encoding (Sec. 2.1): True -> -1, False -> +1.  A literal with sign s on
variable v is true at a corner x when s * x_v == -1.

The constraint types are the symmetric PB constraints of Sec. 2.2 and
Appendix A: OR (t>=1), XOR (t odd), CARD_GE (t>=k), CARD_LE (t<=k),
NAE (0<t<L), EO (t==1), EK (t==k), AMO (t<=1), SPECTRUM (explicit truth
table over t), with t the number of true literals.
"""
from dataclasses import dataclass, field
from typing import Optional
import numpy as np

TYPE_OR, TYPE_XOR, TYPE_CARD_GE, TYPE_CARD_LE, TYPE_NAE = 0, 1, 2, 3, 4
TYPE_EO, TYPE_EK, TYPE_AMO, TYPE_SPECTRUM = 5, 6, 7, 8
TYPE_NAMES = {TYPE_OR: "OR", TYPE_XOR: "XOR", TYPE_CARD_GE: "CARD_GE",
              TYPE_CARD_LE: "CARD_LE", TYPE_NAE: "NAE", TYPE_EO: "EO",
              TYPE_EK: "EK", TYPE_AMO: "AMO", TYPE_SPECTRUM: "SPECTRUM"}


@dataclass
class Instance:
    n: int
    offsets: np.ndarray
    lit_var: np.ndarray
    lit_sign: np.ndarray
    ctype: np.ndarray
    k: np.ndarray
    weight: np.ndarray
    spectra: Optional[np.ndarray] = None
    fixed: Optional[np.ndarray] = None
    fixed_val: Optional[np.ndarray] = None
    plant: Optional[np.ndarray] = None
    name: str = ""
    meta: dict = field(default_factory=dict)

    @property
    def m(self) -> int:
        return int(len(self.offsets) - 1)

    @property
    def nnz(self) -> int:
        return int(self.offsets[-1])

    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets).astype(np.int64)


# ---------------------------------------------------------------------------
# planting: the generator's own truth test, used only to make instances
# satisfiable by a known assignment
# ---------------------------------------------------------------------------
def _holds(ct: int, L: int, k: int, t: int, spec=None) -> bool:
    if ct == TYPE_OR:
        return t >= 1
    if ct == TYPE_XOR:
        return t % 2 == 1
    if ct == TYPE_CARD_GE:
        return t >= k
    if ct == TYPE_CARD_LE:
        return t <= k
    if ct == TYPE_NAE:
        return 0 < t < L
    if ct == TYPE_EO:
        return t == 1
    if ct == TYPE_EK:
        return t == k
    if ct == TYPE_AMO:
        return t <= 1
    if ct == TYPE_SPECTRUM:
        return spec[t] == -1
    raise ValueError(ct)


def _plant_signs(rng, ct, L, k, vars_, signs, z):
    """Flip the fewest literal signs so the constraint holds under plant z."""
    true = (signs * z[vars_]) == -1
    t = int(true.sum())
    if _holds(ct, L, k, t):
        return signs
    if ct in (TYPE_OR, TYPE_XOR, TYPE_NAE):
        i = rng.integers(L)
        signs[i] = -signs[i]
    elif ct in (TYPE_CARD_GE, TYPE_EO, TYPE_EK) and t < {TYPE_CARD_GE: k, TYPE_EO: 1, TYPE_EK: k}[ct]:
        need = {TYPE_CARD_GE: k, TYPE_EO: 1, TYPE_EK: k}[ct] - t
        idx = rng.choice(np.flatnonzero(~true), size=need, replace=False)
        signs[idx] = -signs[idx]
    else:  # too many true literals: CARD_LE, AMO, EO, EK
        target = {TYPE_CARD_LE: k, TYPE_AMO: 1, TYPE_EO: 1, TYPE_EK: k}[ct]
        idx = rng.choice(np.flatnonzero(true), size=t - target, replace=False)
        signs[idx] = -signs[idx]
    t2 = int(((signs * z[vars_]) == -1).sum())
    assert _holds(ct, L, k, t2)
    return signs


def build(n, rows, rng=None, plant=None, name="", weights=None, fixed=None,
          fixed_val=None, spectra=None, meta=None) -> Instance:
    """rows: list of (ctype, k, vars(array), signs(array))."""
    offsets = np.zeros(len(rows) + 1, dtype=np.int32)
    offsets[1:] = np.cumsum([len(r[2]) for r in rows])
    nnz = int(offsets[-1])
    lit_var = np.empty(nnz, dtype=np.int32)
    lit_sign = np.empty(nnz, dtype=np.int8)
    ctype = np.empty(len(rows), dtype=np.int32)
    kk = np.zeros(len(rows), dtype=np.int32)
    for c, (ct, k, v, s) in enumerate(rows):
        lit_var[offsets[c]:offsets[c + 1]] = v
        lit_sign[offsets[c]:offsets[c + 1]] = s
        ctype[c] = ct
        kk[c] = k
    w = np.ones(len(rows), dtype=np.float32) if weights is None else np.asarray(weights, np.float32)
    return Instance(n=int(n), offsets=offsets, lit_var=lit_var, lit_sign=lit_sign,
                    ctype=ctype, k=kk, weight=w, spectra=spectra, fixed=fixed,
                    fixed_val=fixed_val, plant=plant, name=name, meta=meta or {})


def _draw_rows(rng, n, spec_list, z=None):
    """spec_list: list of (ctype, L, k). Distinct variables, uniform signs;
    planted when z is given."""
    rows = []
    for ct, L, k in spec_list:
        v = rng.choice(n, size=L, replace=False).astype(np.int32)
        s = np.where(rng.random(L) < 0.5, -1, 1).astype(np.int8)
        if z is not None:
            s = _plant_signs(rng, ct, L, k, v, s, z)
        rows.append((ct, k, v, s))
    return rows


# ---------------------------------------------------------------------------
# workloads (sizes follow the benchmark configurations)
# ---------------------------------------------------------------------------
def random_ksat(n=100, m=426, kl=3, seed=1100) -> Instance:
    """Uniform random k-SAT: kl distinct variables per clause, signs +-1
    uniform, weights 1 (3-SAT at clause ratio 4.26 mirrors Sec. 3.2)."""
    rng = np.random.default_rng(seed)
    rows = _draw_rows(rng, n, [(TYPE_OR, kl, 0)] * m)
    return build(n, rows, name=f"random{kl}sat_n{n}_m{m}",
                 meta=dict(seed=seed))


def planted_ksat(n=550, m=None, kl=3, seed=1600) -> Instance:
    """Random k-SAT with a planted solution at clause ratio 4.26 by default
    (stands in for the satisfiable phase-transition 3-SAT instances of
    Sec. 3.2, 450-650 variables): kl distinct variables per clause, uniform
    signs, then each clause the plant violates gets one literal's sign
    flipped (the generator's planting rule)."""
    m = int(round(4.26 * n)) if m is None else m
    rng = np.random.default_rng(seed)
    z = np.where(rng.random(n) < 0.5, -1, 1).astype(np.int8)
    rows = _draw_rows(rng, n, [(TYPE_OR, kl, 0)] * m, z)
    return build(n, rows, plant=z, name=f"planted{kl}sat_n{n}_m{m}", meta=dict(seed=seed))


def mixed_pb(n=5000, n_or=20000, or_len=(2, 8), n_xor=2000, xor_len=(3, 20),
             n_card=500, card_len=(10, 300), seed=1200, planted=True) -> Instance:
    """Batched mixed symmetric PB, planted satisfiable: clauses of length
    U{or_len}, XOR of length U{xor_len}, cardinality at-least-k or at-most-k
    (probability 1/2 each) of length U{card_len}, k ~ U{1..L-1}."""
    rng = np.random.default_rng(seed)
    z = np.where(rng.random(n) < 0.5, -1, 1).astype(np.int8) if planted else None
    spec = []
    for _ in range(n_or):
        spec.append((TYPE_OR, int(rng.integers(or_len[0], or_len[1] + 1)), 0))
    for _ in range(n_xor):
        spec.append((TYPE_XOR, int(rng.integers(xor_len[0], xor_len[1] + 1)), 0))
    for _ in range(n_card):
        L = int(rng.integers(card_len[0], min(card_len[1], n) + 1))
        ct = TYPE_CARD_GE if rng.random() < 0.5 else TYPE_CARD_LE
        spec.append((ct, L, int(rng.integers(1, L))))
    rows = _draw_rows(rng, n, spec, z)
    return build(n, rows, plant=z, name=f"mixedpb_n{n}_m{len(rows)}",
                 meta=dict(seed=seed))


def redundant_5sat(n=2000, m=40000, redundancy=0.0, red_len=(50, 200), seed=1300) -> Instance:
    """Planted 5-SAT plus round(redundancy*m) redundant at-least-1
    constraints (clauses) of length U{red_len} that the plant satisfies
    (mirrors the redundant-constraint study of Sec. 3.1.1)."""
    rng = np.random.default_rng(seed)
    z = np.where(rng.random(n) < 0.5, -1, 1).astype(np.int8)
    spec = [(TYPE_OR, 5, 0)] * m
    spec += [(TYPE_OR, int(rng.integers(red_len[0], red_len[1] + 1)), 0)
             for _ in range(int(round(redundancy * m)))]
    rows = _draw_rows(rng, n, spec, z)
    return build(n, rows, plant=z, name=f"red5sat_n{n}_m{m}_r{redundancy}",
                 meta=dict(seed=seed, redundancy=redundancy))


def ramsey_balanced(V=16, C=3, redundant=False) -> Instance:
    """Balanced edge colouring of the complete graph K_V with C colours
    (Sec. 3.1).  Variable c(e, i) = e*C + i is True when edge e (pairs u < v
    in lexicographic order) takes colour i.  Constraints, in this order:
      * per edge: EO over c(e, 0..C-1) (each edge takes exactly one colour);
      * per vertex v and colour i: CARD_GE, k = ceil((V-1)/C), over
        c({v, w}, i) for the V-1 neighbours w (balanced colour degrees);
      * redundant=True adds, per edge, the decomposed form of the same
        exactly-one condition: CARD_GE over the negated literals with
        k = C-1 (at most one colour; CARD>=2(not x) for C = 3) and OR over
        the positive ones (at least one colour).
    With V even and C dividing V-1 the plant is a round-robin
    1-factorisation of K_V (V-1 perfect matchings, (V-1)/C of them per
    colour), which gives every vertex exactly (V-1)/C edges of each colour;
    otherwise plant is None (and for C not dividing V-1 the balance
    thresholds sum past V-1 at every vertex, so no assignment exists)."""
    edges = [(u, v) for u in range(V) for v in range(u + 1, V)]
    eid = {e: i for i, e in enumerate(edges)}
    E = len(edges)
    n = E * C
    pos = np.ones(C, dtype=np.int8)
    rows = [(TYPE_EO, 0, np.arange(e * C, (e + 1) * C, dtype=np.int32), pos) for e in range(E)]
    k = -(-(V - 1) // C)
    for v in range(V):
        for i in range(C):
            vs = np.array([eid[(min(v, w), max(v, w))] * C + i for w in range(V) if w != v],
                          dtype=np.int32)
            rows.append((TYPE_CARD_GE, k, vs, np.ones(V - 1, dtype=np.int8)))
    if redundant:
        for e in range(E):
            vs = np.arange(e * C, (e + 1) * C, dtype=np.int32)
            rows.append((TYPE_CARD_GE, C - 1, vs, -pos))
            rows.append((TYPE_OR, 0, vs.copy(), pos))
    plant = None
    if V % 2 == 0 and (V - 1) % C == 0:
        colour = np.full(E, -1)
        per = (V - 1) // C
        inf, mod = V - 1, V - 1
        for r in range(V - 1):
            pairs = [(inf, r)] + [((r + j) % mod, (r - j) % mod) for j in range(1, V // 2)]
            for a, b in pairs:
                colour[eid[(min(a, b), max(a, b))]] = r // per
        plant = np.ones(n, dtype=np.int8)
        plant[np.arange(E) * C + colour] = -1
    return build(n, rows, plant=plant,
                 name=f"ramsey_V{V}_C{C}" + ("_redundant" if redundant else ""),
                 meta=dict(V=V, C=C, redundant=redundant, edges=E, k=k))


def partial_assignment(inst: Instance, frac_fixed=0.9, seed=1500) -> Instance:
    """Pin frac_fixed of the variables to the plant (Sec. 3.2's partial
    assignment completion)."""
    rng = np.random.default_rng(seed)
    fixed = np.zeros(inst.n, dtype=np.uint8)
    idx = rng.choice(inst.n, size=int(round(frac_fixed * inst.n)), replace=False)
    fixed[idx] = 1
    fixed_val = np.where(fixed == 1, inst.plant.astype(np.float32), 0.0).astype(np.float32)
    out = Instance(**{**inst.__dict__})
    out.fixed, out.fixed_val = fixed, fixed_val
    out.name = inst.name + f"_fix{frac_fixed}"
    return out


def mixed_instance(i, n_range=(1000, 4000), ratio=4.5, seed=1400):
    """The i-th instance of mixed_instances(..., seed): planted mixed PB with
    m = ratio*n in the 20000:2000:500 (clause:XOR:cardinality) proportions."""
    rng = np.random.default_rng(seed + i)
    n = int(rng.integers(n_range[0], n_range[1] + 1))
    m = int(round(ratio * n))
    n_card = max(1, int(round(m * 500 / 22500)))
    n_xor = max(1, int(round(m * 2000 / 22500)))
    n_or = m - n_card - n_xor
    return mixed_pb(n=n, n_or=n_or, n_xor=n_xor, n_card=n_card,
                    card_len=(10, min(300, n)), seed=seed * 7 + i)


def mixed_instances(count, n_range=(1000, 4000), ratio=4.5, seed=1400, workers=1):
    """Planted mixed-PB instances with m = ratio*n in the 20000:2000:500
    (clause:XOR:cardinality) proportions.  workers > 1 draws them in that
    many spawned processes (same instances, same order)."""
    if workers > 1 and count > 1:
        import functools
        import multiprocessing as mp
        fn = functools.partial(mixed_instance, n_range=n_range, ratio=ratio, seed=seed)
        with mp.get_context("spawn").Pool(min(workers, count)) as pool:
            return pool.map(fn, range(count), chunksize=1)
    return [mixed_instance(i, n_range, ratio, seed) for i in range(count)]


def random_constraint_set(rng, n, m, types, L_range, weights="ones", spectra_for=None):
    """Unplanted random constraints of the given types for parity tests.
    L ~ U{L_range}; k ~ U{0..L} for thresholded types; random spectra for
    TYPE_SPECTRUM."""
    rows, spectra = [], []
    for _ in range(m):
        ct = int(types[rng.integers(len(types))])
        L = int(rng.integers(L_range[0], min(L_range[1], n) + 1))
        k = int(rng.integers(0, L + 1)) if ct in (TYPE_CARD_GE, TYPE_CARD_LE, TYPE_EK) else 0
        if ct == TYPE_SPECTRUM:
            spectra.append(np.where(rng.random(L + 1) < 0.5, -1, 1).astype(np.int8))
        v = rng.choice(n, size=L, replace=False).astype(np.int32)
        s = np.where(rng.random(L) < 0.5, -1, 1).astype(np.int8)
        rows.append((ct, k, v, s))
    if weights == "ones":
        w = None
    else:
        w = rng.uniform(0.25, 2.0, size=m).astype(np.float32)
    sp = np.concatenate(spectra) if spectra else None
    return build(n, rows, weights=w, spectra=sp)


# ---------------------------------------------------------------------------
# starting points / test inputs (restart-minor layout: x[v, r])
# ---------------------------------------------------------------------------
def uniform_points(n, R, seed, low=-1.0, high=1.0):
    rng = np.random.default_rng(seed)
    return rng.uniform(low, high, size=(n, R)).astype(np.float32)


def corner_points(n, R, seed):
    rng = np.random.default_rng(seed)
    return np.where(rng.random((n, R)) < 0.5, -1.0, 1.0).astype(np.float32)


def near_corner_points(n, R, seed, eps=1e-3):
    rng = np.random.default_rng(seed)
    c = np.where(rng.random((n, R)) < 0.5, -1.0, 1.0)
    return (c * (1.0 - eps * rng.random((n, R)))).astype(np.float32)


def mixed_points(n, R, seed):
    """Per entry: a corner, exactly 0, or interior, with +-0.0 and tiny values
    sprinkled in (edge cases for rounding)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(-1, 1, size=(n, R))
    u = rng.random((n, R))
    x[u < 0.2] = -1.0
    x[(u >= 0.2) & (u < 0.4)] = 1.0
    x[(u >= 0.4) & (u < 0.45)] = 0.0
    x = x.astype(np.float32)
    x[(u >= 0.45) & (u < 0.48)] = np.float32(-0.0)
    x[(u >= 0.48) & (u < 0.5)] = np.float32(1e-30)
    x[(u >= 0.5) & (u < 0.52)] = np.float32(-1e-30)
    return x
