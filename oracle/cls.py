"""Whole-problem CLS oracle -- test-only (see package docstring).

Assignments are arrays x[v, r] (variable-major, restart-minor), r indexing
independent restarts (Sec. 3.3: all batch elements iterate together).

* objective / gradient -- Sec. 2.3, Eq. 5: F(x) = sum_c w_c FE_c(s_c o x_c)
  (the paper's sum is unweighted: w_c = 1), dF/dx_v = sum over literals e on
  v of w_c s_e dFE_c/dy_e.  FP64.
* projected gradient step -- Sec. 2.3 (PGD on the cube Q^n): the step is
  x' = clamp(x - lr*g, -1, 1), computed in FP32 as two roundings
  (t = fl(lr*g), x' = fl(x - t)) so that it is reproducible bit for bit;
  the clamp is IEEE fmax/fmin (NaN -> the bound); pinned variables
  (partial assignment, Sec. 3.2) never move.
* rounding -- Sec. 2.3 sign(X): a variable is True (-1) iff x < 0; +0, -0
  and NaN round to False (+1).
* score -- Sec. 2.3: sign(X) satisfies the formula iff sum_c FE_c = -m;
  each constraint is satisfied iff its predicate holds on t, the number of
  true literals at the rounded point.  Integer counts.
* init -- x ~ U[-1, 1) from Philox4x64-10 (Salmon, Moraes, Dror, Shaw,
  "Parallel random numbers: as easy as 1, 2, 3", SC'11), keyed by the seed,
  counter (restart id, v div 4, 0, 0), output word v mod 4; x = (u >> 40) *
  2^-23 - 1.  (Random draws are an input convention, not paper arithmetic.)
* per-restart tracking, refills, movement and convergence (Sec. 3.3,
  Sec. 3.3) -- plain definitions, pinned by hand-worked traces and by the
  projected step's own displacement.
* adaptive constraint weighting (Sec. 3.1) -- per-constraint gradient-norm
  sums and violation counts (plain definitions, pinned to the OR/XOR closed
  forms and direct counts) and the library's update rule (pinned to a
  hand-worked example).
"""
import numpy as np

from . import fe as _fe
from . import spectra as _sp


def literal_values(inst, X):
    """y_e = s_e * x[v_e, r] for every literal e: array (nnz, R), FP64."""
    X = np.asarray(X, dtype=np.float64)
    return inst.lit_sign.astype(np.float64)[:, None] * X[inst.lit_var]


def objective_grad(inst, X, spectra=None):
    """Returns (obj[R], grad[n, R], fe_con[m, R]) in FP64.
    fe_con[c] = FE_c (unweighted); obj = sum_c w_c fe_con[c]."""
    X = np.asarray(X, dtype=np.float64)
    n, R = X.shape
    sps = spectra if spectra is not None else _sp.instance_spectra(inst)
    Y = literal_values(inst, X)
    fe_con = np.zeros((inst.m, R))
    grad = np.zeros((n, R))
    for c in range(inst.m):
        a, b = int(inst.offsets[c]), int(inst.offsets[c + 1])
        fe, g = _fe.fe_grad_dp(sps[c], Y[a:b])
        fe_con[c] = fe
        w = float(inst.weight[c])
        for j in range(a, b):
            grad[inst.lit_var[j]] += w * float(inst.lit_sign[j]) * g[j - a]
    obj = (inst.weight.astype(np.float64)[:, None] * fe_con).sum(axis=0)
    return obj, grad, fe_con


def pgd_step(X, G, lr, fixed=None):
    """One projected gradient step in FP32 (see module docstring)."""
    X = np.asarray(X, dtype=np.float32)
    G = np.asarray(G, dtype=np.float32)
    t = np.float32(lr) * G                      # fl(lr * g)
    # IEEE fmax/fmin (a NaN operand yields the other operand)
    Xn = np.fmin(np.fmax(X - t, np.float32(-1.0)), np.float32(1.0))
    if fixed is not None:
        keep = np.asarray(fixed).astype(bool)
        Xn[keep] = X[keep]
    return Xn.astype(np.float32)


def round_true(X):
    """Boolean array: variable is True (x < 0) at the rounded point."""
    return np.asarray(X, dtype=np.float32) < np.float32(0.0)


def true_counts(inst, X):
    """t[c, r] = number of true literals of constraint c at sign(X[:, r])."""
    vt = round_true(X)                                   # (n, R)
    lit_true = vt[inst.lit_var] ^ (inst.lit_sign < 0)[:, None]
    cs = np.concatenate([np.zeros((1, lit_true.shape[1]), np.int64),
                         np.cumsum(lit_true, axis=0, dtype=np.int64)])
    return cs[inst.offsets[1:]] - cs[inst.offsets[:-1]]


def score(inst, X, spectra=None):
    """Returns (nsat[R] int64, wsat[R] float64, sat[m, R] bool)."""
    t = true_counts(inst, X)
    sps = spectra if spectra is not None else _sp.instance_spectra(inst)
    sat = np.zeros(t.shape, dtype=bool)
    for c in range(inst.m):
        sat[c] = np.asarray(sps[c])[t[c]] == -1
    nsat = sat.sum(axis=0).astype(np.int64)
    wsat = (inst.weight.astype(np.float64)[:, None] * sat).sum(axis=0)
    return nsat, wsat, sat


def pack_bits(B):
    """Pack a boolean (n, R) array into words[n, ceil(R/32)] uint32, bit
    (r mod 32) of word r div 32 -- the bitset format of the library."""
    B = np.asarray(B, dtype=bool)
    n, R = B.shape
    RW = (R + 31) // 32
    pad = np.zeros((n, RW * 32), dtype=np.uint64)
    pad[:, :R] = B
    w = pad.reshape(n, RW, 32) << np.arange(32, dtype=np.uint64)
    return w.sum(axis=2).astype(np.uint32)


# --- Philox4x64-10 (Salmon et al., SC'11) --------------------------------
_M0, _M1 = 0xD2E7470EE14C6C93, 0xCA5A826395121157
_W0, _W1 = 0x9E3779B97F4A7C15, 0xBB67AE8584CAA73B
_MASK = (1 << 64) - 1


def philox4x64(ctr, key, rounds=10):
    """One Philox4x64 block: 4 counter words, 2 key words -> 4 words."""
    x0, x1, x2, x3 = (int(c) & _MASK for c in ctr)
    k0, k1 = (int(k) & _MASK for k in key)
    for _ in range(rounds):
        p0, p1 = _M0 * x0, _M1 * x2
        x0, x1, x2, x3 = ((p1 >> 64) ^ x1 ^ k0, p1 & _MASK,
                          (p0 >> 64) ^ x3 ^ k1, p0 & _MASK)
        k0, k1 = (k0 + _W0) & _MASK, (k1 + _W1) & _MASK
    return x0, x1, x2, x3


def init_uniform(n, R, seed, r_offset=0, fixed=None, fixed_val=None):
    """x[v, r] ~ U[-1, 1) as described in the module docstring; pinned
    variables take fixed_val."""
    X = np.empty((n, R), dtype=np.float32)
    for r in range(R):
        for q in range((n + 3) // 4):
            words = philox4x64((r + r_offset, q, 0, 0), (seed, 0))
            for j in range(4):
                v = 4 * q + j
                if v < n:
                    X[v, r] = np.float32((words[j] >> 40) * 2.0 ** -23 - 1.0)
    if fixed is not None:
        f = np.asarray(fixed).astype(bool)
        X[f] = np.asarray(fixed_val, dtype=np.float32)[f][:, None]
    return X


# --- per-restart convergence tracking and refills (Sec. 3.3) -------------
# Sec. 3.3 observes that in a lockstep batch converged restarts idle and
# waste compute, and studies the distribution of steps to convergence.
# These are the plain definitions the tracking kernels must reproduce.

def track_reset(R):
    """State rows: best satisfied count (-1), step it was reached (-1),
    steps since the last improvement (0), first step with every constraint
    satisfied (-1)."""
    S = np.zeros((4, R), dtype=np.int64)
    S[0] = -1
    S[1] = -1
    S[3] = -1
    return S


def track_step(S, nsat, step, m):
    """One step's counts: improve or age, and record the first solution."""
    S = S.copy()
    nsat = np.asarray(nsat, dtype=np.int64)
    up = nsat > S[0]
    S[0] = np.where(up, nsat, S[0])
    S[1] = np.where(up, step, S[1])
    S[2] = np.where(up, 0, S[2] + 1)
    S[3] = np.where((nsat == m) & (S[3] < 0), step, S[3])
    return S


def refill(X, S, patience, seed, generation, r_offset=0, fixed=None, fixed_val=None):
    """Restarts not solved and without improvement for `patience` steps get
    fresh uniform points: the draw of init_uniform with counter word 2 =
    generation (>= 1; generation 0 is the first draw); their tracking
    restarts.  Returns (X', S', number refilled)."""
    X = np.array(X, dtype=np.float32, copy=True)
    S = S.copy()
    n, R = X.shape
    mask = (S[3] < 0) & (S[2] >= patience)
    for r in np.nonzero(mask)[0]:
        for q in range((n + 3) // 4):
            words = philox4x64((int(r) + r_offset, q, generation, 0), (seed, 0))
            for j in range(4):
                v = 4 * q + j
                if v < n and not (fixed is not None and fixed[v]):
                    X[v, r] = np.float32((words[j] >> 40) * 2.0 ** -23 - 1.0)
    S[0, mask] = -1
    S[1, mask] = -1
    S[2, mask] = 0
    return X, S, int(mask.sum())


def unsat_histogram(nsat, m):
    """h[k] = number of restarts with exactly k unsatisfied constraints."""
    return np.bincount(m - np.asarray(nsat, dtype=np.int64), minlength=m + 1)


# --- adaptive constraint weighting (Sec. 3.1) -------------------------------
# Sec. 3.1 finds that a doubled edge-constraint gradient overwhelms the
# balancing constraints and proposes weights informed by the constraints'
# gradient magnitudes, without a rule.  The statistics are plain
# definitions; the update is the library's rule (stated in reweight).

def constraint_stats(inst, X, free_only=False, spectra=None):
    """gnorm[c] = sum_r ||dFE_c/dy(x_r)||_2 over the literals entering FE
    (all, or with free_only those on unpinned variables; 0 where w_c = 0);
    unsat[c] = restarts whose rounded point violates c.  Also returns
    has_fe[c]: the constraint's spectrum, restricted to the counts its free
    literals can reach, is not constant (it has a gradient at all)."""
    X = np.asarray(X, dtype=np.float32)
    n, R = X.shape
    sps = spectra if spectra is not None else _sp.instance_spectra(inst)
    Y = literal_values(inst, X)
    fixed = np.zeros(n, bool) if (not free_only or inst.fixed is None) \
        else np.asarray(inst.fixed).astype(bool)
    gnorm = np.zeros(inst.m)
    has_fe = np.zeros(inst.m, bool)
    for c in range(inst.m):
        a, b = int(inst.offsets[c]), int(inst.offsets[c + 1])
        free = ~fixed[inst.lit_var[a:b]]
        # pinned literals that are true shift the reachable counts
        if free.all():
            f_true = 0
        else:
            fv = np.asarray(inst.fixed_val, np.float64)[inst.lit_var[a:b]]
            f_true = int(((inst.lit_sign[a:b] * fv == -1.0) & ~free).sum())
        sp = np.asarray(sps[c])
        reach = sp[f_true:f_true + int(free.sum()) + 1]
        has_fe[c] = len(np.unique(reach)) > 1
        if not has_fe[c] or float(inst.weight[c]) == 0.0:
            continue
        _, g = _fe.fe_grad_dp(sps[c], Y[a:b])
        gnorm[c] = np.sqrt((g[free] ** 2).sum(axis=0)).sum()
    _, _, sat = score(inst, X, spectra=sps)
    unsat = (~sat).sum(axis=1).astype(np.int64)
    return gnorm, unsat, has_fe


def reweight(w, gnorm, unsat, has_fe, R, eta, kappa, w_max):
    """w'_c = min(w_max, w_c (1 + eta u_c rho_c)) with u_c = unsat_c / R,
    g_c = gnorm_c / R, gbar = mean of g_c over the constraints with FE work,
    rho_c = kappa if g_c kappa <= gbar else gbar / g_c: constraints that many
    restarts violate gain weight, the more the weaker their pull.  FP64,
    result rounded to FP32."""
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(gnorm, dtype=np.float64) / R
    u = np.asarray(unsat, dtype=np.float64) / R
    has_fe = np.asarray(has_fe, bool)
    gbar = g[has_fe].mean() if has_fe.any() else 0.0
    rho = np.array([kappa if gc * kappa <= gbar else gbar / gc for gc in g])
    return np.minimum(w_max, w * (1.0 + eta * u * rho)).astype(np.float32)


# --- convergence of the descent per restart (Sec. 3.3) ----------------------

def movement(X_prev, X):
    """max over variables of |x - x_prev| per restart, FP32 subtraction."""
    d = np.abs(np.asarray(X, np.float32) - np.asarray(X_prev, np.float32))
    return d.max(axis=0) if d.shape[0] else np.zeros(d.shape[1], np.float32)


def track_converged(conv, maxdelta, tol, step):
    """First step at which the movement is at most tol (-1 until then)."""
    conv = np.array(conv, dtype=np.int64, copy=True)
    hit = (conv < 0) & (np.asarray(maxdelta, np.float32) <= np.float32(tol))
    conv[hit] = step
    return conv
