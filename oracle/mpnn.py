"""Message-passing initialiser -- oracle, test-only.

The paper has no learned component; this model is this library's learned
initialiser (a 2-layer message-passing network, hidden width 64, on the
constraint-variable incidence graph) and is defined here, FP64, as the
reference the GPU kernels are checked against.

Graph: variable nodes v, constraint nodes c, one edge per literal e with sign
s_e = +-1 (Sec. 2.2's literals).  Node features
  f_v = [1, deg_v/16, pos_v/deg_v, neg_v/deg_v]                (4)
  f_c = [onehot(type, 9), L_c/64, k_c/L_c, w_c]                (12)
(pos/neg = literals of v with sign +1/-1, k only for CARD_GE/CARD_LE/EK).
Embedding  h_v = relu(W_vin f_v + b_vin),  h_c = relu(W_cin f_c + b_cin).
Two layers, l = 1, 2:
  a_c = L_c^{-1/2}   sum_{e in c} s_e h_v[v_e]
  h_c = relu(W_cl [h_c, a_c] + b_cl)
  a_v = deg_v^{-1/2} sum_{e on v} s_e h_c[c_e]          (the updated h_c)
  h_v = relu(W_vl [h_v, a_v] + b_vl)
Head  z_v = w_out . h_v + b_out;  initial points x0[v, r] = tanh(z_v + tau u[v, r])
with u[v, r] the U[-1, 1) draws of the initialiser (pinned variables keep
their fixed value).
Training loss per instance (R restarts, n_free free variables, targets t_v in
{-1, +1} from local minima the solver reached, weight lam):
  J = 1/(R m) sum_r F(x0_r) + lam/n_free sum_{free v} softplus(-2 t_v z_v)
(F the CLS objective of Sec. 2.3, Eq. 5).

`emulate_bf16=True` rounds the operands of the four 128-wide dense layers
(forward and both backward products) to bfloat16 exactly as the tensor-core
kernels do, so that GPU and oracle differ only by FP32 accumulation order.
"""
import numpy as np

HID, FV, FC = 64, 4, 12
N_TYPES = 9
PARAM_LAYOUT = [
    ("W_vin", (HID, FV)), ("b_vin", (HID,)), ("W_cin", (HID, FC)), ("b_cin", (HID,)),
    ("W_c1", (HID, 2 * HID)), ("b_c1", (HID,)), ("W_v1", (HID, 2 * HID)), ("b_v1", (HID,)),
    ("W_c2", (HID, 2 * HID)), ("b_c2", (HID,)), ("W_v2", (HID, 2 * HID)), ("b_v2", (HID,)),
    ("w_out", (HID,)), ("b_out", (1,)),
]
N_PARAMS = sum(int(np.prod(s)) for _, s in PARAM_LAYOUT)
THRESH_TYPES = (2, 3, 6)   # CARD_GE, CARD_LE, EK


def unflatten(theta):
    out, off = {}, 0
    for name, shape in PARAM_LAYOUT:
        k = int(np.prod(shape))
        out[name] = np.asarray(theta[off:off + k], dtype=np.float64).reshape(shape)
        off += k
    return out


def flatten(d):
    return np.concatenate([np.asarray(d[name], np.float64).reshape(-1)
                           for name, _ in PARAM_LAYOUT])


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    a32 = np.asarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    rounded = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    out = rounded.astype(np.uint32).view(np.float32).astype(np.float64)
    return np.where(np.isfinite(a32), out, a32.astype(np.float64))


def features(inst):
    n, m = inst.n, inst.m
    L = np.diff(inst.offsets).astype(np.float64)
    deg = np.bincount(inst.lit_var, minlength=n).astype(np.float64)
    pos = np.bincount(inst.lit_var[inst.lit_sign > 0], minlength=n).astype(np.float64)
    neg = deg - pos
    d1 = np.maximum(deg, 1.0)
    fv = np.stack([np.ones(n), deg / 16.0, pos / d1, neg / d1], axis=1)
    fc = np.zeros((m, FC))
    fc[np.arange(m), inst.ctype] = 1.0
    fc[:, 9] = L / 64.0
    kk = np.where(np.isin(inst.ctype, THRESH_TYPES), inst.k, 0).astype(np.float64)
    fc[:, 10] = kk / L
    fc[:, 11] = inst.weight.astype(np.float64)
    return fv, fc, L, deg


def _edges(inst):
    con_of = np.repeat(np.arange(inst.m), np.diff(inst.offsets))
    return con_of, inst.lit_var.astype(np.int64), inst.lit_sign.astype(np.float64)


def _agg_to_con(inst, hv, scale_src=None):
    """sum_{e in c} s_e (scale_src[v_e]) hv[v_e] for every constraint c."""
    con_of, var_of, sg = _edges(inst)
    w = sg if scale_src is None else sg * scale_src[var_of]
    out = np.zeros((inst.m, hv.shape[1]))
    np.add.at(out, con_of, w[:, None] * hv[var_of])
    return out


def _agg_to_var(inst, hc, scale_src=None):
    """sum_{e on v} s_e (scale_src[c_e]) hc[c_e] for every variable v."""
    con_of, var_of, sg = _edges(inst)
    w = sg if scale_src is None else sg * scale_src[con_of]
    out = np.zeros((inst.n, hc.shape[1]))
    np.add.at(out, var_of, w[:, None] * hc[con_of])
    return out


def forward(inst, theta, emulate_bf16=True):
    """Returns (z[n], cache)."""
    P = unflatten(theta)
    q = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    fv, fc, L, deg = features(inst)
    isL = 1.0 / np.sqrt(L)
    isd = 1.0 / np.sqrt(np.maximum(deg, 1.0))
    hv = np.maximum(fv @ P["W_vin"].T + P["b_vin"], 0.0)
    hc = np.maximum(fc @ P["W_cin"].T + P["b_cin"], 0.0)
    cache = dict(fv=fv, fc=fc, isL=isL, isd=isd, hv0=hv, hc0=hc, layers=[])
    for l in (1, 2):
        ac = isL[:, None] * _agg_to_con(inst, hv)
        Xc = np.concatenate([hc, ac], axis=1)
        hc_new = np.maximum(q(Xc) @ q(P[f"W_c{l}"]).T + P[f"b_c{l}"], 0.0)
        av = isd[:, None] * _agg_to_var(inst, hc_new)
        Xv = np.concatenate([hv, av], axis=1)
        hv_new = np.maximum(q(Xv) @ q(P[f"W_v{l}"]).T + P[f"b_v{l}"], 0.0)
        cache["layers"].append(dict(Xc=Xc, hc=hc_new, Xv=Xv, hv=hv_new))
        hc, hv = hc_new, hv_new
    z = hv @ P["w_out"] + P["b_out"][0]
    cache["hv_last"] = hv
    return z, cache


def backward(inst, theta, cache, dz, emulate_bf16=True):
    """Gradient of sum_v dz_v z_v with respect to theta (flat)."""
    P = unflatten(theta)
    q = bf16 if emulate_bf16 else (lambda a: np.asarray(a, np.float64))
    G = {name: np.zeros(shape) for name, shape in PARAM_LAYOUT}
    dz = np.asarray(dz, np.float64)
    hv = cache["hv_last"]
    G["w_out"] = hv.T @ dz
    G["b_out"] = np.array([dz.sum()])
    dhv = np.outer(dz, P["w_out"])
    dhc = np.zeros((inst.m, HID))
    isL, isd = cache["isL"], cache["isd"]
    for l in (2, 1):
        lay = cache["layers"][l - 1]
        # variable update
        dpre = dhv * (lay["hv"] > 0)
        G[f"W_v{l}"] = q(dpre).T @ q(lay["Xv"])
        G[f"b_v{l}"] = dpre.sum(axis=0)
        dX = q(dpre) @ q(P[f"W_v{l}"])
        dhv = dX[:, :HID].copy()
        dav = dX[:, HID:]
        dhc = dhc + _agg_to_con(inst, dav, scale_src=isd)
        # constraint update
        dpre = dhc * (lay["hc"] > 0)
        G[f"W_c{l}"] = q(dpre).T @ q(lay["Xc"])
        G[f"b_c{l}"] = dpre.sum(axis=0)
        dX = q(dpre) @ q(P[f"W_c{l}"])
        dhc = dX[:, :HID].copy()
        dac = dX[:, HID:]
        dhv = dhv + _agg_to_var(inst, dac, scale_src=isL)
    dpre = dhv * (cache["hv0"] > 0)
    G["W_vin"] = dpre.T @ cache["fv"]
    G["b_vin"] = dpre.sum(axis=0)
    dpre = dhc * (cache["hc0"] > 0)
    G["W_cin"] = dpre.T @ cache["fc"]
    G["b_cin"] = dpre.sum(axis=0)
    return flatten(G)


def init_points(z, u, tau, fixed=None, fixed_val=None):
    x0 = np.tanh(np.asarray(z, np.float64)[:, None] + tau * np.asarray(u, np.float64))
    if fixed is not None:
        f = np.asarray(fixed).astype(bool)
        x0[f] = np.asarray(fixed_val, np.float64)[f][:, None]
    return x0


def softplus(a):
    return np.logaddexp(0.0, a)


def head_grad(z, x0, gx0, target, lam, fixed=None):
    """dJ/dz from dJ/dx0 (through the tanh) plus the target term."""
    z = np.asarray(z, np.float64)
    free = np.ones(len(z), bool) if fixed is None else ~np.asarray(fixed).astype(bool)
    dz = ((1.0 - x0 ** 2) * gx0).sum(axis=1)
    dz = np.where(free, dz, 0.0)
    if target is not None and lam != 0.0:
        t = np.asarray(target, np.float64)
        nf = max(1, int(free.sum()))
        sig = 1.0 / (1.0 + np.exp(2.0 * t * z))         # sigma(-2 t z)
        dz = dz + np.where(free, lam / nf * (-2.0 * t) * sig, 0.0)
    return dz


def target_loss(z, target, lam, fixed=None):
    free = np.ones(len(z), bool) if fixed is None else ~np.asarray(fixed).astype(bool)
    nf = max(1, int(free.sum()))
    return lam / nf * softplus(-2.0 * np.asarray(target, np.float64) * z)[free].sum()


def adam(theta, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, ICLR 2015), bias-corrected, FP64."""
    m = b1 * m + (1 - b1) * g
    v = b2 * v + (1 - b2) * g * g
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
