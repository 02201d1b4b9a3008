"""Pins for the FP64 message-passing oracle (the learned initialiser).

The model is not from the paper, so it is pinned against its own definition
by routes other than its code: central finite differences of the forward
(which pin the hand-written backward), a tiny graph evaluated by hand,
equivariance under relabelling variables and constraints, and the bf16
rounding rule against torch's own bfloat16 conversion.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import mpnn as om


def small_instance(seed=0, n=14, m=18):
    rng = np.random.default_rng(seed)
    types = [W.TYPE_OR, W.TYPE_XOR, W.TYPE_CARD_GE, W.TYPE_CARD_LE, W.TYPE_NAE,
             W.TYPE_EO, W.TYPE_EK, W.TYPE_AMO]
    return W.random_constraint_set(rng, n, m, types, (2, 6), weights="random")


def rand_theta(seed=1, scale=0.4):
    return np.random.default_rng(seed).normal(0, scale, om.N_PARAMS)


def test_param_count():
    assert om.N_PARAMS == 64 * 4 + 64 + 64 * 12 + 64 + 4 * (64 * 128 + 64) + 64 + 1


@pytest.mark.parametrize("emulate", [False, True])
def test_backward_matches_central_differences(emulate):
    inst = small_instance()
    theta = rand_theta()
    rng = np.random.default_rng(3)
    dz = rng.normal(size=inst.n)
    z, cache = om.forward(inst, theta, emulate_bf16=False)
    g = om.backward(inst, theta, cache, dz, emulate_bf16=False)
    eps = 1e-6
    for _ in range(12):
        d = rng.normal(size=om.N_PARAMS)
        zp, _ = om.forward(inst, theta + eps * d, emulate_bf16=False)
        zm, _ = om.forward(inst, theta - eps * d, emulate_bf16=False)
        fd = (dz @ zp - dz @ zm) / (2 * eps)
        assert abs(fd - g @ d) <= 1e-6 * max(1.0, abs(fd)), (fd, g @ d)
    if emulate:     # with bf16 operands the gradient is a bf16-rounded version
        g2 = om.backward(inst, theta, cache, dz, emulate_bf16=True)
        assert np.linalg.norm(g2 - g) <= 2e-2 * np.linalg.norm(g)


def test_tiny_graph_by_hand():
    """One OR clause (x0 or not x1): every weight zero except a few, so the
    forward can be written out by hand."""
    inst = W.build(2, [(W.TYPE_OR, 0, np.array([0, 1], np.int32), np.array([1, -1], np.int8))])
    P = {name: np.zeros(shape) for name, shape in om.PARAM_LAYOUT}
    P["W_vin"][0, 0] = 1.0            # h_v[0] = relu(1 * f_v[0]) = 1
    P["W_cin"][0, 0] = 2.0            # h_c[0] = relu(2 * onehot_OR) = 2
    P["W_c1"][0, 64] = 1.0            # h_c1[0] = relu(a_c[0]) with a_c = (1 - 1)/sqrt2 = 0
    P["b_c1"][0] = 0.5                # -> 0.5
    P["W_v1"][0, 64] = 1.0            # h_v1[0] = relu(a_v[0]) = relu(s_e * 0.5)
    P["W_c2"][0, 0] = 1.0             # h_c2[0] = relu(h_c1[0]) = 0.5
    P["W_v2"][0, 0] = 1.0             # h_v2[0] = relu(h_v1[0])
    P["W_v2"][1, 64] = 3.0            # h_v2[1] = relu(3 * a_v[0]) = relu(3 s_e 0.5)
    P["w_out"][0], P["w_out"][1] = 1.0, 1.0
    P["b_out"][0] = -0.25
    z, _ = om.forward(inst, om.flatten(P), emulate_bf16=False)
    # variable 0 (positive literal): h_v1 = 0.5, a_v2 = +0.5 -> z = 0.5 + 1.5 - 0.25
    # variable 1 (negated literal): h_v1 = 0,   a_v2 = -0.5 -> z = 0 + 0 - 0.25
    assert np.allclose(z, [1.75, -0.25])


def test_equivariance_under_relabelling():
    inst = small_instance(seed=5)
    theta = rand_theta(seed=6)
    z, _ = om.forward(inst, theta, emulate_bf16=False)
    rng = np.random.default_rng(7)
    pv = rng.permutation(inst.n)           # new index of old variable v
    pc = rng.permutation(inst.m)           # constraint order
    rows = []
    for c in pc:
        a, b = inst.offsets[c], inst.offsets[c + 1]
        rows.append((int(inst.ctype[c]), int(inst.k[c]), pv[inst.lit_var[a:b]].astype(np.int32),
                     inst.lit_sign[a:b].copy()))
    inst2 = W.build(inst.n, rows, weights=inst.weight[pc])
    z2, _ = om.forward(inst2, theta, emulate_bf16=False)
    assert np.allclose(z2[pv], z, atol=1e-12)


def test_bf16_rounding_matches_torch():
    rng = np.random.default_rng(0)
    a = np.concatenate([rng.normal(size=2000) * 10 ** rng.uniform(-8, 8, 2000),
                        [0.0, -0.0, 1.0, 1.00390625, 1.01171875, 3.3895e38]])
    want = torch.from_numpy(a.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(om.bf16(a), want)


def test_head_grad_matches_differences():
    rng = np.random.default_rng(2)
    n, R = 9, 6
    z = rng.normal(size=n)
    u = rng.uniform(-1, 1, (n, R))
    t = np.where(rng.random(n) < 0.5, -1.0, 1.0)
    gx0 = rng.normal(size=(n, R))
    fixed = np.zeros(n, np.uint8)
    fixed[2] = 1
    fv = np.zeros(n)
    fv[2] = 1.0

    def J(zz):
        x0 = om.init_points(zz, u, 0.7, fixed, fv)
        return (gx0 * x0).sum() + om.target_loss(zz, t, 0.3, fixed)

    x0 = om.init_points(z, u, 0.7, fixed, fv)
    dz = om.head_grad(z, x0, gx0, t, 0.3, fixed)
    for v in range(n):
        e = np.zeros(n)
        e[v] = 1e-6
        assert abs((J(z + e) - J(z - e)) / 2e-6 - dz[v]) < 1e-6


def test_adam_matches_torch():
    rng = np.random.default_rng(4)
    th = rng.normal(size=50)
    tt = torch.tensor(th, requires_grad=True)
    opt = torch.optim.Adam([tt], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros(50)
    v = np.zeros(50)
    for step in range(1, 6):
        g = rng.normal(size=50)
        tt.grad = torch.tensor(g)
        opt.step()
        th, m, v = om.adam(th, g, m, v, step, 1e-2)
    assert np.allclose(th, tt.detach().numpy(), atol=1e-12)
