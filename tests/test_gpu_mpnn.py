"""Learned initialiser on the GPU vs the FP64 oracle (oracle/mpnn.py).

The oracle rounds the operands of the tensor-core products to bf16 exactly as
the kernels do, so the remaining differences are FP32 accumulation order and
(rarely) a bf16 rounding or ReLU decision flipped by it; the tolerances are
relative to the norm of each tensor: 1e-3 for the forward and 2e-3 for the
gradients.
"""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cls as ocls
from oracle import mpnn as om

pytestmark = pytest.mark.gpu


def _inst(seed=3):
    return W.mixed_pb(n=300, n_or=700, n_xor=70, n_card=15, card_len=(10, 80), seed=seed)


def _theta(seed=1, scale=0.15):
    return np.random.default_rng(seed).normal(0, scale, om.N_PARAMS).astype(np.float32)


def _net(inst):
    from paper_2606_06656_b300 import Problem
    from paper_2606_06656_b300.learned import GraphNet
    p = Problem(inst)
    return p, GraphNet(p)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-30))


def test_param_layout_matches_oracle():
    inst = _inst()
    _, net = _net(inst)
    assert net.n_params == om.N_PARAMS


@pytest.mark.parametrize("seed", [3, 4])
def test_forward_matches_oracle(seed):
    inst = _inst(seed)
    _, net = _net(inst)
    th = _theta(seed)
    z = net.forward(torch.from_numpy(th).cuda()).cpu().numpy()
    zo, _ = om.forward(inst, th.astype(np.float64), emulate_bf16=True)
    assert _rel(z, zo) <= 1e-3, _rel(z, zo)
    assert np.std(zo) > 1e-3             # a non-degenerate network


def test_backward_matches_oracle():
    inst = _inst(5)
    _, net = _net(inst)
    th = _theta(5)
    dz = np.random.default_rng(6).normal(size=inst.n).astype(np.float32)
    params = torch.from_numpy(th).cuda()
    net.forward(params)
    dp = net.backward(params, torch.from_numpy(dz).cuda()).cpu().numpy()
    _, cache = om.forward(inst, th.astype(np.float64), emulate_bf16=True)
    dpo = om.backward(inst, th.astype(np.float64), cache, dz.astype(np.float64), emulate_bf16=True)
    off = 0
    for name, shape in om.PARAM_LAYOUT:
        k = int(np.prod(shape))
        r = _rel(dp[off:off + k], dpo[off:off + k])
        assert r <= 2e-3, (name, r)
        off += k


def test_points_and_head_grad_match_oracle():
    inst = W.partial_assignment(_inst(7), 0.3)
    _, net = _net(inst)
    R, tau, seed = 40, 0.8, 12
    z = np.random.default_rng(8).normal(size=inst.n).astype(np.float32)
    x0 = net.points(torch.from_numpy(z).cuda(), R, seed, tau).cpu().numpy()
    u = ocls.init_uniform(inst.n, R, seed).astype(np.float64)      # same draws, same convention
    want = om.init_points(z, u, tau, inst.fixed, inst.fixed_val)
    free = inst.fixed == 0
    assert np.abs(x0[free] - want[free]).max() <= 2e-6
    assert np.array_equal(x0[~free], want[~free].astype(np.float32))
    gx0 = np.random.default_rng(9).normal(size=(inst.n, R)).astype(np.float32)
    t = np.where(np.random.default_rng(10).random(inst.n) < 0.5, -1, 1).astype(np.int8)
    dz = net.head_grad(torch.from_numpy(z).cuda(), torch.from_numpy(x0).cuda(),
                       torch.from_numpy(gx0).cuda(), torch.from_numpy(t).cuda(), 0.4).cpu().numpy()
    dzo = om.head_grad(z.astype(np.float64), x0.astype(np.float64), gx0.astype(np.float64),
                       t, 0.4, inst.fixed)
    assert np.abs(dz - dzo).max() <= 1e-4 * max(1.0, np.abs(dzo).max())


def test_adam_matches_oracle():
    from paper_2606_06656_b300.learned import Adam
    rng = np.random.default_rng(11)
    th = rng.normal(size=1000).astype(np.float32)
    p = torch.from_numpy(th.copy()).cuda()
    opt = Adam(p, lr=1e-2)
    m = np.zeros(1000)
    v = np.zeros(1000)
    tho = th.astype(np.float64)
    for step in range(1, 6):
        g = rng.normal(size=1000).astype(np.float32)
        opt.step(p, torch.from_numpy(g).cuda())
        tho, m, v = om.adam(tho, g.astype(np.float64), m, v, step, 1e-2)
    assert np.abs(p.cpu().numpy() - tho).max() <= 1e-5


def test_param_init_distribution():
    inst = _inst()
    _, net = _net(inst)
    p = net.init_params(5).cpu().numpy()
    off = 0
    for name, shape in om.PARAM_LAYOUT:
        k = int(np.prod(shape))
        block = p[off:off + k]
        if name.startswith("W") or name == "w_out":
            a = 1.0 / np.sqrt(shape[-1] if len(shape) == 2 else 64)
            assert np.all(np.abs(block) <= a * (1 + 1e-6)) and np.std(block) > 0.3 * a
        off += k
    p2 = net.init_params(5).cpu().numpy()
    assert np.array_equal(p, p2)


def test_training_reduces_loss_and_objective():
    """A few hundred Adam steps through the CLS objective lower the mean
    objective at the network's initial points on the training instances."""
    from paper_2606_06656_b300.learned import build_entries, train
    insts = W.mixed_instances(6, n_range=(300, 500), seed=77)
    entries = build_entries(insts, harvest_R=32, harvest_steps=100)
    params = entries[0][1].init_params(3)

    def mean_obj(params):
        vals = []
        for p, net, _ in entries:
            z = net.forward(params)
            x0 = net.points(z, 64, seed=5, tau=1.0)
            obj, _, _ = p.eval(x0, obj=True, grad=False)
            vals.append(float(obj.mean().item()) / p.m)
        return float(np.mean(vals))

    before = mean_obj(params)
    train(entries, params, steps=300, R=32, lam=0.5, tau=1.0, lr=3e-3)
    after = mean_obj(params)
    assert after < before - 0.02, (before, after)


def test_training_gradient_flows_through_autograd_objective(monkeypatch):
    """learned.train differentiates the CLS objective through CLSObjective:
    its backward (the hand-written adjoint) runs once per training step, and
    the gradient it returns is the oracle-checked objective gradient scaled
    by 1/(R m)."""
    from paper_2606_06656_b300 import autograd as AG
    from paper_2606_06656_b300.learned import build_entries, train
    calls = []
    orig = AG.CLSObjective.backward

    def counting(ctx, gout):
        calls.append(float(gout[0].item()))
        return orig(ctx, gout)

    monkeypatch.setattr(AG.CLSObjective, "backward", staticmethod(counting))
    insts = W.mixed_instances(2, n_range=(200, 300), seed=78)
    entries = build_entries(insts, harvest_R=8, harvest_steps=10)
    params = entries[0][1].init_params(3)
    train(entries, params, steps=5, R=16, lam=0.5, tau=1.0, lr=1e-3)
    assert len(calls) == 5
    ms = {p.m for p, _, _ in entries}
    assert all(any(abs(c * 16 * m - 1.0) < 1e-6 for m in ms) for c in calls)


def test_learned_initialisation_gains_over_uniform():
    """Trained on planted mixed instances through the CLS objective, the
    network's initial points reach the satisfied fraction that uniform starts
    reach after 100 steps in fewer steps, on held-out instances."""
    from paper_2606_06656_b300 import learned as Lr
    train = W.mixed_instances(20, n_range=(600, 900), seed=1400)
    held = W.mixed_instances(3, n_range=(600, 900), seed=91400)
    tr = Lr.build_entries(train, harvest_R=64, harvest_steps=150)
    te = Lr.build_entries(held, harvest_R=8, harvest_steps=1)
    params = tr[0][1].init_params(3)
    Lr.train(tr, params, steps=800, R=32, lam=0.5, tau=1.0, lr=2e-3)
    res = Lr.compare(te, params, R=256, S=100, tau=1.0)
    gain = 0
    for r in res:
        assert r["steps_learned"] is not None
        gain += r["steps_learned"] < r["steps_uniform"]
    assert gain >= 2, res
    # wall-clock on the device, network inference included
    assert np.median([r["s_learned"] for r in res]) < np.median([r["s_uniform"] for r in res]), res
    f0u = np.median([Lr.median_fraction_after(p, p.init_uniform(256, 5), 1) for p, _, _ in te])
    f0l = np.median([Lr.median_fraction_after(p, n.points(n.forward(params), 256, 5, 1.0), 1)
                     for p, n, _ in te])
    assert f0l > f0u, (f0l, f0u)
