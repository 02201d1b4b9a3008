"""Ramsey balanced-colouring instances (Sec. 3.1) on the CUDA path: FE and
gradient against the FP64 oracle (1e-4 per constraint / of the gradient's
norm), counts bit-exact at the plant and at single-edge changes of it."""
import numpy as np
import pytest
import torch

import workloads as W
from oracle import cls as ocls

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("V,C,red", [(16, 3, False), (16, 3, True), (16, 5, True), (16, 4, False)])
def test_ramsey_parity(V, C, red):
    from paper_2606_06656_b300 import Problem
    inst = W.ramsey_balanced(V, C, redundant=red)
    p = Problem(inst)
    # FP32 floor near corners, where the exact gradient can be tiny: a few
    # L*u per DFT literal partial (EO and CARD_GE are both evaluated at the
    # roots of unity), summed over each variable's constraints
    L = np.diff(inst.offsets).astype(np.float64)
    per_var = np.zeros(inst.n)
    np.add.at(per_var, inst.lit_var, np.repeat(4.0 * L * 2.0 ** -24, L.astype(int)))
    floor = float(np.linalg.norm(per_var))
    for X, fl in ((W.uniform_points(inst.n, 70, seed=V + C), 0.0),
                  (W.near_corner_points(inst.n, 40, seed=3), floor)):
        x = torch.from_numpy(np.ascontiguousarray(X)).cuda()
        obj, grad, fe = p.eval(x, obj=True, grad=True, fe_con=True)
        torch.cuda.synchronize()
        oobj, ograd, ofe = ocls.objective_grad(inst, X.astype(np.float64))
        assert np.max(np.abs(fe.cpu().numpy() - ofe)) <= 1e-4
        g = grad.cpu().numpy()
        assert (np.linalg.norm(g - ograd, axis=0)
                <= 1e-4 * np.linalg.norm(ograd, axis=0) + fl + 1e-30).all()
        assert np.max(np.abs(obj.cpu().numpy() - oobj)) <= 1e-4 * inst.m


def test_ramsey_counts_at_plant_and_changes():
    from paper_2606_06656_b300 import Problem
    for red in (False, True):
        inst = W.ramsey_balanced(16, 3, redundant=red)
        base = inst.plant.astype(np.float32)
        rng = np.random.default_rng(5)
        cols = [base]
        for _ in range(63):
            x = base.copy()
            flip = rng.choice(inst.n, size=int(rng.integers(1, 6)), replace=False)
            x[flip] = -x[flip]
            cols.append(x)
        X = np.stack(cols, axis=1)
        p = Problem(inst)
        nsat, _, _ = p.round_score(torch.from_numpy(X).cuda())
        onsat, _, _ = ocls.score(inst, X)
        assert np.array_equal(nsat.cpu().numpy(), onsat)
        assert onsat[0] == inst.m
