"""cls_step_noalloc: the step entry point that allocates nothing.

It serves callers that cannot allocate device memory while running (real-time
loops, processes held to a fixed device-memory budget, host languages with no
route to cudaMalloc); its scratch is a fixed 32 MiB device array inside the
library.  This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import workloads as W

pytestmark = pytest.mark.gpu


def _p(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("make", [
    lambda: W.random_ksat(),                                         # 3-SAT, closed forms
    lambda: W.mixed_pb(n=400, n_or=900, n_xor=90, n_card=20, card_len=(10, 120), seed=6),
])
def test_noalloc_step_matches_workspace_step(make):
    from paper_2606_06656_b300 import Problem, _lib
    from paper_2606_06656_b300 import binding as B
    lib = _lib.load()
    inst = make()
    p = Problem(inst)
    R, lr, steps = 64, 0.1, 5
    X0 = W.uniform_points(inst.n, R, seed=3)
    xa = torch.from_numpy(X0.copy()).cuda()
    xb = xa.clone()
    RW = (R + 31) // 32
    for _ in range(2):                      # two calls in a row share the array
        ba = torch.empty((inst.n, RW), dtype=torch.int32, device="cuda")
        bb = torch.empty_like(ba)
        na = torch.empty(R, dtype=torch.int32, device="cuda")
        nb = torch.empty_like(na)
        wa = torch.empty(R, dtype=torch.float64, device="cuda")
        wb = torch.empty_like(wa)
        B.cls_step(p.handle, R, xa, lr, steps, ba, na, wa, p.workspace(R))
        rc = lib.cls_step_noalloc(p.handle, R, _p(xb), C.c_float(lr), steps, _p(bb), _p(nb),
                                  _p(wb), _stream())
        assert rc == 0, lib.cls_last_error()
        torch.cuda.synchronize()
        assert torch.equal(xa, xb)           # same kernels, same inputs: same bits
        assert torch.equal(na, nb) and torch.equal(ba, bb)
        assert torch.equal(wa, wb)


def test_noalloc_rejects_oversized_problem():
    from paper_2606_06656_b300 import Problem, _lib
    lib = _lib.load()
    inst = W.mixed_pb(n=2000, n_or=8000, n_xor=800, n_card=200, seed=7)
    p = Problem(inst)
    R = 1024                                 # partials alone exceed 32 MiB
    x = torch.zeros((inst.n, R), dtype=torch.float32, device="cuda")
    n = torch.empty(R, dtype=torch.int32, device="cuda")
    rc = lib.cls_step_noalloc(p.handle, R, _p(x), C.c_float(0.1), 1, None, _p(n), None,
                              _stream())
    assert rc == -5
    assert b"static limit" in lib.cls_last_error()
