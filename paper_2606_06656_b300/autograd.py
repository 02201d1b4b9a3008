"""CLSObjective: the per-restart CLS objective as a torch.autograd.Function.

    obj = CLSObjective.apply(problem, x)       # x: (n, R) float32 CUDA tensor
    obj.sum().backward()                        # x.grad = dF/dx, restart by restart

Forward runs the fused FE + literal-partial kernels and the variable-major
gradient accumulation (cls_eval), returning obj[r] = sum_c w_c FE_c(x_r)
(Sec. 2.3, Eq. 5) and keeping the gradient.  Backward is the hand-written
adjoint: the saved gradient scaled restart by restart by dLoss/dobj
(cls_restart_scale).  The objective is multilinear in x, so its gradient is
exact up to FP32 rounding; no autograd graph is built through the kernels.
"""
import torch

from . import binding as B


class CLSObjective(torch.autograd.Function):
    @staticmethod
    def forward(ctx, problem, x):
        R = problem._x(x)
        obj = torch.empty(R, dtype=torch.float32, device=x.device)
        grad = torch.empty_like(x)
        B.cls_eval(problem.handle, R, x.contiguous(), obj, grad, None, problem.workspace(R))
        ctx.problem = problem
        ctx.save_for_backward(grad)
        return obj

    @staticmethod
    def backward(ctx, gout):
        (grad,) = ctx.saved_tensors
        p = ctx.problem
        R = grad.shape[1]
        out = torch.empty_like(grad)
        B.cls_restart_scale(p.handle, R, grad, gout.contiguous().float(), out)
        return None, out


def cls_objective(problem, x):
    return CLSObjective.apply(problem, x)
