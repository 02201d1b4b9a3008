"""Learned initial points: the message-passing network of include/cls.h
(cls_mpnn_*) trained through the CLS objective, and its comparison with the
uniform initialisation.  The paper has no learned component; its CLS solver
starts from uniform random points, which remain the fallback and the judge.

Every numeric step runs in the CUDA library (network forward/backward on
tensor cores, objective and gradient, Adam, CLS steps); this module only
sequences the calls and keeps the tensors.

Training signal, per instance and step (R restarts, m constraints):
  J = 1/(R m) sum_r F(x0_r) + lam/n_free sum_v softplus(-2 t_v z_v)
with x0 = tanh(z + tau u) and t the signs of the best assignment the solver
itself reached from uniform starts (its local minimum).  The objective
term's gradient with respect to x0 comes through CLSObjective (the
torch.autograd.Function whose backward is the hand-written adjoint); the
head and network backward are the library's own kernels.
"""
import time

import numpy as np
import torch

from . import binding as B
from .api import Problem
from .autograd import CLSObjective


def _aligned(nbytes, device):
    buf = torch.empty(max(nbytes, 1) + 256, dtype=torch.uint8, device=device)
    off = (-buf.data_ptr()) % 256
    return buf[off:off + max(nbytes, 1)]


class GraphNet:
    """The network bound to one problem's incidence graph."""

    def __init__(self, problem: Problem):
        self.problem = problem
        self.handle = B.cls_mpnn_create(problem.handle)
        self.n_params, act_bytes = B.cls_mpnn_sizes(self.handle)
        self.act = _aligned(act_bytes, problem.device)
        self.n = problem.n

    def close(self):
        if getattr(self, "handle", None):
            B.cls_mpnn_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_params(self, seed):
        p = torch.empty(self.n_params, dtype=torch.float32, device=self.problem.device)
        B.cls_mpnn_param_init(self.handle, seed, p)
        return p

    def forward(self, params):
        z = torch.empty(self.n, dtype=torch.float32, device=self.problem.device)
        B.cls_mpnn_forward(self.handle, params, z, self.act)
        return z

    def points(self, z, R, seed, tau, r_offset=0):
        x0 = torch.empty((self.n, R), dtype=torch.float32, device=self.problem.device)
        B.cls_mpnn_points(self.handle, z, R, seed, r_offset, tau, x0)
        return x0

    def head_grad(self, z, x0, gx0, target=None, lam=0.0):
        dz = torch.empty_like(z)
        R = x0.shape[1] if x0 is not None else 0
        B.cls_mpnn_head_grad(self.handle, z, x0, gx0, R, target, lam, dz)
        return dz

    def backward(self, params, dz):
        dp = torch.empty_like(params)
        B.cls_mpnn_backward(self.handle, params, dz, dp, self.act)
        return dp


class Adam:
    def __init__(self, params, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, params, grads):
        self.t += 1
        B.cls_adam_step(params, grads, self.m, self.v, self.lr, self.b1, self.b2, self.eps, self.t)


def harvest_targets(problem: Problem, R=64, steps=200, lr=0.1, seed=7):
    """Signs (+-1, int8) of the best rounded assignment reached by `steps` CLS
    steps from R uniform starts: the method's own local minimum."""
    x = problem.init_uniform(R, seed)
    nsat, _, bits = problem.step(x, lr, n_steps=steps)
    best = int(torch.argmax(nsat).item())
    col = x[:, best]
    return torch.where(col < 0, -1, 1).to(torch.int8), int(nsat[best].item())


def train(entries, params, steps, R=32, lam=0.5, tau=1.0, lr=2e-3, seed=11, log_every=0):
    """entries: list of (Problem, GraphNet, targets).  Returns the loss log."""
    opt = Adam(params, lr=lr)
    log = []
    rng = np.random.default_rng(seed)
    for it in range(steps):
        p, net, tgt = entries[int(rng.integers(len(entries)))]
        z = net.forward(params)
        x0 = net.points(z, R, seed=seed * 100003 + it, tau=tau).requires_grad_(True)
        # the objective term through the autograd path: forward = FE and
        # literal partials, backward = the hand-written adjoint scaled by
        # d(mean objective / m)/dobj_r = 1/(R m)
        obj = CLSObjective.apply(p, x0)
        obj.backward(torch.full_like(obj, 1.0 / (R * p.m)))
        gx0 = x0.grad
        x0 = x0.detach()
        dz = net.head_grad(z, x0, gx0, tgt, lam)
        dp = net.backward(params, dz)
        opt.step(params, dp)
        if log_every and it % log_every == 0:
            log.append((it, float(obj.detach().mean().item()) / p.m))
    return log


def run_chunks(problem: Problem, x0, lr, steps, chunk=10):
    """`steps` CLS steps from x0 in chunks of `chunk`, with no host
    synchronisation inside: each chunk's satisfied counts land in one row of
    a device buffer and a CUDA event is recorded after it.  Returns (x after
    the run, median satisfied fraction per chunk, device seconds from the
    start to the end of each chunk)."""
    x = x0.clone()
    R = x.shape[1]
    K = max(1, steps // chunk)
    nsat = torch.empty((K, R), dtype=torch.int32, device=x.device)
    ws = problem.workspace(R)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    evs[0].record()
    for k in range(K):
        B.cls_step(problem.handle, R, x, lr, chunk, None, nsat[k], None, ws)
        evs[k + 1].record()
    torch.cuda.synchronize()
    med = (torch.median(nsat.float(), dim=1).values / problem.m).cpu().numpy()
    secs = np.array([evs[0].elapsed_time(evs[k + 1]) / 1e3 for k in range(K)])
    return x, med, secs


def _first_reach(med, frac):
    hit = np.nonzero(med >= frac)[0]
    return int(hit[0]) if len(hit) else None


def time_to_fraction(problem: Problem, x0, frac, lr=0.1, max_steps=500, chunk=10):
    """Steps and device seconds (CUDA events) until the median over restarts
    of the satisfied fraction reaches `frac`, checked after every chunk;
    (None, None) if it does not within max_steps."""
    _, med, secs = run_chunks(problem, x0, lr, max_steps, chunk)
    k = _first_reach(med, frac)
    return (None, None) if k is None else ((k + 1) * chunk, float(secs[k]))


def median_fraction_after(problem: Problem, x0, steps, lr=0.1):
    x = x0.clone()
    nsat, _, _ = problem.step(x, lr, n_steps=steps, bits=False)
    return float(torch.median(nsat.float()).item()) / problem.m


def compare(entries, params, R=1024, S=500, tau=1.0, lr=0.1, seed=99, chunk=10):
    """Learned vs uniform initialisation on held-out instances.

    tau_i = median over restarts of the satisfied fraction that uniform
    starts reach after S steps on instance i.  One uniform run of S steps
    gives both tau_i and the uniform time: the device time until the median,
    checked every `chunk` steps, first reaches tau_i.  The learned time is
    the network forward + points (device time) plus the steps from the
    network's points until the median reaches tau_i (runs of S steps, at
    most 4 S in all).  Returns per-instance records."""
    out = []
    for i, (p, net, _) in enumerate(entries):
        xu = p.init_uniform(R, seed + i)
        _, med_u, secs_u = run_chunks(p, xu, lr, S, chunk)
        tau_i = float(med_u[-1])
        ku = _first_reach(med_u, tau_i)
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record()
        z = net.forward(params)
        xl = net.points(z, R, seed + i, tau)
        t1.record()
        torch.cuda.synchronize()
        t_inf = t0.elapsed_time(t1) / 1e3
        steps_l, t_l, done, elapsed = None, None, 0, 0.0
        while done < 4 * S:
            xl, med_l, secs_l = run_chunks(p, xl, lr, S, chunk)
            kl = _first_reach(med_l, tau_i)
            if kl is not None:
                steps_l, t_l = done + (kl + 1) * chunk, elapsed + float(secs_l[kl])
                break
            done += S
            elapsed += float(secs_l[-1])
        out.append(dict(instance=i, n=p.n, m=p.m, tau=tau_i, steps_uniform=(ku + 1) * chunk,
                        s_uniform=float(secs_u[ku]), steps_learned=steps_l,
                        s_learned=None if t_l is None else t_l + t_inf, s_inference=t_inf))
    return out


def build_entries(instances, harvest_R=64, harvest_steps=200, lr=0.1):
    entries = []
    for k, inst in enumerate(instances):
        p = Problem(inst)
        net = GraphNet(p)
        tgt, _ = harvest_targets(p, harvest_R, harvest_steps, lr, seed=1000 + k)
        entries.append((p, net, tgt))
    return entries
