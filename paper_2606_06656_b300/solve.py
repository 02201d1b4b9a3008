"""Command-line solver: parallel continuous local search on a DIMACS CNF or
OPB file (Sec. 3.3: R restarts advance in lockstep; a restart whose best
count has not improved for `patience` steps is given a fresh point).

    python -m paper_2606_06656_b300.solve formula.cnf --restarts 4096 --steps 2000

Prints "s SATISFIABLE" and a "v" line (DIMACS: signed variable numbers
ending in 0; OPB: x<i> / -x<i>) as soon as one restart's rounded point
satisfies every constraint, else "s UNKNOWN" and the fewest unsatisfied
constraints seen.  Every step runs on the GPU (cls_step, cls_track_step,
cls_refill); the host only reads the best count once per check interval.
"""
import argparse
import sys
import time

import numpy as np

from .formats import read_dimacs, read_opb


def read_any(path):
    with open(path) as f:
        text = f.read()
    for line in text.splitlines():
        s = line.strip()
        if not s or s[0] in "c%*":
            continue
        if s.startswith("p cnf"):
            return read_dimacs(text, name=path), "dimacs"
        break
    return read_opb(text, name=path), "opb"


def solve(inst, restarts=1024, steps=1000, lr=0.1, seed=1, patience=50,
          refill_every=10, check_every=1, deadline=None, reweight=0.0):
    """Runs the loop; returns (solved, assignment or None, best unsatisfied
    count, steps run).  assignment[v] is True where variable v is True.
    reweight > 0: every refill_every steps the constraint weights are
    updated from the batch's statistics (cls_reweight with eta = reweight,
    kappa 4, w_max 10), raising often-violated constraints with weak
    gradients (Sec. 3.1)."""
    import torch
    from .api import Problem
    from . import binding as B
    p = Problem(inst)
    R = int(restarts)
    x = p.init_uniform(R, seed)
    ws = p.workspace(R)
    dev = x.device
    nsat = torch.empty(R, dtype=torch.int32, device=dev)
    wsat = torch.empty(R, dtype=torch.float64, device=dev)
    bits = torch.empty((inst.n, (R + 31) // 32), dtype=torch.int32, device=dev)
    trk = torch.empty((4, R), dtype=torch.int32, device=dev)
    cnt = torch.zeros(1, dtype=torch.int32, device=dev)
    B.cls_track_reset(p.handle, R, trk)
    m, gen, best = inst.m, 0, -1
    for k in range(steps):
        B.cls_step(p.handle, R, x, lr, 1, bits, nsat, wsat, ws)
        B.cls_track_step(p.handle, R, nsat, k, trk)
        if (k + 1) % check_every == 0 or k + 1 == steps:
            top, r = torch.max(nsat, dim=0)
            top = int(top)
            best = max(best, top)
            if top == m:
                r = int(r)
                word = bits[:, r // 32].cpu().numpy().view(np.uint32)
                return True, ((word >> np.uint32(r % 32)) & 1).astype(bool), 0, k + 1
            if deadline is not None and time.monotonic() > deadline:
                return False, None, m - best, k + 1
        if (k + 1) % refill_every == 0:
            if reweight > 0:
                g, u = p.constraint_stats(bits, R)
                p.reweight(g, u, R, reweight)
            gen += 1
            B.cls_refill(p.handle, R, x, trk, patience, seed, 0, gen, cnt)
    return False, None, m - best, steps


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("file")
    ap.add_argument("--restarts", type=int, default=1024)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--lr", type=float, default=0.1)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--patience", type=int, default=50)
    ap.add_argument("--check-every", type=int, default=1)
    ap.add_argument("--time-limit", type=float, default=0.0, help="seconds (0 = none)")
    ap.add_argument("--reweight", type=float, default=0.0,
                    help="adaptive constraint weighting rate eta (0 = off)")
    a = ap.parse_args(argv)
    inst, kind = read_any(a.file)
    print(f"c {kind}: n={inst.n} m={inst.m} literals={inst.nnz} dropped={inst.dropped}")
    for note in inst.notes:
        print(f"c {note}")
    t0 = time.monotonic()
    ok, asg, unsat, k = solve(inst, a.restarts, a.steps, a.lr, a.seed, a.patience,
                              check_every=a.check_every,
                              deadline=t0 + a.time_limit if a.time_limit > 0 else None,
                              reweight=a.reweight)
    print(f"c steps={k} time={time.monotonic() - t0:.3f}s")
    if not ok:
        print(f"c fewest unsatisfied constraints: {unsat}")
        print("s UNKNOWN")
        return 0
    print("s SATISFIABLE")
    if kind == "dimacs":
        lits = [str(v + 1) if asg[v] else str(-(v + 1)) for v in range(inst.n)]
        print("v " + " ".join(lits) + " 0")
    else:
        print("v " + " ".join(f"x{v + 1}" if asg[v] else f"-x{v + 1}" for v in range(inst.n)))
    return 10


if __name__ == "__main__":
    sys.exit(main())
