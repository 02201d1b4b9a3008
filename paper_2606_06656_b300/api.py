"""Problem handle with torch-managed device memory.

    p = Problem(instance)                 # cls_problem_create
    x = p.init_uniform(R, seed)           # (n, R) float32 on the device
    obj, grad, fe = p.eval(x, fe_con=True)
    nsat, wsat, bits = p.step(x, lr=0.1, n_steps=200)

All arithmetic runs in libcls_b300.so; this class only allocates tensors
(outputs and the workspace) and passes pointers.
"""
import torch

from . import binding as B


class Problem:
    def __init__(self, inst, device=None, simplify_fixed=False):
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.handle = B.cls_problem_create(
                inst, B.CLS_SIMPLIFY_FIXED if simplify_fixed else 0)
        info = B.cls_problem_info(self.handle)
        self.info = info
        self.n, self.m, self.nnz = info["n"], info["m"], info["nnz"]
        self._ws = {}

    def close(self):
        if getattr(self, "handle", None):
            B.cls_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- memory ---------------------------------------------------------
    def workspace(self, R, host_solve=False):
        key = (int(R), bool(host_solve))
        ws = self._ws.get(key)
        if ws is None:
            nbytes = (B.cls_solve_host_workspace_size(self.handle, R) if host_solve
                      else B.cls_workspace_size(self.handle, R))
            ws = torch.empty(max(nbytes, 1) + 256, dtype=torch.uint8, device=self.device)
            off = (-ws.data_ptr()) % 256
            ws = ws[off:off + max(nbytes, 1)]
            self._ws[key] = ws
        return ws

    def _x(self, x):
        if not (x.is_cuda and x.dtype == torch.float32 and x.is_contiguous()
                and x.dim() == 2 and x.shape[0] == self.n):
            raise ValueError("x must be a contiguous float32 CUDA tensor of shape (n, R)")
        return x.shape[1]

    # -- calls ----------------------------------------------------------
    def init_uniform(self, R, seed, r_offset=0, out=None):
        x = out if out is not None else torch.empty((self.n, R), dtype=torch.float32,
                                                    device=self.device)
        B.cls_init_uniform(self.handle, R, seed, r_offset, x)
        return x

    def eval(self, x, obj=True, grad=True, fe_con=False):
        R = self._x(x)
        o = torch.empty(R, dtype=torch.float32, device=self.device) if obj else None
        g = torch.empty_like(x) if grad else None
        f = torch.empty((self.m, R), dtype=torch.float32, device=self.device) if fe_con else None
        B.cls_eval(self.handle, R, x, o, g, f, self.workspace(R))
        return o, g, f

    def pgd_update(self, x, grad, lr, bits=True):
        R = self._x(x)
        b = torch.empty((self.n, (R + 31) // 32), dtype=torch.int32, device=self.device) \
            if bits else None
        B.cls_pgd_update(self.handle, R, x, grad, lr, b)
        return b

    def round_score(self, x):
        R = self._x(x)
        b = torch.empty((self.n, (R + 31) // 32), dtype=torch.int32, device=self.device)
        nsat = torch.empty(R, dtype=torch.int32, device=self.device)
        wsat = torch.empty(R, dtype=torch.float64, device=self.device)
        B.cls_round_score(self.handle, R, x, b, nsat, wsat, self.workspace(R))
        return nsat, wsat, b

    def step(self, x, lr, n_steps=1, bits=True, score=True):
        R = self._x(x)
        b = torch.empty((self.n, (R + 31) // 32), dtype=torch.int32, device=self.device) \
            if bits else None
        nsat = torch.empty(R, dtype=torch.int32, device=self.device) if score else None
        wsat = torch.empty(R, dtype=torch.float64, device=self.device) if score else None
        B.cls_step(self.handle, R, x, lr, n_steps, b, nsat, wsat, self.workspace(R))
        return nsat, wsat, b

    def step_persistent(self, x, lr, n_steps=1, bits=True, score=True):
        """Same results as step(), the whole loop in one cooperative launch
        (problems whose FE work is all short closed forms).  Raises if a
        grid barrier timed out."""
        R = self._x(x)
        b = torch.empty((self.n, (R + 31) // 32), dtype=torch.int32, device=self.device) \
            if bits else None
        nsat = torch.empty(R, dtype=torch.int32, device=self.device) if score else None
        wsat = torch.empty(R, dtype=torch.float64, device=self.device) if score else None
        ws = self.workspace(R)
        B.cls_step_persistent(self.handle, R, x, lr, n_steps, b, nsat, wsat, ws)
        if n_steps > 0 and R > 0 and B.cls_persistent_status(self.handle, R, ws) != 0:
            raise RuntimeError("cls_step_persistent: a grid barrier timed out")
        return nsat, wsat, b

    def solve_host(self, x0_host, lr, n_steps, nsat_host, x_host=None):
        """x0_host: (n, R) float32 CPU tensor (pinned for async copies)."""
        R = x0_host.shape[1]
        B.cls_solve_host(self.handle, R, x0_host, lr, n_steps, nsat_host, x_host,
                         self.workspace(R, host_solve=True))
        return nsat_host

    # -- per-restart tracking and refills (Sec. 3.3) ----------------------
    def track_reset(self, R, trk=None):
        """Tracking state int32[4, R]: best count, its step, steps since the
        last improvement, first solved step."""
        t = trk if trk is not None else torch.empty((4, R), dtype=torch.int32,
                                                     device=self.device)
        B.cls_track_reset(self.handle, R, t)
        return t

    def track_step(self, nsat, step, trk):
        B.cls_track_step(self.handle, trk.shape[1], nsat, step, trk)

    def refill(self, x, trk, patience, seed, generation, count, r_offset=0):
        B.cls_refill(self.handle, self._x(x), x, trk, patience, seed, r_offset, generation, count)

    # -- adaptive constraint weighting (Sec. 3.1) -------------------------
    def constraint_stats(self, bits, R):
        """(gnorm float64[m], unsat int32[m]) from the partials of the last
        eval/step with R restarts and the bitset of the rounded points."""
        g = torch.empty(self.m, dtype=torch.float64, device=self.device)
        u = torch.empty(self.m, dtype=torch.int32, device=self.device)
        B.cls_constraint_stats(self.handle, R, bits, self.workspace(R), g, u)
        return g, u

    def reweight(self, gnorm, unsat, R, eta, kappa=4.0, w_max=10.0):
        """New weights (float32[m]) from constraint_stats' output; they also
        become the problem's weights."""
        w = torch.empty(self.m, dtype=torch.float32, device=self.device)
        B.cls_reweight(self.handle, R, gnorm, unsat, eta, kappa, w_max, w)
        return w

    def set_weights(self, w):
        if not (w.is_cuda and w.dtype == torch.float32 and w.is_contiguous()
                and w.numel() == self.m):
            raise ValueError("w must be a contiguous float32 CUDA tensor of m entries")
        B.cls_set_weights(self.handle, w)
