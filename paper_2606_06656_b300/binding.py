"""Thin Python binding over the C ABI (include/cls.h): argument marshalling
only.  Every computation runs in the CUDA library; PyTorch provides device
memory and the current stream.

Function names follow the C ABI.  Assignments are torch float32 CUDA tensors
of shape (n, R) (variable-major, restart-minor), i.e. x[v, r].
"""
import ctypes as C

import numpy as np
import torch

from . import _lib

i64 = C.c_int64


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, torch.Tensor):
        return C.c_void_p(a.data_ptr()) if a.numel() else None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p) if a.size else None
    raise TypeError(type(a))


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _arrays(inst):
    """Contiguous host arrays of a constraint set (workloads.Instance-like)."""
    a = dict(
        offsets=np.ascontiguousarray(inst.offsets, dtype=np.int32),
        lit_var=np.ascontiguousarray(inst.lit_var, dtype=np.int32),
        lit_sign=np.ascontiguousarray(inst.lit_sign, dtype=np.int8),
        ctype=np.ascontiguousarray(inst.ctype, dtype=np.int32),
        k=np.ascontiguousarray(inst.k, dtype=np.int32),
        weight=np.ascontiguousarray(inst.weight, dtype=np.float32),
        spectra=None if getattr(inst, "spectra", None) is None
        else np.ascontiguousarray(inst.spectra, dtype=np.int8),
        fixed=None if getattr(inst, "fixed", None) is None
        else np.ascontiguousarray(inst.fixed, dtype=np.uint8),
        fixed_val=None if getattr(inst, "fixed_val", None) is None
        else np.ascontiguousarray(inst.fixed_val, dtype=np.float32),
    )
    return a


def cls_problem_check(inst):
    lib = _lib.load()
    a = _arrays(inst)
    rc = lib.cls_problem_check(int(inst.n), len(a["offsets"]) - 1, _ptr(a["offsets"]),
                               _ptr(a["lit_var"]), _ptr(a["lit_sign"]), _ptr(a["ctype"]),
                               _ptr(a["k"]), _ptr(a["weight"]), _ptr(a["spectra"]),
                               _ptr(a["fixed"]), _ptr(a["fixed_val"]))
    return rc, (lib.cls_last_error() or b"").decode()


CLS_SIMPLIFY_FIXED = 1


def cls_problem_create(inst, flags=0):
    lib = _lib.load()
    a = _arrays(inst)
    h = C.c_void_p()
    rc = lib.cls_problem_create_ex(int(inst.n), len(a["offsets"]) - 1, _ptr(a["offsets"]),
                                   _ptr(a["lit_var"]), _ptr(a["lit_sign"]), _ptr(a["ctype"]),
                                   _ptr(a["k"]), _ptr(a["weight"]), _ptr(a["spectra"]),
                                   _ptr(a["fixed"]), _ptr(a["fixed_val"]), int(flags),
                                   C.byref(h))
    _lib.check(rc, "cls_problem_create_ex")
    return h


def cls_problem_destroy(h):
    if h:
        _lib.check(_lib.load().cls_problem_destroy(h), "cls_problem_destroy")


def cls_problem_info(h):
    info = (i64 * 10)()
    _lib.check(_lib.load().cls_problem_info(h, info), "cls_problem_info")
    keys = ["n", "m", "nnz", "n_thread", "n_group_real", "n_group_dft", "dft_roots",
            "dft_lroots", "nnz_fe", "n_const"]
    return dict(zip(keys, [int(v) for v in info]))


def cls_workspace_size(h, R):
    b = C.c_size_t()
    _lib.check(_lib.load().cls_workspace_size(h, int(R), C.byref(b)), "cls_workspace_size")
    return int(b.value)


def cls_solve_host_workspace_size(h, R):
    b = C.c_size_t()
    _lib.check(_lib.load().cls_solve_host_workspace_size(h, int(R), C.byref(b)),
               "cls_solve_host_workspace_size")
    return int(b.value)


def cls_init_uniform(h, R, seed, r_offset, x, stream=None):
    _lib.check(_lib.load().cls_init_uniform(h, int(R), int(seed), int(r_offset), _ptr(x),
                                            _stream(stream)), "cls_init_uniform")


def cls_track_reset(h, R, trk, stream=None):
    """Per-restart tracking state (int32[4, R] device tensor) to its start."""
    _lib.check(_lib.load().cls_track_reset(h, int(R), _ptr(trk), _stream(stream)),
               "cls_track_reset")


def cls_track_step(h, R, nsat, step, trk, stream=None):
    """Fold one step's satisfied counts into the tracking state."""
    _lib.check(_lib.load().cls_track_step(h, int(R), _ptr(nsat), int(step), _ptr(trk),
                                          _stream(stream)), "cls_track_step")


def cls_refill(h, R, x, trk, patience, seed, r_offset, generation, count, stream=None):
    """Fresh points for the unsolved restarts without improvement for
    `patience` steps; count (device int32[1]) is increased by their number."""
    _lib.check(_lib.load().cls_refill(h, int(R), _ptr(x), _ptr(trk), int(patience), int(seed),
                                      int(r_offset), int(generation), _ptr(count),
                                      _stream(stream)), "cls_refill")


def cls_unsat_histogram(h, R, nsat, hist, stream=None):
    """hist[k] = restarts with k unsatisfied constraints (device int32[m + 1])."""
    _lib.check(_lib.load().cls_unsat_histogram(h, int(R), _ptr(nsat), _ptr(hist),
                                               _stream(stream)), "cls_unsat_histogram")


def cls_constraint_stats(h, R, bits, ws, gnorm, unsat, stream=None):
    """Per constraint over the restarts: gnorm (device float64[m]) = sum of
    the restarts' gradient norms from the workspace's partials of the last
    evaluation; unsat (device int32[m]) = restarts violating it at bits."""
    _lib.check(_lib.load().cls_constraint_stats(h, int(R), _ptr(bits), _ptr(ws),
                                                ws.numel() if ws is not None else 0,
                                                _ptr(gnorm), _ptr(unsat), _stream(stream)),
               "cls_constraint_stats")


def cls_reweight(h, R, gnorm, unsat, eta, kappa, w_max, w_out, stream=None):
    """Weight update from cls_constraint_stats' output; new weights in w_out
    (device float32[m]) and in the problem."""
    _lib.check(_lib.load().cls_reweight(h, int(R), _ptr(gnorm), _ptr(unsat), float(eta),
                                        float(kappa), float(w_max), _ptr(w_out),
                                        _stream(stream)), "cls_reweight")


def cls_set_weights(h, w, stream=None):
    """w (device float32[m]) become the constraint weights."""
    _lib.check(_lib.load().cls_set_weights(h, _ptr(w), _stream(stream)), "cls_set_weights")


def cls_movement(h, R, x_prev, x, maxdelta, stream=None):
    """maxdelta (device float32[R]) = per restart max_v |x - x_prev|."""
    _lib.check(_lib.load().cls_movement(h, int(R), _ptr(x_prev), _ptr(x), _ptr(maxdelta),
                                        _stream(stream)), "cls_movement")


def cls_track_converged(h, R, maxdelta, tol, step, conv, stream=None):
    """conv (device int32[R], -1 = not yet) takes `step` the first time the
    restart's movement is at most tol."""
    _lib.check(_lib.load().cls_track_converged(h, int(R), _ptr(maxdelta), float(tol), int(step),
                                               _ptr(conv), _stream(stream)),
               "cls_track_converged")


def cls_eval(h, R, x, obj, grad, fe_con, ws, stream=None):
    _lib.check(_lib.load().cls_eval(h, int(R), _ptr(x), _ptr(obj), _ptr(grad), _ptr(fe_con),
                                    _ptr(ws), ws.numel() if ws is not None else 0,
                                    _stream(stream)), "cls_eval")


def cls_restart_scale(h, R, g, scale, out, stream=None):
    _lib.check(_lib.load().cls_restart_scale(h, int(R), _ptr(g), _ptr(scale), _ptr(out),
                                             _stream(stream)), "cls_restart_scale")


def cls_pgd_update(h, R, x, grad, lr, bits, stream=None):
    _lib.check(_lib.load().cls_pgd_update(h, int(R), _ptr(x), _ptr(grad), float(lr), _ptr(bits),
                                          _stream(stream)), "cls_pgd_update")


def cls_round_score(h, R, x, bits, nsat, wsat, ws, stream=None):
    _lib.check(_lib.load().cls_round_score(h, int(R), _ptr(x), _ptr(bits), _ptr(nsat),
                                           _ptr(wsat), _ptr(ws),
                                           ws.numel() if ws is not None else 0, _stream(stream)),
               "cls_round_score")


def cls_step(h, R, x, lr, n_steps, bits, nsat, wsat, ws, stream=None):
    _lib.check(_lib.load().cls_step(h, int(R), _ptr(x), float(lr), int(n_steps), _ptr(bits),
                                    _ptr(nsat), _ptr(wsat), _ptr(ws),
                                    ws.numel() if ws is not None else 0, _stream(stream)),
               "cls_step")


def cls_solve_host(h, R, x0_host, lr, n_steps, nsat_host, x_host, ws, stream=None):
    _lib.check(_lib.load().cls_solve_host(h, int(R), _ptr(x0_host), float(lr), int(n_steps),
                                          _ptr(nsat_host), _ptr(x_host), _ptr(ws),
                                          ws.numel() if ws is not None else 0, _stream(stream)),
               "cls_solve_host")


def cls_profile_enable(h, on):
    _lib.check(_lib.load().cls_profile_enable(h, 1 if on else 0), "cls_profile_enable")


def cls_profile_reset(h):
    _lib.check(_lib.load().cls_profile_reset(h), "cls_profile_reset")


def cls_profile_read(h, kc):
    n, ms = C.c_int64(), C.c_double()
    _lib.check(_lib.load().cls_profile_read(h, int(kc), C.byref(n), C.byref(ms)),
               "cls_profile_read")
    return int(n.value), float(ms.value)


N_BUCKETS = 25


def cls_autotune(h, R, x, reps, ws, stream=None):
    _lib.check(_lib.load().cls_autotune(h, int(R), _ptr(x), int(reps), _ptr(ws),
                                        ws.numel() if ws is not None else 0, _stream(stream)),
               "cls_autotune")


def cls_tuning_get(h):
    buf = (C.c_int32 * N_BUCKETS)()
    _lib.check(_lib.load().cls_tuning_get(h, buf, N_BUCKETS), "cls_tuning_get")
    return [int(v) for v in buf]


def cls_tuning_set(h, cfg):
    buf = (C.c_int32 * N_BUCKETS)(*[int(v) for v in cfg])
    _lib.check(_lib.load().cls_tuning_set(h, buf, len(cfg)), "cls_tuning_set")


def cls_config_info(cid):
    buf = (C.c_int32 * 4)()
    _lib.check(_lib.load().cls_config_info(int(cid), buf), "cls_config_info")
    return [int(v) for v in buf]


def cls_graph_create(h, R, x, lr, n_steps, bits, nsat, wsat, ws):
    g = C.c_void_p()
    _lib.check(_lib.load().cls_graph_create(h, int(R), _ptr(x), float(lr), int(n_steps),
                                            _ptr(bits), _ptr(nsat), _ptr(wsat), _ptr(ws),
                                            ws.numel() if ws is not None else 0, C.byref(g)),
               "cls_graph_create")
    return g


def cls_graph_launch(g, stream=None):
    _lib.check(_lib.load().cls_graph_launch(g, _stream(stream)), "cls_graph_launch")


def cls_graph_kernel_count(g):
    n = C.c_int64()
    _lib.check(_lib.load().cls_graph_kernel_count(g, C.byref(n)), "cls_graph_kernel_count")
    return int(n.value)


def cls_graph_destroy(g):
    if g:
        _lib.check(_lib.load().cls_graph_destroy(g), "cls_graph_destroy")


def cls_mpnn_create(h):
    g = C.c_void_p()
    _lib.check(_lib.load().cls_mpnn_create(h, C.byref(g)), "cls_mpnn_create")
    return g


def cls_mpnn_destroy(g):
    if g:
        _lib.check(_lib.load().cls_mpnn_destroy(g), "cls_mpnn_destroy")


def cls_mpnn_sizes(g):
    n, b = C.c_int64(), C.c_size_t()
    _lib.check(_lib.load().cls_mpnn_sizes(g, C.byref(n), C.byref(b)), "cls_mpnn_sizes")
    return int(n.value), int(b.value)


def cls_mpnn_param_init(g, seed, params, stream=None):
    _lib.check(_lib.load().cls_mpnn_param_init(g, int(seed), _ptr(params), _stream(stream)),
               "cls_mpnn_param_init")


def cls_mpnn_forward(g, params, z, act, stream=None):
    _lib.check(_lib.load().cls_mpnn_forward(g, _ptr(params), _ptr(z), _ptr(act), act.numel(),
                                            _stream(stream)), "cls_mpnn_forward")


def cls_mpnn_points(g, z, R, seed, r_offset, tau, x0, stream=None):
    _lib.check(_lib.load().cls_mpnn_points(g, _ptr(z), int(R), int(seed), int(r_offset),
                                           float(tau), _ptr(x0), _stream(stream)),
               "cls_mpnn_points")


def cls_mpnn_head_grad(g, z, x0, gx0, R, target, lam, dz, stream=None):
    _lib.check(_lib.load().cls_mpnn_head_grad(g, _ptr(z), _ptr(x0), _ptr(gx0), int(R),
                                              _ptr(target), float(lam), _ptr(dz),
                                              _stream(stream)), "cls_mpnn_head_grad")


def cls_mpnn_backward(g, params, dz, dparams, act, stream=None):
    _lib.check(_lib.load().cls_mpnn_backward(g, _ptr(params), _ptr(dz), _ptr(dparams), _ptr(act),
                                             act.numel(), _stream(stream)), "cls_mpnn_backward")


def cls_adam_step(params, grads, m, v, lr, b1, b2, eps, t, stream=None):
    _lib.check(_lib.load().cls_adam_step(params.numel(), _ptr(params), _ptr(grads), _ptr(m),
                                         _ptr(v), float(lr), float(b1), float(b2), float(eps),
                                         int(t), _stream(stream)), "cls_adam_step")


def cls_batch_graph_create(handles, Rs, xs, lr, n_steps, nsats, wss):
    """One graph over several problems (each with its own restarts)."""
    n = len(handles)
    VP = C.c_void_p * n
    hs = VP(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    rs = (C.c_int32 * n)(*[int(r) for r in Rs])
    xp = VP(*[t.data_ptr() for t in xs])
    npp = VP(*[t.data_ptr() if t is not None else None for t in nsats])
    wp = VP(*[t.data_ptr() for t in wss])
    wb = (C.c_size_t * n)(*[t.numel() for t in wss])
    g = C.c_void_p()
    _lib.check(_lib.load().cls_batch_graph_create(n, hs, rs, xp, float(lr), int(n_steps), None,
                                                  npp, None, wp, wb, C.byref(g)),
               "cls_batch_graph_create")
    return g


def cls_step_persistent(h, R, x, lr, n_steps, bits, nsat, wsat, ws, stream=None):
    _lib.check(_lib.load().cls_step_persistent(h, int(R), _ptr(x), float(lr), int(n_steps),
                                               _ptr(bits), _ptr(nsat), _ptr(wsat), _ptr(ws),
                                               ws.numel() if ws is not None else 0,
                                               _stream(stream)), "cls_step_persistent")


def cls_persistent_status(h, R, ws):
    st = C.c_int32()
    _lib.check(_lib.load().cls_persistent_status(h, int(R), _ptr(ws), ws.numel(), C.byref(st)),
               "cls_persistent_status")
    return int(st.value)


def cls_grid_barrier_check(rounds, extra, spin_limit, scratch):
    st, passed = C.c_int32(), C.c_int32()
    _lib.check(_lib.load().cls_grid_barrier_check(int(rounds), int(extra), int(spin_limit),
                                                  _ptr(scratch), scratch.numel(), C.byref(st),
                                                  C.byref(passed)), "cls_grid_barrier_check")
    return int(st.value), int(passed.value)


def cls_dft_work(h):
    """(flops per restart, (literal, root) pairs per restart) of the DFT
    buckets under the current tuning."""
    out = (C.c_int64 * 2)()
    _lib.check(_lib.load().cls_dft_work(h, out), "cls_dft_work")
    return int(out[0]), int(out[1])


def cls_series_range(L, K):
    """Low roots j = 1..js of a length-L constraint in range of the power-sum
    pass with K terms (host-only)."""
    js = _lib.load().cls_series_range(int(L), int(K))
    if js < 0:
        _lib.check(js, "cls_series_range")
    return int(js)


def cls_dft_flops_counter(h, reset=False):
    """Flops of the DFT roots evaluated by the dense factored kernel since the
    last reset (synchronises the device)."""
    v = C.c_int64()
    _lib.check(_lib.load().cls_dft_flops_counter(h, C.byref(v), 1 if reset else 0),
               "cls_dft_flops_counter")
    return int(v.value)
