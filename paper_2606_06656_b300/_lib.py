"""ctypes loader for libcls_b300.so (the C ABI of include/cls.h).

The library is built in-tree (paper_2606_06656_b300/csrc/build.py).  There is
no fallback: if the shared library is missing or fails to load, every call
raises.
"""
import ctypes as C
import os
import re

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcls_b300.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "cls.h")

_lib = None

i32, i64, u64, f32, vp, sz = C.c_int32, C.c_int64, C.c_uint64, C.c_float, C.c_void_p, C.c_size_t
u32 = C.c_uint32
P = C.POINTER

SIGNATURES = {
    "cls_problem_check": (i32, [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
    "cls_problem_create": (i32, [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, P(vp)]),
    "cls_problem_create_ex": (i32, [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, C.c_uint32,
                                    P(vp)]),
    "cls_problem_destroy": (i32, [vp]),
    "cls_problem_info": (i32, [vp, P(i64)]),
    "cls_workspace_size": (i32, [vp, i32, P(sz)]),
    "cls_init_uniform": (i32, [vp, i32, u64, i64, vp, vp]),
    "cls_eval": (i32, [vp, i32, vp, vp, vp, vp, vp, sz, vp]),
    "cls_pgd_update": (i32, [vp, i32, vp, vp, f32, vp, vp]),
    "cls_restart_scale": (i32, [vp, i32, vp, vp, vp, vp]),
    "cls_round_score": (i32, [vp, i32, vp, vp, vp, vp, vp, sz, vp]),
    "cls_step": (i32, [vp, i32, vp, f32, i32, vp, vp, vp, vp, sz, vp]),
    "cls_step_persistent": (i32, [vp, i32, vp, f32, i32, vp, vp, vp, vp, sz, vp]),
    "cls_persistent_status": (i32, [vp, i32, vp, sz, P(i32)]),
    "cls_grid_barrier_check": (i32, [i32, i32, u32, vp, sz, P(i32), P(i32)]),
    "cls_dft_work": (i32, [vp, P(i64)]),
    "cls_dft_flops_counter": (i32, [vp, P(i64), i32]),
    "cls_series_range": (i32, [i32, i32]),
    "cls_track_reset": (i32, [vp, i32, vp, vp]),
    "cls_track_step": (i32, [vp, i32, vp, i32, vp, vp]),
    "cls_refill": (i32, [vp, i32, vp, vp, i32, u64, i64, i32, vp, vp]),
    "cls_unsat_histogram": (i32, [vp, i32, vp, vp, vp]),
    "cls_constraint_stats": (i32, [vp, i32, vp, vp, sz, vp, vp, vp]),
    "cls_reweight": (i32, [vp, i32, vp, vp, C.c_double, C.c_double, C.c_double, vp, vp]),
    "cls_set_weights": (i32, [vp, vp, vp]),
    "cls_movement": (i32, [vp, i32, vp, vp, vp, vp]),
    "cls_track_converged": (i32, [vp, i32, vp, f32, i32, vp, vp]),
    "cls_solve_host_workspace_size": (i32, [vp, i32, P(sz)]),
    "cls_solve_host": (i32, [vp, i32, vp, f32, i32, vp, vp, vp, sz, vp]),
    "cls_autotune": (i32, [vp, i32, vp, i32, vp, sz, vp]),
    "cls_tuning_get": (i32, [vp, P(i32), i32]),
    "cls_tuning_set": (i32, [vp, P(i32), i32]),
    "cls_config_info": (i32, [i32, P(i32)]),
    "cls_graph_create": (i32, [vp, i32, vp, f32, i32, vp, vp, vp, vp, sz, P(vp)]),
    "cls_batch_graph_create": (i32, [i32, vp, vp, vp, f32, i32, vp, vp, vp, vp, vp, P(vp)]),
    "cls_graph_launch": (i32, [vp, vp]),
    "cls_graph_kernel_count": (i32, [vp, P(i64)]),
    "cls_graph_destroy": (i32, [vp]),
    "cls_step_noalloc": (i32, [vp, i32, vp, f32, i32, vp, vp, vp, vp]),
    "cls_mpnn_create": (i32, [vp, P(vp)]),
    "cls_mpnn_destroy": (i32, [vp]),
    "cls_mpnn_sizes": (i32, [vp, P(i64), P(sz)]),
    "cls_mpnn_param_init": (i32, [vp, u64, vp, vp]),
    "cls_mpnn_forward": (i32, [vp, vp, vp, vp, sz, vp]),
    "cls_mpnn_points": (i32, [vp, vp, i32, u64, i64, f32, vp, vp]),
    "cls_mpnn_head_grad": (i32, [vp, vp, vp, vp, i32, vp, f32, vp, vp]),
    "cls_mpnn_backward": (i32, [vp, vp, vp, vp, vp, sz, vp]),
    "cls_adam_step": (i32, [i64, vp, vp, vp, vp, f32, f32, f32, f32, i32, vp]),
    "cls_profile_enable": (i32, [vp, i32]),
    "cls_profile_read": (i32, [vp, i32, P(i64), P(C.c_double)]),
    "cls_profile_reset": (i32, [vp]),
    "cls_strerror": (C.c_char_p, [i32]),
    "cls_last_error": (C.c_char_p, []),
}


class ClsError(RuntimeError):
    def __init__(self, code, fn, msg):
        super().__init__(f"{fn} failed with {code}: {msg}")
        self.code = code


def header_symbols():
    """Names of the functions declared in include/cls.h."""
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char\*)\s+(cls_\w+)\s*\(", txt, re.M)))


def load():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          "`python -m paper_2606_06656_b300.csrc.build` (no CPU fallback)")
    lib = C.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def check(rc, fn):
    if rc != 0:
        lib = load()
        raise ClsError(rc, fn, (lib.cls_last_error() or b"").decode())
    return rc
