"""C ABI checks that need no GPU: the library loads, exports every symbol the
header declares, validates constraint sets and reports errors by code."""
import ctypes as C

import numpy as np
import pytest

import workloads as W
from paper_2606_06656_b300 import _lib
from paper_2606_06656_b300 import binding as B


def test_library_exports_every_header_symbol():
    lib = _lib.load()
    syms = _lib.header_symbols()
    assert len(syms) >= 15
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) <= set(_lib.SIGNATURES)


def test_strerror_codes():
    lib = _lib.load()
    assert lib.cls_strerror(0) == b"ok"
    for code in (-1, -2, -3, -4, -5):
        assert lib.cls_strerror(code) not in (b"", b"unknown error")


def _clone(inst):
    return W.Instance(**{k: (v.copy() if isinstance(v, np.ndarray) else v)
                         for k, v in inst.__dict__.items()})


def test_problem_check_accepts_workloads():
    for inst in [W.random_ksat(), W.mixed_pb(n=600, n_or=500, n_xor=50, n_card=20,
                                              card_len=(10, 300)),
                 W.redundant_5sat(n=300, m=900, redundancy=0.5, red_len=(50, 200))]:
        rc, msg = B.cls_problem_check(inst)
        assert rc == 0, msg


@pytest.mark.parametrize("mutate,needle", [
    (lambda i: i.lit_var.__setitem__(4, i.lit_var[3]), "appears twice"),
    (lambda i: i.lit_var.__setitem__(0, i.n), "out of range"),
    (lambda i: i.lit_var.__setitem__(0, -1), "out of range"),
    (lambda i: i.lit_sign.__setitem__(2, 0), "sign"),
    (lambda i: i.ctype.__setitem__(1, 9), "unknown type"),
    (lambda i: i.weight.__setitem__(1, np.inf), "weight"),
    (lambda i: i.offsets.__setitem__(2, i.offsets[1]), "length"),
])
def test_problem_check_rejects(mutate, needle):
    inst = _clone(W.random_ksat())
    mutate(inst)
    rc, msg = B.cls_problem_check(inst)
    assert rc == -1 and needle in msg, msg


def test_problem_check_thresholds_and_spectra():
    rng = np.random.default_rng(0)
    inst = W.random_constraint_set(rng, 20, 10, [W.TYPE_CARD_GE], (3, 6))
    inst.k[0] = inst.offsets[1] - inst.offsets[0] + 1          # k > L
    rc, msg = B.cls_problem_check(inst)
    assert rc == -1 and "k=" in msg
    inst = W.random_constraint_set(rng, 20, 5, [W.TYPE_SPECTRUM], (3, 6))
    inst.spectra[0] = 0
    rc, msg = B.cls_problem_check(inst)
    assert rc == -1 and "spectra" in msg
    inst.spectra = None
    rc, msg = B.cls_problem_check(inst)
    assert rc == -1
    # too long
    inst = W.build(2000, [(W.TYPE_OR, 0, np.arange(1025, dtype=np.int32),
                           np.ones(1025, np.int8))])
    rc, msg = B.cls_problem_check(inst)
    assert rc == -1 and "1024" in msg


def test_problem_check_fixed_values():
    inst = _clone(W.random_ksat())
    inst.fixed = np.zeros(inst.n, np.uint8)
    inst.fixed[3] = 1
    inst.fixed_val = np.zeros(inst.n, np.float32)
    rc, msg = B.cls_problem_check(inst)
    assert rc == -1 and "fixed value" in msg
    inst.fixed_val[3] = -1.0
    assert B.cls_problem_check(inst)[0] == 0


def test_empty_constraint_set_is_valid():
    inst = W.build(5, [])
    assert B.cls_problem_check(inst)[0] == 0


def test_null_arguments_do_not_crash():
    lib = _lib.load()
    assert lib.cls_problem_destroy(None) == 0
    assert lib.cls_workspace_size(None, 4, C.byref(C.c_size_t())) == -1
    assert lib.cls_step(None, 4, None, 0.1, 1, None, None, None, None, 0, None) == -1
    assert lib.cls_problem_create(0, 0, None, None, None, None, None, None, None, None,
                                  None, None) == -1


def test_config_table_describes_buckets_and_configs():
    from paper_2606_06656_b300 import binding as B
    seen_dft = seen_real = 0
    for cid in range(99):
        G, Q, cplx, ys = B.cls_config_info(cid)
        assert G in (8, 16, 32) and Q >= 1 and cplx in (0, 1, 2, 3) and ys in (0, 1)
        seen_dft += cplx > 0
        seen_real += cplx == 0
    assert seen_dft > 0 and seen_real > 0
    maxes = [B.cls_config_info(1000 + b)[1] for b in range(B.N_BUCKETS)]
    assert maxes[-1] == 1024
    with pytest.raises(Exception):
        B.cls_config_info(99)
