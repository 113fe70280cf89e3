"""The C-ABI library loads, exports every symbol include/smnn.h declares, and rejects bad
arguments before touching the GPU (runs on CPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "smnn.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(smnn_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2410_06074_b300 import binding
    names = declared_symbols()
    assert len(names) >= 9
    lib = ctypes.CDLL(binding.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n
        assert n in binding.SYMBOLS, n


def test_status_strings_and_counter():
    from paper_2410_06074_b300 import binding
    for st in range(5):
        assert binding.status_string(st).startswith("SMNN_")
    assert binding.launch_count() >= 0


@pytest.mark.parametrize("field,value", [("R", 0), ("R", 4), ("R_init", 3), ("T_init", 0),
                                         ("precision", 7), ("algo", 5), ("max_refine", -1),
                                         ("chunk", 1), ("adjoint_refine", -1), ("adjoint_refine", 17),
                                         ("precision", 4), ("num_seq", 0),
                                         ("w_gov", -1.0), ("T", 0)])
def test_plan_create_rejects_invalid_descriptors(field, value):
    from paper_2410_06074_b300 import binding as B
    d = B.Desc(2, 1, 1, B.F32_REFINED, B.ALGO_AUTO, 2, 0, 0, 1.0, 1.0, 1.0, 0.0, 2, 2, 16, None)
    setattr(d, field, value)
    h = ctypes.c_void_p()
    assert B.lib.smnn_plan_create(ctypes.byref(d), ctypes.byref(h)) == B.SMNN_ERR_INVALID_ARG
    assert not h.value


def test_null_arguments_are_rejected():
    from paper_2410_06074_b300 import binding as B
    assert B.lib.smnn_plan_create(None, None) == B.SMNN_ERR_INVALID_ARG
    assert B.lib.smnn_plan_destroy(None) == B.SMNN_OK
    assert B.lib.smnn_workspace_size(None, None, None) == B.SMNN_ERR_INVALID_ARG
    assert B.lib.smnn_factor_solve(*([None] * 10)) == B.SMNN_ERR_INVALID_ARG
    assert B.lib.smnn_backward(*([None] * 16)) == B.SMNN_ERR_INVALID_ARG


def test_ragged_seq_T_validation():
    from paper_2410_06074_b300 import binding as B
    seq = (ctypes.c_int64 * 3)(5, 0, 7)   # a zero-length sequence is invalid
    d = B.Desc(2, 1, 1, 0, 0, 2, 0, 0, 1.0, 1.0, 1.0, 0.0, 3, 1, 0,
               ctypes.cast(seq, ctypes.POINTER(ctypes.c_int64)))
    h = ctypes.c_void_p()
    assert B.lib.smnn_plan_create(ctypes.byref(d), ctypes.byref(h)) == B.SMNN_ERR_INVALID_ARG


def test_fused_pass_needs_every_system_within_one_cta():
    """SMNN_ALGO_CR_FUSED runs all levels of a system in one CTA (128 level-0 chunks at
    most); a longer system is refused at plan creation, before any device call."""
    from paper_2410_06074_b300 import binding as B
    d = B.Desc(2, 1, 1, B.F32_REFINED, B.ALGO_CR_FUSED, 2, 8, 0, 1.0, 1.0, 1.0, 0.0, 2, 2, 8 * 129, None)
    h = ctypes.c_void_p()
    assert B.lib.smnn_plan_create(ctypes.byref(d), ctypes.byref(h)) == B.SMNN_ERR_UNSUPPORTED
    assert not h.value


@pytest.mark.parametrize("V,Q,R,ok", [(2, 1, 1, True), (2, 2, 1, True), (3, 3, 1, True), (2, 2, 2, True),
                                      (1, 2, 2, False), (2, 1, 2, False), (3, 1, 1, False),
                                      (4, 1, 1, False), (2, 3, 1, False), (2, 4, 2, False),
                                      (3, 3, 2, True), (3, 2, 2, False), (4, 2, 2, False),
                                      (2, 3, 3, False), (0, 0, 2, True)])
def test_coupled_descriptor_validation(V, Q, R, ok):
    """V variables x (R+1) orders must fit a block of SMNN_MAX_NB = 9 and Q <= 3; shapes
    outside the instantiated ones (V = Q = 1; V = 2, R = 1, Q <= 2; V = 3, R = 1, Q = 3;
    V = 2, R = 2, Q = 2; V = 3, R = 2, Q = 3) are refused or reported unsupported at plan
    creation, before any device call; 0 means 1 for both fields."""
    from paper_2410_06074_b300 import binding as B
    d = B.Desc(R, 0, 1, B.F32_REFINED, B.ALGO_CR, 2, 0, 0, 1.0, 1.0, 1.0, 0.0, 2, 2, 16, None, V, Q)
    h = ctypes.c_void_p()
    rc = B.lib.smnn_plan_create(ctypes.byref(d), ctypes.byref(h))
    if ok:
        assert rc in (B.SMNN_OK, B.SMNN_ERR_CUDA)   # CUDA: no device in this container
        if h.value:
            B.lib.smnn_plan_destroy(h)
    else:
        assert rc in (B.SMNN_ERR_INVALID_ARG, B.SMNN_ERR_UNSUPPORTED) and not h.value


def test_graph_calls_reject_null_arguments():
    """smnn_graph_create checks its arguments before any device call (no GPU here) and
    leaves *graph NULL; launching a NULL graph is refused; destroying NULL is a no-op."""
    from paper_2410_06074_b300 import binding as B
    h = ctypes.c_void_p(1234)
    rc = B.lib.smnn_graph_create(None, *([None] * 15), ctypes.byref(h))
    assert rc == B.SMNN_ERR_INVALID_ARG and not h.value
    assert B.lib.smnn_graph_create(None, *([None] * 15), None) == B.SMNN_ERR_INVALID_ARG
    assert B.lib.smnn_graph_launch(None, None) == B.SMNN_ERR_INVALID_ARG
    assert B.lib.smnn_graph_destroy(None) == B.SMNN_OK
