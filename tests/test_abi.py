"""The C ABI library builds, loads without a GPU and exports every call of include/ba.h."""
import ctypes
import os

import pytest

from paper_2110_04015_gb300 import binding
from paper_2110_04015_gb300 import build as B


@pytest.fixture(scope="module")
def libba():
    if not os.path.exists(B.LIB):
        B.build()
    return ctypes.CDLL(B.LIB)


def test_header_declares_the_boundary_calls():
    names = binding.header_functions()
    for required in ["ba_problem_create", "ba_set_stream", "ba_build_normal", "ba_solve_pcg", "ba_solve_mcg",
                     "ba_get_delta", "ba_lm_step", "ba_problem_destroy", "ba_last_error"]:
        assert required in names


def test_library_exports_every_declared_call(libba):
    missing = [n for n in binding.header_functions() if not hasattr(libba, n)]
    assert not missing


def test_binding_covers_every_declared_call():
    assert sorted(binding._SIGNATURES) == binding.header_functions()


def test_struct_layouts_match_header():
    # sizes implied by include/ba.h (int32 fields, then doubles, natural alignment)
    assert ctypes.sizeof(binding.ba_options) == 4 * 4 + 8 + 4 * 8
    assert ctypes.sizeof(binding.ba_solve_stats) == 6 * 4 + 3 * 8
    assert ctypes.sizeof(binding.ba_lm_stats) == 4 * 4 + 6 * 8


def test_default_options_and_errors_without_device(libba):
    L = binding.lib()
    opt = binding.ba_options()
    L.ba_default_options(ctypes.byref(opt))
    assert opt.precision == 0 and opt.damping == 0 and opt.chunk_iters == 8 and opt.inner_tol == 1e-6
    assert opt.max_refine == 64 and opt.max_history == 0 and opt.item_blocks == 0
    # argument checks run before any device work
    out = ctypes.c_void_p()
    code = L.ba_problem_create(None, 0, 1, 1, None, None, None, None, None, ctypes.byref(out))
    assert code == binding.BA_ERR_INVALID_ARG
    assert b"n_cams" in L.ba_last_error(None)
    assert L.ba_project(0, 1, 1, None, None, None, None, None, None) == binding.BA_ERR_INVALID_ARG


def test_batch_create_argument_errors_without_device(libba):
    L = binding.lib()
    out = ctypes.c_void_p()
    # n_problems out of range and a missing offsets array are rejected before any device work
    code = L.ba_batch_create(None, 0, None, 4, 4, 4, None, None, None, None, None, ctypes.byref(out))
    assert code == binding.BA_ERR_INVALID_ARG
    code = L.ba_batch_create(None, 2, None, 4, 4, 4, None, None, None, None, None, ctypes.byref(out))
    assert code == binding.BA_ERR_INVALID_ARG
    assert b"cam_off" in L.ba_last_error(None)
    for name in ["ba_get_batch_size", "ba_get_batch_stats", "ba_get_batch_history", "ba_autotune"]:
        assert getattr(L, name)(None, *([0] * (len(binding._SIGNATURES[name][1]) - 1))) == binding.BA_ERR_INVALID_ARG


def test_grouping_network_parameter_layout(libba):
    # 3 layers of (Ws, Wn, b) with widths 8 -> 64 -> 64 -> 64, then wo (64) and bo (1)
    from paper_2110_04015_gb300 import learn

    n = ctypes.c_int64()
    assert binding.lib().ba_gnn_param_count(ctypes.byref(n)) == binding.BA_OK
    assert n.value == 2 * 8 * 64 + 64 + 2 * (2 * 64 * 64 + 64) + 64 + 1
    assert n.value == sum(int(__import__("numpy").prod(s)) for _, s in learn.layer_shapes())
    assert learn.init_params(0).size == n.value
