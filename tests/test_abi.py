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
    assert ctypes.sizeof(binding.ba_solve_stats) == 8 * 4 + 3 * 8
    assert ctypes.sizeof(binding.ba_lm_stats) == 4 * 4 + 6 * 8


def test_default_options_and_errors_without_device(libba):
    L = binding.lib()
    opt = binding.ba_options()
    L.ba_default_options(ctypes.byref(opt))
    assert opt.precision == 0 and opt.damping == 0 and opt.chunk_iters == 8 and opt.inner_tol == 1e-6
    assert opt.max_refine == 64 and opt.max_history == 0 and opt.item_blocks == 0 and opt.wait_polls == 0
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


def test_static_residual_binding_rejects_bad_arrays():
    """ba_schur_residual_static receives raw device pointers and no lengths, so the binding rejects
    host arrays, wrong dtypes and wrong sizes before the library is called (checked here on CPU
    tensors: every other property right, the device check comes last)."""
    import numpy as np
    import torch

    n = 3
    good = {"row_ptr": torch.zeros(n + 1, dtype=torch.int64), "col": torch.zeros(2, dtype=torch.int32),
            "blocks": torch.zeros(2 * 81, dtype=torch.float64), "btilde": torch.zeros(9 * n, dtype=torch.float64),
            "x": torch.zeros(9 * n, dtype=torch.float64), "out": torch.zeros(2, dtype=torch.float64)}

    def call(**over):
        a = dict(good, **over)
        binding.ba_schur_residual_static(n, a["row_ptr"], a["col"], a["blocks"], a["btilde"], a["x"], a["out"])

    with pytest.raises(TypeError, match="row_ptr"):
        call(row_ptr=np.zeros(n + 1, np.int64))
    for name, bad in [("row_ptr", torch.zeros(n + 1, dtype=torch.int32)), ("col", torch.zeros(2, dtype=torch.int64)),
                      ("blocks", torch.zeros(2 * 81, dtype=torch.float32)),
                      ("btilde", torch.zeros(9 * n, dtype=torch.float32)), ("x", torch.zeros(9 * n, dtype=torch.int64)),
                      ("out", torch.zeros(2, dtype=torch.float32))]:
        with pytest.raises(TypeError, match=name):
            call(**{name: bad})
    for name, bad in [("row_ptr", torch.zeros(n, dtype=torch.int64)), ("btilde", torch.zeros(9 * n - 1, dtype=torch.float64)),
                      ("x", torch.zeros(9 * n + 9, dtype=torch.float64)), ("out", torch.zeros(1, dtype=torch.float64)),
                      ("blocks", torch.zeros(81, dtype=torch.float64))]:
        with pytest.raises(ValueError):
            call(**{name: bad})
    with pytest.raises(ValueError, match="contiguous"):
        call(blocks=torch.zeros(2 * 81 * 2, dtype=torch.float64)[::2])
    with pytest.raises(ValueError, match="CUDA"):
        call()
