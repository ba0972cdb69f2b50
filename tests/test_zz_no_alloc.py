"""The allocation-free residual check agrees with the solver's own float64 true residual.

``ba_schur_residual_static`` is for callers that cannot allocate device memory where they
check a solution (under a fixed memory budget, or behind an allocator that owns the device).
It works in a file-scope device array instead of allocating.
This file is named to be collected last, so a run that stops at its first failure has already
run every other test; it also passes on its own in a fresh process.
"""
import numpy as np
import pytest

from paper_2110_04015_gb300 import binding, problem
from paper_2110_04015_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu


def _system(name, **kw):
    import torch

    sc = sy.make(name, 0, **kw)
    p = problem.from_scene(sc)
    p.ba_build_normal(1e-4)
    st = p.ba_solve_pcg(1e-6, 1000)
    row_ptr, col, B, bt = p.ba_get_schur()
    x = p.ba_get_delta()
    p.close()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return sc, st, dev(row_ptr), dev(col), dev(B), dev(bt), dev(x)


@pytest.mark.parametrize("name,kw", [("tiny", {}), ("sequential", {"n_cams": 120, "n_pts": 8000})])
def test_static_residual_matches_solver_twice(name, kw):
    import torch

    from oracle import lm as olm
    from tests._gpu import bsr_from_gpu

    sc, st, row_ptr, col, B, bt, x = _system(name, **kw)
    n_cams = sc.n_cams
    outs = []
    for _ in range(2):
        out = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
        binding.ba_schur_residual_static(n_cams, row_ptr, col, B, bt, x, out)
        torch.cuda.synchronize()
        outs.append(out.cpu().numpy())
    xh = x.cpu().numpy().ravel()
    bth = bt.cpu().numpy().ravel()
    # |-b~ - S x| with this S on the host (scipy, another summation order)
    S = bsr_from_gpu(row_ptr.cpu().numpy(), col.cpu().numpy(), B.cpu().numpy().reshape(-1, 9, 9), n_cams)
    res_host = np.linalg.norm(-bth - S @ xh)
    # the same residual with the float64 oracle's own S and b~ (Eqs. 13-14): by the triangle
    # inequality it differs from the library's by at most |b~ - b~_o| + |(S - S_o) x|
    m = olm.measurements(sc)
    lin = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, 1e-4)
    res_oracle = np.linalg.norm(-lin.btilde - lin.S @ xh)
    bound = np.linalg.norm(bth - lin.btilde) + np.linalg.norm((S - lin.S) @ xh) + 1e-9 * res_oracle
    assert bound <= 0.05 * res_oracle   # the two systems agree well enough for this to mean something
    for o in outs:
        rel = o[0] / o[1]
        # the same float64 quantity as the solver's true residual, summed in another order
        assert abs(rel - st["true_rel_residual"]) <= 1e-6 * st["true_rel_residual"]
        assert abs(o[1] - np.linalg.norm(bth)) <= 1e-12 * o[1]
        assert abs(o[0] - res_host) <= 1e-9 * res_host
        assert abs(o[0] - res_oracle) <= bound
        assert abs(o[1] - np.linalg.norm(lin.btilde)) <= 1e-10 * o[1]
    # the shared scratch is fully rewritten by every call: repeated calls agree exactly
    assert np.array_equal(outs[0], outs[1])


def test_static_residual_rejects_oversized_problems():
    import torch

    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    i = torch.zeros(8, dtype=torch.int64, device="cuda")
    c = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(binding.BAError) as e:
        binding.ba_schur_residual_static(binding.BA_STATIC_MAX_CAMS + 1, i, c, z, z, z, z)
    assert e.value.code == binding.BA_ERR_INVALID_ARG
    assert "n_cams" in str(e.value)
