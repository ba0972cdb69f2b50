"""Batched problems (``ba_batch_create``): many independent problems in the same launches.

Every problem of a batch is solved by its own Algorithm 1 / Algorithm 2 iteration; the batch only
shares the kernel launches.  The library sums every per-problem quantity in an order fixed by the
problem alone, so a problem solved in a batch must give bit-for-bit the solution, iteration count
and residual history it gives when solved alone; the single-problem path is itself checked against
the oracle in test_gpu_solve.py, and here one batch is also checked against the oracle directly.
"""
import numpy as np
import pytest

from oracle import lm as olm
from oracle import solvers as osol
from paper_2110_04015_gb300 import binding, problem
from paper_2110_04015_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

LAM = 1e-4


def _scenes():
    # uneven sizes and shapes: a ring, two sequences and a clustered dense problem; the 13-camera
    # ring has fewer cameras than some subset counts below
    return [
        sy.make("tiny", 3, n_cams=13, n_pts=700),
        sy.make("sequential", 1, n_cams=90, n_pts=5000),
        sy.make("dense", 2, n_cams=70, n_pts=6000, n_clusters=3),
        sy.make("sequential", 4, n_cams=41, n_pts=2500, window=12),
    ]


_SCENES = None


def scenes():
    global _SCENES
    if _SCENES is None:
        _SCENES = _scenes()
    return _SCENES


def _solve(p, solver, **kw):
    p.ba_build_normal(LAM)
    if solver == "pcg":
        st = p.ba_solve_pcg(1e-6, 1000)
    else:
        st = p.ba_solve_mcg(1e-6, 1000, kw.get("n_dirs", 4), kw.get("tau", 10.0))
    return st, p.ba_get_delta()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("solver,kw", [("pcg", {}), ("mcg", {"n_dirs": 4, "tau": 10.0}),
                                       ("mcg", {"n_dirs": 16, "tau": 1e9})])
def test_batch_equals_solo_bit_for_bit(precision, solver, kw):
    scs = scenes()
    cam_off, _ = problem.concat_offsets(scs)
    pb = problem.from_scenes(scs, precision=precision)
    assert pb.ba_get_batch_size() == len(scs)
    st_b, x_b = _solve(pb, solver, **kw)
    per = pb.ba_get_batch_stats()
    hist_b = [pb.ba_get_batch_history(b) for b in range(len(scs))]
    pb.close()
    for b, sc in enumerate(scs):
        ps = problem.from_scene(sc, precision=precision)
        st_s, x_s = _solve(ps, solver, **kw)
        h_s = ps.ba_get_residual_history()
        ps.close()
        assert per[b]["status"] == st_s["status"] == 0
        assert per[b]["iters"] == st_s["iters"]
        assert per[b]["local_steps"] == st_s["local_steps"]
        assert per[b]["refinements"] == st_s["refinements"]
        assert per[b]["n_dirs_eff"] == st_s["n_dirs_eff"]
        assert np.array_equal(hist_b[b], h_s)
        assert np.array_equal(x_b[cam_off[b]:cam_off[b + 1]], x_s)
        assert per[b]["true_rel_residual"] == st_s["true_rel_residual"]
        assert per[b]["true_rel_residual"] <= 1e-6
    # the summary is the worst problem
    assert st_b["iters"] == max(s["iters"] for s in per)
    assert st_b["true_rel_residual"] == max(s["true_rel_residual"] for s in per)


def test_batch_matches_oracle_per_problem():
    scs = scenes()
    cam_off, _ = problem.concat_offsets(scs)
    pb = problem.from_scenes(scs)
    pb.ba_build_normal(LAM)
    pb.ba_solve_mcg(1e-6, 1000, 4, 10.0)
    x = pb.ba_get_delta()
    per = pb.ba_get_batch_stats()
    pb.close()
    for b, sc in enumerate(scs):
        m = olm.measurements(sc)
        lin = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, LAM)
        ref = osol.dense_solve(lin.S, lin.btilde)
        xb = x[cam_off[b]:cam_off[b + 1]].ravel()
        d = xb - ref
        # S-energy error of the Krylov solution against the exact solve (tolerance 1e-6 on the residual)
        assert np.sqrt(d @ (lin.S @ d) / (ref @ (lin.S @ ref))) < 1e-4
        assert osol.true_rel_residual(lin.S, lin.btilde, xb) <= 1.01e-6
        o = osol.mcg(lin.S, lin.btilde, osol.block_jacobi_inverse(lin.S, sc.n_cams), 4, 10.0)
        # same iteration count as the oracle's Algorithm 2, within rounding-sensitive plateaus
        assert abs(per[b]["iters"] - o.iters) <= max(1, int(0.05 * o.iters))


def test_problems_finish_independently():
    # a problem that needs many more iterations keeps iterating after the others have stopped,
    # and max_iters applies per problem
    scs = [sy.make("tiny", 0), sy.make("sequential", 0, n_cams=150, n_pts=9000)]
    pb = problem.from_scenes(scs)
    pb.ba_build_normal(LAM)
    st = pb.ba_solve_pcg(1e-6, 1000)
    per = pb.ba_get_batch_stats()
    assert st["status"] == 0 and all(s["status"] == 0 for s in per)
    assert per[0]["iters"] < per[1]["iters"]
    k = (per[0]["iters"] + per[1]["iters"]) // 2
    st = pb.ba_solve_pcg(1e-6, k)
    assert st["status"] == binding.BA_ERR_NOT_CONVERGED
    per = pb.ba_get_batch_stats()
    assert per[0]["status"] == 0 and per[1]["status"] == binding.BA_ERR_NOT_CONVERGED
    assert per[1]["iters"] == k
    pb.close()


def test_batch_rejects_shared_landmarks_and_lm():
    sc = sy.make("tiny", 0)
    xy = problem.device_measurements(sc)
    # split the 16 cameras of one connected problem into two "problems": landmarks straddle them
    with pytest.raises(binding.BAError) as e:
        binding.Problem(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, xy, cam_off=np.array([0, 8, 16], np.int32))
    assert e.value.code == binding.BA_ERR_INVALID_ARG and "landmark" in str(e.value)
    with pytest.raises(binding.BAError):
        binding.Problem(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, xy, cam_off=np.array([0, 16, 16], np.int32))
    pb = problem.from_scenes([sc, sy.make("tiny", 1)])
    with pytest.raises(binding.BAError) as e:
        pb.ba_lm_step("pcg")
    assert e.value.code == binding.BA_ERR_INVALID_ARG
    pb.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_autotune_picks_a_candidate_and_keeps_results(precision):
    scs = scenes()
    pb = problem.from_scenes(scs, precision=precision)
    pb.ba_build_normal(LAM)
    st0 = pb.ba_solve_mcg(1e-6, 1000, 4, 10.0)
    x0 = pb.ba_get_delta()
    cb, ms, cfg = pb.ba_autotune(reps=3)
    assert cb in (32, 64, 128, 256, 512, 1024) and ms > 0 and cfg in (0, 1, 2)
    st1 = pb.ba_solve_mcg(1e-6, 1000, 4, 10.0)
    x1 = pb.ba_get_delta()
    pb.close()
    # the choice is kept for handles of the same precision and size: taken again without timing
    pc = problem.from_scenes(scs, precision=precision)
    pc.ba_build_normal(LAM)
    assert pc.ba_autotune(reps=3) == (cb, ms, cfg)
    pc.close()
    assert st1["status"] == 0 and st1["true_rel_residual"] <= 1e-6
    # another work-item size changes only the summation order of the products
    assert abs(st1["iters"] - st0["iters"]) <= max(1, st0["iters"] // 10)
    assert np.abs(x1 - x0).max() <= 1e-3 * np.abs(x0).max()
