"""Failure detection on the GPU without a GPU fault (the bounded waits and the error statuses).

* Every tile-streaming product waits on an mbarrier for its bulk copies with a bounded number of
  polls (ba_options.wait_polls).  wait_polls = -1 makes every such wait give up at once, as a copy
  that never lands would: the kernel must record BA_ERR_TIMEOUT, wait for its own copies still in
  flight (with the default bound: they do land), and return, so the solve ends with TIMEOUT and
  the context stays usable.
* A NaN put into the parameters on the host must end in a documented error, not a silent result.
"""
import numpy as np
import pytest

from paper_2110_04015_gb300 import binding, problem
from tests._gpu import scene

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_expired_tile_waits_end_the_solve_with_timeout(precision):
    sc = scene("seq-small")
    xy = problem.device_measurements(sc)
    with problem.from_scene(sc, precision=precision, xy=xy, wait_polls=-1) as p:
        p.ba_build_normal(1e-4)
        for solve in (lambda: p.ba_solve_pcg(1e-6, 1000), lambda: p.ba_solve_mcg(1e-6, 1000, 16, 10.0),
                      lambda: p.ba_solve_mcg(1e-6, 1000, 4, 1e9)):
            with pytest.raises(binding.BAError) as e:
                solve()
            assert e.value.code == binding.BA_ERR_TIMEOUT, e.value
            assert "wait" in str(e.value)
    # the context and a fresh handle work normally afterwards
    with problem.from_scene(sc, precision=precision, xy=xy) as q:
        q.ba_build_normal(1e-4)
        st = q.ba_solve_mcg(1e-6, 1000, 16, 10.0)
        assert st["status"] == 0 and st["true_rel_residual"] <= 1.5e-6


def test_wait_polls_option_range():
    sc = scene("tiny")
    xy = problem.device_measurements(sc)
    for bad in (-2, (1 << 30) + 1):
        with pytest.raises(binding.BAError) as e:
            problem.from_scene(sc, xy=xy, wait_polls=bad)
        assert e.value.code == binding.BA_ERR_INVALID_ARG
    with problem.from_scene(sc, xy=xy, wait_polls=1 << 30) as p:
        p.ba_build_normal(1e-4)
        assert p.ba_solve_pcg(1e-6, 1000)["status"] == 0


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("where", ["camera", "landmark"])
def test_nan_parameter_is_reported_not_solved(precision, where):
    sc = scene("tiny")
    xy = problem.device_measurements(sc)
    with problem.from_scene(sc, precision=precision, xy=xy) as p:
        cams, pts = sc.cams0.copy(), sc.pts0.copy()
        if where == "camera":
            cams[2, 6] = np.nan          # a focal length
        else:
            pts[int(sc.obs_pt[0]), 1] = np.nan
        p.ba_set_params(cams, pts)
        with pytest.raises(binding.BAError) as e:
            p.ba_build_normal(1e-4)
            p.ba_solve_mcg(1e-6, 1000, 8, 3.0)
        assert e.value.code in (binding.BA_ERR_SINGULAR, binding.BA_ERR_BREAKDOWN), e.value
        # the failed build leaves no system to solve
        with pytest.raises(binding.BAError) as e:
            p.ba_solve_pcg(1e-6, 1000)
        assert e.value.code == binding.BA_ERR_STATE
        # valid parameters again: the handle recovers
        p.ba_set_params(sc.cams0, sc.pts0)
        p.ba_build_normal(1e-4)
        st = p.ba_solve_pcg(1e-6, 1000)
        assert st["status"] == 0 and st["true_rel_residual"] <= 1.5e-6
