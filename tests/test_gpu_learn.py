"""The pose-grouping network (ba_gnn_*): graph, forward, gradient and Adam against the float64
oracle (oracle/gnn.py), and what the trained network gains for MCG on held-out problems whose
camera numbering carries no geometry."""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gnn as ognn
from oracle import lm as olm
from oracle import solvers as osol
from paper_2110_04015_gb300 import binding, learn, problem
from paper_2110_04015_gb300 import synthetic as sy

pytestmark = pytest.mark.gpu

LAM = 1e-4


def _oracle_graph(sc):
    m = olm.measurements(sc)
    lin = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, LAM)
    C = ognn.coupling(lin.S, sc.n_cams)
    return C, ognn.features(sc.cams0, C)


def _coupling_from_gpu(p, c):
    row_ptr, col, _, _ = p.ba_get_schur(blocks=False)
    return sp.csr_matrix((c.astype(np.float64), col, row_ptr), shape=(p.n_cams, p.n_cams))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [("tiny", {}), ("sequential", {"n_cams": 120, "n_pts": 8000})])
def test_graph_and_features_match_oracle(precision, case):
    sc = sy.shuffled(sy.make(case[0], 0, **case[1]), 5)
    C, X = _oracle_graph(sc)
    p = problem.from_scene(sc, precision=precision)
    p.ba_build_normal(LAM)
    g = binding.GNN(learn.init_params(0))
    Xg, c = g.ba_gnn_graph(p)
    Cg = _coupling_from_gpu(p, c)
    assert abs(Cg - C).max() <= 1e-5 * abs(C).max()
    assert np.abs(Xg - X).max() <= 1e-4
    g.close()
    p.close()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_loss_scores_and_gradient_match_oracle(precision):
    sc = sy.shuffled(sy.make("sequential", 3, n_cams=150, n_pts=9000), 3)
    C, X = _oracle_graph(sc)
    theta = learn.init_params(7)
    L_o, g_o, s_o = ognn.loss_and_grad(theta.astype(np.float64), X, C)
    p = problem.from_scene(sc, precision=precision)
    p.ba_build_normal(LAM)
    g = binding.GNN(theta)
    L, s, grad = g.ba_gnn_loss(p, grad=True)
    assert abs(L - L_o) <= 1e-4 * abs(L_o)
    assert np.abs(s - s_o).max() <= 1e-4 * np.abs(s_o).max()
    assert np.abs(grad - g_o).max() <= 2e-3 * np.abs(g_o).max()
    # per parameter block (each layer's Ws, Wn, b and the read-out); the loss does not change when
    # a constant is added to every score, so the gradient of bo is zero up to rounding
    o = 0
    for _, shp in learn.layer_shapes()[:-1]:
        k = int(np.prod(shp))
        a, b = grad[o:o + k], g_o[o:o + k]
        assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b), shp
        o += k
    assert abs(g_o[-1]) <= 1e-12 * np.abs(g_o).max() and abs(grad[-1]) <= 1e-5 * np.abs(g_o).max()
    g.close()
    p.close()


def test_adam_step_matches_oracle_update():
    sc = sy.shuffled(sy.make("sequential", 4, n_cams=90, n_pts=5000), 4)
    p = problem.from_scene(sc)
    p.ba_build_normal(LAM)
    theta = learn.init_params(3)
    g = binding.GNN(theta)
    L0, _, grad = g.ba_gnn_loss(p, grad=True)
    L1 = g.ba_gnn_train_step(p, lr=1e-3)
    assert L1 == L0
    th_o, _, _ = ognn.adam(theta.astype(np.float64), grad.astype(np.float64), np.zeros(theta.size),
                           np.zeros(theta.size), 1, 1e-3)
    assert np.abs(g.ba_gnn_get_params() - th_o).max() <= 1e-6
    g.close()
    p.close()


def test_order_is_the_score_ranking_and_bf16_inference_agrees():
    sc = sy.shuffled(sy.make("sequential", 5, n_cams=110, n_pts=6000), 5)
    p = problem.from_scene(sc)
    p.ba_build_normal(LAM)
    g = binding.GNN(learn.init_params(1))
    L, s = g.ba_gnn_loss(p)
    order, L32 = g.ba_gnn_order(p)
    assert L32 == L
    assert list(order) == list(np.lexsort((np.arange(s.size), s)))
    o16, L16 = g.ba_gnn_order(p, bf16=True)
    assert sorted(o16) == list(range(p.n_cams))
    assert abs(L16 - L) <= 0.05 * L + 1e-3
    g.close()
    p.close()


def _held_out_losses(g):
    out = []
    for seed in (2000, 2001):
        p = problem.from_scene(learn.training_scene("sequential", seed))
        p.ba_build_normal(LAM)
        out.append(g.ba_gnn_loss(p)[0])
        p.close()
    return out


@pytest.fixture(scope="module")
def trained():
    g = binding.GNN(learn.init_params(0))
    before = _held_out_losses(g)
    losses = learn.harvest_train(g, seeds=range(24), kinds=("sequential",), lm_steps=4, lr=3e-3)
    after = _held_out_losses(g)
    yield g, losses, before, after
    g.close()


def test_training_lowers_the_loss(trained):
    g, losses, before, after = trained
    assert len(losses) == 96 and all(np.isfinite(losses))
    # on problems it never saw, the Rayleigh quotient of the scores drops by more than half
    assert np.mean(after) < 0.5 * np.mean(before), (before, after)


@pytest.mark.parametrize("seed", [1000, 1001])
def test_learned_grouping_cuts_mcg_iterations_on_held_out_problems(trained, seed):
    g = trained[0]
    sc = sy.shuffled(sy.sequential(seed, n_cams=200, n_pts=12000), seed)
    # without the network: Algorithm 2's consecutive subsets of the given (random) camera order
    p = problem.from_scene(sc)
    p.ba_build_normal(LAM)
    base = p.ba_solve_mcg(1e-6, 1000, 8, 10.0)
    x_base = p.ba_get_delta()
    p.close()
    res = learn.solve_grouped(g, sc, 8, 10.0, precision="fp64")
    st = res["stats"]
    assert res["grouping"] == "learned" and st["status"] == 0 and st["true_rel_residual"] <= 1e-6
    assert st["iters"] <= 0.8 * base["iters"], (st["iters"], base["iters"])
    # the same solution: both solves reach 1e-6 on the same system
    m = olm.measurements(sc)
    lin = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, LAM)
    ref = osol.dense_solve(lin.S, lin.btilde)
    for x in (x_base.ravel(), res["x"].ravel()):
        d = x - ref
        assert np.sqrt(d @ (lin.S @ d) / (ref @ (lin.S @ ref))) < 1e-4
    # bfloat16 inference gives a grouping of the same quality
    r16 = learn.solve_grouped(g, sc, 8, 10.0, precision="fp64", bf16=True)
    assert r16["stats"]["iters"] <= 0.8 * base["iters"]


def test_solve_grouped_falls_back_to_the_given_order(trained):
    g = trained[0]
    sc = sy.shuffled(sy.make("tiny", 9), 9)
    # a budget of 2 iterations cannot reach 1e-6: the learned grouping fails and plain MCG runs
    res = learn.solve_grouped(g, sc, 4, 10.0, precision="fp64", max_iters=2)
    assert res["grouping"] == "fallback"
    assert res["stats"]["iters"] == 2
