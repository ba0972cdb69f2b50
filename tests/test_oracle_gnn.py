"""Pins of the grouping network's oracle (oracle/gnn.py) against closed forms and finite differences."""
import numpy as np
import scipy.sparse as sp

from oracle import gnn
from oracle import lm as olm
from paper_2110_04015_gb300 import synthetic as sy


def _cycle(n, w=0.7):
    i = np.arange(n)
    rows = np.concatenate([i, i])
    cols = np.concatenate([(i + 1) % n, (i - 1) % n])
    return sp.csr_matrix((np.full(2 * n, w), (rows, cols)), shape=(n, n))


def test_loss_on_a_cycle_matches_its_spectrum():
    # uniform cycle: D = 2w I, and the generalised eigenvalues of (D - C, D) are 1 - cos(2 pi k / n);
    # cos(2 pi j / n) is an eigenvector of the second one (the Fiedler value)
    n = 24
    C = _cycle(n)
    s = np.cos(2 * np.pi * np.arange(n) / n)
    lam2 = 1.0 - np.cos(2 * np.pi / n)
    assert abs(gnn.loss(s, C) - lam2) < 1e-14
    # any other score has a quotient at least the Fiedler value, and the Fiedler vector is stationary
    rng = np.random.default_rng(0)
    for _ in range(20):
        assert gnn.loss(rng.standard_normal(n), C) >= lam2 - 1e-12
    L, g = gnn.loss_grad_s(3.0 * s + 5.0, C)
    assert abs(L - lam2) < 1e-13 and np.abs(g).max() < 1e-13
    # the k-th eigenvector has quotient 1 - cos(2 pi k / n)
    for k in (3, 7):
        assert abs(gnn.loss(np.sin(2 * np.pi * k * np.arange(n) / n), C) - (1 - np.cos(2 * np.pi * k / n))) < 1e-13


def _random_graph(n, rng, p=0.4):
    A = rng.random((n, n)) * (rng.random((n, n)) < p)
    A = np.triu(A, 1)
    A = A + A.T
    A[0, 1] = A[1, 0] = 0.5          # keep node degrees positive
    for j in range(n):
        A[j, (j + 1) % n] = A[(j + 1) % n, j] = max(A[j, (j + 1) % n], 0.1)
    return sp.csr_matrix(A)


def test_network_gradient_matches_finite_differences():
    rng = np.random.default_rng(1)
    n = 14
    C = _random_graph(n, rng)
    X = rng.standard_normal((n, gnn.N_FEATURES))
    theta = 0.3 * rng.standard_normal(gnn.param_count())
    L, g, _ = gnn.loss_and_grad(theta, X, C)
    idx = rng.choice(theta.size, 60, replace=False)
    # every block of the parameter vector: each layer's Ws, Wn, b and the read-out
    shapes = gnn.layer_shapes()
    starts = np.cumsum([0] + [int(np.prod(s)) for _, s in shapes])
    idx = np.concatenate([idx, starts[:-1], [theta.size - 1]])
    h = 1e-6
    for i in idx:
        e = np.zeros_like(theta)
        e[i] = h
        fd = (gnn.loss_and_grad(theta + e, X, C)[0] - gnn.loss_and_grad(theta - e, X, C)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-8, (i, fd, g[i])


def test_features_follow_their_definition_on_hand_made_cameras():
    # camera 0: no rotation; camera 1: 90 degrees about z (R maps x -> y); camera 2: 180 about x
    cams = np.zeros((3, 9))
    cams[0, 3:6] = [1.0, 2.0, 3.0]
    cams[1, :3] = [0.0, 0.0, np.pi / 2]
    cams[1, 3:6] = [1.0, 0.0, 0.0]
    cams[2, :3] = [np.pi, 0.0, 0.0]
    cams[2, 3:6] = [0.0, 0.0, 2.0]
    centres = np.array([[-1.0, -2.0, -3.0],      # -t
                        [0.0, 1.0, 0.0],          # -R^T t with R^T (1, 0, 0) = (0, -1, 0)
                        [0.0, 0.0, 2.0]])         # R = diag(1, -1, -1): -R^T t = (0, 0, 2)
    axes = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 1.0], [0.0, 0.0, -1.0]])
    C = sp.csr_matrix(np.array([[0, 1.0, 2.0], [1.0, 0, 0.5], [2.0, 0.5, 0]]))
    X = gnn.features(cams, C)
    c = centres - centres.mean(0)
    assert np.allclose(X[:, :3], c / np.sqrt((c ** 2).mean(0)), atol=1e-12)
    assert np.allclose(X[:, 3:6], axes, atol=1e-12)
    ld = np.log1p(np.array([3.0, 1.5, 2.5]))
    ld = ld - ld.mean()
    assert np.allclose(X[:, 6], ld / np.sqrt((ld ** 2).mean()), atol=1e-12)
    assert np.all(X[:, 7] == 1.0)


def test_coupling_is_symmetric_and_invariant_to_parameter_scaling():
    sc = sy.make("tiny", 0)
    m = olm.measurements(sc)
    lin = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, 1e-4)
    C = gnn.coupling(lin.S, sc.n_cams)
    Cd = C.toarray()
    assert np.allclose(Cd, Cd.T, rtol=1e-12, atol=0)
    assert np.all(np.diag(Cd) == 0) and np.all(Cd >= 0) and (Cd > 0).sum() > 0
    # rescaling the camera parameters (S -> E S E, E diagonal) leaves the Jacobi-scaled blocks as they are
    E = sp.diags(np.exp(np.random.default_rng(2).uniform(-3, 3, 9 * sc.n_cams)))
    C2 = gnn.coupling(E @ lin.S @ E, sc.n_cams).toarray()
    assert np.allclose(C2, Cd, rtol=1e-10, atol=1e-14)


def test_first_adam_step_moves_each_parameter_by_lr():
    g = np.array([3.0, -0.5, 1e-3, -2e-2])
    th, m, v = gnn.adam(np.zeros(4), g, np.zeros(4), np.zeros(4), 1, 0.01)
    # bias correction makes m_hat = g and v_hat = g^2 on the first step
    assert np.allclose(th, -0.01 * np.sign(g) * np.abs(g) / (np.abs(g) + 1e-8), rtol=1e-12)


def test_order_sorts_by_score_with_index_ties():
    s = np.array([0.5, -1.0, 0.5, 2.0, -1.0])
    assert list(gnn.order(s)) == [1, 4, 0, 2, 3]
