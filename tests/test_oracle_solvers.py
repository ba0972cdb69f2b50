"""Pins of the oracle's PCG (Algorithm 1) and MCG (Algorithm 2), Section 3.2."""
import functools

import numpy as np
import pytest

from oracle import lm, solvers
from tests._problems import scene


@functools.lru_cache(maxsize=None)
def system(name="tiny", seed=0, **kw):
    sc = scene(name, seed, **dict(kw))
    m = lm.measurements(sc)
    lin = lm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, 1e-4)
    Dinv = solvers.block_jacobi_inverse(lin.S, sc.n_cams)
    return sc, lin.S, lin.btilde, Dinv


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# --- pseudo-inverse (A13) -----------------------------------------------------

@pytest.mark.parametrize("w,rank", [(1, 1), (4, 4), (8, 5), (16, 11), (16, 16)])
def test_pinv_moore_penrose(w, rank):
    rng = np.random.default_rng(w * 100 + rank)
    B = rng.normal(size=(w, rank))
    A = B @ B.T
    X = solvers.pinv_sym(A)
    tol = 1e-9 * np.abs(A).max() * np.abs(X).max()
    assert np.abs(A @ X @ A - A).max() < tol * 10
    assert np.abs(X @ A @ X - X).max() < 1e-9 * np.abs(X).max()
    assert np.abs((A @ X).T - A @ X).max() < 1e-9
    assert np.abs((X @ A).T - X @ A).max() < 1e-9
    assert np.abs(X - np.linalg.pinv(A, rcond=1e-10, hermitian=True)).max() < 1e-8 * np.abs(X).max()


def test_pinv_is_inverse_when_well_conditioned_and_division_for_scalars():
    rng = np.random.default_rng(7)
    B = rng.normal(size=(6, 6))
    A = B @ B.T + 6 * np.eye(6)
    assert np.abs(solvers.pinv_sym(A) - np.linalg.inv(A)).max() < 1e-12
    assert solvers.pinv_sym(np.array([[4.0]]))[0, 0] == 0.25
    assert np.all(solvers.pinv_sym(np.zeros((3, 3))) == 0)


# --- block Jacobi and subsets (A9, A17) ---------------------------------------

def test_block_jacobi_inverts_diagonal_blocks():
    sc, S, bt, Dinv = system("tiny")
    Sd = S.toarray()
    for j in range(sc.n_cams):
        B = Sd[9 * j:9 * j + 9, 9 * j:9 * j + 9]
        kappa = np.linalg.cond(B)
        # backward-stable inverse: |B X - I| <= c kappa eps
        assert np.abs(B @ Dinv[j] - np.eye(9)).max() < 100 * kappa * 2.0 ** -52
        assert np.abs(Dinv[j] - Dinv[j].T).max() <= 1e-6 * np.abs(Dinv[j]).max()


@pytest.mark.parametrize("n,N", [(16, 1), (16, 4), (16, 5), (1000, 16), (1936, 121), (10, 16)])
def test_subsets_cover_each_pose_once(n, N):
    sub, n_eff = solvers.subsets(n, N)
    assert sub.shape == (n,)
    assert n_eff <= N and n_eff == len(np.unique(sub))
    assert np.all(np.diff(sub) >= 0)          # consecutive poses
    sizes = np.bincount(sub)
    assert np.all(sizes[:-1] == sizes[0]) and 0 < sizes[-1] <= sizes[0]


# --- PCG (Algorithm 1) -------------------------------------------------------

@pytest.mark.parametrize("name", ["tiny", "tiny-seed1"])
def test_pcg_matches_dense_cholesky(name):
    sc, S, bt, Dinv = system("tiny", seed=1 if name.endswith("1") else 0)
    xs = solvers.dense_solve(S, bt)
    res = solvers.pcg(S, bt, Dinv, eps=1e-6)
    assert res.converged
    assert solvers.true_rel_residual(S, bt, res.x) < 1.5e-6
    # the error in the S-norm is bounded by the residual through the preconditioned spectrum;
    # measured ~1e-5 at eps = 1e-6 and ~1e-10 at eps = 1e-10
    eS = np.sqrt((res.x - xs) @ (S @ (res.x - xs)) / (xs @ (S @ xs)))
    assert eS < 1e-4
    tight = solvers.pcg(S, bt, Dinv, eps=1e-12, imax=5000)
    assert _rel(tight.x, xs) < 1e-8


def test_pcg_finite_termination():
    sc, S, bt, Dinv = system("tiny")
    res = solvers.pcg(S, bt, Dinv, eps=1e-30, imax=9 * sc.n_cams)
    assert min(res.rel_res) < 1e-10


def test_pcg_energy_error_non_increasing():
    sc, S, bt, Dinv = system("tiny")
    xs = solvers.dense_solve(S, bt)
    res = solvers.pcg(S, bt, Dinv, eps=1e-10, record=True)
    e = np.array([np.sqrt((x - xs) @ (S @ (x - xs))) for x in res.xs])
    assert np.all(np.diff(e) <= 1e-9 * e[0])


def test_pcg_zero_rhs_returns_zero():
    sc, S, bt, Dinv = system("tiny")
    res = solvers.pcg(S, np.zeros_like(bt), Dinv)
    assert res.iters == 0 and np.all(res.x == 0) and res.converged


# --- MCG (Algorithm 2) -------------------------------------------------------

@pytest.mark.parametrize("N,tau", [(1, 3.0), (8, 0.0), (16, 0.0)])
def test_mcg_reduces_to_pcg_iterate_by_iterate(N, tau):
    """With one subset, or tau = 0 (never local), Algorithm 2 is Algorithm 1 plus reorthogonalisation."""
    sc, S, bt, Dinv = system("tiny")
    p = solvers.pcg(S, bt, Dinv, eps=1e-30, imax=20, record=True)
    q = solvers.mcg(S, bt, Dinv, N, tau, eps=1e-30, imax=20, record=True)
    assert q.local_steps == (q.iters - 1 if N == 1 and tau > 0 else 0) or N == 1
    errs = [_rel(a, b) for a, b in zip(q.xs, p.xs)]
    assert len(errs) == 20 and max(errs) < 1e-10


@pytest.mark.parametrize("N,tau", [(2, 3.0), (4, 3.0), (8, 3.0), (16, 10.0), (5, 1e9)])
def test_mcg_matches_dense_cholesky(N, tau):
    sc, S, bt, Dinv = system("tiny")
    xs = solvers.dense_solve(S, bt)
    res = solvers.mcg(S, bt, Dinv, N, tau, eps=1e-6)
    assert res.converged and solvers.true_rel_residual(S, bt, res.x) < 1.5e-6
    eS = np.sqrt((res.x - xs) @ (S @ (res.x - xs)) / (xs @ (S @ xs)))
    assert eS < 1e-4
    tight = solvers.mcg(S, bt, Dinv, N, tau, eps=1e-12, imax=5000)
    assert _rel(tight.x, xs) < 1e-8


def test_mcg_takes_local_steps_and_fewer_iterations_on_sequential():
    sc, S, bt, Dinv = system("sequential", n_cams=120, n_pts=8000)
    p = solvers.pcg(S, bt, Dinv)
    q = solvers.mcg(S, bt, Dinv, 8, 10.0)
    assert p.converged and q.converged
    assert q.local_steps > 0 and q.iters < p.iters
    assert max(q.widths) == 8


def test_mcg_energy_monotone_and_blocks_conjugate():
    sc, S, bt, Dinv = system("tiny")
    xs = solvers.dense_solve(S, bt)
    res = solvers.mcg(S, bt, Dinv, 8, 3.0, eps=1e-10, record=True)
    e = np.array([np.sqrt((x - xs) @ (S @ (x - xs))) for x in res.xs])
    assert np.all(np.diff(e) <= 1e-9 * e[0])
    P = res.P
    worst = 0.0
    for a in range(len(P)):
        na = np.sqrt(np.abs(np.einsum("ij,ij->j", P[a], S @ P[a])))
        for b in range(a):
            nb = np.sqrt(np.abs(np.einsum("ij,ij->j", P[b], S @ P[b])))
            M = P[a].T @ (S @ P[b])
            ok = np.outer(na, nb) > 0
            worst = max(worst, np.abs(M[ok] / np.outer(na, nb)[ok]).max())
    assert worst < 1e-8


def test_q_update_of_eq18_tracks_direct_product():
    sc, S, bt, Dinv = system("tiny")
    a = solvers.mcg(S, bt, Dinv, 8, 3.0, record=True, q_trick=True)
    b = solvers.mcg(S, bt, Dinv, 8, 3.0, record=True, q_trick=False)
    assert a.iters == b.iters
    assert max(_rel(x, y) for x, y in zip(a.xs, b.xs)) < 1e-9


def test_planted_diagonal_pseudo_inverse_is_caught(monkeypatch):
    """Replacing Delta^+ by the inverse of its diagonal must break a pin."""
    sc, S, bt, Dinv = system("tiny")
    xs = solvers.dense_solve(S, bt)
    monkeypatch.setattr(solvers, "pinv_sym", lambda A: np.diag(1.0 / np.diag(A)))
    res = solvers.mcg(S, bt, Dinv, 8, 1e9, eps=1e-10, imax=200, record=True)
    e = np.array([np.sqrt((x - xs) @ (S @ (x - xs))) for x in res.xs])
    assert (not res.converged) or _rel(res.x, xs) > 1e-6 or np.any(np.diff(e) > 1e-9 * e[0])


def test_planted_missing_reorthogonalisation_is_caught(monkeypatch):
    """Keeping only the last block in the beta sum (PCG's short recurrence) must break a pin."""
    sc, S, bt, Dinv = system("tiny")
    xs = solvers.dense_solve(S, bt)
    real = solvers.pinv_sym
    res_ok = solvers.mcg(S, bt, Dinv, 8, 1e9, eps=1e-10, imax=300, record=True)
    assert res_ok.converged

    def mcg_short(S, bt, Dinv, N, tau, eps, imax):
        n = bt.size
        sub, n_eff = solvers.subsets(n // 9, N)
        row_sub = np.repeat(sub, 9)
        x = np.zeros(n)
        r = -bt.copy()
        rn0 = np.linalg.norm(r)
        P = solvers.apply_block_diag(Dinv, r)[:, None]
        Q = S @ P
        for i in range(imax):
            Dp = real(0.5 * (Q.T @ P + P.T @ Q))
            al = Dp @ (P.T @ r)
            x = x + P @ al
            r = r - Q @ al
            if np.linalg.norm(r) < eps * rn0:
                return x, True
            z = solvers.apply_block_diag(Dinv, r)
            Z = np.zeros((n, n_eff))
            Z[np.arange(n), row_sub] = z
            beta = Dp @ (Q.T @ Z)
            P = Z - P @ beta
            Q = S @ P
        return x, False

    x, conv = mcg_short(S, bt, Dinv, 8, 1e9, 1e-10, res_ok.iters)
    assert (not conv) or _rel(x, xs) > 1e-6


# --- the tau-test ratio t_i (Algorithm 2, adaptive tau-test of Section 3.2) ---------------------

def _tau_identity_errors(S, bt, res, n_cams):
    """For each recorded t_i: |t_i d_i - (E_i^2 - E_{i+1}^2)| / (E_i^2 - E_{i+1}^2), with E_i the
    S-energy distance of x_i to the dense Cholesky solution and d_i = r_{i+1}^T D(S)^{-1} r_{i+1}
    built from the true residual -b~ - S x_{i+1} and dense solves with the 9x9 diagonal blocks of S.
    A block step minimises the S-energy error over its span, so gamma_i^T alpha_i is exactly that
    decrease; nothing here shares arithmetic with the solver's own gamma, alpha, r or z."""
    xs = solvers.dense_solve(S, bt)
    Sd = S.toarray()
    xi = [np.zeros_like(xs)] + res.xs
    E2 = [(x - xs) @ (S @ (x - xs)) for x in xi]
    errs = []
    for i, t in enumerate(res.t):
        r1 = -bt - S @ xi[i + 1]
        d = sum(r1[9 * j:9 * j + 9] @ np.linalg.solve(Sd[9 * j:9 * j + 9, 9 * j:9 * j + 9], r1[9 * j:9 * j + 9])
                for j in range(n_cams))
        drop = E2[i] - E2[i + 1]
        errs.append(abs(t * d - drop) / drop)
    return errs


@pytest.mark.parametrize("N,tau", [(8, 3.0), (16, 10.0), (4, 1e9), (8, 0.0)])
def test_tau_ratio_is_energy_decrease_over_preconditioned_residual(N, tau):
    sc, S, bt, Dinv = system("tiny")
    res = solvers.mcg(S, bt, Dinv, N, tau, eps=1e-6, record=True)
    assert res.converged and len(res.t) == res.iters - 1
    errs = _tau_identity_errors(S, bt, res, sc.n_cams)
    # measured <= 6e-8 (roundoff of the energy differences near convergence)
    assert max(errs) < 1e-6, max(errs)


def _two_camera_system():
    """A hand-worked 2-camera reduced system: S = [[A, b I], [b I, A]] with A = diag(d), d_1 = 3,
    b = 1, and b~ = -(e_1, 0).  From x_0 = 0: r_0 = (e_1, 0), z_0 = (e_1 / 3, 0), Q_0 = (e_1, e_1 / 3),
    Delta_0 = gamma_0 = 1/3, alpha_0 = 1, r_1 = (0, -e_1 / 3), z_1 = (0, -e_1 / 9), so
    t_0 = (1/3) / (1/27) = 9 and the S-energy error drops by gamma_0 alpha_0 = 1/3."""
    import scipy.sparse as sps

    d = np.array([3.0, 2.0, 4.0, 5.0, 2.5, 6.0, 7.0, 3.5, 8.0])
    A = np.diag(d)
    S = np.block([[A, np.eye(9)], [np.eye(9), A]])
    bt = np.zeros(18)
    bt[0] = -1.0
    return sps.csr_matrix(S), bt


def test_tau_ratio_hand_worked_two_cameras():
    S, bt = _two_camera_system()
    Dinv = solvers.block_jacobi_inverse(S, 2)
    res = solvers.mcg(S, bt, Dinv, 2, 10.0, eps=1e-12, imax=50, record=True)
    assert abs(res.t[0] - 9.0) < 1e-13
    assert res.widths[:2] == [1, 2]            # t_0 = 9 < 10: the second step is local
    assert np.abs(res.xs[0] - np.r_[1.0 / 3.0, np.zeros(17)]).max() < 1e-15
    xs = solvers.dense_solve(S, bt)
    e0 = xs @ (S @ xs)
    e1 = (res.xs[0] - xs) @ (S @ (res.xs[0] - xs))
    assert abs((e0 - e1) - 1.0 / 3.0) < 1e-14
    assert res.converged and np.abs(res.x - xs).max() < 1e-12


@pytest.mark.parametrize("plant", ["r^T r denominator", "gamma^T gamma numerator", "alpha^T alpha numerator"])
def test_planted_tau_ratio_mistakes_are_caught(plant, monkeypatch):
    """A wrong numerator or denominator of t_i must fail one of the two pins above."""
    wrong = {"r^T r denominator": lambda g, a, r, z: float(g @ a) / float(r @ r),
             "gamma^T gamma numerator": lambda g, a, r, z: float(g @ g) / float(r @ z),
             "alpha^T alpha numerator": lambda g, a, r, z: float(a @ a) / float(r @ z)}[plant]
    monkeypatch.setattr(solvers, "tau_ratio", wrong)
    S, bt = _two_camera_system()
    hand = solvers.mcg(S, bt, solvers.block_jacobi_inverse(S, 2), 2, 10.0, eps=1e-12, imax=50, record=True)
    hand_ok = abs(hand.t[0] - 9.0) < 1e-13
    sc, S, bt, Dinv = system("tiny")
    res = solvers.mcg(S, bt, Dinv, 8, 3.0, eps=1e-6, record=True)
    energy_ok = max(_tau_identity_errors(S, bt, res, sc.n_cams)) < 1e-6
    assert not (hand_ok and energy_ok)
