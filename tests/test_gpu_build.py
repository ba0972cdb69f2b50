"""GPU parity of the linearisation and the reduced camera system (Eqs. 1-14) with the oracle.

Tolerances (float64 on both sides, different summation orders):
  * projections, residuals, Jacobians: 1e-11 of the array's largest entry - a
    handful of roundings on values of the same magnitude;
  * U, V, b_p, b_l: 1e-11 of the largest entry - sums of at most a few
    thousand products, each rounding at 1.1e-16;
  * S, b~: 1e-9 of the largest entry of S - U minus sums of G G^T cancels,
    so the error is set by the size of U, not of the result;
  * D(S)^{-1}: S_jj D_j = I to 1e-8 relative to kappa(S_jj) * 1e-16.
"""
import os

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import camera as ocam
from oracle import lm as olm
from oracle import schur as osch
from paper_2110_04015_gb300 import problem
from tests._gpu import CASES, bsr_from_gpu, oracle_system, rel_max, scene

pytestmark = pytest.mark.gpu

BUILD_CASES = ["tiny", "tiny-s3", "seq-small", "dense-small", "sequential"]


@pytest.fixture(scope="module")
def built():
    cache = {}

    def get(case, lam=1e-4, damping="marquardt"):
        key = (case, lam, damping)
        if key not in cache:
            sc = scene(case)
            p = problem.from_scene(sc, damping=damping)
            p.ba_build_normal(lam)
            cache[key] = p
        return cache[key]

    yield get
    for p in cache.values():
        p.close()


@pytest.mark.parametrize("case", BUILD_CASES)
def test_projection_matches_oracle(case):
    sc = scene(case)
    xy = problem.device_measurements(sc).cpu().numpy()
    m = olm.measurements(sc)
    assert rel_max(xy, m) < 1e-11


def test_projection_matches_hand_worked_example():
    import torch

    from paper_2110_04015_gb300 import binding

    rows = np.loadtxt(os.path.join(os.path.dirname(__file__), "golden", "bal_projection_worked_example.txt"))
    dev = "cuda"
    cams = torch.from_numpy(np.ascontiguousarray(rows[:, :9])).to(dev)
    pts = torch.from_numpy(np.ascontiguousarray(rows[:, 9:12])).to(dev)
    idx = torch.arange(rows.shape[0], dtype=torch.int32, device=dev)
    out = torch.empty((rows.shape[0], 2), dtype=torch.float64, device=dev)
    binding.ba_project(cams, pts, idx, idx, out)
    torch.cuda.synchronize()
    assert np.allclose(out.cpu().numpy(), rows[:, 12:14], rtol=1e-13, atol=1e-11)


@pytest.mark.parametrize("case", BUILD_CASES)
def test_residuals_and_jacobians_match_oracle(case, built):
    sc = scene(case)
    m, lin, _ = oracle_system(case)
    r, Jp, Jl = built(case).ba_get_linearization()
    assert rel_max(r, lin.r) < 1e-11
    assert rel_max(Jp, lin.Jp) < 1e-11
    assert rel_max(Jl, lin.Jl) < 1e-11


@pytest.mark.parametrize("case", BUILD_CASES)
def test_normal_equation_matches_oracle(case, built):
    m, lin, _ = oracle_system(case)
    U, V, bp, bl = built(case).ba_get_normal()
    assert rel_max(U, lin.ne.U) < 1e-11
    assert rel_max(V, lin.ne.V) < 1e-11
    assert rel_max(bp, lin.ne.b_p) < 1e-11
    assert rel_max(bl, lin.ne.b_l) < 1e-11


@pytest.mark.parametrize("case", BUILD_CASES)
def test_schur_matches_oracle(case, built):
    sc = scene(case)
    m, lin, _ = oracle_system(case)
    row_ptr, col, B, bt = built(case).ba_get_schur()
    Sg = bsr_from_gpu(row_ptr, col, B, sc.n_cams)
    So = lin.S
    # same block pattern: camera co-visibility (Section 3.2)
    Bo = sp.bsr_matrix(So, blocksize=(9, 9))
    Bo.sort_indices()
    assert np.array_equal(Bo.indptr, row_ptr) and np.array_equal(Bo.indices, col)
    assert np.all(np.diff(col[row_ptr[0]:row_ptr[1]]) > 0)
    scale = abs(So).max()
    assert abs(Sg - So).max() < 1e-9 * scale
    assert rel_max(bt, lin.btilde) < 1e-9
    # symmetric
    assert abs(Sg - Sg.T).max() < 1e-12 * scale


@pytest.mark.parametrize("case", ["tiny", "seq-small", "dense-small"])
def test_preconditioner_inverts_diagonal_blocks(case, built):
    sc = scene(case)
    m, lin, Dinv_o = oracle_system(case)
    D = built(case).ba_get_preconditioner()
    Sd = lin.S
    for j in range(0, sc.n_cams, max(1, sc.n_cams // 16)):
        Bj = Sd[9 * j:9 * j + 9, 9 * j:9 * j + 9].toarray()
        kappa = np.linalg.cond(Bj)
        assert np.abs(Bj @ D[j] - np.eye(9)).max() < 1e-8 * max(1.0, kappa * 1e-16 * 1e8)
        assert np.abs(D[j] - Dinv_o[j]).max() < 1e-6 * np.abs(Dinv_o[j]).max() * max(1.0, kappa * 1e-10)


def test_identity_damping_matches_oracle(built):
    m, lin, _ = oracle_system("tiny", damping="identity", lam=0.5)
    U, V, bp, bl = built("tiny", lam=0.5, damping="identity").ba_get_normal()
    assert rel_max(U, lin.ne.U) < 1e-11
    assert rel_max(V, lin.ne.V) < 1e-11


def test_dense_full_size_sampled_blocks():
    """F-1936-shaped problem: sampled S blocks and b~ rows computed one by one by the oracle."""
    from paper_2110_04015_gb300 import synthetic as sy

    sc = sy.dense(seed=0)
    m = olm.measurements(sc)
    rng = np.random.default_rng(0)
    with problem.from_scene(sc) as p:
        p.ba_build_normal(1e-4)
        row_ptr, col, B, bt = p.ba_get_schur()
        r, Jp, Jl = p.ba_get_linearization()
    # linearisation on a sample of observations
    idx = rng.choice(sc.n_obs, 20000, replace=False)
    ro = ocam.residuals(sc.cams0, sc.pts0, sc.obs_cam[idx], sc.obs_pt[idx], m[idx])
    Jpo, Jlo = ocam.jacobians(sc.cams0, sc.pts0, sc.obs_cam[idx], sc.obs_pt[idx])
    assert rel_max(r[idx], ro) < 1e-11 and rel_max(Jp[idx], Jpo) < 1e-11 and rel_max(Jl[idx], Jlo) < 1e-11
    # blocks of S for sampled camera pairs, and rows of b~
    ne = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, 1e-4, with_schur=False).ne
    jj = np.repeat(np.arange(sc.n_cams), np.diff(row_ptr))
    picks = list(rng.choice(len(col), 6, replace=False))
    picks += [int(row_ptr[j] + np.searchsorted(col[row_ptr[j]:row_ptr[j + 1]], j)) for j in (0, 1935)]
    for q in picks:
        j, k = int(jj[q]), int(col[q])
        ref = osch.schur_block(ne, j, k)
        scale = max(np.abs(ne.U[j]).max(), np.abs(ne.U[k]).max())
        assert np.abs(B[q] - ref).max() < 1e-9 * scale, (j, k)
    for j in (0, 977, 1935):
        ref = osch.btilde_block(ne, j)
        assert np.abs(bt[j] - ref).max() < 1e-9 * np.abs(ref).max()


def test_mixed_precision_schur_matches_oracle_to_float32():
    """Mixed precision keeps S as float32 Lam S Lam (Lam = diag(S)^-1/2), built from float32 Jacobians."""
    sc = scene("seq-small")
    m, lin, _ = oracle_system("seq-small")
    with problem.from_scene(sc, precision="mixed") as p:
        p.ba_build_normal(1e-4)
        row_ptr, col, B, bt = p.ba_get_schur()
    Sg = bsr_from_gpu(row_ptr, col, B, sc.n_cams)
    So = lin.S
    d = np.sqrt(np.abs(So.diagonal()))
    # relative to the scaled entries |S_ij| / (sqrt(S_ii) sqrt(S_jj)): float32 accumulation of
    # the pair products (~1e-7 each, tens of terms)
    diff = (Sg - So).tocoo()
    rel = np.abs(diff.data) / (d[diff.row] * d[diff.col])
    assert rel.max() < 1e-5
    assert rel_max(bt, lin.btilde) < 1e-9   # b~ stays float64


@pytest.mark.parametrize("case", ["tiny", "seq-small", "dense-small"])
def test_mixed_precision_build_arrays_match_oracle(case):
    """The mixed-precision build, array by array, against the float64 oracle (Eqs. 2-14).

    Float64 arrays (stated error: 1e-11 of the largest entry, as in the float64 build): r, J_p, J_l,
    V, b_l, and U, b_p (formed on request); b~ to 1e-9 (it is sum J_p^T (r - J_l V^-1 b_l), whose
    terms cancel down to the size of b~).  Float32 arrays, from float32 Jacobians recomputed from
    float32 parameters: every block of S relative to sqrt(S_aa S_bb) (the entries of Lam S Lam,
    which is what the float32 sweeps use) within 1e-5; measured ~1e-6 on the diagonal blocks (sums
    of positive semi-definite float32 terms) and off the diagonal."""
    sc = scene(case)
    m, lin, _ = oracle_system(case)
    with problem.from_scene(sc, precision="mixed") as p:
        p.ba_build_normal(1e-4)
        r, Jp, Jl = p.ba_get_linearization()
        U, V, bp, bl = p.ba_get_normal()
        row_ptr, col, B, bt = p.ba_get_schur()
    assert rel_max(r, lin.r) < 1e-11 and rel_max(Jp, lin.Jp) < 1e-11 and rel_max(Jl, lin.Jl) < 1e-11
    assert rel_max(V, lin.ne.V) < 1e-11 and rel_max(bl, lin.ne.b_l) < 1e-11
    assert rel_max(U, lin.ne.U) < 1e-11
    assert rel_max(bp, lin.ne.b_p) < 1e-11
    assert rel_max(bt, lin.btilde) < 1e-9
    Sg = bsr_from_gpu(row_ptr, col, B, sc.n_cams)
    d = np.sqrt(np.abs(lin.S.diagonal()))
    diff = (Sg - lin.S).tocoo()
    rel = np.abs(diff.data) / (d[diff.row] * d[diff.col])
    on_diag = (diff.row // 9) == (diff.col // 9)
    assert rel[on_diag].max() < 1e-5, rel[on_diag].max()
    assert rel[~on_diag].max() < 1e-5, rel[~on_diag].max()


@pytest.mark.parametrize("case", ["tiny", "dense-small"])
def test_mixed_precision_true_residual_is_the_oracle_residual(case):
    """The float64 true residual of a mixed solve (the J form S x = sum_o J_p^T (J_p x - J_l V^-1 sum
    J_l^T J_p x) + lambda D_p x, no explicit S) equals |-b~ - S x| / |b~| with the oracle's S and b~,
    up to the difference of the two systems (triangle inequality)."""
    sc = scene(case)
    m, lin, _ = oracle_system(case)
    with problem.from_scene(sc, precision="mixed") as p:
        p.ba_build_normal(1e-4)
        st = p.ba_solve_pcg(1e-6, 1000)
        x = p.ba_get_delta().ravel()
        _, _, _, bt = p.ba_get_schur()
    res_o = np.linalg.norm(-lin.btilde - lin.S @ x) / np.linalg.norm(lin.btilde)
    # the library's b~ against the oracle's, and 1e-13 of |S x| for the two operators
    bound = (np.linalg.norm(bt.ravel() - lin.btilde) + 1e-12 * np.linalg.norm(lin.S @ x)) / np.linalg.norm(lin.btilde)
    assert bound < 0.1 * res_o
    assert abs(st["true_rel_residual"] - res_o) <= bound + 1e-9 * res_o, (st["true_rel_residual"], res_o, bound)


def test_duplicate_observations_are_rejected():
    from paper_2110_04015_gb300 import binding

    sc = scene("tiny")
    xy = problem.device_measurements(sc).cpu().numpy()
    oc = np.concatenate([sc.obs_cam, sc.obs_cam[:1]])
    op = np.concatenate([sc.obs_pt, sc.obs_pt[:1]])
    with pytest.raises(binding.BAError) as e:
        binding.Problem(sc.cams0, sc.pts0, oc, op, np.concatenate([xy, xy[:1]]))
    assert e.value.code == binding.BA_ERR_INVALID_ARG and "more than once" in str(e.value)
