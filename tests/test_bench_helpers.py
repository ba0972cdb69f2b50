"""Host-side arithmetic of the benchmark's roofline figures (no GPU).

The algorithmic bytes of one product q = S p follow from the stored blocks alone: every block's
81 values and column index once, the row pointers, and three vectors of 9 n_cams values.  The
float32 symmetric product stores the upper triangle with the diagonal, (nnzb + n_cams) / 2 blocks
of a symmetric pattern.  The expected values below are that count written out for the dense
1936-camera problem (nnzb = 3,509,916) and a hand-sized case.
"""
import importlib.util
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def test_product_bytes_dense_1936():
    b = _bench()
    nnzb, nc = 3_509_916, 1936
    # float64: 3,509,916 blocks of 81 doubles + an int32 column index, 1937 int64 row pointers,
    # three vectors of 17,424 doubles
    assert b.spmv_bytes("fp64", nnzb, nc) == 3_509_916 * 652 + 8 * 1937 + 3 * 17_424 * 8 == 2_288_898_904
    # float32 symmetric: (3,509,916 + 1936) / 2 = 1,755,926 upper blocks of 81 floats + index
    assert b.spmv_bytes("mixed", nnzb, nc) == 1_755_926 * 328 + 8 * 1937 + 3 * 17_424 * 4 == 576_168_312


def test_product_bytes_tiny_symmetric_pattern():
    b = _bench()
    # 3 cameras, fully coupled: 9 stored blocks, 6 of them in the upper triangle with the diagonal
    assert b.spmv_bytes("fp64", 9, 3) == 9 * 652 + 8 * 4 + 3 * 27 * 8
    assert b.spmv_bytes("mixed", 9, 3) == 6 * 328 + 8 * 4 + 3 * 27 * 4


class _FakeHandle:
    def __init__(self, ms):
        self.ms = ms

    def ba_time_kernel(self, key, reps):
        return self.ms[key]


def test_build_roofline_fractions_and_bound():
    b = _bench()
    counts = {"o": 1_000_000, "l": 250_000, "c": 1000, "p": 2_000_000, "u": 300_000}
    ms = {k: 0.1 for k in ("linearize", "landmarks", "cam_rhs", "schur_diag", "block_jacobi", "schur_off")}
    peaks = {"hbm_gbs": 6000.0}
    rows = b.build_roofline(_FakeHandle(ms), counts, peaks)
    assert [r["kernel"].split(":")[0] for r in rows][:2] == ["k_cam_prep + k_linearize_df", "k_landmarks_df"]
    lin = rows[0]
    # 260 B per observation + 48 per landmark in 0.1 ms
    assert lin["bytes_per_launch"] == 260 * 1_000_000 + 48 * 250_000
    assert lin["achieved_gbs"] == pytest.approx(lin["bytes_per_launch"] / 0.1 / 1e6)
    assert lin["frac_hbm"] == pytest.approx(lin["achieved_gbs"] / 6000.0)
    assert lin["achieved_fp32_tflops"] == pytest.approx(1548.0 * 1_000_000 / 0.1 / 1e9)
    for r in rows:
        fr = {k[5:]: v for k, v in r.items() if k.startswith("frac_")}
        assert r["bound"] == max(fr, key=fr.get) and r["frac"] == fr[r["bound"]]
    # the preconditioner has no arithmetic count: bounded by HBM only
    assert rows[4]["bound"] == "hbm" and "frac_fp32" not in rows[4]
    off = rows[5]
    assert off["fp32_ops_per_launch"] == 486.0 * 2_000_000 + 162.0 * 300_000
