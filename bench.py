#!/usr/bin/env python3
"""Benchmark: time to relative residual 1e-6 per LM normal-equation solve, PCG and MCG.

One step is one pass of the whole hot path over one synthetic problem at the first
LM iteration (lambda = 1e-4): linearisation and reduced camera system (build), a
block-Jacobi PCG solve to |r| < 1e-6 |r_0| (Algorithm 1), an MCG solve to the same
tolerance (Algorithm 2), and the float64 true residual of each.  ``value`` is
milliseconds per step (lower is better); with N ranks each rank solves its own
problem (replicas, no collective on the data path) and value = T_max / (N * K).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload dense-1936]
                    [--precision fp64|mixed] [--impl ours|reference]

``--impl reference`` times the float64 CPU oracle instead (host cores only).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2110_04015_gb300 import synthetic  # noqa: E402

WORKLOADS = {
    # name: (generator, kwargs, description)
    "dense-1936": ("dense", {}, "1936 cameras on a sphere, 1.3M landmarks, ~5.2M observations, "
                                "64 co-visibility clusters, d~0.94 (F-1936-shaped)"),
    "sequential-1000": ("sequential", {}, "1000 cameras on a helix, 100k landmarks, ~700k observations, "
                                          "window 32 (banded S, d~0.04)"),
    "tiny-16": ("tiny", {}, "16 cameras on a circle, 1000 landmarks, ~4.5k observations"),
}
LAMBDA = 1e-4
TOL = 1e-6
MAX_ITERS = 1000
LM_MAX_STEPS, LM_FTOL = 25, 1e-6   # Section 4.1: at most 25 LM iterations, relative cost tolerance
METRIC = "time to rel. residual 1e-6 per LM solve (MCG vs PCG, FP64 vs mixed); HBM GB/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="dense-1936", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed"])
    ap.add_argument("--no-compare", action="store_true", help="skip the float64 comparison solves")
    ap.add_argument("--n-dirs", type=int, default=16)
    ap.add_argument("--inner-tol", type=float, default=None,
                    help="mixed precision: relative residual reduction of one float32 sweep (library default)")
    ap.add_argument("--tau", type=float, default=10.0)
    ap.add_argument("--full-size", action="store_true",
                    help="kernel cases: the benchmark's workload (--workload) instead of the 1000-camera problem")
    ap.add_argument("--kernel-case", choices=["spmv", "schur", "linearize", "mcg", "build", "pcg", "step"],
                    help="profiling mode: time one kernel on a mid-size dense problem (1000 cameras, "
                         "400k landmarks, ~1.6M observations) and exit; 'mcg' runs one MCG solve (N = 16) "
                         "with every step local, so each iteration launches the 16-column kernels; 'build' "
                         "runs three whole builds; 'pcg' two PCG solves")
    ap.add_argument("--sweep", choices=["tau", "ndirs", "density"],
                    help="sensitivity mode (Figs. 3-5 of the paper): MCG vs PCG time-to-1e-6 over tau, N or the "
                         "density of S; prints one JSON line per point and exits")
    ap.add_argument("--lm-run", action="store_true",
                    help="whole-run mode: Levenberg-Marquardt (ba_lm_step, at most 25 iterations, lambda0 1e-4, "
                         "stop at a relative cost decrease below 1e-6) once with PCG and once with MCG from the same "
                         "start; the paper's solver runtime ratio over the whole run; one JSON line")
    ap.add_argument("--batched", action="store_true",
                    help="batch mode: 64 uneven problems (50-600 cameras, 300 landmarks per camera, tracks mean 8) "
                         "solved by MCG in the same launches, against looping single-problem solves; one JSON line")
    ap.add_argument("--learned", action="store_true",
                    help="learned-grouping mode: train the grouping network on normal equations harvested from LM "
                         "iterations of shuffled synthetic problems, then MCG with and without it on held-out seeds")
    ap.add_argument("--learn-problems", type=int, default=100,
                    help="training problems per family (each gives 10 normal equations)")
    ap.add_argument("--batch-problems", type=int, default=64)
    ap.add_argument("--no-loop", action="store_true", help="batch mode: skip the looped single-problem solves")
    ap.add_argument("--no-batched", action="store_true",
                    help="default line: skip the batched 64-problem measurement reported under `batched`")
    ap.add_argument("--batch-scale", type=float, default=1.0, help="landmarks per camera x this factor")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--oracle-sample", action="store_true", help=argparse.SUPPRESS)
    ap.add_argument("--cpu-sample", action="store_true",
                    help="CPU baseline from the 1/32 landmark sample, scaled (seconds) instead of one measured "
                         "oracle step on the whole workload (about two minutes)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--host-loop", action="store_true",
                    help="drive the solve loops from the host (ba_options.host_loop), so that a profiler sees "
                         "the iteration kernels; the default device-side loops run in graphs with conditional "
                         "nodes, whose kernels ncu does not profile")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default work-item size instead of ba_autotune's choice")
    return ap.parse_args()


def load_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        d["source"] = "measured"
        return d
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "source": "fallback"}


# DRAM bytes per stored upper 9x9 block of one float32 symmetric product (k_spmv<float,1,true,true> and
# k_spmv_col together: dram__bytes_read.sum + dram__bytes_write.sum, one ncu capture of the dense
# 1936-camera product timed by ba_time_kernel, mean of two launch pairs: 594.5 + 11.4 + 0.2 + 0.6 MB
# over 1,755,926 upper blocks).
SPMV_F32_TRAFFIC_PER_UPPER_BLOCK = 345.5

# FP64 arithmetic peak of this GB300: 1.06 TFLOP/s measured with an FMA-chain kernel
# (1216 CTAs x 256 threads x 8 independent chains; 1.69 FMA per clock per SM at 2.07 GHz).
# NVIDIA's nominal figure for the part is 1.25 TFLOP/s.
FP64_PEAK_TFLOPS = 1.06
# Float32 FMA peak (nominal: 128 FMA per clock per SM, 152 SMs, 2.07 GHz; no measured figure).
FP32_PEAK_TFLOPS = 2 * 128 * 152 * 2.07e9 / 1e12

# The mixed-precision build kernel by kernel (ba_time_kernel keys), with the work of one launch in the
# counts of the problem: o observations, l landmarks, c cameras, p observation pairs of shared landmarks
# (the terms of the off-diagonal Schur blocks), u stored upper blocks off the diagonal.  Bytes: every
# array element the kernel reads or writes, once (gathered rows counted once).  Operations: floating-
# point operations per unit, FMA counted twice.  The double-float kernels (the float64 parts of the
# mixed build, on the float32 pipe) and the float32 diagonal pass count the float32 instructions they
# execute (FFMA x 2 + FADD + FMUL per observation, ncu on the 1000-camera dense build); the
# off-diagonal blocks count the algorithm's 243 FMA per pair and the scaling (2 multiplies per entry
# of a block).
BUILD_WORK = [
    ("linearize", "k_cam_prep + k_linearize_df: r, J_p, J_l per observation in double-float (Eqs. 2-4)",
     lambda n: 260 * n["o"] + 48 * n["l"], None, lambda n: 1548.0 * n["o"]),
    ("landmarks", "k_landmarks_df: V_lambda, its Cholesky factor, b_l, y_l per landmark (double-float)",
     lambda n: 64 * n["o"] + 132 * n["l"], None, lambda n: 510.0 * n["o"]),
    ("cam_rhs", "k_cam_rhs_df: b~ (Eq. 14) and the damping per camera (double-float)",
     lambda n: 216 * n["o"] + 24 * n["l"] + 144 * n["c"], None, lambda n: 1009.0 * n["o"]),
    ("schur_diag", "k_schur_diag32: S_jj and the float32 G rows (Eq. 13)",
     lambda n: 136 * n["o"] + 24 * n["l"] + 816 * n["c"], None, lambda n: 483.0 * n["o"]),
    ("block_jacobi", "k_block_jacobi: Lam and the inverse scaled diagonal blocks",
     lambda n: 1400 * n["c"], None, None),
    ("schur_off", "k_schur_off_sub + k_put_diag: the float32 blocks of Lam S Lam (Eq. 13)",
     lambda n: 8 * n["p"] + 108 * n["o"] + 1012 * n["u"] + 1944 * n["c"], None,
     lambda n: 486.0 * n["p"] + 162.0 * n["u"]),
]


def spmv_bytes(precision: str, nnzb: int, n_cams: int) -> int:
    """Algorithmic bytes of one product q = S p: the stored blocks of S once (81 values and a 4-byte
    column index each; float64 streams every block, the float32 symmetric product the upper triangle
    with the diagonal, (nnzb + n_cams) / 2 blocks, each serving S_jk p_k and S_jk^T p_j), the row
    pointers, and three vectors of 9 n_cams values (p read, q written, one more read for the
    per-camera sums).  The transposed terms the symmetric product writes and reads back are
    implementation traffic, not counted."""
    elt = 8 if precision == "fp64" else 4
    blocks = nnzb if precision == "fp64" else (nnzb + n_cams) // 2
    return blocks * (81 * elt + 4) + 8 * (n_cams + 1) + 3 * 9 * n_cams * elt


def build_roofline(p, counts, peaks, reps=3):
    """Each kernel of the mixed build timed alone (ba_time_kernel, L2 evicted before each launch),
    against the HBM copy peak and the arithmetic peak of its precision; `bound` is the larger fraction."""
    out = []
    for key, what, fbytes, f64, f32 in BUILD_WORK:
        t = p.ba_time_kernel(key, reps)
        e = {"kernel": what, "ms_per_launch": t, "bytes_per_launch": fbytes(counts)}
        e["achieved_gbs"] = e["bytes_per_launch"] / t / 1e6
        e["frac_hbm"] = e["achieved_gbs"] / peaks["hbm_gbs"]
        fr = {"hbm": e["frac_hbm"]}
        if f64:
            e["fp64_ops_per_launch"] = f64(counts)
            e["achieved_fp64_tflops"] = e["fp64_ops_per_launch"] / t / 1e9
            e["frac_fp64"] = fr["fp64"] = e["achieved_fp64_tflops"] / FP64_PEAK_TFLOPS
        if f32:
            e["fp32_ops_per_launch"] = f32(counts)
            e["achieved_fp32_tflops"] = e["fp32_ops_per_launch"] / t / 1e9
            e["frac_fp32"] = fr["fp32"] = e["achieved_fp32_tflops"] / FP32_PEAK_TFLOPS
        e["bound"] = max(fr, key=fr.get)
        e["frac"] = fr[e["bound"]]
        out.append(e)
    return out


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 200 ms while running."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------------------------------
# CPU oracle timing (the baseline and the reference arm)

def oracle_sample_step(sc, frac: int = 32) -> dict:
    """The float64 oracle on a bounded sample of the workload, scaled to the full problem.

    Sample: every frac-th landmark of the same scene with all its observations.  The
    oracle linearises and forms S, b~ (Eqs. 2-14), then solves to 1e-6 by PCG and MCG.
    Build time is scaled by the observation ratio, solve times by the ratio of nonzero
    9x9 blocks of S (the cost of one product with S).
    """
    from oracle import camera as ocam
    from oracle import lm as olm
    from oracle import schur as osch
    from oracle import solvers as osol

    keep = (sc.obs_pt % frac) == 0
    oc, op = sc.obs_cam[keep], sc.obs_pt[keep]
    m = ocam.project(sc.cams_true, sc.pts_true, oc, op) + sc.noise[keep]
    t0 = time.perf_counter()
    lin = olm.linearise(sc.cams0, sc.pts0, oc, op, m, LAMBDA)
    Dinv = osol.block_jacobi_inverse(lin.S, sc.n_cams)
    t1 = time.perf_counter()
    pcg = osol.pcg(lin.S, lin.btilde, Dinv, TOL, MAX_ITERS)
    t2 = time.perf_counter()
    mcg = osol.mcg(lin.S, lin.btilde, Dinv, 16, 10.0, TOL, MAX_ITERS)
    t3 = time.perf_counter()
    nnzb_s = osch.density(lin.S, sc.n_cams) * sc.n_cams ** 2
    return {"t_build": t1 - t0, "t_pcg": t2 - t1, "t_mcg": t3 - t2, "n_obs_sample": int(keep.sum()),
            "n_obs": sc.n_obs, "nnzb_sample": nnzb_s, "pcg_iters": pcg.iters, "mcg_iters": mcg.iters,
            "n_cams": sc.n_cams, "frac": frac}


def cpu_info() -> dict:
    """Host cores and CPU model of the machine the oracle runs on."""
    import platform

    model = ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or platform.machine()}


def oracle_full_step(sc) -> dict:
    """One step of the float64 oracle on the whole workload, every part timed (nothing scaled):
    linearisation and reduced camera system (Eqs. 2-14) with its block-Jacobi preconditioner, then
    PCG (Algorithm 1) and MCG (Algorithm 2, N = 16, tau = 10) to 1e-6.  The measurements (the
    scene's input) are formed before the clock starts, as on the GPU side."""
    from oracle import camera as ocam
    from oracle import lm as olm
    from oracle import solvers as osol

    m = ocam.project(sc.cams_true, sc.pts_true, sc.obs_cam, sc.obs_pt) + sc.noise
    t0 = time.perf_counter()
    lin = olm.linearise(sc.cams0, sc.pts0, sc.obs_cam, sc.obs_pt, m, LAMBDA)
    Dinv = osol.block_jacobi_inverse(lin.S, sc.n_cams)
    t1 = time.perf_counter()
    pcg = osol.pcg(lin.S, lin.btilde, Dinv, TOL, MAX_ITERS)
    t2 = time.perf_counter()
    mcg = osol.mcg(lin.S, lin.btilde, Dinv, 16, 10.0, TOL, MAX_ITERS)
    t3 = time.perf_counter()
    return {"t_build": t1 - t0, "t_pcg": t2 - t1, "t_mcg": t3 - t2, "ms": 1e3 * (t3 - t0),
            "pcg_iters": pcg.iters, "mcg_iters": mcg.iters, "mcg_local": mcg.local_steps,
            "true_rel_residual": [osol.true_rel_residual(lin.S, lin.btilde, pcg.x),
                                  osol.true_rel_residual(lin.S, lin.btilde, mcg.x)]}


def full_text(f: dict, sc) -> str:
    return (f"the whole workload ({sc.n_cams} cameras, {sc.n_obs} observations), one step measured: build "
            f"{f['t_build']:.1f} s, PCG {f['t_pcg']:.1f} s ({f['pcg_iters']} it), MCG N=16 tau=10 {f['t_mcg']:.1f} s "
            f"({f['mcg_iters']} it, {f['mcg_local']} local); numpy/scipy float64, the sparse products on one thread")


THREAD_VARS = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS")


def thread_scaling(workload: str, counts=(1, 4, None)) -> dict:
    """The oracle step on the 1/32 landmark sample with 1, 4 and all BLAS/OpenMP threads, each in a
    fresh child process (the thread count of numpy's BLAS is fixed when it loads).  The dense parts
    of the oracle use these threads; scipy's sparse products run on one."""
    out = {}
    for n in counts:
        k = n if n else (os.cpu_count() or 1)
        env = dict(os.environ)
        for v in THREAD_VARS:
            env[v] = str(k)
        try:
            res = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-sample", "--workload", workload],
                                 env=env, capture_output=True, text=True, timeout=600)
            out[str(k)] = json.loads(res.stdout.strip().splitlines()[-1])["seconds"]
        except (subprocess.SubprocessError, ValueError, IndexError, KeyError) as e:
            out[str(k)] = f"failed: {type(e).__name__}"
    return {"sample": "landmarks with index % 32 == 0: build + PCG + MCG N=16 tau=10, seconds by thread count "
                      "(OMP/BLAS thread variables of a child process)", "seconds": out}


def run_oracle_sample(a):
    """Child process of thread_scaling: one oracle step on the 1/32 sample, printed as JSON."""
    gen, kw, _ = WORKLOADS[a.workload]
    sc = synthetic.make(gen, 0, **kw)
    s = oracle_sample_step(sc)
    print(json.dumps({"seconds": round(s["t_build"] + s["t_pcg"] + s["t_mcg"], 3)}), flush=True)


def sample_text(s: dict, nnzb_full) -> str:
    return (f"landmarks with index % {s['frac']} == 0 ({s['n_obs_sample']} of {s['n_obs']} observations): oracle "
            f"build + PCG ({s['pcg_iters']} it) + MCG N=16 tau=10 ({s['mcg_iters']} it) to 1e-6 in "
            f"{s['t_build'] + s['t_pcg'] + s['t_mcg']:.1f} s; build scaled by observations, solves by nonzero "
            f"blocks of S ({s['nnzb_sample']:.0f} -> {nnzb_full:.0f})")


def scale_oracle(s: dict, nnzb_full: float) -> float:
    """Estimated ms of one full step from a sample step."""
    b = s["t_build"] * s["n_obs"] / s["n_obs_sample"]
    r = nnzb_full / s["nnzb_sample"]
    return 1e3 * (b + (s["t_pcg"] + s["t_mcg"]) * r)


def cpu_threads() -> int:
    try:
        import threadpoolctl

        info = threadpoolctl.threadpool_info()
        n = max((d.get("num_threads", 1) for d in info), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


def nnzb_estimate(sc) -> float:
    """Nonzero 9x9 blocks of S for the full scene: camera pairs sharing a landmark."""
    import scipy.sparse as sp

    A = sp.csr_matrix((np.ones(sc.n_obs, np.float32), (sc.obs_cam, sc.obs_pt)), shape=(sc.n_cams, sc.n_pts))
    return float((A @ A.T).nnz)


def run_reference(a, rank: int, world: int):
    """The reference arm: the float64 oracle on the same workload, on the host cores.

    The paper ships no code, so the oracle written from it stands in for the reference.  Its warm-up
    steps run on the 1/32 landmark sample; then ONE step on the whole workload is measured (build,
    PCG and MCG, nothing scaled): a full step takes about two minutes, so the requested K timed steps
    are not repeated (``steps`` is 1, ``steps_requested`` K)."""
    if rank != 0:
        return
    gen, kw, desc = WORKLOADS[a.workload]
    sc = synthetic.make(gen, 0, **kw)
    t_start = time.perf_counter()
    for _ in range(min(a.warmup, 2)):
        oracle_sample_step(sc)
    t0 = time.perf_counter()
    f = oracle_full_step(sc)
    t1 = time.perf_counter()
    v = f["ms"]
    info = cpu_info()
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "ms/step", "n_gpus": world,
            "steps": 1, "steps_requested": a.steps, "warmup": a.warmup, "ms_per_step": v,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded generator; BAL/1dSfM datasets absent)",
            "config": {"workload": a.workload, "description": desc, "n_cams": sc.n_cams, "n_pts": sc.n_pts,
                       "n_obs": sc.n_obs, "lambda": LAMBDA, "tol": TOL, "max_iters": MAX_ITERS,
                       "mcg": {"n_dirs": 16, "tau": 10.0}, "precision": "fp64"},
            "cpu_baseline": {"value": v, "unit": "ms/step", "cores": cpu_threads(), "kind": "oracle",
                             "sample": full_text(f, sc), **info},
            "breakdown": {"build_s": f["t_build"], "pcg_s": f["t_pcg"], "mcg_s": f["t_mcg"],
                          "pcg_iters": f["pcg_iters"], "mcg_iters": f["mcg_iters"], "mcg_local": f["mcg_local"],
                          "true_rel_residual": f["true_rel_residual"]},
            "e2e": {"value": v, "unit": "ms/step", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "timed_s": t1 - t0, "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------------------------------
# replicas: every rank solves its own problem; only the timing is combined

def rank_seed(rank: int) -> int:
    """Scene seed of a rank: independent problems, no data exchanged between ranks."""
    return rank


def aggregate_ms(t_local_ms: float, steps: int, world: int, dist=None, device=None) -> tuple[float, float]:
    """(T_max over ranks, whole-job ms per step = T_max / (world * steps))."""
    T = float(t_local_ms)
    if dist is not None and world > 1:
        import torch

        t = torch.tensor([T], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        T = float(t.item())
    return T, T / (steps * world)


def run_ours(a, rank: int, world: int, local_rank: int):
    import torch

    from paper_2110_04015_gb300 import problem

    dist = None
    if world > 1:
        import torch.distributed as dist

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    gen, kw, desc = WORKLOADS[a.workload]
    sc = synthetic.make(gen, seed=rank_seed(rank), **kw)
    xy = problem.device_measurements(sc, device=str(dev))
    torch.cuda.synchronize()
    t_create = time.perf_counter()
    p = problem.from_scene(sc, precision=a.precision, xy=xy, host_loop=int(a.host_loop),
                           **({} if a.inner_tol is None else {"inner_tol": a.inner_tol}))
    create_ms = (time.perf_counter() - t_create) * 1e3
    stream = torch.cuda.current_stream()
    p.ba_set_stream(stream)

    def step():
        p.ba_build_normal(LAMBDA)
        s1 = p.ba_solve_pcg(TOL, MAX_ITERS)
        s2 = p.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau)
        return s1, s2

    # work-item size of the tile-streaming products, measured once before the warm-up (setup,
    # outside the timed region; ba_autotune times the S p product for each candidate size)
    tuned = None
    if not a.no_autotune:
        p.ba_build_normal(LAMBDA)
        cb, t_cb, cfg = p.ba_autotune(reps=5)
        tuned = {"item_blocks": cb, "spmv_config": cfg, "spmv_ms": t_cb}
    for _ in range(a.warmup):
        step()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local_rank)
    clocks.start()
    l0 = p.ba_get_launch_count()
    times, stats = [], []
    for _ in range(a.steps):
        flush.zero_()
        e0.record(stream)
        st = step()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        stats.append(st)
    torch.cuda.synchronize()
    launches = p.ba_get_launch_count() - l0
    if dist:
        dist.barrier()
    clk = clocks.stop()
    T, value = aggregate_ms(sum(times), a.steps, world, dist, dev)

    # breakdown of the last step
    s_pcg, s_mcg = stats[-1]
    for s1, s2 in stats:
        assert s1["true_rel_residual"] <= 1.5e-6 and s2["true_rel_residual"] <= 1.5e-6, (s1, s2)

    # roofline of the dominant kernel: the product q = S p of the Krylov solves
    nnzb = p.ba_get_schur_nnzb()
    nnzb_u = (nnzb + sc.n_cams) // 2       # upper triangle with the diagonal
    t_spmv = p.ba_time_kernel("spmv", reps=10)
    t_schur = p.ba_time_kernel("schur", reps=3)
    peaks = load_peaks()
    spmv_flops = 162.0 * nnzb
    # the float32 symmetric product streams the upper triangle once; the 9 transposed terms per
    # strict upper block it writes and reads back (72 B) are not counted as algorithmic
    sbytes = spmv_bytes(a.precision, nnzb, sc.n_cams)
    if a.precision == "fp64":
        roof = {"kernel": "k_spmv<double,1,true> (q = S p, Algorithm 1)", "bound": "alu", "achieved": spmv_flops / t_spmv / 1e9,
                "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "traffic": None,
                "bytes_per_launch": sbytes, "flops_per_launch": spmv_flops, "ms_per_launch": t_spmv,
                "achieved_gbs": sbytes / t_spmv / 1e6, "hbm_peak_gbs": peaks["hbm_gbs"],
                "peak_source": "measured FP64 FMA throughput 1.06 TFLOP/s (nominal 1.25)"}
        roof["frac"] = roof["achieved"] / roof["peak"]
    else:
        traffic = None if SPMV_F32_TRAFFIC_PER_UPPER_BLOCK is None else SPMV_F32_TRAFFIC_PER_UPPER_BLOCK * nnzb_u
        roof = {"kernel": "k_spmv<float,1,true,true> + k_spmv_col (q = S p from the upper triangle of S, Algorithm 1)",
                "bound": "hbm", "achieved": sbytes / t_spmv / 1e6,
                "peak": peaks["hbm_gbs"], "unit": "GB/s", "traffic": traffic,
                "traffic_source": "ncu dram bytes of this product on dense-1936 (both launches), per upper block",
                "bytes_per_launch": sbytes, "upper_blocks": nnzb_u,
                "bytes_moved_model": sbytes + 72 * (nnzb_u - sc.n_cams),
                "ms_per_launch": t_spmv, "peak_source": peaks["source"]}
        roof["frac"] = roof["achieved"] / roof["peak"]
    # the build kernel by kernel (mixed precision)
    roof_build = None
    if a.precision == "mixed":
        track = np.bincount(sc.obs_pt, minlength=sc.n_pts).astype(np.int64)
        counts = {"o": sc.n_obs, "l": sc.n_pts, "c": sc.n_cams, "p": int((track * (track - 1) // 2).sum()),
                  "u": (nnzb - sc.n_cams) // 2}
        roof_build = {"counts": counts, "schur_ms": t_schur, "kernels": build_roofline(p, counts, peaks)}

    # end to end through the host-buffer API: parameters in, both solutions out
    e2e = None
    if not a.no_e2e:
        # inputs and the result through pinned host buffers
        cams_h = torch.from_numpy(np.ascontiguousarray(sc.cams0)).pin_memory()
        pts_h = torch.from_numpy(np.ascontiguousarray(sc.pts0)).pin_memory()
        dx_h = torch.empty((sc.n_cams, 9), dtype=torch.float64).pin_memory()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(a.steps):
            p.ba_set_params(cams_h, pts_h)
            p.ba_build_normal(LAMBDA)
            p.ba_solve_pcg(TOL, MAX_ITERS)
            p.ba_get_delta(dx_h)
            p.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau)
            p.ba_get_delta(dx_h)
        torch.cuda.synchronize()
        Te, e2e_value = aggregate_ms((time.perf_counter() - t0) * 1e3, a.steps, world, dist, dev)
        nbytes = lambda t: t.numel() * t.element_size()
        e2e = {"value": e2e_value, "unit": "ms/step", "host_buffers": "pinned",
               "h2d_bytes_per_step": int(nbytes(cams_h) + nbytes(pts_h)), "d2h_bytes_per_step": int(2 * nbytes(dx_h))}

    # the solutions of this precision (outside the timed region), for the comparison with float64
    p.ba_build_normal(LAMBDA)
    p.ba_solve_pcg(TOL, MAX_ITERS)
    dx_pcg = p.ba_get_delta().copy()
    p.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau)
    dx_mcg = p.ba_get_delta().copy()
    p.close()

    # the same step in float64 throughout, for the FP64-vs-mixed comparison of the metric
    fp64 = None
    if a.precision == "mixed" and not a.no_compare:
        q = problem.from_scene(sc, precision="fp64", xy=xy, host_loop=int(a.host_loop))
        q.ba_set_stream(stream)
        if not a.no_autotune:
            q.ba_build_normal(LAMBDA)
            q.ba_autotune(reps=3)

        def step64():
            q.ba_build_normal(LAMBDA)
            return q.ba_solve_pcg(TOL, MAX_ITERS), q.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau)

        step64()
        t64 = []
        for _ in range(2):
            flush.zero_()
            e0.record(stream)
            s1, s2 = step64()
            e1.record(stream)
            e1.synchronize()
            t64.append(e0.elapsed_time(e1))
        t_sp64 = q.ba_time_kernel("spmv", reps=5)
        # each mixed solution against the float64 solution of the same algorithm: both meet the float64
        # true residual 1e-6, so they differ by at most about the condition of S times that
        q.ba_build_normal(LAMBDA)
        q.ba_solve_pcg(TOL, MAX_ITERS)
        d64_pcg = q.ba_get_delta().copy()
        q.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau)
        d64_mcg = q.ba_get_delta().copy()
        rel = lambda d, r: float(np.linalg.norm(d - r) / np.linalg.norm(r))
        colrel = lambda d, r: float((np.abs(d - r).max(axis=0) / np.abs(r).max(axis=0)).max())
        mixed_err = {"pcg_dx_rel_diff": rel(dx_pcg, d64_pcg), "mcg_dx_rel_diff": rel(dx_mcg, d64_mcg),
                     "pcg_dx_max_param_rel_diff": colrel(dx_pcg, d64_pcg),
                     "mcg_dx_max_param_rel_diff": colrel(dx_mcg, d64_mcg),
                     "true_rel_residual_float64": [s_pcg["true_rel_residual"], s_mcg["true_rel_residual"]],
                     "note": "mixed precision against the float64 GPU solve of the same normal equation (itself "
                             "parity-tested against the float64 oracle); the true residuals are float64"}
        fp64 = {"step_ms": float(np.mean(t64)), "pcg": {k: s1[k] for k in ("iters", "ms", "true_rel_residual")},
                "mcg": {k: s2[k] for k in ("iters", "local_steps", "ms", "true_rel_residual")},
                "build_ms": float(np.mean(t64)) - s1["ms"] - s2["ms"],
                "spmv": {"kernel": "k_spmv<double,1,true>", "ms_per_launch": t_sp64,
                         "achieved_tflops": 162.0 * nnzb / t_sp64 / 1e9, "peak_tflops": FP64_PEAK_TFLOPS},
                "mixed_vs_fp64": mixed_err}
        q.close()

    # 64 uneven problems in one handle against a loop over 64 handles (the batched solve of the
    # hot path), on rank 0 of a one-GPU run
    batched = None
    if rank == 0 and world == 1 and not a.no_batched:
        batched = measure_batched(a, 3, 1, True)

    cpu = None
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        if a.cpu_sample:
            s = oracle_sample_step(sc)
            cpu = {"value": scale_oracle(s, nnzb), "unit": "ms/step", "cores": cpu_threads(), "kind": "oracle",
                   "sample": sample_text(s, nnzb), **cpu_info()}
        else:
            f = oracle_full_step(sc)
            cpu = {"value": f["ms"], "unit": "ms/step", "cores": cpu_threads(), "kind": "oracle",
                   "sample": full_text(f, sc), **cpu_info(), "thread_scaling": thread_scaling(a.workload)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "ms/step", "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": T / a.steps, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else "f32+f64",
            "data": "synthetic (seeded generator; BAL/1dSfM datasets absent)",
            "config": {"workload": a.workload, "description": desc, "n_cams": sc.n_cams, "n_pts": sc.n_pts,
                       "n_obs": sc.n_obs, "nnzb": nnzb, "lambda": LAMBDA, "tol": TOL, "max_iters": MAX_ITERS,
                       "mcg": {"n_dirs": a.n_dirs, "tau": a.tau}, "precision": a.precision,
                       "parallelism": f"replicas x{world}", "create_ms": create_ms,
                       "l2": "256 MiB buffer written before every timed step; S and the observation arrays exceed L2"},
            "breakdown": {
                "step_ms": [round(x, 4) for x in times],
                "pcg": {k: s_pcg[k] for k in ("iters", "ms", "true_rel_residual", "status", "refinements")},
                "mcg": {k: s_mcg[k] for k in ("iters", "local_steps", "ms", "true_rel_residual", "status",
                                              "history_cols", "n_dirs_eff", "refinements")},
                "build_ms": T / a.steps - s_pcg["ms"] - s_mcg["ms"],
            },
            "roofline": roof,
            "roofline_build": roof_build,
            "fp64": fp64,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(launches),
            "clocks": clk,
            "autotune": tuned,
            "batched": batched,
        }
        print(json.dumps(line), flush=True)


def run_kernel_case(a):
    """A problem small enough for multi-pass ncu captures (S ~0.3 GB float32), larger than L2; or
    (`step`) two steps of the benchmark's own workload with the solve loops driven from the host, for
    a profiler's launch list (ncu does not profile kernels in graphs with conditional nodes)."""
    import torch

    from paper_2110_04015_gb300 import problem

    if a.kernel_case == "step":
        gen, kw, _ = WORKLOADS[a.workload]
        sc = synthetic.make(gen, 0, **kw)
        p = problem.from_scene(sc, precision=a.precision, host_loop=1, item_blocks=256)
        for rep in range(2):
            t0 = time.perf_counter()
            p.ba_build_normal(LAMBDA)
            s1 = p.ba_solve_pcg(TOL, MAX_ITERS)
            s2 = p.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau)
            torch.cuda.synchronize()
            print(json.dumps({"kernel_case": "step", "workload": a.workload, "rep": rep,
                              "host_ms": (time.perf_counter() - t0) * 1e3, "pcg_iters": s1["iters"],
                              "mcg_iters": s2["iters"], "mcg_local": s2["local_steps"]}), flush=True)
        p.close()
        return
    if a.full_size:
        gen, kw, _ = WORKLOADS[a.workload]
        sc = synthetic.make(gen, 0, **kw)
    else:
        sc = synthetic.dense(seed=0, n_cams=1000, n_pts=400_000, n_clusters=33)
    # work items of 256 blocks: what ba_autotune picks for the 1000-camera problem
    p = problem.from_scene(sc, precision=a.precision, host_loop=int(a.host_loop), item_blocks=256)
    p.ba_build_normal(LAMBDA)
    if a.kernel_case == "build":
        import torch as _t

        e0, e1 = _t.cuda.Event(enable_timing=True), _t.cuda.Event(enable_timing=True)
        for rep in range(3):
            e0.record()
            p.ba_build_normal(LAMBDA)
            e1.record()
            e1.synchronize()
            print(json.dumps({"kernel_case": "build", "precision": a.precision, "rep": rep,
                              "ms": e0.elapsed_time(e1)}), flush=True)
        p.close()
        return
    if a.kernel_case == "pcg":
        for rep in range(2):
            st = p.ba_solve_pcg(TOL, MAX_ITERS)
            print(json.dumps({"kernel_case": "pcg", "precision": a.precision, "rep": rep, "ms": st["ms"],
                              "iters": st["iters"], "true_rel_residual": st["true_rel_residual"]}), flush=True)
        p.close()
        return
    if a.kernel_case == "mcg":
        for rep in range(2):
            st = p.ba_solve_mcg(TOL, MAX_ITERS, 16, 1e9)
            print(json.dumps({"kernel_case": "mcg", "precision": a.precision, "rep": rep, "ms": st["ms"],
                              "iters": st["iters"], "local_steps": st["local_steps"],
                              "true_rel_residual": st["true_rel_residual"]}), flush=True)
        p.close()
        torch.cuda.synchronize()
        return
    ms = p.ba_time_kernel(a.kernel_case, 3)
    print(json.dumps({"kernel_case": a.kernel_case, "precision": a.precision, "nnzb": p.ba_get_schur_nnzb(),
                      "n_obs": sc.n_obs, "ms_per_launch": ms}), flush=True)
    p.close()
    torch.cuda.synchronize()


def run_sweep(a):
    """Solver time ratio t_MCG / t_PCG (the paper's "solver runtime ratio") against tau, N or density."""
    import torch

    from paper_2110_04015_gb300 import problem

    def measure(p, reps=2):
        p.ba_build_normal(LAMBDA)
        pcg = [p.ba_solve_pcg(TOL, MAX_ITERS) for _ in range(reps)]
        return min(s["ms"] for s in pcg), pcg[-1]["iters"]

    def one(sc, label, points):
        p = problem.from_scene(sc, precision=a.precision)
        t_pcg, it_pcg = measure(p)
        for N, tau in points:
            runs = [p.ba_solve_mcg(TOL, MAX_ITERS, N, tau) for _ in range(2)]
            m = min(r["ms"] for r in runs)
            print(json.dumps({"sweep": a.sweep, **label, "n_dirs": N, "tau": tau, "precision": a.precision,
                              "pcg_ms": t_pcg, "pcg_iters": it_pcg, "mcg_ms": m, "mcg_iters": runs[-1]["iters"],
                              "local_steps": runs[-1]["local_steps"], "ratio": m / t_pcg,
                              "true_rel_residual": runs[-1]["true_rel_residual"]}), flush=True)
        p.close()
        torch.cuda.synchronize()

    gen, kw, _ = WORKLOADS[a.workload]
    if a.sweep == "tau":
        one(synthetic.make(gen, 0, **kw), {"workload": a.workload},
            [(16, t) for t in (0.0, 1.0, 2.0, 3.0, 6.0, 10.0, 30.0, 1e9)])
    elif a.sweep == "ndirs":
        one(synthetic.make(gen, 0, **kw), {"workload": a.workload}, [(N, 10.0) for N in (1, 2, 4, 8, 16)])
    else:
        for pu in (0.01, 0.03, 0.1, 0.25, 0.6):
            sc = synthetic.dense(seed=0, n_cams=1000, n_pts=400_000, n_clusters=33, p_uniform=pu)
            d = nnzb_estimate(sc) / sc.n_cams ** 2
            one(sc, {"workload": "dense-1000x400k", "p_uniform": pu, "density": d}, [(16, 10.0)])


def run_lm(a):
    """The paper's solver runtime ratio over a whole bundle-adjustment run (Section 5): the LM loop
    with each solver from the same start, summing the solve times of its normal equations."""
    import torch

    from paper_2110_04015_gb300 import problem

    gen, kw, desc = WORKLOADS[a.workload]
    sc = synthetic.make(gen, 0, **kw)
    xy = problem.device_measurements(sc)
    runs = {}
    for solver in ("pcg", "mcg"):
        for rep in range(2):   # the first run pays for graph capture and buffer growth
            p = problem.from_scene(sc, precision=a.precision, xy=xy)
            cost0 = p.ba_cost()
            steps = []
            for _ in range(LM_MAX_STEPS):
                st = p.ba_lm_step(solver, lambda0=LAMBDA, tol=TOL, max_iters=MAX_ITERS, n_dirs=a.n_dirs, tau=a.tau,
                                  ftol=LM_FTOL)
                steps.append(st)
                if st["converged"]:
                    break
            cost_end = p.ba_cost()
            p.close()
            torch.cuda.synchronize()
        runs[solver] = {
            "lm_iterations": len(steps), "accepted": sum(s["accepted"] for s in steps),
            "converged": bool(steps[-1]["converged"]), "cost_start": cost0,
            "cost_end": cost_end,
            "solver_iters": sum(s["solver_iters"] for s in steps),
            "solve_ms": sum(s["solve_ms"] for s in steps), "total_ms": sum(s["ms"] for s in steps),
        }
    r_solve = runs["mcg"]["solve_ms"] / runs["pcg"]["solve_ms"]
    print(json.dumps({
        "mode": "lm-run", "metric": "solver runtime ratio t_MCG / t_PCG over a whole LM run (Section 5)",
        "value": r_solve, "unit": "ratio", "higher_is_better": False, "precision": a.precision,
        "config": {"workload": a.workload, "description": desc, "n_cams": sc.n_cams, "n_obs": sc.n_obs,
                   "lambda0": LAMBDA, "tol": TOL, "lm_max_steps": LM_MAX_STEPS, "lm_ftol": LM_FTOL,
                   "mcg": {"n_dirs": a.n_dirs, "tau": a.tau}},
        "pcg": runs["pcg"], "mcg": runs["mcg"],
        "total_ratio": runs["mcg"]["total_ms"] / runs["pcg"]["total_ms"],
    }), flush=True)


def run_batched(a):
    """Batched uneven problems (`--batched`): one JSON line."""
    print(json.dumps(measure_batched(a, a.steps, a.warmup, not a.no_loop)), flush=True)


def measure_batched(a, steps, warmup, loop):
    """Batched uneven problems: one handle (ba_batch_create) against a loop over single-problem handles.

    A step is the build and the MCG solve of every problem to the float64 tolerance; both arms use
    the same precision, tolerance, N and tau.  The batch's work-item size is chosen by ba_autotune.
    """
    import torch

    from paper_2110_04015_gb300 import problem

    scs = synthetic.batched(seed=0, n_problems=a.batch_problems, scale=a.batch_scale)
    n_cams = sum(sc.n_cams for sc in scs)
    n_obs = sum(sc.n_obs for sc in scs)
    stream = torch.cuda.current_stream()
    pb = problem.from_scenes(scs, precision=a.precision)
    pb.ba_set_stream(stream)
    pb.ba_build_normal(LAMBDA)
    t_heur = pb.ba_time_kernel("spmv", reps=5)
    cb, t_tuned, cfg = pb.ba_autotune(reps=5)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)

    def timed(fn):
        flush.zero_()
        e0.record(stream)
        out = fn()
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1), out

    def step_batch():
        pb.ba_build_normal(LAMBDA)
        return pb.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau)

    for _ in range(warmup):
        step_batch()
    l0 = pb.ba_get_launch_count()
    clocks = ClockSampler(0)
    clocks.start()
    tb = []
    for _ in range(steps):
        t, st = timed(step_batch)
        tb.append(t)
    clk = clocks.stop()
    launches = (pb.ba_get_launch_count() - l0) // steps
    per = pb.ba_get_batch_stats()
    assert all(s["status"] == 0 and s["true_rel_residual"] <= 1.5e-6 for s in per), per
    nnzb = pb.ba_get_schur_nnzb()
    peaks = load_peaks()
    elt = 8 if a.precision == "fp64" else 4
    sbytes = spmv_bytes(a.precision, nnzb, n_cams)
    pb.close()

    tl = []
    if loop:
        singles = [problem.from_scene(sc, precision=a.precision) for sc in scs]
        for q in singles:
            q.ba_set_stream(stream)

        def step_loop():
            out = []
            for q in singles:
                q.ba_build_normal(LAMBDA)
                out.append(q.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau))
            return out

        step_loop()
        for _ in range(max(1, min(steps, 3))):
            t, sts = timed(step_loop)
            tl.append(t)
        assert all(s["status"] == 0 for s in sts)
        for q in singles:
            q.close()
    torch.cuda.synchronize()
    ms_b = float(np.mean(tb))
    ms_l = float(np.mean(tl)) if tl else None
    line = {
        "mode": "batched", "metric": "time to rel. residual 1e-6, all problems of a batch (MCG)",
        "value": ms_b, "unit": "ms/batch", "higher_is_better": False, "steps": steps, "warmup": warmup,
        "dtype": "f64" if a.precision == "fp64" else "f32+f64", "data": "synthetic (seeded generator)",
        "config": {"workload": f"batched-{len(scs)}", "n_problems": len(scs),
                   "cams": [sc.n_cams for sc in scs], "n_cams": n_cams, "n_obs": n_obs, "nnzb": nnzb,
                   "mcg": {"n_dirs": a.n_dirs, "tau": a.tau}, "precision": a.precision, "tol": TOL,
                   "l2": "256 MiB buffer written before every timed step"},
        "looped_single_ms": ms_l, "speedup_vs_loop": ms_l / ms_b if ms_l else None,
        "per_problem_iters": [s["iters"] for s in per],
        "autotune": {"item_blocks": cb, "spmv_config": cfg, "spmv_ms_tuned": t_tuned, "spmv_ms_heuristic": t_heur},
        "roofline": {"kernel": "q = S p over all problems (float32: the symmetric product over the upper triangle)",
                     "bound": "hbm" if elt == 4 else "alu", "bytes_per_launch": sbytes,
                     "achieved_gbs": sbytes / t_tuned / 1e6, "peak_gbs": peaks["hbm_gbs"],
                     "frac": sbytes / t_tuned / 1e6 / peaks["hbm_gbs"]},
        "gpu_launches_per_step": int(launches), "clocks": clk,
        "step_ms": [round(x, 3) for x in tb], "loop_ms": [round(x, 3) for x in tl],
    }
    return line


def run_learned(a):
    """Learned pose grouping: training cost, then MCG iterations and time with and without it.

    Training: one Adam step per normal equation of 10 LM iterations of each of ``--learn-problems``
    shuffled problems per family (sequential and clustered dense, 80-240 cameras).  Evaluation on
    held-out seeds (1000+): MCG (N = 16, tau = 10) on the problem in its given random camera order,
    against MCG on the problem renumbered in the network's order (float32 and bfloat16 inference);
    the time with the network includes its inference on the built system.
    """
    import torch

    from paper_2110_04015_gb300 import binding, learn, problem

    g = binding.GNN(learn.init_params(0))

    def held_out_loss():
        out = {}
        for kind in ("sequential", "dense"):
            ls = []
            for seed in (5000, 5001, 5002):
                q = problem.from_scene(learn.training_scene(kind, seed), precision=a.precision)
                q.ba_build_normal(LAMBDA)
                ls.append(g.ba_gnn_loss(q)[0])
                q.close()
            out[kind] = float(np.mean(ls))
        return out

    loss_before = held_out_loss()
    t0 = time.perf_counter()
    l0 = g.ba_gnn_launch_count()
    losses = learn.harvest_train(g, seeds=range(a.learn_problems), kinds=("sequential", "dense"), lm_steps=10,
                                 lr=3e-3, precision=a.precision)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    train_launches = g.ba_gnn_launch_count() - l0
    loss_after = held_out_loss()
    evals = []
    for kind, seed, n in [("sequential", 1000, 1000), ("sequential", 1001, 400), ("dense", 1002, 600)]:
        if kind == "sequential":
            sc = synthetic.sequential(seed, n_cams=n, n_pts=100 * n)
        else:
            sc = synthetic.dense(seed, n_cams=n, n_pts=300 * n, n_clusters=n // 30)
        sc = synthetic.shuffled(sc, seed)
        p = problem.from_scene(sc, precision=a.precision)
        p.ba_build_normal(LAMBDA)
        base = min((p.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau) for _ in range(2)), key=lambda s: s["ms"])
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        row = {"workload": f"{kind}-{n} shuffled", "seed": seed, "n_cams": n,
               "without": {k: base[k] for k in ("iters", "local_steps", "ms", "true_rel_residual")}}
        for bf16 in (False, True):
            e0.record()
            order, L = g.ba_gnn_order(p, bf16=bf16)
            e1.record()
            e1.synchronize()
            t_inf = e0.elapsed_time(e1)
            q = problem.from_scene(synthetic.permute_cameras(sc, order), precision=a.precision)
            q.ba_build_normal(LAMBDA)
            st = min((q.ba_solve_mcg(TOL, MAX_ITERS, a.n_dirs, a.tau) for _ in range(2)), key=lambda s: s["ms"])
            q.close()
            row["bf16" if bf16 else "fp32"] = {"iters": st["iters"], "local_steps": st["local_steps"], "ms": st["ms"],
                                               "inference_ms": t_inf, "loss": L,
                                               "true_rel_residual": st["true_rel_residual"],
                                               "iters_ratio": st["iters"] / base["iters"],
                                               "time_ratio": (st["ms"] + t_inf) / base["ms"]}
        p.close()
        evals.append(row)
        print(json.dumps(row), file=sys.stderr, flush=True)
    line = {"mode": "learned", "metric": "MCG time to rel. residual 1e-6 with the learned grouping / without",
            "value": float(np.mean([r["fp32"]["time_ratio"] for r in evals])), "unit": "ratio",
            "higher_is_better": False, "precision": a.precision, "mcg": {"n_dirs": a.n_dirs, "tau": a.tau},
            "training": {"normal_equations": len(losses), "seconds": t_train, "gpu_launches": int(train_launches),
                         "held_out_loss_before": loss_before, "held_out_loss_after": loss_after},
            "eval": evals}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    if a.oracle_sample:
        run_oracle_sample(a)
        return
    if a.learned:
        run_learned(a)
        return
    if a.batched:
        run_batched(a)
        return
    if a.sweep:
        run_sweep(a)
        return
    if a.kernel_case:
        run_kernel_case(a)
        return
    if a.lm_run:
        run_lm(a)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if a.impl == "reference":
        run_reference(a, rank, world)
        return
    if world > 1:
        import torch.distributed as dist

        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl")
    try:
        run_ours(a, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist

            dist.destroy_process_group()


if __name__ == "__main__":
    main()
