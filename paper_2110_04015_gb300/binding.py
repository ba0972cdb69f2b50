"""Thin ctypes binding of libba (include/ba.h): same names, argument marshalling only.

Every computation happens in the CUDA library.  Arrays may be numpy arrays
(host memory) or torch tensors (host or CUDA); they are passed by pointer.
When the library is missing this module raises instead of falling back to
anything else.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

from .build import LIB, ROOT

BA_OK = 0
BA_ERR_INVALID_ARG = -1
BA_ERR_OOM = -2
BA_ERR_CUDA = -3
BA_ERR_SINGULAR = -4
BA_ERR_BREAKDOWN = -5
BA_ERR_NOT_CONVERGED = -6
BA_ERR_TIMEOUT = -7
BA_ERR_STATE = -8
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA", -4: "SINGULAR", -5: "BREAKDOWN",
                -6: "NOT_CONVERGED", -7: "TIMEOUT", -8: "STATE"}

DAMPING = {"marquardt": 0, "identity": 1}
PRECISION = {"fp64": 0, "mixed": 1}
SOLVER = {"pcg": 0, "mcg": 1}


class ba_options(ctypes.Structure):
    _fields_ = [("damping", ctypes.c_int32), ("precision", ctypes.c_int32), ("chunk_iters", ctypes.c_int32),
                ("max_history", ctypes.c_int32), ("inner_tol", ctypes.c_double), ("max_refine", ctypes.c_int32),
                ("item_blocks", ctypes.c_int32), ("wait_polls", ctypes.c_int32), ("spmv_config", ctypes.c_int32),
                ("host_loop", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class ba_solve_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("iters", ctypes.c_int32), ("local_steps", ctypes.c_int32),
                ("n_dirs_eff", ctypes.c_int32), ("refinements", ctypes.c_int32), ("history_cols", ctypes.c_int32),
                ("pinv_steps", ctypes.c_int32), ("host_waits", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("true_rel_residual", ctypes.c_double), ("ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class ba_lm_stats(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("accepted", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("solver_iters", ctypes.c_int32), ("cost_before", ctypes.c_double), ("cost_after", ctypes.c_double),
                ("lambda_used", ctypes.c_double), ("lambda_next", ctypes.c_double), ("ms", ctypes.c_double),
                ("solve_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class BAError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


_P = ctypes.c_void_p
_I32, _I64, _D = ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_SIGNATURES = {
    "ba_default_options": (None, [_P]),
    "ba_problem_create": (_I32, [_P, _I32, _I32, _I64, _P, _P, _P, _P, _P, _P]),
    "ba_batch_create": (_I32, [_P, _I32, _P, _I32, _I32, _I64, _P, _P, _P, _P, _P, _P]),
    "ba_problem_destroy": (None, [_P]),
    "ba_last_error": (ctypes.c_char_p, [_P]),
    "ba_set_stream": (_I32, [_P, _P]),
    "ba_set_params": (_I32, [_P, _P, _P]),
    "ba_get_params": (_I32, [_P, _P, _P]),
    "ba_build_normal": (_I32, [_P, _D]),
    "ba_solve_pcg": (_I32, [_P, _D, _I32, _P]),
    "ba_solve_mcg": (_I32, [_P, _D, _I32, _I32, _D, _P]),
    "ba_get_delta": (_I32, [_P, _P, _P]),
    "ba_lm_step": (_I32, [_P, _I32, _D, _D, _I32, _I32, _D, _D, _P]),
    "ba_cost": (_I32, [_P, _P]),
    "ba_project": (_I32, [_I32, _I32, _I64, _P, _P, _P, _P, _P, _P]),
    "ba_get_linearization": (_I32, [_P, _P, _P, _P]),
    "ba_get_normal": (_I32, [_P, _P, _P, _P, _P]),
    "ba_get_schur_nnzb": (_I32, [_P, _P]),
    "ba_get_schur": (_I32, [_P, _P, _P, _P, _P]),
    "ba_get_preconditioner": (_I32, [_P, _P]),
    "ba_get_residual_history": (_I32, [_P, _P, _I32, _P]),
    "ba_get_batch_size": (_I32, [_P, _P]),
    "ba_get_batch_stats": (_I32, [_P, _P, _I32]),
    "ba_get_batch_history": (_I32, [_P, _I32, _P, _I32, _P]),
    "ba_autotune": (_I32, [_P, _I32, _P, _P, _P]),
    "ba_get_launch_count": (_I32, [_P, _P]),
    "ba_time_kernel": (_I32, [_P, _I32, _I32, _P]),
    "ba_schur_residual_static": (_I32, [_I32, _P, _P, _P, _P, _P, _P, _P]),
    "ba_gnn_create": (_I32, [_P]),
    "ba_gnn_destroy": (None, [_P]),
    "ba_gnn_last_error": (ctypes.c_char_p, [_P]),
    "ba_gnn_param_count": (_I32, [_P]),
    "ba_gnn_set_params": (_I32, [_P, _P]),
    "ba_gnn_get_params": (_I32, [_P, _P]),
    "ba_gnn_graph": (_I32, [_P, _P, _P, _P]),
    "ba_gnn_loss": (_I32, [_P, _P, _P, _P, _P]),
    "ba_gnn_train_step": (_I32, [_P, _P, _D, _P]),
    "ba_gnn_order": (_I32, [_P, _P, _I32, _P, _P]),
    "ba_gnn_launch_count": (_I32, [_P, _P]),
}
BA_STATIC_MAX_CAMS = 65536
KERNEL = {"spmv": 0, "schur": 1, "linearize": 2, "landmarks": 3, "cam_rhs": 4, "schur_diag": 5, "schur_off": 6,
          "block_jacobi": 7}

_lib = None


def header_functions() -> list[str]:
    """Names of the functions declared in include/ba.h."""
    with open(os.path.join(ROOT, "include", "ba.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(ba_[a-z0-9_]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    """Load libba; raise if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise RuntimeError(f"{LIB} is missing: build it with paper_2110_04015_gb300.build.build()")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)}")


def _check(code: int, handle=None, allow=(BA_OK,)) -> int:
    if code in allow:
        return code
    msg = lib().ba_last_error(handle).decode() if handle is not None or code != BA_OK else ""
    raise BAError(code, msg)


def _f64(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.float64)
    return a


def _i32(a):
    if isinstance(a, np.ndarray):
        return np.ascontiguousarray(a, dtype=np.int32)
    return a


def ba_project(cams, pts, obs_cam, obs_pt, out, stream=None) -> None:
    """pi(c_j, X_l) per observation on the device (all arguments CUDA tensors)."""
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    code = lib().ba_project(int(cams.shape[0]), int(pts.shape[0]), int(obs_cam.shape[0]), _ptr(cams), _ptr(pts),
                            _ptr(obs_cam), _ptr(obs_pt), _ptr(out), st)
    _check(code)


def _static_args_check(n_cams, row_ptr, col, blocks, btilde, x, out) -> None:
    """Reject what the library cannot check itself: it receives raw device pointers and no lengths,
    so a wrong dtype, a short array or a host array would be read out of bounds on the device."""
    import torch

    named = {"row_ptr": row_ptr, "col": col, "blocks": blocks, "btilde": btilde, "x": x, "out": out}
    for name, t in named.items():
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor on the current CUDA device, got {type(t).__name__}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
    want = {"row_ptr": torch.int64, "col": torch.int32, "blocks": torch.float64, "btilde": torch.float64,
            "x": torch.float64, "out": torch.float64}
    for name, dt in want.items():
        if named[name].dtype != dt:
            raise TypeError(f"{name} must be {dt}, got {named[name].dtype}")
    n = int(n_cams)
    if 1 <= n <= BA_STATIC_MAX_CAMS:
        if row_ptr.numel() != n + 1:
            raise ValueError(f"row_ptr must hold n_cams + 1 = {n + 1} offsets, got {row_ptr.numel()}")
        if btilde.numel() != 9 * n or x.numel() != 9 * n:
            raise ValueError(f"btilde and x must hold 9 n_cams = {9 * n} values")
        if out.numel() < 2:
            raise ValueError("out must hold 2 values")
    for name, t in named.items():
        if not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor")
    dev = torch.cuda.current_device()
    for name, t in named.items():
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
    if 1 <= n <= BA_STATIC_MAX_CAMS and (blocks.numel() % 81 != 0 or blocks.numel() // 81 != col.numel()):
        raise ValueError(f"blocks must hold 81 values per entry of col ({col.numel()}), got {blocks.numel()}")


def ba_schur_residual_static(n_cams, row_ptr, col, blocks, btilde, x, out, stream=None) -> None:
    """|-b~ - S x| and |b~| into out[0:2] without any device allocation.

    Every array is a contiguous torch tensor on the current CUDA device: row_ptr int64 (n_cams + 1),
    col int32, blocks float64 (81 per entry of col), btilde and x float64 (9 n_cams), out float64
    (>= 2).  Anything else is rejected here from the tensors' metadata alone, before the library is
    called; the contents of row_ptr and col (offsets within col, columns within [0, n_cams)) are the
    caller's to keep valid, since checking them would mean reading device memory back.
    """
    _static_args_check(n_cams, row_ptr, col, blocks, btilde, x, out)
    st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
    code = lib().ba_schur_residual_static(int(n_cams), _ptr(row_ptr), _ptr(col), _ptr(blocks), _ptr(btilde),
                                          _ptr(x), _ptr(out), st)
    _check(code)


class Problem:
    """One bundle-adjustment problem held by the library (a ``ba_problem`` handle).

    With ``cam_off`` (n_problems + 1 camera offsets) the handle holds a batch of independent
    problems over the concatenated arrays (``ba_batch_create``).
    """

    def __init__(self, cams, pts, obs_cam, obs_pt, obs_xy, damping="marquardt", precision="fp64",
                 chunk_iters=8, max_history=0, inner_tol=1e-6, max_refine=64, item_blocks=0, wait_polls=0,
                 host_loop=0, spmv_config=0, cam_off=None):
        L = lib()
        opt = ba_options()
        L.ba_default_options(ctypes.byref(opt))
        opt.damping = DAMPING[damping]
        opt.precision = PRECISION[precision]
        opt.chunk_iters = chunk_iters
        opt.max_history = max_history
        opt.inner_tol = inner_tol
        opt.max_refine = max_refine
        opt.item_blocks = item_blocks
        opt.wait_polls = wait_polls
        opt.host_loop = host_loop
        opt.spmv_config = spmv_config
        self._keep = [_f64(cams), _f64(pts), _i32(obs_cam), _i32(obs_pt), _f64(obs_xy)]
        cams, pts, obs_cam, obs_pt, obs_xy = self._keep
        self.n_cams = int(cams.shape[0])
        self.n_pts = int(pts.shape[0])
        self.n_obs = int(obs_cam.shape[0])
        h = ctypes.c_void_p()
        if cam_off is None:
            self.n_problems = 1
            code = L.ba_problem_create(ctypes.byref(opt), self.n_cams, self.n_pts, self.n_obs, _ptr(cams),
                                       _ptr(pts), _ptr(obs_cam), _ptr(obs_pt), _ptr(obs_xy), ctypes.byref(h))
        else:
            off = _i32(np.asarray(cam_off))
            self.n_problems = int(off.shape[0]) - 1
            code = L.ba_batch_create(ctypes.byref(opt), self.n_problems, _ptr(off), self.n_cams, self.n_pts,
                                     self.n_obs, _ptr(cams), _ptr(pts), _ptr(obs_cam), _ptr(obs_pt), _ptr(obs_xy),
                                     ctypes.byref(h))
        self._keep = None
        if code != BA_OK:
            raise BAError(code, L.ba_last_error(None).decode())
        self.h = h
        self.precision = precision

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            lib().ba_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # -- the calls of include/ba.h
    def ba_set_stream(self, stream):
        st = stream.cuda_stream if hasattr(stream, "cuda_stream") else stream
        _check(lib().ba_set_stream(self.h, st), self.h)

    def ba_set_params(self, cams=None, pts=None):
        cams, pts = _f64(cams), _f64(pts)
        _check(lib().ba_set_params(self.h, _ptr(cams), _ptr(pts)), self.h)

    def ba_get_params(self, cams=None, pts=None):
        if cams is None and pts is None:
            cams = np.empty((self.n_cams, 9))
            pts = np.empty((self.n_pts, 3))
        _check(lib().ba_get_params(self.h, _ptr(cams), _ptr(pts)), self.h)
        return cams, pts

    def ba_build_normal(self, lam: float):
        _check(lib().ba_build_normal(self.h, float(lam)), self.h)

    def ba_solve_pcg(self, tol=1e-6, max_iters=1000) -> dict:
        st = ba_solve_stats()
        code = lib().ba_solve_pcg(self.h, float(tol), int(max_iters), ctypes.byref(st))
        _check(code, self.h, allow=(BA_OK, BA_ERR_NOT_CONVERGED))
        return st.as_dict()

    def ba_solve_mcg(self, tol=1e-6, max_iters=1000, n_dirs=8, tau=3.0) -> dict:
        st = ba_solve_stats()
        code = lib().ba_solve_mcg(self.h, float(tol), int(max_iters), int(n_dirs), float(tau), ctypes.byref(st))
        _check(code, self.h, allow=(BA_OK, BA_ERR_NOT_CONVERGED))
        return st.as_dict()

    def ba_get_delta(self, dxp=None, dxl=None, landmarks=False):
        if dxp is None:
            dxp = np.empty((self.n_cams, 9))
        if dxl is None and landmarks:
            dxl = np.empty((self.n_pts, 3))
        _check(lib().ba_get_delta(self.h, _ptr(dxp), _ptr(dxl)), self.h)
        return (dxp, dxl) if landmarks else dxp

    def ba_lm_step(self, solver="pcg", lambda0=1e-4, tol=1e-6, max_iters=1000, n_dirs=8, tau=3.0,
                   ftol=1e-6) -> dict:
        st = ba_lm_stats()
        code = lib().ba_lm_step(self.h, SOLVER[solver], float(lambda0), float(tol), int(max_iters), int(n_dirs),
                                float(tau), float(ftol), ctypes.byref(st))
        _check(code, self.h)
        return st.as_dict()

    def ba_cost(self) -> float:
        c = ctypes.c_double()
        _check(lib().ba_cost(self.h, ctypes.byref(c)), self.h)
        return c.value

    def ba_get_linearization(self):
        r = np.empty((self.n_obs, 2))
        Jp = np.empty((self.n_obs, 2, 9))
        Jl = np.empty((self.n_obs, 2, 3))
        _check(lib().ba_get_linearization(self.h, _ptr(r), _ptr(Jp), _ptr(Jl)), self.h)
        return r, Jp, Jl

    def ba_get_normal(self):
        U = np.empty((self.n_cams, 9, 9))
        V = np.empty((self.n_pts, 3, 3))
        bp = np.empty((self.n_cams, 9))
        bl = np.empty((self.n_pts, 3))
        _check(lib().ba_get_normal(self.h, _ptr(U), _ptr(V), _ptr(bp), _ptr(bl)), self.h)
        return U, V, bp, bl

    def ba_get_schur_nnzb(self) -> int:
        n = ctypes.c_int64()
        _check(lib().ba_get_schur_nnzb(self.h, ctypes.byref(n)), self.h)
        return n.value

    def ba_get_schur(self, blocks=True):
        nnzb = self.ba_get_schur_nnzb()
        row_ptr = np.empty(self.n_cams + 1, np.int64)
        col = np.empty(nnzb, np.int32)
        B = np.empty((nnzb, 9, 9)) if blocks else None
        bt = np.empty((self.n_cams, 9))
        _check(lib().ba_get_schur(self.h, _ptr(row_ptr), _ptr(col), _ptr(B), _ptr(bt)), self.h)
        return row_ptr, col, B, bt

    def ba_get_preconditioner(self):
        D = np.empty((self.n_cams, 9, 9))
        _check(lib().ba_get_preconditioner(self.h, _ptr(D)), self.h)
        return D

    def ba_get_residual_history(self, cap=100000):
        h = np.empty(cap)
        n = ctypes.c_int32()
        _check(lib().ba_get_residual_history(self.h, _ptr(h), int(cap), ctypes.byref(n)), self.h)
        return h[:min(n.value, cap)].copy()

    def ba_get_batch_size(self) -> int:
        n = ctypes.c_int32()
        _check(lib().ba_get_batch_size(self.h, ctypes.byref(n)), self.h)
        return n.value

    def ba_get_batch_stats(self) -> list[dict]:
        nb = self.ba_get_batch_size()
        arr = (ba_solve_stats * nb)()
        _check(lib().ba_get_batch_stats(self.h, arr, nb), self.h)
        return [arr[b].as_dict() for b in range(nb)]

    def ba_get_batch_history(self, problem: int, cap=100000):
        h = np.empty(cap)
        n = ctypes.c_int32()
        _check(lib().ba_get_batch_history(self.h, int(problem), _ptr(h), int(cap), ctypes.byref(n)), self.h)
        return h[:min(n.value, cap)].copy()

    def ba_autotune(self, reps=5) -> tuple[int, float, int]:
        """(blocks per work item, mean ms of the tuned product, warps x stages shape)."""
        cb = ctypes.c_int32()
        cfg = ctypes.c_int32()
        ms = ctypes.c_double()
        _check(lib().ba_autotune(self.h, int(reps), ctypes.byref(cb), ctypes.byref(cfg), ctypes.byref(ms)), self.h)
        return cb.value, ms.value, cfg.value

    def ba_get_launch_count(self) -> int:
        n = ctypes.c_int64()
        _check(lib().ba_get_launch_count(self.h, ctypes.byref(n)), self.h)
        return n.value

    def ba_time_kernel(self, kernel="spmv", reps=10) -> float:
        ms = ctypes.c_double()
        _check(lib().ba_time_kernel(self.h, KERNEL[kernel], int(reps), ctypes.byref(ms)), self.h)
        return ms.value

    # short aliases
    build_normal = ba_build_normal
    solve_pcg = ba_solve_pcg
    solve_mcg = ba_solve_mcg
    get_delta = ba_get_delta
    lm_step = ba_lm_step
    cost = ba_cost


def _gcheck(code: int, g) -> None:
    if code != BA_OK:
        raise BAError(code, lib().ba_gnn_last_error(g).decode())


class GNN:
    """The pose-grouping network held by the library (a ``ba_gnn`` handle)."""

    def __init__(self, params=None):
        L = lib()
        h = ctypes.c_void_p()
        code = L.ba_gnn_create(ctypes.byref(h))
        if code != BA_OK:
            raise BAError(code, L.ba_last_error(None).decode())
        self.h = h
        n = ctypes.c_int64()
        _check(L.ba_gnn_param_count(ctypes.byref(n)))
        self.n_params = n.value
        if params is not None:
            self.ba_gnn_set_params(params)

    def close(self):
        if getattr(self, "h", None):
            lib().ba_gnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def ba_gnn_set_params(self, params):
        params = np.ascontiguousarray(params, dtype=np.float32) if isinstance(params, np.ndarray) else params
        _gcheck(lib().ba_gnn_set_params(self.h, _ptr(params)), self.h)

    def ba_gnn_get_params(self):
        out = np.empty(self.n_params, np.float32)
        _gcheck(lib().ba_gnn_get_params(self.h, _ptr(out)), self.h)
        return out

    def ba_gnn_graph(self, p: "Problem"):
        X = np.empty((p.n_cams, 8), np.float32)
        c = np.empty(p.ba_get_schur_nnzb(), np.float32)
        _gcheck(lib().ba_gnn_graph(self.h, p.h, _ptr(X), _ptr(c)), self.h)
        return X, c

    def ba_gnn_loss(self, p: "Problem", grad=False):
        loss = ctypes.c_double()
        s = np.empty(p.n_cams, np.float32)
        g = np.empty(self.n_params, np.float32) if grad else None
        _gcheck(lib().ba_gnn_loss(self.h, p.h, ctypes.byref(loss), _ptr(s), _ptr(g)), self.h)
        return (loss.value, s, g) if grad else (loss.value, s)

    def ba_gnn_train_step(self, p: "Problem", lr=1e-3) -> float:
        loss = ctypes.c_double()
        _gcheck(lib().ba_gnn_train_step(self.h, p.h, float(lr), ctypes.byref(loss)), self.h)
        return loss.value

    def ba_gnn_order(self, p: "Problem", bf16=False):
        order = np.empty(p.n_cams, np.int32)
        loss = ctypes.c_double()
        _gcheck(lib().ba_gnn_order(self.h, p.h, int(bool(bf16)), _ptr(order), ctypes.byref(loss)), self.h)
        return order, loss.value

    def ba_gnn_launch_count(self) -> int:
        n = ctypes.c_int64()
        _gcheck(lib().ba_gnn_launch_count(self.h, ctypes.byref(n)), self.h)
        return n.value
