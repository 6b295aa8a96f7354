"""Thin Python binding of the C ABI in include/segsalsa_str.h (ctypes; argument marshalling only).

Every compute step runs in libsegsalsa_str.so. Arrays may be numpy arrays (host memory) or
torch tensors (device tensors are passed by data_ptr() with on_device=1). There is no CPU
fallback: if the shared library is missing this module raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

SEGSALSA_OK = 0
SEGSALSA_ERR_ARG = -1
SEGSALSA_ERR_OOM = -2
SEGSALSA_ERR_CUDA = -3
SEGSALSA_ERR_NUMERIC = -4
SEGSALSA_ERR_TIMEOUT = -5
SEGSALSA_ERR_STATE = -6
SEGSALSA_FP32 = 0
SEGSALSA_FP64 = 1
SEGSALSA_LAYOUT_KHW = 0
SEGSALSA_LAYOUT_HWK = 1
SEGSALSA_SCHATTEN_INF = 0
SEGSALSA_G4_AFFINE = 0
SEGSALSA_G4_SIMPLEX = 1

KERNEL_KINDS = ("sweep", "row_fft_forward", "column_solve", "row_fft_inverse", "diagnostics",
                "other", "mlr", "adjoint", "zupdate_fused")

SYMBOLS = (
    "segsalsa_str_workspace_bytes", "segsalsa_str_create", "segsalsa_str_set_probs",
    "segsalsa_str_solve", "segsalsa_str_get_labels", "segsalsa_str_get_z",
    "segsalsa_str_get_iteration", "segsalsa_str_get_state", "segsalsa_str_set_state",
    "segsalsa_str_linear_solve", "segsalsa_str_set_profiling", "segsalsa_str_kernel_stats",
    "segsalsa_str_reset_stats", "segsalsa_str_traffic_model", "segsalsa_str_destroy",
    "segsalsa_str_last_error", "segsalsa_str_linear_solve_static",
    "segsalsa_str_workspace_bytes_tiled", "segsalsa_str_create_tiled", "segsalsa_str_get_tiling",
    "segsalsa_str_batch_create", "segsalsa_str_batch_image", "segsalsa_str_batch_solve",
    "segsalsa_str_batch_autotune", "segsalsa_str_batch_set_lanes", "segsalsa_str_batch_get_lanes",
    "segsalsa_str_batch_destroy", "segsalsa_str_batch_last_error",
    "segsalsa_str_set_spectra", "segsalsa_str_get_probs", "segsalsa_str_solve_until",
    "segsalsa_str_set_g4", "segsalsa_str_set_log_probs", "segsalsa_str_set_lambda",
    "segsalsa_str_set_weights", "segsalsa_str_backward", "segsalsa_str_set_wait_budget",
)


class Params(C.Structure):
    _fields_ = [
        ("H", C.c_int32), ("W", C.c_int32), ("K", C.c_int32), ("M", C.c_int32),
        ("weights", C.POINTER(C.c_double)), ("sigma", C.c_double), ("lambda_", C.c_double),
        ("mu", C.c_double), ("schatten_p", C.c_int32), ("precision", C.c_int32),
        ("stream", C.c_void_p),
    ]


class Tiling(C.Structure):
    _fields_ = [("tile_rows", C.c_int32), ("row_pairs", C.c_int32), ("col_block", C.c_int32),
                ("row_threads", C.c_int32), ("col_rows", C.c_int32), ("zfuse", C.c_int32),
                ("row_pipe", C.c_int32)]

    def as_tuple(self):
        return (self.tile_rows, self.row_pairs, self.col_block, self.row_threads, self.col_rows,
                self.zfuse, self.row_pipe)


def make_tiling(tile_rows=0, row_pairs=0, col_block=0, row_threads=0, col_rows=0,
                zfuse=0, row_pipe=0) -> Tiling:
    t = Tiling()
    t.tile_rows, t.row_pairs, t.col_block = int(tile_rows), int(row_pairs), int(col_block)
    t.row_threads, t.col_rows, t.zfuse = int(row_threads), int(col_rows), int(zfuse)
    t.row_pipe = int(row_pipe)
    return t


class SegsalsaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"segsalsa_str error {code}: {msg}")
        self.code = code


_LIB = None


def library_path() -> str:
    return _build.LIB


def load(path: str | None = None):
    """Load libsegsalsa_str.so (built in-tree by paper_1504_07028_gb300.build)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: run paper_1504_07028_gb300.build.build() first")
    lib = C.CDLL(p)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    sig = {
        "segsalsa_str_workspace_bytes": (C.c_int, [C.POINTER(Params), C.POINTER(C.c_size_t)]),
        "segsalsa_str_create": (C.c_int, [C.POINTER(Params), vp, C.c_size_t, C.POINTER(vp)]),
        "segsalsa_str_set_probs": (C.c_int, [vp, vp, i32, i32]),
        "segsalsa_str_solve": (C.c_int, [vp, i32, C.POINTER(C.c_double), i32, C.POINTER(i32)]),
        "segsalsa_str_get_labels": (C.c_int, [vp, vp, i32]),
        "segsalsa_str_get_z": (C.c_int, [vp, vp, i32, i32]),
        "segsalsa_str_get_iteration": (C.c_int, [vp, C.POINTER(i32)]),
        "segsalsa_str_get_state": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, i32]),
        "segsalsa_str_set_state": (C.c_int, [vp, vp, vp, vp, vp, vp, vp, i32, i32]),
        "segsalsa_str_linear_solve": (C.c_int, [vp, vp, vp, i32]),
        "segsalsa_str_set_profiling": (C.c_int, [vp, i32]),
        "segsalsa_str_kernel_stats": (C.c_int, [vp, C.POINTER(i64), C.POINTER(C.c_double)]),
        "segsalsa_str_reset_stats": (C.c_int, [vp]),
        "segsalsa_str_traffic_model": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "segsalsa_str_destroy": (None, [vp]),
        "segsalsa_str_last_error": (C.c_char_p, [vp]),
        "segsalsa_str_linear_solve_static": (C.c_int, [vp, vp, i32, i32, i32, C.c_double, vp]),
        "segsalsa_str_workspace_bytes_tiled": (C.c_int, [C.POINTER(Params), C.POINTER(Tiling),
                                                         C.POINTER(C.c_size_t)]),
        "segsalsa_str_create_tiled": (C.c_int, [C.POINTER(Params), C.POINTER(Tiling), vp,
                                                C.c_size_t, C.POINTER(vp)]),
        "segsalsa_str_get_tiling": (C.c_int, [vp, C.POINTER(Tiling)]),
        "segsalsa_str_batch_create": (C.c_int, [i32, C.POINTER(Params), C.POINTER(Tiling), vp,
                                                C.POINTER(vp)]),
        "segsalsa_str_batch_image": (C.c_int, [vp, i32, C.POINTER(vp)]),
        "segsalsa_str_batch_solve": (C.c_int, [vp, i32]),
        "segsalsa_str_batch_autotune": (C.c_int, [vp, i32, C.POINTER(Tiling)]),
        "segsalsa_str_batch_set_lanes": (C.c_int, [vp, i32]),
        "segsalsa_str_batch_get_lanes": (C.c_int, [vp, C.POINTER(i32)]),
        "segsalsa_str_batch_destroy": (None, [vp]),
        "segsalsa_str_set_spectra": (C.c_int, [vp, vp, vp, vp, i32, i32]),
        "segsalsa_str_get_probs": (C.c_int, [vp, vp, i32, i32]),
        "segsalsa_str_set_g4": (C.c_int, [vp, i32]),
        "segsalsa_str_set_wait_budget": (C.c_int, [vp, C.c_int64, i32]),
        "segsalsa_str_set_log_probs": (C.c_int, [vp, vp, i32, i32]),
        "segsalsa_str_set_lambda": (C.c_int, [vp, C.c_double]),
        "segsalsa_str_set_weights": (C.c_int, [vp, C.POINTER(C.c_double)]),
        "segsalsa_str_backward": (C.c_int, [vp, i32, vp, i32, vp, C.POINTER(C.c_double),
                                            C.POINTER(C.c_double), i32, i32]),
        "segsalsa_str_solve_until": (C.c_int, [vp, i32, C.c_double, C.c_double, i32,
                                               C.POINTER(i32), C.POINTER(C.c_double)]),
        "segsalsa_str_batch_last_error": (C.c_char_p, [vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _LIB = lib
    return lib


def _ptr(a, dtype):
    """(pointer, on_device) of a contiguous numpy array or torch tensor of `dtype`."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if a.dtype != dtype:
            raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    # torch tensor
    import torch
    tmap = {np.float32: torch.float32, np.float64: torch.float64, np.int32: torch.int32}
    if a.dtype != tmap[np.dtype(dtype).type]:
        raise TypeError(f"expected {np.dtype(dtype)}, got {a.dtype}")
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), int(a.is_cuda)


def _ptr_bf16(a):
    """(pointer, on_device) of a contiguous BF16 array: a torch.bfloat16 tensor or a numpy
    uint16 array holding BF16 bit patterns."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.uint16:
            raise TypeError("numpy BF16 data must be uint16 bit patterns")
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return a.ctypes.data, 0
    import torch
    if a.dtype != torch.bfloat16:
        raise TypeError(f"expected torch.bfloat16, got {a.dtype}")
    if not a.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return a.data_ptr(), int(a.is_cuda)


def _check(lib, h, rc):
    if rc != SEGSALSA_OK:
        msg = lib.segsalsa_str_last_error(h).decode()
        raise SegsalsaError(rc, msg)


# ------------------------------------------------------------------ C-ABI-named functions

def segsalsa_str_workspace_bytes(params: Params) -> int:
    lib = load()
    n = C.c_size_t(0)
    _check(lib, None, lib.segsalsa_str_workspace_bytes(C.byref(params), C.byref(n)))
    return n.value


def segsalsa_str_create(params: Params, workspace_ptr: int | None = None, workspace_bytes: int = 0,
                        tiling: Tiling | None = None):
    lib = load()
    h = C.c_void_p()
    if tiling is None:
        rc = lib.segsalsa_str_create(C.byref(params), workspace_ptr, workspace_bytes, C.byref(h))
    else:
        rc = lib.segsalsa_str_create_tiled(C.byref(params), C.byref(tiling), workspace_ptr,
                                           workspace_bytes, C.byref(h))
    _check(lib, None, rc)
    return h


def segsalsa_str_workspace_bytes_tiled(params: Params, tiling: Tiling | None) -> int:
    lib = load()
    n = C.c_size_t(0)
    _check(lib, None, lib.segsalsa_str_workspace_bytes_tiled(
        C.byref(params), C.byref(tiling) if tiling is not None else None, C.byref(n)))
    return n.value


def segsalsa_str_destroy(h):
    load().segsalsa_str_destroy(h)


def segsalsa_str_last_error(h=None) -> str:
    return load().segsalsa_str_last_error(h).decode()


def segsalsa_str_linear_solve_static(rhs, z, c_omega: float = 1.0, stream=None) -> int:
    """Allocation-free z-update for callers that cannot allocate device memory: rhs and z are
    FP32 device tensors of shape (H, W, K); the scratch is the library's static device array.
    Returns the status code (0 on success) without raising."""
    H, W, K = (int(v) for v in rhs.shape)
    if tuple(z.shape) != (H, W, K):
        raise ValueError("rhs and z must have the same (H, W, K) shape")
    p1, d1 = _ptr(rhs, np.float32)
    p2, d2 = _ptr(z, np.float32)
    if not (d1 and d2):
        raise ValueError("rhs and z must be device tensors")
    return load().segsalsa_str_linear_solve_static(p1, p2, H, W, K, float(c_omega), stream)


def make_params(H, W, K, M=1, sigma=0.5, lam=1.5, mu=1.0, schatten_p=1, precision="fp32",
                weights=None, stream=None) -> Params:
    pr = Params()
    pr.H, pr.W, pr.K, pr.M = int(H), int(W), int(K), int(M)
    if weights is not None:
        w = np.ascontiguousarray(weights, dtype=np.float64)
        pr._weights_keep = w
        pr.weights = w.ctypes.data_as(C.POINTER(C.c_double))
    else:
        pr.weights = None
    pr.sigma = float(sigma)
    pr.lambda_ = float(lam)
    pr.mu = float(mu)
    sp = schatten_p
    pr.schatten_p = SEGSALSA_SCHATTEN_INF if sp in (np.inf, float("inf"), "inf", 0) else int(sp)
    pr.precision = SEGSALSA_FP64 if precision in ("fp64", np.float64, SEGSALSA_FP64) else SEGSALSA_FP32
    pr.stream = stream
    return pr


class Solver:
    """One solver handle (wraps segsalsa_str_*). Arrays: numpy (host) or torch (device)."""

    def __init__(self, params: Params, workspace=None, tiling: Tiling | None = None,
                 _borrowed=None):
        self.lib = load()
        self.params = params
        self.dtype = np.float64 if params.precision == SEGSALSA_FP64 else np.float32
        self.H, self.W, self.K, self.M = params.H, params.W, params.K, params.M
        self.L = (2 * self.M + 1) ** 2
        self._ws = workspace  # keep the caller's memory alive
        self._owned = _borrowed is None
        if _borrowed is not None:
            self.h = _borrowed
            return
        ptr, nbytes = (None, 0)
        if workspace is not None:
            ptr, nbytes = workspace.data_ptr(), workspace.numel() * workspace.element_size()
        self.h = segsalsa_str_create(params, ptr, nbytes, tiling)

    def close(self):
        if getattr(self, "h", None):
            if self._owned:
                self.lib.segsalsa_str_destroy(self.h)
            self.h = None

    # segsalsa_str_get_tiling
    def tiling(self) -> tuple:
        t = Tiling()
        self._c(self.lib.segsalsa_str_get_tiling(self.h, C.byref(t)))
        return t.as_tuple()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, rc):
        _check(self.lib, self.h, rc)

    # segsalsa_str_set_probs
    def set_probs(self, p, layout=SEGSALSA_LAYOUT_KHW):
        ptr, dev = _ptr(p, self.dtype)
        self._c(self.lib.segsalsa_str_set_probs(self.h, ptr, layout, dev))

    # segsalsa_str_solve
    def solve(self, iters, trace_every=0):
        if trace_every:
            cap = iters // trace_every + 2
            tr = np.zeros((cap, 6), dtype=np.float64)
            n = C.c_int32(0)
            self._c(self.lib.segsalsa_str_solve(
                self.h, int(iters), tr.ctypes.data_as(C.POINTER(C.c_double)), int(trace_every),
                C.byref(n)))
            return tr[: n.value]
        self._c(self.lib.segsalsa_str_solve(self.h, int(iters), None, 0, None))
        return None

    # segsalsa_str_set_spectra
    def set_spectra(self, x, w, bias=None):
        """x: (H, W, d) BF16, w: (K, d) BF16 (torch.bfloat16 or numpy uint16 bit patterns),
        bias: (K,) float32 or None; x, w and bias on the same side (host or device)."""
        d = int(x.shape[-1])
        if tuple(x.shape) != (self.H, self.W, d) or tuple(w.shape) != (self.K, d):
            raise ValueError("x must be (H, W, d) and w (K, d)")
        px_, dx = _ptr_bf16(x)
        pw, dw = _ptr_bf16(w)
        pb, db = (None, dx)
        if bias is not None:
            pb, db = _ptr(bias, np.float32)
        if not (dx == dw == db):
            raise ValueError("x, w and bias must all be host or all device arrays")
        self._c(self.lib.segsalsa_str_set_spectra(self.h, px_, pw, pb, d, dx))

    # segsalsa_str_get_probs
    def get_probs(self, out=None, layout=SEGSALSA_LAYOUT_KHW):
        if out is None:
            shape = (self.K, self.H, self.W) if layout == SEGSALSA_LAYOUT_KHW else (self.H, self.W, self.K)
            out = np.empty(shape, dtype=self.dtype)
        ptr, dev = _ptr(out, self.dtype)
        self._c(self.lib.segsalsa_str_get_probs(self.h, ptr, layout, dev))
        return out

    # segsalsa_str_set_log_probs
    def set_log_probs(self, log_p, layout=SEGSALSA_LAYOUT_KHW):
        ptr, dev = _ptr(log_p, self.dtype)
        self._c(self.lib.segsalsa_str_set_log_probs(self.h, ptr, layout, dev))

    # segsalsa_str_set_lambda
    def set_lambda(self, lam):
        self._c(self.lib.segsalsa_str_set_lambda(self.h, float(lam)))

    # segsalsa_str_set_weights
    def set_weights(self, weights):
        w = np.ascontiguousarray(weights, dtype=np.float64)
        if w.shape != (self.L,):
            raise ValueError(f"weights must have {self.L} entries")
        self._c(self.lib.segsalsa_str_set_weights(self.h, w.ctypes.data_as(C.POINTER(C.c_double))))

    # segsalsa_str_backward
    def backward(self, iters, zbar, checkpoint_every=10, out=None, layout=SEGSALSA_LAYOUT_KHW):
        """Returns (dLoss/dlog p, dLoss/dlambda, dLoss/domega) for zbar = dLoss/dz^T."""
        if out is None:
            out = np.empty_like(zbar) if isinstance(zbar, np.ndarray) else zbar.new_empty(zbar.shape)
        p1, d1 = _ptr(zbar, self.dtype)
        p2, d2 = _ptr(out, self.dtype)
        if d1 != d2:
            raise ValueError("zbar and the output must both be host or both device arrays")
        glam = C.c_double(0)
        gom = (C.c_double * self.L)()
        self._c(self.lib.segsalsa_str_backward(self.h, int(iters), p1, layout, p2, C.byref(glam),
                                               gom, int(checkpoint_every), d1))
        return out, glam.value, np.array(gom[:], dtype=np.float64)

    # segsalsa_str_set_g4
    def set_wait_budget(self, cycles: int, probe: bool = False):
        """Clock-cycle limit of the bounded device-side waits; probe=True makes the next
        bulk-copy waits run out (a test of the timeout path)."""
        self._c(self.lib.segsalsa_str_set_wait_budget(self.h, int(cycles), int(probe)))

    def set_g4(self, mode):
        m = {"affine": SEGSALSA_G4_AFFINE, "simplex": SEGSALSA_G4_SIMPLEX}.get(mode, mode)
        self._c(self.lib.segsalsa_str_set_g4(self.h, int(m)))

    # segsalsa_str_solve_until
    def solve_until(self, max_iters, tol_primal, tol_dual, check_every=10):
        """Returns (iterations run, last trace record as a 6-vector)."""
        n = C.c_int32(0)
        rec = (C.c_double * 6)()
        self._c(self.lib.segsalsa_str_solve_until(self.h, int(max_iters), float(tol_primal),
                                                  float(tol_dual), int(check_every),
                                                  C.byref(n), rec))
        return n.value, np.array(rec[:], dtype=np.float64)

    # segsalsa_str_get_labels
    def get_labels(self, out=None):
        if out is None:
            out = np.empty((self.H, self.W), dtype=np.int32)
        ptr, dev = _ptr(out, np.int32)
        self._c(self.lib.segsalsa_str_get_labels(self.h, ptr, dev))
        return out

    # segsalsa_str_get_z
    def get_z(self, out=None, layout=SEGSALSA_LAYOUT_KHW):
        if out is None:
            shape = (self.K, self.H, self.W) if layout == SEGSALSA_LAYOUT_KHW else (self.H, self.W, self.K)
            out = np.empty(shape, dtype=self.dtype)
        ptr, dev = _ptr(out, self.dtype)
        self._c(self.lib.segsalsa_str_get_z(self.h, ptr, layout, dev))
        return out

    def get_iteration(self) -> int:
        k = C.c_int32(0)
        self._c(self.lib.segsalsa_str_get_iteration(self.h, C.byref(k)))
        return k.value

    def state_shapes(self):
        H, W, K, L = self.H, self.W, self.K, self.L
        return {"z": (H, W, K), "d1": (H, W, K), "d2": (H, W, L, K, 2), "d3": (H, W, K),
                "d4": (H, W, K), "rhs": (H, W, K)}

    # segsalsa_str_get_state
    def get_state(self):
        sh = self.state_shapes()
        out = {k: np.empty(v, dtype=self.dtype) for k, v in sh.items()}
        ptrs = [_ptr(out[k], self.dtype)[0] for k in ("z", "d1", "d2", "d3", "d4", "rhs")]
        self._c(self.lib.segsalsa_str_get_state(self.h, *ptrs, 0))
        return out

    # segsalsa_str_set_state
    def set_state(self, st: dict, k: int):
        arrs = [np.ascontiguousarray(st[n], dtype=self.dtype) if st.get(n) is not None else None
                for n in ("z", "d1", "d2", "d3", "d4", "rhs")]
        ptrs = [_ptr(a, self.dtype)[0] for a in arrs]
        self._c(self.lib.segsalsa_str_set_state(self.h, *ptrs, int(k), 0))

    # segsalsa_str_linear_solve
    def linear_solve(self, rhs, out=None):
        if out is None:
            out = np.empty_like(rhs) if isinstance(rhs, np.ndarray) else rhs.new_empty(rhs.shape)
        p1, d1 = _ptr(rhs, self.dtype)
        p2, d2 = _ptr(out, self.dtype)
        if d1 != d2:
            raise ValueError("rhs and z must both be host or both be device arrays")
        self._c(self.lib.segsalsa_str_linear_solve(self.h, p1, p2, d1))
        return out

    def set_profiling(self, on: bool):
        self._c(self.lib.segsalsa_str_set_profiling(self.h, int(bool(on))))

    def kernel_stats(self):
        n = (C.c_int64 * len(KERNEL_KINDS))()
        ms = (C.c_double * len(KERNEL_KINDS))()
        self._c(self.lib.segsalsa_str_kernel_stats(self.h, n, ms))
        return {KERNEL_KINDS[i]: (int(n[i]), float(ms[i])) for i in range(len(KERNEL_KINDS))}

    def reset_stats(self):
        self._c(self.lib.segsalsa_str_reset_stats(self.h))

    def traffic_model(self):
        a, b = C.c_double(0), C.c_double(0)
        self._c(self.lib.segsalsa_str_traffic_model(self.h, C.byref(a), C.byref(b)))
        return a.value, b.value


class Batch:
    """A batch of independent images (wraps segsalsa_str_batch_*). `params` is a list of
    Params (stream NULL); `tilings` an optional list of Tiling. image(i) gives a borrowed
    Solver view of image i for set_probs / get_labels / get_z / get_state."""

    def __init__(self, params: list, tilings: list | None = None, stream=None):
        self.lib = load()
        n = len(params)
        self._params = (Params * n)(*params)
        self._keep = params  # the weights arrays referenced by the Params
        tl = None
        if tilings is not None:
            if len(tilings) != n:
                raise ValueError("one tiling per image")
            tl = (Tiling * n)(*tilings)
        self.b = C.c_void_p()
        rc = self.lib.segsalsa_str_batch_create(n, self._params, tl, stream, C.byref(self.b))
        if rc != SEGSALSA_OK:
            raise SegsalsaError(rc, self.lib.segsalsa_str_batch_last_error(None).decode())
        self.n = n
        self.images = []
        for i in range(n):
            h = C.c_void_p()
            self._c(self.lib.segsalsa_str_batch_image(self.b, i, C.byref(h)))
            self.images.append(Solver(params[i], _borrowed=h))

    def _c(self, rc):
        if rc != SEGSALSA_OK:
            raise SegsalsaError(rc, self.lib.segsalsa_str_batch_last_error(self.b).decode())

    def image(self, i: int) -> Solver:
        return self.images[i]

    # segsalsa_str_batch_solve
    def solve(self, iters: int):
        self._c(self.lib.segsalsa_str_batch_solve(self.b, int(iters)))

    # segsalsa_str_batch_autotune
    def autotune(self, trial_iters: int = 4) -> list:
        out = (Tiling * self.n)()
        self._c(self.lib.segsalsa_str_batch_autotune(self.b, int(trial_iters), out))
        return [t.as_tuple() for t in out]

    def set_lanes(self, lanes: int):
        self._c(self.lib.segsalsa_str_batch_set_lanes(self.b, int(lanes)))

    def lanes(self) -> int:
        v = C.c_int32(0)
        self._c(self.lib.segsalsa_str_batch_get_lanes(self.b, C.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "b", None):
            for s in self.images:
                s.h = None
            self.lib.segsalsa_str_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
