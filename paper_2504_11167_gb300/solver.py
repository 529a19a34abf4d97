"""ctypes binding of ``liblrspike.so`` (C ABI in include/lrspike.h).

Argument marshalling only: every step of the factorisation and of the solve
runs in the library's CUDA kernels.  PyTorch provides device memory and the
stream.  If the shared library is missing the binding raises; there is no
fallback path.

Layouts (the C ABI's, expressed as row-major torch tensors):
  band : float64 tensor of shape (2k+1, ld), ld >= n, band[k + i - j, j] = A[i, j]
  f, x : float64 tensor of shape (n,) or (nrhs, ld); row q is right-hand side q
Tensors may live on the GPU or on the host; host tensors are copied by the
library (that is the end-to-end path).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "liblrspike.so")

STATUS = {0: "OK", 1: "INVALID_ARG", 2: "STATE", 3: "OOM", 4: "CUDA", 5: "SINGULAR",
          6: "NOT_CONVERGED", 7: "UNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
COMPRESS = {"spike": 0, "coupling": 1}
REDUCED = {"full": 0, "truncated": 1, "otf": 2}
OUTER = {"ir": 0, "bicgstab": 1, "none": 2}


class LRSpikeError(RuntimeError):
    def __init__(self, status: int, message: str):
        self.status = status
        self.name = STATUS.get(status, str(status))
        super().__init__(f"{self.name}: {message}")


class Options(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("k", ctypes.c_int32), ("p", ctypes.c_int32),
                ("r", ctypes.c_int32), ("precision", ctypes.c_int32), ("pivoting", ctypes.c_int32),
                ("compress", ctypes.c_int32), ("reduced", ctypes.c_int32), ("outer", ctypes.c_int32),
                ("max_iter", ctypes.c_int32), ("tol", ctypes.c_double), ("rank_tol", ctypes.c_double),
                ("max_nrhs", ctypes.c_int32), ("profile", ctypes.c_int32),
                ("oversample", ctypes.c_int32), ("power_iters", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("graph_safe", ctypes.c_int32), ("block", ctypes.c_int32),
                ("otf_tol", ctypes.c_double), ("otf_max_iter", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("max_rel_residual", ctypes.c_double),
                ("rel_residual", ctypes.POINTER(ctypes.c_double)), ("reduced_iterations", ctypes.c_int32)]


_lib = None
EXPORTS = ["lrspike_options_default", "lrspike_create", "lrspike_factor", "lrspike_solve",
           "lrspike_solve_transpose", "lrspike_destroy", "lrspike_last_error",
           "lrspike_launch_count", "lrspike_profile_get", "lrspike_profile_reset",
           "lrspike_get_reduced", "lrspike_residual_noalloc", "lrspike_band_outer", "lrspike_finish",
           "lrspike_fp64_fma_probe"]


def load_library(path: str = LIB_PATH):
    """Loads the CUDA library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise LRSpikeError(4, f"{path} is missing: build it with __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    H = ctypes.c_void_p
    dp = ctypes.POINTER(ctypes.c_double)
    lib.lrspike_options_default.argtypes = [ctypes.POINTER(Options), ctypes.c_int64, ctypes.c_int32,
                                            ctypes.c_int32, ctypes.c_int32]
    lib.lrspike_create.argtypes = [ctypes.POINTER(Options), ctypes.c_void_p, ctypes.POINTER(H)]
    lib.lrspike_factor.argtypes = [H, ctypes.c_void_p, ctypes.c_int64]
    lib.lrspike_solve.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                  ctypes.POINTER(Info)]
    lib.lrspike_solve_transpose.argtypes = lib.lrspike_solve.argtypes
    lib.lrspike_finish.argtypes = [H, ctypes.POINTER(Info)]
    lib.lrspike_destroy.argtypes = [H]
    lib.lrspike_last_error.argtypes = [H]
    lib.lrspike_last_error.restype = ctypes.c_char_p
    lib.lrspike_launch_count.argtypes = [H]
    lib.lrspike_launch_count.restype = ctypes.c_int64
    lib.lrspike_profile_get.argtypes = [H, ctypes.c_int32, ctypes.POINTER(ctypes.c_char_p),
                                        ctypes.POINTER(ctypes.c_int64), dp]
    lib.lrspike_profile_reset.argtypes = [H]
    lib.lrspike_get_reduced.argtypes = [H, ctypes.c_void_p, ctypes.c_void_p]
    lib.lrspike_residual_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                             ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                             ctypes.c_void_p, ctypes.c_void_p]
    lib.lrspike_band_outer.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64,
                                        ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p,
                                        ctypes.c_int64, ctypes.c_void_p]
    lib.lrspike_fp64_fma_probe.argtypes = [ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    for name in EXPORTS:
        if name not in ("lrspike_last_error", "lrspike_launch_count"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _ptr(t) -> int:
    return t.data_ptr()


def residual_noalloc(band, k: int, f, x, r, norms, stream=None) -> None:
    """r = f - A x and the column norms of r, through the allocation-free
    entry point (no handle; scratch is a static device array).  band: device
    (2k+1, ld_band); f, x: device (nrhs, ld); r: device (nrhs, n); norms:
    device (nrhs,).  Enqueued on ``stream`` (default: torch's current stream)."""
    import torch
    lib = load_library()
    F = f.unsqueeze(0) if f.dim() == 1 else f
    X = x.unsqueeze(0) if x.dim() == 1 else x
    R = r.unsqueeze(0) if r.dim() == 1 else r
    nrhs, ld = F.shape
    n = R.shape[-1]
    # the C entry point sees raw pointers only: every extent it will touch is
    # checked here against the tensors
    for name, t in (("band", band), ("f", F), ("x", X), ("r", R), ("norms", norms)):
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous float64 CUDA tensor")
    if X.shape != F.shape:
        raise ValueError("x must have the shape of f")
    if R.shape != (nrhs, n) or ld < n:
        raise ValueError("r must be (nrhs, n) with n <= the leading dimension of f")
    if norms.numel() < nrhs:
        raise ValueError("norms must hold nrhs values")
    if band.dim() != 2 or band.shape[0] != 2 * k + 1 or band.shape[1] < n:
        raise ValueError("band must be (2k+1, ld_band) with ld_band >= n")
    if stream is None:
        stream = torch.cuda.current_stream()
    st = lib.lrspike_residual_noalloc(ctypes.c_void_p(_ptr(band)), band.shape[1], n, k,
                                      ctypes.c_void_p(_ptr(F)), ctypes.c_void_p(_ptr(X)),
                                      ctypes.c_void_p(_ptr(R)), nrhs, ld,
                                      ctypes.c_void_p(_ptr(norms)),
                                      ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise LRSpikeError(st, lib.lrspike_last_error(None).decode(errors="replace"))


def fp64_fma_tflops(iters: int = 1 << 16, stream=None) -> float:
    """Measured FP64 FMA rate of the current GPU in TFLOP/s (one probe
    kernel timed with CUDA events on ``stream``, default torch's current)."""
    import torch
    lib = load_library()
    if stream is None:
        stream = torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    st = lib.lrspike_fp64_fma_probe(int(iters), ctypes.byref(out), ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise LRSpikeError(st, lib.lrspike_last_error(None).decode(errors="replace"))
    return float(out.value)


def band_outer(lam, x, k: int, alpha: float, grad_band, stream=None) -> None:
    """grad_band[k + i - j, j] = alpha * sum_q lam[q, i] x[q, j] on the band
    (0 outside the matrix): with alpha = -1 the band part of dL/dA = -lam x^T.
    lam, x: device (nrhs, ld) or (n,); grad_band: device (2k+1, ld_band)."""
    import torch
    lib = load_library()
    L = lam.unsqueeze(0) if lam.dim() == 1 else lam
    X = x.unsqueeze(0) if x.dim() == 1 else x
    assert L.shape == X.shape and L.is_contiguous() and X.is_contiguous() and grad_band.is_contiguous()
    nrhs, ld = L.shape
    n = grad_band.shape[1] if grad_band.shape[1] <= ld else ld
    if stream is None:
        stream = torch.cuda.current_stream()
    st = lib.lrspike_band_outer(ctypes.c_void_p(_ptr(L)), ctypes.c_void_p(_ptr(X)), nrhs, ld, n, k, alpha,
                                ctypes.c_void_p(_ptr(grad_band)), grad_band.shape[1],
                                ctypes.c_void_p(stream.cuda_stream))
    if st != 0:
        raise LRSpikeError(st, lib.lrspike_last_error(None).decode(errors="replace"))


class LRSpike:
    """One LR-SPIKE handle: ``factor`` once, then ``solve`` / ``solve_transpose``."""

    def __init__(self, n: int, k: int, p: int, r: int, precision: str = "fp64",
                 compress: str = "spike", reduced: str = "full", outer: str = "ir",
                 pivoting: bool = False, tol: Optional[float] = None, max_iter: int = 50,
                 rank_tol: Optional[float] = None, max_nrhs: int = 16, profile: bool = False,
                 stream=None, graph_safe: bool = False, block: int = 0, oversample: Optional[int] = None,
                 power_iters: int = 2, otf_tol: float = 1e-8, otf_max_iter: int = 100):
        import torch
        self._lib = load_library()
        o = Options()
        self._check(self._lib.lrspike_options_default(ctypes.byref(o), n, k, p, r), None)
        o.precision = PRECISION[precision]
        o.compress = COMPRESS[compress]
        o.reduced = REDUCED[reduced]
        o.outer = OUTER[outer]
        o.pivoting = int(bool(pivoting))
        o.max_iter = max_iter
        o.tol = tol if tol is not None else (1e-12 if precision == "fp64" else 1e-10)
        o.rank_tol = rank_tol if rank_tol is not None else (1e-13 if precision == "fp64" else 1e-6)
        o.max_nrhs = max_nrhs
        o.profile = int(bool(profile))
        o.graph_safe = int(bool(graph_safe))
        o.block = block
        if oversample is not None:
            o.oversample = oversample
        o.power_iters = power_iters
        o.otf_tol = otf_tol
        o.otf_max_iter = otf_max_iter
        self.opt = o
        self.n, self.k, self.p, self.r = n, k, p, r
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        self._stream = stream
        sptr = ctypes.c_void_p(stream.cuda_stream if stream is not None else 0)
        h = ctypes.c_void_p()
        self._check(self._lib.lrspike_create(ctypes.byref(o), sptr, ctypes.byref(h)), None)
        self._h = h
        self._band = None

    # -- helpers ---------------------------------------------------------
    def _check(self, st: int, h):
        if st != 0:
            msg = self._lib.lrspike_last_error(h).decode(errors="replace")
            raise LRSpikeError(st, msg)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lrspike_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- API --------------------------------------------------------------
    def factor(self, band):
        """LR-SPIKE factorisation of the banded matrix held in ``band``."""
        assert band.dtype.is_floating_point and band.element_size() == 8, "band must be float64"
        assert band.dim() == 2 and band.shape[0] == 2 * self.k + 1 and band.is_contiguous()
        self._check(self._lib.lrspike_factor(self._h, ctypes.c_void_p(_ptr(band)), band.shape[1]),
                    self._h)
        self._band = band  # borrowed by the library: keep it alive

    def _solve(self, fn, f, x, allow_unconverged):
        import torch
        squeeze = f.dim() == 1
        F = f.unsqueeze(0) if squeeze else f
        assert F.dtype == torch.float64 and F.is_contiguous()
        nrhs, ld = F.shape
        if x is None:
            x = torch.empty_like(F)
        X = x.unsqueeze(0) if x.dim() == 1 else x
        assert X.shape == F.shape and X.is_contiguous() and X.device == F.device
        rel = (ctypes.c_double * nrhs)()
        info = Info(0, 0, 0.0, ctypes.cast(rel, ctypes.POINTER(ctypes.c_double)))
        st = fn(self._h, ctypes.c_void_p(_ptr(F)), ctypes.c_void_p(_ptr(X)), nrhs, ld,
                ctypes.byref(info))
        if st != 0 and not (allow_unconverged and st == 6):
            self._check(st, self._h)
        out = {"iterations": info.iterations, "converged": bool(info.converged),
               "max_rel_residual": info.max_rel_residual, "rel_residual": list(rel),
               "reduced_iterations": info.reduced_iterations}
        return (X[0] if squeeze else X), out

    def solve(self, f, x=None, allow_unconverged=False):
        """x = A^{-1} f (or M^{-1} f with outer='none'); returns (x, info)."""
        return self._solve(self._lib.lrspike_solve, f, x, allow_unconverged)

    def solve_transpose(self, h, x=None, allow_unconverged=False):
        """lambda = A^{-T} h (or M^{-T} h with outer='none'); returns (lambda, info)."""
        return self._solve(self._lib.lrspike_solve_transpose, h, x, allow_unconverged)

    def finish(self, nrhs: int = 16, allow_unconverged: bool = False) -> dict:
        """graph_safe handles: wait for the enqueued work and report the last
        factorisation and solve (raises on SINGULAR, and on NOT_CONVERGED
        unless allowed)."""
        rel = (ctypes.c_double * nrhs)()
        info = Info(0, 0, 0.0, ctypes.cast(rel, ctypes.POINTER(ctypes.c_double)))
        st = self._lib.lrspike_finish(self._h, ctypes.byref(info))
        if st != 0 and not (allow_unconverged and st == 6):
            self._check(st, self._h)
        return {"iterations": info.iterations, "converged": bool(info.converged),
                "max_rel_residual": info.max_rel_residual, "rel_residual": list(rel)}

    def launch_count(self) -> int:
        return int(self._lib.lrspike_launch_count(self._h))

    def profile(self) -> dict:
        """Per-kernel (launches, total ms) measured with CUDA events (profile=True)."""
        out = {}
        i = 0
        name = ctypes.c_char_p()
        cnt = ctypes.c_int64()
        ms = ctypes.c_double()
        while self._lib.lrspike_profile_get(self._h, i, ctypes.byref(name), ctypes.byref(cnt),
                                            ctypes.byref(ms)) == 0:
            out[name.value.decode()] = (int(cnt.value), float(ms.value))
            i += 1
        return out

    def profile_reset(self):
        self._check(self._lib.lrspike_profile_reset(self._h), self._h)

    def reduced(self):
        """(sigma [p, 2, r], R) as numpy arrays: singular values kept per spike
        (T_i then W_i) and the reduced matrix that the solve uses."""
        import numpy as np
        sig = np.zeros((self.p, 2, self.r))
        nz = 2 * self.r * max(self.p - 1, 0)
        R = np.zeros((nz, nz))
        self._check(self._lib.lrspike_get_reduced(self._h, ctypes.c_void_p(sig.ctypes.data),
                                                  ctypes.c_void_p(R.ctypes.data if nz else 0)),
                    self._h)
        return sig, R
