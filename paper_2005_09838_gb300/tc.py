"""Thin ctypes binding of the C ABI in include/tctf2r.h.

Argument marshalling only: every step of the method runs in libtctf2r.so.
The library is loaded on first use; if it is missing the call raises
(there is no CPU fallback).  Arrays are passed as raw pointers: numpy arrays
(host) or torch tensors (host or device) in the C ABI's column-major element
order (first index fastest).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtctf2r.so")

TC_OK, TC_ERR_ARG, TC_ERR_NOMEM, TC_ERR_CUDA, TC_ERR_NUMERIC, TC_ERR_TIMEOUT, TC_ERR_STATE, TC_ERR_UNSUPPORTED = range(8)
TC_FP64, TC_FP32, TC_TF32, TC_BF16 = range(4)
TC_FLAG_SINGLE_PASS = 1
TC_STEP_EXACT, TC_STEP_SCALED = range(2)

STATUS_NAMES = {0: "TC_OK", 1: "TC_ERR_ARG", 2: "TC_ERR_NOMEM", 3: "TC_ERR_CUDA", 4: "TC_ERR_NUMERIC",
                5: "TC_ERR_TIMEOUT", 6: "TC_ERR_STATE", 7: "TC_ERR_UNSUPPORTED"}

# Entry points declared in include/tctf2r.h (checked by the tests).
EXPORTS = ("tc_init", "tc_iterate", "tc_objective", "tc_result", "tc_profile", "tc_free", "tc_last_error",
           "tc_version", "tc_rank_rule", "tc_ranks", "tc_tile", "tc_batch_launches")


class tc_params(ctypes.Structure):
    _fields_ = [
        ("n1", ctypes.c_int64), ("n2", ctypes.c_int64), ("n3", ctypes.c_int64),
        ("r", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("mu", ctypes.c_double), ("rho1", ctypes.c_double), ("rho2", ctypes.c_double),
        ("step", ctypes.c_int32), ("flags", ctypes.c_int32),
        ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
        ("eps", ctypes.c_double), ("pinv_rtol", ctypes.c_double),
    ]


assert ctypes.sizeof(tc_params) == 96


class TCError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path: str | None = None):
    """Load libtctf2r.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with `python -m paper_2005_09838_gb300.build` "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.tc_init.argtypes = [ctypes.POINTER(P), ctypes.POINTER(tc_params), P, P, P, P, ctypes.c_int32, P]
    lib.tc_init.restype = ctypes.c_int
    lib.tc_iterate.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]
    lib.tc_iterate.restype = ctypes.c_int
    lib.tc_objective.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.tc_objective.restype = ctypes.c_int
    lib.tc_result.argtypes = [P, P, P, P, ctypes.c_int32]
    lib.tc_result.restype = ctypes.c_int
    lib.tc_profile.argtypes = [P, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)]
    lib.tc_profile.restype = ctypes.c_int
    lib.tc_convergence.argtypes = [P, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32),
                                   ctypes.POINTER(ctypes.c_int64)]
    lib.tc_convergence.restype = ctypes.c_int
    lib.tc_rank_rule.argtypes = [P, ctypes.c_double, ctypes.c_int32]
    lib.tc_rank_rule.restype = ctypes.c_int
    lib.tc_ranks.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.tc_ranks.restype = ctypes.c_int
    lib.tc_complete_static.argtypes = [ctypes.POINTER(tc_params), P, P, P, P, ctypes.c_int32, P,
                                       ctypes.POINTER(ctypes.c_double), P]
    lib.tc_complete_static.restype = ctypes.c_int
    lib.tc_grad_init.argtypes = [ctypes.POINTER(P), ctypes.POINTER(tc_params), P, P, ctypes.c_int32, P]
    lib.tc_grad_init.restype = ctypes.c_int
    lib.tc_grad_eval.argtypes = [P, P, P, ctypes.POINTER(ctypes.c_double), P, P, ctypes.c_int32]
    lib.tc_grad_eval.restype = ctypes.c_int
    lib.tc_grad_free.argtypes = [P]
    lib.tc_grad_free.restype = ctypes.c_int
    lib.tc_batch_create.argtypes = [ctypes.POINTER(P), ctypes.POINTER(P), ctypes.c_int32, P]
    lib.tc_batch_create.restype = ctypes.c_int
    lib.tc_batch_iterate.argtypes = [P, ctypes.c_int32]
    lib.tc_batch_iterate.restype = ctypes.c_int
    lib.tc_batch_branches.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.tc_batch_branches.restype = ctypes.c_int
    lib.tc_batch_launches.argtypes = [P, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)]
    lib.tc_batch_launches.restype = ctypes.c_int
    lib.tc_tile.argtypes = [P, ctypes.POINTER(ctypes.c_int32)]
    lib.tc_tile.restype = ctypes.c_int
    lib.tc_batch_free.argtypes = [P]
    lib.tc_batch_free.restype = ctypes.c_int
    lib.tc_free.argtypes = [P]
    lib.tc_free.restype = ctypes.c_int
    lib.tc_last_error.argtypes = []
    lib.tc_last_error.restype = ctypes.c_char_p
    lib.tc_version.argtypes = []
    lib.tc_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int):
    if status != TC_OK:
        msg = load().tc_last_error().decode(errors="replace")
        raise TCError(status, msg)


def _ptr(a) -> int | None:
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("numpy buffers must be contiguous flat arrays in column-major element order")
        return a.ctypes.data
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous flat buffers in column-major element order")
        return a.data_ptr()
    raise TypeError(f"unsupported buffer type {type(a)}")


def make_params(n1, n2, n3, r, mu=0.0, rho1=0.0, rho2=0.0, precision=TC_FP32, step=TC_STEP_EXACT,
                alpha=1.0, beta=1.0, eps=0.0, pinv_rtol=0.0, flags=0) -> tc_params:
    return tc_params(n1, n2, n3, r, precision, mu, rho1, rho2, step, flags, alpha, beta, eps, pinv_rtol)


class Completion:
    """One TCTF2R context (tc_init ... tc_free)."""

    def __init__(self, params: tc_params, G, mask, Y0, X0=None, on_device: bool = False, stream: int | None = None):
        lib = load()
        self._lib = lib
        self.params = params
        self._ctx = ctypes.c_void_p()
        st = lib.tc_init(ctypes.byref(self._ctx), ctypes.byref(params), _ptr(G), _ptr(mask), _ptr(Y0), _ptr(X0),
                         1 if on_device else 0, stream)
        _check(st)

    @property
    def dtype(self):
        return np.float64 if self.params.precision == TC_FP64 else np.float32

    def iterate(self, n: int, count: bool = True) -> int:
        """Run n iterations; returns the number run (fewer once the stopping
        test of a context with eps > 0 has held).  count=False skips the
        count (no stream synchronisation) and returns n."""
        if not count:
            _check(self._lib.tc_iterate(self._ctx, int(n), None))
            return int(n)
        done = ctypes.c_int32(0)
        _check(self._lib.tc_iterate(self._ctx, int(n), ctypes.byref(done)))
        return done.value

    def convergence(self):
        """(||dX~||_inf, ||dY~||_inf, ||dW||_F) of the last iteration, whether
        the stopping test has held, and the iterations run since init."""
        ch = (ctypes.c_double * 3)()
        stopped = ctypes.c_int32(0)
        it = ctypes.c_int64(0)
        _check(self._lib.tc_convergence(self._ctx, ch, ctypes.byref(stopped), ctypes.byref(it)))
        return tuple(ch), bool(stopped.value), int(it.value)

    def rank_rule(self, tol: float, patience: int = 1):
        """Step 5 of the Algorithm (tc_rank_rule): rank decrease of the slices whose
        Y-step Gram has eigenvalues at or below tol * lambda_max for patience
        consecutive iterations; tol = 0 turns it off."""
        _check(self._lib.tc_rank_rule(self._ctx, float(tol), int(patience)))

    def tile(self) -> int:
        """Tile of the generic-length transform chosen at init (tc_tile; 0 for a
        dedicated-kernel length)."""
        t = ctypes.c_int32(0)
        _check(self._lib.tc_tile(self._ctx, ctypes.byref(t)))
        return t.value

    def ranks(self):
        """The rank of every frontal slice (n3 values, tc_ranks)."""
        out = (ctypes.c_int32 * int(self.params.n3))()
        _check(self._lib.tc_ranks(self._ctx, out))
        return list(out)

    def objective(self):
        f0 = ctypes.c_double()
        res = ctypes.c_double()
        _check(self._lib.tc_objective(self._ctx, ctypes.byref(f0), ctypes.byref(res)))
        return f0.value, res.value

    def result(self, W=None, X=None, Y=None, on_device: bool = False):
        _check(self._lib.tc_result(self._ctx, _ptr(W), _ptr(X), _ptr(Y), 1 if on_device else 0))

    def result_numpy(self, want_factors: bool = False):
        p = self.params
        W = np.empty(p.n1 * p.n2 * p.n3, dtype=self.dtype)
        X = np.empty(p.n1 * p.r * p.n3, dtype=self.dtype) if want_factors else None
        Y = np.empty(p.r * p.n2 * p.n3, dtype=self.dtype) if want_factors else None
        self.result(W, X, Y)
        return W, X, Y

    def profile(self, n: int):
        """Run n iterations with per-kernel CUDA events; returns the mean
        milliseconds per launch of (qcon, xstep, ystep, slab)."""
        ms = (ctypes.c_double * 4)()
        _check(self._lib.tc_profile(self._ctx, int(n), ms))
        return tuple(ms)

    def close(self):
        if self._ctx:
            self._lib.tc_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch:
    """Batched form (tc_batch_*): the given Completion contexts advanced by one
    CUDA graph launch per iteration.  The contexts stay usable (results,
    objective) and must outlive the batch."""

    def __init__(self, completions, stream: int | None = None):
        self._lib = load()
        self._members = list(completions)
        arr = (ctypes.c_void_p * len(self._members))(*[c._ctx.value for c in self._members])
        self._b = ctypes.c_void_p()
        _check(self._lib.tc_batch_create(ctypes.byref(self._b), arr, len(self._members), stream))

    def iterate(self, n: int):
        _check(self._lib.tc_batch_iterate(self._b, int(n)))

    def branches(self) -> int:
        k = ctypes.c_int32(0)
        _check(self._lib.tc_batch_branches(self._b, ctypes.byref(k)))
        return k.value

    def launches(self):
        """(graph launches made by iterate so far, 1 once the device-side loop runs
        whole calls in one launch)."""
        n = ctypes.c_int64(0)
        loop = ctypes.c_int32(0)
        _check(self._lib.tc_batch_launches(self._b, ctypes.byref(n), ctypes.byref(loop)))
        return n.value, loop.value

    def close(self):
        if self._b:
            self._lib.tc_batch_free(self._b)
            self._b = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class GradContext:
    """Differentiation form (tc_grad_*): loss of the factor model and its
    gradient.  X (n1*r*n3) and Y (r*n2*n3) in the column-major layout of
    tc_init's X0, Y0, as numpy arrays or torch tensors."""

    def __init__(self, params: tc_params, G, mask, on_device: bool = False, stream: int | None = None):
        self._lib = load()
        self.params = params
        self._ctx = ctypes.c_void_p()
        _check(self._lib.tc_grad_init(ctypes.byref(self._ctx), ctypes.byref(params), _ptr(G), _ptr(mask),
                                      1 if on_device else 0, stream))

    def eval(self, X, Y, dX=None, dY=None, on_device: bool = False) -> float:
        loss = ctypes.c_double()
        _check(self._lib.tc_grad_eval(self._ctx, _ptr(X), _ptr(Y), ctypes.byref(loss), _ptr(dX), _ptr(dY),
                                      1 if on_device else 0))
        return loss.value

    def close(self):
        if self._ctx:
            self._lib.tc_grad_free(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _check_static_buffers(params: tc_params, G, mask, Y0, X0, W):
    """The buffers of tc_complete_static must be contiguous CUDA tensors on the
    current device with the element type and element count the parameters
    imply; anything else is refused here, before the kernels could read or
    write outside a buffer."""
    import torch
    real = torch.float64 if params.precision == TC_FP64 else torch.float32
    n1, n2, n3, r = params.n1, params.n2, params.n3, params.r
    want = {"G": (G, real, n1 * n2 * n3), "mask": (mask, torch.uint8, n1 * n2 * n3),
            "Y0": (Y0, real, r * n2 * n3), "W": (W, real, n1 * n2 * n3)}
    if X0 is not None:
        want["X0"] = (X0, real, n1 * r * n3)
    dev = torch.cuda.current_device()
    for name, (t, dtype, numel) in want.items():
        if not isinstance(t, torch.Tensor) or not t.is_cuda:
            raise ValueError(f"{name} must be a CUDA tensor (tc_complete_static takes device buffers only)")
        if t.device.index != dev:
            raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{dev}")
        if t.dtype != dtype:
            raise ValueError(f"{name} must be {dtype} for this precision, got {t.dtype}")
        if t.numel() != numel:
            raise ValueError(f"{name} must hold {numel} elements, got {t.numel()}")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")


def complete_static(params: tc_params, G, mask, Y0, n_iters: int, W, X0=None, stream: int | None = None,
                    want_f0: bool = True):
    """tc_complete_static: the whole completion with no device allocation, for
    callers that cannot call cudaMalloc (their device memory belongs to a host
    framework's allocator, or a cudaMalloc would stall a latency-critical
    loop).  All buffers are CUDA tensors on the current device, checked for
    element type and count before the call; returns f0 (or None)."""
    _check_static_buffers(params, G, mask, Y0, X0, W)
    lib = load()
    f0 = ctypes.c_double()
    st = lib.tc_complete_static(ctypes.byref(params), _ptr(G), _ptr(mask), _ptr(Y0), _ptr(X0), int(n_iters), _ptr(W),
                                ctypes.byref(f0) if want_f0 else None, stream)
    _check(st)
    return f0.value if want_f0 else None


def version() -> str:
    return load().tc_version().decode()
