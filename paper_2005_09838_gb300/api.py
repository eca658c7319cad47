"""Convenience wrapper: numpy tensors indexed [i1, i2, i3] in, numpy out.

Marshalling only (layout conversion to the C ABI's column-major order and
back); the completion itself runs in libtctf2r.so.
"""
from __future__ import annotations

import numpy as np

from . import tc


def _colmajor(a: np.ndarray, dtype) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a).transpose(2, 1, 0)).astype(dtype, copy=False).reshape(-1)


def _from_colmajor(flat: np.ndarray, shape) -> np.ndarray:
    a, b, c = shape
    return flat.reshape(c, b, a).transpose(2, 1, 0)


def complete(G, mask, Y0, r, iters, mu=0.0, rho1=0.0, rho2=0.0, precision="fp32", X0=None,
             want_factors=False, objective=True, step="exact", alpha=1.0, beta=1.0, eps=0.0,
             single_pass=False, rank_tol=0.0, rank_patience=1):
    """Run up to ``iters`` TCTF2R iterations on the GPU (fewer when ``eps`` > 0
    and the stopping test holds).  Returns a dict with W (and X, Y spatial with
    ``want_factors``), f0, resid_obs, the iterations run and, with ``eps`` > 0,
    the last changes (||dX~||_inf, ||dY~||_inf, ||dW||_F).  ``precision`` is
    "fp64", "fp32", or the precision form "tf32" / "bf16" (float data; see
    tc_precision in the C header), where ``single_pass`` rounds the tensor-core
    operands once instead of splitting them.  ``rank_tol`` > 0 turns on step 5
    of the Algorithm (tc_rank_rule) with ``rank_patience``; the result then
    holds the final rank vector under "ranks"."""
    prec = {"fp32": tc.TC_FP32, "fp64": tc.TC_FP64, "tf32": tc.TC_TF32, "bf16": tc.TC_BF16}[precision]
    dt = np.float64 if prec == tc.TC_FP64 else np.float32
    n1, n2, n3 = G.shape
    st = {"exact": tc.TC_STEP_EXACT, "scaled": tc.TC_STEP_SCALED}[step]
    p = tc.make_params(n1, n2, n3, r, mu=mu, rho1=rho1, rho2=rho2, precision=prec, step=st, alpha=alpha,
                       beta=beta, eps=eps, flags=tc.TC_FLAG_SINGLE_PASS if single_pass else 0)
    g = _colmajor(G, dt)
    m = _colmajor(np.asarray(mask, dtype=bool), np.uint8)
    y = _colmajor(Y0, dt)
    x = None if X0 is None else _colmajor(X0, dt)
    with tc.Completion(p, g, m, y, x) as c:
        if rank_tol > 0:
            c.rank_rule(rank_tol, rank_patience)
        out = {"iters": c.iterate(iters)}
        if rank_tol > 0:
            out["ranks"] = c.ranks()
        if eps > 0:
            out["changes"], out["stopped"], out["iters_total"] = c.convergence()
        if objective:
            out["f0"], out["resid_obs"] = c.objective()
        W, X, Y = c.result_numpy(want_factors)
        out["W"] = _from_colmajor(W, (n1, n2, n3)).astype(np.float64)
        if want_factors:
            out["X"] = _from_colmajor(X, (n1, r, n3)).astype(np.float64)
            out["Y"] = _from_colmajor(Y, (r, n2, n3)).astype(np.float64)
    return out
