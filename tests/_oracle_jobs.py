"""Oracle runs for the GPU tests, in worker processes.

The full 100-iteration trajectories of the 144 x 288 x 168 workload take the
FP64 oracle a minute or more each; the GPU tests start them together in a
pool of spawned processes (a forked child of a process that already holds a
CUDA context can hang) and compare when each result is ready.  Test
infrastructure only: nothing outside tests/ imports this module.
"""
from __future__ import annotations

import concurrent.futures
import multiprocessing
import os

import numpy as np


def _c2_trajectory(observed: float, iters: int, setting):
    import workloads as wl
    from oracle import method as O
    w = wl.c2(observed)
    inst = wl.as_precision(wl.generate(w), np.float32)
    mu, rho1, rho2 = setting
    ref = O.tctf2r(inst["G"], inst["mask"], w.r, mu, rho1, rho2, inst["Y0"], iters=iters)
    return {"W": ref["W"], "f0": ref["f0"], "nmse": wl.nmse(inst["M"], ref["W"], inst["mask"])}


def start_c2_trajectories(observed_list, iters, setting):
    """Submit one oracle trajectory per observed ratio; returns (pool, futures).
    Each worker gets an equal share of the host's cores for its BLAS threads."""
    n = len(observed_list)
    share = str(max(1, (os.cpu_count() or 1) // n))
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = share
    try:
        pool = concurrent.futures.ProcessPoolExecutor(max_workers=n, mp_context=multiprocessing.get_context("spawn"))
        futs = {obs: pool.submit(_c2_trajectory, obs, iters, setting) for obs in observed_list}
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return pool, futs


def c4_inputs():
    """The 529 x 288 x 168 differentiation workload (r = 16, 20% observed) in
    FP32-representable values, and seeded initial factors X ~ N(0,1), Y = Y0."""
    import workloads as wl
    w = wl.c4(0.2)
    inst = wl.as_precision(wl.generate(w), np.float32)
    rng = np.random.default_rng(w.seed + 17)
    X = rng.standard_normal((w.n1, w.r, w.n3)).astype(np.float32).astype(np.float64)
    return w, inst, X


def _c4_loss_grad(rho1: float):
    from oracle import method as O
    w, inst, X = c4_inputs()
    Y = inst["Y0"]
    f = O.factor_loss(X, Y, inst["G"], inst["mask"], rho1)
    gX, gY = O.factor_loss_grad(X, Y, inst["G"], inst["mask"], rho1)
    return {"f": f, "gX": gX, "gY": gY}


def start_c4_loss_grad(rho1: float):
    """The oracle's loss and gradients of the differentiation form at the C4
    initial factors, in one spawned worker; returns (pool, future)."""
    pool = concurrent.futures.ProcessPoolExecutor(max_workers=1, mp_context=multiprocessing.get_context("spawn"))
    return pool, pool.submit(_c4_loss_grad, rho1)
