"""The timed bench workload, end to end, against the FP64 oracle.

bench.py times completions of 100 TCTF2R iterations of the 144 x 288 x 168
traffic tensor (r = 8, FP32, mu = rho1 = 1e-3, rho2 = 0.1) at 10, 20, 40 and
60% observed.  Each test runs that completion through the C ABI and compares
it with the oracle's 100 iterations on the same seeded inputs, with the
oracle's default pseudo-inverse cutoff (r 2^-52): relative Frobenius error of
W and relative error of f0 within 1e-5 (the FP32 bar), recovery NMSE within
1e-4.  At 40 and 60% observed the Y-step Gram of the DC slice reaches a
condition number near 2e6 late in the run; these cases check the FP64
real-slice solve of the FP32 path.
"""
import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

OBSERVED = (0.1, 0.2, 0.4, 0.6)
ITERS = 100
SETTING = (1e-3, 1e-3, 1e-1)


@pytest.fixture(scope="module")
def oracle_runs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import _oracle_jobs
    pool, futs = _oracle_jobs.start_c2_trajectories(OBSERVED, ITERS, SETTING)
    from paper_2005_09838_gb300 import build
    build.build()
    yield futs
    pool.shutdown(cancel_futures=True)


@pytest.mark.parametrize("observed", OBSERVED)
def test_bench_workload_100_iterations_fp32(oracle_runs, observed):
    from paper_2005_09838_gb300 import api
    w = wl.c2(observed)
    inst = wl.as_precision(wl.generate(w), np.float32)
    got = api.complete(inst["G"], inst["mask"], inst["Y0"], w.r, ITERS, *SETTING, precision="fp32")
    ref = oracle_runs[observed].result()
    err_w = np.linalg.norm(got["W"] - ref["W"]) / np.linalg.norm(ref["W"])
    err_f = abs(got["f0"] - ref["f0"]) / abs(ref["f0"])
    d_nmse = abs(wl.nmse(inst["M"], got["W"], inst["mask"]) - ref["nmse"])
    print(f"{observed:.0%} observed: W {err_w:.2e}, f0 {err_f:.2e}, NMSE difference {d_nmse:.1e}")
    assert err_w <= 1e-5
    assert err_f <= 1e-5
    assert d_nmse <= 1e-4
