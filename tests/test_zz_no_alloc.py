"""tc_complete_static: the allocation-free entry point.

Callers that cannot call cudaMalloc (a host framework owns the device memory,
or an allocation would synchronise the device inside a latency-critical loop)
get the whole completion from one call whose work arrays live in the library's
fixed 16 MiB device array.  This file checks, through the C ABI, that it
returns the same W and f0 as the allocating path (tc_init / tc_iterate /
tc_result / tc_objective), on two calls in a row with different inputs (the
shared array keeps the previous call's contents), and that an oversized
problem is rejected with a clear error.  It is collected last so a run that
stops at the first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import workloads as wl

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09838_gb300 import build
    build.build()


def _case(shape, r, obs, seed, precision):
    w = wl.custom(*shape, r, obs, seed=seed)
    inst = wl.generate(w)
    dt = np.float64 if precision == "fp64" else np.float32
    if precision == "fp32":
        inst = wl.as_precision(inst, np.float32)
    return w, inst, dt


def _allocating_path(tc, p, g, m, y, iters):
    with tc.Completion(p, g, m, y) as c:
        c.iterate(iters)
        f0, _ = c.objective()
        W, _, _ = c.result_numpy()
    return W, f0


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_entry_matches_allocating_path_twice(precision):
    import torch
    from paper_2005_09838_gb300 import tc
    prec = tc.TC_FP64 if precision == "fp64" else tc.TC_FP32
    stream = torch.cuda.current_stream().cuda_stream
    # the third case has r > 16: the entry point's one-CTA-per-slice X-step with
    # FP64-storage solves, against the engine's four-kernel X-step
    cases = [((16, 48, 7), 2, 0.5, 901), ((12, 40, 12), 3, 0.3, 902), ((60, 40, 8), 20, 0.4, 903)]
    for shape, r, obs, seed in cases:  # calls in a row, different sizes and data
        w, inst, dt = _case(shape, r, obs, seed, precision)
        p = tc.make_params(w.n1, w.n2, w.n3, w.r, 1e-3, 1e-3, 1e-1, precision=prec)
        g = wl.to_colmajor(inst["G"], dt)
        m = wl.to_colmajor(inst["mask"], np.uint8)
        y = wl.to_colmajor(inst["Y0"], dt)
        W_ref, f_ref = _allocating_path(tc, p, g, m, y, 15)
        dg, dm, dy = (torch.from_numpy(a).cuda() for a in (g, m, y))
        Wd = torch.full((w.N,), float("nan"), dtype=torch.float64 if dt == np.float64 else torch.float32,
                        device="cuda")
        f0 = tc.complete_static(p, dg, dm, dy, 15, Wd, stream=stream)
        W = Wd.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(W - W_ref) / np.linalg.norm(W_ref)
        assert rel <= TOL[precision], (shape, rel)
        assert abs(f0 - f_ref) <= TOL[precision] * abs(f_ref)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_static_entry_with_initial_x_and_cutoff(precision):
    # a seeded X0 (the static path's own DFT of X0) and a pseudo-inverse cutoff
    # other than the default, against Completion(..., X0=X0) with the same
    # parameters, on two calls in a row
    import torch
    from paper_2005_09838_gb300 import tc
    prec = tc.TC_FP64 if precision == "fp64" else tc.TC_FP32
    stream = torch.cuda.current_stream().cuda_stream
    for shape, r, obs, seed in [((14, 36, 7), 3, 0.4, 911), ((20, 30, 9), 4, 0.5, 912)]:
        w, inst, dt = _case(shape, r, obs, seed, precision)
        rng = np.random.default_rng(seed)
        X0 = rng.standard_normal((w.n1, w.r, w.n3)).astype(dt).astype(np.float64)
        p = tc.make_params(w.n1, w.n2, w.n3, w.r, 1e-3, 1e-3, 1e-1, precision=prec, pinv_rtol=1e-4)
        g = wl.to_colmajor(inst["G"], dt)
        m = wl.to_colmajor(inst["mask"], np.uint8)
        y = wl.to_colmajor(inst["Y0"], dt)
        x = wl.to_colmajor(X0, dt)
        with tc.Completion(p, g, m, y, x) as c:
            c.iterate(12)
            f_ref, _ = c.objective()
            W_ref, _, _ = c.result_numpy()
        dg, dm, dy, dx = (torch.from_numpy(a).cuda() for a in (g, m, y, x))
        Wd = torch.full((w.N,), float("nan"), dtype=torch.from_numpy(g).dtype, device="cuda")
        f0 = tc.complete_static(p, dg, dm, dy, 12, Wd, X0=dx, stream=stream)
        W = Wd.cpu().numpy().astype(np.float64)
        rel = np.linalg.norm(W - W_ref) / np.linalg.norm(W_ref)
        assert rel <= TOL[precision], (shape, rel)
        assert abs(f0 - f_ref) <= TOL[precision] * abs(f_ref)


def test_static_entry_refuses_host_and_mismatched_buffers():
    # host buffers, a W of the wrong element type and a short Y0 are refused
    # before anything reaches the device
    import torch
    from paper_2005_09838_gb300 import tc
    n1, n2, n3, r = 8, 16, 5, 2
    p = tc.make_params(n1, n2, n3, r, precision=tc.TC_FP32)
    N = n1 * n2 * n3
    g = torch.zeros(N, dtype=torch.float32, device="cuda")
    m = torch.zeros(N, dtype=torch.uint8, device="cuda")
    y = torch.zeros(r * n2 * n3, dtype=torch.float32, device="cuda")
    W = torch.zeros(N, dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError, match="CUDA tensor"):
        tc.complete_static(p, g.cpu(), m, y, 1, W)
    with pytest.raises(ValueError, match="must be torch.float32"):
        tc.complete_static(p, g, m, y, 1, W.double())
    with pytest.raises(ValueError, match="elements"):
        tc.complete_static(p, g, m, y[:-1], 1, W)
    # the C entry point itself refuses a host pointer for W
    lib = tc.load()
    host_w = np.zeros(N, dtype=np.float32)
    st = lib.tc_complete_static(ctypes.byref(p), g.data_ptr(), m.data_ptr(), y.data_ptr(), None, 1,
                                host_w.ctypes.data, None, torch.cuda.current_stream().cuda_stream)
    assert st == tc.TC_ERR_ARG
    assert "device memory" in lib.tc_last_error().decode()


def test_static_entry_rejects_oversized_problem():
    import torch
    from paper_2005_09838_gb300 import tc
    n1, n2, n3, r = 144, 288, 168, 8  # about 60 MB of state: beyond the 16 MiB array
    p = tc.make_params(n1, n2, n3, r, precision=tc.TC_FP32)
    g = torch.zeros(n1 * n2 * n3, dtype=torch.float32, device="cuda")
    m = torch.zeros(n1 * n2 * n3, dtype=torch.uint8, device="cuda")
    y = torch.zeros(r * n2 * n3, dtype=torch.float32, device="cuda")
    with pytest.raises(tc.TCError) as ei:
        tc.complete_static(p, g, m, y, 1, g)
    assert "TC_ERR_ARG" in str(ei.value) and "bytes of scratch" in str(ei.value)
