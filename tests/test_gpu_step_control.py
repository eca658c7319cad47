"""Step control of the TCTF2R Algorithm on the GPU against the FP64 oracle.

* Scaled steps (Eq. (updataXYW1)): X <- X + (alpha / L1) d_X with
  L1 = ||H_rho1||_2 ||Y~Y~^*||_2, Y <- Y + (beta / L2) d_Y with
  L2 = ||X~^* H_rho1 X~||_2, no line search.
* Stopping test (step 6 of the Algorithm): the loop ends after the first
  iteration with ||X~' - X~||_inf <= eps, ||Y~' - Y~||_inf <= eps and
  ||W' - W||_F <= eps.  eps is placed between the largest change of two
  consecutive oracle iterations (5% or more apart, far beyond the FP32 error
  of the changes), so both sides must stop at the same one.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import method as O

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5, "tf32": 1e-3}
SETTING = (1e-3, 1e-3, 1e-1)


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09838_gb300 import build
    build.build()


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _inst(w, precision):
    inst = wl.generate(w)
    return inst if precision == "fp64" else wl.as_precision(inst, np.float32)


@pytest.mark.parametrize("precision,shape,r,obs,iters", [
    ("fp64", (16, 48, 7), 2, 0.5, 40),      # the 16x48x7 workload (register FFT, n3 = 7)
    ("fp32", (20, 40, 112), 4, 0.3, 25),    # shared-memory transform, n3 = 112
    ("fp64", (9, 30, 12), 3, 0.4, 25),      # generic transform
    ("tf32", (200, 96, 12), 32, 0.3, 12),   # precision form: lambda_max from the block Jacobi
])
@pytest.mark.parametrize("alpha,beta", [(1.0, 1.0), (0.6, 0.8)])
def test_scaled_steps_match_oracle(precision, shape, r, obs, iters, alpha, beta):
    # X0 ~ N(0, 1) (seeded): from X0 = 0 the first scaled X-step is tiny, G = X~^*H X~
    # nearly vanishes and beta / L2 grows without bound, overflowing FP32 within a
    # few iterations (the FP64 trajectory shows the same growth)
    from paper_2005_09838_gb300 import api
    w = wl.custom(*shape, r, obs, seed=4100 + shape[2])
    inst = _inst(w, precision)
    dt = np.float64 if precision == "fp64" else np.float32
    X0 = np.random.default_rng(4100 + shape[0]).standard_normal((shape[0], r, shape[2])).astype(dt)
    ref = O.tctf2r(inst["G"], inst["mask"], r, *SETTING, inst["Y0"], X0=X0, iters=iters, step="scaled",
                   alpha=alpha, beta=beta)
    got = api.complete(inst["G"], inst["mask"], inst["Y0"], r, iters, *SETTING, precision, X0=X0, step="scaled",
                       alpha=alpha, beta=beta)
    assert got["iters"] == iters
    assert _rel(got["W"], ref["W"]) <= TOL[precision]
    assert abs(got["f0"] - ref["f0"]) <= TOL[precision] * abs(ref["f0"])


def test_scaled_steps_differ_from_exact_steps():
    # the scaled rule is a different trajectory: guards against the step being ignored
    from paper_2005_09838_gb300 import api
    w = wl.custom(16, 48, 7, 2, 0.5, seed=4107)
    inst = wl.generate(w)
    X0 = np.random.default_rng(4107).standard_normal((16, 2, 7))
    a = api.complete(inst["G"], inst["mask"], inst["Y0"], 2, 10, *SETTING, "fp64", X0=X0, step="scaled",
                     alpha=0.5, beta=0.5)
    b = api.complete(inst["G"], inst["mask"], inst["Y0"], 2, 10, *SETTING, "fp64", X0=X0)
    assert _rel(a["W"], b["W"]) > 1e-6


def _eps_between(hist, lo=4, margin=1.5):
    """An eps with max change(j) <= eps < max change(i) for all i < j, for the
    first j >= lo where the largest change has dropped by the margin."""
    m = np.maximum(np.maximum(hist["dX"], hist["dY"]), hist["dW"])
    for j in range(lo, len(m)):
        prev = m[:j].min()
        if m[j] < prev / margin:
            return float(np.sqrt(m[j] * prev)), j + 1
    raise AssertionError("no iteration with a clear drop of the largest change")


@pytest.mark.parametrize("precision,shape,r,obs", [
    ("fp64", (16, 48, 7), 2, 0.5),
    ("fp32", (20, 40, 112), 4, 0.3),
    ("fp32", (24, 36, 168), 4, 0.3),
    ("fp64", (9, 30, 12), 3, 0.4),
    ("tf32", (200, 96, 12), 32, 0.3),   # precision form: changes from the tensor-core Z~ and split X-step
])
def test_stopping_test_stops_at_the_oracle_iteration(precision, shape, r, obs):
    from paper_2005_09838_gb300 import api
    w = wl.custom(*shape, r, obs, seed=4200 + shape[2])
    inst = _inst(w, precision)
    full = O.tctf2r(inst["G"], inst["mask"], r, *SETTING, inst["Y0"], iters=60, record=True)
    eps, j = _eps_between(full["hist"], lo=4, margin=1.05)
    ref = O.tctf2r(inst["G"], inst["mask"], r, *SETTING, inst["Y0"], iters=60, eps=eps)
    assert ref["iters"] == j
    got = api.complete(inst["G"], inst["mask"], inst["Y0"], r, 60, *SETTING, precision, eps=eps)
    assert got["iters"] == j and got["iters_total"] == j and got["stopped"]
    assert _rel(got["W"], ref["W"]) <= TOL[precision]
    # the reported changes are those of iteration j
    h = full["hist"]
    want = np.array([h["dX"][j - 1], h["dY"][j - 1], h["dW"][j - 1]])
    tol = 1e-8 if precision == "fp64" else 0.2
    assert np.all(np.abs(np.array(got["changes"]) - want) <= tol * np.maximum(want, 1e-300) + 1e-12)


def test_stopping_test_off_runs_every_iteration_and_reports_state_error():
    from paper_2005_09838_gb300 import tc
    w = wl.custom(16, 48, 7, 2, 0.5, seed=4300)
    inst = wl.generate(w)
    p = tc.make_params(16, 48, 7, 2, *SETTING, precision=tc.TC_FP64)
    with tc.Completion(p, wl.to_colmajor(inst["G"], np.float64), wl.to_colmajor(inst["mask"], np.uint8),
                       wl.to_colmajor(inst["Y0"], np.float64)) as c:
        assert c.iterate(7) == 7
        with pytest.raises(tc.TCError) as ei:
            c.convergence()
        assert "TC_ERR_STATE" in str(ei.value)


def test_iterations_after_the_stop_do_no_work():
    # once the test has held, further calls leave the state unchanged
    from paper_2005_09838_gb300 import tc
    w = wl.custom(16, 48, 7, 2, 0.5, seed=4301)
    inst = wl.generate(w)
    p = tc.make_params(16, 48, 7, 2, *SETTING, precision=tc.TC_FP64, eps=1e30)
    with tc.Completion(p, wl.to_colmajor(inst["G"], np.float64), wl.to_colmajor(inst["mask"], np.uint8),
                       wl.to_colmajor(inst["Y0"], np.float64)) as c:
        assert c.iterate(5) == 1
        W1, _, _ = c.result_numpy()
        assert c.iterate(5) == 0
        W2, _, _ = c.result_numpy()
        _, stopped, total = c.convergence()
    assert stopped and total == 1
    assert np.array_equal(W1, W2)
    ref = O.tctf2r(inst["G"], inst["mask"], 2, *SETTING, inst["Y0"], iters=1)
    assert _rel(wl.from_colmajor(W1, (16, 48, 7)), ref["W"]) <= TOL["fp64"]
