"""Differentiation form on the GPU: loss and adjoint of the factor model
L(X, Y) = 1/2 ||P_Omega(X*Y - G)||_F^2 + rho1/2 ||H unfold(X*Y, 1)||_F^2
against the oracle's loss and gradient (itself pinned by central differences),
central differences of the GPU loss (h = 1e-3, FP64, 12 x 24 x 8), the
torch.autograd face and block gradient descent.
"""
import numpy as np
import pytest

import workloads as wl
from oracle import method as O

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32": 1e-5}


C4_RHO1 = 1e-3


@pytest.fixture(scope="module", autouse=True)
def _built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2005_09838_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def c4_oracle():
    # the oracle's loss and gradients at the 529 x 288 x 168 initial factors, in a
    # spawned worker (about a minute of CPU work)
    import _oracle_jobs
    pool, fut = _oracle_jobs.start_c4_loss_grad(C4_RHO1)
    yield fut
    pool.shutdown(cancel_futures=True)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(shape, r, obs, seed, precision):
    w = wl.custom(*shape, r, obs, seed=seed)
    inst = wl.generate(w)
    rng = np.random.default_rng(seed + 1)
    X = rng.standard_normal((shape[0], r, shape[2]))
    Y = inst["Y0"]
    G, mask = inst["G"], inst["mask"]
    if precision == "fp32":
        X, Y, G = (a.astype(np.float32).astype(np.float64) for a in (X, Y, G))
    return X, Y, G, mask


def _gpu(shape, r, X, Y, G, mask, rho1, precision, want_grad=True):
    from paper_2005_09838_gb300 import tc
    dt = np.float64 if precision == "fp64" else np.float32
    n1, n2, n3 = shape
    p = tc.make_params(n1, n2, n3, r, rho1=rho1, precision=tc.TC_FP64 if precision == "fp64" else tc.TC_FP32)
    with tc.GradContext(p, wl.to_colmajor(G, dt), wl.to_colmajor(mask, np.uint8)) as g:
        dX = np.empty(n1 * r * n3, dt) if want_grad else None
        dY = np.empty(r * n2 * n3, dt) if want_grad else None
        loss = g.eval(wl.to_colmajor(X, dt), wl.to_colmajor(Y, dt), dX, dY)
    if not want_grad:
        return loss, None, None
    return loss, wl.from_colmajor(dX, (n1, r, n3)).astype(np.float64), \
        wl.from_colmajor(dY, (r, n2, n3)).astype(np.float64)


@pytest.mark.parametrize("precision,shape,r", [
    ("fp64", (12, 24, 8), 3),      # generic transform
    ("fp64", (16, 48, 7), 2),      # register transform, n3 = 7
    ("fp32", (20, 40, 112), 4),    # shared-memory transform, n3 = 112
    ("fp32", (24, 36, 168), 8),    # shared-memory transform, n3 = 168
    ("fp32", (9, 30, 12), 3),      # generic transform, FP32
])
@pytest.mark.parametrize("rho1", [0.0, 0.3])
def test_loss_and_gradient_match_oracle(precision, shape, r, rho1):
    X, Y, G, mask = _case(shape, r, 0.3, 5000 + shape[2] + r, precision)
    f_ref = O.factor_loss(X, Y, G, mask, rho1)
    gX_ref, gY_ref = O.factor_loss_grad(X, Y, G, mask, rho1)
    f, gX, gY = _gpu(shape, r, X, Y, G, mask, rho1, precision)
    assert abs(f - f_ref) <= TOL[precision] * abs(f_ref)
    assert _rel(gX, gX_ref) <= TOL[precision]
    assert _rel(gY, gY_ref) <= TOL[precision]


def test_gradient_matches_central_differences_of_the_gpu_loss():
    # h = 1e-3, FP64, 12 x 24 x 8: L is quadratic in each single entry, so the
    # central difference of the GPU loss equals the partial derivative
    shape, r, rho1 = (12, 24, 8), 3, 0.3
    X, Y, G, mask = _case(shape, r, 0.3, 5100, "fp64")
    _, gX, gY = _gpu(shape, r, X, Y, G, mask, rho1, "fp64")
    h = 1e-3
    rng = np.random.default_rng(9)
    for A, g in ((X, gX), (Y, gY)):
        for _ in range(6):
            idx = tuple(int(rng.integers(0, n)) for n in A.shape)
            old = A[idx]
            A[idx] = old + h
            fp = _gpu(shape, r, X, Y, G, mask, rho1, "fp64", want_grad=False)[0]
            A[idx] = old - h
            fm = _gpu(shape, r, X, Y, G, mask, rho1, "fp64", want_grad=False)[0]
            A[idx] = old
            assert abs((fp - fm) / (2 * h) - g[idx]) <= 1e-7 * max(1.0, abs(g[idx]))


def test_autograd_function_and_block_gradient_descent():
    import torch
    from paper_2005_09838_gb300 import autograd as ag
    shape, r, rho1 = (20, 40, 112), 4, 1e-3
    X, Y, G, mask = _case(shape, r, 0.3, 5200, "fp32")
    g = ag.grad_context(G, mask, r, rho1, dtype=torch.float32)
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda", requires_grad=True)
    Yt = torch.tensor(Y, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = ag.factor_loss(Xt, Yt, g)
    loss.backward()
    gX_ref, gY_ref = O.factor_loss_grad(X, Y, G, mask, rho1)
    assert _rel(Xt.grad.cpu().numpy().astype(np.float64), gX_ref) <= TOL["fp32"]
    assert _rel(Yt.grad.cpu().numpy().astype(np.float64), gY_ref) <= TOL["fp32"]
    f_ref = O.factor_loss(X, Y, G, mask, rho1)
    assert abs(float(loss.detach()) - f_ref) <= 1e-5 * f_ref
    # block gradient descent (backtracking from 1/L of the initial factors): the
    # loss decreases at every block step and ends well below the start
    Yt_f = np.fft.fft(Y, axis=2)
    Xt_f = np.fft.fft(X, axis=2)
    Ly = max(np.linalg.norm(Yt_f[:, :, k] @ Yt_f[:, :, k].conj().T, 2) for k in range(shape[2]))
    Lx = max(np.linalg.norm(Xt_f[:, :, k].conj().T @ Xt_f[:, :, k], 2) for k in range(shape[2]))
    X1, Y1, hist = ag.block_gradient_descent(g, torch.tensor(X, dtype=torch.float32, device="cuda"),
                                             torch.tensor(Y, dtype=torch.float32, device="cuda"), 6,
                                             1.0 / Ly, 1.0 / Lx)
    assert all(b < a for a, b in zip(hist, hist[1:]))
    assert hist[-1] < 0.5 * hist[0]
    g.close()


def test_differentiation_form_c4_first_evaluation_and_block_descent(c4_oracle):
    # the differentiation form's own workload: 529 x 288 x 168, r = 16, 20%
    # observed, FP32.  The loss and both gradients at the initial factors against
    # the oracle; then block gradient descent through torch.autograd, whose loss
    # falls at every accepted block step
    import torch
    import _oracle_jobs
    from paper_2005_09838_gb300 import autograd as ag
    w, inst, X = _oracle_jobs.c4_inputs()
    Y = inst["Y0"]
    g = ag.grad_context(inst["G"], inst["mask"], w.r, C4_RHO1, dtype=torch.float32)
    Xt = torch.tensor(X, dtype=torch.float32, device="cuda", requires_grad=True)
    Yt = torch.tensor(Y, dtype=torch.float32, device="cuda", requires_grad=True)
    loss = ag.factor_loss(Xt, Yt, g)
    loss.backward()
    ref = c4_oracle.result()
    err_f = abs(float(loss.detach()) - ref["f"]) / ref["f"]
    err_x = _rel(Xt.grad.cpu().numpy().astype(np.float64), ref["gX"])
    err_y = _rel(Yt.grad.cpu().numpy().astype(np.float64), ref["gY"])
    print(f"C4 loss {err_f:.2e}, dL/dX {err_x:.2e}, dL/dY {err_y:.2e}")
    assert err_f <= TOL["fp32"]
    assert err_x <= TOL["fp32"]
    assert err_y <= TOL["fp32"]
    # steps from 1/L of the initial factors (L over the slices of the block's Gram)
    Xf, Yf = np.fft.fft(X, axis=2), np.fft.fft(Y, axis=2)
    Ly = max(np.linalg.norm(Yf[:, :, k] @ Yf[:, :, k].conj().T, 2) for k in range(w.n3))
    Lx = max(np.linalg.norm(Xf[:, :, k].conj().T @ Xf[:, :, k], 2) for k in range(w.n3))
    X1, Y1, hist = ag.block_gradient_descent(g, Xt.detach(), Yt.detach(), 2, 1.0 / Ly, 1.0 / Lx)
    assert all(b < a for a, b in zip(hist, hist[1:]))
    g.close()
