"""FP64 CPU oracle for the TCTF2R iteration (test infrastructure only).

This module is the plain, slow, literal statement of what the GPU path must
compute.  It is test infrastructure: only the tests, ``__graft_entry__.smoke``
and the ``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import
it.  It shares no code with the CUDA library (``paper_2005_09838_gb300``);
the two meet only through the seeded inputs of ``workloads``.

Everything is float64 / complex128.  Tensors are numpy arrays indexed
``[i1, i2, i3]`` (paper: m1 x m2 x m3).  Library primitives used as single
steps: matrix products, ``numpy.linalg.eigh`` (Hermitian eigensolver for the
Moore-Penrose inverse), ``numpy.linalg.solve`` / ``scipy.linalg.solve_banded``
(linear solves).  There is no FFT: the mode-3 transform is the direct sum of
Eq. (bar BA-k).

Sections followed (PAPER = arXiv 2005.09838, "A Parallelizable Method for
Missing Internet Traffic Tensor Data"):

* Sec. 2.2, Definition "t-product", Eq. (BDFT), Eq. (bar BA-k),
  Eq. (barAAk), Remark "blockcon" (conjugate symmetry).
* Sec. 3.2, Eq. (Toeplitz) (H and K), Eq. (TETP-optim) (objective f0).
* Sec. 3.3, Eq. (fun-XYW) (slice-separable f0), Eq. (subquKKT), Eq. (Wkiom)
  (W sub-problem).
* Sec. 4.1, Eq. (hkXYDer) (slice gradients), Eq. (KKTcondition),
  Eq. (updataXYW1) (generalized-inverse X/Y updates), the TCTF2R Algorithm
  (steps 1-7) and the half-spectrum remark after it.
* Sec. 4.2, Lemma "SVPMPI" (pseudo-inverse through a unitary
  eigen/singular decomposition).

Readings taken where the paper is silent (listed in the design notes too):

* step size: ``step="exact"`` takes alpha_kl = L_k1 and beta_kl = L_k2, i.e.
  a unit step along d_X / d_Y (exact block minimisation of the quadratic
  h_k); ``step="scaled"`` uses fixed user alpha, beta divided by L_k1, L_k2.
* pseudo-inverse cutoff: eigenvalues lambda <= rtol * lambda_max of the
  Hermitian PSD Gram are treated as zero; rtol defaults to r * 2**-52.
* rank vector (step 5): fixed r for every slice in ``tctf2r``;
  ``tctf2r_rank`` carries out step 5 as a rank decrease: a slice drops the
  directions whose Y-step Gram eigenvalue stayed at or below
  rank_tol * lambda_max for ``patience`` consecutive iterations.
* initial point: W0 = P_Omega(G), X0 given (default 0), Y0 given.
* DFT sign: the paper's omega = exp(+2 pi i / m3); ``sign=-1`` gives the
  other convention (every real output is the same).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.linalg

EPS64 = 2.0 ** -52


# ---------------------------------------------------------------------------
# Sec. 2.2: block-circulant algebra and the mode-3 DFT
# ---------------------------------------------------------------------------

def bcirc(A: np.ndarray) -> np.ndarray:
    """Block-circulant matrix of the frontal slices (Sec. 2.2): block (k, l)
    is A_{(k-l) mod m3}, size m1*m3 x m2*m3."""
    m1, m2, m3 = A.shape
    out = np.zeros((m1 * m3, m2 * m3), dtype=A.dtype)
    for k in range(m3):
        for l in range(m3):
            out[k * m1:(k + 1) * m1, l * m2:(l + 1) * m2] = A[:, :, (k - l) % m3]
    return out


def bvec(A: np.ndarray) -> np.ndarray:
    """Stack the frontal slices vertically: [A_1; A_2; ...; A_m3]."""
    m1, m2, m3 = A.shape
    return np.concatenate([A[:, :, k] for k in range(m3)], axis=0)


def bvfold(M: np.ndarray, m3: int) -> np.ndarray:
    """Inverse of bvec."""
    m1 = M.shape[0] // m3
    return np.stack([M[k * m1:(k + 1) * m1, :] for k in range(m3)], axis=2)


def tprod_definition(A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Definition "t-product": A*B = bvfold(bcirc(A) . bvec(B))."""
    return bvfold(bcirc(A) @ bvec(B), A.shape[2])


def dft_matrix(m3: int, sign: int = +1) -> np.ndarray:
    """Entries omega^((k-1)(l-1)) with omega = exp(sign * 2 pi i / m3)
    (Eq. (bar BA-k), unnormalised)."""
    k = np.arange(m3)
    ang = (2.0 * math.pi / m3) * np.outer(k, k)
    return np.cos(ang) + 1j * sign * np.sin(ang)


def dft3(A: np.ndarray, nslices: int | None = None, sign: int = +1) -> np.ndarray:
    """Eq. (bar BA-k): A~_k = sum_l omega^((k-1)(l-1)) A_l, for the first
    ``nslices`` slices (default all m3).  Direct sum, no FFT."""
    m3 = A.shape[2]
    F = dft_matrix(m3, sign)
    if nslices is not None:
        F = F[:nslices]
    # sum over l of F[k, l] * A[:, :, l]
    return np.tensordot(A, F, axes=([2], [1]))


def idft3(At: np.ndarray, sign: int = +1) -> np.ndarray:
    """Eq. (barAAk): A_k = (1/m3) sum_l conj(omega)^((k-1)(l-1)) A~_l over all
    m3 slices (complex result; real iff Remark "blockcon" symmetry holds)."""
    m3 = At.shape[2]
    Fc = np.conj(dft_matrix(m3, sign))
    return np.tensordot(At, Fc, axes=([2], [1])) / m3


def mirror_half(half: np.ndarray, m3: int) -> np.ndarray:
    """Complete a half spectrum (slices 1..floor(m3/2)+1) by the conjugate
    relation A~_k = conj(A~_{m3-k+2}) (Remark "blockcon", end of Sec. 4.1)."""
    S = m3 // 2 + 1
    full = np.zeros(half.shape[:2] + (m3,), dtype=np.complex128)
    full[:, :, :S] = half[:, :, :S]
    for k in range(S, m3):
        full[:, :, k] = np.conj(half[:, :, m3 - k])
    return full


def tprod(A: np.ndarray, B: np.ndarray, sign: int = +1) -> np.ndarray:
    """t-product through the block diagonalisation Eq. (BDFT): C~_k = A~_k B~_k
    for every slice, then Eq. (barAAk)."""
    At, Bt = dft3(A, sign=sign), dft3(B, sign=sign)
    Ct = np.einsum("isk,sjk->ijk", At, Bt)
    C = idft3(Ct, sign=sign)
    return C.real


# ---------------------------------------------------------------------------
# Sec. 3.2: the difference operators H, K and the objective f0
# ---------------------------------------------------------------------------

def toeplitz_D(m: int) -> np.ndarray:
    """Eq. (Toeplitz): (m-1) x m matrix with ones on the diagonal and -1 on
    the first upper diagonal."""
    D = np.zeros((m - 1, m))
    for i in range(m - 1):
        D[i, i] = 1.0
        D[i, i + 1] = -1.0
    return D


def H_rho(m1: int, rho1: float) -> np.ndarray:
    """H_rho1 = I + rho1 H^T H (Eq. (KKTcondition))."""
    H = toeplitz_D(m1)
    return np.eye(m1) + rho1 * (H.T @ H)


def K_murho(m2: int, mu: float, rho2: float) -> np.ndarray:
    """K_{mu rho2} = (1 + mu) I + rho2 K^T K (Eq. (subquKKT))."""
    K = toeplitz_D(m2)
    return (1.0 + mu) * np.eye(m2) + rho2 * (K.T @ K)


def unfold(A: np.ndarray, mode: int) -> np.ndarray:
    """Mode-k unfolding of Sec. 2.1 (first index fastest): unfold(A,1) =
    [A_1, ..., A_m3], unfold(A,2) = [A_1^T, ..., A_m3^T]."""
    m1, m2, m3 = A.shape
    if mode == 1:
        return np.concatenate([A[:, :, k] for k in range(m3)], axis=1)
    if mode == 2:
        return np.concatenate([A[:, :, k].T for k in range(m3)], axis=1)
    raise ValueError(mode)


def objective(X, Y, W, mu, rho1, rho2, sign: int = +1) -> float:
    """f0 of Eq. (TETP-optim), spatial form."""
    Z = tprod(X, Y, sign=sign)
    m1, m2, _ = W.shape
    H, K = toeplitz_D(m1), toeplitz_D(m2)
    f = 0.5 * np.sum((Z - W) ** 2) + 0.5 * mu * np.sum(W ** 2)
    if m1 > 1:
        f += 0.5 * rho1 * np.sum((H @ unfold(Z, 1)) ** 2)
    if m2 > 1:
        f += 0.5 * rho2 * np.sum((K @ unfold(W, 2)) ** 2)
    return float(f)


def objective_freq(Xt, Yt, Wt, mu, rho1, rho2) -> float:
    """f0 in the slice-separable form Eq. (fun-XYW); every argument holds all
    m3 slices."""
    m1, m2, m3 = Wt.shape
    H, K = toeplitz_D(m1), toeplitz_D(m2)
    f = 0.0
    for k in range(m3):
        Zk = Xt[:, :, k] @ Yt[:, :, k]
        Wk = Wt[:, :, k]
        f += np.sum(np.abs(Zk - Wk) ** 2) + mu * np.sum(np.abs(Wk) ** 2)
        if m1 > 1:
            f += rho1 * np.sum(np.abs(H @ Zk) ** 2)
        if m2 > 1:
            f += rho2 * np.sum(np.abs(Wk @ K.T) ** 2)
    return float(f / (2.0 * m3))


# ---------------------------------------------------------------------------
# Lemma "SVPMPI": Moore-Penrose inverse of a Hermitian PSD Gram
# ---------------------------------------------------------------------------

def default_rtol(r: int) -> float:
    return r * EPS64


def pinv_herm(A: np.ndarray, rtol: float | None = None) -> np.ndarray:
    """A^+ = V diag(1/lambda) V^* over the eigenvalues above the cutoff
    rtol * lambda_max (Lemma "SVPMPI" applied to a Hermitian PSD matrix,
    whose SVD is its eigendecomposition)."""
    r = A.shape[0]
    rtol = default_rtol(r) if rtol is None or rtol <= 0 else rtol
    Ah = 0.5 * (A + A.conj().T)
    lam, V = np.linalg.eigh(Ah)
    lmax = float(np.max(lam)) if lam.size else 0.0
    if lmax <= 0.0:
        return np.zeros_like(Ah)
    keep = lam > rtol * lmax
    inv = np.where(keep, 1.0 / np.where(keep, lam, 1.0), 0.0)
    return (V * inv[None, :]) @ V.conj().T


# ---------------------------------------------------------------------------
# Sec. 4.1: slice gradients and the generalized-inverse updates
# ---------------------------------------------------------------------------

def grad_X(Xk, Yk, Wk, rho1):
    """Eq. (hkXYDer), first line."""
    m1 = Xk.shape[0]
    HtH = toeplitz_D(m1).T @ toeplitz_D(m1) if m1 > 1 else np.zeros((1, 1))
    Zk = Xk @ Yk
    YYh = Yk @ Yk.conj().T
    return (Zk - Wk) @ Yk.conj().T + rho1 * (HtH @ Xk @ YYh)


def grad_Y(Xk, Yk, Wk, rho1):
    """Eq. (hkXYDer), second line."""
    m1 = Xk.shape[0]
    HtH = toeplitz_D(m1).T @ toeplitz_D(m1) if m1 > 1 else np.zeros((1, 1))
    Zk = Xk @ Yk
    return Xk.conj().T @ (Zk - Wk) + rho1 * (Xk.conj().T @ HtH @ Xk @ Yk)


def x_update(Xk, Yk, Wk, rho1, step="exact", alpha=1.0, rtol=None):
    """First line of Eq. (updataXYW1): X <- X + (alpha/L1) d_X with
    d_X = -H_rho1^{-1} grad_X (Y Y^*)^+ and L1 = ||H_rho1||_2 ||Y Y^*||_2."""
    m1 = Xk.shape[0]
    Hr = H_rho(m1, rho1)
    A = Yk @ Yk.conj().T
    Ap = pinv_herm(A, rtol)
    dX = -np.linalg.solve(Hr, grad_X(Xk, Yk, Wk, rho1)) @ Ap
    if step == "exact":
        t = 1.0
    else:
        L1 = np.linalg.norm(Hr, 2) * np.linalg.norm(A, 2)
        t = alpha / L1 if L1 > 0 else 0.0
    return Xk + t * dX


def y_update(Xk, Yk, Wk, rho1, step="exact", beta=1.0, rtol=None):
    """Second line of Eq. (updataXYW1) with the new X: Y <- Y + (beta/L2) d_Y,
    d_Y = -(X^* H_rho1 X)^+ grad_Y and L2 = ||X^* H_rho1 X||_2."""
    m1 = Xk.shape[0]
    Hr = H_rho(m1, rho1)
    Gx = Xk.conj().T @ Hr @ Xk
    Gp = pinv_herm(Gx, rtol)
    dY = -Gp @ grad_Y(Xk, Yk, Wk, rho1)
    if step == "exact":
        t = 1.0
    else:
        L2 = np.linalg.norm(Gx, 2)
        t = beta / L2 if L2 > 0 else 0.0
    return Yk + t * dY


# ---------------------------------------------------------------------------
# Sec. 3.3: the W sub-problem
# ---------------------------------------------------------------------------

def w_step_dense(Z, G, mask, mu, rho2):
    """Eq. (Wkiom) row by row: for each (i, k) with missing set C and observed
    set O, W_iC = (Z_iC - rho2 G_iO K1^T K2) ((1+mu) I + rho2 K2^T K2)^{-1},
    W_iO = G_iO, with K = [K1, K2] split by columns.  Dense solves."""
    m1, m2, m3 = Z.shape
    K = toeplitz_D(m2) if m2 > 1 else np.zeros((0, 1))
    W = np.where(mask, G, 0.0).astype(np.float64)
    for k in range(m3):
        for i in range(m1):
            obs = mask[i, :, k]
            C = np.flatnonzero(~obs)
            O = np.flatnonzero(obs)
            if C.size == 0:
                continue
            K1, K2 = K[:, O], K[:, C]
            rhs = Z[i, C, k] - rho2 * (G[i, O, k] @ K1.T @ K2)
            Amat = (1.0 + mu) * np.eye(C.size) + rho2 * (K2.T @ K2)
            # row vector w_C with w_C Amat = rhs; Amat is symmetric
            W[i, C, k] = np.linalg.solve(Amat, rhs)
    return W


def w_step_kkt(Z, G, mask, mu, rho2):
    """Eq. (subquKKT) solved as one banded system per (i, k) row:
    (W_k K_{mu rho2})_ij = (Z_k)_ij for missing (i,j), W_ij = G_ij for observed.
    K_{mu rho2} is tridiagonal, so every row is a tridiagonal system; all rows
    are stacked into one block-diagonal banded system (scipy solve_banded)."""
    m1, m2, m3 = Z.shape
    Kmr = K_murho(m2, mu, rho2)
    diag = np.diag(Kmr)
    off = np.diag(Kmr, 1) if m2 > 1 else np.zeros(0)
    # rows of the system ordered (k, i, j) with j fastest
    obs = np.transpose(mask, (2, 0, 1)).reshape(-1, m2)
    g = np.transpose(G, (2, 0, 1)).reshape(-1, m2)
    z = np.transpose(Z, (2, 0, 1)).reshape(-1, m2)
    nrow = obs.shape[0]
    # (w K)_j = sum_m w_m K[m, j]: sub-diagonal coefficient K[j-1, j], super K[j+1, j]
    sub = np.zeros((nrow, m2))
    sup = np.zeros((nrow, m2))
    dia = np.broadcast_to(diag, (nrow, m2)).copy()
    if m2 > 1:
        sub[:, 1:] = off[None, :]
        sup[:, :-1] = off[None, :]
    rhs = z.copy()
    dia[obs] = 1.0
    sub[obs] = 0.0
    sup[obs] = 0.0
    rhs[obs] = g[obs]
    # banded storage for scipy: ab[0, 1:] super, ab[1] diag, ab[2, :-1] sub
    n = nrow * m2
    ab = np.zeros((3, n))
    ab[1] = dia.reshape(-1)
    supf = sup.reshape(-1)
    subf = sub.reshape(-1)
    ab[0, 1:] = supf[:-1]
    ab[2, :-1] = subf[1:]
    w = scipy.linalg.solve_banded((1, 1), ab, rhs.reshape(-1))
    return np.transpose(w.reshape(m3, m1, m2), (1, 2, 0))


# ---------------------------------------------------------------------------
# The TCTF2R Algorithm (Sec. 4.1)
# ---------------------------------------------------------------------------

def tctf2r(G, mask, r, mu, rho1, rho2, Y0, X0=None, iters=10, step="exact",
           alpha=1.0, beta=1.0, rtol=None, half=True, sign=+1,
           wstep="kkt", record=False, eps=0.0):
    """Run ``iters`` iterations of the TCTF2R Algorithm.

    Steps per iteration l (Sec. 4.1): 1. X-update of every slice with Y, W
    fixed; 2. Y-update of every slice with the new X; 3. Z~ = X~ Y~ and Z by
    Eq. (barAAk); 4. W-update (Eq. (subquKKT)); 7. W~ by Eq. (bar BA-k).
    With ``half`` only floor(m3/2)+1 slices are solved and the rest mirrored
    (remark after the algorithm).  Step 5 keeps r fixed.  Step 6: with
    ``eps`` > 0 the loop ends after the first iteration with
    ||X~' - X~||_inf <= eps, ||Y~' - Y~||_inf <= eps and ||W' - W||_F <= eps
    (||.||_inf: largest modulus of an entry), else it runs ``iters`` times.

    Returns a dict with W, Z, X, Y (spatial), Xt, Yt (all slices), f0, the
    number of iterations run and, with ``record``, per-iteration histories.
    """
    G = np.asarray(G, dtype=np.float64)
    mask = np.asarray(mask, dtype=bool)
    m1, m2, m3 = G.shape
    S = m3 // 2 + 1 if half else m3
    X0 = np.zeros((m1, r, m3)) if X0 is None else np.asarray(X0, np.float64)
    W = np.where(mask, G, 0.0)
    Wt = dft3(W, sign=sign)
    Xt = dft3(X0, sign=sign)
    Yt = dft3(np.asarray(Y0, np.float64), sign=sign)
    hist = {"f0": [], "f0_after_x": [], "f0_after_y": [], "dX": [], "dY": [], "dW": []}
    run = 0
    for _ in range(iters):
        Xold, Yold, Wold = Xt.copy(), Yt.copy(), W.copy()
        Xn = np.zeros_like(Xt)
        for k in range(S):
            Xn[:, :, k] = x_update(Xt[:, :, k], Yt[:, :, k], Wt[:, :, k], rho1, step, alpha, rtol)
        Xt = mirror_half(Xn, m3) if half else Xn
        if record:
            hist["f0_after_x"].append(objective_freq(Xt, Yt, Wt, mu, rho1, rho2))
        Yn = np.zeros_like(Yt)
        for k in range(S):
            Yn[:, :, k] = y_update(Xt[:, :, k], Yt[:, :, k], Wt[:, :, k], rho1, step, beta, rtol)
        Yt = mirror_half(Yn, m3) if half else Yn
        if record:
            hist["f0_after_y"].append(objective_freq(Xt, Yt, Wt, mu, rho1, rho2))
        Zt = np.einsum("isk,sjk->ijk", Xt, Yt)
        Zc = idft3(Zt, sign=sign)
        zscale = max(1.0, float(np.max(np.abs(Zc))))
        if np.max(np.abs(Zc.imag)) > 1e-9 * zscale:
            raise AssertionError("inverse DFT of a conjugate-symmetric spectrum is not real")
        Z = Zc.real
        if wstep == "dense":
            W = w_step_dense(Z, G, mask, mu, rho2)
        else:
            W = w_step_kkt(Z, G, mask, mu, rho2)
        Wt = dft3(W, sign=sign)
        run += 1
        dX = float(np.max(np.abs(Xt - Xold)))
        dY = float(np.max(np.abs(Yt - Yold)))
        dW = float(np.linalg.norm(W - Wold))
        if record:
            hist["f0"].append(objective_freq(Xt, Yt, Wt, mu, rho1, rho2))
            hist["dX"].append(dX)
            hist["dY"].append(dY)
            hist["dW"].append(dW)
        if eps > 0 and dX <= eps and dY <= eps and dW <= eps:
            break
    X = idft3(Xt, sign=sign).real
    Y = idft3(Yt, sign=sign).real
    Z = tprod(X, Y, sign=sign)
    out = {"W": W, "Z": Z, "X": X, "Y": Y, "Xt": Xt, "Yt": Yt, "Wt": Wt,
           "f0": objective(X, Y, W, mu, rho1, rho2, sign=sign)}
    out["resid_obs"] = float(np.sqrt(np.sum(((Z - G) * mask) ** 2)))
    out["iters"] = run
    if record:
        out["hist"] = hist
    return out


# ---------------------------------------------------------------------------
# Step 5 of the TCTF2R Algorithm: the rank vector (reading of this build)
# ---------------------------------------------------------------------------

def rank_adjust_slice(Xk, Yk, rho1, tol):
    """One rank decrease of slice k (step 5 reading): the eigendecomposition
    G = V diag(lambda) V^* of G = X~_k^* H_rho1 X~_k; the directions with
    lambda <= tol * lambda_max are dropped, X~_k <- X~_k V_keep and
    Y~_k <- V_keep^* Y~_k (the sizes of X~_k and Y~_k shrink to the kept count).
    Returns (X, Y, dropped)."""
    m1 = Xk.shape[0]
    Gx = Xk.conj().T @ H_rho(m1, rho1) @ Xk
    lam, V = np.linalg.eigh(0.5 * (Gx + Gx.conj().T))
    lmax = float(lam.max()) if lam.size else 0.0
    keep = lam > tol * lmax
    if keep.all() or not keep.any():
        return Xk, Yk, 0
    Vk = V[:, keep]
    return Xk @ Vk, Vk.conj().T @ Yk, int((~keep).sum())


def tctf2r_rank(G, mask, r, mu, rho1, rho2, Y0, X0=None, iters=10, rank_tol=0.0, patience=1, rtol=None,
                sign=+1):
    """The TCTF2R Algorithm with step 5 carried out (exact steps).

    Reading of step 5 ("adjust the rank vector and the sizes of X~_k, Y~_k"):
    after the W-update of iteration l, every solved slice k checks the
    eigenvalues of its Y-step Gram G_k = X~_k^* H_rho1 X~_k; when at least one
    of them has been <= rank_tol * lambda_max(G_k) for ``patience`` consecutive
    iterations, those directions are dropped (rank_adjust_slice) and the count
    restarts.  W~ is not changed by the step.  Slices k > floor(m3/2) follow
    by the conjugate relation, so r_k = r_{m3-k+2}.  The factors are kept as
    one matrix per slice, of width r_k.

    Returns a dict with W, f0 (the objective of the final iterate) and the
    rank vector of all m3 slices."""
    G = np.asarray(G, dtype=np.float64)
    mask = np.asarray(mask, dtype=bool)
    m1, m2, m3 = G.shape
    S = m3 // 2 + 1
    X0 = np.zeros((m1, r, m3)) if X0 is None else np.asarray(X0, np.float64)
    W = np.where(mask, G, 0.0)
    Wt = dft3(W, sign=sign)
    X0t, Y0t = dft3(X0, sign=sign), dft3(np.asarray(Y0, np.float64), sign=sign)
    Xs = [X0t[:, :, k].copy() for k in range(S)]
    Ys = [Y0t[:, :, k].copy() for k in range(S)]
    count = [0] * S
    for _ in range(iters):
        for k in range(S):                                            # step 1
            Xs[k] = x_update(Xs[k], Ys[k], Wt[:, :, k], rho1, rtol=rtol)
        for k in range(S):                                            # step 2
            Ys[k] = y_update(Xs[k], Ys[k], Wt[:, :, k], rho1, rtol=rtol)
        Zt = np.zeros((m1, m2, m3), dtype=np.complex128)              # step 3
        for k in range(S):
            Zt[:, :, k] = Xs[k] @ Ys[k]
        Zt = mirror_half(Zt[:, :, :S], m3)
        Z = idft3(Zt, sign=sign).real
        W = w_step_kkt(Z, G, mask, mu, rho2)                          # step 4
        if rank_tol > 0:                                              # step 5
            for k in range(S):
                m = Xs[k].shape[0]
                Gx = Xs[k].conj().T @ H_rho(m, rho1) @ Xs[k]
                lam = np.linalg.eigvalsh(0.5 * (Gx + Gx.conj().T))
                small = lam.size > 1 and bool(np.any(lam <= rank_tol * lam.max()))
                count[k] = count[k] + 1 if small else 0
                if count[k] >= patience:
                    Xs[k], Ys[k], _ = rank_adjust_slice(Xs[k], Ys[k], rho1, rank_tol)
                    count[k] = 0
        Wt = dft3(W, sign=sign)                                       # step 7
    ranks = [Xs[k].shape[1] for k in range(S)]
    full = ranks + [ranks[m3 - k] for k in range(S, m3)]
    # f0 of the final iterate: X*Y from the slices (mirrored), W
    Zt = np.zeros((m1, m2, m3), dtype=np.complex128)
    for k in range(S):
        Zt[:, :, k] = Xs[k] @ Ys[k]
    Z = idft3(mirror_half(Zt[:, :, :S], m3), sign=sign).real
    Hd, Kd = toeplitz_D(m1), toeplitz_D(m2)
    f = 0.5 * np.sum((Z - W) ** 2) + 0.5 * mu * np.sum(W ** 2)
    if m1 > 1:
        f += 0.5 * rho1 * np.sum((Hd @ unfold(Z, 1)) ** 2)
    if m2 > 1:
        f += 0.5 * rho2 * np.sum((Kd @ unfold(W, 2)) ** 2)
    return {"W": W, "Z": Z, "f0": float(f), "ranks": full}


# ---------------------------------------------------------------------------
# Differentiation form: the factor terms of f0 as a loss of (X, Y)
# ---------------------------------------------------------------------------

def ttranspose(A: np.ndarray) -> np.ndarray:
    """Conjugate transpose A^* of a real third-order tensor (Sec. 2, after
    Definition "T-ProdDef"): every frontal slice transposed, the order of
    frontal slices 2..m3 reversed."""
    At = np.transpose(np.asarray(A), (1, 0, 2))
    return np.concatenate([At[:, :, :1], At[:, :, :0:-1]], axis=2)


def factor_loss(X, Y, G, mask, rho1) -> float:
    """L(X, Y) = 1/2 ||P_Omega(X*Y - G)||_F^2 + rho1/2 ||H unfold(X*Y, 1)||_F^2:
    the terms of f0 (Eq. (TETP-optim)) that involve the factors, with W held at
    G on the mask."""
    Z = tprod(X, Y)
    m1 = Z.shape[0]
    R = np.where(mask, Z - G, 0.0)
    f = 0.5 * np.sum(R ** 2)
    if m1 > 1:
        f += 0.5 * rho1 * np.sum((toeplitz_D(m1) @ unfold(Z, 1)) ** 2)
    return float(f)


def factor_loss_grad(X, Y, G, mask, rho1):
    """Gradients of factor_loss.  With E = P_Omega(X*Y - G) + rho1 (H^T H) x_1
    (X*Y), the gradient with respect to Z = X*Y, they are dL/dX = E * Y^* and
    dL/dY = X^* * E (t-products with the conjugate transpose)."""
    Z = tprod(X, Y)
    m1 = Z.shape[0]
    E = np.where(mask, Z - G, 0.0)
    if m1 > 1:
        D = toeplitz_D(m1)
        E = E + rho1 * np.einsum("ab,bjk->ajk", D.T @ D, Z)
    return tprod(E, ttranspose(Y)), tprod(ttranspose(X), E)
