"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these tests re-types an oracle formula: each checks the oracle
against a printed example (tests/golden), a library routine run on a
different route, a closed form, an invariant proved in the paper, or brute
force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest
import scipy.optimize

import workloads as wl
from oracle import method as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _rng(seed=0):
    return np.random.default_rng(seed)


# --------------------------------------------------------------------------
# Sec. 2.2 / 3.2 printed matrices
# --------------------------------------------------------------------------

def test_toeplitz_matches_printed_H():
    # Eq. (Toeplitz)
    np.testing.assert_array_equal(O.toeplitz_D(5), _load("toeplitz_H_m5.txt"))


def test_dtd_matches_printed_matrix_and_spectrum_bounds():
    # Proposition "KKProp": printed D^T D, lambda_min = 0, lambda_max <= 4
    D = O.toeplitz_D(6)
    np.testing.assert_array_equal(D.T @ D, _load("dtd_m6.txt"))
    for m in (2, 3, 7, 48, 144):
        D = O.toeplitz_D(m)
        lam = np.linalg.eigvalsh(D.T @ D)
        # closed form of the path-graph Laplacian: 2 - 2 cos(pi j / m)
        closed = np.sort(2.0 - 2.0 * np.cos(math.pi * np.arange(m) / m))
        np.testing.assert_allclose(np.sort(lam), closed, atol=1e-12)
        assert abs(lam.min()) < 1e-12 and lam.max() <= 4.0


def test_bcirc_block_pattern_matches_printed_layout():
    m1, m2, m3 = 2, 3, 5
    A = np.zeros((m1, m2, m3))
    for j in range(m3):
        A[:, :, j] = j + 1  # slice j (0-based) filled with its 1-based number
    B = O.bcirc(A)
    blocks = np.array([[B[k * m1, l * m2] for l in range(m3)] for k in range(m3)])
    np.testing.assert_array_equal(blocks, _load("bcirc_blocks_m3_5.txt"))


# --------------------------------------------------------------------------
# Sec. 2.2: DFT, t-product, conjugate symmetry
# --------------------------------------------------------------------------

@pytest.mark.parametrize("m3", [1, 2, 5, 7, 8])
def test_dft3_against_numpy_fft(m3):
    A = _rng(m3).standard_normal((3, 4, m3))
    # omega = exp(+2 pi i / m3): sum_l omega^(kl) A_l = m3 * ifft(A)_k
    np.testing.assert_allclose(O.dft3(A), m3 * np.fft.ifft(A, axis=2), atol=1e-12)
    np.testing.assert_allclose(O.dft3(A, sign=-1), np.fft.fft(A, axis=2), atol=1e-12)
    np.testing.assert_allclose(O.idft3(O.dft3(A)).real, A, atol=1e-12)


def test_orthogonality_sum_lsm3():
    # Eq. (lsm3): sum_k omega^{(k)(l)} conj(omega)^{(k)(s)} = m3 delta_ls
    for m3 in (3, 6, 7):
        F = O.dft_matrix(m3)
        np.testing.assert_allclose(F.T @ np.conj(F), m3 * np.eye(m3), atol=1e-12)


@pytest.mark.parametrize("m3", [1, 4, 5, 7])
def test_tproduct_slices_equal_bcirc_definition(m3):
    rng = _rng(10 + m3)
    A = rng.standard_normal((4, 3, m3))
    B = rng.standard_normal((3, 5, m3))
    np.testing.assert_allclose(O.tprod(A, B), O.tprod_definition(A, B), rtol=1e-13, atol=1e-13)
    # Eq. (BDFT): (F (x) I) bcirc(A) (F^* (x) I) is block diagonal with A~_k
    F = O.dft_matrix(m3) / math.sqrt(m3)
    L = np.kron(F, np.eye(4)) @ O.bcirc(A) @ np.kron(np.conj(F).T, np.eye(3))
    At = O.dft3(A)
    for k in range(m3):
        np.testing.assert_allclose(L[4 * k:4 * k + 4, 3 * k:3 * k + 3], At[:, :, k], atol=1e-12)


@pytest.mark.parametrize("m3", [6, 7])
def test_conjugate_symmetry_of_real_spectrum(m3):
    # Eq. (rcm_3-k+2): A~_1 real, A~_k = conj(A~_{m3-k+2})
    A = _rng(3).standard_normal((3, 4, m3))
    At = O.dft3(A)
    assert np.max(np.abs(At[:, :, 0].imag)) < 1e-12
    for k in range(1, m3):
        np.testing.assert_allclose(At[:, :, k], np.conj(At[:, :, m3 - k]), atol=1e-12)
    np.testing.assert_allclose(O.mirror_half(At[:, :, : m3 // 2 + 1], m3), At, atol=1e-12)


def test_tubal_rank_of_generated_truth():
    # Proposition "tubrank": rank_t(A*B) <= r; every DFT slice of the generated
    # truth has rank <= r
    w = wl.custom(12, 20, 6, 3, 0.5, 99)
    inst = wl.generate(w)
    Tt = O.dft3(inst["T"])
    for k in range(w.n3):
        sv = np.linalg.svd(Tt[:, :, k], compute_uv=False)
        assert sv[w.r] < 1e-10 * sv[0]


# --------------------------------------------------------------------------
# Sec. 3.3: Parseval form of f0
# --------------------------------------------------------------------------

def test_objective_spatial_equals_frequency_form():
    rng = _rng(5)
    m1, m2, m3, r = 6, 7, 5, 2
    X = rng.standard_normal((m1, r, m3))
    Y = rng.standard_normal((r, m2, m3))
    W = rng.standard_normal((m1, m2, m3))
    mu, rho1, rho2 = 0.3, 0.7, 1.1
    f_sp = O.objective(X, Y, W, mu, rho1, rho2)
    f_fr = O.objective_freq(O.dft3(X), O.dft3(Y), O.dft3(W), mu, rho1, rho2)
    assert abs(f_sp - f_fr) < 1e-11 * abs(f_sp)
    # brute-force spatial form: explicit sums of squared neighbour differences
    Z = O.tprod_definition(X, Y)
    brute = 0.5 * np.sum((Z - W) ** 2) + 0.5 * mu * np.sum(W ** 2)
    brute += 0.5 * rho1 * np.sum((Z[:-1, :, :] - Z[1:, :, :]) ** 2)
    brute += 0.5 * rho2 * np.sum((W[:, :-1, :] - W[:, 1:, :]) ** 2)
    assert abs(f_sp - brute) < 1e-11 * abs(brute)


# --------------------------------------------------------------------------
# Lemma "SVPMPI": pseudo-inverse
# --------------------------------------------------------------------------

@pytest.mark.parametrize("rank", [1, 3, 5])
def test_pinv_penrose_conditions(rank):
    rng = _rng(rank)
    r = 5
    F = rng.standard_normal((r, rank)) + 1j * rng.standard_normal((r, rank))
    A = F @ F.conj().T
    P = O.pinv_herm(A)
    scale = np.linalg.norm(A) * np.linalg.norm(P)
    assert np.linalg.norm(A @ P @ A - A) < 1e-12 * scale * np.linalg.norm(A)
    assert np.linalg.norm(P @ A @ P - P) < 1e-12 * scale * np.linalg.norm(P)
    assert np.linalg.norm((A @ P).conj().T - A @ P) < 1e-12 * scale
    assert np.linalg.norm((P @ A).conj().T - P @ A) < 1e-12 * scale
    np.testing.assert_allclose(P, np.linalg.pinv(A, rcond=1e-10, hermitian=True), atol=1e-10 * np.abs(P).max())


# --------------------------------------------------------------------------
# Sec. 3.3: the W sub-problem
# --------------------------------------------------------------------------

def _wcase(seed=7, m1=4, m2=9, m3=3, p=0.4):
    rng = _rng(seed)
    Z = rng.standard_normal((m1, m2, m3))
    G = rng.standard_normal((m1, m2, m3))
    mask = rng.random((m1, m2, m3)) < p
    mask[0, :, 0] = True  # a fully observed row
    mask[1, :, 0] = False  # a fully missing row
    return Z, G, mask


@pytest.mark.parametrize("mu,rho2", [(0.0, 0.0), (1e-3, 0.1), (0.5, 3.0)])
def test_wstep_minimises_g_k_bruteforce(mu, rho2):
    # Eq. (WETP-optim20): W_k minimises g_k over the missing entries; compare
    # with a generic numerical minimiser of g_k written from its definition.
    Z, G, mask = _wcase()
    m1, m2, m3 = Z.shape
    K = O.toeplitz_D(m2)
    W = O.w_step_dense(Z, G, mask, mu, rho2)
    for k in range(m3):
        for i in range(m1):
            C = np.flatnonzero(~mask[i, :, k])
            if C.size == 0:
                np.testing.assert_array_equal(W[i, :, k], G[i, :, k])
                continue

            def g(v):
                w = np.where(mask[i, :, k], G[i, :, k], 0.0)
                w[C] = v
                return 0.5 * (np.sum((Z[i, :, k] - w) ** 2) + rho2 * np.sum((K @ w) ** 2) + mu * np.sum(w ** 2))

            res = scipy.optimize.minimize(g, np.zeros(C.size), method="BFGS", options={"gtol": 1e-12})
            np.testing.assert_allclose(W[i, C, k], res.x, atol=1e-6)
            np.testing.assert_array_equal(W[i, mask[i, :, k], k], G[i, mask[i, :, k], k])


@pytest.mark.parametrize("mu,rho2", [(0.0, 0.0), (1e-3, 0.1), (0.5, 3.0)])
def test_wstep_kkt_banded_equals_dense_and_kkt_residual(mu, rho2):
    Z, G, mask = _wcase(11, 5, 13, 4)
    Wd = O.w_step_dense(Z, G, mask, mu, rho2)
    Wb = O.w_step_kkt(Z, G, mask, mu, rho2)
    np.testing.assert_allclose(Wb, Wd, rtol=1e-12, atol=1e-12)
    # Eq. (subquKKT): (W_k K_{mu rho2})_ij = (Z_k)_ij off the mask
    Kmr = O.K_murho(Z.shape[1], mu, rho2)
    for k in range(Z.shape[2]):
        lhs = Wd[:, :, k] @ Kmr
        miss = ~mask[:, :, k]
        np.testing.assert_allclose(lhs[miss], Z[:, :, k][miss], atol=1e-12)


def test_wstep_closed_form_without_periodicity_term():
    # rho2 = 0: g_k separates per entry, W = Z / (1 + mu) off the mask
    Z, G, mask = _wcase(2)
    W = O.w_step_kkt(Z, G, mask, 0.25, 0.0)
    np.testing.assert_allclose(W[~mask], Z[~mask] / 1.25, atol=1e-14)
    np.testing.assert_array_equal(W[mask], G[mask])


def test_wz_gap_bound():
    # bound after Proposition "KKProp": sum ||(W-Z)_{Omega^c}|| <= (mu+4 rho2) sum ||W_k||
    Z, G, mask = _wcase(3, 6, 20, 5, 0.3)
    for mu, rho2 in ((1e-3, 0.1), (0.2, 1.0)):
        W = O.w_step_kkt(Z, G, mask, mu, rho2)
        lhs = sum(np.linalg.norm((W[:, :, k] - Z[:, :, k]) * ~mask[:, :, k]) for k in range(Z.shape[2]))
        rhs = (mu + 4 * rho2) * sum(np.linalg.norm(W[:, :, k]) for k in range(Z.shape[2]))
        assert lhs <= rhs


# --------------------------------------------------------------------------
# Sec. 4.1: gradients, exact steps and the KKT system
# --------------------------------------------------------------------------

def _slice_case(seed=4, m1=6, m2=8, r=3):
    rng = _rng(seed)
    c = lambda *s: rng.standard_normal(s) + 1j * rng.standard_normal(s)  # noqa: E731
    return c(m1, r), c(r, m2), c(m1, m2)


def test_slice_gradients_against_finite_differences():
    # Eq. (hkXYDer) under Theorem "PDconj": the stated gradient equals
    # d h/d Re + i d h/d Im of the real function h_k (central differences).
    X, Y, W = _slice_case()
    rho1 = 0.7
    m1 = X.shape[0]
    H = O.toeplitz_D(m1)

    def h(Xv, Yv):
        Z = Xv @ Yv
        return 0.5 * (np.sum(np.abs(Z - W) ** 2) + rho1 * np.sum(np.abs(H @ Z) ** 2))

    eps = 1e-6
    for name, grad, arr in (("X", O.grad_X(X, Y, W, rho1), X), ("Y", O.grad_Y(X, Y, W, rho1), Y)):
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            for part, unit in ((1.0, 1.0), (1j, 1j)):
                P = arr.copy()
                P[idx] += eps * unit
                M = arr.copy()
                M[idx] -= eps * unit
                args_p = (P, Y) if name == "X" else (X, P)
                args_m = (M, Y) if name == "X" else (X, M)
                fd[idx] += part * (h(*args_p) - h(*args_m)) / (2 * eps)
        np.testing.assert_allclose(grad, fd, rtol=1e-6, atol=1e-6)


def test_exact_steps_solve_kkt_system():
    # Eq. (KKTcondition): with full-rank Y and X the exact X-step satisfies
    # H_rho1 X (Y Y^*) = W Y^*, and the exact Y-step (X^* H_rho1 X) Y = X^* W.
    X, Y, W = _slice_case(8)
    rho1 = 0.4
    Hr = O.H_rho(X.shape[0], rho1)
    Xn = O.x_update(X, Y, W, rho1)
    lhs, rhs = Hr @ Xn @ (Y @ Y.conj().T), W @ Y.conj().T
    assert np.linalg.norm(lhs - rhs) < 1e-10 * np.linalg.norm(rhs)
    Yn = O.y_update(Xn, Y, W, rho1)
    lhs, rhs = (Xn.conj().T @ Hr @ Xn) @ Yn, Xn.conj().T @ W
    assert np.linalg.norm(lhs - rhs) < 1e-10 * np.linalg.norm(rhs)


def test_scaled_steps_are_descent_directions():
    # Propositions "DirecX" / "DirecY": d_X, d_Y are descent directions; a
    # small scaled step decreases h_k
    X, Y, W = _slice_case(9)
    rho1 = 0.3
    H = O.toeplitz_D(X.shape[0])

    def h(Xv, Yv):
        Z = Xv @ Yv
        return 0.5 * (np.sum(np.abs(Z - W) ** 2) + rho1 * np.sum(np.abs(H @ Z) ** 2))

    Xn = O.x_update(X, Y, W, rho1, step="scaled", alpha=0.5)
    assert h(Xn, Y) < h(X, Y)
    Yn = O.y_update(Xn, Y, W, rho1, step="scaled", beta=0.5)
    assert h(Xn, Yn) < h(Xn, Y)


def _path_laplacian_norm(m):
    # H^T H for the first-difference matrix of Eq. (Toeplitz) is the Laplacian
    # of the path on m nodes, with eigenvalues 2 - 2 cos(pi k / m), k = 0..m-1
    return 2.0 + 2.0 * math.cos(math.pi / m)


def test_scaled_x_step_length_is_alpha_over_closed_form_L1():
    # Eq. (updataXYW1): the scaled X-step is X + (alpha / L1) d_X with
    # L1 = ||H_rho1||_2 ||Y Y^*||_2.  Rows of Y~ with disjoint supports make the
    # Gram diagonal, diag(d_s^2), so ||Y Y^*||_2 = max d_s^2 (not a Frobenius
    # norm), and ||H_rho1||_2 = 1 + rho1 (2 + 2 cos(pi / m1)).  The scaled step
    # divided by the unit step is alpha / L1.
    rng = _rng(41)
    m1, m2, r = 7, 11, 3
    d = np.array([0.7, 2.5, 1.3])
    Y = np.zeros((r, m2), complex)
    for s in range(r):
        Y[s, 2 * s + 1] = d[s] * np.exp(1j * rng.uniform(0, 2 * np.pi))
    X = rng.standard_normal((m1, r)) + 1j * rng.standard_normal((m1, r))
    W = rng.standard_normal((m1, m2)) + 1j * rng.standard_normal((m1, m2))
    rho1, alpha = 0.4, 0.9
    L1 = (1.0 + rho1 * _path_laplacian_norm(m1)) * d.max() ** 2
    step_unit = O.x_update(X, Y, W, rho1) - X
    step_scaled = O.x_update(X, Y, W, rho1, step="scaled", alpha=alpha) - X
    np.testing.assert_allclose(step_scaled, (alpha / L1) * step_unit, rtol=1e-12, atol=0)


def test_scaled_y_step_length_is_beta_over_closed_form_L2():
    # L2 = ||X^* H_rho1 X||_2.  The DCT-II vectors v_k(i) = cos(pi k (i + 1/2) / m1)
    # are the eigenvectors of the path Laplacian H^T H (eigenvalues
    # 2 - 2 cos(pi k / m1)); with the columns of X~ equal to c_k v_k / ||v_k|| (and a
    # phase each), X^* H_rho1 X = diag(c_k^2 (1 + rho1 (2 - 2 cos(pi k / m1)))).
    rng = _rng(42)
    m1, m2 = 9, 10
    ks, c = [1, 4, 8], [1.5, 0.8, 1.1]
    i = np.arange(m1)
    cols = []
    for k, ck in zip(ks, c):
        v = np.cos(math.pi * k * (i + 0.5) / m1)
        cols.append(ck * np.exp(1j * rng.uniform(0, 2 * np.pi)) * v / np.linalg.norm(v))
    X = np.stack(cols, axis=1)
    Y = rng.standard_normal((3, m2)) + 1j * rng.standard_normal((3, m2))
    W = rng.standard_normal((m1, m2)) + 1j * rng.standard_normal((m1, m2))
    rho1, beta = 0.7, 0.6
    L2 = max(ck ** 2 * (1.0 + rho1 * (2.0 - 2.0 * math.cos(math.pi * k / m1))) for k, ck in zip(ks, c))
    step_unit = O.y_update(X, Y, W, rho1) - Y
    step_scaled = O.y_update(X, Y, W, rho1, step="scaled", beta=beta) - Y
    np.testing.assert_allclose(step_scaled, (beta / L2) * step_unit, rtol=1e-12, atol=0)


# --------------------------------------------------------------------------
# The TCTF2R Algorithm: invariants and special cases
# --------------------------------------------------------------------------

def test_objective_monotone_at_every_half_step():
    # Theorem "GlobConvergM" and Proposition "inWWk"
    w = wl.custom(10, 16, 7, 2, 0.4, 321, iters=15)
    inst = wl.generate(w)
    out = O.tctf2r(inst["G"], inst["mask"], w.r, 1e-3, 0.05, 0.2, inst["Y0"], iters=15, record=True)
    h = out["hist"]
    seq = []
    for a, b, c in zip(h["f0_after_x"], h["f0_after_y"], h["f0"]):
        seq += [a, b, c]
    d = np.diff(seq)
    assert np.all(d <= 1e-10 * np.abs(np.array(seq[:-1])))


def test_exact_recovery_fully_observed_rank_r():
    # Proposition "tubrank": a noise-free tensor of tubal rank r, fully
    # observed, mu = rho = 0, is recovered to machine precision
    rng = _rng(12)
    A = rng.standard_normal((9, 2, 5))
    B = rng.standard_normal((2, 11, 5))
    T = O.tprod_definition(A, B)
    mask = np.ones(T.shape, bool)
    out = O.tctf2r(T, mask, 2, 0.0, 0.0, 0.0, rng.standard_normal((2, 11, 5)), iters=30)
    assert np.linalg.norm(out["Z"] - T) <= 1e-10 * np.linalg.norm(T)


def test_converged_objective_equals_eckart_young():
    # fully observed, mu = rho = 0: the optimum of Eq. (fun-XYW) is the best
    # rank-r approximation of every slice, f0 = (1/2m3) sum_k sum_{i>r} sigma_i^2
    rng = _rng(13)
    M = rng.standard_normal((8, 10, 5))
    mask = np.ones(M.shape, bool)
    r = 2
    out = O.tctf2r(M, mask, r, 0.0, 0.0, 0.0, rng.standard_normal((r, 10, 5)), iters=400)
    Mt = O.dft3(M)
    ey = sum(np.sum(np.linalg.svd(Mt[:, :, k], compute_uv=False)[r:] ** 2) for k in range(5)) / 10.0
    assert abs(out["f0"] - ey) <= 1e-8 * ey


def test_half_spectrum_equals_full_spectrum():
    # remark after the TCTF2R Algorithm: floor(m3/2)+1 slices suffice
    for n3 in (6, 7):
        w = wl.custom(7, 9, n3, 2, 0.5, 50 + n3, iters=6)
        inst = wl.generate(w)
        a = O.tctf2r(inst["G"], inst["mask"], 2, 1e-2, 0.1, 0.3, inst["Y0"], iters=6, half=True)
        b = O.tctf2r(inst["G"], inst["mask"], 2, 1e-2, 0.1, 0.3, inst["Y0"], iters=6, half=False)
        np.testing.assert_allclose(a["W"], b["W"], rtol=1e-10, atol=1e-10)


def test_dft_sign_convention_does_not_change_real_outputs():
    w = wl.custom(6, 10, 5, 2, 0.5, 77, iters=5)
    inst = wl.generate(w)
    a = O.tctf2r(inst["G"], inst["mask"], 2, 1e-2, 0.1, 0.3, inst["Y0"], iters=5, sign=+1)
    b = O.tctf2r(inst["G"], inst["mask"], 2, 1e-2, 0.1, 0.3, inst["Y0"], iters=5, sign=-1)
    np.testing.assert_allclose(a["W"], b["W"], rtol=1e-10, atol=1e-10)
    assert abs(a["f0"] - b["f0"]) < 1e-10 * a["f0"]


def test_matrix_case_m3_1_is_rank_r_fit():
    # m3 = 1: the model is plain matrix factorisation; fully observed and
    # mu = rho = 0 it converges to the truncated SVD (numpy)
    rng = _rng(21)
    M = rng.standard_normal((7, 9, 1))
    out = O.tctf2r(M, np.ones(M.shape, bool), 2, 0.0, 0.0, 0.0, rng.standard_normal((2, 9, 1)), iters=500)
    U, s, Vh = np.linalg.svd(M[:, :, 0])
    best = (U[:, :2] * s[:2]) @ Vh[:2]
    np.testing.assert_allclose(out["Z"][:, :, 0], best, atol=1e-7)


def test_dense_and_banded_wstep_agree_in_the_loop():
    w = wl.custom(5, 12, 4, 2, 0.4, 31, iters=4)
    inst = wl.generate(w)
    a = O.tctf2r(inst["G"], inst["mask"], 2, 1e-3, 0.1, 0.5, inst["Y0"], iters=4, wstep="dense")
    b = O.tctf2r(inst["G"], inst["mask"], 2, 1e-3, 0.1, 0.5, inst["Y0"], iters=4, wstep="kkt")
    np.testing.assert_allclose(a["W"], b["W"], rtol=1e-11, atol=1e-11)


def test_stopping_test_ends_at_the_first_iteration_meeting_all_three_bounds():
    # Algorithm step 6: stop after the first iteration l with ||X~' - X~||_inf,
    # ||Y~' - Y~||_inf and ||W' - W||_F all <= eps
    w = wl.custom(8, 12, 5, 2, 0.5, seed=77)
    inst = wl.generate(w)
    full = O.tctf2r(inst["G"], inst["mask"], 2, 1e-3, 1e-3, 1e-1, inst["Y0"], iters=30, record=True)
    h = full["hist"]
    m = np.maximum(np.maximum(h["dX"], h["dY"]), h["dW"])
    for eps in (m[3] * 1.0000001, m[7], 0.5 * (m[10] + m[11])):
        first = next(i for i in range(30) if m[i] <= eps) + 1
        out = O.tctf2r(inst["G"], inst["mask"], 2, 1e-3, 1e-3, 1e-1, inst["Y0"], iters=30, eps=eps)
        assert out["iters"] == first
        short = O.tctf2r(inst["G"], inst["mask"], 2, 1e-3, 1e-3, 1e-1, inst["Y0"], iters=first)
        assert np.array_equal(out["W"], short["W"])
    assert O.tctf2r(inst["G"], inst["mask"], 2, 1e-3, 1e-3, 1e-1, inst["Y0"], iters=6, eps=0.0)["iters"] == 6
    assert O.tctf2r(inst["G"], inst["mask"], 2, 1e-3, 1e-3, 1e-1, inst["Y0"], iters=6, eps=1e300)["iters"] == 1


# ---------------------------------------------------------------------------
# Differentiation form: loss of the factors and its gradient
# ---------------------------------------------------------------------------

def _grad_case(m1=12, m2=24, m3=8, r=3, seed=11):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((m1, r, m3))
    Y = rng.standard_normal((r, m2, m3))
    G = rng.standard_normal((m1, m2, m3))
    mask = rng.random((m1, m2, m3)) < 0.3
    return X, Y, G, mask


def test_conjugate_transpose_reverses_the_t_product():
    # (A*B)^* = B^* * A^* and (A^*)^* = A, with the t-product by its definition
    rng = np.random.default_rng(5)
    A, B = rng.standard_normal((4, 3, 6)), rng.standard_normal((3, 5, 6))
    lhs = O.ttranspose(O.tprod_definition(A, B))
    rhs = O.tprod_definition(O.ttranspose(B), O.ttranspose(A))
    assert np.allclose(lhs, rhs, rtol=0, atol=1e-12)
    assert np.array_equal(O.ttranspose(O.ttranspose(A)), A)


@pytest.mark.parametrize("rho1", [0.0, 0.3])
def test_factor_loss_gradient_matches_central_differences(rho1):
    # L is quadratic in any single entry of X (or of Y), so a central
    # difference equals the partial derivative up to rounding
    X, Y, G, mask = _grad_case()
    gX, gY = O.factor_loss_grad(X, Y, G, mask, rho1)
    h = 1e-3
    rng = np.random.default_rng(3)
    for A, g in ((X, gX), (Y, gY)):
        for _ in range(12):
            idx = tuple(int(rng.integers(0, n)) for n in A.shape)
            old = A[idx]
            A[idx] = old + h
            fp = O.factor_loss(X, Y, G, mask, rho1)
            A[idx] = old - h
            fm = O.factor_loss(X, Y, G, mask, rho1)
            A[idx] = old
            fd = (fp - fm) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-7 * max(1.0, abs(g[idx]))


def test_factor_loss_gradient_with_one_slice_is_the_matrix_gradient():
    # m3 = 1: L = 1/2 ||P(XY - G)||^2 + rho1/2 ||H X Y||^2, dL/dX = E Y^T, dL/dY = X^T E
    X, Y, G, mask = _grad_case(m3=1)
    rho1 = 0.2
    x, y, g, m = X[:, :, 0], Y[:, :, 0], G[:, :, 0], mask[:, :, 0]
    D = O.toeplitz_D(x.shape[0])
    E = np.where(m, x @ y - g, 0.0) + rho1 * D.T @ D @ x @ y
    gX, gY = O.factor_loss_grad(X, Y, G, mask, rho1)
    assert np.allclose(gX[:, :, 0], E @ y.T, rtol=1e-12, atol=1e-12)
    assert np.allclose(gY[:, :, 0], x.T @ E, rtol=1e-12, atol=1e-12)


# --------------------------------------------------------------------------
# Step 5 (rank vector): the rank-decreasing reading
# --------------------------------------------------------------------------

def _slice_rank_data(m1, m2, m3, obs, noise, seed):
    # t-product of factors whose third column of A is constant along mode 3:
    # its DFT is zero off the DC slice, so slice 0 has rank 3 and the others 2
    rng = _rng(seed)
    A = rng.standard_normal((m1, 3, m3))
    B = rng.standard_normal((3, m2, m3))
    A[:, 2, :] = A[:, 2, :1]
    T = O.tprod_definition(A, B)
    M = T + noise * math.sqrt(float(np.mean(T * T))) * rng.standard_normal(T.shape)
    mask = rng.random(T.shape) < obs
    return T, M, mask, rng.standard_normal((3, m2, m3))


def test_rank_rule_off_is_the_fixed_rank_algorithm():
    _, M, mask, Y0 = _slice_rank_data(12, 20, 7, 0.5, 0.01, 61)
    G = np.where(mask, M, 0.0)
    a = O.tctf2r_rank(G, mask, 3, 1e-3, 1e-3, 1e-1, Y0, iters=8, rank_tol=0.0)
    b = O.tctf2r(G, mask, 3, 1e-3, 1e-3, 1e-1, Y0, iters=8)
    assert np.linalg.norm(a["W"] - b["W"]) <= 1e-12 * np.linalg.norm(b["W"])
    assert abs(a["f0"] - b["f0"]) <= 1e-12 * b["f0"]
    assert a["ranks"] == [3] * 7


def test_rank_rule_finds_the_slice_ranks_of_the_data():
    # fully observed, 1% noise: the third direction of the rank-2 slices fits
    # noise only (Gram eigenvalue ratio ~1e-4), the DC slice keeps rank 3; the
    # rank vector is symmetric (r_k = r_{m3-k+2}) and the fit stays at the
    # noise level
    T, M, mask, Y0 = _slice_rank_data(40, 60, 8, 1.0, 0.01, 7)
    out = O.tctf2r_rank(M, mask, 3, 0.0, 1e-3, 0.0, Y0, iters=15, rank_tol=1e-2, patience=2)
    assert out["ranks"] == [3, 2, 2, 2, 2, 2, 2, 2]
    assert all(out["ranks"][k] == out["ranks"][(8 - k) % 8] for k in range(8))
    assert np.linalg.norm(out["Z"] - T) <= 0.02 * np.linalg.norm(T)


def test_rank_adjustment_of_a_dependent_factor_keeps_the_product():
    # X~ with an exactly dependent third column: dropping the zero-eigenvalue
    # direction of X~^* H_rho1 X~ leaves X~ Y~ unchanged and the width 2
    rng = _rng(62)
    X = rng.standard_normal((9, 3)) + 1j * rng.standard_normal((9, 3))
    X[:, 2] = 0.3 * X[:, 0] - (0.2 + 0.5j) * X[:, 1]
    Y = rng.standard_normal((3, 11)) + 1j * rng.standard_normal((3, 11))
    Xn, Yn, dropped = O.rank_adjust_slice(X, Y, 0.4, 1e-10)
    assert dropped == 1 and Xn.shape == (9, 2) and Yn.shape == (2, 11)
    assert np.linalg.norm(Xn @ Yn - X @ Y) <= 1e-12 * np.linalg.norm(X @ Y)


def test_rank_rule_at_true_ranks_recovers_better():
    # 60% observed: with the rule the slices settle at their data ranks and the
    # recovery error on the missing entries is lower than at the fixed rank 3
    _, M, mask, Y0 = _slice_rank_data(40, 60, 8, 0.6, 0.01, 7)
    G = np.where(mask, M, 0.0)
    out = O.tctf2r_rank(G, mask, 3, 1e-3, 1e-3, 1e-1, Y0, iters=20, rank_tol=0.08, patience=2)
    ref = O.tctf2r(G, mask, 3, 1e-3, 1e-3, 1e-1, Y0, iters=20)
    assert out["ranks"] == [3, 2, 2, 2, 2, 2, 2, 2]
    assert wl.nmse(M, out["W"], mask) < 0.8 * wl.nmse(M, ref["W"], mask)
