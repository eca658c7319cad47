"""The acceptance rule of the refined r x r inverse (FP32 engines, r > 16).

The kernels invert a Hermitian positive definite Gram by an FP32 Gauss-Jordan
elimination X0, form the residual R = I - G X0 without rounding error (error-
free products and compensated sums), and accept X1 = X0 + X0 R (the
correction rounded to FP32) when ||R||_F <= 2^-14, on the claim that the
error of X1 is then about ||R||^2, below 2^-27 relative.  This emulates those
steps in numpy (FP32 elimination with the kernels' update rules, the residual
in FP64 standing in for the error-free one) on complex Hermitian matrices of
condition 10 to 3e3 and checks the claim.
"""
import numpy as np


def _gj32(A):
    # in-place Gauss-Jordan without pivoting in complex64, the update rules of
    # the kernels: a_pp <- 1/a_pp, a_pj <- a_pj / a_pp, a_ip <- -a_ip / a_pp,
    # a_ij <- a_ij - a_ip a_pj / a_pp
    W = A.astype(np.complex64).copy()
    for p in range(W.shape[0]):
        ip = np.float32(1) / W[p, p].real
        t = W[p, :] * ip
        c = W[:, p].copy()
        W = W - np.outer(c, t)
        W[p, :] = t
        W[:, p] = -c * ip
        W[p, p] = ip
    return W


def _gram(rng, r, kappa):
    Q, _ = np.linalg.qr(rng.standard_normal((r, r)) + 1j * rng.standard_normal((r, r)))
    A = (Q * np.logspace(0, np.log10(kappa), r)) @ Q.conj().T
    return ((A + A.conj().T) / 2).astype(np.complex64)


def test_accepted_refinement_is_below_2_pow_minus_27():
    rng = np.random.default_rng(0)
    accepted = 0
    for kappa in (10.0, 1e2, 1e3, 3e3):
        for _ in range(6):
            G = _gram(rng, 32, kappa)
            X0 = _gj32(G)
            R = np.eye(32) - G.astype(np.complex128) @ X0.astype(np.complex128)
            C = (X0 @ R.astype(np.complex64)).astype(np.complex64)
            X1 = X0.astype(np.complex128) + C.astype(np.complex128)
            X1 = (X1 + X1.conj().T) / 2
            Xt = np.linalg.inv(G.astype(np.complex128))
            rn = float(np.linalg.norm(R))
            err = float(np.linalg.norm(X1 - Xt) / np.linalg.norm(Xt))
            # the step's error follows ||R||^2 (plus the FP32 rounding of the correction)
            assert err <= 8 * rn * rn + 2.0 ** -40
            if rn <= 2.0 ** -14:
                accepted += 1
                assert err <= 2.0 ** -27
    assert accepted >= 6  # the well-conditioned cases pass the bar
