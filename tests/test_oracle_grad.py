"""Pins for the oracle's gradients of the truncated factorization with Pi held fixed.

Both the closed-form gradient of L = ||A - Q1 [R11 R12] Pi^T||_F^2 and the general
thin-QR adjoint (upstream gradients on Q1, R11, R12) are checked against FP64 central
finite differences along random directions, at 256 x 128 with k = 16.
"""
import numpy as np
import pytest

from paper_1804_05138_gb300 import inputs


def _setup(orc, m=256, n=128, k=16, seed=0):
    A = inputs.spectrum_matrix(m, n, inputs.sigma_inverse_square(n))
    res = orc.rqrcp(A, k, 8, 8, inputs.gaussian_sketch(16, m, seed=seed))
    return A, res.jpvt


def test_loss_gradient_closed_form_vs_fd(orc):
    A, jpvt = _setup(orc)
    k = 16
    G = orc.truncated_loss_grad(A, jpvt, k)
    rng = np.random.default_rng(1)
    h = 1e-6
    for _ in range(6):
        E = rng.standard_normal(A.shape)
        E /= np.linalg.norm(E)           # keep h*E far below sigma_k of A
        fd = (orc.truncated_loss(A + h * E, jpvt, k) - orc.truncated_loss(A - h * E, jpvt, k)) / (2 * h)
        an = float(np.sum(G * E))
        assert abs(fd - an) <= 1e-6 * max(1.0, abs(an)), (fd, an)


def test_general_adjoint_vs_fd(orc):
    A, jpvt = _setup(orc, seed=2)
    k = 16
    rng = np.random.default_rng(3)
    m, n = A.shape
    dQ1 = rng.standard_normal((m, k))
    dR11 = np.triu(rng.standard_normal((k, k)))
    dR12 = rng.standard_normal((k, n - k))

    def f(Ain):
        X = Ain[:, jpvt]
        Q1, R11, R12 = orc.truncated_qr_forward(X, k)
        return float(np.sum(dQ1 * Q1) + np.sum(dR11 * R11) + np.sum(dR12 * R12))

    X = A[:, jpvt]
    Q1, R11, R12 = orc.truncated_qr_forward(X, k)
    dX = orc.truncated_qr_adjoint(X, Q1, R11, R12, dQ1, dR11, dR12)
    dA = np.empty_like(dX)
    dA[:, jpvt] = dX
    h = 1e-6
    for _ in range(6):
        E = rng.standard_normal(A.shape)
        E /= np.linalg.norm(E)           # keep h*E far below sigma_k of A
        fd = (f(A + h * E) - f(A - h * E)) / (2 * h)
        an = float(np.sum(dA * E))
        assert abs(fd - an) <= 1e-5 * max(1.0, abs(an)), (fd, an)


def test_loss_gradient_matches_general_adjoint(orc):
    """The loss gradient equals the general adjoint with the upstream gradients of L."""
    A, jpvt = _setup(orc, m=64, n=40, k=8, seed=4)
    k = 8
    X = A[:, jpvt]
    Q1, R11, R12 = orc.truncated_qr_forward(X, k)
    Rk = np.concatenate([R11, R12], axis=1)
    E = X - Q1 @ Rk
    dQ1 = -2.0 * E @ Rk.T
    dRk = -2.0 * Q1.T @ E
    dX = orc.truncated_qr_adjoint(X, Q1, R11, R12, dQ1, np.triu(dRk[:, :k]), dRk[:, k:])
    dX = dX + 2.0 * E       # explicit dependence of L on X
    dA = np.empty_like(dX)
    dA[:, jpvt] = dX
    G = orc.truncated_loss_grad(A, jpvt, k)
    assert np.allclose(dA, G, rtol=1e-8, atol=1e-10 * np.abs(G).max())


@pytest.mark.parametrize("m,k", [(50, 7), (120, 20)])
def test_cholqr_reorth_keeps_product_and_orthogonalises(orc, m, k):
    rng = np.random.default_rng(m)
    Q, _ = np.linalg.qr(rng.standard_normal((m, k)))
    Q1 = Q + 1e-5 * rng.standard_normal((m, k))      # perturbed orthonormal basis
    Rk = np.triu(rng.standard_normal((k, 3 * k)))
    Qn, Rn = orc.cholqr_reorth(Q1, Rk)
    assert orc.orth_error(Qn) < 1e-12
    assert np.allclose(Qn @ Rn, Q1 @ Rk, rtol=0, atol=1e-12 * np.abs(Q1 @ Rk).max())
    assert np.allclose(np.tril(Rn[:, :k], -1), 0.0)
