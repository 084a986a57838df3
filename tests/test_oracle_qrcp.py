"""Pins for Alg. 1 (QRCP) and for RQRCP's reduction to QRCP when Omega is orthogonal.

* Alg. 1 against LAPACK dgeqp3 (scipy.linalg.qr with pivoting) on small inputs with
  well-separated column norms: same pivots, same R (dgeqp3 uses the same xLARFG signs).
* Lemma 1 (QRCP pseudo-diagonal dominance): |r_ii| >= ||R(i:m, j)|| for j > i, exactly.
* Sec. III-B: with Omega = I_m (l = m) the sketch is A itself, R_hat = R and Eq. (4)
  leaves B = [0; R22], so RQRCP makes QRCP's pivot choices.  Any orthogonal Omega
  preserves column norms and gives the same pivots.
"""
import numpy as np
import pytest
import scipy.linalg as sla

from paper_1804_05138_gb300 import inputs


def _well_separated(m, n, seed):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((m, n)) * (1.5 ** rng.permutation(n))[None, :]
    return np.asfortranarray(A)


@pytest.mark.parametrize("m,n,seed", [(12, 9, 0), (30, 30, 1), (40, 25, 2), (20, 35, 3)])
def test_qrcp_matches_lapack_dgeqp3(orc, m, n, seed):
    A = _well_separated(m, n, seed)
    k = min(m, n)
    Af, jpvt, tau = orc.qrcp(A, k)
    Qs, Rs, Ps = sla.qr(A, pivoting=True, mode="economic")
    assert np.array_equal(jpvt, Ps)
    R = np.triu(Af[:k, :])
    assert np.allclose(R, Rs[:k, :], rtol=0, atol=1e-13 * np.abs(Rs).max())


def test_qrcp_lemma1_pseudo_diagonal_dominance(orc):
    A = inputs.gaussian(60, 40, seed=5)
    k = 25
    Af, jpvt, tau = orc.qrcp(A, k)
    R = orc.r_factor(Af, k)
    for i in range(k):
        tail = np.linalg.norm(R[i:, i + 1:], axis=0)
        assert abs(R[i, i]) >= tail.max() * (1 - 1e-13)


@pytest.mark.parametrize("m,n,b,k", [(24, 20, 4, 16), (24, 30, 5, 24), (30, 18, 7, 18)])
def test_rqrcp_identity_sketch_is_qrcp(orc, m, n, b, k):
    A = _well_separated(m, n, seed=m + n)
    p = m - b
    res = orc.rqrcp(A, k, b, p, np.eye(m), formula=4)
    Af, jpvt, tau = orc.qrcp(A, k)
    assert np.array_equal(res.jpvt, jpvt)
    assert np.allclose(res.A, Af, rtol=0, atol=1e-12 * np.abs(A).max())
    assert np.allclose(res.tau, tau, rtol=0, atol=1e-13)
    # Eq. (4) with Omega = I: the top block rows of B are annihilated, the rest is R22.
    if k < n:
        R22 = res.A[k:, k:]
        Btrail = res.B[:, k:]
        bb_last = k - ((k - 1) // b) * b
        assert np.abs(Btrail[:bb_last]).max() < 1e-11 * np.abs(A).max()
        assert np.allclose(np.linalg.norm(Btrail, axis=0), np.linalg.norm(R22, axis=0),
                           rtol=1e-10, atol=1e-11 * np.abs(A).max())


def test_rqrcp_orthogonal_sketch_is_qrcp(orc):
    m, n, b, k = 28, 22, 6, 18
    A = _well_separated(m, n, seed=9)
    Om = inputs.haar(m, m, seed=11).T.copy()
    res = orc.rqrcp(A, k, b, m - b, Om, formula=4)
    _, jpvt, _ = orc.qrcp(A, k)
    assert np.array_equal(res.jpvt, jpvt)
