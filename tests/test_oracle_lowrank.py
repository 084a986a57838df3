"""Pins for the oracle's Q formation, Q x and low-rank product (Sec. I-A: A Pi ~ Q1 [R11 R12]),
against LAPACK and against what the mathematics fixes -- nothing here compares the oracle with
itself.

L1  form_q and apply_q on LAPACK's own Householder factor (scipy.linalg.qr, mode='raw': the
    xGEQP3 layout with xLARFG reflectors, the convention the oracle reads) reproduce LAPACK's
    explicit Q (xORGQR): Q(:, 0:k) to rounding, and Q x for unit and random vectors.
L2  lowrank on that factor equals the product of LAPACK's explicit Q1 and [R11 R12], scattered to
    the input's column order: L(:, jpvt[c]) = Q1 R(0:k, c).
L3  k = n <= m: L equals A (the factorization is exact up to rounding), for a matrix whose
    column norms force a non-trivial permutation.
L4  k < n: ||A - L||_F = ||R22||_F, the trailing block of LAPACK's R (Q is orthogonal).
L5  planted mistakes in a copy of the oracle's C source (the column scatter, the length of the
    triangular column, the order and sign of the reflectors in Q x) each fail L1-L4.
"""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest
import scipy.linalg as sl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_SRC = os.path.join(ROOT, "oracle", "rqrcp_oracle.c")
U = 2.0 ** -53


def _input(m, n, seed):
    rng = np.random.default_rng(seed)
    # column scales spread over six orders of magnitude: the pivot order is far from identity
    return np.asfortranarray(rng.standard_normal((m, n)) * (10.0 ** rng.uniform(-3, 3, n))[None, :])


def _lapack(A):
    (raw, tau), _, P = sl.qr(A, pivoting=True, mode="raw")
    Q, R, P2 = sl.qr(A, pivoting=True, mode="economic")
    assert np.array_equal(P, P2)
    return np.asfortranarray(raw), tau, P.astype(np.int32), Q, R


class _Orc:
    """The three oracle routines loaded from a given shared library (the real oracle, or a copy
    of its source with one planted mistake)."""

    def __init__(self, lib):
        d, i64 = ctypes.POINTER(ctypes.c_double), ctypes.c_int64
        lib.orc_form_q.argtypes = [i64, i64, d, i64, d, i64, d, i64]
        lib.orc_apply_q.argtypes = [i64, i64, d, i64, d, d]
        lib.orc_lowrank.argtypes = [i64, i64, i64, d, i64, d, ctypes.POINTER(ctypes.c_int32), d, i64, d]
        lib.orc_lowrank.restype = ctypes.c_int
        self.lib = lib

    @staticmethod
    def _p(a):
        return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))

    def form_q(self, raw, tau, k, ncols):
        m = raw.shape[0]
        Q = np.zeros((m, ncols), order="F")
        self.lib.orc_form_q(m, k, self._p(raw), m, self._p(np.ascontiguousarray(tau)), ncols, self._p(Q), m)
        return Q

    def apply_q(self, raw, tau, k, x):
        y = np.array(x, dtype=np.float64, copy=True)
        self.lib.orc_apply_q(raw.shape[0], k, self._p(raw), raw.shape[0], self._p(np.ascontiguousarray(tau)),
                             self._p(y))
        return y

    def lowrank(self, raw, tau, jpvt, k):
        m, n = raw.shape
        L = np.zeros((m, n), order="F")
        Q1 = np.zeros((m, k), order="F")
        jp = np.ascontiguousarray(jpvt, dtype=np.int32)
        rc = self.lib.orc_lowrank(m, n, k, self._p(raw), m, self._p(np.ascontiguousarray(tau)),
                                  jp.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), self._p(L), m, self._p(Q1))
        assert rc == 0
        return L, Q1


@pytest.fixture(scope="module")
def real(orc):
    return _Orc(orc._load())


def _check_all(o):
    """Every pin of this file on one oracle; raises AssertionError at the first that fails."""
    # L1: Q and Q x against LAPACK's explicit Q
    for (m, n, k, seed) in [(40, 30, 30, 1), (37, 50, 20, 2)]:
        A = _input(m, n, seed)
        raw, tau, P, Q, R = _lapack(A)
        Qo = o.form_q(raw, tau, min(m, n), Q.shape[1])
        assert np.abs(Qo - Q).max() <= 50 * m * U, "form_q vs LAPACK Q"
        Qfull = sl.qr(A, pivoting=True, mode="full")[0]
        for j in range(0, m, 7):
            e = np.zeros(m)
            e[j] = 1.0
            assert np.abs(o.apply_q(raw, tau, min(m, n), e) - Qfull[:, j]).max() <= 50 * m * U, "apply_q(e_j)"
        x = np.random.default_rng(seed + 10).standard_normal(m)
        assert np.abs(o.apply_q(raw, tau, min(m, n), x) - Qfull @ x).max() <= 50 * m * U * np.abs(x).sum(), "Q x"
        # L2: the scattered product of LAPACK's Q1 and [R11 R12]
        L, Q1 = o.lowrank(raw, tau, P, k)
        Lref = np.zeros_like(L)
        Lref[:, P] = Q[:, :k] @ R[:k, :]
        assert np.abs(Q1 - Q[:, :k]).max() <= 50 * m * U, "Q1"
        assert np.linalg.norm(L - Lref) <= 100 * m * U * np.linalg.norm(Lref), "L vs LAPACK Q1 R"
    # L3: k = n <= m reproduces A
    for (m, n, seed) in [(30, 30, 3), (45, 20, 4), (1, 1, 5)]:
        A = _input(m, n, seed)
        raw, tau, P, Q, R = _lapack(A)
        L, _ = o.lowrank(raw, tau, P, n)
        assert np.linalg.norm(L - A) <= 100 * m * U * np.linalg.norm(A), "L == A at k = n"
    # L4: k < n leaves exactly R22
    for (m, n, k, seed) in [(40, 30, 10, 6), (25, 60, 24, 7)]:
        A = _input(m, n, seed)
        raw, tau, P, Q, R = _lapack(A)
        L, _ = o.lowrank(raw, tau, P, k)
        r22 = np.linalg.norm(np.triu(raw)[k:, k:])
        assert abs(np.linalg.norm(A - L) - r22) <= 100 * m * U * np.linalg.norm(A), "||A - L|| = ||R22||"


def test_lowrank_and_q_against_lapack(real):
    _check_all(real)


def test_lowrank_of_oracle_rqrcp_with_identity_sketch(orc):
    """The oracle's own RQRCP with Omega = I is QRCP: its low-rank product at k = n is A again and,
    at k < n, leaves ||R22||_F."""
    A = _input(36, 28, 8)
    res = orc.rqrcp(A, 28, 8, 28, np.eye(36))
    L, Q1 = orc.lowrank(res.A, res.tau, res.jpvt, 28)
    assert np.linalg.norm(L - A) <= 100 * 36 * U * np.linalg.norm(A)
    res = orc.rqrcp(A, 12, 4, 32, np.eye(36))
    L, Q1 = orc.lowrank(res.A, res.tau, res.jpvt, 12)
    r22 = np.linalg.norm(orc.r_factor(res.A, 12)[12:, 12:])
    assert abs(np.linalg.norm(A - L) - r22) <= 100 * 36 * U * np.linalg.norm(A)
    assert orc.orth_error(Q1) <= 100 * 36 * U


MUTATIONS = [
    ("scatter to L(:, c) instead of L(:, jpvt[c])",
     r"double\* out = &AT\(L, ldl, 0, jpvt\[c\]\);", "double* out = &AT(L, ldl, 0, c);"),
    ("triangular column one entry short",
     r"int64_t top = \(c \+ 1 < k\) \? c \+ 1 : k;", "int64_t top = (c < k) ? c : k;"),
    ("triangular column one entry long (reads the reflector tail)",
     r"int64_t top = \(c \+ 1 < k\) \? c \+ 1 : k;", "int64_t top = (c + 2 < k) ? c + 2 : k;"),
    ("reflectors applied in the wrong order in Q x (Q^T x)",
     r"for \(int64_t h = k - 1; h >= 0; --h\) house_apply\(m - h, &AT\(A, lda, h, h\), tau\[h\], x \+ h\);",
     "for (int64_t h = 0; h < k; ++h) house_apply(m - h, &AT(A, lda, h, h), tau[h], x + h);"),
    ("wrong sign of tau in Q x",
     r"house_apply\(m - h, &AT\(A, lda, h, h\), tau\[h\], x \+ h\);",
     "house_apply(m - h, &AT(A, lda, h, h), -tau[h], x + h);"),
]


@pytest.mark.parametrize("what,pattern,repl", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistakes_fail_the_pins(tmp_path, what, pattern, repl):
    src = open(ORACLE_SRC).read()
    bad, count = re.subn(pattern, repl, src)
    assert count == 1, f"mutation pattern for '{what}' must match exactly once"
    cpath = tmp_path / "mutant.c"
    cpath.write_text(bad)
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE", "-fvisibility=hidden",
                    str(cpath), "-o", str(so), "-lm"], check=True)
    with pytest.raises(AssertionError):
        _check_all(_Orc(ctypes.CDLL(str(so))))
