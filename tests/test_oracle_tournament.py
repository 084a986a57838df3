"""Pins for the oracle's QR with tournament pivoting on the sketch (the paper's future work,
Sec. VI: tournament pivoting in place of the partial QRCP on B; Demmel, Grigori, Gu, Xiang,
SIAM J. Matrix Anal. Appl. 36 (2015)), against LAPACK and against what the definition fixes.

T1  One leaf holding every column: the tournament is Alg. 1 on B, so its choices are LAPACK
    dgeqp3's first bb pivots (scipy.linalg.qr with pivoting, a library routine).
T2  Mutually orthogonal columns with distinct norms: a reflector leaves the other columns' norms
    unchanged, so every group keeps its largest columns and the root takes the bb largest of
    all, largest first, whatever the grouping.
T3  The definition step by step, with dgeqp3 as each node's choice: leaves of gs consecutive
    columns, runs of `fanin` consecutive groups merged in order, min(bb, candidates) chosen at
    every node; several (nc, gs, bb, fanin) with ragged last groups and two to four levels.
T4  Ties: exactly repeated columns go to the smallest position, at the leaves and at the nodes.
T5  RQRCP with the tournament and one leaf per block equals the greedy RQRCP (pivots and R);
    with several leaves per block the factorization stays backward stable (residual at
    rounding level), its R22 is within a small factor of the greedy one, and on an exactly
    rank-r input the rank guard stops at r.
T6  Planted mistakes in a copy of the oracle's C source (group boundary, fan-in, leaf choice
    count, norm rows, tie rule, the position map) each fail at least one of T1-T5.
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
_i64, _dp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
_i64p, _i32p = ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int32)


class _Orc:
    """The two entry points these pins need, on a given build of the oracle's source."""

    def __init__(self, lib):
        lib.orc_tournament.argtypes = [_dp, _i64, _i64, _i64, _i64, _i64, _i64, _i64p, _dp]
        lib.orc_tournament.restype = ctypes.c_int64
        lib.orc_rqrcp3.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, _i64, _dp, ctypes.c_int, ctypes.c_int,
                                   _i64p, _i64, _i32p, _dp, _i64p, _dp, _dp]
        lib.orc_rqrcp3.restype = ctypes.c_int
        self.lib = lib

    def tournament(self, X, bb, gs, fanin, pos0=0):
        Xf = np.asfortranarray(X, dtype=np.float64)
        l, nc = Xf.shape
        sel = np.zeros(bb, dtype=np.int64)
        gap = np.zeros(1)
        ns = self.lib.orc_tournament(Xf.ctypes.data_as(_dp), l, nc, pos0, bb, gs, fanin, sel.ctypes.data_as(_i64p),
                                     gap.ctypes.data_as(_dp))
        assert ns >= 0
        return sel[:ns]

    def rqrcp(self, A, k, b, p, Om, tgs=None, fanin=4):
        Af = np.array(A, dtype=np.float64, order="F", copy=True)
        m, n = Af.shape
        jpvt = np.zeros(n, dtype=np.int32)
        tau = np.zeros(k)
        rank = np.zeros(1, dtype=np.int64)
        gaps = np.zeros(k)
        B = np.zeros((b + p, n), order="F")
        nblk = (k + b - 1) // b
        tg = None if tgs is None else np.full(nblk, tgs, dtype=np.int64)
        rc = self.lib.orc_rqrcp3(m, n, Af.ctypes.data_as(_dp), m, k, b, p,
                                 np.ascontiguousarray(Om, dtype=np.float64).ctypes.data_as(_dp), 4, 0,
                                 tg.ctypes.data_as(_i64p) if tg is not None else _i64p(), fanin,
                                 jpvt.ctypes.data_as(_i32p), tau.ctypes.data_as(_dp), rank.ctypes.data_as(_i64p),
                                 gaps.ctypes.data_as(_dp), B.ctypes.data_as(_dp))
        assert rc == 0
        return Af, jpvt, tau, int(rank[0])


def _dgeqp3_choice(X, cols, steps):
    """The first `steps` pivots of LAPACK dgeqp3 on X(:, cols), as positions from cols."""
    _, _, P = sl.qr(X[:, cols], pivoting=True, mode="economic")
    return [cols[j] for j in P[:steps]]


def _definition(X, bb, gs, fanin):
    nc = X.shape[1]
    groups = [_dgeqp3_choice(X, list(range(g, min(g + gs, nc))), min(bb, min(g + gs, nc) - g))
              for g in range(0, nc, gs)]
    while len(groups) > 1:
        nxt = []
        for q in range(0, len(groups), fanin):
            cand = [c for grp in groups[q:q + fanin] for c in grp]
            nxt.append(_dgeqp3_choice(X, cand, min(bb, len(cand))))
        groups = nxt
    return groups[0]


def _rfac(Af, k):
    """R of the partial factorization: the first k columns upper triangular, R12 and R22 full."""
    R = Af.copy()
    for j in range(k):
        R[j + 1:, j] = 0.0
    return R


def _residual(A, Af, tau, jpvt, k):
    m, n = A.shape
    R = _rfac(Af, k)
    Q = np.eye(m)
    for j in reversed(range(k)):
        v = np.zeros(m)
        v[j] = 1.0
        v[j + 1:] = Af[j + 1:, j]
        Q -= tau[j] * np.outer(v, v @ Q)
    return np.linalg.norm(A[:, jpvt] - Q @ R) / np.linalg.norm(A)


def _r22(Af, k):
    return np.linalg.norm(Af[k:, k:], 2)


T3_CASES = [(60, 10, 3, 2), (97, 12, 4, 4), (130, 16, 5, 3), (45, 45, 6, 4), (200, 9, 4, 2), (77, 20, 8, 4)]


def _check_all(o):
    rng = np.random.default_rng(0)
    # T1
    for (l, nc, bb) in [(20, 50, 4), (12, 30, 12), (33, 70, 9)]:
        X = rng.standard_normal((l, nc))
        assert list(o.tournament(X, bb, nc + 5, 4)) == _dgeqp3_choice(X, list(range(nc)), bb), "T1"
    # T2
    l, nc, bb = 64, 60, 7
    d = rng.permutation(np.linspace(1.0, 60.0, nc))
    Qo, _ = np.linalg.qr(rng.standard_normal((l, l)))
    X = Qo[:, :nc] * d
    want = list(np.argsort(-d)[:bb])
    for gs, fanin in [(5, 2), (8, 4), (13, 3), (60, 4)]:
        assert list(o.tournament(X, bb, gs, fanin)) == want, ("T2", gs, fanin)
    # T3
    for (nc, gs, bb, fanin) in T3_CASES:
        X = rng.standard_normal((bb + 6, nc))
        assert list(o.tournament(X, bb, gs, fanin)) == _definition(X, bb, gs, fanin), ("T3", nc, gs, bb, fanin)
    # T4: column 3 repeated at 7 and 11 (different leaves of gs = 4), column 2 repeated at 9
    X = rng.standard_normal((10, 16)) * 0.1
    X[:, 3] = X[:, 7] = X[:, 11] = 5.0 * rng.standard_normal(10)
    X[:, 2] = X[:, 9] = 3.0 * rng.standard_normal(10)
    sel = list(o.tournament(X, 2, 4, 2))
    assert sel[0] == 3, "T4 tie at the nodes"
    assert list(o.tournament(X, 2, 16, 2)) == [3, 2], "T4 ties in one leaf"
    # T5
    m, n, k, b, p = 90, 70, 24, 8, 6
    A = rng.standard_normal((m, n)) @ np.diag(np.exp(-np.arange(n) / 15.0))
    Om = rng.standard_normal((b + p, m))
    Ag, jg, tg, rg = o.rqrcp(A, k, b, p, Om)
    At, jt, tt, rt = o.rqrcp(A, k, b, p, Om, tgs=n + 1)
    assert np.array_equal(jg, jt) and rg == rt == k, "T5 one leaf"
    assert np.linalg.norm(_rfac(Ag, k) - _rfac(At, k)) <= 1e-12 * np.linalg.norm(_rfac(Ag, k)), "T5 one leaf R"
    for gs, fanin in [(10, 2), (16, 4), (9, 3)]:
        At, jt, tt, rt = o.rqrcp(A, k, b, p, Om, tgs=gs, fanin=fanin)
        assert sorted(jt) == list(range(n)) and rt == k
        assert _residual(A, At, tt, jt, k) <= 1e-14, ("T5 residual", gs, fanin)
        assert _r22(At, k) <= 2.0 * _r22(Ag, k), ("T5 R22", gs, fanin)
    G = rng.standard_normal((m, 11)) @ rng.standard_normal((11, n))
    Om2 = rng.standard_normal((b + p, m))
    _, _, _, rr = o.rqrcp(G, k, b, p, Om2, tgs=12, fanin=2)
    assert rr == 11, "T5 rank guard"


def test_tournament_pins(orc):
    _check_all(_Orc(ctypes.CDLL(orc.build())))


def test_tournament_python_wrapper(orc):
    rng = np.random.default_rng(3)
    X = rng.standard_normal((14, 40))
    sel, gap = orc.tournament(X, 5, 9, 2)
    assert list(sel) == _definition(X, 5, 9, 2) and 0.0 < gap <= 1.0
    A = rng.standard_normal((50, 40))
    res = orc.rqrcp(A, 16, 8, 4, rng.standard_normal((12, 50)), tgs=[10, 12], fanin=3)
    assert res.rank == 16 and sorted(res.jpvt) == list(range(40))


MUTATIONS = [
    ("leaf skips the first column of every group but the first",
     r"const int64_t c0 = g \* gs, c1", "const int64_t c0 = g * gs + (g > 0), c1"),
    ("a node after the first drops its first child",
     r"for \(int64_t g = q \* fanin; g < \(q \+ 1\) \* fanin && g < P; \+\+g\)",
     "for (int64_t g = q * fanin + (q > 0); g < (q + 1) * fanin && g < P; ++g)"),
    ("leaves choose one column fewer",
     r"cnt\[g\] = bb < c1 - c0 \? bb : c1 - c0;", "cnt[g] = bb - 1 < c1 - c0 ? bb - 1 : c1 - c0;"),
    ("norms over all rows instead of the trailing rows",
     r"for \(int64_t r = t; r < l; \+\+r\) nu \+= AT\(W, l, r, s\) \* AT\(W, l, r, s\);",
     "for (int64_t r = 0; r < l; ++r) nu += AT(W, l, r, s) * AT(W, l, r, s);"),
    ("ties to the larger position",
     r"\(nu == v1 && cand\[s\] < cand\[best\]\)", "(nu == v1 && cand[s] > cand[best])"),
    ("position map: the displaced column's new position wrong",
     r"where\[ob\] = c; where\[oc\] = best;", "where[ob] = c; where[oc] = c;"),
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
