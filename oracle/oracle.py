"""FP64 CPU oracle for randomized QR with column pivoting (Xiao, Gu, Langou, HiPC 2017).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this module.  It never imports the CUDA
package and the CUDA package never imports it.

The step-by-step algorithms live in ``rqrcp_oracle.c`` (plain C loops, no BLAS);
this module compiles that file with gcc on first use, loads it with ctypes and adds
numpy-level helpers for quantities that have a plain definition (residuals, the
CholQR reorthogonalisation, the closed-form gradient).  numpy/scipy library
primitives (matmul, cholesky, triangular solve, SVD) serve as single steps only.

Pins (tests/test_oracle_*.py): Philox against numpy's Philox bit generator; Alg. 1
against LAPACK dgeqp3; RQRCP with Omega = I against Alg. 1 (special case, Sec. III-B);
Eq. (4) against Eq. (5) (same permutations, Sec. III-B); the Kahan matrix against
Tables I and II (Sec. V-B); Lemma 1 and Lemma 3 inequalities; Theorem 1's p bound
against the worked example in Sec. III-C; the gradient against finite differences; Alg. 3
(SRQR) against Tables I and II's SRQR columns, the factorization identity through forced
swaps, exact estimates with a scaled identity sketch, the bound of Sec. IV-D and the exact g2.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rqrcp_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle_rqrcp.so")
_lock = threading.Lock()
_lib = None

_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_dp = ctypes.POINTER(ctypes.c_double)
_i32p = ctypes.POINTER(ctypes.c_int32)
_i64p = ctypes.POINTER(ctypes.c_int64)
_u64p = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile rqrcp_oracle.c into oracle/_build/liboracle_rqrcp.so (gcc -O3 -fopenmp)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c11", "-D_GNU_SOURCE",
           "-fvisibility=hidden", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        lib.orc_philox4x64_10.argtypes = [_u64p, _u64p, _u64p]
        lib.orc_philox4x64_10.restype = None
        lib.orc_omega.argtypes = [_i64, _i64, _u64, _dp]
        lib.orc_omega.restype = None
        lib.orc_qrcp.argtypes = [_i64, _i64, _dp, _i64, _i64, _i32p, _dp]
        lib.orc_qrcp.restype = ctypes.c_int
        lib.orc_rqrcp.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, _i64, _dp, ctypes.c_int,
                                  _i32p, _dp, _i64p, _dp, _dp]
        lib.orc_rqrcp.restype = ctypes.c_int
        lib.orc_rqrcp2.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, _i64, _dp, ctypes.c_int, ctypes.c_int,
                                   _i32p, _dp, _i64p, _dp, _dp]
        lib.orc_rqrcp2.restype = ctypes.c_int
        lib.orc_rqrcp3.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, _i64, _dp, ctypes.c_int, ctypes.c_int,
                                   _i64p, _i64, _i32p, _dp, _i64p, _dp, _dp]
        lib.orc_rqrcp3.restype = ctypes.c_int
        lib.orc_tournament.argtypes = [_dp, _i64, _i64, _i64, _i64, _i64, _i64, _i64p, _dp]
        lib.orc_tournament.restype = ctypes.c_int64
        lib.orc_round_bf16.argtypes = [_i64, _dp, _dp]
        lib.orc_round_bf16.restype = None
        lib.orc_form_q.argtypes = [_i64, _i64, _dp, _i64, _dp, _i64, _dp, _i64]
        lib.orc_form_q.restype = None
        lib.orc_apply_q.argtypes = [_i64, _i64, _dp, _i64, _dp, _dp]
        lib.orc_apply_q.restype = None
        lib.orc_lowrank.argtypes = [_i64, _i64, _i64, _dp, _i64, _dp, _i32p, _dp, _i64, _dp]
        lib.orc_lowrank.restype = ctypes.c_int
        lib.orc_srqr.argtypes = [_i64, _i64, _dp, _i64, _i64, _i64, _i64, _dp, ctypes.c_double, _i64, _u64, _i64,
                                 _dp, _i32p, _i64p, _dp, _dp, _i64p]
        lib.orc_srqr.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _fortran64(A: np.ndarray) -> np.ndarray:
    return np.array(A, dtype=np.float64, order="F", copy=True)


# --------------------------------------------------------------------------- RNG
def philox4x64_10(ctr, key) -> np.ndarray:
    """One Philox4x64-10 block (Salmon et al., SC'11) -> 4 uint64 words."""
    lib = _load()
    c = np.asarray(ctr, dtype=np.uint64).copy()
    k = np.asarray(key, dtype=np.uint64).copy()
    out = np.zeros(4, dtype=np.uint64)
    lib.orc_philox4x64_10(_ptr(c, ctypes.c_uint64), _ptr(k, ctypes.c_uint64), _ptr(out, ctypes.c_uint64))
    return out


def omega(l: int, m: int, seed: int) -> np.ndarray:
    """Gaussian sketching matrix Omega (l x m, Alg. 2) drawn from Philox4x64-10 + Box-Muller."""
    lib = _load()
    out = np.empty((l, m), dtype=np.float64)  # row-major, as the C routine writes it
    lib.orc_omega(l, m, seed, _ptr(out, ctypes.c_double))
    return out


# --------------------------------------------------------------------------- Alg. 1
def qrcp(A: np.ndarray, k: int):
    """Alg. 1 (QRCP, k steps).  Returns (A_fact, jpvt, tau), LAPACK-style in-place layout."""
    lib = _load()
    Af = _fortran64(A)
    m, n = Af.shape
    jpvt = np.zeros(n, dtype=np.int32)
    tau = np.zeros(k, dtype=np.float64)
    rc = lib.orc_qrcp(m, n, _ptr(Af, ctypes.c_double), max(m, 1), k, _ptr(jpvt, ctypes.c_int32),
                      _ptr(tau, ctypes.c_double))
    if rc != 0:
        raise ValueError(f"orc_qrcp: invalid argument ({rc})")
    return Af, jpvt, tau


# --------------------------------------------------------------------------- Alg. 2
class RQRCPResult:
    def __init__(self, A, jpvt, tau, rank, gaps, B):
        self.A, self.jpvt, self.tau, self.rank, self.gaps, self.B = A, jpvt, tau, rank, gaps, B


def tournament(X: np.ndarray, bb: int, gs: int, fanin: int = 4, pos0: int = 0):
    """QR with tournament pivoting on the l x nc matrix X (column s has position pos0 + s):
    leaves of gs consecutive columns, fan-in `fanin`, every choice Alg. 1 with ties to the
    smallest position.  Returns (the min(bb, nc) chosen positions in order, the smallest
    relative gap of all choices)."""
    lib = _load()
    Xf = _fortran64(X)
    l, nc = Xf.shape
    sel = np.zeros(max(bb, 1), dtype=np.int64)
    gap = np.zeros(1, dtype=np.float64)
    ns = lib.orc_tournament(_ptr(Xf, ctypes.c_double), l, nc, pos0, bb, gs, fanin, _ptr(sel, ctypes.c_int64),
                            _ptr(gap, ctypes.c_double))
    if ns < 0:
        raise ValueError("orc_tournament: invalid arguments")
    return sel[:ns], float(gap[0])


def rqrcp(A: np.ndarray, k: int, b: int, p: int, Omega: np.ndarray, formula: int = 4,
          sketch_bf16: bool = False, tgs=None, fanin: int = 4) -> RQRCPResult:
    """Alg. 2 (RQRCP) with the sketch Omega given explicitly (l x m, l = b + p).

    formula=4 updates B with Eq. (4) (Duersch-Gu), formula=5 with Eq. (5) (Martinsson et al.).
    sketch_bf16: the mixed form's BF16 sketch (Omega and A rounded to FP32 then BF16 for the
    initial B = Omega A only; exact products and FP64 sums).
    tgs: None for the partial QRCP of Alg. 2; else QR with tournament pivoting on B, tgs[q] the
    leaf group size of block q (an int gives every block the same size) with fan-in `fanin`.
    """
    lib = _load()
    Af = _fortran64(A)
    m, n = Af.shape
    l = b + p
    Om = np.ascontiguousarray(Omega, dtype=np.float64)
    if Om.shape != (l, m):
        raise ValueError(f"Omega must be {l}x{m}, got {Om.shape}")
    jpvt = np.zeros(n, dtype=np.int32)
    tau = np.zeros(max(k, 1), dtype=np.float64)
    rank = np.zeros(1, dtype=np.int64)
    gaps = np.zeros(max(k, 1), dtype=np.float64)
    B = np.zeros((l, n), dtype=np.float64, order="F")
    nblk = (k + b - 1) // b
    if tgs is None:
        tg = None
        tgp = ctypes.POINTER(ctypes.c_int64)()
    else:
        tg = np.array([tgs] * nblk if np.isscalar(tgs) else list(tgs), dtype=np.int64)
        if tg.shape != (nblk,):
            raise ValueError(f"tgs needs {nblk} group sizes")
        tgp = _ptr(tg, ctypes.c_int64)
    rc = lib.orc_rqrcp3(m, n, _ptr(Af, ctypes.c_double), max(m, 1), k, b, p, _ptr(Om, ctypes.c_double),
                        formula, 1 if sketch_bf16 else 0, tgp, fanin, _ptr(jpvt, ctypes.c_int32),
                        _ptr(tau, ctypes.c_double), _ptr(rank, ctypes.c_int64), _ptr(gaps, ctypes.c_double),
                        _ptr(B, ctypes.c_double))
    if rc != 0:
        raise ValueError(f"orc_rqrcp: error {rc}")
    return RQRCPResult(Af, jpvt, tau[:k], int(rank[0]), gaps[:k], B)


def rqrcp_seeded(A: np.ndarray, k: int, b: int, p: int, seed: int, formula: int = 4,
                 sketch_bf16: bool = False, tgs=None, fanin: int = 4) -> RQRCPResult:
    """Alg. 2 with Omega drawn from the seed by the oracle's own Philox generator."""
    return rqrcp(A, k, b, p, omega(b + p, A.shape[0], seed), formula, sketch_bf16, tgs, fanin)


# --------------------------------------------------------------------------- Alg. 3
class SRQRResult:
    def __init__(self, R, jpvt, swaps, g2, alpha, l, rank):
        self.R, self.jpvt, self.swaps, self.g2, self.alpha, self.l, self.rank = R, jpvt, swaps, g2, alpha, l, rank


def srqr(A: np.ndarray, l: int, b: int, p: int, Omega: np.ndarray, g: float = 5.0, d: int = 8,
         seed_g: int = 0, max_swaps: int = 1000) -> SRQRResult:
    """Alg. 3 (SRQR): RQRCP to rank l with the sketch Omega ((b+p) x m), the extra pivot, the
    randomized g_2 estimate (d x (l+1) Gaussian matrices from seeds seed_g, seed_g+1, ...) and
    the swap loop while g_2 > g.  Returns the explicit R (m x n), jpvt, the swap count, the last
    g_2 estimate, |alpha| = |R(l, l)| and the RQRCP stage's rank (the swap loop is skipped when
    its rank guard fired before l pivots)."""
    lib = _load()
    A64 = _fortran64(A)
    m, n = A64.shape
    Om = np.ascontiguousarray(Omega, dtype=np.float64)
    if Om.shape != (b + p, m):
        raise ValueError(f"Omega must be {b + p}x{m}, got {Om.shape}")
    R = np.zeros((m, n), dtype=np.float64, order="F")
    jpvt = np.zeros(n, dtype=np.int32)
    swaps = np.zeros(1, dtype=np.int64)
    g2 = np.zeros(1, dtype=np.float64)
    alpha = np.zeros(1, dtype=np.float64)
    rank = np.zeros(1, dtype=np.int64)
    rc = lib.orc_srqr(m, n, _ptr(A64, ctypes.c_double), m, l, b, p, _ptr(Om, ctypes.c_double), float(g), d,
                      seed_g, max_swaps, _ptr(R, ctypes.c_double), _ptr(jpvt, ctypes.c_int32),
                      _ptr(swaps, ctypes.c_int64), _ptr(g2, ctypes.c_double), _ptr(alpha, ctypes.c_double),
                      _ptr(rank, ctypes.c_int64))
    if rc != 0:
        raise ValueError(f"orc_srqr: error {rc}")
    return SRQRResult(R, jpvt, int(swaps[0]), float(g2[0]), float(alpha[0]), l, int(rank[0]))


def round_bf16(x: np.ndarray) -> np.ndarray:
    """Each element rounded to FP32, then to BF16 (round to nearest, ties to even), as FP64."""
    lib = _load()
    xa = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(xa)
    lib.orc_round_bf16(xa.size, _ptr(xa, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


# --------------------------------------------------------------------------- Q, R, low rank
def form_q(Af: np.ndarray, tau: np.ndarray, k: int, ncols: int) -> np.ndarray:
    """First ncols columns of Q = H_0 ... H_{k-1} (Alg. 2 output)."""
    lib = _load()
    A = np.asfortranarray(Af, dtype=np.float64)
    t = np.ascontiguousarray(tau, dtype=np.float64)
    m = A.shape[0]
    Q = np.zeros((m, ncols), dtype=np.float64, order="F")
    lib.orc_form_q(m, k, _ptr(A, ctypes.c_double), m, _ptr(t, ctypes.c_double), ncols,
                   _ptr(Q, ctypes.c_double), m)
    return Q


def apply_q(Af: np.ndarray, tau: np.ndarray, k: int, x: np.ndarray) -> np.ndarray:
    """Q x = H_0 ... H_{k-1} x for one vector (reflectors read from the factored array)."""
    lib = _load()
    A = np.asfortranarray(Af, dtype=np.float64)
    t = np.ascontiguousarray(tau, dtype=np.float64)
    y = np.array(x, dtype=np.float64, copy=True)
    lib.orc_apply_q(A.shape[0], k, _ptr(A, ctypes.c_double), A.shape[0], _ptr(t, ctypes.c_double),
                    _ptr(y, ctypes.c_double))
    return y


def sketch(A: np.ndarray, Omega: np.ndarray) -> np.ndarray:
    """B = Omega A (Alg. 2), the plain definition."""
    return np.asarray(Omega, dtype=np.float64) @ np.asarray(A, dtype=np.float64)


def r_factor(Af: np.ndarray, k: int) -> np.ndarray:
    """R of A*Pi = Q R: the factored array with the reflector tails of columns 0..k-1 zeroed.
    Rows k..m-1 of columns k..n-1 hold R22 (the updated trailing block)."""
    R = np.array(Af, dtype=np.float64, copy=True)
    for j in range(k):
        R[j + 1:, j] = 0.0
    return R


def lowrank(Af: np.ndarray, tau: np.ndarray, jpvt: np.ndarray, k: int):
    """L = Q1 [R11 R12] Pi^T (Sec. I-A) and Q1."""
    lib = _load()
    A = np.asfortranarray(Af, dtype=np.float64)
    m, n = A.shape
    t = np.ascontiguousarray(tau, dtype=np.float64)
    jp = np.ascontiguousarray(jpvt, dtype=np.int32)
    L = np.zeros((m, n), dtype=np.float64, order="F")
    Q1 = np.zeros((m, k), dtype=np.float64, order="F")
    rc = lib.orc_lowrank(m, n, k, _ptr(A, ctypes.c_double), m, _ptr(t, ctypes.c_double),
                         _ptr(jp, ctypes.c_int32), _ptr(L, ctypes.c_double), m, _ptr(Q1, ctypes.c_double))
    if rc != 0:
        raise MemoryError("orc_lowrank")
    return L, Q1


def rel_residual(A0: np.ndarray, Af: np.ndarray, tau: np.ndarray, jpvt: np.ndarray, k: int) -> float:
    """||A Pi - Q R||_F / ||A||_F with Q the full m x m product and R including R22."""
    m = A0.shape[0]
    Q = form_q(Af, tau, k, m)
    R = r_factor(Af, k)
    AP = np.asarray(A0, dtype=np.float64)[:, jpvt]
    return float(np.linalg.norm(AP - Q @ R) / np.linalg.norm(A0))


def orth_error(Q1: np.ndarray) -> float:
    """||Q1^T Q1 - I||_F."""
    k = Q1.shape[1]
    return float(np.linalg.norm(Q1.T @ Q1 - np.eye(k)))


# --------------------------------------------------------------------------- Theorem 1
def p_min(n: int, k: int, eps: float, delta: float) -> int:
    """Theorem 1 oversampling bound: p >= ceil(4/(eps^2 - eps^3) * log(2nk/delta)) - 1."""
    return int(math.ceil(4.0 / (eps * eps - eps ** 3) * math.log(2.0 * n * k / delta))) - 1


# --------------------------------------------------------------------------- FP64 CholQR
def cholqr_reorth(Q1: np.ndarray, Rk: np.ndarray):
    """One CholQR pass: G = Q1^T Q1, S = chol(G) (upper), Q1 <- Q1 S^{-1}, [R11 R12] <- S [R11 R12].
    Keeps Q1 [R11 R12] unchanged in exact arithmetic while restoring orthogonality of Q1."""
    import scipy.linalg as sla
    G = Q1.T @ Q1
    S = np.linalg.cholesky(G).T
    Qn = sla.solve_triangular(S, Q1.T, trans="T", lower=False).T
    return Qn, S @ Rk


# --------------------------------------------------------------------------- gradient
def truncated_qr_adjoint(X: np.ndarray, Q1: np.ndarray, R11: np.ndarray, R12: np.ndarray,
                         dQ1: np.ndarray, dR11: np.ndarray, dR12: np.ndarray) -> np.ndarray:
    """Adjoint of the truncated QR X Pi = [X1 X2], X1 = Q1 R11, R12 = Q1^T X2 with Pi fixed.

    Returns dX (same column order as X Pi).  Thin-QR adjoint extended to the wide block:
      dX2 = Q1 dR12;  dQ' = dQ1 + X2 dR12^T;  M = R11 dR11^T - dQ'^T Q1;
      dX1 = (dQ' + Q1 copyltu(M)) R11^{-T},  copyltu(M) = tril(M) + tril(M,-1)^T.
    """
    import scipy.linalg as sla
    k = Q1.shape[1]
    X2 = X[:, k:]
    dX2 = Q1 @ dR12
    dQp = dQ1 + X2 @ dR12.T
    M = R11 @ dR11.T - dQp.T @ Q1
    C = np.tril(M) + np.tril(M, -1).T
    rhs = dQp + Q1 @ C
    dX1 = sla.solve_triangular(R11, rhs.T, trans="N", lower=False).T  # rhs R11^{-T}
    return np.concatenate([dX1, dX2], axis=1)


def truncated_qr_forward(X: np.ndarray, k: int):
    """Unpivoted thin QR of the first k columns of X (already permuted), R12 = Q1^T X2.
    Uses the oracle's own Householder QR so signs follow the xLARFG convention."""
    Af, jp, tau = _householder_qr_nopivot(X[:, :k])
    Q1 = form_q(Af, tau, k, k)
    R11 = np.triu(Af[:k, :k])
    R12 = Q1.T @ X[:, k:]
    return Q1, R11, R12


def _householder_qr_nopivot(X1: np.ndarray):
    """Unpivoted Householder QR of X1 (the panel step of Alg. 2), reflector by reflector,
    each applied to the columns on its right.  Returns (factored X1, identity jpvt, tau)."""
    m, k = X1.shape
    A = _fortran64(X1)
    tau = np.zeros(k)
    for j in range(k):
        x = A[j:, j]
        tau[j] = _house_gen_py(x)
        A[j:, j] = x
        for s in range(j + 1, k):
            y = A[j:, s]
            if tau[j] != 0.0:
                v = np.concatenate([[1.0], x[1:]])
                y = y - tau[j] * v * (v @ y)
            A[j:, s] = y
    return A, np.arange(k, dtype=np.int32), tau


def _house_gen_py(x: np.ndarray) -> float:
    """xLARFG convention reflector (as in rqrcp_oracle.c), in place on x; returns tau."""
    if x.shape[0] <= 1:
        return 0.0
    ss = float(np.sum(x[1:] * x[1:]))
    if ss == 0.0:
        return 0.0
    alpha = float(x[0])
    nrm = math.sqrt(alpha * alpha + ss)
    beta = -nrm if alpha >= 0.0 else nrm
    tau = (beta - alpha) / beta
    x[1:] *= 1.0 / (alpha - beta)
    x[0] = beta
    return tau


def truncated_loss(A: np.ndarray, jpvt: np.ndarray, k: int) -> float:
    """L = ||A - Q1 [R11 R12] Pi^T||_F^2 for fixed Pi (the projection residual of X2)."""
    X = A[:, jpvt]
    Q1, R11, R12 = truncated_qr_forward(X, k)
    E = X - Q1 @ np.concatenate([R11, R12], axis=1)
    return float(np.sum(E * E))


def truncated_loss_grad(A: np.ndarray, jpvt: np.ndarray, k: int) -> np.ndarray:
    """Closed form: L = ||P_perp X2||_F^2, dL/dX2 = 2 P_perp X2, dL/dX1 = -2 P_perp X2 R12^T R11^{-T},
    dA = [dX1 dX2] Pi^T."""
    import scipy.linalg as sla
    X = A[:, jpvt]
    Q1, R11, R12 = truncated_qr_forward(X, k)
    X2 = X[:, k:]
    P = X2 - Q1 @ (Q1.T @ X2)
    dX2 = 2.0 * P
    dX1 = sla.solve_triangular(R11, (-2.0 * P @ R12.T).T, trans="N", lower=False).T
    dX = np.concatenate([dX1, dX2], axis=1)
    dA = np.empty_like(dX)
    dA[:, jpvt] = dX
    return dA
