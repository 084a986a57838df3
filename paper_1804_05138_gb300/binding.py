"""ctypes binding of librqrcp (include/rqrcp.h): argument marshalling only.

Functions named ``rqrcp_*`` mirror the C entry points one to one and take torch CUDA
tensors for the device pointers (column-major matrices are tensors of shape (m, n) with
stride (1, ld)).  ``factor``/``factor_mixed``/``lowrank`` add workspace allocation through
torch and status checking.  There is no fallback: if the library is missing or no GPU is
present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from dataclasses import dataclass

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librqrcp.so")

RQRCP_OK = 0
RQRCP_ERR_CUDA = 1
RQRCP_ERR_NONFINITE = 2
RQRCP_ERR_TIMEOUT = 3
RQRCP_ERR_WORKSPACE = 4
RQRCP_ERR_UNSUPPORTED = 5
RQRCP_PREC_FP64 = 0
RQRCP_PREC_MIXED = 1
RQRCP_SKETCH_BF16 = 0
RQRCP_SKETCH_FP32 = 1
RQRCP_UPDATE_EQ4 = 4
RQRCP_UPDATE_EQ5 = 5

# Every symbol include/rqrcp.h declares.
ABI_SYMBOLS = (
    "rqrcp_error_string", "rqrcp_workspace_size", "rqrcp_generate_omega_host", "rqrcp_generate_omega",
    "rqrcp_generate_omega_f32",
    "rqrcp_sketch", "rqrcp_factor", "rqrcp_factor_with_omega", "rqrcp_factor_mixed", "rqrcp_factor_mixed_ex",
    "rqrcp_read_status", "rqrcp_lowrank_workspace_size", "rqrcp_lowrank",
    "rqrcp_profile_begin", "rqrcp_profile_end", "rqrcp_profile_class_name",
    "rqrcp_sketch_noalloc", "rqrcp_lowrank_f32", "rqrcp_backward_workspace_size", "rqrcp_backward",
    "rqrcp_backward_f32", "rqrcp_reorth_workspace_size", "rqrcp_lowrank_reorth",
    "rqrcp_batched_workspace_size", "rqrcp_factor_batched", "rqrcp_factor_ex",
    "rqrcp_srqr_workspace_size", "rqrcp_srqr", "rqrcp_peak_probe", "rqrcp_factor_tournament",
    "rqrcp_factor_mixed_tournament", "rqrcp_tournament_config",
)
RQRCP_PROFILE_CLASSES = 14

_lock = threading.Lock()
_lib = None

_i64, _u64, _vp, _sz = ctypes.c_int64, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_size_t


class RQRCPError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {code} ({error_string(code)})")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librqrcp.so (built by paper_1804_05138_gb300.build) and declare its signatures."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(path):
            raise RuntimeError(f"librqrcp.so not built ({path}); run paper_1804_05138_gb300.build.build()")
        lib = ctypes.CDLL(path)
        sig = {
            "rqrcp_error_string": (ctypes.c_char_p, [ctypes.c_int]),
            "rqrcp_workspace_size": (_sz, [_i64, _i64, _i64, _i64, _i64, ctypes.c_int]),
            "rqrcp_generate_omega_host": (ctypes.c_int, [_i64, _i64, _u64, _vp, _i64]),
            "rqrcp_generate_omega": (ctypes.c_int, [_i64, _i64, _u64, _vp, _i64, _vp]),
            "rqrcp_generate_omega_f32": (ctypes.c_int, [_i64, _i64, _u64, _vp, _i64, _vp]),
            "rqrcp_sketch": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp, _sz, _vp]),
            "rqrcp_factor": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _u64, _vp, _vp, _vp, _vp, _sz,
                                            _vp]),
            "rqrcp_factor_with_omega": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _vp, _i64, _vp,
                                                       _vp, _vp, _vp, _sz, _vp]),
            "rqrcp_factor_ex": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _u64, _vp, _i64, ctypes.c_int,
                                               _vp, _vp, _vp, _vp, _sz, _vp]),
            "rqrcp_srqr_workspace_size": (_sz, [_i64, _i64, _i64, _i64, _i64, _i64]),
            "rqrcp_srqr": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _u64, _vp, _i64, ctypes.c_double,
                                          _i64, _u64, _i64, _vp, ctypes.POINTER(ctypes.c_double), _vp, _sz, _vp]),
            "rqrcp_factor_mixed": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _u64, _vp, _vp, _vp, _vp,
                                                  _sz, _vp]),
            "rqrcp_factor_mixed_ex": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _u64, _vp, _i64,
                                                     ctypes.c_int, _vp, _vp, _vp, _vp, _sz, _vp]),
            "rqrcp_factor_tournament": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _u64, _vp, _i64,
                                                       _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
            "rqrcp_factor_mixed_tournament": (ctypes.c_int, [_i64, _i64, _vp, _i64, _i64, _i64, _i64, _u64, _vp,
                                                             _i64, ctypes.c_int, _i64, _vp, _vp, _vp, _vp, _sz, _vp]),
            "rqrcp_tournament_config": (ctypes.c_int, [_i64, _i64, _i64, _i64, ctypes.c_int, _i64,
                                                       ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
            "rqrcp_read_status": (ctypes.c_int, [_vp, ctypes.POINTER(_i64), _vp]),
            "rqrcp_lowrank_workspace_size": (_sz, [_i64, _i64, _i64]),
            "rqrcp_lowrank": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _vp, _vp, _i64, _vp, _i64, _vp,
                                             _sz, _vp]),
            "rqrcp_profile_begin": (ctypes.c_int, []),
            "rqrcp_profile_end": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_i64),
                                                 ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                                 ctypes.POINTER(ctypes.c_double)]),
            "rqrcp_profile_class_name": (ctypes.c_char_p, [ctypes.c_int]),
            "rqrcp_peak_probe": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                ctypes.POINTER(ctypes.c_double), _vp]),
            "rqrcp_sketch_noalloc": (ctypes.c_int, [_i64, _i64, _vp, _i64, _vp, _i64, _i64, _vp, _i64, _vp]),
            "rqrcp_lowrank_f32": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _vp, _vp, _i64, _vp, _i64, _vp,
                                                 _sz, _vp]),
            "rqrcp_backward_workspace_size": (_sz, [_i64, _i64, _i64, ctypes.c_int]),
            "rqrcp_reorth_workspace_size": (_sz, [_i64, _i64, _i64]),
            "rqrcp_batched_workspace_size": (_sz, [_i64, _i64, _i64, _i64]),
            "rqrcp_factor_batched": (ctypes.c_int, [_i64, _vp, _vp, _i64, _i64, _i64, _i64, _vp, _i64, _vp, _sz,
                                                    _vp]),
            "rqrcp_lowrank_reorth": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64,
                                                    ctypes.c_double, _vp, _vp, _sz, _vp]),
            "rqrcp_backward": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _i64,
                                              _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
            "rqrcp_backward_f32": (ctypes.c_int, [_i64, _i64, _i64, _vp, _i64, _vp, _vp, _i64, _vp, _i64, _vp, _i64,
                                                  _vp, _i64, _vp, _i64, _vp, _sz, _vp]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def error_string(code: int) -> str:
    return load().rqrcp_error_string(int(code)).decode()


# --------------------------------------------------------------------------- tensor helpers
def _ptr(t) -> int | None:
    return None if t is None else int(t.data_ptr())


def _ld(t) -> int:
    """Leading dimension of a column-major (m, n) tensor."""
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("expected a column-major 2-D tensor (stride(0) == 1)")
    return max(int(t.stride(1)), int(t.shape[0]), 1)


def _ld_rowmajor(t) -> int:
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError("expected a row-major 2-D tensor (stride(1) == 1)")
    return max(int(t.stride(0)), int(t.shape[1]), 1)


def _stream(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def colmajor(A):
    """Column-major copy (or view) of a 2-D tensor: shape (m, n), stride (1, m)."""
    if A.dim() == 2 and A.stride(0) == 1 and A.stride(1) >= A.shape[0]:
        return A
    return A.t().contiguous().t()


def _check(code: int, where: str):
    if code != RQRCP_OK:
        raise RQRCPError(code, where)


def workspace(nbytes: int, device):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# --------------------------------------------------------------------------- 1:1 entry points
def rqrcp_workspace_size(m, n, k, b, p, precision=RQRCP_PREC_FP64) -> int:
    return int(load().rqrcp_workspace_size(m, n, k, b, p, precision))


def rqrcp_lowrank_workspace_size(m, n, k) -> int:
    return int(load().rqrcp_lowrank_workspace_size(m, n, k))


def rqrcp_generate_omega_host(l, m, seed):
    """The library's host draw of Omega (l x m, row-major float64 numpy array)."""
    import numpy as np
    out = np.empty((l, m), dtype=np.float64)
    _check(load().rqrcp_generate_omega_host(l, m, seed, out.ctypes.data, m), "rqrcp_generate_omega_host")
    return out


def rqrcp_generate_omega(l, m, seed, Omega, stream=None) -> int:
    fn = load().rqrcp_generate_omega if Omega.element_size() == 8 else load().rqrcp_generate_omega_f32
    return fn(l, m, seed, _ptr(Omega), _ld_rowmajor(Omega), _stream(stream))


def rqrcp_sketch(A, Omega, B, work, stream=None) -> int:
    m, n = A.shape
    l = Omega.shape[0]
    return load().rqrcp_sketch(m, n, _ptr(A), _ld(A), _ptr(Omega), l, _ld_rowmajor(Omega), _ptr(B), _ld(B),
                               _ptr(work), work.numel(), _stream(stream))


def rqrcp_sketch_noalloc(A, Omega, B, stream=None) -> int:
    """B = Omega A with the library's fixed device scratch (no workspace argument)."""
    m, n = A.shape
    l = Omega.shape[0]
    return load().rqrcp_sketch_noalloc(m, n, _ptr(A), _ld(A), _ptr(Omega), l, _ld_rowmajor(Omega), _ptr(B),
                                       _ld(B), _stream(stream))


def rqrcp_factor(A, k, b, p, seed, jpvt, tau, work, stream=None, rank_out=None) -> int:
    """rank_out: optional int64 CUDA tensor of one element that receives the rank."""
    m, n = A.shape
    return load().rqrcp_factor(m, n, _ptr(A), _ld(A), k, b, p, seed, _ptr(jpvt), _ptr(tau), _ptr(rank_out),
                               _ptr(work), work.numel(), _stream(stream))


def rqrcp_factor_with_omega(A, k, b, p, Omega, jpvt, tau, work, stream=None, rank_out=None) -> int:
    m, n = A.shape
    return load().rqrcp_factor_with_omega(m, n, _ptr(A), _ld(A), k, b, p, _ptr(Omega), _ld_rowmajor(Omega),
                                          _ptr(jpvt), _ptr(tau), _ptr(rank_out), _ptr(work), work.numel(),
                                          _stream(stream))


def rqrcp_factor_ex(A, k, b, p, seed, Omega, formula, jpvt, tau, work, stream=None, rank_out=None) -> int:
    m, n = A.shape
    om, ldo = (None, 0) if Omega is None else (_ptr(Omega), _ld_rowmajor(Omega))
    return load().rqrcp_factor_ex(m, n, _ptr(A), _ld(A), k, b, p, seed, om, ldo, formula, _ptr(jpvt), _ptr(tau),
                                  _ptr(rank_out), _ptr(work), work.numel(), _stream(stream))


def rqrcp_factor_mixed(A, k, b, p, seed, jpvt, tau, work, stream=None, rank_out=None) -> int:
    m, n = A.shape
    return load().rqrcp_factor_mixed(m, n, _ptr(A), _ld(A), k, b, p, seed, _ptr(jpvt), _ptr(tau), _ptr(rank_out),
                                     _ptr(work), work.numel(), _stream(stream))


def rqrcp_factor_mixed_ex(A, k, b, p, seed, sketch, jpvt, tau, work, stream=None, Omega=None,
                          rank_out=None) -> int:
    """Omega: optional row-major float32 CUDA tensor ((b+p) x m) replacing the seeded sketch."""
    m, n = A.shape
    om, ldo = (None, 0) if Omega is None else (_ptr(Omega), _ld_rowmajor(Omega))
    return load().rqrcp_factor_mixed_ex(m, n, _ptr(A), _ld(A), k, b, p, seed, om, ldo, sketch, _ptr(jpvt),
                                        _ptr(tau), _ptr(rank_out), _ptr(work), work.numel(), _stream(stream))


def rqrcp_factor_tournament(A, k, b, p, seed, Omega, group_cols, jpvt, tau, work, stream=None,
                            rank_out=None) -> int:
    m, n = A.shape
    om, ldo = (None, 0) if Omega is None else (_ptr(Omega), _ld_rowmajor(Omega))
    return load().rqrcp_factor_tournament(m, n, _ptr(A), _ld(A), k, b, p, seed, om, ldo, group_cols, _ptr(jpvt),
                                          _ptr(tau), _ptr(rank_out), _ptr(work), work.numel(), _stream(stream))


def rqrcp_factor_mixed_tournament(A, k, b, p, seed, sketch, group_cols, jpvt, tau, work, stream=None, Omega=None,
                                  rank_out=None) -> int:
    m, n = A.shape
    om, ldo = (None, 0) if Omega is None else (_ptr(Omega), _ld_rowmajor(Omega))
    return load().rqrcp_factor_mixed_tournament(m, n, _ptr(A), _ld(A), k, b, p, seed, om, ldo, sketch, group_cols,
                                                _ptr(jpvt), _ptr(tau), _ptr(rank_out), _ptr(work), work.numel(),
                                                _stream(stream))


def rqrcp_tournament_config(ncols, bb, b, p, elem_bytes, group_cols=0) -> tuple[int, int]:
    """(leaf group size, fan-in) that the tournament entry points use for one block."""
    g, f = _i64(0), _i64(0)
    _check(load().rqrcp_tournament_config(ncols, bb, b, p, elem_bytes, group_cols, ctypes.byref(g), ctypes.byref(f)),
           "rqrcp_tournament_config")
    return int(g.value), int(f.value)


def rqrcp_read_status(work, stream=None) -> tuple[int, int]:
    rank = _i64(0)
    code = load().rqrcp_read_status(_ptr(work), ctypes.byref(rank), _stream(stream))
    return int(code), int(rank.value)


def rqrcp_lowrank(Afact, k, tau, jpvt, L, Q1, work, stream=None) -> int:
    """L may be None (only Q1 is formed).  Dispatches on Afact's dtype (FP64 or FP32 twin)."""
    m, n = Afact.shape
    fn = load().rqrcp_lowrank if Afact.element_size() == 8 else load().rqrcp_lowrank_f32
    return fn(m, n, k, _ptr(Afact), _ld(Afact), _ptr(tau), _ptr(jpvt), _ptr(L), _ld(L) if L is not None else m,
              _ptr(Q1), _ld(Q1), _ptr(work), work.numel(), _stream(stream))


def rqrcp_reorth_workspace_size(m, n, k) -> int:
    return int(load().rqrcp_reorth_workspace_size(m, n, k))


def rqrcp_lowrank_reorth(Afact, k, tau, Q1, R, tol, orth, work, stream=None) -> int:
    """FP64 Q1 (m x k) and R (k x n) from a mixed factorization; CholQR pass when ||Q1^T Q1 - I||_F > tol."""
    m, n = Afact.shape
    return load().rqrcp_lowrank_reorth(m, n, k, _ptr(Afact), _ld(Afact), _ptr(tau), _ptr(Q1), _ld(Q1), _ptr(R),
                                       _ld(R), float(tol), _ptr(orth), _ptr(work), work.numel(), _stream(stream))


def rqrcp_batched_workspace_size(m_max, n_max, b_max, p) -> int:
    return int(load().rqrcp_batched_workspace_size(m_max, n_max, b_max, p))


def rqrcp_factor_batched(count, descs, order, m_max, n_max, b_max, p, Omega, work, stream=None) -> int:
    """descs: device uint8 tensor of count x 72-byte descriptors; order: device int32 tensor; Omega: row-major
    float32 CUDA tensor of at least (b_max + p) x m_max."""
    return load().rqrcp_factor_batched(count, _ptr(descs), _ptr(order), m_max, n_max, b_max, p, _ptr(Omega),
                                       _ld_rowmajor(Omega), _ptr(work), work.numel(), _stream(stream))


BATCH_DESC_BYTES = 72


RQRCP_TILES_UPDATE_SIMT, RQRCP_TILES_UPDATE_TC, RQRCP_TILES_SKETCH_SIMT, RQRCP_TILES_GRAM_RT64 = 1, 2, 4, 8


def batch_descriptors(mats, jpvts, taus, ranks, ks, bs, tiles=None):
    """Pack the 72-byte descriptors (layout of include/rqrcp.h) into a host uint8 array."""
    import numpy as np
    dt = np.dtype([("A", "<u8"), ("jpvt", "<u8"), ("tau", "<u8"), ("rank", "<u8"), ("m", "<i8"), ("n", "<i8"),
                   ("k", "<i8"), ("lda", "<i8"), ("b", "<i4"), ("tiles", "<i4")])
    assert dt.itemsize == BATCH_DESC_BYTES
    tiles = [0] * len(mats) if tiles is None else list(tiles)
    rec = np.zeros(len(mats), dtype=dt)
    for i, (A, jp, tu, rk, k, b, t) in enumerate(zip(mats, jpvts, taus, ranks, ks, bs, tiles)):
        rec[i] = (A.data_ptr(), jp.data_ptr(), tu.data_ptr(), rk.data_ptr(), A.shape[0], A.shape[1], k, _ld(A), b, t)
    return rec.view(np.uint8)


def batch_cost(m, n, k, b, p):
    """Counted flops of one RQRCP (sketch + Householder QR to rank k): the order key."""
    l = b + p
    return 2.0 * l * m * n + 4.0 * m * n * k - 2.0 * (m + n) * k * k + 4.0 * k ** 3 / 3.0


class Batch:
    """Prepared batched call: descriptors, order and workspace on the device; `run()` enqueues it."""

    def __init__(self, mats, ks, bs, p=8, seed=0, tiles=None):
        import numpy as np
        import torch
        self.mats = [colmajor(A) for A in mats]
        dev = self.mats[0].device
        self.ks, self.bs, self.p, self.seed = list(ks), list(bs), p, seed
        self.tiles = [0] * len(self.mats) if tiles is None else [int(t) for t in tiles]
        self.jpvts = [torch.empty(A.shape[1], dtype=torch.int32, device=dev) for A in self.mats]
        self.taus = [torch.empty(k, dtype=torch.float64, device=dev) for k in self.ks]
        self.ranks = torch.zeros(len(self.mats), dtype=torch.int64, device=dev)
        rank_views = [self.ranks[i:i + 1] for i in range(len(self.mats))]
        host = batch_descriptors(self.mats, self.jpvts, self.taus, rank_views, self.ks, self.bs, self.tiles)
        self.descs = torch.from_numpy(host.copy()).to(dev)
        cost = [batch_cost(A.shape[0], A.shape[1], k, b, p) for A, k, b in zip(self.mats, self.ks, self.bs)]
        self.order = torch.from_numpy(np.argsort(-np.asarray(cost), kind="stable").astype(np.int32)).to(dev)
        self.m_max = max(A.shape[0] for A in self.mats)
        self.n_max = max(A.shape[1] for A in self.mats)
        self.b_max = max(self.bs)
        need = rqrcp_batched_workspace_size(self.m_max, self.n_max, self.b_max, p)
        if need == 0:
            raise ValueError("invalid batch limits")
        self.work = workspace(need, dev)
        self.flops = float(sum(cost))
        # the shared sketching matrix, drawn once from the seed (host draw, one copy)
        self.omega = torch.empty((self.b_max + p, self.m_max), dtype=torch.float32, device=dev)
        _check(rqrcp_generate_omega(self.b_max + p, self.m_max, seed, self.omega), "rqrcp_generate_omega_f32")

    def run(self, stream=None) -> int:
        return rqrcp_factor_batched(len(self.mats), self.descs, self.order, self.m_max, self.n_max, self.b_max,
                                    self.p, self.omega, self.work, stream)


def rqrcp_backward_workspace_size(m, n, k, precision=RQRCP_PREC_FP64) -> int:
    return int(load().rqrcp_backward_workspace_size(m, n, k, precision))


def rqrcp_backward(A, jpvt, Q1, R, dQ1, dR, dA, work, stream=None) -> int:
    """dA from the upstream gradients of (Q1, R); dispatches on dtype (FP64 or FP32 twin)."""
    m, n = A.shape
    k = Q1.shape[1]
    fn = load().rqrcp_backward if A.element_size() == 8 else load().rqrcp_backward_f32
    return fn(m, n, k, _ptr(A), _ld(A), _ptr(jpvt), _ptr(Q1), _ld(Q1), _ptr(R), _ld(R), _ptr(dQ1), _ld(dQ1),
              _ptr(dR), _ld(dR), _ptr(dA), _ld(dA), _ptr(work), work.numel(), _stream(stream))


RQRCP_PROBE_DFMA, RQRCP_PROBE_FFMA, RQRCP_PROBE_TC_TF32, RQRCP_PROBE_TC_BF16 = 0, 1, 2, 3


def rqrcp_peak_probe(kind, stream=None) -> tuple[float, float]:
    """(TFLOP/s, ms) of one timed launch of the probe `kind` (RQRCP_PROBE_*)."""
    tf, ms = ctypes.c_double(0.0), ctypes.c_double(0.0)
    _check(load().rqrcp_peak_probe(int(kind), ctypes.byref(tf), ctypes.byref(ms), _stream(stream)),
           "rqrcp_peak_probe")
    return float(tf.value), float(ms.value)


def rqrcp_profile_begin() -> int:
    return int(load().rqrcp_profile_begin())


def rqrcp_profile_end() -> dict:
    """Per kernel class: {name: {"launches", "ms", "flops", "bytes"}} since rqrcp_profile_begin."""
    n = RQRCP_PROFILE_CLASSES
    launches = (_i64 * n)()
    ms = (ctypes.c_double * n)()
    fl = (ctypes.c_double * n)()
    by = (ctypes.c_double * n)()
    _check(load().rqrcp_profile_end(n, launches, ms, fl, by), "rqrcp_profile_end")
    out = {}
    for c in range(n):
        name = load().rqrcp_profile_class_name(c).decode()
        out[name] = {"launches": int(launches[c]), "ms": float(ms[c]), "flops": float(fl[c]), "bytes": float(by[c])}
    return out


# --------------------------------------------------------------------------- convenience layer
@dataclass
class Factorization:
    A: object      # factored matrix (R above the diagonal, reflectors below), column-major
    jpvt: object   # int32 permutation, column c of A*Pi is input column jpvt[c]
    tau: object    # float64 Householder scalars, length k
    rank: int      # pivots chosen before the rank guard fired
    k: int


def _run_factor(A, k, b, p, seed, omega, mixed, work, stream, sketch=RQRCP_SKETCH_BF16, formula=RQRCP_UPDATE_EQ4,
                tournament=None):
    import torch
    m, n = A.shape
    dev = A.device
    jpvt = torch.empty(n, dtype=torch.int32, device=dev)
    tau = torch.empty(k, dtype=torch.float64, device=dev)
    need = rqrcp_workspace_size(m, n, k, b, p, RQRCP_PREC_MIXED if mixed else RQRCP_PREC_FP64)
    if need == 0:
        raise ValueError("invalid factorization arguments")
    if work is None or work.numel() < need:
        work = workspace(need, dev)
    if tournament is not None:
        if mixed:
            code = rqrcp_factor_mixed_tournament(A, k, b, p, seed, sketch, tournament, jpvt, tau, work, stream,
                                                 Omega=omega)
        else:
            code = rqrcp_factor_tournament(A, k, b, p, seed, omega, tournament, jpvt, tau, work, stream)
    elif mixed:
        code = rqrcp_factor_mixed_ex(A, k, b, p, seed, sketch, jpvt, tau, work, stream, Omega=omega)
    elif formula != RQRCP_UPDATE_EQ4:
        code = rqrcp_factor_ex(A, k, b, p, seed, omega, formula, jpvt, tau, work, stream)
    elif omega is None:
        code = rqrcp_factor(A, k, b, p, seed, jpvt, tau, work, stream)
    else:
        code = rqrcp_factor_with_omega(A, k, b, p, omega, jpvt, tau, work, stream)
    _check(code, "rqrcp_factor_mixed" if mixed else "rqrcp_factor")
    status, rank = rqrcp_read_status(work, stream)
    _check(status, "device status")
    return Factorization(A, jpvt, tau, rank, k)


def factor(A, k: int, b: int = 64, p: int = 8, seed: int = 0, omega=None, work=None, stream=None,
           overwrite: bool = False, formula: int = 4, tournament=None) -> Factorization:
    """Randomized QRCP of a float64 CUDA matrix (plain FP64 form).  ``omega`` (row-major
    (b+p) x m float64 CUDA tensor) replaces the seeded sketch when given.  ``formula``: 4 updates
    the sketch between blocks with Eq. (4) (Duersch-Gu), 5 with Eq. (5) (Martinsson et al.).
    ``tournament``: None for Alg. 2's partial QRCP on B, else QR with tournament pivoting on B
    with that leaf group size (0: automatic; rqrcp_factor_tournament)."""
    import torch
    if A.dtype != torch.float64:
        raise TypeError("factor expects float64; use factor_mixed for float32")
    Acm = colmajor(A)
    if not overwrite:
        Acm = Acm.t().clone().t()
    if formula not in (RQRCP_UPDATE_EQ4, RQRCP_UPDATE_EQ5):
        raise ValueError("formula must be 4 or 5")
    if tournament is not None and formula != RQRCP_UPDATE_EQ4:
        raise ValueError("tournament pivoting runs with Eq. (4) only")
    return _run_factor(Acm, k, b, p, seed, omega, False, work, stream, formula=formula, tournament=tournament)


class SRQRFactorization:
    """Output of srqr: R (the overwritten A: explicit, upper trapezoidal in rows 0..l, trailing
    block R22 below), jpvt, the swap count, the last g2 estimate, |alpha| = |R(l, l)| and the
    RQRCP stage's rank."""

    def __init__(self, R, jpvt, l, swaps, g2, alpha, rank):
        self.R, self.jpvt, self.l, self.swaps, self.g2, self.alpha, self.rank = R, jpvt, l, swaps, g2, alpha, rank


def srqr(A, l: int, b: int = 64, p: int = 8, seed: int = 0, omega=None, g: float = 5.0, d: int = 8,
         seed_g: int = 0, max_swaps: int = 1000, work=None, stream=None, overwrite: bool = False) -> SRQRFactorization:
    """Spectrum-revealing QR (Alg. 3) of a float64 CUDA matrix: RQRCP to rank l, the extra pivot,
    the randomized g2 estimate and the swap loop while g2 > g (rqrcp_srqr)."""
    import torch
    if A.dtype != torch.float64:
        raise TypeError("srqr expects float64")
    Acm = colmajor(A)
    if not overwrite:
        Acm = Acm.t().clone().t()
    m, n = Acm.shape
    need = load().rqrcp_srqr_workspace_size(m, n, l, b, p, d)
    if need == 0:
        raise ValueError("invalid srqr arguments")
    if work is None or work.numel() < need:
        work = workspace(need, Acm.device)
    jpvt = torch.empty(n, dtype=torch.int32, device=Acm.device)
    info = (ctypes.c_double * 4)()
    om, ldo = (None, 0) if omega is None else (_ptr(omega), _ld_rowmajor(omega))
    code = load().rqrcp_srqr(m, n, _ptr(Acm), _ld(Acm), l, b, p, seed, om, ldo, float(g), d, seed_g, max_swaps,
                             _ptr(jpvt), info, _ptr(work), work.numel(), _stream(stream))
    _check(code, "rqrcp_srqr")
    return SRQRFactorization(Acm, jpvt, l, int(info[0]), float(info[1]), float(info[2]), int(info[3]))


def factor_mixed(A, k: int, b: int = 64, p: int = 16, seed: int = 0, work=None, stream=None,
                 overwrite: bool = False, sketch: str = "bf16", omega=None, tournament=None) -> Factorization:
    """Randomized QRCP of a float32 CUDA matrix (mixed form, FP64 reflectors).

    sketch: "bf16" (operands rounded to BF16, FP32 accumulation) or "fp32" (FP32-level sketch).
    omega: optional row-major (b+p) x m float32 CUDA tensor replacing the seeded sketch.
    tournament: None, or the leaf group size of QR with tournament pivoting on B (0: automatic).
    """
    import torch
    if A.dtype != torch.float32:
        raise TypeError("factor_mixed expects float32")
    if sketch not in ("bf16", "fp32"):
        raise ValueError("sketch must be 'bf16' or 'fp32'")
    Acm = colmajor(A)
    if not overwrite:
        Acm = Acm.t().clone().t()
    return _run_factor(Acm, k, b, p, seed, omega, True, work, stream,
                       RQRCP_SKETCH_BF16 if sketch == "bf16" else RQRCP_SKETCH_FP32, tournament=tournament)


def lowrank(f: Factorization, stream=None):
    """L = Q1 [R11 R12] Pi^T and Q1 from a factorization (FP64, or FP32 from the mixed form)."""
    import torch
    m, n = f.A.shape
    k = f.k
    dev = f.A.device
    L = torch.empty((n, m), dtype=f.A.dtype, device=dev).t()
    Q1 = torch.empty((k, m), dtype=f.A.dtype, device=dev).t()
    work = workspace(rqrcp_lowrank_workspace_size(m, n, k), dev)
    _check(rqrcp_lowrank(f.A, k, f.tau, f.jpvt, L, Q1, work, stream), "rqrcp_lowrank")
    status, _ = rqrcp_read_status(work, stream)
    _check(status, "device status")
    return L, Q1
