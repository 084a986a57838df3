"""C-ABI checks that need no GPU: the library builds, loads, exports every symbol that
include/rqrcp.h declares, and rejects invalid arguments before touching the device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1804_05138_gb300 import binding, build
    build.build()
    return binding.load()


def _declared_symbols():
    with open(os.path.join(ROOT, "include", "rqrcp.h")) as f:
        text = f.read()
    return sorted(set(re.findall(r"\b(rqrcp_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    from paper_1804_05138_gb300 import binding
    declared = _declared_symbols()
    assert len(declared) >= 10
    for name in declared:
        assert hasattr(lib, name), name
    assert set(binding.ABI_SYMBOLS) == set(declared)


def test_error_strings(lib):
    from paper_1804_05138_gb300 import binding
    for code in range(0, 6):
        assert binding.error_string(code)
    assert "invalid argument" in binding.error_string(-3)


def test_workspace_size_rejects_bad_arguments(lib):
    from paper_1804_05138_gb300 import binding as b
    assert b.rqrcp_workspace_size(0, 10, 1, 4, 2) == 0
    assert b.rqrcp_workspace_size(10, 10, 1, 0, 2) == 0
    assert b.rqrcp_workspace_size(10, 10, 1, 4, -1) == 0
    assert b.rqrcp_workspace_size(10, 10, 1, 4, 2, 7) == 0
    assert b.rqrcp_workspace_size(1000, 1000, 64, 32, 8) > 0
    assert b.rqrcp_workspace_size(1000, 1000, 64, 32, 8, b.RQRCP_PREC_MIXED) > 0
    assert b.rqrcp_lowrank_workspace_size(100, 80, 10) > 0


def test_factor_argument_codes(lib):
    fake = ctypes.c_void_p(0x1000)   # never dereferenced: validation happens first
    f = lib.rqrcp_factor
    #            m    n    A     lda  k   b   p  seed jpvt  tau  rank  work  bytes stream
    assert f(0, 5, fake, 1, 1, 1, 0, 0, fake, fake, None, None, 0, None) == -1
    assert f(5, 0, fake, 5, 1, 1, 0, 0, fake, fake, None, None, 0, None) == -2
    assert f(5, 5, None, 5, 1, 1, 0, 0, fake, fake, None, None, 0, None) == -3
    assert f(5, 5, fake, 4, 1, 1, 0, 0, fake, fake, None, None, 0, None) == -4
    assert f(5, 5, fake, 5, 6, 1, 0, 0, fake, fake, None, None, 0, None) == -5
    assert f(5, 5, fake, 5, 0, 1, 0, 0, fake, fake, None, None, 0, None) == -5
    assert f(5, 5, fake, 5, 2, 0, 0, 0, fake, fake, None, None, 0, None) == -6
    assert f(5, 5, fake, 5, 2, 1, -1, 0, fake, fake, None, None, 0, None) == -7
    assert f(5, 5, fake, 5, 2, 1, 0, 0, None, fake, None, None, 0, None) == -9
    assert f(5, 5, fake, 5, 2, 1, 0, 0, fake, None, None, None, 0, None) == -10
    assert f(5, 5, fake, 5, 2, 1, 0, 0, fake, fake, None, None, 0, None) == 4      # no workspace
    assert f(5, 5, fake, 5, 2, 1, 0, 0, fake, fake, fake, None, 0, None) == 4      # rank_out given
    g = lib.rqrcp_factor_with_omega
    assert g(5, 5, fake, 5, 2, 1, 0, None, 5, fake, fake, None, None, 0, None) == -8
    assert g(5, 5, fake, 5, 2, 1, 0, fake, 4, fake, fake, None, None, 0, None) == -9
    assert g(5, 5, fake, 5, 2, 1, 0, fake, 5, None, fake, None, None, 0, None) == -10
    assert g(5, 5, fake, 5, 2, 1, 0, fake, 5, fake, None, None, None, 0, None) == -11
    h = lib.rqrcp_factor_mixed
    assert h(5, 5, fake, 5, 2, 1, 0, 0, fake, fake, None, fake, 16, None) == 4     # too small
    hx = lib.rqrcp_factor_mixed_ex
    #             m  n  A    lda k  b  p  seed Omega ldo sketch jpvt tau rank work bytes stream
    assert hx(5, 5, fake, 5, 2, 1, 0, 0, fake, 4, 0, fake, fake, None, None, 0, None) == -10
    assert hx(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 2, fake, fake, None, None, 0, None) == -11
    assert hx(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 0, None, fake, None, None, 0, None) == -12
    assert hx(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 1, fake, None, None, None, 0, None) == -13
    assert hx(5, 5, fake, 5, 2, 1, 0, 0, fake, 5, 1, fake, fake, None, None, 0, None) == 4  # no workspace
    x = lib.rqrcp_factor_ex
    #            m  n  A    lda k  b  p  seed Omega ldo formula jpvt tau rank work bytes stream
    assert x(5, 5, None, 5, 2, 1, 0, 0, None, 0, 5, fake, fake, None, None, 0, None) == -3
    assert x(5, 5, fake, 5, 2, 1, 0, 0, fake, 4, 5, fake, fake, None, None, 0, None) == -10
    assert x(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 3, fake, fake, None, None, 0, None) == -11
    assert x(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 5, None, fake, None, None, 0, None) == -12
    assert x(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 5, fake, None, None, None, 0, None) == -13
    assert x(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 5, fake, fake, None, None, 0, None) == 4  # no workspace
    assert x(5, 5, fake, 5, 2, 1, 0, 0, fake, 5, 4, fake, fake, None, None, 0, None) == 4
    tf = lib.rqrcp_factor_tournament
    #             m  n  A    lda k  b  p  seed Omega ldo group jpvt tau rank work bytes stream
    assert tf(5, 5, fake, 5, 2, 1, 0, 0, fake, 4, 0, fake, fake, None, None, 0, None) == -10
    assert tf(5, 5, fake, 5, 2, 1, 0, 0, None, 0, -1, fake, fake, None, None, 0, None) == -11
    assert tf(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 0, None, fake, None, None, 0, None) == -12
    assert tf(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 0, fake, None, None, None, 0, None) == -13
    assert tf(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 0, fake, fake, None, None, 0, None) == 4  # no workspace
    tm = lib.rqrcp_factor_mixed_tournament
    #             m  n  A    lda k  b  p  seed Omega ldo sketch group jpvt tau rank work bytes stream
    assert tm(5, 5, fake, 5, 2, 1, 0, 0, fake, 4, 0, 0, fake, fake, None, None, 0, None) == -10
    assert tm(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 2, 0, fake, fake, None, None, 0, None) == -11
    assert tm(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 0, -1, fake, fake, None, None, 0, None) == -12
    assert tm(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 0, 0, None, fake, None, None, 0, None) == -13
    assert tm(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 0, 0, fake, None, None, None, 0, None) == -14
    assert tm(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 1, 0, fake, fake, None, None, 0, None) == 4  # no workspace
    tc = lib.rqrcp_tournament_config
    g64, f64 = ctypes.c_int64(0), ctypes.c_int64(0)
    #          ncols bb  b   p  bytes group  out
    assert tc(0, 1, 1, 0, 8, 0, ctypes.byref(g64), ctypes.byref(f64)) == -1
    assert tc(10, 11, 16, 0, 8, 0, ctypes.byref(g64), ctypes.byref(f64)) == -2
    assert tc(10, 4, 2, 0, 8, 0, ctypes.byref(g64), ctypes.byref(f64)) == -3
    assert tc(10, 4, 4, -1, 8, 0, ctypes.byref(g64), ctypes.byref(f64)) == -4
    assert tc(10, 4, 4, 0, 2, 0, ctypes.byref(g64), ctypes.byref(f64)) == -5
    assert tc(10, 4, 4, 0, 8, -1, ctypes.byref(g64), ctypes.byref(f64)) == -6
    assert tc(10, 4, 4, 0, 8, 0, None, ctypes.byref(f64)) == -7
    assert tc(10, 4, 4, 0, 8, 0, ctypes.byref(g64), None) == -8
    sr = lib.rqrcp_srqr
    #      m  n  A    lda l  b  p  seed Omega ldo g    d  seed_g swaps jpvt info work bytes stream
    assert sr(1, 5, fake, 5, 1, 1, 0, 0, None, 0, 5.0, 8, 0, 10, fake, None, None, 0, None) == -1
    assert sr(5, 5, fake, 5, 5, 1, 0, 0, None, 0, 5.0, 8, 0, 10, fake, None, None, 0, None) == -5
    assert sr(5, 5, fake, 5, 2, 1, 0, 0, fake, 4, 5.0, 8, 0, 10, fake, None, None, 0, None) == -10
    assert sr(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 1.0, 8, 0, 10, fake, None, None, 0, None) == -11
    assert sr(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 5.0, 0, 0, 10, fake, None, None, 0, None) == -12
    assert sr(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 5.0, 8, 0, -1, fake, None, None, 0, None) == -14
    assert sr(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 5.0, 8, 0, 10, None, None, None, 0, None) == -15
    assert sr(5, 5, fake, 5, 2, 1, 0, 0, None, 0, 5.0, 8, 0, 10, fake, None, None, 0, None) == 4  # no workspace
    ws = lib.rqrcp_srqr_workspace_size
    assert ws(5, 5, 5, 1, 0, 8) == 0 and ws(5, 5, 2, 1, 0, 0) == 0
    assert ws(5, 5, 2, 1, 0, 8) > lib.rqrcp_workspace_size(5, 5, 2, 1, 0, 0)


def test_other_entry_point_argument_codes(lib):
    fake = ctypes.c_void_p(0x1000)
    assert lib.rqrcp_generate_omega(0, 5, 0, fake, 5, None) == -1
    assert lib.rqrcp_generate_omega(2, 5, 0, fake, 4, None) == -5
    assert lib.rqrcp_generate_omega_host(0, 5, 0, fake, 5) == -1
    assert lib.rqrcp_generate_omega_host(2, 0, 0, fake, 5) == -2
    assert lib.rqrcp_generate_omega_host(2, 5, 0, None, 5) == -4
    assert lib.rqrcp_generate_omega_host(2, 5, 0, fake, 4) == -5
    bt = lib.rqrcp_factor_batched
    #        count descs order m_max n_max b_max p Omega ldo work bytes stream
    assert bt(1, fake, fake, 8, 8, 4, 2, None, 8, None, 0, None) == -8
    assert bt(1, fake, fake, 8, 8, 4, 2, fake, 7, None, 0, None) == -9
    assert bt(1, fake, fake, 8, 8, 4, 2, fake, 8, None, 0, None) == 4   # no workspace
    assert lib.rqrcp_sketch(5, 5, fake, 5, fake, 3, 4, fake, 3, None, 0, None) == -7
    assert lib.rqrcp_sketch(5, 5, fake, 5, fake, 3, 5, fake, 2, None, 0, None) == -9
    assert lib.rqrcp_lowrank(5, 5, 6, fake, 5, fake, fake, fake, 5, fake, 5, None, 0, None) == -3
    assert lib.rqrcp_lowrank(5, 5, 2, fake, 5, fake, fake, fake, 5, None, 5, None, 0, None) == -10
    assert lib.rqrcp_read_status(None, None, None) == -1


def test_binding_rejects_bad_python_arguments(lib):
    """The Python wrappers check dtype and the sketch-update choice before any device call."""
    import torch
    from paper_1804_05138_gb300 import binding
    A64 = torch.zeros((8, 6), dtype=torch.float64)
    with pytest.raises(ValueError):
        binding.factor(A64, 2, 2, 1, formula=3)
    with pytest.raises(TypeError):
        binding.factor(A64.float(), 2, 2, 1)
    with pytest.raises(TypeError):
        binding.srqr(A64.float(), 2, 2, 1)
    with pytest.raises(ValueError):
        binding.srqr(A64, 6, 2, 1)          # l must be below min(m, n): workspace size 0


def test_host_omega_matches_oracle_bit_for_bit(lib, orc):
    """The library's host draw of Omega (its own Philox4x64-10 + Box-Muller) equals the oracle's
    independent implementation of the same published definition, bit for bit, at sizes that use
    one host thread and several; the seeded factorizations use exactly this draw."""
    import numpy as np
    from paper_1804_05138_gb300 import binding
    for (l, m, seed) in [(1, 1, 0), (3, 7, 5), (40, 1000, 0), (80, 32768, 0), (72, 8193, 2**63 + 11)]:
        got = binding.rqrcp_generate_omega_host(l, m, seed)
        want = orc.omega(l, m, seed)
        assert got.shape == want.shape
        assert np.array_equal(got.view(np.uint64), want.view(np.uint64)), (l, m, seed)


def test_host_omega_respects_leading_dimension(lib):
    import numpy as np
    from paper_1804_05138_gb300 import binding
    l, m, ldo = 5, 9, 13
    buf = np.full((l, ldo), 7.0)
    assert lib.rqrcp_generate_omega_host(l, m, 3, buf.ctypes.data, ldo) == 0
    dense = binding.rqrcp_generate_omega_host(l, m, 3)
    assert np.array_equal(buf[:, :m], dense)
    assert np.all(buf[:, m:] == 7.0)
