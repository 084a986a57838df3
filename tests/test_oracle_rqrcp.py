"""Pins for the oracle's Alg. 2 (RQRCP) against what the paper and the mathematics fix.

P2  Kahan matrix, Tables I/II (Sec. V-B): QRCP makes no interchanges; printed ratios.
P3  exactly rank-r input: R22 vanishes to rounding and the rank guard stops at r.
P4  interlacing ||R22||_2 >= sigma_{k+1} (Sec. IV-A) and the reported ratio on a known spectrum.
P5  Theorem 1 (Sec. III-C) with the oversampling it prescribes.
P6  Eq. (4) and Eq. (5) give identical permutations (Sec. III-B).
P7  the updated sketch is (Omega Q)(:, k:m) R22 column-norm-wise (Sec. III-C, Eq. (3)).
P8  Lemma 3 / Eq. (7): sigma_j(A)^2 <= sigma_j([R11 R12])^2 + ||R22||_2^2.
P9  Theorem 1's worked example p >= 508 (golden file).
P10 Householder backward stability: residual and ||Q1^T Q1 - I|| at rounding level.
"""
import os

import numpy as np
import pytest

from paper_1804_05138_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                rows.append(line.split())
    return rows


# ------------------------------------------------------------------------------ P2
def test_kahan_table1_qrcp_column(orc):
    rows = [r for r in _read_golden("kahan_tables.txt") if len(r) == 3]
    assert len(rows) == 3
    for n_s, k_s, printed in rows:
        n, k = int(n_s), int(k_s)
        K = inputs.kahan(n)
        Af, jpvt, tau = orc.qrcp(K, k)
        assert np.array_equal(jpvt, np.arange(n)), "QRCP must make no interchanges on Kahan"
        R = orc.r_factor(Af, k)
        ratio = np.linalg.norm(R[k:, k:]) / np.linalg.norm(K)
        # computed s^{n-1}/||K||_F sits 0.5-2% from the printed digits (their s differs
        # slightly from the stated one); 3% tolerance
        assert abs(ratio / float(printed) - 1.0) < 0.03, (n, ratio, printed)
        # RQRCP with the identity sketch reproduces QRCP here too, up to the first
        # pivot step whose top-two sketch norms are tied to rounding (gap < 1e-10)
        res = orc.rqrcp(K, k, 16, n - 16, np.eye(n), formula=4)
        sep = res.gaps >= 1e-10
        upto = k if sep.all() else int(np.argmin(sep))
        assert upto >= min(k, 96)
        assert np.array_equal(res.jpvt[:upto], np.arange(upto))


def test_kahan_table2_qrcp_column(orc):
    rows = [r for r in _read_golden("kahan_tables.txt") if len(r) == 2]
    n, k = 192, 191
    K = inputs.kahan(n)
    Af, jpvt, tau = orc.qrcp(K, k)
    R11 = np.triu(Af[:k, :k])
    sA = np.linalg.svd(K, compute_uv=False)
    sR = np.linalg.svd(R11, compute_uv=False)
    for j_s, printed in rows:
        j = int(j_s)
        ratio = sR[j - 1] / sA[j - 1]
        if j < 191:
            assert abs(ratio - float(printed)) < 6e-5, (j, ratio, printed)
        else:  # rounding-level quantity: pinned to order of magnitude only
            assert 1e-18 < ratio < 1e-17, (j, ratio)


# ------------------------------------------------------------------------------ P3
@pytest.mark.parametrize("m,n,r,k,b,p", [(120, 100, 30, 60, 8, 6), (90, 140, 24, 80, 16, 4)])
def test_exact_rank_r22_vanishes_and_guard(orc, m, n, r, k, b, p):
    A = inputs.rank_r_product(m, n, r)
    res = orc.rqrcp(A, k, b, p, inputs.gaussian_sketch(b + p, m, seed=0))
    assert res.rank == r
    R = orc.r_factor(res.A, k)
    assert np.linalg.norm(R[r:, r:]) / np.linalg.norm(A) < 1e-12
    d = np.abs(np.diag(R[:k, :k]))
    assert d[r:].max() <= 1e-12 * d[0]
    assert d[:r].min() > 1e-6 * d[0]
    assert orc.rel_residual(A, res.A, res.tau, res.jpvt, k) < 1e-14


# ------------------------------------------------------------------------------ P4, P8, P10
def test_spectrum_c1_like(orc):
    """Scaled-down version of the 1000^2, sigma_i = 10^(-6 i/1000) workload."""
    m = n = 300
    k, b, p = 48, 16, 8
    sig = inputs.sigma_log_decay(n)
    A = inputs.spectrum_matrix(m, n, sig)
    res = orc.rqrcp(A, k, b, p, inputs.gaussian_sketch(b + p, m, seed=0))
    assert res.rank == k
    R = orc.r_factor(res.A, k)
    nrm22 = np.linalg.norm(R[k:, k:], 2)
    s = np.linalg.svd(A, compute_uv=False)
    assert nrm22 >= s[k] * (1 - 1e-10)                 # interlacing
    assert nrm22 <= 4.0 * s[k]                         # RQRCP reveals the spectrum
    Rt = R[:k, :]
    sR = np.linalg.svd(Rt, compute_uv=False)
    assert np.all(s[:k] ** 2 <= sR ** 2 + nrm22 ** 2 * (1 + 1e-10))   # Lemma 3, Eq. (7)
    resid = orc.rel_residual(A, res.A, res.tau, res.jpvt, k)
    assert resid < 10 * np.sqrt(m * n) * U
    Q1 = orc.form_q(res.A, res.tau, k, k)
    assert orc.orth_error(Q1) < 10 * np.sqrt(m * k) * U


def test_c1_full_size_oracle(orc):
    """The 1000 x 1000, k=64, b=32, p=8 workload itself (seconds on the CPU)."""
    m = n = 1000
    A = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(n))
    Om = orc.omega(40, m, seed=0)
    res = orc.rqrcp(A, 64, 32, 8, Om)
    assert res.rank == 64
    resid = orc.rel_residual(A, res.A, res.tau, res.jpvt, 64)
    assert resid < 10 * np.sqrt(m * n) * U
    R = orc.r_factor(res.A, 64)
    s = np.linalg.svd(A, compute_uv=False)
    ratio = np.linalg.norm(R[64:, 64:], 2) / s[64]
    assert 1.0 - 1e-10 <= ratio < 4.0


# ------------------------------------------------------------------------------ P5, P9
def test_theorem1_pmin_worked_example(orc):
    rows = _read_golden("theorem1_pmin.txt")
    for n, k, eps, delta, want in rows:
        assert orc.p_min(int(n), int(k), float(eps), float(delta)) == int(want)


def test_theorem1_pseudo_diagonal_dominance(orc):
    m, n, k, b = 400, 60, 10, 5
    eps, delta = 0.5, 0.05
    p = orc.p_min(n, k, eps, delta)
    assert b + p <= m
    A = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(n, 8.0))
    res = orc.rqrcp(A, k, b, p, inputs.gaussian_sketch(b + p, m, seed=3))
    R = orc.r_factor(res.A, k)
    c = np.sqrt((1 - eps) / (1 + eps))
    for i in range(k):
        tail = np.linalg.norm(R[i:, i + 1:], axis=0).max()
        assert abs(R[i, i]) >= c * tail


# ------------------------------------------------------------------------------ P6, P7
@pytest.mark.parametrize("m,n,k,b,p", [(80, 70, 40, 8, 5), (64, 100, 50, 16, 8), (50, 50, 50, 7, 3)])
def test_formula4_equals_formula5(orc, m, n, k, b, p):
    A = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(min(m, n), 12.0))
    Om = inputs.gaussian_sketch(b + p, m, seed=1)
    r4 = orc.rqrcp(A, k, b, p, Om, formula=4)
    r5 = orc.rqrcp(A, k, b, p, Om, formula=5)
    sep = r4.gaps > 1e-8
    first_tie = np.argmin(sep) if not sep.all() else k
    assert np.array_equal(r4.jpvt[:first_tie], r5.jpvt[:first_tie])
    if first_tie == k and k < n:
        assert np.allclose(np.linalg.norm(r4.B[:, k:], axis=0), np.linalg.norm(r5.B[:, k:], axis=0),
                           rtol=1e-9, atol=1e-12 * np.abs(r4.B).max())


@pytest.mark.parametrize("formula", [4, 5])
def test_sketch_invariant_after_last_block(orc, formula):
    m, n, k, b, p = 70, 60, 24, 8, 6
    A = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(n, 15.0))
    Om = inputs.gaussian_sketch(b + p, m, seed=2)
    res = orc.rqrcp(A, k, b, p, Om, formula=formula)
    Q = orc.form_q(res.A, res.tau, k, m)
    R22 = res.A[k:, k:]
    want = (Om @ Q)[:, k:] @ R22
    if formula == 5:
        assert np.allclose(res.B[:, k:], want, rtol=0, atol=1e-12 * np.abs(want).max())
    got = np.linalg.norm(res.B[:, k:], axis=0)
    assert np.allclose(got, np.linalg.norm(want, axis=0), rtol=1e-10, atol=1e-13 * got.max())


# ------------------------------------------------------------------------------ shapes and edge cases
@pytest.mark.parametrize("m,n,k,b,p", [
    (1, 1, 1, 1, 0), (5, 1, 1, 3, 2), (1, 7, 1, 2, 0), (9, 9, 9, 4, 0), (7, 12, 7, 3, 1),
    (33, 17, 17, 5, 40), (40, 40, 13, 64, 2),
])
def test_edge_shapes_residual(orc, m, n, k, b, p):
    A = inputs.gaussian(m, n, seed=m * 100 + n)
    res = orc.rqrcp(A, k, b, p, inputs.gaussian_sketch(b + p, m, seed=7))
    assert sorted(res.jpvt.tolist()) == list(range(n))
    assert orc.rel_residual(A, res.A, res.tau, res.jpvt, k) < 1e-14


def test_argument_errors(orc):
    A = inputs.gaussian(5, 4, seed=0)
    with pytest.raises(ValueError):
        orc.rqrcp(A, 5, 2, 1, inputs.gaussian_sketch(3, 5, 0))   # k > min(m, n)
    with pytest.raises(ValueError):
        orc.rqrcp(A, 0, 2, 1, inputs.gaussian_sketch(3, 5, 0))   # k < 1


# ------------------------------------------------------------------------------ P11
# The mixed form's BF16 sketch, the oracle's reading of it: Omega and A rounded to FP32, then to
# BF16 (round to nearest, ties to even) for the initial sketch only.
def test_round_bf16_matches_library_conversion(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    x = np.concatenate([
        rng.standard_normal(20000) * 10.0 ** rng.integers(-30, 30, 20000),
        # exact ties between two BF16 neighbours (even and odd kept patterns), and near-ties
        1.0 + np.array([1, 3, 5, 7]) * 2.0 ** -8, -(2.0 + np.array([1, 3]) * 2.0 ** -7),
        1.0 + 2.0 ** -8 + np.array([2.0 ** -20, -2.0 ** -20]),
        [0.0, -0.0, 1e-40, -3e-39],                   # zeros and FP32 subnormals
    ])
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    got = orc.round_bf16(x)
    assert np.array_equal(got, ref)
    assert np.array_equal(orc.round_bf16(got), got)  # BF16 values are fixed points


def test_bf16_sketch_is_identity_on_bf16_inputs(orc):
    # inputs already representable in BF16: the rounding is the identity, so the BF16-sketch
    # oracle must reproduce the FP64-sketch oracle bit for bit
    m, n, k, b, p = 120, 90, 40, 16, 6
    A = orc.round_bf16(inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(n, 30.0)))
    Om = orc.round_bf16(inputs.gaussian_sketch(b + p, m, seed=4))
    r64 = orc.rqrcp(A, k, b, p, Om)
    r16 = orc.rqrcp(A, k, b, p, Om, sketch_bf16=True)
    assert np.array_equal(r64.jpvt, r16.jpvt)
    assert np.array_equal(r64.A, r16.A)
    assert np.array_equal(r64.tau, r16.tau)


def test_bf16_sketch_changes_only_pivot_choice(orc):
    # the rounding only steers pivots: the factorization stays backward stable, and where the
    # sketch norms are well separated the pivots agree with the FP64 sketch
    m, n, k, b, p = 300, 200, 60, 20, 10
    A = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(n, 40.0))
    Om = inputs.gaussian_sketch(b + p, m, seed=5)
    r64 = orc.rqrcp(A, k, b, p, Om)
    r16 = orc.rqrcp(A, k, b, p, Om, sketch_bf16=True)
    assert orc.rel_residual(A, r16.A, r16.tau, r16.jpvt, k) < 1e-14
    sep = r64.gaps >= 1e-2  # BF16 moves the sketch norms by ~1e-3 relative
    upto = k if sep.all() else int(np.argmin(sep))
    assert upto >= 1
    assert np.array_equal(r64.jpvt[:upto], r16.jpvt[:upto])
