"""SRQR (Alg. 3) on the GPU against the FP64 oracle's Alg. 3 (orc_srqr), through the C ABI.

Bar: the swap count and the permutation equal to the oracle's (when every pivot step of the
RQRCP stage is separated by more than 1e-10 relative in the oracle), R within 1e-12 normwise,
the g2 estimate within 1e-9 relative; on the Kahan matrix, Table I's and Table II's SRQR
columns (Sec. V-B) as in the oracle's pins; after forced swaps, A(:, jpvt) = Q R to rounding.
"""
import os

import numpy as np
import pytest

from paper_1804_05138_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
U = 2.0 ** -53


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_1804_05138_gb300 import binding, build
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build.build()
    binding.load()
    return binding


def _golden(tag):
    rows = []
    with open(os.path.join(GOLDEN, "kahan_srqr.txt")) as f:
        for line in f:
            parts = line.split()
            if parts and parts[0] == tag:
                rows.append(parts[1:])
    return rows


def _run(gpu, A0, l, b, p, Om, g=5.0, max_swaps=1000, seed=0):
    import torch
    from paper_1804_05138_gb300.binding import colmajor
    Ag = colmajor(torch.from_numpy(np.asfortranarray(A0)).cuda())
    om = None if Om is None else torch.from_numpy(np.ascontiguousarray(Om)).cuda()
    f = gpu.srqr(Ag, l, b, p, seed=seed, omega=om, g=g, d=8, seed_g=0, max_swaps=max_swaps)
    torch.cuda.synchronize()
    return f.R.cpu().numpy(), f.jpvt.cpu().numpy(), f


def _separated(orc, A0, l, b, p, Om):
    ref = orc.rqrcp(A0, l, b, p, Om)
    return bool((ref.gaps >= 1e-10).all())


def _compare(orc, A0, l, b, p, Om, g=5.0, max_swaps=1000, gpu=None, seed=0):
    R, jp, f = _run(gpu, A0, l, b, p, None if seed else Om, g, max_swaps, seed)
    ref = orc.srqr(A0, l, b, p, Om, g=g, d=8, seed_g=0, max_swaps=max_swaps)
    assert sorted(jp.tolist()) == list(range(A0.shape[1]))
    if _separated(orc, A0, l, b, p, Om):
        assert f.swaps == ref.swaps, (f.swaps, ref.swaps)
        assert np.array_equal(jp, ref.jpvt)
        assert np.linalg.norm(R - ref.R) <= 1e-12 * np.linalg.norm(ref.R)
        if np.isfinite(ref.g2):
            assert abs(f.g2 - ref.g2) <= 1e-9 * ref.g2, (f.g2, ref.g2)
    return R, jp, f, ref


def _check_factor(A0, R, jp, l):
    m, n = A0.shape
    Ap = A0[:, jp]
    gram = Ap.T @ Ap
    assert np.linalg.norm(R.T @ R - gram) <= 200 * np.sqrt(m * n) * U * np.linalg.norm(gram)
    assert np.all(np.tril(R[:l + 1, :], -1) == 0.0)
    assert np.all(R[l + 1:, :l + 1] == 0.0)


def test_kahan_qrcp_start_table1(gpu, orc):
    """QRCP start (identity sketch): the loop must repair the Kahan matrix with a swap."""
    n = 96
    K = inputs.kahan(n)
    R, jp, f, ref = _compare(orc, K, n - 1, 16, n - 16, np.eye(n), gpu=gpu)
    assert f.swaps >= 1 and f.g2 <= 5.0
    printed = float([r for r in _golden("T1") if r[0] == "96"][0][2])
    ratio = np.linalg.norm(R[n - 1:, n - 1:]) / np.linalg.norm(K)
    assert abs(ratio / printed - 1.0) < 0.03, ratio


def test_kahan_rqrcp_start_tables(gpu, orc):
    n = 192
    K = inputs.kahan(n)
    R, jp, f, ref = _compare(orc, K, n - 1, 64, 10, inputs.gaussian_sketch(74, n, seed=0), gpu=gpu)
    assert f.g2 <= 5.0
    printed = float([r for r in _golden("T1") if r[0] == "192"][0][2])
    ratio = np.linalg.norm(R[n - 1:, n - 1:]) / np.linalg.norm(K)
    assert abs(ratio / printed - 1.0) < 0.03, ratio
    sA = np.linalg.svd(K, compute_uv=False)
    sR = np.linalg.svd(np.triu(R[:n - 1, :n - 1]), compute_uv=False)
    for j_s, pr in _golden("T2"):
        j = int(j_s)
        assert abs(sR[j - 1] / sA[j - 1] - float(pr)) < 5e-4, j


def test_random_matrix_matches_oracle(gpu, orc):
    A0 = inputs.spectrum_matrix(300, 250, inputs.sigma_exp_decay(250, 10.0))
    R, jp, f, ref = _compare(orc, A0, 60, 16, 8, inputs.gaussian_sketch(24, 300, seed=4), gpu=gpu)
    _check_factor(A0, R, jp, 60)


def test_forced_swaps_match_oracle(gpu, orc):
    A0 = inputs.spectrum_matrix(200, 160, inputs.sigma_exp_decay(160, 8.0))
    R, jp, f, ref = _compare(orc, A0, 40, 16, 8, inputs.gaussian_sketch(24, 200, seed=5), g=1.0 + 1e-12,
                             max_swaps=4, gpu=gpu)
    assert f.swaps == 4
    _check_factor(A0, R, jp, 40)


def test_seeded_sketch_matches_oracle(gpu, orc):
    m, n, l, b, p, seed = 400, 300, 100, 32, 8, 7
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    R, jp, f, ref = _compare(orc, A0, l, b, p, orc.omega(b + p, m, seed), gpu=gpu, seed=seed)
    _check_factor(A0, R, jp, l)


def test_rank_below_l_skips_the_swap_loop(gpu, orc):
    """Ten nonzero columns among forty, l = 15: the RQRCP stage stops at rank 10, R_hat has
    exact zeros on its diagonal and the loop is skipped, as in the oracle."""
    rng = np.random.default_rng(3)
    A0 = np.zeros((60, 40))
    A0[:, ::4] = rng.standard_normal((60, 10))
    Om = inputs.gaussian_sketch(14, 60, seed=0)
    R, jp, f = _run(gpu, A0, 15, 8, 6, Om)
    ref = orc.srqr(A0, 15, 8, 6, Om, g=5.0, d=8)
    assert f.rank == ref.rank == 10
    assert f.swaps == ref.swaps == 0 and f.g2 == np.inf
    assert np.array_equal(jp[:10], ref.jpvt[:10])
    assert np.all(R[10:, 10:] == 0.0)
    _check_factor(A0, R, jp, 15)
