"""GPU path vs the FP64 CPU oracle, element by element, through the C ABI.

Bar (plain FP64 form):
  * pivots identical up to the first step whose top-two sketch norms are within 1e-10
    relative of each other in the oracle (near-ties may resolve either way under different
    summation orders); with every step separated, the whole permutation is identical;
  * R (upper trapezoid and R22) within 1e-12 normwise: ||R_gpu - R_oracle||_F / ||R_oracle||_F;
  * the GPU factorization's own backward error ||A Pi - Q R||_F / ||A||_F (computed by the
    oracle from the GPU's reflectors) at rounding level (<= 10 sqrt(mn) 2^-53) and within
    1e-12 of the oracle's;
  * tau within 1e-10 normwise.
Entry-wise differences of tiny entries of R reach kappa(A) * 2^-53 on ill-conditioned
spectra (two backward-stable computations in different summation orders); that is forward
error, not a parity defect, so the bar is normwise.
"""
import numpy as np
import pytest

from paper_1804_05138_gb300 import inputs

pytestmark = pytest.mark.gpu

GAP_TOL = 1e-10
RTOL = 1e-12
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


def _to_gpu(A, dtype=None):
    import torch
    t = torch.from_numpy(np.asfortranarray(A)).to("cuda")
    if dtype is not None:
        t = t.to(dtype)
    from paper_1804_05138_gb300.binding import colmajor
    return colmajor(t)


def _compare(orc, ref, Ag, jpvt, tau, k, A0, rtol=RTOL):
    sep = ref.gaps >= GAP_TOL
    upto = k if sep.all() else int(np.argmin(sep))
    assert np.array_equal(jpvt[:upto], ref.jpvt[:upto]), (upto, jpvt[:upto][:20], ref.jpvt[:upto][:20])
    m, n = A0.shape
    if upto == k:
        assert np.array_equal(jpvt, ref.jpvt)
        Rg, Ro = orc.r_factor(Ag, k), orc.r_factor(ref.A, k)
        nerr = np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro)
        assert nerr <= rtol, nerr
        assert np.linalg.norm(tau - ref.tau) <= 1e-10 * np.linalg.norm(ref.tau)
    res = orc.rel_residual(A0, Ag, tau, jpvt, k)
    assert res <= 10 * np.sqrt(m * n) * U, res
    if upto == k:
        res_o = orc.rel_residual(A0, ref.A, ref.tau, ref.jpvt, k)
        assert abs(res - res_o) <= rtol
    return upto


CASES = [  # m, n, k, b, p
    (1000, 1000, 64, 32, 8),    # the 1000 x 1000 workload
    (257, 190, 100, 16, 5),     # ragged tails everywhere
    (300, 500, 250, 64, 8),     # wide
    (130, 70, 70, 32, 4),       # full k = n
    (64, 64, 64, 7, 3),         # k = m = n, odd block
    (33, 17, 17, 5, 40),        # l > m
    (1, 1, 1, 1, 0),            # 1 x 1
    (5, 7, 5, 2, 0),            # p = 0, full k = m < n
    (2000, 64, 64, 64, 8),      # tall-skinny, one block
]


@pytest.mark.parametrize("m,n,k,b,p", CASES)
def test_factor_with_omega_matches_oracle(gpu, orc, m, n, k, b, p):
    import torch
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    Om = inputs.gaussian_sketch(b + p, m, seed=3)
    ref = orc.rqrcp(A0, k, b, p, Om)
    f = gpu.factor(_to_gpu(A0), k, b, p, omega=torch.from_numpy(Om).cuda())
    torch.cuda.synchronize()
    _compare(orc, ref, f.A.cpu().numpy(), f.jpvt.cpu().numpy(), f.tau.cpu().numpy(), k, A0)
    assert f.rank == ref.rank


@pytest.mark.parametrize("m,n,k,b,p,seed", [(1000, 1000, 64, 32, 8, 0), (400, 300, 200, 32, 8, 5),
                                             (400, 300, 200, 32, 8, 7)])
def test_factor_seeded_matches_oracle(gpu, orc, m, n, k, b, p, seed):
    """The seeded entry point draws the same Omega as the oracle, bit for bit, so the whole
    permutation must match wherever the oracle's pivot steps are separated (all of them here)."""
    import torch
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    ref = orc.rqrcp_seeded(A0, k, b, p, seed)
    assert (ref.gaps >= GAP_TOL).all()
    rank = torch.full((1,), -7, dtype=torch.int64, device="cuda")
    A = _to_gpu(A0)
    jpvt = torch.empty(n, dtype=torch.int32, device="cuda")
    tau = torch.empty(k, dtype=torch.float64, device="cuda")
    work = gpu.workspace(gpu.rqrcp_workspace_size(m, n, k, b, p), "cuda")
    assert gpu.rqrcp_factor(A, k, b, p, seed, jpvt, tau, work, rank_out=rank) == 0
    code, rk = gpu.rqrcp_read_status(work)
    assert code == 0 and rk == k == int(rank.item())
    upto = _compare(orc, ref, A.cpu().numpy(), jpvt.cpu().numpy(), tau.cpu().numpy(), k, A0)
    assert upto == k


def test_omega_matches_oracle(gpu, orc):
    """Device copies of the seeded Omega are the oracle's draw bit for bit (FP64) and that draw
    rounded to float (FP32)."""
    import torch
    for (l, m, seed) in [(40, 1000, 0), (80, 32768, 3), (9, 13, 2)]:
        want = orc.omega(l, m, seed)
        Om = torch.empty((l, m), dtype=torch.float64, device="cuda")
        assert gpu.rqrcp_generate_omega(l, m, seed, Om) == 0
        assert np.array_equal(Om.cpu().numpy().view(np.uint64), want.view(np.uint64))
        Om32 = torch.empty((l, m), dtype=torch.float32, device="cuda")
        assert gpu.rqrcp_generate_omega(l, m, seed, Om32) == 0
        assert np.array_equal(Om32.cpu().numpy(), want.astype(np.float32))


def test_rank_out_reports_the_guard(gpu, orc):
    """rank_out receives the rank on the device, equal to rqrcp_read_status's and to the oracle's
    on an exactly rank-deficient input."""
    import torch
    m, n, r, k, b, p = 300, 200, 37, 120, 16, 8
    A0 = inputs.rank_r_product(m, n, r)
    Om = inputs.gaussian_sketch(b + p, m, seed=4)
    ref = orc.rqrcp(A0, k, b, p, Om)
    A = _to_gpu(A0)
    jpvt = torch.empty(n, dtype=torch.int32, device="cuda")
    tau = torch.empty(k, dtype=torch.float64, device="cuda")
    rank = torch.zeros(1, dtype=torch.int64, device="cuda")
    work = gpu.workspace(gpu.rqrcp_workspace_size(m, n, k, b, p), "cuda")
    assert gpu.rqrcp_factor_with_omega(A, k, b, p, torch.from_numpy(Om).cuda(), jpvt, tau, work,
                                       rank_out=rank) == 0
    code, rk = gpu.rqrcp_read_status(work)
    assert code == 0 and int(rank.item()) == rk == ref.rank


@pytest.mark.parametrize("m,n,l", [(1000, 1000, 40), (777, 333, 72), (64, 3000, 80), (500, 700, 96), (300, 257, 130)])
def test_sketch_matches_oracle(gpu, orc, m, n, l):
    import torch
    A0 = inputs.gaussian(m, n, seed=1)
    Om = inputs.gaussian_sketch(l, m, seed=2)
    want = orc.sketch(A0, Om)
    Ag = _to_gpu(A0)
    B = torch.empty((n, l), dtype=torch.float64, device="cuda").t()
    work = gpu.workspace(gpu.rqrcp_workspace_size(m, n, 1, l, 0), "cuda")
    assert gpu.rqrcp_sketch(Ag, torch.from_numpy(Om).cuda(), B, work) == 0
    code, _ = gpu.rqrcp_read_status(work)
    assert code == 0
    got = B.cpu().numpy()
    # |error| <= m * u * (|Omega| |A|) componentwise bound
    bound = m * 2.0 ** -53 * (np.abs(Om) @ np.abs(A0))
    assert np.all(np.abs(got - want) <= bound)


def test_identity_sketch_is_qrcp(gpu, orc):
    import torch
    m, n, b = 48, 40, 8
    rng = np.random.default_rng(0)
    A0 = np.asfortranarray(rng.standard_normal((m, n)) * (1.3 ** rng.permutation(n))[None, :])
    Af, jpvt, tau = orc.qrcp(A0, 32)
    f = gpu.factor(_to_gpu(A0), 32, b, m - b, omega=torch.eye(m, dtype=torch.float64, device="cuda"))
    assert np.array_equal(f.jpvt.cpu().numpy(), jpvt)
    assert np.abs(f.A.cpu().numpy() - Af).max() <= 1e-12 * np.abs(Af).max()


@pytest.mark.parametrize("m,n,r,k,b,p", [(600, 500, 50, 200, 32, 8), (512, 512, 64, 512, 64, 8)])
def test_rank_deficient_guard(gpu, orc, m, n, r, k, b, p):
    import torch
    A0 = inputs.rank_r_product(m, n, r)
    Om = inputs.gaussian_sketch(b + p, m, seed=0)
    ref = orc.rqrcp(A0, k, b, p, Om)
    f = gpu.factor(_to_gpu(A0), k, b, p, omega=torch.from_numpy(Om).cuda())
    assert ref.rank == r and f.rank == r
    Ag = f.A.cpu().numpy()
    assert np.array_equal(f.jpvt.cpu().numpy()[:r], ref.jpvt[:r])
    R = orc.r_factor(Ag, k)
    assert np.linalg.norm(R[r:, r:]) / np.linalg.norm(A0) < 1e-12
    assert orc.rel_residual(A0, Ag, f.tau.cpu().numpy(), f.jpvt.cpu().numpy(), k) < 1e-13


EQ5_CASES = [  # m, n, k, b, p
    (1000, 1000, 64, 32, 8),    # the 1000 x 1000 workload
    (257, 190, 100, 16, 5),     # ragged tails everywhere
    (300, 500, 250, 64, 8),     # wide
    (64, 64, 64, 7, 3),         # k = m = n, odd block
    (33, 17, 17, 5, 40),        # l > m
]


@pytest.mark.parametrize("m,n,k,b,p", EQ5_CASES)
def test_factor_eq5_matches_oracle(gpu, orc, m, n, k, b, p):
    """Eq. (5) (Omega_bar = Omega Q kept on the device, B2 - Omega_bar_1 R12) against the
    oracle's Eq. (5) path, with the bar of the Eq. (4) runs; the caller's Omega is not written."""
    import torch
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    Om = inputs.gaussian_sketch(b + p, m, seed=3)
    ref = orc.rqrcp(A0, k, b, p, Om, formula=5)
    Omg = torch.from_numpy(Om).cuda()
    f = gpu.factor(_to_gpu(A0), k, b, p, omega=Omg, formula=5)
    torch.cuda.synchronize()
    _compare(orc, ref, f.A.cpu().numpy(), f.jpvt.cpu().numpy(), f.tau.cpu().numpy(), k, A0)
    assert f.rank == ref.rank
    assert np.array_equal(Omg.cpu().numpy(), Om)


def test_factor_eq5_seeded_and_rank_guard(gpu, orc):
    m, n, k, b, p = 400, 300, 200, 32, 8
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    ref = orc.rqrcp_seeded(A0, k, b, p, 5, formula=5)
    assert (ref.gaps >= GAP_TOL).all()
    f = gpu.factor(_to_gpu(A0), k, b, p, seed=5, formula=5)
    upto = _compare(orc, ref, f.A.cpu().numpy(), f.jpvt.cpu().numpy(), f.tau.cpu().numpy(), k, A0)
    assert upto == k
    m, n, r, k, b, p = 600, 500, 50, 200, 32, 8
    A0 = inputs.rank_r_product(m, n, r)
    ref = orc.rqrcp_seeded(A0, k, b, p, 0, formula=5)
    f = gpu.factor(_to_gpu(A0), k, b, p, seed=0, formula=5)
    assert ref.rank == r and f.rank == r
    assert np.array_equal(f.jpvt.cpu().numpy()[:r], ref.jpvt[:r])
    assert orc.rel_residual(A0, f.A.cpu().numpy(), f.tau.cpu().numpy(), f.jpvt.cpu().numpy(), k) < 1e-13


def test_nonfinite_input_reports_error(gpu):
    import torch
    A = torch.randn(100, 80, dtype=torch.float64, device="cuda").t().contiguous().t()
    A[17, 33] = float("nan")
    with pytest.raises(gpu.RQRCPError) as ei:
        gpu.factor(A, 10, 8, 4)
    assert ei.value.code == gpu.RQRCP_ERR_NONFINITE


@pytest.mark.parametrize("m,n,k", [(300, 200, 70), (1000, 1000, 64), (129, 129, 129)])
def test_lowrank_matches_oracle(gpu, orc, m, n, k):
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    f = gpu.factor(_to_gpu(A0), k, 32, 8, seed=1)
    Af, tau, jpvt = f.A.cpu().numpy(), f.tau.cpu().numpy(), f.jpvt.cpu().numpy()
    L, Q1 = gpu.lowrank(f)
    Lref, Q1ref = orc.lowrank(Af, tau, jpvt, k)
    assert np.abs(Q1.cpu().numpy() - Q1ref).max() <= 1e-13
    assert np.abs(L.cpu().numpy() - Lref).max() <= 1e-12 * np.abs(Lref).max()
