"""QR with tournament pivoting on the sketch (the paper's future work, Sec. VI) on the GPU
against the oracle's tournament (orc_rqrcp3), through the C ABI, on the same seeded inputs.

The oracle takes the leaf group size of every block and the fan-in from
rqrcp_tournament_config, the rule the GPU itself uses (automatic sizes and explicit ones), so
both sides run the same tree.

Bar (plain FP64 form): pivots identical up to the first block whose tournament made a choice
within 1e-10 relative of the runner-up (all k where every choice is separated, asserted for most
cases); R within 1e-12 normwise; tau within 1e-10; backward error at rounding level.  A single
leaf per block reproduces the greedy GPU factorization (Alg. 2's partial QRCP) exactly.
FP32 form (FP32-accurate sketch, FP32 selection steps): pivots up to the first 1e-4 near-tie,
backward error <= 1e-6, rank.  Exactly rank-r inputs stop at r.  At 8192 x 4096 the mixed form
keeps ||R22||_2 within 1.2x of the greedy search's and the low-rank identity
||A - Q1 [R11 R12] Pi^T||_F = ||R22||_F.
"""
import numpy as np
import pytest

from paper_1804_05138_gb300 import inputs

pytestmark = pytest.mark.gpu

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
    from paper_1804_05138_gb300.binding import colmajor
    t = torch.from_numpy(np.asfortranarray(A)).to("cuda")
    return colmajor(t if dtype is None else t.to(dtype))


def _tree(gpu, n, k, b, p, es, group):
    """Per-block leaf group sizes and the common fan-in the GPU uses."""
    gs, fans = [], set()
    for i in range(0, k, b):
        g, f = gpu.rqrcp_tournament_config(n - i, min(b, k - i), b, p, es, group)
        gs.append(g)
        fans.add(f)
    assert len(fans) == 1
    return gs, fans.pop()


def _upto(gaps, tol, k):
    sep = gaps >= tol
    return k if sep.all() else int(np.argmin(sep))


CASES64 = [  # m, n, k, b, p, group (0: automatic), want the whole permutation
    (300, 200, 48, 16, 8, 0, True),
    (257, 301, 70, 32, 5, 40, True),
    (2000, 1500, 128, 64, 8, 0, True),
    (600, 900, 96, 24, 6, 24, True),
    (129, 77, 77, 16, 4, 16, False),
]


@pytest.mark.parametrize("m,n,k,b,p,group,full", CASES64)
def test_tournament_fp64_matches_oracle(gpu, orc, m, n, k, b, p, group, full):
    import torch
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    Om = inputs.gaussian_sketch(b + p, m, seed=3)
    tgs, fan = _tree(gpu, n, k, b, p, 8, group)
    ref = orc.rqrcp(A0, k, b, p, Om, tgs=tgs, fanin=fan)
    f = gpu.factor(_to_gpu(A0), k, b, p, omega=torch.from_numpy(Om).cuda(), tournament=group)
    Ag, jp, tau = f.A.cpu().numpy(), f.jpvt.cpu().numpy(), f.tau.cpu().numpy()
    assert sorted(jp.tolist()) == list(range(n))
    assert f.rank == ref.rank
    upto = _upto(ref.gaps, 1e-10, k)
    if full:
        assert upto == k
    assert np.array_equal(jp[:upto], ref.jpvt[:upto]), (upto, jp[:upto][:16], ref.jpvt[:upto][:16])
    if upto == k:
        assert np.array_equal(jp, ref.jpvt)
        Rg, Ro = orc.r_factor(Ag, k), orc.r_factor(ref.A, k)
        assert np.linalg.norm(Rg - Ro) <= 1e-12 * np.linalg.norm(Ro)
        assert np.linalg.norm(tau - ref.tau) <= 1e-10 * np.linalg.norm(ref.tau)
    assert orc.rel_residual(A0, Ag, tau, jp, k) <= 10 * np.sqrt(m * n) * U


def test_tournament_one_leaf_is_the_greedy_search(gpu):
    import torch
    m, n, k, b, p = 500, 400, 96, 32, 8
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_log_decay(min(m, n)))
    Om = torch.from_numpy(inputs.gaussian_sketch(b + p, m, seed=4)).cuda()
    g = gpu.factor(_to_gpu(A0), k, b, p, omega=Om)
    t = gpu.factor(_to_gpu(A0), k, b, p, omega=Om, tournament=n)  # one leaf holds all n - i columns
    assert torch.equal(g.jpvt, t.jpvt)
    Rg, Rt = np.triu(g.A.cpu().numpy()[:k]), np.triu(t.A.cpu().numpy()[:k])
    assert np.linalg.norm(Rg - Rt) <= 1e-13 * np.linalg.norm(Rg)


def test_tournament_group_too_large_is_unsupported(gpu):
    import torch
    A = torch.zeros((400, 300), dtype=torch.float64, device="cuda").t().contiguous().t()
    with pytest.raises(gpu.RQRCPError) as e:
        gpu.factor(A, 64, 32, 8, tournament=4096)
    assert e.value.code == gpu.RQRCP_ERR_UNSUPPORTED


def test_tournament_rank_deficient_stops_at_rank(gpu, orc):
    m, n, k, b, p, r = 400, 300, 120, 32, 8, 37
    A0 = inputs.rank_r_product(m, n, r)
    f = gpu.factor(_to_gpu(A0), k, b, p, seed=1, tournament=0)
    assert f.rank == r
    Ag = f.A.cpu().numpy()
    assert np.linalg.norm(orc.r_factor(Ag, k)[r:, r:]) <= 1e-12 * np.linalg.norm(A0)


@pytest.mark.parametrize("m,n,k,b,p,group", [(1400, 800, 192, 64, 16, 0), (1000, 1000, 128, 32, 8, 48)])
def test_tournament_fp32_matches_oracle(gpu, orc, m, n, k, b, p, group):
    import torch
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(n, 100.0))
    A32 = A0.astype(np.float32).astype(np.float64)
    tgs, fan = _tree(gpu, n, k, b, p, 4, group)
    ref = orc.rqrcp_seeded(A32, k, b, p, seed=0, tgs=tgs, fanin=fan)
    f = gpu.factor_mixed(_to_gpu(A0, torch.float32), k, b, p, seed=0, sketch="fp32", tournament=group)
    Af, jp, tau = f.A.cpu().double().numpy(), f.jpvt.cpu().numpy(), f.tau.cpu().numpy()
    assert sorted(jp.tolist()) == list(range(n))
    assert f.rank == ref.rank == k
    upto = _upto(ref.gaps, 1e-4, k)
    assert np.array_equal(jp[:upto], ref.jpvt[:upto]), upto
    assert orc.rel_residual(A32, Af, tau, jp, k) <= 1e-6


def test_tournament_mixed_8192x4096_quality(gpu):
    import torch
    m, n, k, b, p = 8192, 4096, 256, 64, 16
    sigma = inputs.sigma_exp_decay(n, 200.0)
    A = inputs.spectrum_matrix_torch(m, n, sigma, dtype=torch.float32)
    g = gpu.factor_mixed(A, k, b, p, seed=5)
    t = gpu.factor_mixed(A, k, b, p, seed=5, tournament=0)
    assert g.rank == t.rank == k
    r22 = {}
    for name, f in (("greedy", g), ("tournament", t)):
        R22 = f.A[k:, k:].double()
        x = torch.randn(n - k, dtype=torch.float64, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
        for _ in range(30):
            x = R22.t() @ (R22 @ x)
            x /= torch.linalg.norm(x)
        r22[name] = torch.linalg.norm(R22 @ x).item()
        L, _ = gpu.lowrank(f)
        lhs = torch.linalg.norm(A.double() - L.double()).item()
        rhs = torch.linalg.norm(R22).item()
        assert abs(lhs - rhs) <= 1e-5 * torch.linalg.norm(A.double()).item(), (name, lhs, rhs)
    assert r22["tournament"] >= sigma[k] * (1 - 1e-3)
    assert r22["tournament"] <= 1.2 * r22["greedy"], r22
