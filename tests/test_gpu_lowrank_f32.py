"""FP32 low-rank outputs of the mixed form (Q1 = H_0 ... H_{k-1} I(:, 0:k) and
L = Q1 [R11 R12] Pi^T, Sec. I-A) on the GPU against the oracle's orc_lowrank run in FP64 on the
same FP32 factorization (reflectors, tau and pivots from the GPU).

For k <= 256 with aligned operands the library forms Q1 from all k reflectors at once on the tensor
cores (T^{-1} = diag(1/tau) + striu(V^T V)); otherwise it applies the blocks one by one.  Both are
checked.  Bars: the products run at FP32 accuracy (3xTF32 operands, FP32 accumulation over m and
k terms), so ||Q1 - Q1_ref||_F <= 2e-6 sqrt(k) (about 30 units of 2^-24 per column of norm 1),
||L - L_ref||_F <= 1e-5 ||L_ref||_F, and ||Q1^T Q1 - I||_F <= 2e-6 k.
"""
import numpy as np
import pytest

from paper_1804_05138_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_1804_05138_gb300 import binding, build
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build.build()
    binding.load()
    return binding


def _check(gpu, orc, A0, k, b, p):
    import torch
    from paper_1804_05138_gb300.binding import colmajor
    A = colmajor(torch.from_numpy(np.asfortranarray(A0)).to("cuda").float())
    f = gpu.factor_mixed(A, k, b, p, seed=2)
    L, Q1 = gpu.lowrank(f)
    Af = f.A.double().cpu().numpy()
    tau, jp = f.tau.cpu().numpy(), f.jpvt.cpu().numpy()
    Lref, Q1ref = orc.lowrank(Af, tau, jp, k)
    Qg, Lg = Q1.double().cpu().numpy(), L.double().cpu().numpy()
    eq = np.linalg.norm(Qg - Q1ref)
    el = np.linalg.norm(Lg - Lref) / np.linalg.norm(Lref)
    eo = np.linalg.norm(Qg.T @ Qg - np.eye(k))
    print(f"{A0.shape} k={k}: Q1 {eq:.3e}, L {el:.3e}, orth {eo:.3e}")
    assert eq <= 2e-6 * np.sqrt(k), eq
    assert el <= 1e-5, el
    assert eo <= 2e-6 * k, eo
    return f


@pytest.mark.parametrize("m,n,k,b", [
    (1000, 800, 200, 64),    # all reflectors at once on the tensor cores
    (516, 300, 129, 32),     # ragged k and tiles
    (4096, 4096, 256, 64),   # the differentiable workload's size
    (600, 300, 300, 64),     # k > 256: block by block
    (1001, 700, 70, 16),     # ldaf % 4 != 0: block by block
    (300, 50, 1, 8),         # one reflector
])
def test_lowrank_f32_matches_oracle(gpu, orc, m, n, k, b):
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(min(m, n), 0.25 * min(m, n)))
    _check(gpu, orc, A0, k, b, 8)


def test_lowrank_f32_rank_deficient(gpu, orc):
    """Exactly rank r < k: the factorization stops at r; Q1's leading r columns match the oracle
    and the low-rank product reproduces A."""
    import torch
    m, n, k, r = 400, 300, 120, 37
    A0 = inputs.rank_r_product(m, n, r)
    f = _check(gpu, orc, A0, k, 32, 8)
    assert f.rank == r
