"""Mixed form (FP32 storage and arithmetic, FP64 reflector generation) against the FP64 oracle.

The error against the FP64 oracle is stated per result:
  * backward error ||A Pi - Q R||_F / ||A||_F (FP64, R including R22) <= 1e-6;
  * ||R22||_2 >= sigma_{k+1} (interlacing) and no worse than max(2, 1.1 x the FP64 oracle's
    own ratio) (the 2 sigma_{k+1} target is statistical: the oracle itself reaches 1.6-2.5 on
    these spectra with these oversamplings);
  * pivots identical to the oracle's (run with the same sketch reading: BF16-rounded operands
    or the exact sketch) up to the first step where the oracle's top-two sketch norms are within
    1e-4 relative (FP32 accumulation resolves only gaps well above 2^-24);
  * R within 1e-5 normwise of the oracle's R when all pivots agree.
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


def _f32_gpu(A, gpu):
    import torch
    return gpu.colmajor(torch.from_numpy(np.asfortranarray(A)).to("cuda").float())


@pytest.mark.parametrize("sketch", ["bf16", "fp32"])
@pytest.mark.parametrize("m,n,k,b,p,scale", [
    (1000, 1000, 64, 32, 8, 100.0),
    (2048, 1536, 200, 64, 16, 200.0),
    (777, 500, 130, 32, 16, 60.0),
    (4096, 256, 256, 64, 16, 40.0),
])
def test_mixed_against_oracle(gpu, orc, m, n, k, b, p, scale, sketch):
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(min(m, n), scale))
    A32 = A0.astype(np.float32).astype(np.float64)          # the matrix the mixed form sees
    # the oracle with the same sketch reading: BF16-rounded operands, or the exact sketch
    ref = orc.rqrcp_seeded(A32, k, b, p, seed=0, sketch_bf16=(sketch == "bf16"))
    f = gpu.factor_mixed(_f32_gpu(A0, gpu), k, b, p, seed=0, sketch=sketch)
    Af = f.A.cpu().double().numpy()
    jp = f.jpvt.cpu().numpy()
    tau = f.tau.cpu().numpy()
    assert sorted(jp.tolist()) == list(range(n))
    res = orc.rel_residual(A32, Af, tau, jp, k)
    assert res <= 1e-6, res
    sep = ref.gaps >= 1e-4
    upto = k if sep.all() else int(np.argmin(sep))
    assert np.array_equal(jp[:upto], ref.jpvt[:upto])
    if upto == k:
        Rg, Ro = orc.r_factor(Af, k), orc.r_factor(ref.A, k)
        assert np.linalg.norm(Rg - Ro) / np.linalg.norm(Ro) <= 1e-5
    if k < min(m, n):
        R = orc.r_factor(Af, k)
        s = np.linalg.svd(A32, compute_uv=False)
        ratio = np.linalg.norm(R[k:, k:], 2) / s[k]
        ratio_o = np.linalg.norm(orc.r_factor(ref.A, k)[k:, k:], 2) / s[k]
        assert 1.0 - 1e-4 <= ratio <= max(2.0, 1.1 * ratio_o), (ratio, ratio_o)


@pytest.mark.parametrize("sketch", ["bf16", "fp32"])
def test_mixed_rank_deficient_guard(gpu, orc, sketch):
    m, n, r, k, b, p = 600, 500, 40, 200, 32, 8
    A0 = inputs.rank_r_product(m, n, r)
    f = gpu.factor_mixed(_f32_gpu(A0, gpu), k, b, p, seed=0, sketch=sketch)
    assert f.rank == r
    R = orc.r_factor(f.A.cpu().double().numpy(), k)
    assert np.linalg.norm(R[r:, r:]) / np.linalg.norm(A0) < 1e-5


def test_mixed_nonfinite(gpu):
    import torch
    A = torch.randn(64, 48, device="cuda").t().contiguous().t()
    A[3, 5] = float("inf")
    with pytest.raises(gpu.RQRCPError) as ei:
        gpu.factor_mixed(A, 8, 8, 4)
    assert ei.value.code == gpu.RQRCP_ERR_NONFINITE
