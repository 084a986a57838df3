"""FP64 Q1/R of the mixed form and the CholQR reorthogonalisation pass, against the oracle.

* tol above the measured error: no pass; Q1 equals the oracle's Q1 built in FP64 from the
  FP32 reflectors (1e-13), R is the FP32 upper trapezoid widened exactly, and the reported
  ||Q1^T Q1 - I||_F matches the host's value.
* tol = 0: the pass runs; Q1 and R equal the oracle's CholQR of the same inputs (1e-12
  normwise), ||Q1^T Q1 - I||_F drops to rounding level and Q1 R is unchanged (1e-13).
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


def _run(gpu, f, k, tol):
    import torch
    m, n = f.A.shape
    Q1 = torch.empty((k, m), dtype=torch.float64, device="cuda").t()
    R = torch.empty((n, k), dtype=torch.float64, device="cuda").t()
    orth = torch.zeros(1, dtype=torch.float64, device="cuda")
    work = gpu.workspace(gpu.rqrcp_reorth_workspace_size(m, n, k), "cuda")
    assert gpu.rqrcp_lowrank_reorth(f.A, k, f.tau, Q1, R, tol, orth, work) == 0
    code, _ = gpu.rqrcp_read_status(work)
    assert code == 0
    return Q1.cpu().numpy(), R.cpu().numpy(), float(orth.item())


@pytest.mark.parametrize("m,n,k", [(2048, 1024, 128), (3000, 700, 200)])
def test_reorth_against_oracle(gpu, orc, m, n, k):
    import torch
    A0 = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(n, 100.0))
    f = gpu.factor_mixed(gpu.colmajor(torch.from_numpy(A0).cuda().float()), k, 64, 16, seed=0)
    Af = f.A.double().cpu().numpy()
    tau = f.tau.cpu().numpy()
    Q0, R0, e0 = _run(gpu, f, k, 1e30)
    Q0ref = orc.form_q(Af, tau, k, k)
    assert np.abs(Q0 - Q0ref).max() <= 1e-13
    assert np.array_equal(R0, np.triu(Af[:k, :]))
    e_host = np.linalg.norm(Q0.T @ Q0 - np.eye(k))
    assert abs(e0 - e_host) <= 1e-10 * e_host + 1e-15
    Q1, R1, e1 = _run(gpu, f, k, 0.0)
    assert e1 == pytest.approx(e0, rel=1e-12)
    Qref, Rref = orc.cholqr_reorth(Q0, R0)
    assert np.linalg.norm(Q1 - Qref) <= 1e-12 * np.linalg.norm(Qref)
    assert np.linalg.norm(R1 - Rref) <= 1e-12 * np.linalg.norm(Rref)
    assert np.linalg.norm(Q1.T @ Q1 - np.eye(k)) <= 10 * np.sqrt(m * k) * 2.0 ** -53
    P0 = Q0 @ R0
    assert np.linalg.norm(Q1 @ R1 - P0) <= 1e-13 * np.linalg.norm(P0)
    assert np.allclose(np.tril(R1[:, :k], -1), 0.0)
