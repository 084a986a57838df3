"""The no-allocation sketch entry point (rqrcp_sketch_noalloc) against the workspace one.

Some callers cannot allocate device memory: they only hold the input and output pointers
(no allocator, no workspace to pass) or must not call cudaMalloc/cudaFree because those
synchronise the device.  rqrcp_sketch_noalloc serves them from a fixed device array inside
the library.  This file runs last (pytest collects it after the others) and also passes in
a fresh process on its own.
"""
import ctypes

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


def _sketch_both(gpu, m, n, l, seed):
    import torch
    A0 = inputs.gaussian(m, n, seed=seed)
    Om = inputs.gaussian_sketch(l, m, seed=seed + 100)
    A = gpu.colmajor(torch.from_numpy(A0).cuda())
    Omg = torch.from_numpy(Om).cuda()
    B_ref = torch.empty((n, l), dtype=torch.float64, device="cuda").t()
    work = gpu.workspace(gpu.rqrcp_workspace_size(m, n, 1, l, 0), "cuda")
    assert gpu.rqrcp_sketch(A, Omg, B_ref, work) == 0
    B_na = torch.full((n, l), float("nan"), dtype=torch.float64, device="cuda").t()
    assert gpu.rqrcp_sketch_noalloc(A, Omg, B_na) == 0
    torch.cuda.synchronize()
    # each result is within m*u*(|Omega||A|) of the exact product, so they differ by at most twice that
    bound = 2.0 * m * U * (np.abs(Om) @ np.abs(A0))
    return B_ref.cpu().numpy(), B_na.cpu().numpy(), bound


def test_noalloc_matches_workspace_sketch_on_two_calls_in_a_row(gpu):
    for (m, n, l, seed) in [(1000, 1000, 40, 1), (777, 333, 72, 2)]:
        ref, got, bound = _sketch_both(gpu, m, n, l, seed)
        assert np.all(np.isfinite(got))
        assert np.all(np.abs(got - ref) <= bound)


def test_noalloc_rejects_sizes_beyond_its_scratch(gpu):
    lib = gpu.load()
    fake = ctypes.c_void_p(0x1000)   # rejected before any pointer is used
    # n * l * 8 bytes for one split must fit the 8 MiB array (minus its 256-byte status block)
    assert lib.rqrcp_sketch_noalloc(10, 16384, fake, 10, fake, 64, 10, fake, 64, None) == gpu.RQRCP_ERR_UNSUPPORTED
    assert lib.rqrcp_sketch_noalloc(0, 5, fake, 1, fake, 2, 1, fake, 2, None) == -1


def test_noalloc_with_a_non_finite_entry_writes_every_column(gpu):
    """An Inf in one column of A makes that column of B non-finite; every other column is still
    written and equals the workspace sketch (status is not reported by this entry point)."""
    import torch
    m, n, l = 600, 500, 24
    A0 = inputs.gaussian(m, n, seed=3)
    A0[17, 123] = np.inf
    Om = inputs.gaussian_sketch(l, m, seed=4)
    A = gpu.colmajor(torch.from_numpy(A0).cuda())
    Omg = torch.from_numpy(Om).cuda()
    B_ref = torch.empty((n, l), dtype=torch.float64, device="cuda").t()
    work = gpu.workspace(gpu.rqrcp_workspace_size(m, n, 1, l, 0), "cuda")
    assert gpu.rqrcp_sketch(A, Omg, B_ref, work) == 0
    code, _ = gpu.rqrcp_read_status(work)
    assert code == gpu.RQRCP_ERR_NONFINITE
    B_na = torch.full((n, l), 12345.0, dtype=torch.float64, device="cuda").t()
    assert gpu.rqrcp_sketch_noalloc(A, Omg, B_na) == 0
    torch.cuda.synchronize()
    got, ref = B_na.cpu().numpy(), B_ref.cpu().numpy()
    assert not np.isfinite(got[:, 123]).any()
    keep = np.ones(n, dtype=bool)
    keep[123] = False
    assert np.all(np.isfinite(got[:, keep]))
    # the two entry points may split the sum over m differently: each is within m*u*(|Omega||A|)
    bound = 2.0 * m * U * (np.abs(Om) @ np.abs(np.where(np.isfinite(A0), A0, 0.0)))
    assert np.all(np.abs(got[:, keep] - ref[:, keep]) <= bound[:, keep])
