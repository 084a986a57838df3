"""Batched randomized QRCP (one persistent launch) against the FP64 oracle.

Each matrix of a small uneven batch is compared with the oracle's Alg. 2 on the same
matrix, the same (shared, sliced) sketch and the same b, p, with the mixed-form bar:
backward error <= 1e-6, pivots equal up to the oracle's first 1e-4 near-tie, rank = k.
The 512-matrix batch (m in [256,4096], n in [128, min(m,2048)], k in [16,256]) is checked on
sampled matrices and sampled columns; a CUDA-graph replay gives the same bits as the eager call.
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


def _spectrum_batch(shapes, seed0=100, torch_gen=False):
    import torch
    mats = []
    for i, (m, n, _) in enumerate(shapes):
        sig = inputs.sigma_exp_decay(min(m, n), 0.1 * n)
        if torch_gen:
            A = inputs.spectrum_matrix_torch(m, n, sig, seed_u=seed0 + 2 * i, seed_v=seed0 + 2 * i + 1,
                                             dtype=torch.float32)
        else:
            A = torch.from_numpy(inputs.spectrum_matrix(m, n, sig, seed0 + 2 * i, seed0 + 2 * i + 1)).float().cuda()
        mats.append(A)
    return mats


SMALL = [(700, 400, 64, 32), (333, 120, 40, 16), (128, 128, 128, 32), (512, 300, 17, 8), (257, 33, 33, 16),
         (64, 40, 30, 64), (900, 500, 100, 64), (1000, 150, 150, 32), (95, 95, 60, 16), (400, 399, 80, 8)]


def test_small_batch_against_oracle(gpu, orc):
    p, seed = 8, 3
    shapes = [(m, n, k) for m, n, k, _ in SMALL]
    bs = [b for *_, b in SMALL]
    mats = _spectrum_batch(shapes)
    A0s = [A.double().cpu().numpy() for A in mats]
    batch = gpu.Batch(mats, [k for _, _, k in shapes], bs, p=p, seed=seed)
    assert batch.run() == 0
    import torch
    torch.cuda.synchronize()
    Om_full = orc.omega(batch.b_max + p, batch.m_max, seed).astype(np.float32).astype(np.float64)
    for i, ((m, n, k), b) in enumerate(zip(shapes, bs)):
        l = b + p
        ref = orc.rqrcp(A0s[i], k, b, p, np.ascontiguousarray(Om_full[:l, :m]))
        Af = batch.mats[i].double().cpu().numpy()
        jp = batch.jpvts[i].cpu().numpy()
        tau = batch.taus[i].cpu().numpy()
        assert int(batch.ranks[i]) == ref.rank == k
        assert sorted(jp.tolist()) == list(range(n))
        res = orc.rel_residual(A0s[i], Af, tau, jp, k)
        assert res <= 1e-6, (i, res)
        sep = ref.gaps >= 1e-4
        upto = k if sep.all() else int(np.argmin(sep))
        assert np.array_equal(jp[:upto], ref.jpvt[:upto]), (i, upto)


@pytest.mark.parametrize("tiles", [1, 2, 4, 8, 2 | 4 | 8])
def test_small_batch_tile_variants_against_oracle(gpu, orc, tiles):
    """Every tile-shape choice the autotuner may pick (RQRCP_TILES_*) meets the same bar as the
    default rules on the same batch."""
    import torch
    p, seed = 8, 3
    shapes = [(m, n, k) for m, n, k, _ in SMALL]
    bs = [b for *_, b in SMALL]
    mats = _spectrum_batch(shapes)
    A0s = [A.double().cpu().numpy() for A in mats]
    batch = gpu.Batch(mats, [k for _, _, k in shapes], bs, p=p, seed=seed, tiles=[tiles] * len(shapes))
    assert batch.run() == 0
    torch.cuda.synchronize()
    Om_full = orc.omega(batch.b_max + p, batch.m_max, seed).astype(np.float32).astype(np.float64)
    for i, ((m, n, k), b) in enumerate(zip(shapes, bs)):
        ref = orc.rqrcp(A0s[i], k, b, p, np.ascontiguousarray(Om_full[:b + p, :m]))
        jp = batch.jpvts[i].cpu().numpy()
        assert int(batch.ranks[i]) == ref.rank == k
        res = orc.rel_residual(A0s[i], batch.mats[i].double().cpu().numpy(), batch.taus[i].cpu().numpy(), jp, k)
        assert res <= 1e-6, (tiles, i, res)
        sep = ref.gaps >= 1e-4
        upto = k if sep.all() else int(np.argmin(sep))
        assert np.array_equal(jp[:upto], ref.jpvt[:upto]), (tiles, i, upto)


def test_graph_replay_matches_eager(gpu):
    import torch
    shapes = [(m, n, k) for m, n, k, _ in SMALL[:6]]
    mats = _spectrum_batch(shapes, seed0=300)
    orig = [A.clone() for A in mats]
    batch = gpu.Batch(mats, [k for _, _, k in shapes], [b for *_, b in SMALL[:6]], p=8, seed=1)
    assert batch.run() == 0
    torch.cuda.synchronize()
    eager = [A.clone() for A in batch.mats]
    eager_j = [j.clone() for j in batch.jpvts]
    for A, O in zip(batch.mats, orig):
        A.copy_(O)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            code = batch.run(stream=s)
    torch.cuda.current_stream().wait_stream(s)
    assert code == 0
    for A, O in zip(batch.mats, orig):
        A.copy_(O)
    g.replay()
    torch.cuda.synchronize()
    for A, E, j, ej in zip(batch.mats, eager, batch.jpvts, eager_j):
        assert torch.equal(A, E) and torch.equal(j, ej)


def test_full_batch_512(gpu, orc):
    import torch
    from paper_1804_05138_gb300 import autotune
    shapes = inputs.batched_shapes(512, seed=0)
    table = autotune.load_or_tune(shapes, p=8)
    bs = [autotune.choose(table, m, n, k) for (m, n, k) in shapes]
    assert all(1 <= b <= min(64, k) for b, (_, _, k) in zip(bs, shapes))
    tiles = [autotune.choose_tiles(table, m, n, k) for (m, n, k) in shapes]
    mats = _spectrum_batch(shapes, seed0=1000, torch_gen=True)
    batch = gpu.Batch(mats, [k for _, _, k in shapes], bs, p=8, seed=0, tiles=tiles)
    picks = [int(np.argmax([m * n for m, n, _ in shapes])), int(np.argmin([m * n for m, n, _ in shapes])), 7, 200, 411]
    A0 = {i: mats[i].double().cpu().numpy() for i in picks}
    assert batch.run() == 0
    torch.cuda.synchronize()
    ranks = batch.ranks.cpu().numpy()
    assert np.array_equal(ranks, np.array([k for _, _, k in shapes]))
    for i in picks:
        m, n, k = shapes[i]
        jp = batch.jpvts[i].cpu().numpy()
        assert sorted(jp.tolist()) == list(range(n))
        Af = batch.mats[i].double().cpu().numpy()
        tau = batch.taus[i].cpu().numpy()
        for j in sorted({0, k - 1, k, min(n - 1, k + 5), n - 1}):
            r = np.array(Af[:, j], copy=True)
            if j < k:
                r[j + 1:] = 0.0
            y = orc.apply_q(Af[:, :k], tau, k, r)
            a = A0[i][:, jp[j]]
            assert np.linalg.norm(y - a) <= 1e-6 * np.linalg.norm(a), (i, j)
