"""The FP32 form's CholeskyQR2 panel with Householder reconstruction against the FP64 oracle (whose
panel is Householder QR, Alg. 2 "Do unpivoted QR"), and against the cooperative Householder panel.

* Well-conditioned panels (spectra as in the mixed workloads): the mixed-form bar (backward error
  <= 1e-6, pivots equal up to the oracle's first 1e-4 near-tie) and R within 1e-5 of the oracle's
  R normwise when all pivots agree: the reconstruction reproduces the xLARFG sign convention, so R
  itself (not only |R|) matches.
* Panels beyond the CholeskyQR2 range: an exactly rank-deficient input (the panel straddling the
  rank boundary mixes columns of norm 1 with columns at rounding level) and a graded matrix
  (column norms spread over 1e7); the fallback flag hands those panels to the Householder panel and
  the same bar holds.
* The same factorizations with RQRCP_PANEL=householder (the switch is read once per process, so
  in a child process): identical pivots, R within 1e-5 normwise of the CholeskyQR2 run's R.
"""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

from paper_1804_05138_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_1804_05138_gb300 import binding, build
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    build.build()
    binding.load()
    return binding


def _graded(m, n, seed=4):
    rng = np.random.default_rng(seed)
    return np.asfortranarray(rng.standard_normal((m, n)) * (10.0 ** rng.uniform(-7, 0, n))[None, :])


CASES = {
    "expspec": lambda: inputs.spectrum_matrix(1400, 800, inputs.sigma_exp_decay(800, 100.0)),
    "logspec": lambda: inputs.spectrum_matrix(1200, 700, inputs.sigma_log_decay(700)),
    "rank37": lambda: inputs.rank_r_product(600, 400, 37),
    "graded": lambda: _graded(800, 300),
}
PARAMS = {"expspec": (192, 64, 16), "logspec": (150, 32, 8), "rank37": (120, 16, 8), "graded": (160, 32, 8)}


def _run(gpu, orc, name):
    import torch
    A0 = CASES[name]()
    k, b, p = PARAMS[name]
    A32 = A0.astype(np.float32).astype(np.float64)
    ref = orc.rqrcp_seeded(A32, k, b, p, seed=0, sketch_bf16=False)
    A = gpu.colmajor(torch.from_numpy(np.asfortranarray(A0)).to("cuda").float())
    f = gpu.factor_mixed(A, k, b, p, seed=0, sketch="fp32")
    return A32, ref, f, k


@pytest.mark.parametrize("name", sorted(CASES))
def test_cholqr_panel_against_oracle(gpu, orc, name):
    A32, ref, f, k = _run(gpu, orc, name)
    Af = f.A.cpu().double().numpy()
    jp = f.jpvt.cpu().numpy()
    tau = f.tau.cpu().numpy()
    n = A32.shape[1]
    assert sorted(jp.tolist()) == list(range(n))
    if name == "rank37":
        # the FP32 input is rank 37 plus rounding noise: the mixed form's guard (FP32 level) stops
        # at 37, the FP64 oracle's guard keeps pivoting the noise; the first 37 pivots are compared
        assert f.rank == 37
    else:
        assert f.rank == ref.rank
    res = orc.rel_residual(A32, Af, tau, jp, k)
    assert res <= 1e-6, (name, res)
    sep = ref.gaps >= 1e-4
    upto = min(k if sep.all() else int(np.argmin(sep)), f.rank)
    assert np.array_equal(jp[:upto], ref.jpvt[:upto]), (name, upto)
    if upto == k and f.rank == k and ref.rank == k:
        Rg, Ro = orc.r_factor(Af, k), orc.r_factor(ref.A, k)
        Rg, Ro = Rg[:k], Ro[:k]
        assert np.linalg.norm(Rg - Ro) <= 1e-5 * np.linalg.norm(Ro), name


CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
from paper_1804_05138_gb300 import binding, build
import test_gpu_cholqr_panel as t
build.build()
binding.load()
out = {}
for name in sorted(t.CASES):
    A0 = t.CASES[name]()
    k, b, p = t.PARAMS[name]
    A = binding.colmajor(torch.from_numpy(np.asfortranarray(A0)).to("cuda").float())
    f = binding.factor_mixed(A, k, b, p, seed=0, sketch="fp32")
    out[name] = {"jpvt": f.jpvt.cpu().numpy().tolist(), "R": np.triu(f.A[:k].cpu().double().numpy()).tolist(),
                 "rank": f.rank}
print(json.dumps(out))
"""


def test_cholqr_panel_matches_householder_panel(gpu):
    import torch
    env = dict(os.environ, RQRCP_PANEL="householder")
    proc = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, cwd=ROOT, capture_output=True, text=True,
                          timeout=1200)
    assert proc.returncode == 0, proc.stderr[-3000:]
    hh = json.loads(proc.stdout.strip().splitlines()[-1])
    for name in sorted(CASES):
        A0 = CASES[name]()
        k, b, p = PARAMS[name]
        A = gpu.colmajor(torch.from_numpy(np.asfortranarray(A0)).to("cuda").float())
        f = gpu.factor_mixed(A, k, b, p, seed=0, sketch="fp32")
        assert f.rank == hh[name]["rank"], name
        jp = f.jpvt.cpu().numpy()
        assert np.array_equal(jp[:f.rank], np.array(hh[name]["jpvt"])[:f.rank]), name
        Rc = np.triu(f.A[:k].cpu().double().numpy())
        Rh = np.array(hh[name]["R"])
        r = f.rank
        assert np.linalg.norm(Rc[:r, :] - Rh[:r, :]) <= 1e-5 * np.linalg.norm(Rh[:r, :]), name
