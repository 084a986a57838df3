"""The FP32 form's paired block step (two blocks share one pass of the trailing update: block i
updates its R12 rows and block i+1's panel columns only, block i+1's Gram is corrected by
(V1^T V0) Y0, then C -= [V0 V1] [Y0; Y1]) against the per-block path.  The library pairs blocks
where the trailing matrix is larger than about the L2; here RQRCP_PAIRED=1 forces pairing at these
sizes and RQRCP_PAIRED=0 turns it off (the switch is read once per process, so both sides run in
child processes).

Both meet the mixed form's backward-error bar (<= 1e-6 against the FP64 oracle's residual).  Block
i+1's pivot search sees identical inputs on both paths (its Eq. (4) update reads only block i's R12
rows, computed identically), so the first two blocks' pivots are identical; later blocks differ
only by rounding, so where the whole permutation agrees R agrees to 1e-5 normwise.  Shapes: four
pairs; a block count that leaves an unpaired full block and a short last block; a steep spectrum
(sigma_i = 1/(1+i)^2, FP32 sketch), where the trailing matrix shrinks by orders of magnitude under
each block.
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
CASES = [(3000, 2500, 256, 64, 16, "exp"), (1500, 1200, 200, 64, 8, "exp"), (1200, 900, 128, 64, 8, "steep")]

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1804_05138_gb300 import binding, build, inputs
build.build()
binding.load()
out = {}
for (m, n, k, b, p, spec) in json.loads(sys.argv[2]):
    sig = inputs.sigma_exp_decay(min(m, n), 0.2 * min(m, n)) if spec == "exp" else inputs.sigma_inverse_square(min(m, n))
    A0 = inputs.spectrum_matrix(m, n, sig)
    A = binding.colmajor(torch.from_numpy(np.asfortranarray(A0)).to("cuda").float())
    f = binding.factor_mixed(A, k, b, p, seed=4, sketch="bf16" if spec == "exp" else "fp32")
    np.save(sys.argv[3] + "_%d_A.npy" % m, f.A.double().cpu().numpy())
    out[str(m)] = {"jpvt": f.jpvt.cpu().numpy().tolist(), "tau": f.tau.cpu().numpy().tolist(), "rank": f.rank}
print(json.dumps(out))
"""


def _run(mode, base):
    env = dict(os.environ, RQRCP_PAIRED=mode)
    r = subprocess.run([sys.executable, "-c", CHILD, ROOT, json.dumps(CASES), base], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-2000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    return {int(mk): (np.load(base + "_%s_A.npy" % mk), np.array(v["jpvt"]), np.array(v["tau"]), v["rank"])
            for mk, v in out.items()}


@pytest.fixture(scope="module")
def runs(tmp_path_factory):
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA GPU required for -m gpu tests")
    d = tmp_path_factory.mktemp("paired")
    return _run("1", str(d / "p")), _run("0", str(d / "u"))


@pytest.mark.parametrize("m,n,k,b,p,spec", CASES)
def test_paired_matches_per_block(orc, runs, m, n, k, b, p, spec):
    sig = inputs.sigma_exp_decay(min(m, n), 0.2 * min(m, n)) if spec == "exp" else inputs.sigma_inverse_square(min(m, n))
    A32 = inputs.spectrum_matrix(m, n, sig).astype(np.float32).astype(np.float64)
    Ap, jp, tp, rp = runs[0][m]
    Au, ju, tu, ru = runs[1][m]
    assert rp == ru and (spec != "exp" or rp == k)
    for Af, jv, tv in ((Ap, jp, tp), (Au, ju, tu)):
        assert sorted(jv.tolist()) == list(range(n))
        assert orc.rel_residual(A32, Af, tv, jv, k) <= 1e-6
    assert np.array_equal(jp[:2 * b], ju[:2 * b])
    if np.array_equal(jp, ju):
        Rp, Ru = orc.r_factor(Ap, k), orc.r_factor(Au, k)
        assert np.linalg.norm(Rp - Ru) <= 1e-5 * np.linalg.norm(Ru)
