"""The SIMT contractions kept beside the tensor-core ones (RQRCP_TENSOR_CORES=0: the FP32 form's
sketch, Gram and trailing update, and the batched kernel's sketch and update) against the FP64
oracle, with the same bars as the tensor-core runs: backward error <= 1e-6 and pivots equal up
to the oracle's first 1e-4 near-tie.  The switch is read once per process, so the cases run in a
child process with the variable set.
"""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np, torch
sys.path.insert(0, sys.argv[1])
from paper_1804_05138_gb300 import binding, build, inputs
from oracle import oracle as orc
orc.build()
build.build()
binding.load()
out = {}

def upto_of(ref, k):
    sep = ref.gaps >= 1e-4
    return k if sep.all() else int(np.argmin(sep))

# single-matrix FP32 form
m, n, k, b, p = 1000, 1000, 64, 32, 8
A0 = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(min(m, n), 100.0))
A32 = A0.astype(np.float32).astype(np.float64)
A = binding.colmajor(torch.from_numpy(np.asfortranarray(A0)).to("cuda").float())
for sk in ("bf16", "fp32"):
    ref = orc.rqrcp_seeded(A32, k, b, p, seed=0, sketch_bf16=(sk == "bf16"))
    f = binding.factor_mixed(A, k, b, p, seed=0, sketch=sk)
    Af = f.A.cpu().double().numpy()
    jp = f.jpvt.cpu().numpy()
    tau = f.tau.cpu().numpy()
    up = upto_of(ref, k)
    out["mixed_" + sk] = {"residual": float(orc.rel_residual(A32, Af, tau, jp, k)),
                          "pivots_equal": bool(np.array_equal(jp[:up], ref.jpvt[:up])),
                          "permutation": sorted(jp.tolist()) == list(range(n))}

# batched kernel
cases = [(700, 400, 64, 32), (333, 120, 40, 16), (900, 500, 100, 64), (257, 33, 33, 16), (1000, 150, 150, 32)]
p, seed = 8, 3
mats, A0s = [], []
for i, (m, n, k, _) in enumerate(cases):
    Ai = inputs.spectrum_matrix(m, n, inputs.sigma_exp_decay(min(m, n), 0.1 * n), 100 + 2 * i, 101 + 2 * i)
    mats.append(torch.from_numpy(Ai).float().cuda())
    A0s.append(mats[-1].double().cpu().numpy())
batch = binding.Batch(mats, [c[2] for c in cases], [c[3] for c in cases], p=p, seed=seed)
assert batch.run() == 0
torch.cuda.synchronize()
Om = orc.omega(batch.b_max + p, batch.m_max, seed).astype(np.float32).astype(np.float64)
for i, (m, n, k, b) in enumerate(cases):
    ref = orc.rqrcp(A0s[i], k, b, p, np.ascontiguousarray(Om[:b + p, :m]))
    Af = batch.mats[i].double().cpu().numpy()
    jp = batch.jpvts[i].cpu().numpy()
    tau = batch.taus[i].cpu().numpy()
    up = upto_of(ref, k)
    out["batched_%d" % i] = {"residual": float(orc.rel_residual(A0s[i], Af, tau, jp, k)),
                             "pivots_equal": bool(np.array_equal(jp[:up], ref.jpvt[:up])),
                             "permutation": sorted(jp.tolist()) == list(range(n)),
                             "rank": int(batch.ranks[i]), "k": k}
print(json.dumps(out))
"""


def test_simt_contractions_against_oracle():
    env = dict(os.environ, RQRCP_TENSOR_CORES="0")
    proc = subprocess.run([sys.executable, "-c", CHILD, ROOT], env=env, cwd=ROOT, capture_output=True, text=True,
                          timeout=1200)
    assert proc.returncode == 0, proc.stderr[-3000:]
    res = json.loads(proc.stdout.strip().splitlines()[-1])
    assert len(res) == 7
    for key, v in res.items():
        assert v["permutation"], key
        assert v["residual"] <= 1e-6, (key, v)
        assert v["pivots_equal"], (key, v)
        if "rank" in v:
            assert v["rank"] == v["k"], (key, v)
