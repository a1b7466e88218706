"""The tcgen05 split-3xTF32 GEMM against the FP32 SIMT GEMM: the mixed
factorization is run in two fresh processes (tensor cores on / off, chosen
by H2_TC) on the same seeded problem; ranks must agree almost everywhere,
the refined solutions must both meet the target and agree, and the mixed
log-determinants must agree to FP32-product accuracy."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SCRIPT = r'''
import sys, json
sys.path.insert(0, %r)
import numpy as np, torch, synth
from paper_2208_10907_gb300 import h2ulv as H
X = synth.sphere_ball(6000, 31)
N = len(X)
pts = torch.from_numpy(X).cuda()
h = H.h2_construct(pts, N, H.make_kernel("yukawa"), H.make_options(leaf=128, tol=1e-8, max_rank=100))
H.h2_factor(h, H.H2_MIXED)
b = torch.from_numpy(synth.rhs(N, 1, 5)[:, 0].copy()).cuda()
x = torch.zeros_like(b)
st, ach, it = H.h2_solve(h, b, x, 1, N, 1e-11, 40)
ld, sg = H.h2_logdet(h)
s = json.loads(H.h2_stats(h))
print(json.dumps(dict(st=st, res=float(ach[0]), it=it, logdet=float(ld[0]), x=x.cpu().numpy().tolist(),
                      ranks=[lv["rank_mean"] for lv in s["levels"]],
                      tc=[k for k in s["kernels"] if k.startswith("gemm_tc")])))
H.h2_destroy(h)
''' % ROOT


def run(tc):
    env = dict(os.environ, H2_TC=tc)
    out = subprocess.run([sys.executable, "-c", SCRIPT], env=env, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    return json.loads(out.stdout.strip().splitlines()[-1])


def test_tensor_core_gemm_matches_simt():
    a = run("1")
    b = run("0")
    assert a["tc"], "tensor-core kernel was not used"
    assert not b["tc"]
    assert a["st"] == 0 and b["st"] == 0 and a["res"] <= 1e-11 and b["res"] <= 1e-11
    xa, xb = np.array(a["x"]), np.array(b["x"])
    assert np.linalg.norm(xa - xb) / np.linalg.norm(xb) < 1e-9
    assert np.allclose(a["ranks"], b["ranks"], rtol=0.05)
    assert abs(a["logdet"] - b["logdet"]) <= 1e-5 * abs(b["logdet"])
