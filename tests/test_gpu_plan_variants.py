"""Every schedule of the plan-driven product kernel against the oracle.

The autotuner picks one schedule per product on the running GPU, so each
schedule is forced in turn (LSQ_PLAN_VARIANT, read when a product is first
launched in a process) and checked in a fresh process: float64 within
1e-12, float32 within 1e-5 of max |A|.|B|, on a product with a truncated
result, a symmetric result and transposed operands.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_VARIANTS = 29

SCRIPT = r"""
import sys, numpy as np, torch
sys.path.insert(0, sys.argv[1]); sys.path.insert(0, sys.argv[1] + '/tests')
import oracle, paper_2002_07704_gb300 as lsq
from gpu_common import cuda, gpu_geometry, si, rel_err
lsq.build()
pos, cell = si(3, 0.1, 1234)
ranges = [6.6, 10.0, 16.6, 23.2]
g = gpu_geometry(pos, cell, ranges)
P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
rng = np.random.default_rng(5)
worst = 0.0
for (ra, rb, rc, ta, tb) in [(16.6, 10.0, 23.2, 0, 1), (6.6, 16.6, 10.0, 0, 0), (23.2, 16.6, 10.0, 1, 1)]:
    A = oracle.Bsr(P[ra], 4, rng.standard_normal((P[ra].nnzb, 4, 4)))
    B = oracle.Bsr(P[rb], 4, rng.standard_normal((P[rb].nnzb, 4, 4)))
    opA = oracle.transpose(A, P[ra]) if ta else A
    opB = oracle.transpose(B, P[rb]) if tb else B
    ref, _ = oracle.matmul(opA, opB, P[rc])
    for prec, dt in ((lsq.F64, torch.float64), (lsq.F32, torch.float32)):
        C = torch.zeros((P[rc].nnzb, 4, 4), dtype=dt, device='cuda')
        lsq.block_matmul(g, 4, cuda(A.val, dt), g.range_id(ra), cuda(B.val, dt), g.range_id(rb),
                         C, g.range_id(rc), precision=prec, trans_a=ta, trans_b=tb)
        got = C.double().cpu().numpy()
        if prec == lsq.F64:
            e = rel_err(got, ref.val)
            assert e <= 1e-12, e
        else:
            bound, _ = oracle.matmul(oracle.Bsr(P[ra], 4, np.abs(opA.val)), oracle.Bsr(P[rb], 4, np.abs(opB.val)), P[rc])
            e = np.abs(got - ref.val).max() / bound.val.max()
            assert e <= 1e-5, e
        worst = max(worst, e)
print('ok', worst)
"""


@pytest.mark.parametrize("variant", range(N_VARIANTS))
def test_plan_variant_matches_oracle(variant):
    env = dict(os.environ, LSQ_PLAN_VARIANT=str(variant))
    r = subprocess.run([sys.executable, "-c", SCRIPT, ROOT], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "ok" in r.stdout, r.stdout + r.stderr
