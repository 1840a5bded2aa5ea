"""The allocation-free trace (lsq_trace_static) against lsq_trace.

lsq_trace_static is for callers that cannot let the library allocate
device memory: their memory is all owned by their own pool, or they must
not stall the device with cudaMalloc/cudaFree.  It keeps its partial sums
in a fixed device array instead.  This file is collected last so that a
run stopping at the first failure has already run every other test; it
also passes on its own in a fresh process.

Tolerance: both entry points accumulate the same float64 products, in a
different order, so they agree to 1e-12 relative.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_2002_07704_gb300 as lsq
from gpu_common import cuda, gpu_geometry, si

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [lsq.F64, lsq.F32])
def test_trace_static_matches_trace_twice(precision):
    lsq.build()
    lib = lsq.load()
    pos, cell = si(3, 0.1, 77)
    ranges = [6.6, 10.0]
    g = gpu_geometry(pos, cell, ranges)
    rng = np.random.default_rng(2024)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    dt = torch.float64 if precision == lsq.F64 else torch.float32
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    for call in range(2):
        X = cuda(rng.standard_normal((P[6.6].nnzb, 4, 4)), dt)
        Y = cuda(rng.standard_normal((P[10.0].nnzb, 4, 4)), dt)
        ref = lsq.trace(g, 4, X, 0, Y, 1, precision=precision)
        rc = lib.lsq_trace_static(g.handle, 4, precision, 0, ctypes.c_void_p(X.data_ptr()), 1,
                                  ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == 0
        torch.cuda.synchronize()
        got = float(out.item())
        assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)), (call, got, ref)


def test_trace_static_rejects_null_geometry():
    """Arguments are checked on the host before any launch."""
    lsq.build()
    lib = lsq.load()
    rc = lib.lsq_trace_static(None, 4, lsq.F64, 0, None, 0, None, None, None)
    assert rc == 1
