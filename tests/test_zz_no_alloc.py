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


def _call(lib, g, b, precision, rx, X, ry, Y, out):
    return lib.lsq_trace_static(g.handle, b, precision, rx, ctypes.c_void_p(X.data_ptr()), ry,
                                ctypes.c_void_p(Y.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def test_trace_static_against_oracle_and_allocates_nothing():
    """Same value as the oracle's trace (1e-12 relative; both accumulate the float64 products
    in a different order), and no device memory taken by the calls: the free device memory
    is the same before and after two calls on a geometry no other trace has touched."""
    lsq.build()
    lib = lsq.load()
    pos, cell = si(2, 0.1, 91)
    ranges = [6.6, 10.0]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(5)
    Xh = rng.standard_normal((P[10.0].nnzb, 4, 4))
    Yh = rng.standard_normal((P[6.6].nnzb, 4, 4))
    ref = oracle.trace(oracle.Bsr(P[10.0], 4, Xh), oracle.Bsr(P[6.6], 4, Yh))
    X, Y = cuda(Xh), cuda(Yh)
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _call(lib, g, 4, lsq.F64, 1, X, 0, Y, out) == 0
        torch.cuda.synchronize()
        assert abs(float(out.item()) - ref) <= 1e-12 * max(1.0, abs(ref))
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_trace_static_b13_and_batched_geometry():
    """13 x 13 blocks, and a block-diagonal geometry of two systems (the binary search then
    runs over concatenated columns): both equal lsq_trace to 1e-12."""
    lsq.build()
    lib = lsq.load()
    rng = np.random.default_rng(13)
    out = torch.zeros((1,), dtype=torch.float64, device="cuda")
    pos, cell = si(1, 0.1, 17)
    g = gpu_geometry(pos, cell, [3.0, 4.0])
    X = torch.randn((g.nnzb(0), 13, 13), dtype=torch.float64, device="cuda")
    Y = torch.randn((g.nnzb(1), 13, 13), dtype=torch.float64, device="cuda")
    ref = lsq.trace(g, 13, X, 0, Y, 1)
    assert _call(lib, g, 13, lsq.F64, 0, X, 1, Y, out) == 0
    torch.cuda.synchronize()
    assert abs(float(out.item()) - ref) <= 1e-12 * max(1.0, abs(ref))
    parts = [gpu_geometry(*si(n, 0.1, 40 + n), [6.6, 10.0]) for n in (1, 2)]
    bg = lsq.concat_geometries(parts)
    X = cuda(rng.standard_normal((bg.nnzb(0), 4, 4)))
    Y = cuda(rng.standard_normal((bg.nnzb(1), 4, 4)))
    ref = lsq.trace(bg, 4, X, 0, Y, 1)
    assert _call(lib, bg, 4, lsq.F64, 0, X, 1, Y, out) == 0
    torch.cuda.synchronize()
    assert abs(float(out.item()) - ref) <= 1e-12 * max(1.0, abs(ref))


def test_trace_static_empty_and_above_limit():
    """No atoms: the trace is 0.  More than 262144 atoms: LSQ_ERR_UNSUPPORTED before any
    launch (a grid of atoms 1 A apart with a 0.5 A range: only self pairs)."""
    lsq.build()
    lib = lsq.load()
    out = torch.full((1,), np.nan, dtype=torch.float64, device="cuda")
    g0 = gpu_geometry(np.zeros((0, 3)), [10.0, 10.0, 10.0], [3.0])
    z = torch.zeros((1, 4, 4), dtype=torch.float64, device="cuda")
    assert _call(lib, g0, 4, lsq.F64, 0, z, 0, z, out) == 0
    torch.cuda.synchronize()
    assert float(out.item()) == 0.0
    n = (65, 65, 63)
    grid = np.stack(np.meshgrid(*[np.arange(k, dtype=np.float64) + 0.25 for k in n], indexing="ij"), -1)
    big = gpu_geometry(grid.reshape(-1, 3), [float(k) for k in n], [0.5])
    assert big.n_atoms == 266175 > 262144 and big.nnzb(0) == big.n_atoms
    X = torch.ones((big.nnzb(0), 1, 1), dtype=torch.float64, device="cuda")
    assert _call(lib, big, 1, lsq.F64, 0, X, 0, X, out) == 7
