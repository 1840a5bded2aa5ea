"""Parity of the GPU Hotelling inverse overlap (lsq_hotelling_inverse) with the oracle.

Float64 within 1e-12 (relative to max |X|), float32 products within 1e-5,
on full-range and truncated ranges, both block sizes, from the scaled start
and from a given X, and sampled rows of a step at 4096 atoms.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import hotelling as OH
from oracle import lnv as OL
import paper_2002_07704_gb300 as lsq
from gpu_common import cuda, gpu_geometry, si
from synth import config_seed, sk_blocks

pytestmark = pytest.mark.gpu


def _setup(n, sigma, seed, b, R_X):
    pos, cell = si(n, sigma, seed)
    R_S = 6.6
    ranges = sorted(set([R_S, R_X, R_X + R_S]))
    g = gpu_geometry(pos, cell, ranges)
    m = OL.System(pos, cell)
    pS = m.pattern(R_S)
    _, S = sk_blocks(pos, cell, pS.rows(), pS.col, b=b, perturb_seed=(seed + 7) if b == 13 else None)
    return g, m, oracle.Bsr(pS, b, S), (g.range_id(R_S), g.range_id(R_X), g.range_id(R_X + R_S))


@pytest.mark.parametrize("b,n,R_X,iters", [(4, 2, 10.0, 30), (13, 2, 10.0, 30), (4, 3, 5.0, 12), (13, 1, 3.0, 8)])
def test_hotelling_float64_matches_oracle(b, n, R_X, iters):
    g, m, S, (rs, rx, rxs) = _setup(n, 0.1, config_seed(0) + 40 + n, b, R_X)
    Xref, href = OH.hotelling(m, S, R_X, iters)
    X = torch.zeros((g.nnzb(rx), b, b), dtype=torch.float64, device="cuda")
    dx = lsq.hotelling_inverse(g, b, cuda(S.val), rs, X, rx, rxs, iters)
    got = X.cpu().numpy()
    scale = np.abs(Xref.val).max()
    assert np.abs(got - Xref.val).max() <= 1e-12 * scale
    # the step sizes agree, down to the rounding of X itself
    normx = float(np.sqrt(np.sum(Xref.val ** 2)))
    for a, r in zip(dx, href):
        assert abs(a - r) <= 1e-9 * r + 1e-13 * normx
    # X stays symmetric to the last bit
    pat = oracle.Pattern(g.n_atoms, *[t.cpu().numpy() for t in g.pattern(rx)], R_X)
    assert np.array_equal(got, oracle.transpose(oracle.Bsr(pat, b, got), pat).val)


def test_hotelling_float32_and_restart_from_given_x():
    b, R_X = 4, 5.0
    g, m, S, (rs, rx, rxs) = _setup(3, 0.1, config_seed(0) + 61, b, R_X)
    X5, _ = OH.hotelling(m, S, R_X, 5)
    X3, _ = OH.hotelling(m, S, R_X, 3)
    # float64, three steps from the oracle's X after two more
    X = cuda(X3.val)
    lsq.hotelling_inverse(g, b, cuda(S.val), rs, X, rx, rxs, 2, start=False)
    assert np.abs(X.cpu().numpy() - X5.val).max() <= 1e-12 * np.abs(X5.val).max()
    # float32 products from the scaled start
    X = torch.zeros((g.nnzb(rx), b, b), dtype=torch.float64, device="cuda")
    lsq.hotelling_inverse(g, b, cuda(S.val), rs, X, rx, rxs, 5, precision=lsq.F32)
    assert np.abs(X.cpu().numpy() - X5.val).max() <= 1e-5 * np.abs(X5.val).max()


def test_hotelling_rejects_a_short_product_range():
    g, m, S, (rs, rx, rxs) = _setup(2, 0.1, config_seed(0), 4, 5.0)
    X = torch.zeros((g.nnzb(rx), 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(lsq.LsqError):
        lsq.hotelling_inverse(g, 4, cuda(S.val), rs, X, rx, rx, 1)


def test_hotelling_full_size_sampled_rows():
    """4096-atom Si, R_X = 10 A: one step from the scaled start, sampled rows vs the oracle."""
    b, R_X = 4, 10.0
    g, m, S, (rs, rx, rxs) = _setup(8, 0.05, config_seed(1), b, R_X)
    X = torch.zeros((g.nnzb(rx), b, b), dtype=torch.float64, device="cuda")
    lsq.hotelling_inverse(g, b, cuda(S.val), rs, X, rx, rxs, 1)
    got = X.cpu().numpy()
    X0 = OH.scaled_start(S, m.pattern(R_X))
    rows = np.array([0, 1, 1234, 2048, 4095], dtype=np.int32)
    XS, _ = oracle.matmul(X0, S, m.pattern(R_X + 6.6), rows=rows)
    XSX, _ = oracle.matmul(XS, X0, m.pattern(R_X), rows=rows)
    ref = 2.0 * X0 - XSX
    p = m.pattern(R_X)
    for i in rows:
        sl = slice(p.ptr[i], p.ptr[i + 1])
        assert np.abs(got[sl] - ref.val[sl]).max() <= 1e-12 * np.abs(ref.val[sl]).max()
