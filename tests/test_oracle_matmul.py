"""Pins of the oracle's truncated atom-block product (Sec. 2.3.2: all
matrices sparse by range, products restricted to the range of the result)."""
import numpy as np
import pytest

import oracle
from synth import diamond_si_positions, config_seed


def _rand_bsr(pat, b, rng):
    return oracle.Bsr(pat, b, rng.standard_normal((pat.nnzb, b, b)))


def _mask(pat, b):
    m = np.zeros((pat.n, pat.n), dtype=bool)
    m[pat.rows(), pat.col] = True
    return np.kron(m, np.ones((b, b), dtype=bool))


@pytest.mark.parametrize("n,b,ra,rb,rc", [
    (1, 4, 3.0, 4.0, 5.0),      # truncated below the natural range
    (2, 4, 4.0, 3.0, 7.0),      # exactly the natural range
    (2, 4, 3.0, 3.0, 8.0),      # beyond the natural range (extra zero blocks)
    (2, 4, 6.6, 8.0, 6.6),      # LSL.SL-like truncation to a short range
    (1, 13, 3.0, 2.5, 4.0),     # 13 x 13 blocks
    (2, 13, 2.5, 2.5, 3.0),
])
def test_truncated_product_equals_dense_masked(n, b, ra, rb, rc):
    pos, cell = diamond_si_positions(n, 0.1, config_seed(0) + 17 * n + b)
    rng = np.random.default_rng(5)
    pa = oracle.neighbour_list(pos, cell, ra)
    pb = oracle.neighbour_list(pos, cell, rb)
    pc = oracle.neighbour_list(pos, cell, rc)
    A, B = _rand_bsr(pa, b, rng), _rand_bsr(pb, b, rng)
    C, triples = oracle.matmul(A, B, pc)
    ref = (A.dense() @ B.dense()) * _mask(pc, b)
    err = np.abs(C.dense() - ref).max() / np.abs(ref).max()
    assert err < 1e-13
    # triple count by brute force over atom indices
    ma = np.zeros((pa.n, pa.n), bool); ma[pa.rows(), pa.col] = True
    mb = np.zeros((pb.n, pb.n), bool); mb[pb.rows(), pb.col] = True
    mc = np.zeros((pc.n, pc.n), bool); mc[pc.rows(), pc.col] = True
    brute = int(np.sum((ma.astype(np.int64) @ mb.astype(np.int64)) * mc))
    assert triples == brute


def test_transpose_identity():
    """(A.B)^T = B^T.A^T on the mirrored (here symmetric) pattern."""
    pos, cell = diamond_si_positions(2, 0.1, 21)
    rng = np.random.default_rng(1)
    pa = oracle.neighbour_list(pos, cell, 4.0)
    pb = oracle.neighbour_list(pos, cell, 6.0)
    pc = oracle.neighbour_list(pos, cell, 7.0)
    A, B = _rand_bsr(pa, 4, rng), _rand_bsr(pb, 4, rng)
    AB, _ = oracle.matmul(A, B, pc)
    BtAt, _ = oracle.matmul(oracle.transpose(B, pb), oracle.transpose(A, pa), pc)
    assert np.abs(oracle.transpose(AB, pc).val - BtAt.val).max() < 1e-12


def test_row_subset_matches_full():
    pos, cell = diamond_si_positions(2, 0.1, 22)
    rng = np.random.default_rng(2)
    p = oracle.neighbour_list(pos, cell, 5.0)
    pc = oracle.neighbour_list(pos, cell, 8.0)
    A, B = _rand_bsr(p, 4, rng), _rand_bsr(p, 4, rng)
    full, _ = oracle.matmul(A, B, pc)
    rows = np.array([0, 7, 33, 63])
    part, _ = oracle.matmul(A, B, pc, rows=rows)
    for i in rows:
        s = slice(pc.ptr[i], pc.ptr[i + 1])
        assert np.array_equal(part.val[s], full.val[s])


def test_trace_equals_dense_trace():
    pos, cell = diamond_si_positions(2, 0.1, 23)
    rng = np.random.default_rng(3)
    px = oracle.neighbour_list(pos, cell, 5.0)
    py = oracle.neighbour_list(pos, cell, 3.0)
    X, Y = _rand_bsr(px, 4, rng), _rand_bsr(py, 4, rng)
    ref = np.trace(X.dense() @ Y.dense())
    assert abs(oracle.trace(X, Y) - ref) < 1e-11 * max(1.0, abs(ref))


def test_identity_and_empty_rows():
    """Identity on the self-only pattern is a neutral factor."""
    pos, cell = diamond_si_positions(1, 0.1, 24)
    p0 = oracle.neighbour_list(pos, cell, 0.5)          # self pairs only
    assert np.all(np.diff(p0.ptr) == 1)
    I = oracle.Bsr(p0, 4, np.broadcast_to(np.eye(4), (p0.nnzb, 4, 4)).copy())
    p = oracle.neighbour_list(pos, cell, 4.0)
    A = _rand_bsr(p, 4, np.random.default_rng(4))
    C, t = oracle.matmul(A, I, p)
    assert np.array_equal(C.val, A.val) and t == p.nnzb
