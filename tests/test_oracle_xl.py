"""Pins of the oracle's extended-Lagrangian propagation of X (Sec. 3.3).

Closed forms of the Verlet recursion (the harmonic oscillator about a fixed
L S), of the dissipation on a history that is a cubic in time (which tells
the index direction and sign of the sum apart), the fixed point, brute-force
pair matching of a matrix moved between the patterns of two geometries, and
dense algebra for the initial L (X S^-1 = L at the centre; masked dense
product when truncated).
"""
import os

import numpy as np
import pytest

import oracle
from oracle import lnv as OL
from oracle import xl as OX
from synth import config_seed, diamond_si_positions, md_trajectory, sk_blocks


def read_dissipation():
    """(kappa, alpha, c) from tests/golden/xl_dissipation_k5.txt (the cited table's K = 5 row)."""
    vals = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "xl_dissipation_k5.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            key, *rest = line.split()
            vals[key] = [float(x) for x in rest]
    return vals["kappa"][0], vals["alpha"][0], np.array(vals["c"])


KAPPA, ALPHA, C5 = read_dissipation()


def test_dissipation_coefficients_annihilate_constant_and_linear_histories():
    m = np.arange(len(C5), dtype=float)
    assert np.sum(C5) == 0.0 and np.sum(m * C5) == 0.0
    assert 0.0 < KAPPA < 4.0                      # the undamped Verlet recursion is stable


def test_binding_default_is_the_golden_row():
    import paper_2002_07704_gb300 as lsq
    kappa, alpha, c = lsq.XL_DISSIPATION_K5
    assert (kappa, alpha) == (KAPPA, ALPHA) and np.array_equal(np.array(c), C5)


def _rand_bsr(pat, b, rng):
    return oracle.Bsr(pat, b, rng.standard_normal((pat.nnzb, b, b)))


@pytest.fixture(scope="module")
def small():
    pos, cell = diamond_si_positions(2, 0.05, config_seed(0))
    m = OL.System(pos, cell)
    return m, m.pattern(6.6)


def test_verlet_without_dissipation_is_the_harmonic_closed_form(small):
    m, p = small
    rng = np.random.default_rng(1)
    D = _rand_bsr(p, 4, rng)
    Xm1, X0 = _rand_bsr(p, 4, rng), _rand_bsr(p, 4, rng)
    hist = [X0, Xm1]
    for _ in range(40):
        hist = [OX.propagate(hist, D, KAPPA), hist[0]]
    # e_{n+1} = (2 - kappa) e_n - e_{n-1}  =>  e_n = A cos(n th) + B sin(n th), cos th = 1 - kappa / 2
    th = np.arccos(1.0 - KAPPA / 2.0)
    A = X0.val - D.val
    Bc = (A * np.cos(th) - (Xm1.val - D.val)) / np.sin(th)
    want = D.val + A * np.cos(40 * th) + Bc * np.sin(40 * th)
    assert np.abs(hist[0].val - want).max() <= 1e-10 * np.abs(want).max()


def test_dissipation_on_a_cubic_history(small):
    m, p = small
    rng = np.random.default_rng(2)
    A = _rand_bsr(p, 4, rng)
    t = 10.0
    hist = [oracle.Bsr(p, 4, (t - k) ** 3 * A.val) for k in range(6)]
    LS = hist[0].copy()                       # kappa term off: L S on X(t)
    got = OX.propagate(hist, LS, 0.0, ALPHA, C5)
    # sum_m c_m (t - m)^3 = t^3 S0 - 3 t^2 S1 + 3 t S2 - S3,  S_k = sum_m m^k c_m
    mm_ = np.arange(6.0)
    S = [float(np.sum(mm_ ** k * C5)) for k in range(4)]
    diss = t ** 3 * S[0] - 3 * t ** 2 * S[1] + 3 * t * S[2] - S[3]
    want = (2 * t ** 3 - (t - 1) ** 3 + ALPHA * diss) * A.val
    assert np.abs(got.val - want).max() <= 1e-12 * np.abs(want).max()
    assert abs(diss - (-18.0 * t)) < 1e-12          # this set's moments: S0 = S1 = S3 = 0, S2 = -6


def test_fixed_point(small):
    m, p = small
    D = _rand_bsr(p, 4, np.random.default_rng(3))
    got = OX.propagate([D] * 6, D, KAPPA, ALPHA, C5)
    assert np.abs(got.val - D.val).max() <= 1e-14 * np.abs(D.val).max()


def test_remap_between_geometries_matches_pairs():
    pos, cell = diamond_si_positions(3, 0.05, config_seed(0) + 3)
    traj = md_trajectory(pos, cell, 6, seed=17, amp=0.3)
    m0, m1 = OL.System(traj[0], cell), OL.System(traj[6], cell)
    p0, p1 = m0.pattern(5.0), m1.pattern(5.0)
    assert not np.array_equal(p0.col, p1.col)          # the motion changed the pairs in range
    X0 = _rand_bsr(p0, 4, np.random.default_rng(4))
    X1 = OX.remap(X0, p1)
    old = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(p0.rows(), p0.col))}
    for k, (i, j) in enumerate(zip(p1.rows(), p1.col)):
        src = old.get((int(i), int(j)))
        if src is None:
            assert not X1.val[k].any()
        else:
            assert np.array_equal(X1.val[k], X0.val[src])
    back = OX.remap(X1, p0)
    new = {(int(i), int(j)) for i, j in zip(p1.rows(), p1.col)}
    for k, (i, j) in enumerate(zip(p0.rows(), p0.col)):
        want = X0.val[k] if (int(i), int(j)) in new else 0.0
        assert np.array_equal(back.val[k], np.broadcast_to(want, (4, 4)))


def test_initial_L_at_the_harmonic_centre_is_L():
    # 64 atoms, every range beyond the largest minimum-image distance (9.4 A): no truncation
    pos, cell = diamond_si_positions(2, 0.05, config_seed(0))
    m = OL.System(pos, cell)
    pf = m.pattern(10.0)
    _, Sv = sk_blocks(pos, cell, pf.rows(), pf.col)
    S = oracle.Bsr(pf, 4, Sv)
    rng = np.random.default_rng(5)
    Lr = rng.standard_normal((256, 256))
    L = oracle.Bsr.from_dense(Lr + Lr.T, pf, 4)
    X = oracle.Bsr.from_dense(L.dense() @ S.dense(), m.pattern(16.6), 4)
    Sinv = oracle.Bsr.from_dense(np.linalg.inv(S.dense()), pf, 4)
    L0 = OX.initial_L(m, X, Sinv, 10.0)
    assert np.abs(L0.val - L.val).max() <= 1e-10 * np.abs(L.val).max()


def test_truncated_initial_L_is_the_masked_dense_product():
    pos, cell = diamond_si_positions(3, 0.1, config_seed(0) + 5)
    m = OL.System(pos, cell)
    R_L, R_X = 5.0, 4.0
    pl, px, ps = m.pattern(R_L), m.pattern(R_L + 6.6), m.pattern(R_X)
    rng = np.random.default_rng(6)
    X = _rand_bsr(px, 4, rng)
    Sinv = _rand_bsr(ps, 4, rng)
    Sinv = oracle.Bsr(ps, 4, 0.5 * (Sinv.val + oracle.transpose(Sinv, ps).val))
    mask = oracle.Bsr(pl, 4, np.ones((pl.nnzb, 4, 4))).dense() != 0
    P = np.where(mask, X.dense() @ Sinv.dense(), 0.0)
    want = 0.5 * (P + P.T)
    got = OX.initial_L(m, X, Sinv, R_L)
    assert np.abs(got.dense() - want).max() <= 1e-12 * np.abs(want).max()
    assert np.array_equal(got.dense(), got.dense().T)
