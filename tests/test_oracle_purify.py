"""Pins of the oracle's initial density matrix by McWeeny purification (Sec. 2.3.2).

Dense linear algebra only: the generalised eigenproblem (H, S) for the
bounds, the spectrum of K_0 S and the occupied projector the full-range
purification must reach; the masked dense iteration the truncated one
must equal.
"""
import numpy as np
import pytest
import scipy.linalg as sl

import oracle
from oracle import hotelling as OH
from oracle import lnv as OL
from oracle import purify as OP
from synth import config_seed, diamond_si_positions, sk_blocks

MU = -2.0


def _problem(n=2, sigma=0.05, seed=config_seed(0)):
    pos, cell = diamond_si_positions(n, sigma, seed)
    m = OL.System(pos, cell)
    pH = m.pattern(6.6)
    H, S = sk_blocks(pos, cell, pH.rows(), pH.col)
    return m, oracle.Bsr(pH, 4, H), oracle.Bsr(pH, 4, S)


@pytest.fixture(scope="module")
def full():
    # 64 atoms, ranges beyond the largest minimum-image distance (9.4 A): nothing truncated
    m, H, S = _problem()
    X, _ = OH.hotelling(m, S, 10.0, 30)
    return m, H, S, X


def test_bounds_contain_the_generalised_spectrum(full):
    m, H, S, X = full
    w = sl.eigh(H.dense(), S.dense(), eigvals_only=True)
    e_min, e_max = OP.gershgorin_bounds(OL.mm(m, X, H))
    assert e_min <= w.min() and w.max() <= e_max


def test_start_spectrum_in_unit_interval(full):
    m, H, S, X = full
    K0, (lam, e_min, e_max) = OP.initial(m, S, H, X, MU, 12.0)
    ev = np.linalg.eigvals(K0.dense() @ S.dense()).real
    assert ev.min() >= -1e-12 and ev.max() <= 1.0 + 1e-12
    # the eigenvalues are 1/2 + lam (mu - e) / 2 for the generalised eigenvalues e
    w = sl.eigh(H.dense(), S.dense(), eigvals_only=True)
    assert np.allclose(np.sort(ev), np.sort(0.5 + 0.5 * lam * (MU - w)), atol=1e-10)


def test_full_range_purification_reaches_the_occupied_projector(full):
    m, H, S, X = full
    K, hist, _ = OP.purify(m, S, H, X, MU, 12.0, 40)
    w, C = sl.eigh(H.dense(), S.dense())
    occ = w < MU
    Kex = C[:, occ] @ C[:, occ].T
    assert np.abs(K.dense() - Kex).max() <= 1e-10 * np.abs(Kex).max()
    assert abs(2.0 * oracle.trace(K, S) - 2.0 * occ.sum()) <= 1e-9


def test_truncated_purification_is_the_masked_dense_one():
    m, H, S = _problem(n=3, sigma=0.1, seed=config_seed(0) + 9)
    R_L = 5.0
    X, _ = OH.hotelling(m, S, 6.6, 12)
    pl = m.pattern(R_L)
    mask = oracle.Bsr(pl, 4, np.ones((pl.nnzb, 4, 4))).dense() != 0
    Xd, Hd, Sd = X.dense(), H.dense(), S.dense()
    XH = Xd @ Hd
    d = np.diag(XH)
    rad = np.abs(XH).sum(axis=1) - np.abs(d)
    e_min, e_max = (d - rad).min(), (d + rad).max()
    lam = min(1.0 / (e_max - MU), 1.0 / (MU - e_min))
    XL = np.where(mask, Xd, 0.0)
    K = 0.5 * lam * (MU * XL - np.where(mask, XH @ Xd, 0.0)) + 0.5 * XL
    K = 0.5 * (K + K.T)
    Ko, _ = OP.initial(m, S, H, X, MU, R_L)
    assert np.abs(Ko.dense() - K).max() <= 1e-12 * np.abs(K).max()
    for _ in range(6):
        KS = K @ Sd
        B = np.where(mask, KS @ K, 0.0)
        Cm = np.where(mask, KS @ B, 0.0)
        K = 3 * B - 2 * Cm
        K = 0.5 * (K + K.T)
        Ko = OP.mcweeny_step(m, S, Ko)
        assert np.abs(Ko.dense() - K).max() <= 1e-11 * np.abs(K).max()
