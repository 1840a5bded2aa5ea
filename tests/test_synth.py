"""Pins of the seeded Slater-Koster inputs (textbook two-centre table)."""
import numpy as np

import oracle
from synth import diamond_si_positions, sk_blocks, SK_H, SK_S, config_seed


def test_dimer_along_x_closed_form():
    pos = np.array([[10.0, 10.0, 10.0], [12.35, 10.0, 10.0]])
    cell = np.array([40.0, 40.0, 40.0])
    H, S = sk_blocks(pos, cell, np.array([0]), np.array([1]))
    h = H[0]
    # r = 2.35: scale factors are exactly 1; bond along +x (l = 1)
    assert np.isclose(h[0, 0], SK_H["sss"])
    assert np.isclose(h[0, 1], SK_H["sps"]) and np.isclose(h[1, 0], -SK_H["sps"])
    assert np.isclose(h[1, 1], SK_H["pps"])
    assert np.isclose(h[2, 2], SK_H["ppp"]) and np.isclose(h[3, 3], SK_H["ppp"])
    assert np.allclose(h[0, 2:], 0) and np.allclose(h[2, 3], 0)
    assert np.isclose(S[0][1, 1], SK_S["pps"])


def test_scaling_laws_and_cutoff():
    cell = np.array([40.0, 40.0, 40.0])
    for r, fc in [(3.0, 1.0), (6.1, 0.5), (6.7, 0.0)]:
        pos = np.array([[5.0, 5.0, 5.0], [5.0, 5.0, 5.0 + r]])
        H, S = sk_blocks(pos, cell, np.array([0]), np.array([1]))
        assert np.isclose(H[0][0, 0], SK_H["sss"] * (2.35 / r) ** 2 * fc)
        assert np.isclose(S[0][0, 0], SK_S["sss"] * np.exp(-2 * (r / 2.35 - 1)) * fc)
        # bond along +z: p_z p_z is sigma
        assert np.isclose(H[0][3, 3], SK_H["pps"] * (2.35 / r) ** 2 * fc)


def _hs(n, sigma, seed, b=4, perturb=None):
    pos, cell = diamond_si_positions(n, sigma, seed)
    p = oracle.neighbour_list(pos, cell, 6.6)
    H, S = sk_blocks(pos, cell, p.rows(), p.col, b=b, perturb_seed=perturb)
    return pos, cell, p, oracle.Bsr(p, b, H), oracle.Bsr(p, b, S)


def test_symmetric_and_positive_definite():
    for n in (1, 2):
        _, _, _, H, S = _hs(n, 0.05, config_seed(0))
        Hd, Sd = H.dense(), S.dense()
        assert np.array_equal(Hd, Hd.T)
        assert np.abs(Sd - Sd.T).max() == 0.0
        np.linalg.cholesky(Sd)


def test_b13_symmetric_and_perturbed():
    _, _, _, H, S = _hs(1, 0.1, 5, b=13, perturb=99)
    Hd = H.dense()
    assert np.abs(Hd - Hd.T).max() == 0.0
    np.linalg.cholesky(S.dense())
    _, _, _, H0, _ = _hs(1, 0.1, 5, b=13)
    dev = np.abs(H.val - H0.val)
    assert dev.max() <= 0.1 and dev.max() > 0.05


def test_perfect_crystal_onsite_blocks_equal():
    _, _, p, H, S = _hs(3, 0.0, 0)
    diag = p.rows() == p.col
    assert np.abs(H.val[diag] - H.val[diag][0]).max() < 1e-12
    assert np.abs(S.val[diag] - S.val[diag][0]).max() < 1e-12


def test_translation_invariance_of_blocks():
    pos, cell = diamond_si_positions(2, 0.1, 31)
    p = oracle.neighbour_list(pos, cell, 6.6)
    H0, S0 = sk_blocks(pos, cell, p.rows(), p.col)
    shifted = np.mod(pos + np.array([0.77, 3.1, -1.9]), cell)
    H1, S1 = sk_blocks(shifted, cell, p.rows(), p.col)
    assert np.abs(H0 - H1).max() < 1e-11 and np.abs(S0 - S1).max() < 1e-11
