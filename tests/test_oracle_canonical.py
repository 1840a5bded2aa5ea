"""Pins of the oracle's canonical (fixed electron number) LNV minimisation (Sec. 2.3.2).

The canonical problem at N0 = N_e of the grand-canonical minimum at mu has
the same minimiser, and its Lagrange multiplier is the chemical potential:
the grand-canonical CG (itself pinned against diagonalisation elsewhere)
pins the canonical one.  Along the way N_e stays at N0 and E_band falls.
"""
import numpy as np
import pytest

import oracle
from oracle import lnv as OL
from synth import config_seed, diamond_si_positions, sk_blocks

MU = -2.0
R_L = 8.0


@pytest.fixture(scope="module")
def both():
    pos, cell = diamond_si_positions(2, 0.05, config_seed(0))
    m = OL.System(pos, cell)
    pH = m.pattern(6.6)
    H, S = sk_blocks(pos, cell, pH.rows(), pH.col)
    Hb, Sb = oracle.Bsr(pH, 4, H), oracle.Bsr(pH, 4, S)
    gc = OL.Lnv(m, Sb, Hb, R_L, MU)
    L0 = OL.onsite_inverse_half(Sb, gc.pat_L)
    Lg, _ = OL.minimise(gc, L0, 150, tol_ha_per_atom=1e-10)
    n0 = gc.energy(Lg)[1]
    le = OL.Lnv(m, Sb, Hb, R_L, 0.0)                       # Omega at mu = 0 is E_band
    ln = OL.Lnv(m, Sb, oracle.restrict(Sb, pH), R_L, 0.0)  # its "Omega" is N_e
    Lc, hc = OL.minimise_canonical(le, ln, L0, n0, 150, tol_ha_per_atom=1e-10)
    return le, ln, Lg, Lc, hc, n0


def test_energy_and_electron_number_views(both):
    le, ln, Lg, Lc, hc, n0 = both
    E, N = le.energy(Lg)
    assert np.isclose(ln.energy(Lg)[0], N, rtol=1e-12)  # 2 Tr[K S] from the S-as-H view
    om_gc = E - MU * N
    assert np.isclose(OL.Lnv(le.sys, le.S, le.H, R_L, MU).energy(Lg)[0], om_gc, rtol=1e-12)


def test_canonical_keeps_the_electron_number_and_lowers_the_energy(both):
    le, ln, Lg, Lc, hc, n0 = both
    for h in hc:
        assert abs(h["ne"] - n0) <= 1e-9 * n0
    e = [h["energy"] for h in hc]
    assert all(b <= a + 1e-9 for a, b in zip(e, e[1:]))


def test_canonical_minimum_is_the_grand_canonical_one(both):
    le, ln, Lg, Lc, hc, n0 = both
    Eg, Ec = le.energy(Lg)[0], le.energy(Lc)[0]
    assert abs(Ec - Eg) <= 1e-8 * abs(Eg)
    assert np.abs(Lc.val - Lg.val).max() <= 1e-4 * np.abs(Lg.val).max()
    # the Lagrange multiplier of the electron number is the chemical potential
    assert abs(hc[-1]["lam"] - MU) <= 1e-3
