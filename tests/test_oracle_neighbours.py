"""Pins of the oracle's range patterns (Sec. 2.3.2: elements are zero when
the inter-atomic distance exceeds the cutoff)."""
import os

import numpy as np
import pytest

import oracle
from synth import diamond_si_positions, config_seed


@pytest.mark.parametrize("n,sigma", [(1, 0.05), (2, 0.05), (3, 0.15)])
@pytest.mark.parametrize("R", [2.0, 4.5, 6.6, 10.0, 16.6, 26.6])
def test_cell_list_equals_brute_force(n, sigma, R):
    pos, cell = diamond_si_positions(n, sigma, config_seed(0) + n)
    pb = oracle.neighbour_list(pos, cell, R, "brute")
    pc = oracle.neighbour_list(pos, cell, R, "cell")
    assert pb == pc


def _min_image_d2_numpy(pos, cell):
    d = pos[None, :, :] - pos[:, None, :]
    d -= cell * np.rint(d / cell)
    return np.sum(d * d, axis=-1)


def test_pattern_is_the_distance_set_sorted_symmetric():
    pos, cell = diamond_si_positions(2, 0.1, 7)
    R = 5.0
    p = oracle.neighbour_list(pos, cell, R, "cell")
    d2 = _min_image_d2_numpy(pos, cell)
    keep = d2 <= R * R
    # same set as an independent numpy evaluation (no value within 1e-9 of the cutoff)
    assert np.all(np.abs(d2 - R * R) > 1e-9)
    dense = np.zeros_like(keep)
    dense[p.rows(), p.col] = True
    assert np.array_equal(dense, keep)
    assert np.array_equal(dense, dense.T)
    assert np.all(np.diag(dense))
    for i in range(p.n):
        c = p.col[p.ptr[i]:p.ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


# Coordination shells of the diamond lattice (tests/golden/diamond_shells.txt): radius in units
# of a, atoms in the shell.
_G = np.loadtxt(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "diamond_shells.txt"))
SHELLS = [(np.sqrt(r2 / 16.0), int(c)) for r2, c in _G]


@pytest.mark.parametrize("k", range(len(SHELLS)))
def test_perfect_crystal_shell_counts(k):
    a = 5.431
    pos, cell = diamond_si_positions(4, 0.0, 0)       # half the cell edge: 10.9 A
    r_lo = SHELLS[k][0] * a
    r_hi = SHELLS[k + 1][0] * a if k + 1 < len(SHELLS) else 1.03 * r_lo
    R = 0.5 * (r_lo + r_hi)
    expect = 1 + sum(c for _, c in SHELLS[:k + 1])
    p = oracle.neighbour_list(pos, cell, R, "cell")
    assert np.all(np.diff(p.ptr) == expect)


def test_translation_invariance():
    pos, cell = diamond_si_positions(2, 0.1, 11)
    p0 = oracle.neighbour_list(pos, cell, 6.6)
    shifted = np.mod(pos + np.array([1.37, -2.11, 4.03]), cell)
    p1 = oracle.neighbour_list(shifted, cell, 6.6)
    assert p0 == p1


def test_permutation_covariance():
    pos, cell = diamond_si_positions(2, 0.1, 12)
    perm = np.random.default_rng(0).permutation(pos.shape[0])
    p0 = oracle.neighbour_list(pos, cell, 6.6)
    p1 = oracle.neighbour_list(pos[perm], cell, 6.6)
    inv = np.argsort(perm)
    a = set(zip(p0.rows().tolist(), p0.col.tolist()))
    b = set((int(perm[i]), int(perm[j])) for i, j in zip(p1.rows(), p1.col))
    assert a == b
    del inv


def test_range_beyond_cell_gives_complete_pattern():
    pos, cell = diamond_si_positions(1, 0.05, 3)
    p = oracle.neighbour_list(pos, cell, 100.0, "cell")
    assert np.all(np.diff(p.ptr) == pos.shape[0])


def test_empty_system():
    pos = np.zeros((0, 3))
    cell = np.array([10.0, 10.0, 10.0])
    p = oracle.neighbour_list(pos, cell, 5.0)
    assert p.n == 0 and p.nnzb == 0
