"""Pins of the oracle's Hotelling inverse overlap (Sec. 2.3.2, after Eq. 8).

The pins use dense linear algebra on small cells, not the oracle's own
sparse code: the Newton-Schulz identity of the untruncated iteration, the
dense inverse it converges to, and the masked dense iteration that the
truncated one must equal.
"""
import numpy as np
import pytest

import oracle
from oracle import hotelling as OH
from oracle import lnv as OL
from synth import diamond_si_positions, sk_blocks, config_seed


def _overlap(b=4, n=2, sigma=0.05, seed=config_seed(0)):
    pos, cell = diamond_si_positions(n, sigma, seed)
    m = OL.System(pos, cell)
    pS = m.pattern(6.6)
    H, S = sk_blocks(pos, cell, pS.rows(), pS.col, b=b,
                     perturb_seed=(seed + 7) if b == 13 else None)
    return m, oracle.Bsr(pS, b, S)


def test_scaled_start_bound_and_spectrum():
    m, S = _overlap()
    ev = np.linalg.eigvalsh(S.dense())
    s = OH.row_abs_max(S)
    assert ev.min() > 0 and ev.max() <= s * (1 + 1e-12)
    # the iteration matrix I - X_0 S of the start has spectrum in [0, 1)
    E0 = np.eye(ev.size) - OH.scaled_start(S, m.pattern(10.0)).dense() @ S.dense()
    lam = np.linalg.eigvals(E0).real
    assert lam.min() >= -1e-12 and lam.max() < 1.0


@pytest.mark.parametrize("b", [4, 13])
def test_untruncated_step_squares_the_residual(b):
    # 64 atoms: every min-image distance is below 9.41 A, so R_X = 10 A keeps every block
    m, S = _overlap(b)
    Sd = S.dense()
    X = OH.scaled_start(S, m.pattern(10.0))
    eye = np.eye(Sd.shape[0])
    for _ in range(3):
        E = eye - X.dense() @ Sd
        Xn = OH.hotelling_step(m, S, X)
        En = eye - Xn.dense() @ Sd
        assert np.abs(En - E @ E).max() <= 1e-12 * max(1.0, np.abs(E).max())
        X = Xn


@pytest.mark.parametrize("b", [4, 13])
def test_untruncated_iteration_reaches_dense_inverse(b):
    m, S = _overlap(b)
    X, hist = OH.hotelling(m, S, 10.0, 30)
    Sinv = np.linalg.inv(S.dense())
    assert np.abs(X.dense() - Sinv).max() <= 1e-12 * np.abs(Sinv).max()
    assert hist[-1] <= 1e-12 * np.sqrt(np.sum(Sinv ** 2))
    # quadratic convergence: the change at least squares (relative) once it is small
    rel = [h / np.sqrt(np.sum(Sinv ** 2)) for h in hist]
    k = next(i for i, r in enumerate(rel) if r < 1e-2)
    assert rel[k + 1] <= 10 * rel[k] ** 2 + 1e-14


def test_truncated_iteration_is_the_masked_dense_one():
    m, S = _overlap(n=3, sigma=0.1, seed=config_seed(0) + 5)
    R_X = 5.0
    pX = m.pattern(R_X)
    X = OH.scaled_start(S, pX)
    mask = oracle.Bsr(pX, 4, np.ones((pX.nnzb, 4, 4))).dense() != 0
    Sd, Xd = S.dense(), X.dense()
    for _ in range(12):
        X = OH.hotelling_step(m, S, X)
        Xd = np.where(mask, 2 * Xd - Xd @ Sd @ Xd, 0.0)
        assert np.abs(X.dense() - Xd).max() <= 1e-12 * np.abs(Xd).max()
    # truncated X stays symmetric and S X approaches the identity on the diagonal blocks
    Xf = X.dense()
    assert np.abs(Xf - Xf.T).max() <= 1e-13 * np.abs(Xf).max()
    assert np.abs(np.diag(Xf @ Sd) - 1.0).max() < 0.05
