"""Sparse approximate inverse overlap by the Hotelling iteration (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.3.2, the paragraph after Eq. 8: the LNV minimisation uses an
approximate, sparse inverse of the overlap matrix as the metric of the
optimisation, found with the iterative Hotelling method.  The paper gives
no formula; the Hotelling (Newton-Schulz) iteration for an inverse is

    X_{n+1} = 2 X_n - X_n S X_n,

for which I - X_{n+1} S = (I - X_n S)^2 when nothing is truncated, so it
converges quadratically once the spectral radius of I - X_0 S is below one.

Readings taken here:
  * X has its own range R_X; the product X S is kept at its natural range
    R_X + R_S and X S X is restricted to R_X (the truncated iteration);
  * X_0 = S / s^2 restricted to R_X, with s the largest absolute row sum
    of S (Gershgorin: s bounds the largest eigenvalue of the positive
    definite S), so that the eigenvalues of I - X_0 S = I - S^2 / s^2 lie in
    [0, 1) and the iteration converges; the block-Jacobi start
    X_0 = S_ii^{-1} does not converge for the Slater-Koster overlaps used
    here (the spectral radius of I - X_0 S exceeds one);
  * the reported change of step n is the Frobenius norm of X_{n+1} - X_n.
"""
import numpy as np

from . import dot, restrict
from .lnv import mm


def row_abs_max(S):
    """Largest absolute row sum of S (over the scalar rows of its blocks)."""
    n, b = S.pat.n, S.b
    sums = np.zeros((n, b))
    np.add.at(sums, S.pat.rows(), np.abs(S.val).sum(axis=2))
    return float(sums.max())


def scaled_start(S, pat_X):
    """X_0 = S / s^2 on X's range, s = row_abs_max(S)."""
    s = row_abs_max(S)
    return (1.0 / (s * s)) * restrict(S, pat_X)


def hotelling_step(sysm, S, X):
    """One truncated step: X S at its natural range, then (X S) X on X's range."""
    XS = mm(sysm, X, S)
    XSX = mm(sysm, XS, X, R=X.pat.R)
    return 2.0 * X - XSX


def hotelling(sysm, S, R_X, n_iter, X0=None):
    """n_iter steps from X0 (default: scaled_start).  Returns (X, [|X_{n+1} - X_n|_F])."""
    X = scaled_start(S, sysm.pattern(R_X)) if X0 is None else X0.copy()
    hist = []
    for _ in range(n_iter):
        Xn = hotelling_step(sysm, S, X)
        d = Xn - X
        hist.append(float(np.sqrt(dot(d, d))))
        X = Xn
    return X, hist
