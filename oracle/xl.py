"""Extended-Lagrangian propagation of the density matrix between MD steps (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 3.3 (molecular dynamics): an auxiliary sparse matrix X, associated with
L S rather than L, moves in a harmonic potential centred on the ground
state L(t) S(t); integrated by Verlet,

    X(t + dt) = 2 X(t) - X(t - dt) + dt^2 w^2 [L(t) S(t) - X(t)],

and X S^-1 is the initial L of the next step's minimisation.  A dissipative
term a sum_{m=0}^{M} c_m X(t - m dt) is added to keep X near the centre.

Readings taken here (the paper gives no more):
  * kappa = dt^2 w^2, a and the c_m are inputs (the paper quotes no values;
    the scheme it cites for the dissipation tabulates sets of them);
  * X lives on the range of L S (R_L + R_S), the natural range of the
    product; every X(t - m dt) of the history is held on the current
    geometry's pattern: when the atoms move, a matrix moves to the new
    pattern block by block, matched by atom pair, blocks of pairs that
    left the range are dropped and pairs that entered start at zero;
  * the initial L is the symmetric part of (X S^-1) restricted to L's range:
    X S^-1 equals L only at the harmonic centre, and L is symmetric.
"""
import numpy as np

from . import Bsr, restrict, transpose
from .lnv import mm


def remap(X, pat_new):
    """X moved to another pattern of the same atoms: block (i, j) kept where both hold it."""
    return restrict(X, pat_new)


def propagate(hist, LS, kappa, alpha=0.0, c=None):
    """X(t + dt) from hist = [X(t), X(t - dt), ..., X(t - M dt)] and LS = L(t) S(t).

    2 X(t) - X(t - dt) + kappa (LS - X(t)) + alpha sum_m c_m X(t - m dt), evaluated in
    that order, every operation rounded once.
    """
    X0, X1 = hist[0], hist[1]
    out = 2.0 * X0.val - X1.val
    out = out + kappa * (LS.val - X0.val)
    if alpha != 0.0:
        assert c is not None and len(c) <= len(hist)
        s = c[0] * hist[0].val
        for m in range(1, len(c)):
            s = s + c[m] * hist[m].val
        out = out + alpha * s
    return Bsr(X0.pat, X0.b, out)


def initial_L(sysm, X, Sinv, R_L):
    """L_0 = symmetric part of (X S^-1) on L's range."""
    P = mm(sysm, X, Sinv, R=R_L)
    return Bsr(P.pat, P.b, 0.5 * (P.val + transpose(P, P.pat).val))
