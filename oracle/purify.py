"""Initial density matrix from the Hamiltonian by McWeeny purification (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.3.2, after Eq. 8: the initial density matrix is generated from the
Hamiltonian by an iterative procedure that generalises the McWeeny
transform (the references are Palser and Manolopoulos, and Bowler and
Gillan).  The paper gives no formula.  Reading taken here: the
grand-canonical purification at the chemical potential mu, written for a
non-orthogonal basis with an approximate inverse overlap X ~ S^-1 (from
the Hotelling iteration):

    K_0 = (lam / 2) (mu X - X H X) + X / 2,
    lam = min(1 / (e_max - mu), 1 / (mu - e_min)),

so that with X = S^-1 the eigenvalues of K_0 S are 1/2 + lam (mu - e) / 2,
in [0, 1] for every generalised eigenvalue e of (H, S) in [e_min, e_max];
then the McWeeny step

    K_{n+1} = 3 K_n S K_n - 2 K_n S K_n S K_n

drives the eigenvalues of K S below 1/2 to 0 and those above to 1 (the
states below mu become occupied).  [e_min, e_max] are the Gershgorin
bounds of X H: over its scalar rows, the diagonal element minus and plus
the sum of the other absolute values in the row.

Truncation: K lives on L's range; X H is kept at its natural range and
(X H) X restricted to L's range; K S is kept at its natural range and
(K S) K and (K S)(K S K) are restricted to L's range.  Each K is
symmetrised, as the CG's gradients are.
"""
import numpy as np

from . import dot, restrict, transpose
from .lnv import mm


def gershgorin_bounds(XH):
    """(e_min, e_max) over the scalar rows of XH (diagonal -/+ off-diagonal absolute sum)."""
    n, b = XH.pat.n, XH.b
    rows = XH.pat.rows()
    absum = np.zeros((n, b))
    np.add.at(absum, rows, np.abs(XH.val).sum(axis=2))
    diag = np.zeros((n, b))
    on = rows == XH.pat.col
    diag[rows[on]] = np.diagonal(XH.val[on], axis1=1, axis2=2)
    radius = absum - np.abs(diag)
    return float((diag - radius).min()), float((diag + radius).max())


def _sym(K):
    return 0.5 * (K + transpose(K, K.pat))


def initial(sysm, S, H, X, mu, R_L):
    """K_0 on L's range and (lam, e_min, e_max)."""
    pl = sysm.pattern(R_L)
    XH = mm(sysm, X, H)
    e_min, e_max = gershgorin_bounds(XH)
    lam = min(1.0 / (e_max - mu), 1.0 / (mu - e_min))
    XHX = mm(sysm, XH, X, R=R_L)
    XL = restrict(X, pl)
    K0 = (0.5 * lam) * (mu * XL - XHX) + 0.5 * XL
    return _sym(K0), (lam, e_min, e_max)


def mcweeny_step(sysm, S, K):
    KS = mm(sysm, K, S)
    KSK = mm(sysm, KS, K, R=K.pat.R)
    KSKSK = mm(sysm, KS, KSK, R=K.pat.R)
    return _sym(3.0 * KSK - 2.0 * KSKSK)


def purify(sysm, S, H, X, mu, R_L, n_iter):
    """K after n_iter McWeeny steps from K_0; returns (K, [|K_{n+1} - K_n|_F], (lam, e_min, e_max))."""
    K, bounds = initial(sysm, S, H, X, mu, R_L)
    hist = []
    for _ in range(n_iter):
        Kn = mcweeny_step(sysm, S, K)
        d = Kn - K
        hist.append(float(np.sqrt(dot(d, d))))
        K = Kn
    return K, hist, bounds
