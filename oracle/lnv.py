"""LNV grand-potential minimisation, written out step by step (oracle side).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Sec. 2.3.2 ("Density matrix: linear scaling") of the paper: the density
matrix is K = 3LSL - 2LSLSL (the McWeeny form, Eq. 8) of an auxiliary
matrix L whose range is restricted; K has the range of H; the band energy
E_band = 2 Tr[K H] is minimised with respect to L using the gradient
dE/dL, with the electron number held by a chemical potential.  The
paper's CG runs reset the search direction every 40 iterations (the
caption of the 17,102-atom gramicidin convergence figure, Sec. 5.3).

Readings taken here (the paper gives no formula for them):
  * grand potential Omega = 2 Tr[K (H - mu S)] = E_band - mu N_e with the
    spin factor 2 of E_band, and electron count N_e = 2 Tr[K S];
  * gradient G_ab = dOmega/dL_ab for every stored entry of L,
    G = 2 [3 X - 2 Y]^T restricted to L's range, where
    X = SLH' + H'LS and Y = SLSLH' + SLH'LS + H'LSLS, H' = H - mu S;
  * L is symmetric (it is a density matrix), so the minimisation runs over
    symmetric L and its search directions use the symmetric part
    (G + G^T) / 2 of the gradient.  At symmetric L this equals G in exact
    arithmetic; taking it explicitly stops rounding from seeding an
    antisymmetric component, along which Omega is unbounded below;
  * conjugate gradients of Polak-Ribiere form, beta = max(0, beta_PR),
    direction reset to -G every 40 steps (or to -X G X with the metric X of
    metric_gradient), and an exact line minimisation:
    Omega(L + a D) is a cubic c0 + c1 a + c2 a^2 + c3 a^3 in a and the step
    is its local minimum.
Intermediate products are kept at their natural range (the sum of their
factors' ranges), so no truncation enters beyond L's own range and the
final restriction of each trace to H's range.
"""
import time

import numpy as np

from . import Bsr, Pattern, dot, matmul, neighbour_list, restrict, trace, transpose

HA_EV = 27.211386245988     # Hartree in eV (CODATA 2018)


class System:
    """Atom positions in an orthorhombic periodic cell, with a pattern cache."""

    def __init__(self, pos, cell):
        self.pos = np.ascontiguousarray(pos, dtype=np.float64)
        self.cell = np.ascontiguousarray(cell, dtype=np.float64)
        self.n = self.pos.shape[0]
        self._pats = {}

    def pattern(self, R):
        R = float(R)
        if R not in self._pats:
            self._pats[R] = neighbour_list(self.pos, self.cell, R, method="cell")
        return self._pats[R]


_sample = {"rows": None, "mm_seconds": 0.0}


class row_sample:
    """Context manager for timing a sample of a large workload: inside it,
    every block product of the LNV steps is evaluated on the given rows of
    its result only (other rows stay zero) and the time spent in products
    is accumulated.  Results are not meaningful inside the context."""

    def __init__(self, rows):
        self.rows = np.ascontiguousarray(rows, dtype=np.int32)

    def __enter__(self):
        _sample["rows"] = self.rows
        _sample["mm_seconds"] = 0.0
        return self

    def __exit__(self, *exc):
        self.mm_seconds = _sample["mm_seconds"]
        _sample["rows"] = None
        return False


def mm(sysm, A, B, R=None):
    """A.B on its natural range R_A + R_B, or truncated to range R."""
    if R is None:
        R = A.pat.R + B.pat.R
    pat = sysm.pattern(R)
    t0 = time.perf_counter()
    C, _ = matmul(A, B, pat, rows=_sample["rows"])
    _sample["mm_seconds"] += time.perf_counter() - t0
    return C


def onsite_inverse_half(S, pat_L):
    """Initial L: one half of the inverse of each on-site block S_ii, zero elsewhere.

    Each block is symmetrised after inversion so that L starts exactly symmetric.
    """
    b = S.b
    L = Bsr(pat_L, b)
    for i in range(pat_L.n):
        ps = np.searchsorted(S.pat.col[S.pat.ptr[i]:S.pat.ptr[i + 1]], i) + S.pat.ptr[i]
        pl = np.searchsorted(pat_L.col[pat_L.ptr[i]:pat_L.ptr[i + 1]], i) + pat_L.ptr[i]
        inv = np.linalg.inv(S.val[ps])
        L.val[pl] = 0.25 * (inv + inv.T)
    return L


class Lnv:
    """Omega, N_e, gradient and CG for fixed S, H (on R_H's range) and mu."""

    def __init__(self, sysm, S, H, R_L, mu, spin=2.0):
        self.sys = sysm
        self.b = S.b
        self.pat_H = H.pat
        self.pat_L = sysm.pattern(R_L)
        self.S = restrict(S, self.pat_H)
        self.H = H
        self.mu = float(mu)
        self.spin = float(spin)
        self.Hp = H - self.mu * self.S          # H' = H - mu S

    # -- Eq. 8 and E_band = 2 Tr[K H] ------------------------------------
    def energy(self, L):
        """(Omega, N_e) in eV and electrons, with K = 3LSL - 2LSLSL on H's range."""
        m = self.sys
        LS = mm(m, L, self.S)
        SL = mm(m, self.S, L)
        LSL = mm(m, LS, L)
        LSLSL_H = mm(m, LSL, SL, R=self.pat_H.R)
        K = 3.0 * restrict(LSL, self.pat_H) - 2.0 * LSLSL_H
        return self.spin * trace(K, self.Hp), self.spin * trace(K, self.S)

    def gradient(self, L):
        """G_ab = dOmega/dL_ab on L's range."""
        m, pl = self.sys, self.pat_L
        LS = mm(m, L, self.S)
        SL = mm(m, self.S, L)
        SLHp = mm(m, SL, self.Hp)
        HpLS = mm(m, self.Hp, LS)
        X = restrict(SLHp, pl) + restrict(HpLS, pl)
        Y = (mm(m, SL, SLHp, R=pl.R) + mm(m, SL, HpLS, R=pl.R) + mm(m, HpLS, LS, R=pl.R))
        return self.spin * transpose(3.0 * X - 2.0 * Y, pl)

    def cubic(self, L, D, G):
        """Coefficients (c1, c2, c3) of Omega(L + a D) - Omega(L) = c1 a + c2 a^2 + c3 a^3.

        Expanding Eq. 8 with L -> L + a D:
          c1 = sum_ab G_ab D_ab,
          c2 = 2 (3 Tr[DSDH'] - 2 (Tr[DSDSLH'] + Tr[DSLSDH'] + Tr[LSDSDH'])),
          c3 = -4 Tr[DSDSDH'].
        """
        m, RH = self.sys, self.pat_H.R
        LS = mm(m, L, self.S)
        DS = mm(m, D, self.S)
        DSD = mm(m, DS, D)
        DSDS = mm(m, DSD, self.S)
        DSLS = mm(m, DS, LS)
        LSDS = mm(m, LS, DS)
        t2 = trace(DSD, self.Hp)
        t3a = trace(mm(m, DSDS, L, R=RH), self.Hp)
        t3b = trace(mm(m, DSLS, D, R=RH), self.Hp)
        t3c = trace(mm(m, LSDS, D, R=RH), self.Hp)
        t4 = trace(mm(m, DSDS, D, R=RH), self.Hp)
        c1 = dot(G, D)
        c2 = self.spin * (3.0 * t2 - 2.0 * (t3a + t3b + t3c))
        c3 = -2.0 * self.spin * t4
        return c1, c2, c3


def line_minimum(c1, c2, c3):
    """Step a > 0 along a descent direction (c1 < 0) for c1 a + c2 a^2 + c3 a^3, or None.

    The stationary points solve 3 c3 a^2 + 2 c2 a + c1 = 0; the one with
    positive curvature is a = -c1 / (c2 + sqrt(c2^2 - 3 c1 c3)).  When the
    cubic has no local minimum (negative discriminant) but positive
    curvature at a = 0 (c2 > 0), the minimum of its quadratic part,
    a = -c1 / (2 c2), is taken; otherwise there is no safe step.
    """
    disc = c2 * c2 - 3.0 * c1 * c3
    if disc >= 0.0:
        den = c2 + np.sqrt(disc)
        if den > 0.0:
            return -c1 / den
    if c2 > 0.0:
        return -c1 / (2.0 * c2)
    return None


def metric_gradient(lnv, G, X):
    """The gradient in the metric X ~ S^-1: P = (X G X) restricted to L's range.

    Sec. 2.3.2 (after Eq. 8): the minimisation uses an approximate sparse
    inverse overlap as its metric.  G is covariant in the non-orthogonal
    basis; X G X is the corresponding contravariant direction.  X G is kept
    at its natural range, then (X G) X is restricted to L's range and
    symmetrised like G.
    """
    m = lnv.sys
    XG = mm(m, X, G)
    P = mm(m, XG, X, R=lnv.pat_L.R)
    return 0.5 * (P + transpose(P, P.pat))


def minimise(lnv, L0, n_iter, reset=40, tol_ha_per_atom=None, metric=None):
    """Polak-Ribiere CG on Omega(L) with exact cubic line minimisation.

    metric: None (plain gradients), or an approximate inverse overlap X on
    its own range, with which the search directions are built from
    P = X G X (preconditioned Polak-Ribiere: beta = <G, P - P_prev> /
    <G_prev, P_prev>).
    Returns (L, history); history[k] holds Omega (eV), N_e, the predicted
    Omega after the step, alpha, beta and max |G| of step k.
    """
    L = L0.copy()
    D = Gp = Pp = None
    hist = []
    n = lnv.sys.n
    for it in range(n_iter):
        om, ne = lnv.energy(L)
        G = lnv.gradient(L)
        G = 0.5 * (G + transpose(G, G.pat))
        P = G if metric is None else metric_gradient(lnv, G, metric)
        beta = 0.0
        if D is None or it % reset == 0:
            D = -1.0 * P
        else:
            beta = max(0.0, dot(G, P - Pp) / dot(Gp, Pp))
            D = -1.0 * P + beta * D
        c1, c2, c3 = lnv.cubic(L, D, G)
        if c1 >= 0.0:                       # not a descent direction: restart
            D = -1.0 * P
            beta = 0.0
            c1, c2, c3 = lnv.cubic(L, D, G)
        a = line_minimum(c1, c2, c3)
        if a is None:
            raise FloatingPointError("no local minimum along the search direction")
        L = L + a * D
        om_next = om + c1 * a + c2 * a * a + c3 * a * a * a
        hist.append(dict(omega=om, ne=ne, omega_next=om_next, alpha=a, beta=beta,
                         gmax=float(np.abs(G.val).max()), c=(c1, c2, c3)))
        Gp, Pp = G, P
        if tol_ha_per_atom is not None and abs(om_next - om) / HA_EV / n < tol_ha_per_atom:
            break
    return L, hist


def minimise_canonical(lnv_e, lnv_n, L0, n_electrons, n_iter, reset=40, tol_ha_per_atom=None,
                       tol_ne=1e-9, max_correct=5):
    """CG on E_band = 2 Tr[K H] at fixed electron number N_e = 2 Tr[K S] (canonical LNV).

    Sec. 2.3.2: during the optimisation the electron number is constrained
    (the paper cites Hernandez, Gillan and Goringe for it).  Reading taken
    here: lnv_e is an Lnv with mu = 0 (so its Omega is E_band and its second
    value N_e), lnv_n the same with H replaced by S (its gradient is
    dN_e/dL).  Each step first restores N_e by moves L += d G_N along the
    electron-number gradient, d = (N0 - N_e) / <G_N, G_N> (Newton on the
    linearisation, at most max_correct moves, until |N_e - N0| <= tol_ne N0);
    then the energy gradient is projected on constant N_e,
    G = G_E - lam G_N with lam = <G_E, G_N> / <G_N, G_N> (the Lagrange
    multiplier, i.e. the chemical potential), Polak-Ribiere directions are
    built from G and projected again, and the step is the exact cubic line
    minimum of E_band.  Returns (L, history) with E_band, N_e, lam, alpha,
    beta per step.
    """
    L = L0.copy()
    D = Gp = None
    hist = []
    n = lnv_e.sys.n
    for it in range(n_iter):
        for c in range(max_correct + 1):
            E, N = lnv_e.energy(L)
            GN = lnv_n.gradient(L)
            GN = 0.5 * (GN + transpose(GN, GN.pat))
            gnn = dot(GN, GN)
            if abs(N - n_electrons) <= tol_ne * abs(n_electrons) or c == max_correct:
                break
            L = L + ((n_electrons - N) / gnn) * GN
        GE = lnv_e.gradient(L)
        GE = 0.5 * (GE + transpose(GE, GE.pat))
        lam = dot(GE, GN) / gnn
        G = GE - lam * GN
        beta = 0.0
        if D is None or it % reset == 0:
            D = -1.0 * G
        else:
            beta = max(0.0, dot(G, G - Gp) / dot(Gp, Gp))
            D = -1.0 * G + beta * D
        D = D - (dot(D, GN) / gnn) * GN
        c1, c2, c3 = lnv_e.cubic(L, D, GE)
        if c1 >= 0.0:
            D = -1.0 * G
            beta = 0.0
            c1, c2, c3 = lnv_e.cubic(L, D, GE)
        a = line_minimum(c1, c2, c3)
        if a is None:
            raise FloatingPointError("no local minimum along the search direction")
        L = L + a * D
        e_next = E + c1 * a + c2 * a * a + c3 * a * a * a
        hist.append(dict(energy=E, ne=N, lam=lam, energy_next=e_next, alpha=a, beta=beta))
        Gp = G
        if tol_ha_per_atom is not None and abs(e_next - E) / HA_EV / n < tol_ha_per_atom:
            break
    return L, hist
