"""Parity of the MD-step density-matrix propagation (Sec. 3.3) with the oracle.

lsq_pattern_remap bit for bit (float64 and float32, b = 4 and 13, between
two geometries of a trajectory and between ranges of one geometry);
lsq_xl_propagate within a few units in the last place (the kernel groups
the terms by history entry), with and without dissipation, in place; lsq_xl_initial_L
within 1e-12 (float32 products: 1e-5 of max |X| |S^-1|) and exactly symmetric; and a short extended-Lagrangian MD run
on 64 atoms (Hotelling S^-1, propagation, moves between geometries, initial
L, 12 float64 CG steps per MD step) against the oracle's run.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import hotelling as OH
from oracle import lnv as OL
from oracle import xl as OX
import paper_2002_07704_gb300 as lsq
from gpu_common import cuda, gpu_geometry, gpu_pattern, rel_err, si
from synth import config_seed, md_trajectory, sk_blocks

pytestmark = pytest.mark.gpu

from test_oracle_xl import read_dissipation

KAPPA, ALPHA, _C = read_dissipation()
C5 = [float(v) for v in _C]


@pytest.mark.parametrize("b,prec", [(4, lsq.F64), (4, lsq.F32), (13, lsq.F64)])
def test_remap_between_geometries_is_exact(b, prec):
    pos, cell = si(3, 0.05, config_seed(0) + 3)
    pos = pos[:-1]                                     # 215 atoms
    traj = md_trajectory(pos, cell, 6, seed=17, amp=0.3)
    ranges = [5.0, 6.6]
    g0, g1 = gpu_geometry(traj[0], cell, ranges), gpu_geometry(traj[6], cell, ranges)
    p0, p1 = gpu_pattern(g0, 0), gpu_pattern(g1, 0)
    assert p0 == oracle.neighbour_list(traj[0], cell, 5.0)
    assert not np.array_equal(p0.col, p1.col)
    dt = torch.float64 if prec == lsq.F64 else torch.float32
    rng = np.random.default_rng(b)
    X0 = oracle.Bsr(p0, b, rng.standard_normal((p0.nnzb, b, b)).astype(np.float32).astype(np.float64))
    want = OX.remap(X0, p1)
    X1 = torch.full((p1.nnzb, b, b), np.nan, dtype=dt, device="cuda")
    lsq.pattern_remap(g0, 0, g1, 0, b, cuda(X0.val, dt), X1, precision=prec)
    assert np.array_equal(X1.double().cpu().numpy(), want.val)
    # within one geometry: to a wider range and back
    pw = gpu_pattern(g0, 1)
    Xw = torch.full((pw.nnzb, b, b), np.nan, dtype=dt, device="cuda")
    lsq.pattern_remap(g0, 0, g0, 1, b, cuda(X0.val, dt), Xw, precision=prec)
    assert np.array_equal(Xw.double().cpu().numpy(), OX.remap(X0, pw).val)
    Xb = torch.zeros((p0.nnzb, b, b), dtype=dt, device="cuda")
    lsq.pattern_remap(g0, 1, g0, 0, b, Xw, Xb, precision=prec)
    assert np.array_equal(Xb.double().cpu().numpy(), X0.val)


def test_remap_rejects_different_atom_counts():
    pos, cell = si(2, 0.05, config_seed(0))
    g0, g1 = gpu_geometry(pos, cell, [5.0]), gpu_geometry(pos[:-1], cell, [5.0])
    X = torch.zeros((g0.nnzb(0), 4, 4), dtype=torch.float64, device="cuda")
    Y = torch.zeros((g1.nnzb(0), 4, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(lsq.LsqError):
        lsq.pattern_remap(g0, 0, g1, 0, 4, X, Y)


@pytest.mark.parametrize("dissipation", [False, True])
def test_propagate_matches_oracle(dissipation):
    pos, cell = si(3, 0.05, config_seed(0) + 4)
    g = gpu_geometry(pos, cell, [11.6])
    p = gpu_pattern(g, 0)
    rng = np.random.default_rng(7)
    hist = [oracle.Bsr(p, 4, rng.standard_normal((p.nnzb, 4, 4))) for _ in range(6)]
    LS = oracle.Bsr(p, 4, rng.standard_normal((p.nnzb, 4, 4)))
    alpha, c = (ALPHA, C5) if dissipation else (0.0, None)
    want = OX.propagate(hist, LS, KAPPA, alpha, c)
    # the kernel groups the terms by history entry: rounding differs from the formula taken
    # term by term by a few units in the last place of the largest term
    scale = np.abs(np.stack([h.val for h in hist] + [LS.val])).max() * (2.0 + KAPPA + 2 * 14 * ALPHA)
    tol = 8 * np.finfo(np.float64).eps * scale
    hg = [cuda(h.val) for h in hist]
    out = torch.zeros_like(hg[0])
    lsq.xl_propagate(g, 4, 0, hg, cuda(LS.val), out, KAPPA, alpha, c)
    got = out.cpu().numpy()
    assert np.abs(got - want.val).max() <= tol
    # in place over the oldest history entry: the same values
    lsq.xl_propagate(g, 4, 0, hg, cuda(LS.val), hg[5], KAPPA, alpha, c)
    assert np.array_equal(hg[5].cpu().numpy(), got)


@pytest.mark.parametrize("prec", [lsq.F64, lsq.F32])
def test_initial_L_matches_oracle(prec):
    pos, cell = si(3, 0.1, config_seed(0) + 5)
    R_L, R_X = 5.0, 4.0
    ranges = sorted({R_L, R_X, R_L + 6.6})
    g = gpu_geometry(pos, cell, ranges)
    m = OL.System(pos, cell)
    px, ps = m.pattern(R_L + 6.6), m.pattern(R_X)
    rng = np.random.default_rng(8)
    X = oracle.Bsr(px, 4, rng.standard_normal((px.nnzb, 4, 4)))
    Sinv = oracle.Bsr(ps, 4, rng.standard_normal((ps.nnzb, 4, 4)))
    Sinv = oracle.Bsr(ps, 4, 0.5 * (Sinv.val + oracle.transpose(Sinv, ps).val))
    want = OX.initial_L(m, X, Sinv, R_L)
    L = torch.full((want.pat.nnzb, 4, 4), np.nan, dtype=torch.float64, device="cuda")
    lsq.xl_initial_L(g, 4, g.range_id(R_L + 6.6), cuda(X.val), g.range_id(R_X), cuda(Sinv.val),
                     g.range_id(R_L), L, precision=prec)
    got = L.cpu().numpy()
    if prec == lsq.F64:
        assert rel_err(got, want.val) <= 1e-12
    else:
        bound, _ = oracle.matmul(oracle.Bsr(px, 4, np.abs(X.val)), oracle.Bsr(ps, 4, np.abs(Sinv.val)), want.pat)
        assert np.abs(got - want.val).max() <= 1e-5 * bound.val.max()
    assert np.array_equal(got, oracle.transpose(oracle.Bsr(want.pat, 4, got), want.pat).val)


def test_xl_md_run_matches_oracle():
    """64 atoms along a prescribed trajectory: each MD step builds the geometry, S^-1 (20
    Hotelling steps on R_L), moves the history of X to the new patterns, propagates X with
    dissipation, starts L from X S^-1 and takes 12 float64 CG steps; GPU and oracle runs
    compared step by step."""
    R_S = R_H = 6.6
    R_L, MU, K = 8.0, -2.0, 5
    pos, cell = si(2, 0.05, config_seed(0))
    traj = md_trajectory(pos, cell, 3, seed=23)
    ranges = lsq.lnv_required_ranges(R_S, R_H, R_L)
    hist_o = hist_g = None
    prev = None
    for n in range(traj.shape[0]):
        m = OL.System(traj[n], cell)
        pH = m.pattern(R_H)
        Hv, Sv = sk_blocks(traj[n], cell, pH.rows(), pH.col)
        Hb, Sb = oracle.Bsr(pH, 4, Hv), oracle.Bsr(pH, 4, Sv)
        ref = OL.Lnv(m, Sb, Hb, R_L, MU)
        g = gpu_geometry(traj[n], cell, ranges)
        rL, rX, rLS = g.range_id(R_L), g.range_id(R_L), g.range_id(R_L + R_S)
        pLS = m.pattern(R_L + R_S)
        ctx = lsq.Lnv(g, 4, R_S, R_H, R_L)
        Sg, Hg = cuda(Sb.val), cuda(Hb.val)
        # S^-1 on L's range
        Xi_o, _ = OH.hotelling(m, Sb, R_L, 20)
        Xi_g = torch.zeros((g.nnzb(rX), 4, 4), dtype=torch.float64, device="cuda")
        lsq.hotelling_inverse(g, 4, Sg, g.range_id(R_S), Xi_g, rX, rLS, 20)
        if n == 0:
            L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
            Lg = cuda(L0.val)
        else:
            g_prev, m_prev = prev
            # X(t + dt) on the previous geometry, then everything moves to this one
            Xn_o = OX.propagate(hist_o, LS_o, KAPPA, ALPHA, C5)
            hist_o = [OX.remap(h, pLS) for h in [Xn_o] + hist_o[:K]]
            Xn_g = torch.zeros_like(hist_g[0])
            lsq.xl_propagate(g_prev, 4, g_prev.range_id(R_L + R_S), hist_g, LS_g, Xn_g, KAPPA, ALPHA, C5)
            moved = []
            for h in [Xn_g] + hist_g[:K]:
                t = torch.zeros((g.nnzb(rLS), 4, 4), dtype=torch.float64, device="cuda")
                lsq.pattern_remap(g_prev, g_prev.range_id(R_L + R_S), g, rLS, 4, h, t)
                moved.append(t)
            hist_g = moved
            L0 = OX.initial_L(m, hist_o[0], Xi_o, R_L)
            Lg = torch.zeros((g.nnzb(rL), 4, 4), dtype=torch.float64, device="cuda")
            lsq.xl_initial_L(g, 4, rLS, hist_g[0], rX, Xi_g, rL, Lg)
            assert rel_err(Lg.cpu().numpy(), L0.val) <= 1e-7, n
        Lr, _ = OL.minimise(ref, L0, 12)
        rep = ctx.minimise(Lg, Sg, Hg, MU, max_iter=12)
        om_ref, _ = ref.energy(Lr)
        assert abs(rep["omega_ev"] - om_ref) <= 1e-9 * abs(om_ref), n
        assert rel_err(Lg.cpu().numpy(), Lr.val) <= 1e-7, n
        # L S on its natural range, the centre of the harmonic potential
        LS_o = OL.mm(m, Lr, Sb)
        LS_g = torch.zeros((g.nnzb(rLS), 4, 4), dtype=torch.float64, device="cuda")
        lsq.block_matmul(g, 4, Lg, rL, Sg, g.range_id(R_S), LS_g, rLS)
        if n == 0:
            hist_o = [LS_o] * (K + 1)
            hist_g = [LS_g.clone() for _ in range(K + 1)]
        prev = (g, m)


def test_adopted_schedules_skip_tuning():
    """lsq_geom_adopt_schedules: a geometry of the next MD step runs the schedules tuned in
    the previous one (far fewer launches on its first product: no tuning run), with results
    that still match the oracle."""
    pos, cell = si(3, 0.05, config_seed(0) + 6)
    traj = md_trajectory(pos, cell, 3, seed=29)
    ranges = [6.6, 10.0, 16.6]
    P1 = {R: oracle.neighbour_list(traj[3], cell, R) for R in ranges}
    rng = np.random.default_rng(9)
    A = oracle.Bsr(P1[10.0], 4, rng.standard_normal((P1[10.0].nnzb, 4, 4)))
    Bm = oracle.Bsr(P1[6.6], 4, rng.standard_normal((P1[6.6].nnzb, 4, 4)))
    ref, _ = oracle.matmul(A, Bm, P1[16.6])
    bound, _ = oracle.matmul(oracle.Bsr(P1[10.0], 4, np.abs(A.val)), oracle.Bsr(P1[6.6], 4, np.abs(Bm.val)),
                             P1[16.6])

    def first_product(g):
        C = torch.zeros((P1[16.6].nnzb, 4, 4), dtype=torch.float32, device="cuda")
        n0 = lsq.launch_count()
        lsq.block_matmul(g, 4, cuda(A.val, torch.float32), 1, cuda(Bm.val, torch.float32), 0, C, 2,
                         precision=lsq.F32)
        torch.cuda.synchronize()
        got = C.double().cpu().numpy()
        assert np.abs(got - ref.val).max() <= 1e-5 * bound.val.max()
        return lsq.launch_count() - n0

    g0 = gpu_geometry(traj[0], cell, ranges)
    Cg = torch.zeros((g0.nnzb(2), 4, 4), dtype=torch.float32, device="cuda")
    lsq.block_matmul(g0, 4, torch.ones((g0.nnzb(1), 4, 4), dtype=torch.float32, device="cuda"), 1,
                     torch.ones((g0.nnzb(0), 4, 4), dtype=torch.float32, device="cuda"), 0, Cg, 2,
                     precision=lsq.F32)                     # tunes g0's plan
    tuned = first_product(gpu_geometry(traj[3], cell, ranges))
    g1 = gpu_geometry(traj[3], cell, ranges)
    g1.adopt_schedules(g0)
    adopted = first_product(g1)
    assert adopted + 20 < tuned, (adopted, tuned)
    with pytest.raises(lsq.LsqError):
        gpu_geometry(traj[3], cell, [6.6, 10.0]).adopt_schedules(g0)
