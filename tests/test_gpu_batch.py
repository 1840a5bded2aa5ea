"""Batched minimisation of independent systems (one block-diagonal geometry).

Each system of the batch must follow the same trajectory as its own
single-system minimisation (float64: 1e-9 relative in Omega after the
same number of steps), which is itself parity-checked against the oracle;
the smallest systems are also checked against the oracle directly.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import lnv as OL
import paper_2002_07704_gb300 as lsq
from gpu_common import cuda, gpu_geometry, gpu_pattern, si
from synth import batch_system_seed, sk_blocks

pytestmark = pytest.mark.gpu

R_S = R_H = 6.6
R_L = 8.0


def _system(n, sigma, seed, b, perturb=None):
    pos, cell = si(n, sigma, seed)
    ranges = lsq.lnv_required_ranges(R_S, R_H, R_L)
    g = gpu_geometry(pos, cell, ranges)
    pH = gpu_pattern(g, 1)
    H, S = sk_blocks(pos, cell, pH.rows(), pH.col, b=b, perturb_seed=perturb)
    return pos, cell, g, pH, H, S


def _batch(specs, b):
    systems = [_system(n, sg, sd, b, pt) for (n, sg, sd, pt) in specs]
    bg = lsq.concat_geometries([s[2] for s in systems])
    H = np.concatenate([s[4] for s in systems])
    S = np.concatenate([s[5] for s in systems])
    return systems, bg, H, S


def _init_L(ctx, g, S, b):
    L = torch.zeros((g.nnzb(2), b, b), dtype=torch.float64, device="cuda")
    ctx.init_L(cuda(S), L)
    return L


@pytest.mark.parametrize("graph", [True, False])
def test_batch_matches_single_systems_float64(graph):
    lsq.build()
    specs = [(2, 0.05, batch_system_seed(0), None), (1, 0.1, batch_system_seed(1), None),
             (3, 0.15, batch_system_seed(2), None)]
    mus = [-2.0, -1.5, -2.2]
    systems, bg, H, S = _batch(specs, 4)
    ctx = lsq.Lnv(bg, 4, R_S, R_H, R_L)
    L = _init_L(ctx, bg, S, 4)
    reps = ctx.minimise_batch(L, cuda(S), cuda(H), mus, max_iter=12, graph=graph)
    for k, (pos, cell, g, pH, Hk, Sk) in enumerate(systems):
        c1 = lsq.Lnv(g, 4, R_S, R_H, R_L)
        Lk = _init_L(c1, g, Sk, 4)
        rep = c1.minimise(Lk, cuda(Sk), cuda(Hk), mus[k], max_iter=12)
        assert reps[k]["iterations"] == rep["iterations"] == 12
        assert abs(reps[k]["omega_ev"] - rep["omega_ev"]) <= 1e-9 * abs(rep["omega_ev"])
        assert abs(reps[k]["ne"] - rep["ne"]) <= 1e-9 * abs(rep["ne"])


def test_batch_block13_against_oracle():
    """13-orbital systems (three s,p copies plus a d-like orbital, perturbed H) in one batch."""
    lsq.build()
    specs = [(1, 0.1, batch_system_seed(24), batch_system_seed(24) + 7),
             (2, 0.05, batch_system_seed(25), batch_system_seed(25) + 7)]
    systems, bg, H, S = _batch(specs, 13)
    ctx = lsq.Lnv(bg, 13, R_S, R_H, R_L)
    L = _init_L(ctx, bg, S, 13)
    mus = [-2.0, -2.0]
    reps = ctx.minimise_batch(L, cuda(S), cuda(H), mus, max_iter=6)
    for k, (pos, cell, g, pH, Hk, Sk) in enumerate(systems):
        m = OL.System(pos, cell)
        pHo = m.pattern(R_H)
        assert pHo == pH
        ref = OL.Lnv(m, oracle.Bsr(pHo, 13, Sk), oracle.Bsr(pHo, 13, Hk), R_L, mus[k])
        L0 = OL.onsite_inverse_half(oracle.Bsr(pHo, 13, Sk), ref.pat_L)
        Lr, hist = OL.minimise(ref, L0, 6)
        om_ref, ne_ref = ref.energy(Lr)
        assert abs(reps[k]["omega_ev"] - om_ref) <= 1e-8 * abs(om_ref)
        assert abs(reps[k]["ne"] - ne_ref) <= 1e-8 * abs(ne_ref)


def test_batch_mixed_precision_converges_to_float64():
    lsq.build()
    specs = [(2, 0.05, batch_system_seed(3), None), (2, 0.1, batch_system_seed(4), None)]
    systems, bg, H, S = _batch(specs, 4)
    ctx = lsq.Lnv(bg, 4, R_S, R_H, R_L)
    L64 = _init_L(ctx, bg, S, 4)
    L32 = L64.clone()
    mus = [-2.0, -2.0]
    r64 = ctx.minimise_batch(L64, cuda(S), cuda(H), mus, max_iter=200, tol_ha_per_atom=1e-11)
    r32 = ctx.minimise_batch(L32, cuda(S), cuda(H), mus, max_iter=200, tol_ha_per_atom=1e-9,
                             precision=lsq.F32, refine_iter=3)
    for a, b in zip(r64, r32):
        assert a["status"] == 0
        assert abs(a["omega_ha_per_atom"] - b["omega_ha_per_atom"]) < 1e-6


def _group_inputs():
    """A batch with 4 x 4 blocks and one with 13 x 13 blocks (uneven systems in each)."""
    specs4 = [(2, 0.05, batch_system_seed(5), None), (1, 0.1, batch_system_seed(6), None),
              (3, 0.15, batch_system_seed(7), None)]
    specs13 = [(1, 0.1, batch_system_seed(26), batch_system_seed(26) + 7),
               (2, 0.05, batch_system_seed(27), batch_system_seed(27) + 7)]
    out = []
    for specs, b in ((specs4, 4), (specs13, 13)):
        systems, bg, H, S = _batch(specs, b)
        ctx = lsq.Lnv(bg, b, R_S, R_H, R_L)
        out.append((systems, bg, ctx, H, S, b))
    return out


def _group_setup(mus):
    parts = _group_inputs()
    Ls, Ss, Hs = [], [], []
    for systems, bg, ctx, H, S, b in parts:
        Ls.append(_init_L(ctx, bg, S, b))
        Ss.append(cuda(S))
        Hs.append(cuda(H))
    return parts, Ls, Ss, Hs


def test_grouped_batch_matches_separate_batches_float64():
    """One lsq_lnv_minimise_batch_group call over a 4 x 4 and a 13 x 13 batch (every product of
    a step after the first one grouped persistent launch over both) against the two batches
    minimised separately with their tuned kernels: the same trajectory to rounding (1e-9
    relative in Omega and N_e after 14 steps; both paths sum each block's terms in float64, in
    different orders)."""
    lsq.build()
    mus = [[-2.0, -1.5, -2.2], [-2.0, -1.8]]
    parts, Ls, Ss, Hs = _group_setup(mus)
    L_sep = [L.clone() for L in Ls]
    reps = lsq.minimise_batch_group([p[2] for p in parts], Ls, Ss, Hs, mus, max_iter=14)
    for c, (systems, bg, ctx, H, S, b) in enumerate(parts):
        sep = ctx.minimise_batch(L_sep[c], Ss[c], Hs[c], mus[c], max_iter=14)
        assert len(reps[c]) == len(sep) == len(systems)
        for a, r in zip(reps[c], sep):
            assert a["iterations"] == r["iterations"] == 14
            assert abs(a["omega_ev"] - r["omega_ev"]) <= 1e-9 * abs(r["omega_ev"])
            assert abs(a["ne"] - r["ne"]) <= 1e-9 * abs(r["ne"])
        scale = L_sep[c].abs().max().item()
        assert (Ls[c] - L_sep[c]).abs().max().item() <= 1e-7 * scale


def test_grouped_batch_mixed_precision_minimum():
    """Float32 products in the grouped launches, then float64 refinement: every system of both
    batches ends within 1e-6 Ha/atom (the metric's tolerance) of its float64 minimum, taken
    from the separate batch run to |dOmega| < 1e-10 Ha/atom."""
    lsq.build()
    mus = [[-2.0, -1.5, -2.2], [-2.0, -1.8]]
    parts, Ls, Ss, Hs = _group_setup(mus)
    L_sep = [L.clone() for L in Ls]
    reps = lsq.minimise_batch_group([p[2] for p in parts], Ls, Ss, Hs, mus, max_iter=300,
                                    tol_ha_per_atom=1e-9, precision=lsq.F32, refine_iter=3)
    for c, (systems, bg, ctx, H, S, b) in enumerate(parts):
        ref = ctx.minimise_batch(L_sep[c], Ss[c], Hs[c], mus[c], max_iter=400, tol_ha_per_atom=1e-10)
        for a, r in zip(reps[c], ref):
            assert r["last_domega_ha_per_atom"] < 1e-9
            assert a["iterations_fp64"] == 3
            assert abs(a["omega_ha_per_atom"] - r["omega_ha_per_atom"]) < 1e-6


def test_grouped_batch_block13_against_oracle():
    """The 13 x 13 systems of a grouped call against the oracle's own minimisation (6 steps)."""
    lsq.build()
    parts = _group_inputs()
    mus = [[-2.0, -2.0, -2.0], [-2.0, -2.0]]
    Ls = [_init_L(p[2], p[1], p[4], p[5]) for p in parts]
    reps = lsq.minimise_batch_group([p[2] for p in parts], Ls, [cuda(p[4]) for p in parts],
                                    [cuda(p[3]) for p in parts], mus, max_iter=6)
    systems = parts[1][0]
    for k, (pos, cell, g, pH, Hk, Sk) in enumerate(systems):
        m = OL.System(pos, cell)
        pHo = m.pattern(R_H)
        ref = OL.Lnv(m, oracle.Bsr(pHo, 13, Sk), oracle.Bsr(pHo, 13, Hk), R_L, mus[1][k])
        L0 = OL.onsite_inverse_half(oracle.Bsr(pHo, 13, Sk), ref.pat_L)
        Lr, _ = OL.minimise(ref, L0, 6)
        om_ref, ne_ref = ref.energy(Lr)
        assert abs(reps[1][k]["omega_ev"] - om_ref) <= 1e-8 * abs(om_ref)
        assert abs(reps[1][k]["ne"] - ne_ref) <= 1e-8 * abs(ne_ref)


def test_grouped_batch_argument_checks():
    """Distinct geometries, a product precision the grouped launch runs, matching list lengths."""
    lsq.build()
    parts = _group_inputs()
    systems, bg, ctx, H, S, b = parts[0]
    L = _init_L(ctx, bg, S, b)
    with pytest.raises(lsq.LsqError):
        lsq.minimise_batch_group([ctx, ctx], [L, L.clone()], [cuda(S)] * 2, [cuda(H)] * 2,
                                 [[-2.0] * 3] * 2, max_iter=1)
    with pytest.raises(lsq.LsqError):
        lsq.minimise_batch_group([ctx], [L], [cuda(S)], [cuda(H)], [[-2.0] * 3], max_iter=1,
                                 precision=lsq.TF32X3)
    with pytest.raises(ValueError):
        lsq.minimise_batch_group([ctx], [L], [cuda(S)], [], [[-2.0] * 3], max_iter=1)


def _metric_X(systems, b):
    """Per system the oracle's Hotelling inverse of S on S's range (30 steps); the blocks of
    all systems in the batch geometry's order."""
    from oracle import hotelling as OH
    Xs = []
    for (pos, cell, g, pH, Hk, Sk) in systems:
        m = OL.System(pos, cell)
        pHo = m.pattern(R_H)
        X, _ = OH.hotelling(m, oracle.Bsr(pHo, b, Sk), R_S, 30)
        Xs.append(X.val)
    return Xs


def test_batch_metric_matches_single_systems_float64():
    """CG in the inverse-overlap metric (lsq_lnv_set_metric on the batch context, X block
    diagonal over the systems): every system follows its own single-system metric trajectory
    (1e-9 relative in Omega and N_e after 12 steps)."""
    lsq.build()
    specs = [(2, 0.05, batch_system_seed(0), None), (1, 0.1, batch_system_seed(1), None),
             (3, 0.15, batch_system_seed(2), None)]
    mus = [-2.0, -1.5, -2.2]
    systems, bg, H, S = _batch(specs, 4)
    Xs = _metric_X(systems, 4)
    ctx = lsq.Lnv(bg, 4, R_S, R_H, R_L)
    r_x, r_xg = bg.range_id(R_S), 3          # X on S's range; X G on L + S's range
    ctx.set_metric(cuda(np.concatenate(Xs)), r_x, r_xg)
    L = _init_L(ctx, bg, S, 4)
    reps = ctx.minimise_batch(L, cuda(S), cuda(H), mus, max_iter=12)
    for k, (pos, cell, g, pH, Hk, Sk) in enumerate(systems):
        c1 = lsq.Lnv(g, 4, R_S, R_H, R_L)
        c1.set_metric(cuda(Xs[k]), g.range_id(R_S), 3)
        Lk = _init_L(c1, g, Sk, 4)
        rep = c1.minimise(Lk, cuda(Sk), cuda(Hk), mus[k], max_iter=12)
        assert reps[k]["iterations"] == rep["iterations"] == 12
        assert abs(reps[k]["omega_ev"] - rep["omega_ev"]) <= 1e-9 * abs(rep["omega_ev"])
        assert abs(reps[k]["ne"] - rep["ne"]) <= 1e-9 * abs(rep["ne"])


def test_grouped_batch_metric_matches_separate_batches_float64():
    """The grouped call with a metric on both contexts (4 x 4 and 13 x 13 batches; the metric's
    two products of each step grouped like the others) against the two batches run separately
    with the same metric: 1e-9 relative in Omega and N_e after 10 steps, L to 1e-7."""
    lsq.build()
    mus = [[-2.0, -1.5, -2.2], [-2.0, -1.8]]
    parts, Ls, Ss, Hs = _group_setup(mus)
    for systems, bg, ctx, H, S, b in parts:
        ctx.set_metric(cuda(np.concatenate(_metric_X(systems, b))), bg.range_id(R_S), 3)
    L_sep = [L.clone() for L in Ls]
    reps = lsq.minimise_batch_group([p[2] for p in parts], Ls, Ss, Hs, mus, max_iter=10)
    for c, (systems, bg, ctx, H, S, b) in enumerate(parts):
        sep = ctx.minimise_batch(L_sep[c], Ss[c], Hs[c], mus[c], max_iter=10)
        for a, r in zip(reps[c], sep):
            assert a["iterations"] == r["iterations"] == 10
            assert abs(a["omega_ev"] - r["omega_ev"]) <= 1e-9 * abs(r["omega_ev"])
            assert abs(a["ne"] - r["ne"]) <= 1e-9 * abs(r["ne"])
        scale = L_sep[c].abs().max().item()
        assert (Ls[c] - L_sep[c]).abs().max().item() <= 1e-7 * scale
    # a metric on one context of a grouped call but not the other is refused
    parts[1][2].set_metric(None, parts[1][1].range_id(R_S), 3)
    with pytest.raises(lsq.LsqError):
        lsq.minimise_batch_group([p[2] for p in parts], [L.clone() for L in Ls], Ss, Hs, mus, max_iter=1)


def _canonical_specs():
    specs = [(2, 0.05, batch_system_seed(0), None), (1, 0.1, batch_system_seed(1), None),
             (3, 0.15, batch_system_seed(2), None)]
    systems, bg, H, S = _batch(specs, 4)
    # 174 electrons for 64 atoms (between the grand-canonical start's count and the minimum's)
    n0 = [174.0 / 64.0 * s[0].shape[0] for s in systems]
    return systems, bg, H, S, n0


@pytest.mark.parametrize("prec", [lsq.F64, lsq.F32])
def test_batch_canonical_matches_single_systems(prec):
    """lsq_lnv_minimise_batch_canonical: every system follows its own single-system canonical
    trajectory (lsq_lnv_minimise_canonical, itself checked against the oracle): float64 to 1e-9
    relative in E_band and N_e and 1e-7 in lambda after 12 steps; float32 products within 1e-4
    of the float64 batch in E_band with N_e held to 1e-5, the single-system float32 bars."""
    lsq.build()
    systems, bg, H, S, n0 = _canonical_specs()
    ctx = lsq.Lnv(bg, 4, R_S, R_H, R_L)
    L = _init_L(ctx, bg, S, 4)
    reps, lams = ctx.minimise_batch_canonical(L, cuda(S), cuda(H), n0, max_iter=12, precision=prec)
    if prec == lsq.F32:
        L64 = _init_L(ctx, bg, S, 4)
        r64, _ = ctx.minimise_batch_canonical(L64, cuda(S), cuda(H), n0, max_iter=12)
        for k, (a, r) in enumerate(zip(reps, r64)):
            assert a["iterations"] == 12
            assert abs(a["ne"] - n0[k]) <= 1e-5 * n0[k]
            assert abs(a["omega_ev"] - r["omega_ev"]) <= 1e-4 * abs(r["omega_ev"])
        return
    for k, (pos, cell, g, pH, Hk, Sk) in enumerate(systems):
        c1 = lsq.Lnv(g, 4, R_S, R_H, R_L)
        Lk = _init_L(c1, g, Sk, 4)
        rep, lam = c1.minimise_canonical(Lk, cuda(Sk), cuda(Hk), n0[k], max_iter=12)
        assert reps[k]["iterations"] == rep["iterations"] == 12
        assert abs(reps[k]["omega_ev"] - rep["omega_ev"]) <= 1e-9 * abs(rep["omega_ev"])
        assert abs(reps[k]["ne"] - rep["ne"]) <= 1e-9 * abs(rep["ne"])
        assert abs(lams[k] - lam) <= 1e-7 * abs(lam)


def test_batch_canonical_argument_checks():
    """One electron count per system, each positive; no metric."""
    lsq.build()
    systems, bg, H, S, n0 = _canonical_specs()
    ctx = lsq.Lnv(bg, 4, R_S, R_H, R_L)
    L = _init_L(ctx, bg, S, 4)
    with pytest.raises(lsq.LsqError):
        ctx.minimise_batch_canonical(L, cuda(S), cuda(H), n0[:2], max_iter=1)
    with pytest.raises(lsq.LsqError):
        ctx.minimise_batch_canonical(L, cuda(S), cuda(H), [n0[0], -1.0, n0[2]], max_iter=1)
    ctx.set_metric(cuda(np.concatenate(_metric_X(systems, 4))), bg.range_id(R_S), 3)
    with pytest.raises(lsq.LsqError):
        ctx.minimise_batch_canonical(L, cuda(S), cuda(H), n0, max_iter=1)
