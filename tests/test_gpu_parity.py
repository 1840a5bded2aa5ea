"""Parity of the CUDA path against the CPU oracle on the same seeded inputs.

Tolerances: range patterns bit-exact; float64 products within 1e-12 of
the oracle (max-norm, relative to the largest reference element); float32
products within 1e-5 of max |A|.|B| (inputs rounded to 24 bits and sums
of up to ~10^4 terms); LNV energy, electron number and gradient in float64
within 1e-12 relative.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import lnv as OL
import paper_2002_07704_gb300 as lsq
from gpu_common import cuda, gpu_geometry, gpu_pattern, rel_err, si, si_hs
from synth import config_seed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lsq.build()
    lsq.load()


@pytest.mark.parametrize("n,sigma,ranges", [
    (1, 0.05, [2.0, 6.6, 10.0, 30.0]),
    (2, 0.05, [6.6, 8.0, 14.6, 22.6, 21.2]),
    (3, 0.15, [6.6, 10.0, 16.6, 26.6, 23.2]),
    (8, 0.05, [6.6, 10.0, 16.6, 26.6, 23.2]),
])
def test_patterns_bit_exact(n, sigma, ranges):
    pos, cell = si(n, sigma, config_seed(1) + n)
    g = gpu_geometry(pos, cell, ranges)
    for r, R in enumerate(ranges):
        assert gpu_pattern(g, r) == oracle.neighbour_list(pos, cell, R, "cell")


def test_pattern_empty_and_single_atom():
    g = gpu_geometry(np.zeros((0, 3)), [10.0, 10.0, 10.0], [3.0])
    assert g.nnzb(0) == 0
    g1 = gpu_geometry(np.array([[1.0, 2.0, 3.0]]), [10.0, 10.0, 10.0], [3.0])
    p = gpu_pattern(g1, 0)
    assert p.nnzb == 1 and p.col[0] == 0


def _rand(pat, b, rng):
    return rng.standard_normal((pat.nnzb, b, b))


@pytest.mark.parametrize("n,b,ra,rb,rc,ta,tb", [
    (2, 4, 10.0, 6.6, 16.6, 0, 0),    # L.S at its natural range (row form)
    (2, 4, 16.6, 10.0, 26.6, 0, 0),   # LS.L
    (2, 4, 26.6, 16.6, 6.6, 0, 1),    # LSL.(LS)^T truncated to R_H (inner form)
    (2, 4, 23.2, 16.6, 10.0, 1, 0),   # Q^T.LS truncated to R_L
    (3, 4, 6.6, 10.0, 8.0, 1, 1),     # both transposed, truncated
    (3, 4, 10.0, 6.6, 16.6, 0, 0),
    (1, 13, 3.0, 2.5, 4.0, 0, 0),     # 13 x 13 blocks (generic kernel)
    (1, 13, 3.0, 2.5, 5.5, 1, 1),
    (2, 7, 4.0, 4.0, 6.0, 0, 1),      # ragged block size
    (1, 13, 4.0, 3.0, 5.5, 0, 1),     # 13 x 13, one operand transposed each way
    (1, 13, 4.0, 3.0, 3.0, 1, 0),
    (1, 9, 3.0, 3.0, 5.0, 0, 1),      # smallest and largest 16 x 16-frame sizes
    (1, 16, 3.0, 2.5, 4.0, 1, 0),
])
@pytest.mark.parametrize("prec", [lsq.F64, lsq.F32])
def test_block_matmul_matches_oracle(n, b, ra, rb, rc, ta, tb, prec):
    pos, cell = si(n, 0.1, config_seed(0) + 31 * n + b)
    ranges = sorted(set([ra, rb, rc]))
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(100 + b)
    A = oracle.Bsr(P[ra], b, _rand(P[ra], b, rng))
    B = oracle.Bsr(P[rb], b, _rand(P[rb], b, rng))
    C0 = oracle.Bsr(P[rc], b, _rand(P[rc], b, rng))
    opA = oracle.transpose(A, P[ra]) if ta else A
    opB = oracle.transpose(B, P[rb]) if tb else B
    ref, triples = oracle.matmul(opA, opB, P[rc])
    alpha, beta = 0.75, -0.5
    ref_val = alpha * ref.val + beta * C0.val
    dt = torch.float64 if prec == lsq.F64 else torch.float32
    Cg = cuda(C0.val, dt)
    t = lsq.block_matmul(g, b, cuda(A.val, dt), g.range_id(ra), cuda(B.val, dt), g.range_id(rb),
                         Cg, g.range_id(rc), precision=prec, trans_a=ta, trans_b=tb,
                         alpha=alpha, beta=beta)
    torch.cuda.synchronize()
    assert t == triples
    got = Cg.double().cpu().numpy()
    if prec == lsq.F64:
        assert rel_err(got, ref_val) <= 1e-12
    else:
        absA = oracle.Bsr(P[ra], b, np.abs(opA.val))
        absB = oracle.Bsr(P[rb], b, np.abs(opB.val))
        bound, _ = oracle.matmul(absA, absB, P[rc])
        scale = abs(alpha) * bound.val.max() + abs(beta) * np.abs(C0.val).max()
        assert np.abs(got - ref_val).max() <= 1e-5 * scale


@pytest.mark.parametrize("b", [4, 13])
@pytest.mark.parametrize("prec", [lsq.F64, lsq.F32])
def test_block_matmul_triangles(b, prec):
    """lsq_block_matmul_tri: the computed triangle equals the oracle's product there; with
    triangle 1 the other blocks are the transposes of the computed ones."""
    n = 2 if b == 4 else 1
    pos, cell = si(n, 0.1, config_seed(0) + 91 + b)
    ra, rb, rc = (16.6, 10.0, 10.0) if b == 4 else (4.0, 3.0, 4.0)
    ranges = sorted(set([ra, rb, rc]))
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(500 + b)
    A = oracle.Bsr(P[ra], b, _rand(P[ra], b, rng))
    B = oracle.Bsr(P[rb], b, _rand(P[rb], b, rng))
    ref, _ = oracle.matmul(A, B, P[rc])
    pc = P[rc]
    rows = np.repeat(np.arange(pc.n), np.diff(pc.ptr))
    upper = pc.col >= rows
    lower = pc.col <= rows
    dt = torch.float64 if prec == lsq.F64 else torch.float32
    absA, absB = oracle.Bsr(P[ra], b, np.abs(A.val)), oracle.Bsr(P[rb], b, np.abs(B.val))
    bound = oracle.matmul(absA, absB, pc)[0].val.max()
    tol = 1e-12 * np.abs(ref.val).max() if prec == lsq.F64 else 1e-5 * bound
    for tri, mask in ((2, upper), (3, lower), (1, upper)):
        C = torch.zeros((pc.nnzb, b, b), dtype=dt, device="cuda")
        lsq.block_matmul(g, b, cuda(A.val, dt), g.range_id(ra), cuda(B.val, dt), g.range_id(rb), C,
                         g.range_id(rc), precision=prec, triangle=tri)
        got = C.double().cpu().numpy()
        assert np.abs(got[mask] - ref.val[mask]).max() <= tol
        if tri == 1:
            # lower blocks hold the transposes of the upper ones, bit for bit
            tpos = {(int(i), int(j)): k for k, (i, j) in enumerate(zip(rows, pc.col))}
            for k in np.nonzero(~upper)[0]:
                kt = tpos[(int(pc.col[k]), int(rows[k]))]
                assert np.array_equal(got[k], got[kt].T)
    with pytest.raises(lsq.LsqError):
        lsq.block_matmul(g, b, cuda(A.val, dt), g.range_id(ra), cuda(B.val, dt), g.range_id(rb), C,
                         g.range_id(rc), precision=prec, triangle=1, beta=0.5)


def _at_offset(x, off):
    """A copy of x whose data starts `off` elements into a fresh allocation."""
    buf = torch.empty(x.numel() + off, dtype=x.dtype, device=x.device)
    v = buf[off:].view(x.shape)
    v.copy_(x)
    return v


@pytest.mark.parametrize("prec,off", [(lsq.F64, 1), (lsq.F64, 2), (lsq.F32, 1), (lsq.F32, 2),
                                      (lsq.F32, 4), (lsq.F32, 8)])
def test_block_matmul_any_alignment(prec, off):
    """4 x 4 blocks at 4-, 8-, 16- and 32-byte offsets: the same product as aligned arrays.

    A first aligned call lets the autotuner pick any schedule (possibly one with
    32-byte loads); the offset call must then take a schedule its pointers allow.
    """
    pos, cell = si(2, 0.1, config_seed(0) + 77)
    ranges = [10.0, 16.6, 23.2]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(300 + off)
    A = oracle.Bsr(P[16.6], 4, _rand(P[16.6], 4, rng))
    B = oracle.Bsr(P[10.0], 4, _rand(P[10.0], 4, rng))
    ref, _ = oracle.matmul(A, B, P[23.2])
    dt = torch.float64 if prec == lsq.F64 else torch.float32
    Ag, Bg = cuda(A.val, dt), cuda(B.val, dt)
    ra, rb, rc = g.range_id(16.6), g.range_id(10.0), g.range_id(23.2)
    C1 = torch.zeros((P[23.2].nnzb, 4, 4), dtype=dt, device="cuda")
    lsq.block_matmul(g, 4, Ag, ra, Bg, rb, C1, rc, precision=prec, trans_b=True)
    ref_t, _ = oracle.matmul(A, oracle.transpose(B, P[10.0]), P[23.2])
    C2 = _at_offset(torch.zeros((P[23.2].nnzb, 4, 4), dtype=dt, device="cuda"), off)
    lsq.block_matmul(g, 4, _at_offset(Ag, off), ra, _at_offset(Bg, off), rb, C2, rc,
                     precision=prec, trans_b=True)
    C3 = _at_offset(torch.zeros((P[23.2].nnzb, 4, 4), dtype=dt, device="cuda"), off)
    lsq.block_matmul(g, 4, _at_offset(Ag, off), ra, _at_offset(Bg, off), rb, C3, rc, precision=prec)
    torch.cuda.synchronize()
    absA = oracle.Bsr(P[16.6], 4, np.abs(A.val))
    absB = oracle.Bsr(P[10.0], 4, np.abs(B.val))
    bound = max(oracle.matmul(absA, absB, P[23.2])[0].val.max(),
                oracle.matmul(absA, oracle.transpose(absB, P[10.0]), P[23.2])[0].val.max())
    tol = 1e-12 * np.abs(ref.val).max() if prec == lsq.F64 else 1e-5 * bound
    for got, want in ((C1, ref_t), (C2, ref_t), (C3, ref)):
        assert np.abs(got.double().cpu().numpy() - want.val).max() <= tol


def test_block_matmul_full_size_sampled_rows():
    """4096-atom Si, LS.L (natural range 26.6 A) in float64: sampled rows against the oracle."""
    pos, cell = si(8, 0.05, config_seed(1))
    ranges = [6.6, 10.0, 16.6, 26.6]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(7)
    A = oracle.Bsr(P[16.6], 4, _rand(P[16.6], 4, rng))
    B = oracle.Bsr(P[10.0], 4, _rand(P[10.0], 4, rng))
    Cg = torch.zeros((P[26.6].nnzb, 4, 4), dtype=torch.float64, device="cuda")
    t = lsq.block_matmul(g, 4, cuda(A.val), 2, cuda(B.val), 1, Cg, 3)
    rows = np.array([0, 1, 777, 2048, 4095])
    ref, _ = oracle.matmul(A, B, P[26.6], rows=rows)
    got = Cg.cpu().numpy()
    for i in rows:
        s = slice(P[26.6].ptr[i], P[26.6].ptr[i + 1])
        assert rel_err(got[s], ref.val[s]) <= 1e-12
    assert t > 0


@pytest.mark.parametrize("shape", ["sl_qt_upper", "p_d_upper", "l_s"])
def test_block_matmul_full_size_float32_sampled_rows(shape):
    """4096-atom Si, float32, the three product shapes whose schedules the autotuner picks for
    the benchmark's mixed step, in the same launch configuration (same geometry, ranges and
    triangle, first call tuned): 32 sampled rows of C against the oracle, within 1e-5 of
    max |A|.|B| over those rows.  At this size rows of C hold ~200 (10 A) to ~2600 (23.2 A)
    blocks and item lists ~900 entries, so the 16-bit offsets and the split lists take their
    full-size paths.
      sl_qt_upper: SL (16.6 A) . Q^T (Q on 23.2 A), upper triangle of 10 A (trans_b);
      p_d_upper:   P (16.6 A) . D^T (D on 10 A), upper triangle of 23.2 A;
      l_s:         L (10 A) . S^T (S on 6.6 A), every block of 16.6 A."""
    ra, rb, rc, tri = {"sl_qt_upper": (16.6, 23.2, 10.0, 2), "p_d_upper": (16.6, 10.0, 23.2, 2),
                       "l_s": (10.0, 6.6, 16.6, 0)}[shape]
    pos, cell = si(8, 0.05, config_seed(1))
    ranges = [6.6, 10.0, 16.6, 23.2]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(17)
    A = oracle.Bsr(P[ra], 4, _rand(P[ra], 4, rng).astype(np.float32).astype(np.float64))
    B = oracle.Bsr(P[rb], 4, _rand(P[rb], 4, rng).astype(np.float32).astype(np.float64))
    Cg = torch.zeros((P[rc].nnzb, 4, 4), dtype=torch.float32, device="cuda")
    args = (g, 4, cuda(A.val, torch.float32), g.range_id(ra), cuda(B.val, torch.float32), g.range_id(rb),
            Cg, g.range_id(rc))
    lsq.block_matmul(*args, precision=lsq.F32, trans_b=True, triangle=tri)   # tunes the schedule
    Cg.zero_()
    lsq.block_matmul(*args, precision=lsq.F32, trans_b=True, triangle=tri)
    torch.cuda.synchronize()
    rows = np.sort(rng.choice(4096, size=32, replace=False))
    Bt = oracle.transpose(B, P[rb])
    ref, _ = oracle.matmul(A, Bt, P[rc], rows=rows)
    bnd, _ = oracle.matmul(oracle.Bsr(P[ra], 4, np.abs(A.val)), oracle.Bsr(P[rb], 4, np.abs(Bt.val)),
                           P[rc], rows=rows)
    pc = P[rc]
    prow = np.repeat(np.arange(pc.n), np.diff(pc.ptr))
    sel = np.isin(prow, rows) & ((pc.col >= prow) if tri == 2 else True)
    got = Cg.double().cpu().numpy()
    assert np.abs(got[sel] - ref.val[sel]).max() <= 1e-5 * bnd.val[sel].max()


@pytest.mark.parametrize("prec", [lsq.F64, lsq.F32, lsq.TF32X3])
def test_block_matmul_64000_atoms_sampled_rows(prec):
    """64,000-atom Si (20 x 20 x 20 cells), beyond the 57,856 atoms a 32-bit shared-memory
    atom map allowed the plan builder: L-like (4 A) . S-like (2.6 A) on the natural 6.6 A range,
    32 sampled rows against the oracle (float64 within 1e-12 of the largest reference element;
    float32 and split-TF32 within 1e-5 of max |A|.|B| over those rows)."""
    pos, cell = si(20, 0.05, config_seed(1) + 20)
    ranges = [2.6, 4.0, 6.6]
    g = gpu_geometry(pos, cell, ranges)
    assert g.n_atoms == 64000
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(21)
    f32 = prec != lsq.F64
    A = _rand(P[4.0], 4, rng)
    B = _rand(P[2.6], 4, rng)
    if f32:
        A, B = A.astype(np.float32).astype(np.float64), B.astype(np.float32).astype(np.float64)
    A, B = oracle.Bsr(P[4.0], 4, A), oracle.Bsr(P[2.6], 4, B)
    dt = torch.float32 if f32 else torch.float64
    Cg = torch.zeros((P[6.6].nnzb, 4, 4), dtype=dt, device="cuda")
    args = (g, 4, cuda(A.val, dt), 1, cuda(B.val, dt), 0, Cg, 2)
    lsq.block_matmul(*args, precision=prec)     # first call: plans (and the kernel choice)
    Cg.zero_()
    lsq.block_matmul(*args, precision=prec)
    g.device_status()
    rows = np.sort(rng.choice(64000, size=32, replace=False))
    rows[0], rows[-1] = 0, 63999
    ref, _ = oracle.matmul(A, B, P[6.6], rows=rows)
    pc = P[6.6]
    prow = np.repeat(np.arange(pc.n), np.diff(pc.ptr))
    sel = np.isin(prow, rows)
    got = Cg.double().cpu().numpy()
    if not f32:
        assert np.abs(got[sel] - ref.val[sel]).max() <= 1e-12 * np.abs(ref.val[sel]).max()
    else:
        bnd, _ = oracle.matmul(oracle.Bsr(P[4.0], 4, np.abs(A.val)), oracle.Bsr(P[2.6], 4, np.abs(B.val)),
                               P[6.6], rows=rows)
        assert np.abs(got[sel] - ref.val[sel]).max() <= 1e-5 * bnd.val[sel].max()


def test_trace_matches_oracle():
    pos, cell = si(2, 0.1, 5)
    g = gpu_geometry(pos, cell, [6.6, 10.0])
    P = {R: oracle.neighbour_list(pos, cell, R) for R in (6.6, 10.0)}
    rng = np.random.default_rng(9)
    X = oracle.Bsr(P[6.6], 4, _rand(P[6.6], 4, rng))
    Y = oracle.Bsr(P[10.0], 4, _rand(P[10.0], 4, rng))
    got = lsq.trace(g, 4, cuda(X.val), 0, cuda(Y.val), 1)
    ref = oracle.trace(X, Y)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref))


# ---- LNV ---------------------------------------------------------------------
R_S = R_H = 6.6
MU = -2.0


def _lnv_setup(n, sigma, seed, R_L, b=4):
    pos, cell = si(n, sigma, seed)
    ranges = lsq.lnv_required_ranges(R_S, R_H, R_L)
    g = gpu_geometry(pos, cell, ranges)
    m = OL.System(pos, cell)
    pH = m.pattern(R_H)
    assert gpu_pattern(g, 1) == pH
    H, S = si_hs(pos, cell, pH, b)
    Hb, Sb = oracle.Bsr(pH, b, H), oracle.Bsr(pH, b, S)
    ref = OL.Lnv(m, Sb, Hb, R_L, MU)
    ctx = lsq.Lnv(g, b, R_S, R_H, R_L)
    return g, ctx, ref, Hb, Sb


def test_lnv_init_energy_gradient_float64():
    g, ctx, ref, Hb, Sb = _lnv_setup(2, 0.05, config_seed(0), 8.0)
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    L1, _ = OL.minimise(ref, L0, 3)
    Lg = torch.zeros((ref.pat_L.nnzb, 4, 4), dtype=torch.float64, device="cuda")
    ctx.init_L(cuda(Sb.val), Lg)
    torch.cuda.synchronize()
    assert rel_err(Lg.cpu().numpy(), L0.val) <= 1e-13
    G = torch.zeros_like(Lg)
    om, ne = ctx.energy_gradient(cuda(L1.val), cuda(Sb.val), cuda(Hb.val), MU, G=G)
    om_ref, ne_ref = ref.energy(L1)
    assert abs(om - om_ref) <= 1e-12 * abs(om_ref)
    assert abs(ne - ne_ref) <= 1e-12 * abs(ne_ref)
    Gr = ref.gradient(L1)
    Gr = 0.5 * (Gr + oracle.transpose(Gr, Gr.pat))
    assert rel_err(G.cpu().numpy(), Gr.val) <= 1e-12
    Gh = G.cpu().numpy()
    assert np.array_equal(Gh, oracle.transpose(oracle.Bsr(ref.pat_L, 4, Gh), ref.pat_L).val)


def test_lnv_energy_float32_within_tolerance():
    g, ctx, ref, Hb, Sb = _lnv_setup(2, 0.05, config_seed(0), 8.0)
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    L1, _ = OL.minimise(ref, L0, 3)
    G = torch.zeros((ref.pat_L.nnzb, 4, 4), dtype=torch.float64, device="cuda")
    om, ne = ctx.energy_gradient(cuda(L1.val), cuda(Sb.val), cuda(Hb.val), MU, G=G,
                                 precision=lsq.F32)
    om_ref, _ = ref.energy(L1)
    assert abs(om - om_ref) / lsq.HARTREE_EV / 64 < 1e-6
    Gr = ref.gradient(L1)
    assert rel_err(G.cpu().numpy(), 0.5 * (Gr.val + oracle.transpose(Gr, Gr.pat).val)) < 1e-5


def test_lnv_minimise_float64_matches_oracle_trajectory():
    """The 64-atom configuration: 20 CG steps, L range 8 A, mu = -2 eV."""
    g, ctx, ref, Hb, Sb = _lnv_setup(2, 0.05, config_seed(0), 8.0)
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    Lr, hist = OL.minimise(ref, L0, 20)
    Lg = cuda(L0.val)
    rep = ctx.minimise(Lg, cuda(Sb.val), cuda(Hb.val), MU, max_iter=20)
    om_ref, ne_ref = ref.energy(Lr)
    assert rep["iterations"] == 20
    assert abs(rep["omega_ev"] - om_ref) <= 1e-9 * abs(om_ref)
    assert abs(rep["ne"] - ne_ref) <= 1e-9 * abs(ne_ref)
    assert rel_err(Lg.cpu().numpy(), Lr.val) <= 1e-7


def test_lnv_mixed_precision_reaches_float64_minimum():
    """Mixed path (float32 products, float64 traces and refinement) vs the oracle's minimum."""
    g, ctx, ref, Hb, Sb = _lnv_setup(2, 0.05, config_seed(0), 8.0)
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    Lr, hist = OL.minimise(ref, L0, 150, tol_ha_per_atom=1e-10)
    om_ref = ref.energy(Lr)[0]
    Lg = cuda(L0.val)
    rep = ctx.minimise(Lg, cuda(Sb.val), cuda(Hb.val), MU, max_iter=150, tol_ha_per_atom=1e-9,
                       precision=lsq.F32, refine_iter=3)
    assert abs(rep["omega_ev"] - om_ref) / lsq.HARTREE_EV / 64 < 1e-6
    # the returned Omega is a float64 evaluation of the returned L
    om_chk, _ = ref.energy(oracle.Bsr(ref.pat_L, 4, Lg.cpu().numpy()))
    assert abs(rep["omega_ev"] - om_chk) <= 1e-10 * abs(om_chk)


def test_lnv_tf32x3_energy_gradient_and_minimum():
    """The mixed path with LSQ_TF32X3 (per product the faster of the FP32 FMA schedules and the
    split-TF32 tensor-core kernel, timed on first use): Omega within 1e-6 Ha/atom and G within
    2e-5 of max |G| of the oracle at an intermediate L (216 atoms; measured 1.4e-7 Ha/atom and
    9.6e-6 with the tensor-core products, 4e-9 and 8.5e-6 with the FP32 FMA ones; which kernel
    each product takes depends on its timing), and the minimum (float64 refinement and final
    Omega) within 1e-6 Ha/atom of the oracle's."""
    g, ctx, ref, Hb, Sb = _lnv_setup(3, 0.05, config_seed(0), 8.0)
    n = g.n_atoms
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    L1, _ = OL.minimise(ref, L0, 3)
    G = torch.zeros((ref.pat_L.nnzb, 4, 4), dtype=torch.float64, device="cuda")
    for _ in range(2):   # the first call times both kernels for every product
        om, _ = ctx.energy_gradient(cuda(L1.val), cuda(Sb.val), cuda(Hb.val), MU, G=G, precision=lsq.TF32X3)
    g.device_status()
    om_ref, _ = ref.energy(L1)
    assert abs(om - om_ref) / lsq.HARTREE_EV / n < 1e-6
    Gr = ref.gradient(L1)
    assert rel_err(G.cpu().numpy(), 0.5 * (Gr.val + oracle.transpose(Gr, Gr.pat).val)) < 2e-5
    Lr, _ = OL.minimise(ref, L0, 200, tol_ha_per_atom=1e-10)
    om_min = ref.energy(Lr)[0]
    Lg = cuda(L0.val)
    rep = ctx.minimise(Lg, cuda(Sb.val), cuda(Hb.val), MU, max_iter=200, tol_ha_per_atom=1e-9,
                       precision=lsq.TF32X3, refine_iter=3)
    g.device_status()
    assert abs(rep["omega_ev"] - om_min) / lsq.HARTREE_EV / n < 1e-6


def test_lnv_metric_cg_matches_oracle_trajectory():
    """CG in the inverse-overlap metric (lsq_lnv_set_metric): 15 steps against the oracle;
    the identity metric reproduces plain CG; the batched minimiser follows it too."""
    from oracle import hotelling as OH
    g, ctx, ref, Hb, Sb = _lnv_setup(2, 0.05, config_seed(0), 8.0)
    X, _ = OH.hotelling(ref.sys, Sb, R_S, 30)
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    Lr, _ = OL.minimise(ref, L0, 15, metric=X)
    r_x, r_xg = g.range_id(R_S), 3          # X on S's range; X G on L + S's range
    ctx.set_metric(cuda(X.val), r_x, r_xg)
    Lg = cuda(L0.val)
    rep = ctx.minimise(Lg, cuda(Sb.val), cuda(Hb.val), MU, max_iter=15)
    om_ref, _ = ref.energy(Lr)
    assert rep["iterations"] == 15
    assert abs(rep["omega_ev"] - om_ref) <= 1e-9 * abs(om_ref)
    assert rel_err(Lg.cpu().numpy(), Lr.val) <= 1e-7
    # the batched minimiser (one system) takes the metric too and follows the same trajectory
    Lb = cuda(L0.val)
    repb = ctx.minimise_batch(Lb, cuda(Sb.val), cuda(Hb.val), [MU], max_iter=15)
    assert repb[0]["iterations"] == 15
    assert abs(repb[0]["omega_ev"] - om_ref) <= 1e-9 * abs(om_ref)
    assert rel_err(Lb.cpu().numpy(), Lr.val) <= 1e-7
    # identity blocks as the metric: the plain trajectory
    pX = ref.sys.pattern(R_S)
    eye = np.zeros((pX.nnzb, 4, 4))
    eye[pX.rows() == pX.col] = np.eye(4)
    ctx.set_metric(cuda(eye), r_x, r_xg)
    L1 = cuda(L0.val)
    rep1 = ctx.minimise(L1, cuda(Sb.val), cuda(Hb.val), MU, max_iter=6)
    ctx.set_metric(None, r_x, r_xg)
    L2 = cuda(L0.val)
    rep2 = ctx.minimise(L2, cuda(Sb.val), cuda(Hb.val), MU, max_iter=6)
    assert abs(rep1["omega_ev"] - rep2["omega_ev"]) <= 1e-12 * abs(rep2["omega_ev"])
    assert rel_err(L1.cpu().numpy(), L2.cpu().numpy()) <= 1e-12


@pytest.mark.parametrize("prec,n_iter", [(lsq.F64, 20), (lsq.F32, 12)])
def test_lnv_purified_start_matches_oracle(prec, n_iter):
    """lsq_lnv_init_purify: the McWeeny-purified start from H against the oracle (64 atoms,
    L range 8 A, X from 30 Hotelling steps on S's range)."""
    from oracle import hotelling as OH
    from oracle import purify as OP
    g, ctx, ref, Hb, Sb = _lnv_setup(2, 0.05, config_seed(0), 8.0)
    X, _ = OH.hotelling(ref.sys, Sb, R_S, 30)
    Kr, hr, _ = OP.purify(ref.sys, Sb, Hb, X, MU, 8.0, n_iter)
    L = torch.zeros((g.nnzb(2), 4, 4), dtype=torch.float64, device="cuda")
    dk = ctx.init_purify(cuda(Sb.val), cuda(Hb.val), MU, cuda(X.val), g.range_id(R_S), 3, L, n_iter,
                         precision=prec)
    tol = 1e-10 if prec == lsq.F64 else 1e-4
    assert rel_err(L.cpu().numpy(), Kr.val) <= tol
    if prec == lsq.F64:
        for a, r in zip(dk, hr):
            assert abs(a - r) <= 1e-8 * r + 1e-12
    # the purified start is a better start: lower Omega than the on-site one
    L0 = cuda(OL.onsite_inverse_half(Sb, ref.pat_L).val)
    om_p, _ = ctx.energy_gradient(L, cuda(Sb.val), cuda(Hb.val), MU)
    om_0, _ = ctx.energy_gradient(L0, cuda(Sb.val), cuda(Hb.val), MU)
    assert om_p < om_0


@pytest.mark.parametrize("prec", [lsq.F64, lsq.F32])
def test_lnv_canonical_matches_oracle_trajectory(prec):
    """Canonical LNV (lsq_lnv_minimise_canonical): 12 steps at N0 = 174 against the oracle."""
    g, ctx, ref, Hb, Sb = _lnv_setup(2, 0.05, config_seed(0), 8.0)
    pH = Hb.pat
    le = OL.Lnv(ref.sys, Sb, Hb, 8.0, 0.0)
    ln = OL.Lnv(ref.sys, Sb, oracle.restrict(Sb, pH), 8.0, 0.0)
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    n0 = 174.0
    Lr, hr = OL.minimise_canonical(le, ln, L0, n0, 12)
    Lg = cuda(L0.val)
    rep, lam = ctx.minimise_canonical(Lg, cuda(Sb.val), cuda(Hb.val), n0, max_iter=12, precision=prec)
    assert rep["iterations"] == 12
    if prec == lsq.F64:
        assert abs(rep["omega_ev"] - hr[-1]["energy"]) <= 1e-9 * abs(hr[-1]["energy"])
        assert abs(lam - hr[-1]["lam"]) <= 1e-7 * max(1.0, abs(hr[-1]["lam"]))
        assert rel_err(Lg.cpu().numpy(), Lr.val) <= 1e-7
        assert abs(rep["ne"] - n0) <= 1e-8 * n0
    else:
        # float32 products: the trajectory stays within float32 accuracy of the oracle's
        E, N = le.energy(oracle.Bsr(ref.pat_L, 4, Lg.cpu().numpy()))
        Er, Nr = le.energy(Lr)
        assert abs(E - Er) <= 1e-4 * abs(Er)
        assert abs(N - Nr) <= 1e-4 * n0          # the last step's drift, before its correction
        assert abs(rep["ne"] - n0) <= 1e-5 * n0  # N_e held at the start of the last step


@pytest.mark.parametrize("setting", ["all=1", "3:2:5:1=1,all=0"])
def test_lnv_tf32x3_all_products_on_tensor_cores(monkeypatch, setting):
    """Kernel choices fixed by LSQ_TC_CHOICE instead of the timing.  "all=1": every 4 x 4
    product of the mixed step on the tensor cores, which also takes the step's fused
    tensor-core forms (the split copy of Q + Q^T formed from Q, SL's split shared by the two
    gradient products, QD^T read through its transpose map).  "3:2:5:1=1,all=0": only
    F = P.D on the tensor cores, every other product on the FMA kernels.  Omega within 1e-6 Ha/atom and G within 2e-5 of max abs G of the oracle at an
    intermediate L (216 atoms), and the minimum (float64 refinement and final Omega) within
    1e-6 Ha/atom of the oracle's."""
    monkeypatch.setenv("LSQ_TC_CHOICE", setting)
    g, ctx, ref, Hb, Sb = _lnv_setup(3, 0.05, config_seed(0), 8.0)
    n = g.n_atoms
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    L1, _ = OL.minimise(ref, L0, 3)
    G = torch.zeros((ref.pat_L.nnzb, 4, 4), dtype=torch.float64, device="cuda")
    for _ in range(2):
        om, _ = ctx.energy_gradient(cuda(L1.val), cuda(Sb.val), cuda(Hb.val), MU, G=G, precision=lsq.TF32X3)
    g.device_status()
    for ra, rb, rc, tri in ((3, 5, 2, 3), (3, 5, 2, 2), (2, 0, 3, 0)):
        assert g.product_plan_info(ra, rb, rc, tri)["auto_choice"] == (1 if setting == "all=1" else 0)
    om_ref, _ = ref.energy(L1)
    assert abs(om - om_ref) / lsq.HARTREE_EV / n < 1e-6
    Gr = ref.gradient(L1)
    assert rel_err(G.cpu().numpy(), 0.5 * (Gr.val + oracle.transpose(Gr, Gr.pat).val)) < 2e-5
    Lr, _ = OL.minimise(ref, L0, 200, tol_ha_per_atom=1e-10)
    om_min = ref.energy(Lr)[0]
    Lg = cuda(L0.val)
    rep = ctx.minimise(Lg, cuda(Sb.val), cuda(Hb.val), MU, max_iter=200, tol_ha_per_atom=1e-9,
                       precision=lsq.TF32X3, refine_iter=3)
    g.device_status()
    assert abs(rep["omega_ev"] - om_min) / lsq.HARTREE_EV / n < 1e-6
