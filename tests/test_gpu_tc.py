"""Parity of the tensor-core product (precision TF32X3) against the CPU oracle.

The product splits every float32 operand value v into hi = tf32(v) and
lo = tf32(v - hi) (22 bits of v) and accumulates hi.hi + hi.lo + lo.hi +
lo.lo in FP32 on the tensor cores, so its error is that of a float32
product: the bound is 1e-5 of max |A|.|B| (plus |beta| max |C0|), as for
the FP32 FMA kernels.  A product that dropped the lo terms would miss it by
an order of magnitude (tf32 alone keeps 11 bits: ~5e-4 relative).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2002_07704_gb300 as lsq
from gpu_common import cuda, gpu_geometry, si
from synth import config_seed

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    lsq.build()
    lsq.load()


def _bound(opA, opB, pc, alpha, beta, C0):
    absA = oracle.Bsr(opA.pat, 4, np.abs(opA.val))
    absB = oracle.Bsr(opB.pat, 4, np.abs(opB.val))
    bnd, _ = oracle.matmul(absA, absB, pc)
    return abs(alpha) * bnd.val.max() + abs(beta) * (np.abs(C0.val).max() if C0 is not None else 0.0)


def _tri_mask(pc, triangle):
    rows = np.repeat(np.arange(pc.n), np.diff(pc.ptr))
    if triangle == 2:
        return pc.col >= rows
    if triangle == 3:
        return pc.col <= rows
    return np.ones(pc.nnzb, dtype=bool)


def _case(pos, cell, ra, rb, rc, ta, tb, triangle, alpha, beta, seed):
    ranges = sorted(set([ra, rb, rc]))
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(seed)
    A = oracle.Bsr(P[ra], 4, rng.standard_normal((P[ra].nnzb, 4, 4)))
    B = oracle.Bsr(P[rb], 4, rng.standard_normal((P[rb].nnzb, 4, 4)))
    C0 = oracle.Bsr(P[rc], 4, rng.standard_normal((P[rc].nnzb, 4, 4)))
    opA = oracle.transpose(A, P[ra]) if ta else A
    opB = oracle.transpose(B, P[rb]) if tb else B
    ref, triples = oracle.matmul(opA, opB, P[rc])
    mask = _tri_mask(P[rc], triangle)
    rows = np.repeat(np.arange(P[rc].n), np.diff(P[rc].ptr))
    if triangle in (1, 2, 3):
        # triples of the computed triangle: with all-ones blocks every triple adds 4 to C_ij[0][0]
        ones_a = oracle.Bsr(opA.pat, 4, np.ones_like(opA.val))
        ones_b = oracle.Bsr(opB.pat, 4, np.ones_like(opB.val))
        cnt, _ = oracle.matmul(ones_a, ones_b, P[rc])
        keep = (P[rc].col >= rows) if triangle in (1, 2) else (P[rc].col <= rows)
        triples = int(round(cnt.val[:, 0, 0][keep].sum() / 4.0))
    Cg = cuda(C0.val, torch.float32)
    t = lsq.block_matmul(g, 4, cuda(A.val, torch.float32), g.range_id(ra), cuda(B.val, torch.float32),
                         g.range_id(rb), Cg, g.range_id(rc), precision=lsq.TF32X3, trans_a=ta, trans_b=tb,
                         alpha=alpha, beta=beta, triangle=triangle)
    torch.cuda.synchronize()
    g.device_status()
    got = Cg.double().cpu().numpy()
    return got, ref, C0, mask, t, triples, _bound(opA, opB, P[rc], alpha, beta, C0), P[rc], rows


@pytest.mark.parametrize("n,ra,rb,rc,ta,tb,triangle", [
    (3, 16.6, 23.2, 10.0, 0, 1, 2),   # SL.Q^T on the upper triangle of R_L (the gradient's shape)
    (3, 16.6, 23.2, 10.0, 0, 1, 3),   # lower triangle
    (3, 10.0, 6.6, 16.6, 0, 0, 0),    # L.S at its natural range, every block
    (3, 16.6, 10.0, 26.6, 0, 1, 0),   # LS.L
    (2, 6.6, 10.0, 8.0, 1, 1, 0),     # both operands transposed, truncated result
    (2, 23.2, 16.6, 10.0, 1, 0, 0),   # a long operand walked as rows
])
def test_tf32x3_matches_oracle(n, ra, rb, rc, ta, tb, triangle):
    pos, cell = si(n, 0.1, config_seed(0) + 7 * n)
    alpha, beta = 0.75, -0.5
    got, ref, C0, mask, t, triples, scale, pc, _ = _case(pos, cell, ra, rb, rc, ta, tb, triangle, alpha, beta,
                                                         300 + n)
    want = alpha * ref.val + beta * C0.val
    assert t == triples
    err = np.abs(got - want)[mask].max()
    assert err <= 1e-5 * scale, (err, scale)
    if triangle in (2, 3):
        # blocks outside the triangle are left as they were
        assert np.array_equal(got[~mask], C0.val[~mask].astype(np.float32).astype(np.float64))


def test_tf32x3_symmetric_result_mirrors():
    """triangle 1: C = LS.L^T style symmetric product, upper blocks computed, lower mirrored."""
    pos, cell = si(3, 0.1, config_seed(0) + 5)
    ranges = [6.6, 16.6]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(11)
    A = oracle.Bsr(P[6.6], 4, rng.standard_normal((P[6.6].nnzb, 4, 4)))
    # C = A.A^T is symmetric
    ref, _ = oracle.matmul(A, oracle.transpose(A, P[6.6]), P[16.6])
    Cg = torch.zeros((P[16.6].nnzb, 4, 4), dtype=torch.float32, device="cuda")
    Ag = cuda(A.val, torch.float32)
    lsq.block_matmul(g, 4, Ag, 0, Ag, 0, Cg, 1, precision=lsq.TF32X3, trans_b=True, triangle=1)
    torch.cuda.synchronize()
    g.device_status()
    absA = oracle.Bsr(P[6.6], 4, np.abs(A.val))
    bnd, _ = oracle.matmul(absA, oracle.transpose(absA, P[6.6]), P[16.6])
    got = Cg.double().cpu().numpy()
    assert np.abs(got - ref.val).max() <= 1e-5 * bnd.val.max()
    # off the diagonal exactly symmetric: lower blocks are copies of the upper ones (the
    # diagonal blocks are computed, symmetric to rounding)
    gt = oracle.transpose(oracle.Bsr(P[16.6], 4, got), P[16.6])
    pc = P[16.6]
    off = pc.col != np.repeat(np.arange(pc.n), np.diff(pc.ptr))
    assert np.array_equal(gt.val[off], got[off])


def test_tf32x3_ragged_group_and_split_precision():
    """61 atoms (the last group of 8 holds 5): every block against the oracle, and the error
    is far below what tf32 without the lo parts allows."""
    pos, cell = si(2, 0.1, config_seed(0) + 17)
    pos = np.delete(pos, [3, 20, 47], axis=0)
    got, ref, C0, mask, t, triples, scale, pc, _ = _case(pos, cell, 10.0, 6.6, 16.6, 0, 0, 0, 1.0, 0.0, 909)
    assert pos.shape[0] == 61 and t == triples
    err = np.abs(got - ref.val).max()
    assert err <= 1e-5 * scale
    assert err <= 2e-6 * scale   # tf32 hi alone: ~2^-11 relative


def test_tf32x3_empty_and_other_block_sizes():
    """No atoms: nothing to do.  b = 13 with TF32X3 runs the float32 FMA kernels."""
    g0 = gpu_geometry(np.zeros((0, 3)), [10.0, 10.0, 10.0], [3.0])
    z = torch.zeros((0, 4, 4), dtype=torch.float32, device="cuda")
    assert lsq.block_matmul(g0, 4, z, 0, z.clone(), 0, z.clone(), 0, precision=lsq.TF32X3) == 0
    pos, cell = si(1, 0.1, config_seed(0) + 3)
    ranges = [3.0, 4.0]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(3)
    A = oracle.Bsr(P[3.0], 13, rng.standard_normal((P[3.0].nnzb, 13, 13)))
    ref, tr = oracle.matmul(A, A, P[4.0])
    Cg = torch.zeros((P[4.0].nnzb, 13, 13), dtype=torch.float32, device="cuda")
    Ag = cuda(A.val, torch.float32)
    assert lsq.block_matmul(g, 13, Ag, 0, Ag.clone(), 0, Cg, 1, precision=lsq.TF32X3) == tr
    torch.cuda.synchronize()
    absA = oracle.Bsr(P[3.0], 13, np.abs(A.val))
    bnd, _ = oracle.matmul(absA, absA, P[4.0])
    assert np.abs(Cg.double().cpu().numpy() - ref.val).max() <= 1e-5 * bnd.val.max()


def test_tf32x3_full_size_sampled_rows():
    """4096-atom Si, SL.Q^T on the upper triangle of the 10 A range (A 16.6 A, B 23.2 A), in
    the launch configuration the benchmark uses: 64 sampled rows against the oracle, and
    every block against the float32 FMA kernels."""
    pos, cell = si(8, 0.05, config_seed(1))
    ranges = [10.0, 16.6, 23.2]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(2002)
    A = oracle.Bsr(P[16.6], 4, rng.standard_normal((P[16.6].nnzb, 4, 4)).astype(np.float32).astype(np.float64))
    Q = oracle.Bsr(P[23.2], 4, rng.standard_normal((P[23.2].nnzb, 4, 4)).astype(np.float32).astype(np.float64))
    rows = np.sort(rng.choice(4096, size=64, replace=False))
    ref, _ = oracle.matmul(A, oracle.transpose(Q, P[23.2]), P[10.0], rows=rows)
    Ag, Qg = cuda(A.val, torch.float32), cuda(Q.val, torch.float32)
    Ct = torch.zeros((P[10.0].nnzb, 4, 4), dtype=torch.float32, device="cuda")
    Cf = torch.zeros_like(Ct)
    tt = lsq.block_matmul(g, 4, Ag, 1, Qg, 2, Ct, 0, precision=lsq.TF32X3, trans_b=True, triangle=2)
    tf = lsq.block_matmul(g, 4, Ag, 1, Qg, 2, Cf, 0, precision=lsq.F32, trans_b=True, triangle=2)
    torch.cuda.synchronize()
    g.device_status()
    assert tt == tf
    pc = P[10.0]
    prow = np.repeat(np.arange(pc.n), np.diff(pc.ptr))
    sel = np.isin(prow, rows) & (pc.col >= prow)
    # |A|.|B| bound of the sampled rows
    absA = oracle.Bsr(P[16.6], 4, np.abs(A.val))
    absQ = oracle.Bsr(P[23.2], 4, np.abs(Q.val))
    bnd, _ = oracle.matmul(absA, oracle.transpose(absQ, P[23.2]), pc, rows=rows)
    scale = bnd.val[sel].max()
    got = Ct.double().cpu().numpy()
    assert np.abs(got[sel] - ref.val[sel]).max() <= 1e-5 * scale
    up = pc.col >= prow
    assert np.abs(got[up] - Cf.double().cpu().numpy()[up]).max() <= 2e-5 * scale



def _step_choices(g, nr):
    """(range_a, range_b, range_c, upper) -> kernel the mixed step chose (1 tensor cores, 0 FMA)."""
    out = {}
    for ra in range(nr):
        for rb in range(nr):
            for rc in range(nr):
                for tri, upper in ((0, 0), (2, 1), (3, 2)):
                    try:
                        info = g.product_plan_info(ra, rb, rc, tri)
                    except lsq.LsqError:
                        continue
                    if info["auto_choice"] >= 0:
                        out[(ra, rb, rc, tri)] = info["auto_choice"]
    return out


def _explicit_products_match(g, choices, seed):
    gen = torch.Generator(device="cuda").manual_seed(seed)
    for (ra, rb, rc, tri) in choices:
        A = torch.randn((g.nnzb(ra), 4, 4), dtype=torch.float32, device="cuda", generator=gen)
        B = torch.randn((g.nnzb(rb), 4, 4), dtype=torch.float32, device="cuda", generator=gen)
        Ct = torch.zeros((g.nnzb(rc), 4, 4), dtype=torch.float32, device="cuda")
        Cf = torch.zeros_like(Ct)
        lsq.block_matmul(g, 4, A, ra, B, rb, Ct, rc, precision=lsq.TF32X3, trans_b=True, triangle=tri)
        lsq.block_matmul(g, 4, A, ra, B, rb, Cf, rc, precision=lsq.F32, trans_b=True, triangle=tri)
        torch.cuda.synchronize()
        g.device_status()
        assert g.product_plan_info(ra, rb, rc, tri)["tiles"] > 0
        assert (Ct - Cf).abs().max().item() <= 2e-5 * Cf.abs().max().item()


def test_explicit_tf32x3_after_the_mixed_choice(monkeypatch):
    """The mixed step (LSQ_TF32X3 requested of the LNV path) keeps one kernel per product and
    drops the other's plan.  A later explicit LSQ_TF32X3 product on the same ranges builds its
    tensor-core plan again and matches LSQ_F32: after the timing (64 atoms, where the FMA
    kernels win most products) and after LSQ_TC_CHOICE=all=0 fixed every choice to FMA."""
    pos, cell = si(2, 0.05, config_seed(0))
    ranges = lsq.lnv_required_ranges(6.6, 6.6, 8.0)
    S_, H_ = None, None
    for forced in (False, True):
        if forced:
            monkeypatch.setenv("LSQ_TC_CHOICE", "all=0")
        g = gpu_geometry(pos, cell, ranges)
        ctx = lsq.Lnv(g, 4, 6.6, 6.6, 8.0)
        if S_ is None:
            from gpu_common import gpu_pattern, si_hs
            pH = gpu_pattern(g, ctx.rH)
            H, S = si_hs(pos, cell, pH, 4)
            S_, H_ = cuda(S), cuda(H)
        L = torch.zeros((g.nnzb(ctx.rL), 4, 4), dtype=torch.float64, device="cuda")
        ctx.init_L(S_, L)
        ctx.energy_gradient(L, S_, H_, -2.0, precision=lsq.TF32X3)
        g.device_status()
        choices = _step_choices(g, len(g.ranges))
        assert len(choices) >= 4
        if forced:
            assert set(choices.values()) == {0}
        _explicit_products_match(g, choices, 4 + forced)
        monkeypatch.delenv("LSQ_TC_CHOICE", raising=False)


def test_tf32x3_expired_wait_reports_timeout(monkeypatch):
    """Failure detection of the tensor-core product without a GPU fault.  With the bound of its
    pipeline waits set to 0 ns (LSQ_TC_WAIT_NS=0) a wait that does not succeed at once expires:
    the kernel records which wait gave up, drains its copies and MMAs (the final drain keeps its
    1 s bound), frees its tensor memory and returns.  lsq_device_status then reports
    LSQ_ERR_TIMEOUT once and clears it, and the geometry stays usable: the same product with the
    default bound matches the float32 FMA product (512 atoms)."""
    pos, cell = si(4, 0.05, config_seed(0))
    ranges = lsq.lnv_required_ranges(6.6, 6.6, 8.0)
    g = gpu_geometry(pos, cell, ranges)
    gen = torch.Generator(device="cuda").manual_seed(11)
    A = torch.randn((g.nnzb(3), 4, 4), dtype=torch.float32, device="cuda", generator=gen)
    B = torch.randn((g.nnzb(5), 4, 4), dtype=torch.float32, device="cuda", generator=gen)
    C = torch.zeros((g.nnzb(2), 4, 4), dtype=torch.float32, device="cuda")
    kw = dict(trans_b=True, triangle=2)
    lsq.block_matmul(g, 4, A, 3, B, 5, C, 2, precision=lsq.TF32X3, **kw)  # plan built, default bound
    g.device_status()
    monkeypatch.setenv("LSQ_TC_WAIT_NS", "0")
    lsq.block_matmul(g, 4, A, 3, B, 5, C, 2, precision=lsq.TF32X3, **kw)
    with pytest.raises(lsq.LsqError) as e:
        g.device_status()
    assert e.value.code == 8
    g.device_status()  # reported once, then cleared
    monkeypatch.delenv("LSQ_TC_WAIT_NS")
    Cf = torch.zeros_like(C)
    lsq.block_matmul(g, 4, A, 3, B, 5, C, 2, precision=lsq.TF32X3, **kw)
    lsq.block_matmul(g, 4, A, 3, B, 5, Cf, 2, precision=lsq.F32, **kw)
    torch.cuda.synchronize()
    g.device_status()
    assert (C - Cf).abs().max().item() <= 2e-5 * Cf.abs().max().item()
