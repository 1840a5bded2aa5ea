"""The hand-written adjoint of the truncated product (autograd) against the oracle.

dOmega/dL from backward must equal the oracle's analytic LNV gradient
(general, unsymmetrised L) and central differences; dOmega/dH must equal
2 K^T (Omega is linear in H).  Float64 throughout; tolerances 1e-10
relative (same products, different summation order) except the finite
differences, whose error is set by the rounding of Omega (~1e-13 |Omega|)
over the step.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import lnv as OL
import paper_2002_07704_gb300 as lsq
from paper_2002_07704_gb300.autograd import BlockMatmulFn, lnv_omega
from gpu_common import cuda, gpu_geometry, gpu_pattern, rel_err, si, si_hs
from synth import config_seed

pytestmark = pytest.mark.gpu

R_S = R_H = 6.6
MU = -2.0


@pytest.fixture(scope="module")
def setup64():
    lsq.build()
    pos, cell = si(2, 0.05, config_seed(0))
    R_L = 8.0
    ranges = lsq.lnv_required_ranges(R_S, R_H, R_L)
    g = gpu_geometry(pos, cell, ranges)
    m = OL.System(pos, cell)
    pH = m.pattern(R_H)
    H, S = si_hs(pos, cell, pH)
    Hb, Sb = oracle.Bsr(pH, 4, H), oracle.Bsr(pH, 4, S)
    ref = OL.Lnv(m, Sb, Hb, R_L, MU)
    L0 = OL.onsite_inverse_half(Sb, ref.pat_L)
    L, _ = OL.minimise(ref, L0, 3)
    # an unsymmetric L: the adjoint must hold for general L
    rng = np.random.default_rng(11)
    L = L + 1e-3 * oracle.Bsr(L.pat, 4, rng.standard_normal(L.val.shape))
    return g, ref, Hb, Sb, L, (0, 1, 2, 3, 5)


def test_omega_and_gradient_match_oracle(setup64):
    g, ref, Hb, Sb, L, rid = setup64
    Lt = cuda(L.val).requires_grad_(True)
    Ht = cuda(Hb.val).requires_grad_(True)
    St = cuda(Sb.val)
    om = lnv_omega(g, 4, Lt, St, Ht, MU, rid)
    om.backward()
    om_ref, _ = ref.energy(L)
    assert abs(om.item() - om_ref) <= 1e-11 * abs(om_ref)
    assert rel_err(Lt.grad.cpu().numpy(), ref.gradient(L).val) <= 1e-10
    # dOmega/dH_ab = 2 K_ba, K = 3LSL - 2LSLSL (dense)
    Ld, Sd = L.dense(), Sb.dense()
    K = 3 * Ld @ Sd @ Ld - 2 * Ld @ Sd @ Ld @ Sd @ Ld
    dH_ref = oracle.Bsr.from_dense(2.0 * K.T, Hb.pat, 4).val
    assert rel_err(Ht.grad.cpu().numpy(), dH_ref) <= 1e-10


def test_gradient_finite_differences(setup64):
    """Omega(L + h e) is a cubic in h, so the Richardson combination of central
    differences at h and 2h is exact up to rounding."""
    g, ref, Hb, Sb, L, rid = setup64
    Lt = cuda(L.val).requires_grad_(True)
    Ht, St = cuda(Hb.val), cuda(Sb.val)
    om = lnv_omega(g, 4, Lt, St, Ht, MU, rid)
    om.backward()
    G = Lt.grad.cpu().numpy().ravel()
    gmax = np.abs(G).max()
    rng = np.random.default_rng(2002)
    h = 1e-3

    def omega_at(delta, flat):
        Lp = L.val.copy()
        Lp.flat[flat] += delta
        with torch.no_grad():
            return lnv_omega(g, 4, cuda(Lp), St, Ht, MU, rid, recompute=False).item()

    for flat in rng.choice(L.val.size, size=12, replace=False):
        d1 = (omega_at(h, flat) - omega_at(-h, flat)) / (2 * h)
        d2 = (omega_at(2 * h, flat) - omega_at(-2 * h, flat)) / (4 * h)
        fd = (4 * d1 - d2) / 3
        assert abs(fd - G[flat]) <= 1e-7 * gmax


def test_block_matmul_adjoint_identity():
    """<dC, (A.dB')> style identity: for C = (A.B)|C, <dC, C(A, dB)> = <B-adjoint(dC), dB>."""
    lsq.build()
    pos, cell = si(2, 0.1, 5)
    ranges = [4.0, 6.0, 7.5]
    g = gpu_geometry(pos, cell, ranges)
    P = {R: oracle.neighbour_list(pos, cell, R) for R in ranges}
    rng = np.random.default_rng(3)
    A = cuda(rng.standard_normal((P[4.0].nnzb, 4, 4))).requires_grad_(True)
    B = cuda(rng.standard_normal((P[6.0].nnzb, 4, 4))).requires_grad_(True)
    dC = cuda(rng.standard_normal((P[7.5].nnzb, 4, 4)))
    C = BlockMatmulFn.apply(A, B, g, 4, 0, 1, 2)
    (C * dC).sum().backward()
    dA, dB = A.grad.clone(), B.grad.clone()
    # directional checks: C is bilinear, so <dC, C(A, dB)> = <dB_grad, dB> exactly (up to rounding)
    eA = cuda(rng.standard_normal(A.shape))
    eB = cuda(rng.standard_normal(B.shape))
    with torch.no_grad():
        lhs_a = (BlockMatmulFn.apply(eA, B.detach(), g, 4, 0, 1, 2) * dC).sum().item()
        lhs_b = (BlockMatmulFn.apply(A.detach(), eB, g, 4, 0, 1, 2) * dC).sum().item()
    assert abs(lhs_a - (dA * eA).sum().item()) <= 1e-11 * max(1.0, abs(lhs_a))
    assert abs(lhs_b - (dB * eB).sum().item()) <= 1e-11 * max(1.0, abs(lhs_b))
    del pos, cell
