"""Shared set-up of the GPU parity tests: the same seeded inputs for both sides."""
import numpy as np
import torch

import oracle
import paper_2002_07704_gb300 as lsq
from synth import diamond_si_positions, sk_blocks


def gpu_geometry(pos, cell, ranges):
    return lsq.Geometry(torch.from_numpy(pos).cuda(), cell, ranges)


def gpu_pattern(geom, r):
    rp, col = geom.pattern(r)
    return oracle.Pattern(geom.n_atoms, rp.cpu().numpy(), col.cpu().numpy(), geom.ranges[r])


def si_hs(pos, cell, pat, b=4, perturb=None):
    """H, S blocks (numpy) on a pattern, from the seeded Slater-Koster generator."""
    return sk_blocks(pos, cell, pat.rows(), pat.col, b=b, perturb_seed=perturb)


def cuda(x, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(x)).to(device="cuda", dtype=dtype)


def rel_err(x, ref):
    x = np.asarray(x, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    m = np.abs(ref).max()
    return float(np.abs(x - ref).max() / (m if m > 0 else 1.0))


def si(n, sigma, seed):
    return diamond_si_positions(n, sigma, seed)
