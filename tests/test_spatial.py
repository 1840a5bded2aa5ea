"""The spatial decomposition of the LNV step over gloo ranks on CPU (Sec. 4.2).

Each rank owns a slab of an elongated Si box (or a box of a 2 x 2 x 1 grid over a
wider one), holds the atoms within the halo depth of it, and runs the distributed
energy, gradient, line-search cubic and CG of
paper_2002_07704_gb300.spatial with the oracle's block algebra as its engine.  That
engine computes the owned rows only and fills every other row of each result with NaN,
so a halo row that the decomposition forgot to fetch poisons the answer.  The results
are compared with the single-process oracle.
"""
import os
import socket

import numpy as np
import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
from oracle import lnv as OL
from paper_2002_07704_gb300 import spatial as SP
from synth import config_seed, diamond_si_positions, sk_blocks

R_S = R_H = 2.6           # first neighbour shell of Si (2.35 A)
R_L = 4.0                 # second shell (3.84 A)
RANGES = (R_S, R_H, R_L)
MU = -2.0
SHAPE = (16, 2, 2)        # conventional cells; slabs cut along the long x axis
B = 4


GRID_SHAPE = (12, 12, 2)   # for a 2 x 2 x 1 grid of boxes


def _geometry(shape=SHAPE):
    return diamond_si_positions(shape, 0.05, config_seed(0) + 40)


def _patterns(pos, cell, rg=RANGES):
    return {R: oracle.neighbour_list(pos, cell, R) for R in SP.lnv_ranges(*rg)}


def _inputs(pos, cell, pats, rg=RANGES):
    """H on R_H's pattern and S on R_S's (the model's blocks of each listed pair)."""
    pS, pH = pats[rg[0]], pats[rg[1]]
    H, _ = sk_blocks(pos, cell, pH.rows(), pH.col)
    _, S = sk_blocks(pos, cell, pS.rows(), pS.col)
    return pH, H, S


class OracleEngine:
    """The oracle's block algebra on the held atoms, owned rows only, NaN elsewhere."""

    def __init__(self, slabs):
        self.sl, self.b = slabs, slabs.b
        self.pats = {R: oracle.Pattern(hp.n, hp.ptr, hp.col, R) for R, hp in slabs.pats.items()}
        self.own = np.zeros(slabs.held.size, dtype=bool)
        self.own[slabs.own] = True

    def _pat(self, R):
        return self.pats[self.sl.pattern(R).R]

    def _poison(self, X):
        X.val[~self.own[X.pat.rows()]] = np.nan
        return X

    def new(self, R):
        return oracle.Bsr(self._pat(R), self.b)

    def from_global(self, R, gvals):
        return oracle.Bsr(self._pat(R), self.b, np.asarray(gvals)[self.sl.pattern(R).gpos])

    def to_host(self, X):
        return X.data.val

    def matmul(self, A, B_, R):
        C, _ = oracle.matmul(A.data, B_.data, self._pat(R), rows=self.sl.own)
        return self._poison(C)

    def lincomb(self, terms, R, rows=None):
        C = self.new(R)
        for c, X in terms:
            C.val += c * oracle.restrict(X.data, C.pat).val
        return C if rows == "held" else self._poison(C)

    def transpose(self, X, R, alpha=1.0):
        T = oracle.transpose(X.data, self._pat(R))
        T.val *= alpha
        return self._poison(T)

    def _owned_blocks(self, X):
        return np.nonzero(self.own[X.pat.rows()])[0]

    def trace(self, X, Y):
        p = self._owned_blocks(X.data)
        i, j = X.data.pat.rows()[p], X.data.pat.col[p].astype(np.int64)
        n = Y.data.pat.n
        keys = Y.data.pat.rows() * n + Y.data.pat.col
        q = np.searchsorted(keys, j * n + i)
        q = np.minimum(q, keys.size - 1)
        hit = keys[q] == j * n + i
        return float(np.sum(X.data.val[p[hit]] * np.transpose(Y.data.val[q[hit]], (0, 2, 1))))

    def dot(self, X, Y):
        p = self._owned_blocks(X.data)
        return float(np.sum(X.data.val[p] * Y.data.val[p]))

    def _idx(self, R, rows):
        return SP.row_blocks(self.sl.pattern(R).ptr, rows)

    def get_rows(self, X, rows):
        return X.data.val[self._idx(X.R, rows)]

    def set_rows(self, X, rows, blocks):
        X.data.val[self._idx(X.R, rows)] = blocks


class DroppingSlabs(SP.Slabs):
    """A planted mistake: every halo request forgets its last row."""

    def exchange(self, engine, X, need):
        need = np.asarray(need, dtype=np.int64)
        ext = need[self.owners[self.held[need]] != self.rank]
        if ext.size:
            need = np.setdiff1d(need, ext[-1:])
        super().exchange(engine, X, need)


def _owned_global(sl, X_host, R):
    hp = sl.pattern(R)
    p = SP.row_blocks(hp.ptr, sl.own)
    return hp.gpos[p], X_host[p]


def _rank(rank, world, port, L2g, L0g, out, drop, shape=SHAPE, grid=None, cg_steps=3, rg=RANGES):
    import datetime
    R_S, R_H, R_L = rg
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        pos, cell = _geometry(shape)
        pats = _patterns(pos, cell, rg)
        _, H, S = _inputs(pos, cell, pats, rg)
        cls = DroppingSlabs if drop else SP.Slabs
        sl = cls(pos, cell, world, rank, {R: (p.ptr, p.col) for R, p in pats.items()}, B, grid=grid)
        en = OracleEngine(sl)
        dl = SP.DistributedLnv(sl, en, SP.Mat(R_S, en.from_global(R_S, S), complete=True),
                               SP.Mat(R_H, en.from_global(R_H, H), complete=True), R_L, MU)
        L2 = SP.Mat(R_L, en._poison(en.from_global(R_L, L2g)))
        om, ne = dl.energy(L2)
        res = dict(omega=om, ne=ne, n_held=int(sl.held.size), n_own=int(sl.own.size))
        if not drop:
            G = dl.symmetric(dl.gradient(L2))
            D = SP.Mat(R_L, en.lincomb([(-1.0, G)], R_L))
            res["c"] = dl.cubic(L2, D, G)
            res["gpos"], res["gval"] = _owned_global(sl, en.to_host(G), R_L)
            L3, hist = dl.minimise(SP.Mat(R_L, en._poison(en.from_global(R_L, L0g))), cg_steps)
            res["lpos"], res["lval"] = _owned_global(sl, en.to_host(L3), R_L)
            res["hist"] = hist
            res["sent"], res["received"] = sl.sent_rows, sl.received_rows
        out[rank] = res
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, L2, L0, drop=False, shape=SHAPE, grid=None, cg_steps=3, rg=RANGES):
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), L2, L0, out, drop, shape, grid, cg_steps, rg),
                 nprocs=world, join=True)
        return dict(out)


def _reference(shape, cg_steps, rg=RANGES):
    R_S, R_H, R_L = rg
    pos, cell = _geometry(shape)
    m = OL.System(pos, cell)
    pS, pH = m.pattern(R_S), m.pattern(R_H)
    H, _ = sk_blocks(pos, cell, pH.rows(), pH.col)
    _, S = sk_blocks(pos, cell, pS.rows(), pS.col)
    # the oracle holds S on H's pattern: zero blocks where R_S < R_ij <= R_H
    lnv = OL.Lnv(m, oracle.Bsr(pS, B, S), oracle.Bsr(pH, B, H), R_L, MU)
    L0 = OL.onsite_inverse_half(lnv.S, lnv.pat_L)
    L2, _ = OL.minimise(lnv, L0, 2)
    om, ne = lnv.energy(L2)
    G = lnv.gradient(L2)
    G = 0.5 * (G + oracle.transpose(G, G.pat))
    c = lnv.cubic(L2, -1.0 * G, G)
    L3, hist = OL.minimise(lnv, L0, cg_steps)
    return dict(n=pos.shape[0], L0=L0.val, L2=L2.val, omega=om, ne=ne, G=G.val, c=c, L3=L3.val, hist=hist)


@pytest.fixture(scope="module")
def ref():
    """The single-process oracle: L after 2 CG steps, its Omega, N_e, symmetric gradient
    and cubic along -G, and 3 CG steps from the on-site start."""
    return _reference(SHAPE, 3)


@pytest.fixture(scope="module")
def ref_short_s():
    """The same with S on a shorter range than H: R_S = 2.6 A, R_H = R_L = 4.0 A."""
    return _reference(SHAPE, 2, (2.6, 4.0, 4.0))


@pytest.fixture(scope="module")
def ref_grid():
    """The same on the 12 x 12 x 2-cell box, with 2 CG steps from the on-site start."""
    return _reference(GRID_SHAPE, 2)


def _check(ref, res, world):
    n = ref["n"]
    assert sum(r["n_own"] for r in res.values()) == n
    for r in res.values():
        assert r["omega"] == pytest.approx(ref["omega"], rel=1e-12, abs=0)
        assert r["ne"] == pytest.approx(ref["ne"], rel=1e-12, abs=0)
        scale = sum(abs(v) for v in ref["c"])
        for a, b in zip(r["c"], ref["c"]):
            assert abs(a - b) <= 1e-12 * scale
        for h, hr in zip(r["hist"], ref["hist"]):
            assert h["omega"] == pytest.approx(hr["omega"], rel=1e-12, abs=0)
            assert h["alpha"] == pytest.approx(hr["alpha"], rel=1e-9, abs=0)
        assert r["received"] > 0 and r["sent"] > 0
    for key, refkey, tol in (("g", "G", 1e-12), ("l", "L3", 1e-11)):
        full = np.full_like(ref[refkey], np.nan)
        for r in res.values():
            assert np.all(np.isnan(full[r[key + "pos"]]))      # each block owned by one rank
            full[r[key + "pos"]] = r[key + "val"]
        assert np.all(np.isfinite(full))
        assert np.max(np.abs(full - ref[refkey])) <= tol * np.max(np.abs(ref[refkey]))


@pytest.mark.parametrize("world", [2, 3, 4])
def test_gloo_ranks_match_single_process(ref, world):
    res = _run(world, ref["L2"], ref["L0"])
    _check(ref, res, world)
    # the halo does not cover the whole box: rows beyond it are never held
    assert all(r["n_held"] < ref["n"] for r in res.values())


def test_gloo_box_grid_matches_single_process(ref_grid):
    """Four ranks on a 2 x 2 x 1 grid of boxes: each holds the atoms within the depth of its
    box along x and along y, fewer than the whole; same bar as the slabs."""
    res = _run(4, ref_grid["L2"], ref_grid["L0"], shape=GRID_SHAPE, grid=(2, 2, 1), cg_steps=2)
    _check(ref_grid, res, 4)
    assert all(r["n_held"] < 0.9 * ref_grid["n"] for r in res.values())


def test_gloo_ranks_with_s_shorter_than_h(ref_short_s):
    """R_S < R_H: S and H on their own ranges, H' = H - mu S on H's; same bar."""
    res = _run(2, ref_short_s["L2"], ref_short_s["L0"], cg_steps=2, rg=(2.6, 4.0, 4.0))
    _check(ref_short_s, res, 2)


def test_forgotten_halo_row_poisons_the_energy(ref):
    res = _run(2, ref["L2"], ref["L0"], drop=True)
    assert not any(np.isfinite(r["omega"]) for r in res.values())


def test_slabs_partition_and_held_atoms_cover_every_reach():
    pos, cell = _geometry()
    pats = _patterns(pos, cell)
    gp = {R: (p.ptr, p.col) for R, p in pats.items()}
    n = pos.shape[0]
    for world in (1, 2, 3, 5):
        seen = np.zeros(n, dtype=np.int64)
        for rank in range(world):
            sl = SP.Slabs(pos, cell, world, rank, gp, B)
            g_own = sl.held[sl.own]
            seen[g_own] += 1
            x = np.mod(pos[g_own, 0], cell[0])
            assert np.all(x >= rank * cell[0] / world - 1e-9) and np.all(x <= (rank + 1) * cell[0] / world + 1e-9)
            for R, p in pats.items():
                # every atom an owned row reaches is held, and the held pattern is the
                # global pattern restricted to the held atoms
                assert np.all(sl.g2l[SP.reach(p.ptr, p.col, g_own)] >= 0)
                hp = sl.pattern(R)
                for l in (0, sl.held.size // 2, sl.held.size - 1):
                    g = sl.held[l]
                    want = [c for c in p.col[p.ptr[g]:p.ptr[g + 1]] if sl.g2l[c] >= 0]
                    assert list(sl.held[hp.col[hp.ptr[l]:hp.ptr[l + 1]]]) == want
                    assert np.array_equal(p.col[hp.gpos[hp.ptr[l]:hp.ptr[l + 1]]], want)
        assert np.all(seen == 1)
        if world == 1:
            assert sl.held.size == n


def test_box_grid_partition_and_held_atoms_cover_every_reach():
    pos, cell = _geometry(GRID_SHAPE)
    pats = _patterns(pos, cell)
    gp = {R: (p.ptr, p.col) for R, p in pats.items()}
    deep = pats[max(pats)]
    n = pos.shape[0]
    for grid in ((2, 2, 1), (1, 3, 1), (3, 1, 2)):
        world = grid[0] * grid[1] * grid[2]
        seen = np.zeros(n, dtype=np.int64)
        for rank in range(world):
            sl = SP.Slabs(pos, cell, world, rank, gp, B, grid=grid)
            g_own = sl.held[sl.own]
            seen[g_own] += 1
            box = (rank // (grid[1] * grid[2]), (rank // grid[2]) % grid[1], rank % grid[2])
            for a in range(3):
                x = np.mod(pos[g_own, a], cell[a])
                assert np.all(x >= box[a] * cell[a] / grid[a] - 1e-9)
                assert np.all(x <= (box[a] + 1) * cell[a] / grid[a] + 1e-9)
            assert np.all(sl.g2l[SP.reach(deep.ptr, deep.col, g_own)] >= 0)
        assert np.all(seen == 1)
    with pytest.raises(ValueError):
        SP.Slabs(pos, cell, 3, 0, gp, B, grid=(2, 2, 1))


def test_lnv_ranges_are_the_product_sums():
    r = SP.lnv_ranges(2.6, 2.6, 4.0)
    assert r == sorted(set(r))
    for want in (2.6, 4.0, 6.6, 10.6, 9.2, 13.2):
        assert min(abs(v - want) for v in r) < 1e-12
    assert len(r) == 6


def test_row_blocks_and_reach():
    ptr = np.array([0, 2, 2, 5, 6])
    col = np.array([1, 3, 0, 2, 3, 1])
    assert list(SP.row_blocks(ptr, [2, 0, 1, 3])) == [2, 3, 4, 0, 1, 5]
    assert list(SP.row_blocks(ptr, [])) == []
    assert list(SP.reach(ptr, col, [0, 3])) == [1, 3]
    assert list(SP.reach(ptr, col, [1])) == []


def test_cubic_step_closed_forms():
    # quadratic: minimum at -c1 / (2 c2)
    assert SP.cubic_step(-3.0, 2.0, 0.0) == pytest.approx(0.75, rel=1e-15)
    # cubics with a local minimum: the derivative vanishes there, the curvature is positive
    for c1, c2, c3 in ((-1.0, -0.5, 0.2), (-1.0, 1.0, -0.1), (-2.0, 0.0, 3.0)):
        a = SP.cubic_step(c1, c2, c3)
        assert a > 0 and abs(c1 + 2 * c2 * a + 3 * c3 * a * a) < 1e-14
        assert 2 * c2 + 6 * c3 * a > 0
    # no stationary point (c2^2 < 3 c1 c3), positive curvature at zero: the quadratic part's minimum
    assert SP.cubic_step(-1.0, 0.1, -1.0) == pytest.approx(5.0, rel=1e-15)
    # nothing to stop at
    assert SP.cubic_step(-1.0, -1.0, -1.0) is None


def _gpu_rank(rank, world, port, L2g, L0g, out):
    import datetime
    import torch
    torch.cuda.set_device(0)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        pos, cell = _geometry()
        pats = _patterns(pos, cell)
        _, H, S = _inputs(pos, cell, pats)
        sl = SP.Slabs(pos, cell, world, rank, {R: (p.ptr, p.col) for R, p in pats.items()}, B)
        en = SP.GpuEngine(sl)
        dl = SP.DistributedLnv(sl, en, SP.Mat(R_S, en.from_global(R_S, S), complete=True),
                               SP.Mat(R_H, en.from_global(R_H, H), complete=True), R_L, MU)
        others = np.setdiff1d(np.arange(sl.held.size), sl.own)

        def owned_only(gvals):
            # rows other ranks own start at zero: a missed halo row changes the result
            X = SP.Mat(R_L, en.from_global(R_L, gvals))
            nb = sl.pattern(R_L).ptr
            en.set_rows(X, others, np.zeros((int(np.sum(nb[others + 1] - nb[others])), B, B)))
            return X

        L2 = owned_only(L2g)
        om, ne = dl.energy(L2)
        G = dl.symmetric(dl.gradient(L2))
        D = SP.Mat(R_L, en.lincomb([(-1.0, G)], R_L))
        res = dict(omega=om, ne=ne, n_held=int(sl.held.size), n_own=int(sl.own.size), c=dl.cubic(L2, D, G))
        res["gpos"], res["gval"] = _owned_global(sl, en.to_host(G), R_L)
        L3, hist = dl.minimise(owned_only(L0g), 3)
        res["lpos"], res["lval"] = _owned_global(sl, en.to_host(L3), R_L)
        res["hist"] = hist
        res["sent"], res["received"] = sl.sent_rows, sl.received_rows
        en.geom.device_status()
        out[rank] = res
    finally:
        dist.destroy_process_group()


@pytest.mark.gpu
def test_gpu_engine_two_gloo_ranks_match_single_process(ref):
    """The library's FP64 products as each rank's engine (both ranks on cuda:0: their
    kernels never wait on one another; the halo rows travel through gloo on the host)."""
    world = 2
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_gpu_rank, args=(world, _free_port(), ref["L2"], ref["L0"], out), nprocs=world, join=True)
        res = dict(out)
    _check(ref, res, world)
