"""Spatial decomposition of the LNV minimisation over ranks: regions of atoms, halo rows.

Sec. 4.2 of the paper spreads the matrix work over processes by space: each process
owns the atoms of a region, and each product stays O(N) because a block of the result
needs only blocks of atoms within the product's reach (Sec. 2.3.2).  Here the cell is
cut into slabs along one axis, or into a px x py x pz grid of boxes, and rank r owns the
block rows of the atoms in region r.

Each rank holds its atoms and every atom within `depth` of its region (the largest range
of any matrix in the step), in global order, with the global range patterns restricted
to them.  A matrix is valid on the owned rows.  Before a product C = A.B the rank fetches
from their owners the rows of B that its rows of A reach: the halo rows.  The rows of
X^T a rank owns are the columns of its rows of X, so a transpose fetches the rows of X
within the pattern's reach.  H and S are known on every held row from the start.  Traces
and dots are summed over owned rows, then over ranks.  One exchange is a row request
(all-gather) and then point-to-point messages of whole block rows (torch.distributed).

The block algebra on the held atoms is an engine's work.  :class:`GpuEngine` does it with
this library's calls on the rank's GPU, on a geometry of the held atoms.  Any object with
the same methods will do.  The GPU engine computes the halo rows of every product too,
and only the owned rows are read.
"""
import numpy as np


def grid_owners(pos, cell, grid):
    """Owner rank of each atom on a px x py x pz grid of boxes of the orthorhombic cell:
    rank (ix py + iy) pz + iz, with i_a = floor(p_a x_a / L_a) of the wrapped coordinate."""
    pos = np.asarray(pos, dtype=np.float64)
    idx = []
    for a in range(3):
        f = np.mod(pos[:, a] / float(cell[a]), 1.0)
        idx.append(np.minimum((f * grid[a]).astype(np.int64), int(grid[a]) - 1))
    return (idx[0] * int(grid[1]) + idx[1]) * int(grid[2]) + idx[2]


def grid_held_atoms(pos, cell, owners, rank, grid, depth):
    """Global ids (ascending) of the atoms rank `rank` holds: its own, and every atom whose
    coordinate along each axis lies within `depth` of the rank's box (periodic).  Any atom
    within distance depth of an owned atom is among them."""
    pos = np.asarray(pos, dtype=np.float64)
    box = (rank // (grid[1] * grid[2]), (rank // grid[2]) % grid[1], rank % grid[2])
    near = np.ones(pos.shape[0], dtype=bool)
    for a in range(3):
        L = float(cell[a])
        x = np.mod(pos[:, a], L)
        lo, hi = box[a] * L / grid[a], (box[a] + 1) * L / grid[a]
        inside = np.mod(x - lo, L) < hi - lo
        d = np.minimum(np.mod(lo - x, L), np.mod(x - hi, L))   # below and above the box
        near &= inside | (d <= depth + 1e-9 * L)
    held = near | (np.asarray(owners) == rank)
    return np.nonzero(held)[0].astype(np.int64)


def _slab_grid(nranks, axis):
    g = [1, 1, 1]
    g[axis] = int(nranks)
    return tuple(g)


def slab_owners(pos, cell, nranks, axis=0):
    """Owner rank of each atom: slab floor(nranks x / L) of its coordinate x along the
    axis of the orthorhombic cell (x wrapped into [0, L))."""
    return grid_owners(pos, cell, _slab_grid(nranks, axis))


def slab_held_atoms(pos, cell, owners, rank, nranks, depth, axis=0):
    """Global ids (ascending) of the atoms rank `rank` holds: its own, and every atom whose
    periodic distance along the axis from the slab is at most `depth`."""
    return grid_held_atoms(pos, cell, owners, rank, _slab_grid(nranks, axis), depth)


def row_blocks(ptr, rows):
    """Block indices of the given rows of a CSR pattern, row after row."""
    ptr = np.asarray(ptr, dtype=np.int64)
    rows = np.asarray(rows, dtype=np.int64)
    starts = ptr[rows]
    lens = ptr[rows + 1] - starts
    first = np.cumsum(lens) - lens
    return np.repeat(starts - first, lens) + np.arange(int(lens.sum()), dtype=np.int64)


def reach(ptr, col, rows):
    """Columns of a CSR pattern over the given rows (sorted, unique): the rows of B that
    those rows of A reach in a product A.B."""
    return np.unique(np.asarray(col)[row_blocks(ptr, rows)]).astype(np.int64)


def lnv_ranges(R_S, R_H, R_L):
    """Every range the distributed energy, gradient and line-search terms form, as the
    float sums the products make (the range of A.B is R_A + R_B).  The largest is the
    halo depth."""
    R_LS = R_L + R_S
    R_DSD = R_LS + R_L
    R_DSDS = R_DSD + R_S
    R_DSLS = R_LS + R_LS
    R_SLH = R_LS + R_H
    out = []
    for r in sorted(float(v) for v in (R_S, R_H, R_L, R_LS, R_DSD, R_DSDS, R_DSLS, R_SLH, R_H + R_LS)):
        if not out or r - out[-1] > 1e-9 * r:       # sums equal up to rounding: one range
            out.append(r)
    return out


class HeldPattern:
    """A global range pattern restricted to the held atoms, in held (local) ids.

    ptr, col: the CSR of the restriction; gpos[p]: the global block index of local block
    p; gptr: the global row pointer (row lengths of the full rows that owners send)."""

    def __init__(self, R, gptr, gcol, held, g2l):
        self.R = float(R)
        gptr = np.asarray(gptr, dtype=np.int64)
        gcol = np.asarray(gcol, dtype=np.int64)
        self.gptr = gptr
        idx = row_blocks(gptr, held)
        rows = np.repeat(np.arange(held.size), gptr[held + 1] - gptr[held])
        keep = g2l[gcol[idx]] >= 0
        self.gpos = idx[keep].astype(np.int64)
        self.col = g2l[gcol[self.gpos]].astype(np.int32)
        counts = np.bincount(rows[keep], minlength=held.size)
        self.ptr = np.zeros(held.size + 1, dtype=np.int64)
        np.cumsum(counts, out=self.ptr[1:])
        self.n = int(held.size)

    @property
    def nnzb(self):
        return int(self.ptr[-1])


class Mat:
    """A distributed block matrix: the engine's data on range R, valid on the owned rows,
    on the halo rows fetched since it was formed, and on every held row if `complete`
    (H and S, which every rank builds for all of its atoms)."""

    __slots__ = ("R", "data", "halo", "complete")

    def __init__(self, R, data, complete=False):
        self.R = float(R)
        self.data = data
        self.halo = np.zeros(0, dtype=np.int64)
        self.complete = bool(complete)


class Slabs:
    """The decomposition of one geometry over the ranks of a process group.

    pos, cell: the whole system (orthorhombic cell); patterns: {R: (ptr, col)}, the global
    range patterns of every range in `ranges` (CSR, columns ascending); b: block size.
    Rank `rank` owns the atoms of slab `rank` along `axis` or, with grid = (px, py, pz),
    of box `rank` of that grid, and holds every atom within the largest range of its
    region.  `sent_rows` and `received_rows` count the block rows exchanged.
    """

    def __init__(self, pos, cell, nranks, rank, patterns, b, axis=0, group=None, grid=None):
        self.nranks, self.rank, self.group, self.b = int(nranks), int(rank), group, int(b)
        self.cell = np.asarray(cell, dtype=np.float64)
        self.ranges = sorted(float(r) for r in patterns)
        self.depth = max(self.ranges)
        n = np.asarray(pos).shape[0]
        self.grid = _slab_grid(nranks, axis) if grid is None else tuple(int(v) for v in grid)
        if int(np.prod(self.grid)) != self.nranks:
            raise ValueError("the grid's boxes must number the ranks")
        self.owners = grid_owners(pos, cell, self.grid)
        self.held = grid_held_atoms(pos, cell, self.owners, rank, self.grid, self.depth)
        self.g2l = np.full(n, -1, dtype=np.int64)
        self.g2l[self.held] = np.arange(self.held.size)
        self.pos = np.ascontiguousarray(np.asarray(pos, dtype=np.float64)[self.held])
        self.own = np.nonzero(self.owners[self.held] == rank)[0].astype(np.int64)
        self.pats = {}
        for R in self.ranges:
            gptr, gcol = patterns[R]
            hp = HeldPattern(R, gptr, gcol, self.held, self.g2l)
            g_own = self.held[self.own]
            if not np.array_equal(hp.ptr[self.own + 1] - hp.ptr[self.own],
                                  np.asarray(gptr)[g_own + 1] - np.asarray(gptr)[g_own]):
                raise ValueError("an owned row of range %g reaches beyond the held atoms" % R)
            self.pats[R] = hp
        self.sent_rows = 0
        self.received_rows = 0

    def pattern(self, R):
        """The held pattern of range R (matched to within 1e-9 relative)."""
        R = float(R)
        for r in self.ranges:
            if abs(r - R) <= 1e-9 * max(1.0, abs(R)):
                return self.pats[r]
        raise KeyError("range %g is not among the decomposition's ranges" % R)

    def reach(self, R, rows=None):
        """Held rows that `rows` (default: the owned rows) reach in the pattern of range R."""
        p = self.pattern(R)
        return reach(p.ptr, p.col, self.own if rows is None else rows)

    def exchange(self, engine, X, need):
        """Make rows `need` (held ids) of X valid, fetching the rows other ranks own.

        Collective: every rank of the group calls it, each with its own list.  The owner
        of a row sends the whole block row; the receiver keeps the blocks whose columns
        it holds."""
        import torch
        import torch.distributed as dist
        if X.complete:          # the same on every rank: all skip the collective together
            return
        need = np.asarray(need, dtype=np.int64)
        need = need[self.owners[self.held[need]] != self.rank]
        need = np.setdiff1d(need, X.halo)
        want = self.held[need]
        requests = [None] * self.nranks
        dist.all_gather_object(requests, want.tolist(), group=self.group)
        hp = self.pattern(X.R)
        bb = self.b * self.b
        recvs, sends = [], []
        for p in range(self.nranks):
            if p == self.rank:
                continue
            rows_in = want[self.owners[want] == p]
            if rows_in.size:
                n_in = int(np.sum(hp.gptr[rows_in + 1] - hp.gptr[rows_in])) * bb
                buf = torch.empty(n_in, dtype=torch.float64)
                recvs.append((rows_in, buf, dist.irecv(buf, src=p, group=self.group, tag=7)))
            rows_out = np.asarray(requests[p], dtype=np.int64)
            rows_out = rows_out[self.owners[rows_out] == self.rank]
            if rows_out.size:
                vals = engine.get_rows(X, self.g2l[rows_out])
                data = torch.from_numpy(np.ascontiguousarray(vals, dtype=np.float64).reshape(-1))
                sends.append((data, dist.isend(data, dst=p, group=self.group, tag=7)))
                self.sent_rows += int(rows_out.size)
        for rows_in, buf, req in recvs:
            req.wait()
            full = buf.numpy().reshape(-1, self.b, self.b)
            lrows = self.g2l[rows_in]
            # the held blocks of each received row: their offsets in the owner's full row,
            # shifted to where that row starts in the message
            glen = hp.gptr[rows_in + 1] - hp.gptr[rows_in]
            llen = hp.ptr[lrows + 1] - hp.ptr[lrows]
            shift = np.repeat(np.cumsum(glen) - glen - hp.gptr[rows_in], llen)
            pick = hp.gpos[row_blocks(hp.ptr, lrows)] + shift
            engine.set_rows(X, lrows, full[pick])
            self.received_rows += int(rows_in.size)
        for _, req in sends:
            req.wait()
        X.halo = np.union1d(X.halo, need)

    def allsum(self, values):
        """Sum of float64 values over the ranks of the group."""
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(v) for v in values], dtype=torch.float64)
        dist.all_reduce(t, group=self.group)
        return [float(v) for v in t.tolist()]


def cubic_step(c1, c2, c3):
    """Step a > 0 to the local minimum of c1 a + c2 a^2 + c3 a^3 along a descent direction
    (c1 < 0), or None.  Its derivative 3 c3 a^2 + 2 c2 a + c1 vanishes at
    a = -c1 / (c2 + sqrt(c2^2 - 3 c1 c3)), the root with positive curvature; with no real
    root but c2 > 0 the quadratic part's minimum -c1 / (2 c2) is taken."""
    disc = c2 * c2 - 3.0 * c1 * c3
    if disc >= 0.0:
        den = c2 + disc ** 0.5
        if den > 0.0:
            return -c1 / den
    if c2 > 0.0:
        return -c1 / (2.0 * c2)
    return None


class DistributedLnv:
    """Omega, N_e, the gradient and the line-search cubic of the LNV functional (Sec. 2.3.2,
    Eq. 8) with the rows spread over the ranks of `slabs`.

    K = 3 LSL - 2 LSLSL on H's range; Omega = spin Tr[K (H - mu S)], N_e = spin Tr[K S];
    G = spin (3 X - 2 Y)^T on L's range with X = SLH' + H'LS restricted to it and
    Y = SL SLH' + SL H'LS + H'LS LS, H' = H - mu S; L is symmetric and the search uses the
    symmetric part of G.  S and H are Mats on R_S and R_H holding every held row.
    """

    def __init__(self, slabs, engine, S, H, R_L, mu, spin=2.0):
        self.sl, self.en = slabs, engine
        self.R_L, self.R_H, self.mu, self.spin = float(R_L), H.R, float(mu), float(spin)
        self.S = S
        self.Hp = Mat(H.R, engine.lincomb([(1.0, H), (-self.mu, S)], H.R, rows="held"), complete=True)

    def _mm(self, A, B, R=None):
        """C = A.B on range R (default R_A + R_B), owned rows; B's halo fetched first."""
        self.sl.exchange(self.en, B, self.sl.reach(A.R))
        R = A.R + B.R if R is None else float(R)
        return Mat(R, self.en.matmul(A, B, R))

    def _comb(self, terms, R):
        return Mat(R, self.en.lincomb(terms, R))

    def _t(self, X, alpha=1.0):
        """alpha X^T on X's range; X's rows within the range's reach fetched first."""
        self.sl.exchange(self.en, X, self.sl.reach(X.R))
        return Mat(X.R, self.en.transpose(X, X.R, alpha))

    def energy(self, L):
        """(Omega, N_e) summed over the ranks."""
        LS = self._mm(L, self.S)
        SL = self._mm(self.S, L)
        LSL = self._mm(LS, L)
        LSLSL = self._mm(LSL, SL, self.R_H)
        K = self._comb([(3.0, LSL), (-2.0, LSLSL)], self.R_H)
        om, ne = self.sl.allsum([self.en.trace(K, self.Hp), self.en.trace(K, self.S)])
        return self.spin * om, self.spin * ne

    def gradient(self, L):
        """G = dOmega/dL on L's range (owned rows valid)."""
        LS = self._mm(L, self.S)
        SL = self._mm(self.S, L)
        SLH = self._mm(SL, self.Hp)
        HLS = self._mm(self.Hp, LS)
        Y1 = self._mm(SL, SLH, self.R_L)
        Y2 = self._mm(SL, HLS, self.R_L)
        Y3 = self._mm(HLS, LS, self.R_L)
        M = self._comb([(3.0, SLH), (3.0, HLS), (-2.0, Y1), (-2.0, Y2), (-2.0, Y3)], self.R_L)
        return self._t(M, self.spin)

    def symmetric(self, G):
        """(G + G^T) / 2."""
        return self._comb([(0.5, G), (1.0, self._t(G, 0.5))], G.R)

    def cubic(self, L, D, G):
        """(c1, c2, c3) of Omega(L + a D) - Omega(L) = c1 a + c2 a^2 + c3 a^3: c1 = <G, D>,
        c2 = spin (3 Tr[DSDH'] - 2 (Tr[DSDSLH'] + Tr[DSLSDH'] + Tr[LSDSDH'])),
        c3 = -2 spin Tr[DSDSDH'] (Eq. 8 expanded in a)."""
        LS = self._mm(L, self.S)
        DS = self._mm(D, self.S)
        DSD = self._mm(DS, D)
        DSDS = self._mm(DSD, self.S)
        DSLS = self._mm(DS, LS)
        LSDS = self._mm(LS, DS)
        tr = self.en.trace
        t = [tr(DSD, self.Hp),
             tr(self._mm(DSDS, L, self.R_H), self.Hp),
             tr(self._mm(DSLS, D, self.R_H), self.Hp),
             tr(self._mm(LSDS, D, self.R_H), self.Hp),
             tr(self._mm(DSDS, D, self.R_H), self.Hp),
             self.en.dot(G, D)]
        t2, t3a, t3b, t3c, t4, c1 = self.sl.allsum(t)
        return c1, self.spin * (3.0 * t2 - 2.0 * (t3a + t3b + t3c)), -2.0 * self.spin * t4

    def minimise(self, L, n_iter, reset=40):
        """Polak-Ribiere CG with the exact cubic line minimum, beta = max(0, beta_PR), the
        direction reset to -G every `reset` steps or when it is not a descent direction.
        Returns (L, history) with Omega, N_e, alpha and beta of each step."""
        D = Gp = None
        hist = []
        for it in range(n_iter):
            om, ne = self.energy(L)
            G = self.symmetric(self.gradient(L))
            beta = 0.0
            if D is None or it % reset == 0:
                D = self._comb([(-1.0, G)], G.R)
            else:
                num, den = self.sl.allsum([self.en.dot(G, G) - self.en.dot(G, Gp), self.en.dot(Gp, Gp)])
                beta = max(0.0, num / den)
                D = self._comb([(-1.0, G), (beta, D)], G.R)
            c1, c2, c3 = self.cubic(L, D, G)
            if c1 >= 0.0:
                D = self._comb([(-1.0, G)], G.R)
                beta = 0.0
                c1, c2, c3 = self.cubic(L, D, G)
            a = cubic_step(c1, c2, c3)
            if a is None:
                raise FloatingPointError("no local minimum along the search direction")
            L = self._comb([(1.0, L), (a, D)], L.R)
            hist.append(dict(omega=om, ne=ne, alpha=a, beta=beta,
                             omega_next=om + c1 * a + c2 * a * a + c3 * a * a * a))
            Gp = G
        return L, hist


class GpuEngine:
    """The block algebra of DistributedLnv on this rank's GPU, with this library's calls in
    float64 on a geometry of the held atoms (same cell, every range of the decomposition
    and a self-only range for the unit and owner matrices).

    Restrictions and linear combinations are products with the unit block matrix I
    (C = alpha I.X + beta C on C's range); a trace or a dot over the owned rows is one of
    Tr[(P X) Y] or Tr[(P X) Y^T], with P the unit blocks on the owned rows and zero blocks
    elsewhere.  Halo rows are packed and unpacked by indexing the block arrays.
    """

    def __init__(self, slabs, stream=None, r_self=0.1):
        import torch
        from . import Geometry
        self.sl, self.b, self.stream = slabs, slabs.b, stream
        self.ranges = list(slabs.ranges) + [float(r_self)]
        self.geom = Geometry(torch.from_numpy(slabs.pos), slabs.cell, self.ranges, stream=stream)
        for r, R in enumerate(slabs.ranges):
            rp, col = self.geom.pattern(r, stream=stream)
            hp = slabs.pats[R]
            if not (np.array_equal(rp.cpu().numpy(), hp.ptr)
                    and np.array_equal(col.cpu().numpy().astype(np.int64), hp.col.astype(np.int64))):
                raise ValueError("the held atoms' pattern of range %g differs from the restricted "
                                 "global pattern" % R)
        n = slabs.pos.shape[0]
        self.r0 = len(self.ranges) - 1
        if self.geom.nnzb(self.r0) != n:
            raise ValueError("r_self %g reaches another atom" % r_self)
        eye = torch.eye(self.b, dtype=torch.float64).expand(n, self.b, self.b)
        self.I = eye.contiguous().view(-1).cuda()
        P = torch.zeros(n, self.b, self.b, dtype=torch.float64)
        P[torch.from_numpy(slabs.own)] = torch.eye(self.b, dtype=torch.float64)
        self.P = P.view(-1).cuda()

    def _rid(self, R):
        hp = self.sl.pattern(R)
        return self.sl.ranges.index(hp.R)

    def new(self, R):
        import torch
        return torch.zeros(self.sl.pattern(R).nnzb * self.b * self.b, dtype=torch.float64, device="cuda")

    def from_global(self, R, gvals):
        """Held blocks of a matrix given by its global blocks [nnzb, b, b] on range R."""
        import torch
        hp = self.sl.pattern(R)
        v = np.ascontiguousarray(np.asarray(gvals, dtype=np.float64).reshape(-1, self.b, self.b)[hp.gpos])
        return torch.from_numpy(v).view(-1).cuda()

    def to_host(self, X):
        """Held blocks of X as float64 [nnzb_held, b, b]."""
        return X.data.view(-1, self.b, self.b).cpu().numpy()

    def matmul(self, A, B, R):
        from . import block_matmul, F64
        C = self.new(R)
        block_matmul(self.geom, self.b, A.data, self._rid(A.R), B.data, self._rid(B.R), C, self._rid(R),
                     precision=F64, stream=self.stream)
        return C

    def lincomb(self, terms, R, rows=None):
        from . import block_matmul, F64
        C = self.new(R)
        for k, (c, X) in enumerate(terms):
            block_matmul(self.geom, self.b, self.I, self.r0, X.data, self._rid(X.R), C, self._rid(R),
                         precision=F64, alpha=float(c), beta=0.0 if k == 0 else 1.0, stream=self.stream)
        return C

    def transpose(self, X, R, alpha=1.0):
        from . import transpose, F64
        out = self.new(R)
        transpose(self.geom, self.b, X.data, self._rid(X.R), out, self._rid(R), alpha=float(alpha),
                  precision=F64, stream=self.stream)
        return out

    def _owned(self, X):
        from . import block_matmul, F64
        Xo = self.new(X.R)
        block_matmul(self.geom, self.b, self.P, self.r0, X.data, self._rid(X.R), Xo, self._rid(X.R),
                     precision=F64, stream=self.stream)
        return Xo

    def trace(self, X, Y):
        from . import trace, F64
        return trace(self.geom, self.b, self._owned(X), self._rid(X.R), Y.data, self._rid(Y.R),
                     precision=F64, stream=self.stream)

    def dot(self, X, Y):
        from . import trace, F64
        Yt = self.transpose(Y, Y.R)
        return trace(self.geom, self.b, self._owned(X), self._rid(X.R), Yt, self._rid(Y.R),
                     precision=F64, stream=self.stream)

    def _blocks(self, R, rows):
        import torch
        return torch.from_numpy(row_blocks(self.sl.pattern(R).ptr, rows)).cuda()

    def get_rows(self, X, rows):
        return X.data.view(-1, self.b, self.b)[self._blocks(X.R, rows)].cpu().numpy()

    def set_rows(self, X, rows, blocks):
        import torch
        X.data.view(-1, self.b, self.b)[self._blocks(X.R, rows)] = \
            torch.from_numpy(np.ascontiguousarray(blocks, dtype=np.float64)).cuda()
