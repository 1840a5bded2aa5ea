"""Diamond-silicon supercells and a two-centre Slater-Koster sp3 model.

The paper's systems are bulk crystalline Si (Sec. 4.2, the O(N) scaling
runs) described in a basis of localised support functions, so that H and
S are matrices of atom blocks H_{i alpha, j beta} (Sec. 2.2, Eqs. 1-2).
Here H and S come from a textbook two-centre Slater-Koster table instead
of DFT integrals; the values are the ones the workload defines.

Units: Angstrom and eV.  Blocks are row-major [b, b]; the row index is
the orbital on atom i, the column index the orbital on atom j; orbital
order (s, px, py, pz).  For b = 13 the first 12 orbitals are three copies
of (s, px, py, pz) and the 13th is a d-like orbital with no off-site
coupling.
"""
import numpy as np

A_SI = 5.431            # conventional-cell lattice constant, Angstrom
R0 = 2.35               # reference bond length of the scaling laws
RC = 6.6                # radius where the smooth cutoff reaches zero
RC_INNER = 5.6          # start of the cosine taper
SEED_BASE = 2002077040

# Hamiltonian: on-site energies and two-centre integrals at r = R0 (eV)
SK_H = dict(Es=-5.25, Ep=1.20, sss=-1.94, sps=1.75, pps=3.05, ppp=-1.08)
# Overlap integrals at r = R0
SK_S = dict(sss=0.10, sps=-0.08, pps=-0.12, ppp=0.04)
D_ONSITE = 8.0          # on-site energy of the 13th orbital (eV)

_FCC = np.array([[0.0, 0.0, 0.0], [0.0, 0.5, 0.5], [0.5, 0.0, 0.5], [0.5, 0.5, 0.0]])
_BASIS = np.concatenate([_FCC, _FCC + 0.25])   # 8 atoms per conventional cell


def config_seed(k):
    """Seed of configuration k of the Si workloads."""
    return SEED_BASE + k


def batch_system_seed(s):
    """Seed of system s of the batched workload."""
    return SEED_BASE + 100 + s


def batch_workload(n_sys=48, n_min=2, n_max=7):
    """The batched workload: n_sys uneven diamond-Si systems.

    System s has n_s x n_s x n_s conventional cells with n_s uniform in
    [n_min, n_max] (64 to 2744 atoms), displacement sigma_s uniform in
    [0.05, 0.15] Angstrom (both drawn once from configuration seed 2), and
    positions seeded by batch_system_seed(s).  The first half of the
    systems uses 4 x 4 blocks, the second half the 13-orbital model with its
    symmetric H perturbation seeded by batch_system_seed(s) + 7.
    Returns a list of dicts (n, sigma, seed, b, perturb_seed).
    """
    rng = np.random.default_rng(config_seed(2))
    ns = rng.integers(n_min, n_max + 1, size=n_sys)
    sig = rng.uniform(0.05, 0.15, size=n_sys)
    out = []
    for s in range(n_sys):
        b = 4 if s < n_sys // 2 else 13
        out.append(dict(n=int(ns[s]), sigma=float(sig[s]), seed=batch_system_seed(s), b=b,
                        perturb_seed=(batch_system_seed(s) + 7) if b == 13 else None))
    return out


def diamond_si_positions(n, sigma, seed, a=A_SI):
    """n x n x n conventional cells of diamond Si with Gaussian displacements;
    n = (nx, ny, nz) gives an orthorhombic box of nx x ny x nz cells.

    Returns (pos [8 nx ny nz, 3] float64 wrapped into [0, L), cell [3] float64).
    Atoms are ordered cell by cell (ix slowest, then iy, iz) and within a
    cell by the 8 basis sites, so consecutive indices are spatially close.
    """
    shape = (int(n),) * 3 if np.isscalar(n) else tuple(int(v) for v in n)
    axes = [np.arange(m) for m in shape]
    cells = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, 3)
    frac = (cells[:, None, :] + _BASIS[None, :, :]).reshape(-1, 3)
    L = np.array(shape, dtype=np.float64) * a
    pos = frac * a
    rng = np.random.default_rng(seed)
    pos = pos + rng.normal(0.0, sigma, size=pos.shape)
    pos = np.mod(pos, L)
    pos = np.where(pos >= L, pos - L, pos)
    pos[pos < 0.0] = 0.0
    cell = np.ascontiguousarray(L)
    return np.ascontiguousarray(pos, dtype=np.float64), cell


def md_trajectory(pos0, cell, n_steps, seed, amp=0.05, period=(20.0, 40.0)):
    """A prescribed atomic motion standing in for a molecular-dynamics run of the crystal.

    Every atom oscillates about its starting position:
    r_i(t_n) = r_i(0) + u_i sin(2 pi n / T_i + phi_i), with a seeded direction
    and amplitude u_i (Gaussian components of standard deviation amp,
    Angstrom), a period T_i uniform in `period` (steps) and a phase phi_i
    uniform in [0, 2 pi).  With amp = 0.05 A and periods of 20-40 steps
    an atom moves ~0.01 A per step, the scale of a 1 fs step of Si at room
    temperature.  Returns [n_steps + 1, N, 3] float64, wrapped into the cell.
    """
    pos0 = np.asarray(pos0, dtype=np.float64)
    rng = np.random.default_rng(seed)
    n = pos0.shape[0]
    u = rng.normal(0.0, amp, size=(n, 3))
    T = rng.uniform(period[0], period[1], size=n)
    phi = rng.uniform(0.0, 2.0 * np.pi, size=n)
    L = np.asarray(cell, dtype=np.float64)
    out = np.empty((n_steps + 1, n, 3))
    for k in range(n_steps + 1):
        p = pos0 + u * np.sin(2.0 * np.pi * k / T + phi)[:, None]
        p = np.mod(p, L)
        p[p >= L] -= L[np.nonzero(p >= L)[1]]
        p[p < 0.0] = 0.0
        out[k] = p
    return out


def _cutoff(r):
    """Smooth cutoff: 1 below 5.6, cosine taper to 0 at 6.6, 0 beyond."""
    f = np.where(r <= RC_INNER, 1.0, 0.5 * (1.0 + np.cos(np.pi * (r - RC_INNER) / (RC - RC_INNER))))
    return np.where(r >= RC, 0.0, f)


def _sk_sp_blocks(vec, p):
    """Two-centre sp3 blocks [m, 4, 4] for bond vectors vec [m, 3] (i -> j).

    p holds (sss, sps, pps, ppp) already scaled to each bond length, each [m].
    """
    r = np.sqrt(np.sum(vec * vec, axis=1))
    c = vec / r[:, None]                      # direction cosines l, m, n
    m = vec.shape[0]
    blk = np.empty((m, 4, 4))
    blk[:, 0, 0] = p["sss"]
    blk[:, 0, 1:] = c * p["sps"][:, None]
    blk[:, 1:, 0] = -c * p["sps"][:, None]
    cc = c[:, :, None] * c[:, None, :]
    eye = np.eye(3)[None]
    blk[:, 1:, 1:] = cc * (p["pps"] - p["ppp"])[:, None, None] + eye * p["ppp"][:, None, None]
    return blk


def _image_vectors(pos, cell, rows, cols):
    """All bond vectors r_j - r_i + T with |.| < RC, over lattice translations T.

    Returns (pair index [m], vectors [m, 3]).  The self term T = 0, i = j
    is excluded (it is the on-site block).
    """
    d = pos[cols] - pos[rows]
    d = d - cell * np.rint(d / cell)           # nearest image first
    reach = [int(np.ceil(RC / L + 0.5)) for L in cell]
    shifts = np.array([[x, y, z] for x in range(-reach[0], reach[0] + 1)
                       for y in range(-reach[1], reach[1] + 1)
                       for z in range(-reach[2], reach[2] + 1)], dtype=np.float64) * cell
    out_p, out_v = [], []
    for t in shifts:
        v = d + t
        r2 = np.sum(v * v, axis=1)
        keep = (r2 < RC * RC) & (r2 > 1e-12)
        if np.any(keep):
            out_p.append(np.nonzero(keep)[0])
            out_v.append(v[keep])
    if not out_p:
        return np.zeros(0, dtype=np.int64), np.zeros((0, 3))
    return np.concatenate(out_p), np.concatenate(out_v)


def sk_blocks(pos, cell, rows, cols, b=4, perturb_seed=None):
    """H and S blocks for the listed atom pairs (i = rows[p], j = cols[p]).

    Every periodic image of atom j within RC of atom i contributes (a
    Gamma-point, image-summed block); pairs with no image inside RC get
    zero off-site blocks.  Diagonal pairs (i == i) carry the on-site
    terms.  The pair list must be symmetric when perturb_seed is given
    (b = 13), because the random perturbation is mirrored to (j, i).

    Returns (H [npair, b, b], S [npair, b, b]) float64.
    """
    pos = np.asarray(pos, dtype=np.float64)
    cell = np.asarray(cell, dtype=np.float64)
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    npair = rows.shape[0]
    H4 = np.zeros((npair, 4, 4))
    S4 = np.zeros((npair, 4, 4))
    pidx, vec = _image_vectors(pos, cell, rows, cols)
    if pidx.size:
        r = np.sqrt(np.sum(vec * vec, axis=1))
        fc = _cutoff(r)
        sh = (R0 / r) ** 2 * fc
        ss = np.exp(-2.0 * (r / R0 - 1.0)) * fc
        ph = {k: SK_H[k] * sh for k in ("sss", "sps", "pps", "ppp")}
        ps = {k: SK_S[k] * ss for k in ("sss", "sps", "pps", "ppp")}
        np.add.at(H4, pidx, _sk_sp_blocks(vec, ph))
        np.add.at(S4, pidx, _sk_sp_blocks(vec, ps))
    diag = rows == cols
    H4[diag] += np.diag([SK_H["Es"], SK_H["Ep"], SK_H["Ep"], SK_H["Ep"]])
    S4[diag] += np.eye(4)
    H4 = _mirror_average(H4, rows, cols)
    S4 = _mirror_average(S4, rows, cols)
    if b == 4:
        return H4, S4
    if b != 13:
        raise ValueError("b must be 4 or 13")
    H = np.zeros((npair, 13, 13))
    S = np.zeros((npair, 13, 13))
    for c in range(3):
        H[:, 4 * c:4 * c + 4, 4 * c:4 * c + 4] = H4
        S[:, 4 * c:4 * c + 4, 4 * c:4 * c + 4] = S4
    H[diag, 12, 12] = D_ONSITE
    S[diag, 12, 12] = 1.0
    if perturb_seed is not None:
        H += _symmetric_perturbation(rows, cols, perturb_seed)
    return H, S


def _mirror_average(X, rows, cols):
    """(X_ij + X_ji^T) / 2 wherever the pair list holds both (i, j) and (j, i).

    The image sums for (i, j) and (j, i) run in different orders; averaging
    makes the matrix symmetric to the last bit.
    """
    n = int(max(rows.max(initial=-1), cols.max(initial=-1))) + 1
    key = rows * n + cols
    order = np.argsort(key)
    mkey = cols * n + rows
    pos = np.searchsorted(key[order], mkey)
    pos = np.minimum(pos, key.size - 1)
    found = key[order][pos] == mkey if key.size else np.zeros(0, bool)
    mirror = order[pos]
    out = X.copy()
    idx = np.nonzero(found)[0]
    out[idx] = 0.5 * (X[idx] + np.transpose(X[mirror[idx]], (0, 2, 1)))
    return out


def _symmetric_perturbation(rows, cols, seed, amp=0.1, b=13):
    """Uniform [-amp, amp] eV on every stored block, mirrored so H stays symmetric.

    Draws, in the order of the pair list, one b x b block for every pair
    with i < j and the upper triangle of every diagonal block.
    """
    npair = rows.shape[0]
    key = {(int(i), int(j)): p for p, (i, j) in enumerate(zip(rows, cols))}
    out = np.zeros((npair, b, b))
    rng = np.random.default_rng(seed)
    iu = np.triu_indices(b)
    for p in range(npair):
        i, j = int(rows[p]), int(cols[p])
        if i < j:
            q = key.get((j, i))
            if q is None:
                raise ValueError("pair list is not symmetric")
            e = rng.uniform(-amp, amp, size=(b, b))
            out[p] = e
            out[q] = e.T
        elif i == j:
            e = np.zeros((b, b))
            e[iu] = rng.uniform(-amp, amp, size=iu[0].size)
            out[p] = e + np.triu(e, 1).T
    return out
