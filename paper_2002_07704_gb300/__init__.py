"""GB300-native linear-scaling density-matrix minimisation (LNV).

Thin Python binding of ``liblsq.so``, whose C ABI is declared in
``include/lsq.h``.  This module only marshals arguments: every step of
the computation (range patterns, truncated atom-block products, traces,
the gradient and the conjugate-gradient minimisation) runs in the
library's CUDA kernels.  PyTorch supplies device memory and streams.

There is no CPU fallback: if the library is not built, or no CUDA device
is present, the calls raise.
"""
import ctypes
import os

from ._build import LIB, build  # noqa: F401

F64 = 0
F32 = 1
TF32X3 = 2   # float32 storage, 4 x 4 blocks on the tensor cores in split TF32
HARTREE_EV = 27.211386245988

ERRORS = {1: "INVALID_ARG", 2: "PATTERN", 3: "OOM", 4: "CUDA", 5: "UNSTABLE",
          6: "NOT_CONVERGED", 7: "UNSUPPORTED", 8: "TIMEOUT"}

_lib = None


class LsqError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("lsq error %d (%s): %s" % (code, ERRORS.get(code, "?"), msg))
        self.code = code


class LnvOpts(ctypes.Structure):
    _fields_ = [("max_iter", ctypes.c_int), ("tol_ha_per_atom", ctypes.c_double),
                ("cg_reset", ctypes.c_int), ("precision", ctypes.c_int),
                ("refine_iter", ctypes.c_int), ("spin", ctypes.c_double),
                ("final_eval", ctypes.c_int), ("verbose", ctypes.c_int), ("graph", ctypes.c_int)]


class LnvReport(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("iterations_fp64", ctypes.c_int),
                ("status", ctypes.c_int), ("omega_ev", ctypes.c_double), ("ne", ctypes.c_double),
                ("omega_ha_per_atom", ctypes.c_double),
                ("last_domega_ha_per_atom", ctypes.c_double), ("seconds", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


def library_path():
    return LIB


def load():
    """Loads liblsq.so (built by build()); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB):
        raise RuntimeError("liblsq.so is not built; call paper_2002_07704_gb300.build()")
    lib = ctypes.CDLL(LIB)
    P, I, D, L64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_int64
    sig = {
        "lsq_last_error": (I, [ctypes.c_char_p, ctypes.c_size_t]),
        "lsq_version": (I, []),
        "lsq_launch_count": (I, [P]),
        "lsq_build_neighbour_lists": (I, [P, I, P, P, I, P, P]),
        "lsq_geom_destroy": (I, [P]),
        "lsq_geom_info": (I, [P, P, P]),
        "lsq_geom_concat": (I, [I, P, P, P]),
        "lsq_geom_systems": (I, [P, P, P]),
        "lsq_pattern": (I, [P, I, P, P, P]),
        "lsq_pattern_copy": (I, [P, I, P, P, P]),
        "lsq_block_matmul": (I, [P, I, I, I, I, P, I, I, P, I, P, D, D, P, P]),
        "lsq_block_matmul_tri": (I, [P, I, I, I, I, P, I, I, P, I, P, D, D, I, P, P]),
        "lsq_trace": (I, [P, I, I, I, P, I, P, P, P]),
        "lsq_transpose": (I, [P, I, I, I, P, I, P, D, P]),
        "lsq_trace_static": (I, [P, I, I, I, P, I, P, P, P]),
        "lsq_hotelling_inverse": (I, [P, I, I, I, P, I, I, P, I, I, P, P]),
        "lsq_lnv_default_opts": (I, [P]),
        "lsq_lnv_required_ranges": (I, [D, D, D, P]),
        "lsq_lnv_create": (I, [P, I, D, D, D, P]),
        "lsq_lnv_destroy": (I, [P]),
        "lsq_lnv_init_L": (I, [P, P, P, P]),
        "lsq_lnv_energy_gradient": (I, [P, P, P, P, D, D, I, P, P, P, P]),
        "lsq_lnv_minimise": (I, [P, P, P, P, D, P, P, P]),
        "lsq_lnv_minimise_batch": (I, [P, P, P, P, P, P, P, P]),
        "lsq_lnv_minimise_batch_group": (I, [I, P, P, P, P, P, P, P, P]),
        "lsq_lnv_set_metric": (I, [P, I, P, I, P]),
        "lsq_lnv_init_purify": (I, [P, P, P, D, I, P, I, I, I, P, P, P]),
        "lsq_lnv_minimise_canonical": (I, [P, P, P, P, D, P, P, P, P]),
        "lsq_lnv_minimise_batch_canonical": (I, [P, P, P, P, P, P, P, P, P]),
        "lsq_pattern_remap": (I, [P, I, P, I, I, I, P, P, P]),
        "lsq_geom_adopt_schedules": (I, [P, P]),
        "lsq_xl_propagate": (I, [P, I, I, I, P, P, D, D, P, I, P, P]),
        "lsq_xl_initial_L": (I, [P, I, I, I, P, I, P, I, P, P]),
        "lsq_device_status": (I, [P, P]),
        "lsq_measure_peak": (I, [I, P, P]),
        "lsq_product_plan_info": (I, [P, I, I, I, I, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    del L64
    _lib = lib
    return lib


def exported_symbols():
    """Names of the C entry points this binding declares."""
    return ["lsq_last_error", "lsq_version", "lsq_launch_count", "lsq_build_neighbour_lists", "lsq_geom_destroy",
            "lsq_geom_info", "lsq_geom_concat", "lsq_geom_systems", "lsq_pattern", "lsq_pattern_copy", "lsq_block_matmul", "lsq_block_matmul_tri", "lsq_trace", "lsq_transpose",
            "lsq_trace_static", "lsq_hotelling_inverse",
            "lsq_lnv_default_opts", "lsq_lnv_required_ranges", "lsq_lnv_create",
            "lsq_lnv_destroy", "lsq_lnv_init_L", "lsq_lnv_energy_gradient", "lsq_lnv_minimise",
            "lsq_lnv_minimise_batch", "lsq_lnv_minimise_batch_group", "lsq_lnv_set_metric", "lsq_lnv_init_purify",
            "lsq_lnv_minimise_canonical", "lsq_lnv_minimise_batch_canonical", "lsq_pattern_remap", "lsq_xl_propagate", "lsq_xl_initial_L",
            "lsq_geom_adopt_schedules", "lsq_device_status", "lsq_measure_peak", "lsq_product_plan_info"]


def measure_peak(precision=F32, stream=None):
    """Measured FMA rate of the current GPU in TFLOP/s (lsq_measure_peak)."""
    t = ctypes.c_double()
    _check(load().lsq_measure_peak(int(precision), ctypes.byref(t), _stream(stream)))
    return t.value


def launch_count():
    """Kernels launched by the library so far in this process."""
    n = ctypes.c_int64()
    _check(load().lsq_launch_count(ctypes.byref(n)))
    return n.value


def _check(rc):
    if rc != 0:
        buf = ctypes.create_string_buffer(512)
        _lib.lsq_last_error(buf, 512)
        raise LsqError(rc, buf.value.decode(errors="replace"))


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _dev(t, dtype=None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return ctypes.c_void_p(t.data_ptr())


def _need(t, geom, r, b, name):
    """Raises LsqError(INVALID_ARG) unless t holds the nnzb(r) b x b blocks of range r of geom
    (a short array would be written or read out of bounds on the device)."""
    if t is None:
        return
    n = geom.nnzb(r) * b * b
    if t.numel() != n:
        raise LsqError(1, "%s has %d values; range %d of the geometry holds %d blocks of %d x %d (%d values)"
                       % (name, t.numel(), r, geom.nnzb(r), b, b, n))


def _darr(vals):
    vals = [float(v) for v in vals]
    return (ctypes.c_double * len(vals))(*vals)


class Geometry:
    """Range patterns of one atomic geometry (lsq_build_neighbour_lists)."""

    def __init__(self, pos, cell, ranges, stream=None):
        import torch
        lib = load()
        pos = pos.to(device="cuda", dtype=torch.float64).contiguous()
        self.ranges = [float(r) for r in ranges]
        self.cell = [float(c) for c in cell]
        h = ctypes.c_void_p()
        _check(lib.lsq_build_neighbour_lists(_dev(pos), pos.shape[0], _darr(self.cell),
                                             _darr(self.ranges), len(self.ranges),
                                             ctypes.byref(h), _stream(stream)))
        self.handle = h
        self.n_atoms = int(pos.shape[0])

    @classmethod
    def _from_handle(cls, handle, n_atoms, ranges):
        self = cls.__new__(cls)
        self.handle = handle
        self.n_atoms = int(n_atoms)
        self.ranges = list(ranges)
        self.cell = None
        return self

    def systems(self):
        """Atom offsets of the systems held by this geometry ([n_sys + 1])."""
        n = ctypes.c_int()
        _check(_lib.lsq_geom_systems(self.handle, ctypes.byref(n), None))
        off = (ctypes.c_int64 * (n.value + 1))()
        _check(_lib.lsq_geom_systems(self.handle, ctypes.byref(n), off))
        return list(off)

    def range_id(self, R):
        return self.ranges.index(float(R))

    def nnzb(self, r):
        n = ctypes.c_int64()
        _check(_lib.lsq_pattern(self.handle, r, None, None, ctypes.byref(n)))
        return n.value

    def pattern(self, r, stream=None):
        """(row_ptr int64 [n+1], col int32 [nnzb]) as new CUDA tensors."""
        import torch
        nnzb = self.nnzb(r)
        rp = torch.empty(self.n_atoms + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(nnzb, 1), dtype=torch.int32, device="cuda")
        _check(_lib.lsq_pattern_copy(self.handle, r, _dev(rp), _dev(col), _stream(stream)))
        return rp, col[:nnzb]

    def device_status(self, stream=None):
        """Raises LsqError(TIMEOUT) if a kernel with bounded waits gave up since the last check."""
        _check(load().lsq_device_status(self.handle, _stream(stream)))

    def product_plan_info(self, range_a, range_b, range_c, triangle=0):
        """Statistics of the tensor-core plan of a product already run (lsq_product_plan_info)."""
        out = (ctypes.c_int64 * 6)()
        _check(load().lsq_product_plan_info(self.handle, range_a, range_b, range_c, triangle, out))
        return {"triples": out[0], "dense_triples": out[1], "block_slots": out[2], "tiles": out[3],
                "auto_choice": out[4], "blocks_copied": out[5]}

    def adopt_schedules(self, other):
        """Use the product schedules tuned in another geometry of the same ranges."""
        _check(load().lsq_geom_adopt_schedules(self.handle, other.handle))

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.lsq_geom_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def build_neighbour_lists(pos, cell, ranges, stream=None):
    return Geometry(pos, cell, ranges, stream)


def concat_geometries(geoms, stream=None):
    """One block-diagonal geometry holding independent systems (lsq_geom_concat)."""
    arr = (ctypes.c_void_p * len(geoms))(*[g.handle.value for g in geoms])
    h = ctypes.c_void_p()
    _check(load().lsq_geom_concat(len(geoms), arr, ctypes.byref(h), _stream(stream)))
    g = Geometry._from_handle(h, sum(x.n_atoms for x in geoms), geoms[0].ranges)
    g.parts = list(geoms)
    return g


def block_matmul(geom, b, A, range_a, B, range_b, C, range_c, precision=F64, trans_a=False,
                 trans_b=False, alpha=1.0, beta=0.0, stream=None, triangle=0):
    """C = alpha op(A) op(B) + beta C on C's range pattern; returns the triple count.

    triangle: 0 every block; 1 symmetric result (upper blocks computed, lower ones
    mirrored); 2 only blocks with j >= i; 3 only blocks with j <= i.
    """
    import torch
    dt = torch.float64 if precision == F64 else torch.float32
    _need(A, geom, range_a, b, "A")
    _need(B, geom, range_b, b, "B")
    _need(C, geom, range_c, b, "C")
    nt = ctypes.c_int64()
    if triangle:
        _check(load().lsq_block_matmul_tri(geom.handle, b, precision, range_a, int(trans_a),
                                           _dev(A, dt), range_b, int(trans_b), _dev(B, dt), range_c,
                                           _dev(C, dt), float(alpha), float(beta), int(triangle),
                                           ctypes.byref(nt), _stream(stream)))
    else:
        _check(load().lsq_block_matmul(geom.handle, b, precision, range_a, int(trans_a), _dev(A, dt),
                                       range_b, int(trans_b), _dev(B, dt), range_c, _dev(C, dt),
                                       float(alpha), float(beta), ctypes.byref(nt), _stream(stream)))
    return nt.value


# A dissipation set (kappa, alpha, c_0..c_5) for lsq_xl_propagate: the K = 5 entry of the
# table of Niklasson et al., J. Chem. Phys. 130, 214109 (2009), the scheme the paper cites
# for its dissipative term (sum c_m = sum m c_m = 0).
XL_DISSIPATION_K5 = (1.82, 0.018, (-6.0, 14.0, -8.0, -3.0, 4.0, -1.0))


def pattern_remap(geom_from, range_from, geom_to, range_to, b, X_from, X_to, precision=F64, stream=None):
    """X_to (on geom_to's range_to) = X_from (on geom_from's range_from) matched by atom pair."""
    import torch
    dt = torch.float64 if precision == F64 else torch.float32
    _need(X_from, geom_from, range_from, b, "X_from")
    _need(X_to, geom_to, range_to, b, "X_to")
    _check(load().lsq_pattern_remap(geom_from.handle, range_from, geom_to.handle, range_to, b, precision,
                                    _dev(X_from, dt), _dev(X_to, dt), _stream(stream)))


def xl_propagate(geom, b, range_x, X_hist, LS, X_next, kappa, alpha=0.0, c=None, stream=None):
    """X_next = 2 X(t) - X(t-dt) + kappa (LS - X(t)) + alpha sum_m c_m X(t - m dt).

    X_hist: [X(t), X(t-dt), ...] (float64 tensors on range_x); X_next may be one of them.
    """
    import torch
    for k, x in enumerate(X_hist):
        _need(x, geom, range_x, b, "X_hist[%d]" % k)
    _need(LS, geom, range_x, b, "LS")
    _need(X_next, geom, range_x, b, "X_next")
    ptrs = (ctypes.c_void_p * len(X_hist))(*[_dev(x, torch.float64) for x in X_hist])
    nc = 0 if c is None else len(c)
    carr = (ctypes.c_double * max(nc, 1))(*([float(v) for v in c] if c is not None else [0.0]))
    _check(load().lsq_xl_propagate(geom.handle, b, range_x, len(X_hist), ptrs, _dev(LS, torch.float64),
                                   float(kappa), float(alpha), carr if nc else None, nc,
                                   _dev(X_next, torch.float64), _stream(stream)))


def xl_initial_L(geom, b, range_x, X, range_sinv, Sinv, range_l, L_out, precision=F64, stream=None):
    """L_out = symmetric part of (X Sinv) on range_l (the MD step's initial L)."""
    import torch
    _need(X, geom, range_x, b, "X")
    _need(Sinv, geom, range_sinv, b, "Sinv")
    _need(L_out, geom, range_l, b, "L_out")
    _check(load().lsq_xl_initial_L(geom.handle, b, precision, range_x, _dev(X, torch.float64), range_sinv,
                                   _dev(Sinv, torch.float64), range_l, _dev(L_out, torch.float64),
                                   _stream(stream)))


def trace(geom, b, X, range_x, Y, range_y, precision=F64, stream=None):
    import torch
    dt = torch.float64 if precision == F64 else torch.float32
    _need(X, geom, range_x, b, "X")
    _need(Y, geom, range_y, b, "Y")
    out = ctypes.c_double()
    _check(load().lsq_trace(geom.handle, b, precision, range_x, _dev(X, dt), range_y, _dev(Y, dt),
                            ctypes.byref(out), _stream(stream)))
    return out.value


def transpose(geom, b, X, range_x, out, range_out, alpha=1.0, precision=F64, stream=None):
    """out = alpha X^T on pattern range_out (zero where X has no (j, i) block)."""
    import torch
    dt = torch.float64 if precision == F64 else torch.float32
    _need(X, geom, range_x, b, "X")
    _need(out, geom, range_out, b, "out")
    _check(load().lsq_transpose(geom.handle, b, precision, range_x, _dev(X, dt), range_out,
                                _dev(out, dt), float(alpha), _stream(stream)))


def trace_static(geom, b, X, range_x, Y, range_y, out, precision=F64, stream=None):
    """Tr[X Y] into the one-element float64 CUDA tensor `out`, allocating no device memory.

    For callers that cannot let the library call cudaMalloc (all device
    memory owned by their own pool, or no device stalls allowed).  At most
    262144 atoms; concurrent calls on unordered streams race (they share
    one fixed scratch array).  Enqueued on the stream; does not synchronise.
    """
    import torch
    dt = torch.float64 if precision == F64 else torch.float32
    _need(X, geom, range_x, b, "X")
    _need(Y, geom, range_y, b, "Y")
    if out is None or out.numel() != 1:
        raise LsqError(1, "out must be a one-element float64 tensor")
    _check(load().lsq_trace_static(geom.handle, b, precision, range_x, _dev(X, dt), range_y,
                                   _dev(Y, dt), _dev(out, torch.float64), _stream(stream)))


def hotelling_inverse(geom, b, S, range_s, X, range_x, range_xs, n_iter, precision=F64, start=True,
                      stream=None):
    """Approximate sparse inverse of S on range_x by the Hotelling iteration (in place in X).

    Returns the list of |X_{n+1} - X_n|_F (one per step).  See lsq_hotelling_inverse.
    """
    import torch
    _need(S, geom, range_s, b, "S")
    _need(X, geom, range_x, b, "X")
    dx = (ctypes.c_double * max(int(n_iter), 1))()
    _check(load().lsq_hotelling_inverse(geom.handle, b, precision, range_s, _dev(S, torch.float64),
                                        range_x, range_xs, _dev(X, torch.float64), int(bool(start)),
                                        int(n_iter), dx, _stream(stream)))
    return [dx[k] for k in range(int(n_iter))]


def lnv_required_ranges(R_S, R_H, R_L):
    out = (ctypes.c_double * 6)()
    _check(load().lsq_lnv_required_ranges(float(R_S), float(R_H), float(R_L), out))
    return list(out)


class Lnv:
    """LNV context: workspace for the products of one CG step (lsq_lnv_create)."""

    def __init__(self, geom, b, R_S, R_H, R_L):
        h = ctypes.c_void_p()
        _check(load().lsq_lnv_create(geom.handle, b, float(R_S), float(R_H), float(R_L),
                                     ctypes.byref(h)))
        self.handle = h
        self.geom = geom
        self.b = b
        self.rS, self.rH, self.rL = geom.range_id(R_S), geom.range_id(R_H), geom.range_id(R_L)

    def _need_lsh(self, L=None, S=None, H=None, G=None):
        for t, r, name in ((L, self.rL, "L"), (S, self.rS, "S"), (H, self.rH, "H"), (G, self.rL, "G")):
            _need(t, self.geom, r, self.b, name)

    def init_L(self, S, L, stream=None):
        import torch
        self._need_lsh(L=L, S=S)
        _check(_lib.lsq_lnv_init_L(self.handle, _dev(S, torch.float64), _dev(L, torch.float64),
                                   _stream(stream)))

    def energy_gradient(self, L, S, H, mu, spin=2.0, precision=F64, G=None, stream=None):
        import torch
        om, ne = ctypes.c_double(), ctypes.c_double()
        self._need_lsh(L=L, S=S, H=H, G=G)
        f = torch.float64
        _check(_lib.lsq_lnv_energy_gradient(self.handle, _dev(L, f), _dev(S, f), _dev(H, f),
                                            float(mu), float(spin), precision, ctypes.byref(om),
                                            ctypes.byref(ne), _dev(G, f), _stream(stream)))
        return om.value, ne.value

    def minimise(self, L, S, H, mu, max_iter=100, tol_ha_per_atom=0.0, cg_reset=40,
                 precision=F64, refine_iter=2, spin=2.0, final_eval=True, verbose=False,
                 stream=None, raise_on_status=False):
        import torch
        o = LnvOpts(max_iter, tol_ha_per_atom, cg_reset, precision, refine_iter, spin,
                    int(bool(final_eval)), int(bool(verbose)), 1)
        self._need_lsh(L=L, S=S, H=H)
        rep = LnvReport()
        f = torch.float64
        rc = _lib.lsq_lnv_minimise(self.handle, _dev(L, f), _dev(S, f), _dev(H, f), float(mu),
                                   ctypes.byref(o), ctypes.byref(rep), _stream(stream))
        if rc != 0 and (raise_on_status or rc not in (5, 6)):
            _check(rc)
        return rep.as_dict()

    def minimise_canonical(self, L, S, H, n_electrons, max_iter=100, tol_ha_per_atom=0.0, cg_reset=40,
                           precision=F64, spin=2.0, verbose=False, stream=None, raise_on_status=False):
        """Minimises E_band at fixed N_e (in place in L).  Returns (report dict, lambda = mu)."""
        import torch
        o = LnvOpts(max_iter, tol_ha_per_atom, cg_reset, precision, 0, spin, 0, int(bool(verbose)), 0)
        self._need_lsh(L=L, S=S, H=H)
        rep = LnvReport()
        lam = ctypes.c_double()
        f = torch.float64
        rc = _lib.lsq_lnv_minimise_canonical(self.handle, _dev(L, f), _dev(S, f), _dev(H, f),
                                             float(n_electrons), ctypes.byref(o), ctypes.byref(rep),
                                             ctypes.byref(lam), _stream(stream))
        if rc != 0 and (raise_on_status or rc not in (5, 6)):
            _check(rc)
        return rep.as_dict(), lam.value

    def init_purify(self, S, H, mu, X, range_x, range_xh, L, n_iter, precision=F64, stream=None):
        """L = McWeeny purification of the grand-canonical start built from H, S^-1 ~ X and mu.

        Returns |K_{n+1} - K_n|_F per step.  See lsq_lnv_init_purify.
        """
        import torch
        dk = (ctypes.c_double * max(int(n_iter), 1))()
        self._need_lsh(L=L, S=S, H=H)
        _need(X, self.geom, int(range_x), self.b, "X")
        f = torch.float64
        _check(_lib.lsq_lnv_init_purify(self.handle, _dev(S, f), _dev(H, f), float(mu), int(range_x),
                                        _dev(X, f), int(range_xh), int(n_iter), int(precision),
                                        _dev(L, f), dk, _stream(stream)))
        return [dk[k] for k in range(int(n_iter))]

    def set_metric(self, X, range_x, range_xg, stream=None):
        """CG metric X ~ S^-1 (float64 blocks on range_x; None removes it)."""
        import torch
        _need(X, self.geom, int(range_x), self.b, "X")
        ptr = None if X is None else _dev(X, torch.float64)
        _check(_lib.lsq_lnv_set_metric(self.handle, int(range_x), ptr, int(range_xg), _stream(stream)))

    def minimise_batch(self, L, S, H, mu, max_iter=100, tol_ha_per_atom=0.0, cg_reset=40,
                       precision=F64, refine_iter=2, spin=2.0, graph=True, stream=None,
                       raise_on_status=False, final_eval=True):
        """Minimises every system of a concatenated geometry; mu: one value per system."""
        import torch
        mu = [float(m) for m in mu]
        if len(mu) != len(self.geom.systems()) - 1:
            raise LsqError(1, "mu needs one value per system of the geometry")
        o = LnvOpts(max_iter, tol_ha_per_atom, cg_reset, precision, refine_iter, spin,
                    int(bool(final_eval)), 0, int(bool(graph)))
        reps = (LnvReport * len(mu))()
        self._need_lsh(L=L, S=S, H=H)
        f = torch.float64
        rc = _lib.lsq_lnv_minimise_batch(self.handle, _dev(L, f), _dev(S, f), _dev(H, f),
                                         _darr(mu), ctypes.byref(o), reps, _stream(stream))
        if rc != 0 and (raise_on_status or rc not in (5, 6)):
            _check(rc)
        return [r.as_dict() for r in reps]

    def minimise_batch_canonical(self, L, S, H, n_electrons, max_iter=100, tol_ha_per_atom=0.0, cg_reset=40,
                                 precision=F64, spin=2.0, stream=None, raise_on_status=False):
        """E_band at fixed N_e for every system of a concatenated geometry (n_electrons: one
        value per system).  Returns (reports, lambdas), one of each per system."""
        import torch
        ne = [float(v) for v in n_electrons]
        if len(ne) != len(self.geom.systems()) - 1:
            raise LsqError(1, "n_electrons needs one value per system of the geometry")
        o = LnvOpts(max_iter, tol_ha_per_atom, cg_reset, precision, 0, spin, 0, 0, 0)
        self._need_lsh(L=L, S=S, H=H)
        reps = (LnvReport * len(ne))()
        lam = (ctypes.c_double * len(ne))()
        f = torch.float64
        rc = _lib.lsq_lnv_minimise_batch_canonical(self.handle, _dev(L, f), _dev(S, f), _dev(H, f),
                                                   _darr(ne), ctypes.byref(o), reps, lam, _stream(stream))
        if rc != 0 and (raise_on_status or rc not in (5, 6)):
            _check(rc)
        return [r.as_dict() for r in reps], [lam[k] for k in range(len(ne))]

    def close(self):
        if getattr(self, "handle", None) is not None and _lib is not None:
            _lib.lsq_lnv_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def minimise_batch_group(ctxs, Ls, Ss, Hs, mus, max_iter=100, tol_ha_per_atom=0.0, cg_reset=40,
                         precision=F64, refine_iter=2, spin=2.0, stream=None, raise_on_status=False,
                         final_eval=True):
    """lsq_lnv_minimise_batch_group: several batched contexts (distinct geometries, any block
    sizes) minimised in one call, each product of a step one grouped launch over all of them.
    Ls, Ss, Hs: one tensor per context; mus: per context, one value per system.  Returns one
    list of reports per context."""
    import torch
    n = len(ctxs)
    if not (len(Ls) == len(Ss) == len(Hs) == len(mus) == n):
        raise ValueError("one L, S, H and mu list per context")
    for c, mu in zip(ctxs, mus):
        if len(mu) != len(c.geom.systems()) - 1:
            raise LsqError(1, "each mu list needs one value per system of its context's geometry")
    o = LnvOpts(max_iter, tol_ha_per_atom, cg_reset, precision, refine_iter, spin,
                int(bool(final_eval)), 0, 1)
    f = torch.float64
    handles = (ctypes.c_void_p * n)(*[c.handle.value for c in ctxs])
    for c, L, S, H in zip(ctxs, Ls, Ss, Hs):
        c._need_lsh(L=L, S=S, H=H)
    Lp = (ctypes.c_void_p * n)(*[_dev(L, f) for L in Ls])
    Sp = (ctypes.c_void_p * n)(*[_dev(S, f) for S in Ss])
    Hp = (ctypes.c_void_p * n)(*[_dev(H, f) for H in Hs])
    mu_arrs = [_darr([float(m) for m in mu]) for mu in mus]
    mup = (ctypes.c_void_p * n)(*[ctypes.cast(a, ctypes.c_void_p).value for a in mu_arrs])
    rep_arrs = [(LnvReport * len(mu))() for mu in mus]
    repp = (ctypes.c_void_p * n)(*[ctypes.cast(r, ctypes.c_void_p).value for r in rep_arrs])
    rc = _lib.lsq_lnv_minimise_batch_group(n, handles, Lp, Sp, Hp, mup, ctypes.byref(o), repp,
                                           _stream(stream))
    if rc != 0 and (raise_on_status or rc not in (5, 6)):
        _check(rc)
    return [[r.as_dict() for r in reps] for reps in rep_arrs]


def lnv_create(geom, b, R_S, R_H, R_L):
    return Lnv(geom, b, R_S, R_H, R_L)


def lnv_energy_gradient(ctx, L, S, H, mu, **kw):
    return ctx.energy_gradient(L, S, H, mu, **kw)


def lnv_minimise(ctx, L, S, H, mu, **kw):
    return ctx.minimise(L, S, H, mu, **kw)
