"""CPU FP64 oracle for the truncated atom-block product and LNV minimisation.

TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
benchmark's CPU-baseline leg may import this package.  It shares no code
with the CUDA path (paper_2002_07704_gb300) and neither imports the other;
both take their inputs from the seeded generators in ``synth``.

The arithmetic core is plain C (``oracle.c``, single-threaded, no FMA
contraction), loaded with ctypes; the LNV steps are written out in numpy
in ``lnv.py``.  Every function cites the passage of the paper it follows.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_oracle.so")
_lib = None


_OMP_PATH = os.path.join(_HERE, "_oracle_omp.so")


def build(force=False, openmp=False):
    """Compile oracle.c with gcc into an in-tree shared library (openmp=True: the OpenMP build
    that times the CPU baseline on all host cores; the tests use the single-threaded one)."""
    path = _OMP_PATH if openmp else _LIB_PATH
    if not force and os.path.exists(path) and os.path.getmtime(path) >= os.path.getmtime(_SRC):
        return path
    tmp = path + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                           "-shared"] + (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
    os.replace(tmp, path)
    return path


_want_omp = False


def use_threads(n):
    """Products on n host threads (the OpenMP build; n = 1: the plain single-threaded build).
    Returns the number of threads the products then use.  For the CPU-baseline timing only."""
    global _lib, _want_omp
    _want_omp = n != 1
    _lib = None
    lib = _load()
    return int(lib.orc_set_threads(int(n))) if _want_omp else 1


def _load():
    global _lib
    if _lib is not None:
        return _lib
    lib = ctypes.CDLL(build(openmp=_want_omp))
    lib.orc_set_threads.restype = ctypes.c_int
    lib.orc_set_threads.argtypes = [ctypes.c_int]
    P = ctypes.c_void_p
    i64, i32, dbl = ctypes.c_int64, ctypes.c_int, ctypes.c_double
    lib.orc_neigh_count.restype = i64
    lib.orc_neigh_count.argtypes = [i32, i32, P, P, dbl, P]
    lib.orc_neigh_fill.restype = None
    lib.orc_neigh_fill.argtypes = [i32, i32, P, P, dbl, P, P]
    lib.orc_bsr_matmul.restype = i64
    lib.orc_bsr_matmul.argtypes = [i32, i32, P, P, P, P, P, P, P, P, P, i32, P]
    lib.orc_trace_xy.restype = dbl
    lib.orc_trace_xy.argtypes = [i32, i32, P, P, P, P, P, P]
    lib.orc_bsr_transpose.restype = None
    lib.orc_bsr_transpose.argtypes = [i32, i32, P, P, P, P, P, P]
    lib.orc_bsr_restrict.restype = None
    lib.orc_bsr_restrict.argtypes = [i32, i32, P, P, P, P, P, P]
    _lib = lib
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


class Pattern:
    """Range pattern of an atom-pair matrix: (i, j) stored iff R_ij <= R.

    Sec. 2.3.2: the range of a matrix is set by the inter-atomic distance;
    elements with R_ij beyond the cutoff are zero.  Columns are sorted
    ascending within each row; self pairs are included.
    """

    def __init__(self, n, ptr, col, R):
        self.n = int(n)
        self.ptr = np.ascontiguousarray(ptr, dtype=np.int64)
        self.col = np.ascontiguousarray(col, dtype=np.int32)
        self.R = float(R)

    @property
    def nnzb(self):
        return int(self.ptr[-1])

    def rows(self):
        return np.repeat(np.arange(self.n, dtype=np.int64), np.diff(self.ptr))

    def __eq__(self, other):
        return (self.n == other.n and np.array_equal(self.ptr, other.ptr)
                and np.array_equal(self.col, other.col))


def neighbour_list(pos, cell, R, method="cell"):
    """Pattern of all pairs with minimum-image distance <= R (Sec. 2.3.2).

    method "brute" tests every pair; "cell" bins atoms into cells of edge
    at least R and scans the 27 adjacent cells.  Both give the same set.
    """
    lib = _load()
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    cell = np.ascontiguousarray(cell, dtype=np.float64)
    n = pos.shape[0]
    m = {"brute": 0, "cell": 1}[method]
    counts = np.zeros(n, dtype=np.int64)
    lib.orc_neigh_count(m, n, _p(pos), _p(cell), float(R), _p(counts))
    ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=ptr[1:])
    col = np.zeros(max(int(ptr[-1]), 1), dtype=np.int32)
    lib.orc_neigh_fill(m, n, _p(pos), _p(cell), float(R), _p(ptr), _p(col))
    return Pattern(n, ptr, col[:int(ptr[-1])], R)


class Bsr:
    """Block-sparse matrix on a range pattern; val is [nnzb, b, b] float64."""

    def __init__(self, pat, b, val=None):
        self.pat = pat
        self.b = int(b)
        if val is None:
            val = np.zeros((pat.nnzb, b, b))
        self.val = np.ascontiguousarray(val, dtype=np.float64)
        assert self.val.shape == (pat.nnzb, b, b)

    def copy(self):
        return Bsr(self.pat, self.b, self.val.copy())

    def __add__(self, o):
        assert o.pat is self.pat
        return Bsr(self.pat, self.b, self.val + o.val)

    def __sub__(self, o):
        assert o.pat is self.pat
        return Bsr(self.pat, self.b, self.val - o.val)

    def __rmul__(self, s):
        return Bsr(self.pat, self.b, float(s) * self.val)

    def dense(self):
        """Expand to a dense [n b, n b] matrix (zeros outside the pattern)."""
        n, b = self.pat.n, self.b
        M = np.zeros((n, b, n, b))
        M[self.pat.rows(), :, self.pat.col, :] = self.val
        return M.reshape(n * b, n * b)

    @staticmethod
    def from_dense(M, pat, b):
        """Blocks of dense M at the stored positions of pat."""
        n = pat.n
        M4 = np.asarray(M, dtype=np.float64).reshape(n, b, n, b)
        return Bsr(pat, b, M4[pat.rows(), :, pat.col, :])


def matmul(A, B, pat_c, rows=None):
    """Truncated product C = A.B restricted to pat_c (Sec. 2.3.2).

    C_ij = sum_k A_ik B_kj for every (i, j) stored in pat_c; blocks with no
    contributing k are zero.  rows (optional) limits the work to those C
    rows; other rows of the result are left zero.  Returns (C, triples),
    triples = number of (i, k, j) block products performed.
    """
    lib = _load()
    assert A.b == B.b
    C = Bsr(pat_c, A.b)
    if rows is None:
        nr, rp = 0, None
    else:
        r = np.ascontiguousarray(rows, dtype=np.int32)
        nr, rp = r.size, _p(r)
    t = lib.orc_bsr_matmul(A.b, pat_c.n,
                           _p(A.pat.ptr), _p(A.pat.col), _p(A.val),
                           _p(B.pat.ptr), _p(B.pat.col), _p(B.val),
                           _p(pat_c.ptr), _p(pat_c.col), _p(C.val), nr, rp)
    return C, int(t)


def trace(X, Y):
    """Tr[X Y] = sum over stored (i, j) of <X_ij, (Y_ji)^T>."""
    lib = _load()
    return float(lib.orc_trace_xy(X.b, X.pat.n, _p(X.pat.ptr), _p(X.pat.col), _p(X.val),
                                  _p(Y.pat.ptr), _p(Y.pat.col), _p(Y.val)))


def dot(X, Y):
    """Elementwise inner product sum_ij <X_ij, Y_ij> of two matrices on one pattern."""
    assert X.pat is Y.pat
    return float(np.sum(X.val * Y.val))


def transpose(X, pat):
    """X^T on pattern pat: out_ij = (X_ji)^T, zero where (j, i) is not stored in X."""
    lib = _load()
    out = Bsr(pat, X.b)
    lib.orc_bsr_transpose(X.b, pat.n, _p(X.pat.ptr), _p(X.pat.col), _p(X.val),
                          _p(pat.ptr), _p(pat.col), _p(out.val))
    return out


def restrict(X, pat):
    """X on pattern pat: out_ij = X_ij, zero where (i, j) is not stored in X."""
    lib = _load()
    out = Bsr(pat, X.b)
    lib.orc_bsr_restrict(X.b, pat.n, _p(X.pat.ptr), _p(X.pat.col), _p(X.val),
                         _p(pat.ptr), _p(pat.col), _p(out.val))
    return out
