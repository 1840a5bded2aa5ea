/*
 * lsq.h -- C ABI of the GB300 linear-scaling density-matrix library.
 *
 * The library implements, on one GPU, the hot path of the O(N) density-
 * matrix method of the CONQUEST paper (arXiv 2002.07704, Sec. 2.3.2,
 * "Density matrix: linear scaling"):
 *   - range patterns of atom-pair matrices: element (i alpha, j beta) is
 *     kept iff the inter-atomic distance R_ij does not exceed the range;
 *   - the truncated atom-block product C = A.B restricted to C's range;
 *   - the LNV grand potential Omega = 2 Tr[(3LSL - 2LSLSL)(H - mu S)]
 *     (McWeeny form of K, Eq. 8; E_band = 2 Tr[K H]), its gradient with
 *     respect to L, and its conjugate-gradient minimisation.
 *
 * Conventions (every entry point):
 *   - Return value: LSQ_OK (0) or an LSQ_ERR_* code; lsq_last_error()
 *     gives a message (thread-local).  On error no output is valid.
 *   - Pointers named *_dev are device pointers (cudaMalloc'd or from
 *     PyTorch); they are borrowed for the duration of the call and never
 *     freed by the library.  Host pointers are named *_host or are
 *     scalars/structs.
 *   - Block storage ("BSR"): a matrix on range pattern r holds
 *     nnzb(r) blocks of b x b values, row-major inside a block, blocks in
 *     the pattern's order (rows ascending, columns ascending in a row).
 *     Blocks hold float64 (LSQ_F64) or float32 (LSQ_F32) values.
 *   - stream is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Work is enqueued asynchronously unless the function returns
 *     host scalars, in which case it synchronises the stream.
 *   - Positions are in Angstrom in an orthorhombic periodic cell
 *     [0, Lx) x [0, Ly) x [0, Lz); energies in eV.
 */
#ifndef LSQ_H
#define LSQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes --------------------------------------------------- */
#define LSQ_OK                 0
#define LSQ_ERR_INVALID_ARG    1   /* bad argument (null, size, range id, dtype) */
#define LSQ_ERR_PATTERN        2   /* a pattern does not fit the operation */
#define LSQ_ERR_OOM            3   /* device allocation failed */
#define LSQ_ERR_CUDA           4   /* a CUDA runtime call or kernel failed */
#define LSQ_ERR_UNSTABLE       5   /* LNV: no local minimum along the line */
#define LSQ_ERR_NOT_CONVERGED  6   /* LNV: iteration limit reached (L holds the last iterate) */
#define LSQ_ERR_UNSUPPORTED    7   /* size beyond a documented kernel limit */
#define LSQ_ERR_TIMEOUT        8   /* a bounded wait inside a kernel expired (see lsq_device_status) */

/* ---- precisions of block products ----------------------------------- */
#define LSQ_F64    0   /* float64 storage, FP64 FMA */
#define LSQ_F32    1   /* float32 storage, FP32 FMA */
#define LSQ_TF32X3 2   /* float32 storage; 4 x 4 blocks multiplied on the tensor cores with
                          split operands: v = hi + lo, hi = tf32(v), lo = tf32(v - hi) (22
                          bits of v), the products hi.hi + hi.lo + lo.hi (and lo.lo)
                          accumulated in FP32; other block sizes as LSQ_F32 */

typedef struct lsq_geom_s *lsq_geom;
typedef struct lsq_lnv_s *lsq_lnv;

/* Copies the message of the last error on this thread into buf (always
 * NUL-terminated when len > 0).  Returns the code of that error. */
int lsq_last_error(char *buf, size_t len);

/* ABI version (major * 10000 + minor * 100 + patch). */
int lsq_version(void);

/* Number of CUDA kernels this library has launched in this process (all
 * devices, all threads).  Host-only; for counting launches in a region. */
int lsq_launch_count(int64_t *out_host);

/* ---- geometry and range patterns (Sec. 2.3.2) ------------------------ */

/*
 * Builds, on the GPU, the range pattern of every requested range: all
 * ordered atom pairs (i, j), self pairs included, whose minimum-image
 * distance satisfies d^2 <= R^2 (Sec. 2.3.2: a matrix's range is set by the
 * interatomic distance, and elements with R_ij beyond the cutoff are zero).  d = r_j - r_i, each component folded as
 * s - L rint(s / L), d^2 = (dx dx + dy dy) + dz dz, every operation
 * correctly rounded and none fused, so the set is reproducible bit for
 * bit on any IEEE host.
 *
 * pos_dev    [n_atoms][3] float64 device array (copied; may be freed after).
 * cell_host  [3] cell lengths; every R must be > 0.
 * ranges_host[n_ranges] cutoffs; the range id of ranges_host[k] is k.
 * out        receives a new handle; release with lsq_geom_destroy.
 * Limits: n_atoms <= 2^30; at most 8192 atoms within the largest range of
 * any atom (LSQ_ERR_UNSUPPORTED otherwise).  Synchronises the stream.
 */
int lsq_build_neighbour_lists(const double *pos_dev, int n_atoms, const double *cell_host,
                              const double *ranges_host, int n_ranges, lsq_geom *out,
                              void *stream);

int lsq_geom_destroy(lsq_geom g);

/* Number of atoms and of ranges of a geometry. */
int lsq_geom_info(lsq_geom g, int *n_atoms, int *n_ranges);

/*
 * Holds n_sys independent systems in one geometry, block-diagonally: the
 * atoms of geoms[k] follow those of geoms[k-1] and every pattern is the
 * concatenation of the systems' patterns (no pair couples two systems).
 * All geometries must have the same list of ranges; each keeps its own
 * cell.  Products, traces and LNV steps on the result run over all systems
 * in single launches (the batched workload; the paper's systems are one at
 * a time).  The inputs stay valid and owned by the caller.  Synchronises.
 */
int lsq_geom_concat(int n_sys, const lsq_geom *geoms, lsq_geom *out, void *stream);

/* Number of systems of a geometry (1 unless made by lsq_geom_concat) and,
 * if atom_off_host is not NULL, the first atom of each system
 * (atom_off_host[n_sys + 1], the last entry is n_atoms). */
int lsq_geom_systems(lsq_geom g, int *n_sys, int64_t *atom_off_host);

/*
 * Device views of pattern range_id (the stored pairs of a range, Sec. 2.3.2):
 * row_ptr_dev [n_atoms+1] int64,
 * col_dev [nnzb] int32 (sorted ascending within a row).  Owned by the
 * geometry; valid until lsq_geom_destroy.  nnzb is returned on the host.
 */
int lsq_pattern(lsq_geom g, int range_id, const int64_t **row_ptr_dev, const int32_t **col_dev,
                int64_t *nnzb);

/* Copies pattern range_id into caller-owned device arrays row_ptr_dev
 * [n_atoms+1] int64 and col_dev [nnzb] int32 (enqueued on stream). */
int lsq_pattern_copy(lsq_geom g, int range_id, int64_t *row_ptr_dev, int32_t *col_dev,
                     void *stream);

/* ---- truncated block-sparse product ----------------------------------- */

/*
 * C = alpha * op(A) . op(B) + beta * C, evaluated only on the stored
 * blocks of C's pattern (Sec. 2.3.2: the product restricted to the range
 * of C; every matrix of the method is sparse by range):
 *     C_ij = alpha * sum_k op(A)_ik op(B)_kj + beta * C_ij
 * over all k with (i, k) stored in op(A)'s pattern and (k, j) in op(B)'s.
 * op(X) = X, or X^T when trans_x != 0 (all patterns are symmetric, so
 * X^T lives on the same pattern, with (X^T)_ik = (X_ki)^T).
 *
 * A_dev, B_dev, C_dev: block arrays on patterns range_a, range_b, range_c
 * of g with block size b (1..16), dtype given by precision.  C must not
 * alias A or B.  Arrays need only the alignment of their value type: with
 * b = 4, 16-byte aligned arrays run the vectorised 4 x 4 kernels (32-byte
 * aligned ones may also use 32-byte loads), others the general kernel.
 * The first call for a (range_a, range_b, range_c, trans)
 * combination builds and caches a product plan (allocates device memory,
 * synchronises); later calls allocate nothing.  n_triples_host (optional)
 * receives the number of block triples (i, k, j) of the product; the
 * algorithmic flop count is 2 b^3 times that number.
 */
int lsq_block_matmul(lsq_geom g, int b, int precision,
                     int range_a, int trans_a, const void *A_dev,
                     int range_b, int trans_b, const void *B_dev,
                     int range_c, void *C_dev, double alpha, double beta,
                     int64_t *n_triples_host, void *stream);

/*
 * lsq_block_matmul restricted to one triangle of C's pattern (the products
 * of the LNV step whose result is symmetric, or of which only one triangle
 * is needed, Sec. 2.3.2):
 *   triangle 0: every block (same as lsq_block_matmul);
 *   triangle 1: C is symmetric in exact arithmetic: the blocks with j >= i
 *               are computed and the others set to their transposes
 *               (requires beta = 0);
 *   triangle 2: only the blocks with j >= i are computed;
 *   triangle 3: only the blocks with j <= i are computed.
 * With 2 and 3 the other blocks of C are left unspecified.  n_triples_host
 * receives the triples of the computed blocks.  Other arguments, errors
 * and plan caching as for lsq_block_matmul (each triangle has its plan).
 */
int lsq_block_matmul_tri(lsq_geom g, int b, int precision,
                         int range_a, int trans_a, const void *A_dev,
                         int range_b, int trans_b, const void *B_dev,
                         int range_c, void *C_dev, double alpha, double beta, int triangle,
                         int64_t *n_triples_host, void *stream);

/*
 * With precision LSQ_TF32X3 and b = 4, lsq_block_matmul(_tri) runs the tensor-core product:
 * atoms i in groups of 8 and the atoms j of their rows of C in tiles of 16; per tile the
 * blocks of op(B)^T and op(A) over the union of the group's rows of op(A) are gathered into
 * shared memory by bulk asynchronous copies and contracted by tcgen05.mma (kind::tf32) into
 * a float32 accumulator in tensor memory.  op(A) and op(B)^T are first copied in split form
 * (a 128-byte hi/lo unit per block) into buffers held by g and grown on demand; the plan of
 * the first call for a (range_a, range_b, range_c, triangle) allocates and synchronises.
 * Arrays need only float alignment.  Limits: rows of at most 65534 blocks and at most
 * 2^31 - 1 blocks in C (LSQ_ERR_UNSUPPORTED).  The kernel bounds every wait on its
 * pipeline barriers (1 s; the environment variable LSQ_TC_WAIT_NS, in ns, lowers it for
 * tests of this path); if one expires it records an error in g, drains its copies and MMAs,
 * frees its tensor memory and returns early, and lsq_device_status reports it.  Calls on
 * different streams race on the split buffers.
 */

/* Measured FMA rate of this GPU in TFLOP/s (2 flop per fused multiply-add): a loop of
 * independent FMAs in float64 (LSQ_F64) or float32 (LSQ_F32) on every SM, the best of three
 * timed launches.  The roofline denominator of the FMA product kernels; no counterpart in the
 * paper.  Synchronises stream; takes a few milliseconds. */
int lsq_measure_peak(int precision, double *tflops_host, void *stream);

/* Statistics of the LSQ_TF32X3 plan of a product already run on g (triangle as for
 * lsq_block_matmul_tri), into info_host[6]: [0] the block triples of the computed blocks;
 * [1] the block triples the MMAs execute (16 j x 8 i x k-list per tile, zero blocks included;
 * each costs 4 x 128 tensor flops with the split operands); [2] the operand block slots a
 * launch fills in shared memory (128 bytes each); [3] the tiles; [5] the slots filled by
 * copying a block (128 bytes from op(A) or op(B)^T; the others are zeros stored in shared
 * memory); [0..3] and [5] are -1 when no plan is held (the LNV path's timing chose the FMA
 * kernel and dropped it); [4], for products the LNV path ran with LSQ_TF32X3, which kernel
 * the timing chose (-1 not timed, 0 FP32 FMA, 1 tensor cores).  Host only.
 * No counterpart in the paper.
 *
 * The LNV path's choice is timed on a product's first call with beta = 0 (both kernels run
 * twice; the call synchronises).  The environment variable LSQ_TC_CHOICE replaces the timing
 * with a fixed choice, read when a product has none yet: a comma-separated list of
 * "range_a:range_b:range_c:t=k" (t = 0 whole C, 1 upper triangle, 2 lower triangle; k = 1
 * tensor cores, 0 FP32 FMA) and "all=k" for the products not listed.  For profiler runs,
 * whose serialised launches distort the timing. */
int lsq_product_plan_info(lsq_geom g, int range_a, int range_b, int range_c, int triangle,
                          int64_t *info_host);

/* Synchronises stream and reports the device error word of g: LSQ_OK, or LSQ_ERR_TIMEOUT
 * when a kernel with bounded waits (the LSQ_TF32X3 product) gave up since the last check
 * (the word is then cleared; the results of that launch are not valid). */
int lsq_device_status(lsq_geom g, void *stream);

/* out = alpha X^T on pattern range_out: out_ij = alpha (X_ji)^T where (j, i)
 * is stored in X's pattern, zero elsewhere (the adjoint of a trace and of a
 * truncation, Sec. 2.3.2).  out must not alias X.  Enqueued on stream; the
 * first call for a (range_x, range_out) pair builds a position map. */
int lsq_transpose(lsq_geom g, int b, int precision, int range_x, const void *X_dev,
                  int range_out, void *out_dev, double alpha, void *stream);

/* Tr[X Y] = sum over stored (i, j) of X, with (j, i) stored in Y, of
 * <X_ij, (Y_ji)^T>, accumulated in float64 (the traces of Sec. 2.3.2's band
 * energy and electron count).  Synchronises the stream. */
int lsq_trace(lsq_geom g, int b, int precision, int range_x, const void *X_dev,
              int range_y, const void *Y_dev, double *out_host, void *stream);

/*
 * The same trace, Tr[X Y], computed without allocating any device memory.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc: code whose device memory is all owned by its own
 * pool or caching allocator, and code that must not stall the device
 * (cudaMalloc and cudaFree can synchronise it).  lsq_trace may allocate on
 * its first call (a position map and reduction buffers); this one never
 * does, and never calls an allocating library routine.
 *
 * Scratch: one float64 partial sum per atom row in a fixed file-scope
 * device array of 262144 entries (2 MiB), which every GPU that loads the
 * library holds until the process exits.  Geometries with more than
 * 262144 atoms are rejected with LSQ_ERR_UNSUPPORTED.  The array is loaded
 * on a device by the creation of a geometry there (lsq_build_neighbour_lists,
 * which allocates in any case); each call then looks up its device address
 * (cudaGetSymbolAddress, with g's device current), which neither allocates
 * nor synchronises once the array is loaded, and stays valid after a device
 * reset.  All calls share the array: calls whose kernels overlap on the GPU
 * (different streams without ordering) race and give wrong results.
 *
 * X_dev, Y_dev: blocks on patterns range_x and range_y (dtype = precision).
 * out_dev: device pointer to one float64 that receives the trace.  The
 * work is enqueued on stream; the call does not synchronise.
 */
int lsq_trace_static(lsq_geom g, int b, int precision, int range_x, const void *X_dev,
                     int range_y, const void *Y_dev, double *out_dev, void *stream);

/* ---- sparse inverse overlap (Sec. 2.3.2, after Eq. 8) ----------------- */

/*
 * Approximate sparse inverse of the overlap S by the Hotelling iteration,
 * the metric the paper's LNV minimisation uses (Sec. 2.3.2, after Eq. 8):
 *     X_{n+1} = 2 X_n - (X_n S) X_n,
 * with X S formed on pattern range_xs (which must cover the natural range
 * R_X + R_S, else LSQ_ERR_INVALID_ARG) and X S X restricted to range_x.
 * Untruncated, I - X_{n+1} S = (I - X_n S)^2.
 *
 * S_dev: float64 blocks on range_s, symmetric (S_ij = S_ji^T, as an overlap
 * is).  X_dev: float64 blocks on range_x, in/out.  start != 0 first sets
 * X_0 = S / s^2 on range_x, s the largest absolute row sum of S (this start
 * converges for any symmetric positive definite S); start = 0 iterates
 * from the X given (which must be symmetric).  n_iter steps are taken; if
 * dx_host is not NULL, dx_host[n] receives |X_{n+1} - X_n|_F.
 * precision: LSQ_F64, or LSQ_F32 for float32 products (X is updated in
 * float64).  The workspace (X S, (X S) X, float32 copies, reductions) is held
 * by g and grown on demand: the first call for given ranges allocates (as do
 * the product plans it builds), later calls of the same or smaller sizes
 * allocate nothing.  Synchronises stream before returning.
 */
int lsq_hotelling_inverse(lsq_geom g, int b, int precision, int range_s, const double *S_dev,
                          int range_x, int range_xs, double *X_dev, int start, int n_iter,
                          double *dx_host, void *stream);

/* ---- LNV grand-potential minimisation (Sec. 2.3.2, Eq. 8) ----------- */

typedef struct {
    int max_iter;              /* CG steps (default 100) */
    double tol_ha_per_atom;    /* stop when |Omega_new - Omega| / N < tol (Hartree); 0: run max_iter */
    int cg_reset;              /* restart the CG direction every cg_reset steps (default 40) */
    int precision;             /* LSQ_F64, or LSQ_F32 for the mixed-precision path */
    int refine_iter;           /* mixed path: FP64 CG steps after the FP32 ones converge (default 2) */
    double spin;               /* spin degeneracy factor of Omega and N_e (default 2) */
    int final_eval;            /* 1 (default): evaluate Omega and N_e of the returned L in
                                  float64 for the report; 0: skip that evaluation, report the
                                  last Omega the steps computed (working precision; the batched
                                  call: the energy at the start of the last step) and N_e = NaN */
    int verbose;               /* 1: print one line per CG step to stderr (default 0) */
    int graph;                 /* batched minimisation: 1 (default) captures one CG step in a
                                  CUDA graph after the first and replays it */
} lsq_lnv_opts;

typedef struct {
    int iterations;            /* CG steps taken (FP32 + FP64) */
    int iterations_fp64;       /* of which FP64 steps */
    int status;                /* LSQ_OK, LSQ_ERR_NOT_CONVERGED or LSQ_ERR_UNSTABLE */
    double omega_ev;           /* Omega(L) of the returned L, evaluated in FP64 */
    double ne;                 /* N_e = 2 Tr[K S] of the returned L, FP64 */
    double omega_ha_per_atom;  /* omega_ev / 27.211386245988 / n_atoms */
    double last_domega_ha_per_atom;
    double seconds;            /* wall time of the minimisation */
} lsq_lnv_report;

/* Fills opts with the defaults listed above. */
int lsq_lnv_default_opts(lsq_lnv_opts *opts);

/*
 * The ranges an LNV context needs in its geometry (a product of ranges R_A
 * and R_B reaches R_A + R_B, Sec. 2.3.2), in this order:
 * R_S, R_H, R_L, R_L + R_S (LS), R_L + R_S + R_L (LSL), R_H + R_L + R_S
 * (H'LS), each computed in float64 exactly as written.  out_host[6].
 */
int lsq_lnv_required_ranges(double R_S, double R_H, double R_L, double *out_host);

/*
 * Creates an LNV context (workspace for all products of one CG step of the
 * LNV minimisation, Sec. 2.3.2) on
 * geometry g, whose ranges must include lsq_lnv_required_ranges(...)
 * (looked up by exact value).  Requires R_S <= R_H.  b: orbitals per atom.
 * Allocates the small, fixed part of the workspace.  The product buffers (LS,
 * LSL, Q, ... on the product ranges: most of the memory) are allocated by the
 * first call that needs them, at 4 bytes per value while every call so far
 * has been float32-only, and at 8 bytes once a call may run float64 work
 * (precision LSQ_F64, refinement steps, the final float64 evaluation, or
 * lsq_lnv_init_purify).  Such a call then reallocates them once.  Product
 * plans and per-system state are allocated on first use too.  Once
 * everything a call needs is allocated, repeating the call allocates
 * nothing.
 */
int lsq_lnv_create(lsq_geom g, int b, double R_S, double R_H, double R_L, lsq_lnv *out);
int lsq_lnv_destroy(lsq_lnv ctx);

/* Initial L = 1/2 (S_ii)^-1 on the diagonal blocks, zero elsewhere
 * (symmetrised): a start for the minimisation of Sec. 2.3.2, which gives none.  S_dev on R_S's pattern, L_dev on R_L's, float64. */
int lsq_lnv_init_L(lsq_lnv ctx, const double *S_dev, double *L_dev, void *stream);

/*
 * Omega = spin Tr[K (H - mu S)], N_e = spin Tr[K S], K = 3LSL - 2LSLSL (Eq. 8) on
 * H's range, and G_ab = dOmega/dL_ab on L's range (symmetrised), for
 * float64 L_dev (R_L), S_dev (R_S), H_dev (R_H).  precision LSQ_F64 or
 * LSQ_F32 (products in FP32, traces accumulated in float64).  G_dev may
 * be NULL.  Synchronises the stream (returns host scalars).
 */
int lsq_lnv_energy_gradient(lsq_lnv ctx, const double *L_dev, const double *S_dev,
                            const double *H_dev, double mu, double spin, int precision,
                            double *omega_host, double *ne_host, double *G_dev, void *stream);

/*
 * Canonical LNV: minimises E_band = 2 Tr[K H] at fixed electron number
 * N_e = 2 Tr[K S] = n_electrons (Sec. 2.3.2: the electron number is
 * constrained during the optimisation).  Each CG step first restores N_e
 * by Newton moves along dN_e/dL (at most 5, to 1e-9 relative in FP64, 1e-6
 * with FP32 products), projects the energy gradient on constant N_e (its
 * multiplier lambda, the chemical potential, goes to *lambda_out), builds
 * Polak-Ribiere directions from the projected gradient, projects them
 * again and takes the exact cubic minimum of E_band.  opts as for
 * lsq_lnv_minimise, with precision applying to every step (no separate
 * FP64 refinement) and refine_iter, final_eval and graph ignored; the
 * report's omega_ev is E_band and ne the last N_e measured.  Near exact
 * idempotency dN_e/dL vanishes and the constraint cannot be held: the call
 * then returns LSQ_ERR_UNSTABLE.  No metric may be set (LSQ_ERR_UNSUPPORTED).
 */
int lsq_lnv_minimise_canonical(lsq_lnv ctx, double *L_dev, const double *S_dev, const double *H_dev,
                               double n_electrons, const lsq_lnv_opts *opts, lsq_lnv_report *report_host,
                               double *lambda_out, void *stream);

/*
 * Initial L from the Hamiltonian (Sec. 2.3.2: the initial density matrix is
 * generated from H by an iterative generalisation of the McWeeny transform):
 * grand-canonical purification at mu with an approximate inverse overlap X:
 *     K_0 = (lam/2) (mu X - X H X) + X/2,  lam = min(1/(e_max - mu), 1/(mu - e_min)),
 *     K_{n+1} = 3 K S K - 2 K S K S K,
 * (the symmetric part of the right side, since K S K is truncated before
 * the last product), [e_min, e_max] the Gershgorin bounds of X H (its
 * scalar rows), X H on
 * range_xh (covering R_X + R_H, else LSQ_ERR_INVALID_ARG; at most as large
 * as the context's widest range), X H X, K S K and K S K S K on L's range.
 * K_n is written to L_dev (float64, L's range), the start for
 * lsq_lnv_minimise.  S_dev on R_S, H_dev on R_H, X_dev on range_x (all
 * float64, symmetric).  precision: LSQ_F64, or LSQ_F32 for float32 products
 * in the McWeeny steps.  dk_host (optional, [n_iter]): |K_{n+1} - K_n|_F.
 * mu outside [e_min, e_max]: LSQ_ERR_INVALID_ARG.  Uses the context's
 * workspace; synchronises stream.
 */
int lsq_lnv_init_purify(lsq_lnv ctx, const double *S_dev, const double *H_dev, double mu, int range_x,
                        const double *X_dev, int range_xh, int n_iter, int precision, double *L_dev,
                        double *dk_host, void *stream);

/*
 * Sets the metric of lsq_lnv_minimise's conjugate gradients (Sec. 2.3.2:
 * an approximate sparse inverse overlap, e.g. from lsq_hotelling_inverse,
 * is the metric of the minimisation).  With a metric X the search
 * directions come from P = (X G X) on L's range instead of the gradient G,
 * and Polak-Ribiere takes beta = <G, P - P_prev> / <G_prev, P_prev>; the
 * line search is unchanged.  X_dev: float64 blocks on range_x, symmetric;
 * the context keeps its own copy.  range_xg: pattern for X G, covering
 * R_X + R_L (else LSQ_ERR_INVALID_ARG).  X_dev = NULL removes the metric.
 * The batched minimisers use it too: on a batch geometry X is block diagonal
 * over the systems, and each system's Polak-Ribiere sums are its own.  The
 * contexts of one lsq_lnv_minimise_batch_group call take a metric all or
 * none (else LSQ_ERR_INVALID_ARG).  Allocates; synchronises stream.
 */
int lsq_lnv_set_metric(lsq_lnv ctx, int range_x, const double *X_dev, int range_xg, void *stream);

/*
 * Conjugate-gradient minimisation of Omega over symmetric L on L's range
 * (Sec. 2.3.2): Polak-Ribiere direction (beta = max(0, beta_PR)) restarted
 * every cg_reset steps (40 in the convergence figure of Sec. 5.3), exact line minimisation of the cubic Omega(L + a D).
 * L_dev (float64, R_L) holds the start on entry and the result on exit.
 * Returns LSQ_OK when converged (or max_iter steps were taken with
 * tol = 0), LSQ_ERR_NOT_CONVERGED, or LSQ_ERR_UNSTABLE; rep (optional)
 * receives the report in every case.
 */
int lsq_lnv_minimise(lsq_lnv ctx, double *L_dev, const double *S_dev, const double *H_dev,
                     double mu, const lsq_lnv_opts *opts, lsq_lnv_report *rep, void *stream);

/*
 * The same minimisation (Sec. 2.3.2) for every system of a geometry made by
 * lsq_geom_concat, all systems at once: each CG step is one sequence of
 * launches over all systems, with each system's Omega, beta, line
 * coefficients and step length reduced and computed on the device, so no
 * step waits for the host; with opts->graph the step is captured in a CUDA
 * graph after the first one (which builds plans and tunes kernels) and
 * replayed.  Systems are independent: each has its own mu (mu_host[n_sys]),
 * its own line search and its own convergence (a converged system is
 * frozen, alpha = 0, while the others continue).  Differences from
 * lsq_lnv_minimise: a direction that is not descent is restarted on the
 * next step (the step is skipped) instead of immediately.  The mixed path
 * refines every system with refine_iter float64 steps.  reps[n_sys]
 * receives one report per system.  Synchronises the stream every 5 steps
 * (convergence check) and at the end.  The first call allocates the
 * per-system state; capture needs no allocation after that.
 */
int lsq_lnv_minimise_batch(lsq_lnv ctx, double *L_dev, const double *S_dev, const double *H_dev,
                           const double *mu_host, const lsq_lnv_opts *opts, lsq_lnv_report *reps,
                           void *stream);

/*
 * The canonical minimisation (lsq_lnv_minimise_canonical: E_band at fixed
 * N_e, Sec. 2.3.2) for every system of a geometry made by lsq_geom_concat,
 * all systems at once.  n_electrons_host[n_sys]: each system's electron
 * count (positive).  Each step restores every system's N_e by Newton moves
 * along its own dN_e/dL (at most 5, until |N_e - N0| <= tol N0 with tol
 * 1e-9 for LSQ_F64 products and 1e-6 otherwise; the host reads one count
 * per round to know whether any system still moves), then projects the
 * energy gradient and the Polak-Ribiere direction on constant N_e, with
 * each system's multiplier lambda = <G_E, G_N> / <G_N, G_N> (its chemical
 * potential), and takes each system's exact cubic step of E_band.  As in
 * lsq_lnv_minimise_batch, a direction that is not descent restarts on the
 * next step, and a converged system is frozen.  No metric (else
 * LSQ_ERR_UNSUPPORTED); no float64 refinement phase.  reps[n_sys] (optional)
 * receives E_band (omega_ev), N_e and the step counts; lambda_host[n_sys]
 * (optional) the multipliers.  Allocates; synchronises the stream after
 * every correction round.
 */
int lsq_lnv_minimise_batch_canonical(lsq_lnv ctx, double *L_dev, const double *S_dev, const double *H_dev,
                                     const double *n_electrons_host, const lsq_lnv_opts *opts,
                                     lsq_lnv_report *reps, double *lambda_host, void *stream);

/*
 * lsq_lnv_minimise_batch over n_ctx contexts at once (1 <= n_ctx <= 16), each on its own
 * lsq_geom_concat geometry with its own block size: a batch of uneven systems whose block
 * sizes differ (4 x 4 and 13 x 13, say) in one call.  Arrays are per context: L_dev[c],
 * S_dev[c], H_dev[c] on ctx[c]'s geometry as for lsq_lnv_minimise_batch, mu_host[c][n_sys of
 * ctx[c]], reps[c][n_sys of ctx[c]] (reps or reps[c] may be null).  The first step of each
 * phase runs context by context (building plans); every later step is one CUDA graph over all
 * contexts in which each product of the step is a single persistent launch serving that
 * product of every context: its thread blocks take work items (a chunk of blocks of C of one
 * context's product) from a queue counter in device memory until the queue is empty, so the
 * systems of all contexts share the GPU within each product.  The products in those launches
 * use one fixed schedule per block size instead of the autotuned ones.  precision: LSQ_F64 or
 * LSQ_F32 (LSQ_ERR_INVALID_ARG otherwise); opts->graph is implied.  The contexts' geometries
 * must be distinct (LSQ_ERR_INVALID_ARG).  Systems, convergence, refinement, reports and
 * return codes as for lsq_lnv_minimise_batch.  The first call of a context allocates its
 * per-system state; each call builds and frees its step graphs.  No counterpart in the paper
 * (Sec. 2.3.2 defines the minimisation of each system).
 */
int lsq_lnv_minimise_batch_group(int n_ctx, lsq_lnv *ctx, double **L_dev, const double **S_dev,
                                 const double **H_dev, const double **mu_host, const lsq_lnv_opts *opts,
                                 lsq_lnv_report **reps, void *stream);

/*
 * Lets g_to use the kernel schedules the product autotuner chose in g_from
 * (and those g_from adopted in turn), for the plans of the same (range_a,
 * range_b, range_c, triangle): a plan of g_to that has not been tuned then
 * runs the adopted schedule instead of timing every schedule on its first
 * call.  Meant for a sequence of geometries of one system (MD steps), whose
 * products have the same shape.  A schedule whose alignment or shared
 * memory the operands do not allow falls back to the adopted 16-byte
 * schedule, as a tuned one does.  Both geometries must hold the same range
 * list (LSQ_ERR_INVALID_ARG otherwise); the atom counts may differ.  Host
 * only, no device work; g_from may be destroyed afterwards.
 */
int lsq_geom_adopt_schedules(lsq_geom g_to, lsq_geom g_from);

/* ---- density matrix between MD steps (Sec. 3.3) ---------------------- */

/*
 * Moves a matrix to another pattern of the same atoms, typically the
 * pattern of the same range after the atoms moved (Sec. 3.3: the matrices
 * carried from one MD step to the next).  Block (i, j) of range_to's
 * pattern in g_to receives block (i, j) of range_from's pattern in g_from
 * where that pattern stores it, and zeros elsewhere: blocks of pairs that
 * left the range are dropped, pairs that entered start at zero.  The
 * copies are exact.
 *
 * g_from and g_to must hold the same atom count (LSQ_ERR_INVALID_ARG
 * otherwise) and may be the same geometry.  X_from_dev: blocks on
 * (g_from, range_from); X_to_dev: blocks on (g_to, range_to), written; both
 * b x b row-major in the precision's value type (LSQ_F64 double, LSQ_F32
 * float) and not aliased.  Enqueued on stream; no allocation, no
 * synchronisation.
 */
int lsq_pattern_remap(lsq_geom g_from, int range_from, lsq_geom g_to, int range_to, int b,
                      int precision, const void *X_from_dev, void *X_to_dev, void *stream);

/*
 * One step of the extended-Lagrangian propagation of X, the auxiliary
 * matrix associated with L S (Sec. 3.3): the Verlet step in the harmonic
 * potential centred on L(t) S(t), plus the dissipative sum,
 *     X(t+dt) = 2 X(t) - X(t-dt) + kappa (LS - X(t)) + alpha sum_{m<n_c} c_m X(t - m dt),
 * kappa = dt^2 w^2, evaluated with the terms grouped by history entry
 * (weights 2 - kappa + alpha c_0, -1 + alpha c_1, alpha c_m, and kappa for
 * LS; one FMA each), so it agrees with the formula as written to a few
 * units in the last place.  alpha = 0 drops the sum (c may then be NULL).
 *
 * X_hist_host: host array of n_hist (2..10) device pointers, X(t), X(t-dt),
 * ..., all float64 blocks on range_x (L S's range R_L + R_S) of g.
 * LS_dev: L(t) S(t) on range_x.  c_host: n_c (1..n_hist) coefficients.
 * X_next_dev: X(t+dt), written; it may be one of the history arrays
 * (each value is read before it is written) but not LS_dev.  Enqueued on
 * stream; no allocation, no synchronisation.
 */
int lsq_xl_propagate(lsq_geom g, int b, int range_x, int n_hist, const double *const *X_hist_host,
                     const double *LS_dev, double kappa, double alpha, const double *c_host, int n_c,
                     double *X_next_dev, void *stream);

/*
 * The initial L of an MD step from the propagated X (Sec. 3.3: X S^-1 is
 * the initial guess for L): L_0 = ((X Sinv) + (X Sinv)^T) / 2 on range_l,
 * the product truncated to range_l and its symmetric part formed in place
 * (exactly symmetric).  X_dev: float64 blocks on range_x; Sinv_dev: an
 * approximate inverse overlap on range_sinv (e.g. from
 * lsq_hotelling_inverse); L_out_dev: float64 blocks on range_l, written,
 * not aliasing the inputs.  precision LSQ_F64, or LSQ_F32: the operands
 * are rounded to float32 and multiplied in float32 (a float32 workspace
 * held by g, grown on demand), the product widened to float64 before its
 * symmetric part is taken.  The product's plan is built on the first call
 * for these ranges (allocates, synchronises) as for lsq_block_matmul.
 */
int lsq_xl_initial_L(lsq_geom g, int b, int precision, int range_x, const double *X_dev, int range_sinv,
                     const double *Sinv_dev, int range_l, double *L_out_dev, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* LSQ_H */
