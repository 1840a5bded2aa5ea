/*
 * oracle.c -- plain, slow CPU FP64 oracle (single-threaded; an OpenMP build of
 * the same source, used only to time the CPU baseline on all host cores, shares
 * the rows of a product among threads without changing any row's arithmetic).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA path and must never be called by it.
 *
 * What it computes, each function following the passage it implements:
 *   - range masks of atom-pair matrices: element (i alpha, j beta) is kept
 *     iff the inter-atomic distance R_ij does not exceed the cutoff R_c
 *     (Sec. 2.3.2, "Density matrix: linear scaling").  R_ij is the
 *     minimum-image distance in an orthorhombic periodic cell.
 *   - the truncated atom-block product C = A.B restricted to the range of C,
 *     written as its definition: C_ij = sum_k A_ik B_kj for every stored
 *     (i, j) of C (Sec. 2.3.2: all matrices sparse, all operations linear).
 *   - traces of block products, Tr[X Y] = sum_ij <X_ij, (Y_ji)^T>, used for
 *     E_band = 2 Tr[K H] (Sec. 2.3.2) and the electron count.
 *   - transposes and restrictions of block-sparse matrices.
 *
 * Distances: d = r_j - r_i, each component folded s -= L * rint(s / L),
 * d^2 = (dx*dx + dy*dy) + dz*dz, compared as d^2 <= R*R.  Compile with
 * -ffp-contract=off so no step is fused.
 *
 * Storage: block-sparse rows (BSR).  row_ptr [N+1] int64, col [nnzb] int32
 * sorted ascending within a row, val [nnzb][b][b] float64 row-major.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double orc_dist2(const double *pi, const double *pj, const double *cell)
{
    double d[3];
    for (int c = 0; c < 3; ++c) {
        double s = pj[c] - pi[c];
        double t = rint(s / cell[c]);
        double u = cell[c] * t;
        d[c] = s - u;
    }
    double xx = d[0] * d[0];
    double yy = d[1] * d[1];
    double zz = d[2] * d[2];
    double xy = xx + yy;
    return xy + zz;
}

/* ---- neighbour lists -------------------------------------------------- */

/* Brute force: every ordered pair (i, j), self pairs included. */
static int64_t orc_row_brute(int n, const double *pos, const double *cell, double r2,
                             int i, int32_t *out)
{
    int64_t cnt = 0;
    for (int j = 0; j < n; ++j) {
        if (orc_dist2(pos + 3 * i, pos + 3 * j, cell) <= r2) {
            if (out) out[cnt] = j;
            ++cnt;
        }
    }
    return cnt;
}

typedef struct {
    int nc[3];
    int *head;      /* [ncell + 1] start of each cell in 'atoms' */
    int *atoms;     /* atom indices sorted by cell, ascending within a cell */
} orc_cells;

static int orc_cell_of(double x, double L, int nc)
{
    double f = x / L;
    f = f - floor(f);
    int c = (int)(f * nc);
    if (c < 0) c = 0;
    if (c >= nc) c = nc - 1;
    return c;
}

static void orc_cells_build(int n, const double *pos, const double *cell, double R, orc_cells *g)
{
    int ntot = 1;
    for (int c = 0; c < 3; ++c) {
        /* cell edge at least R (with margin), so in-range pairs sit in adjacent cells */
        int k = (int)floor(cell[c] / (R * (1.0 + 1e-6)));
        if (k < 1) k = 1;
        g->nc[c] = k;
        ntot *= k;
    }
    g->head = (int *)calloc((size_t)ntot + 1, sizeof(int));
    g->atoms = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    int *cid = (int *)malloc(sizeof(int) * (size_t)(n > 0 ? n : 1));
    for (int i = 0; i < n; ++i) {
        int cx = orc_cell_of(pos[3 * i + 0], cell[0], g->nc[0]);
        int cy = orc_cell_of(pos[3 * i + 1], cell[1], g->nc[1]);
        int cz = orc_cell_of(pos[3 * i + 2], cell[2], g->nc[2]);
        cid[i] = (cx * g->nc[1] + cy) * g->nc[2] + cz;
        g->head[cid[i] + 1]++;
    }
    for (int c = 0; c < ntot; ++c) g->head[c + 1] += g->head[c];
    int *fill = (int *)malloc(sizeof(int) * (size_t)ntot);
    memcpy(fill, g->head, sizeof(int) * (size_t)ntot);
    for (int i = 0; i < n; ++i) g->atoms[fill[cid[i]]++] = i;
    free(fill);
    free(cid);
}

static int orc_cmp_int32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Neighbour offsets -1, 0, +1 folded into [0, nc), without repeats. */
static int orc_offsets(int c, int nc, int out[3])
{
    int m = 0;
    for (int d = -1; d <= 1; ++d) {
        int v = ((c + d) % nc + nc) % nc;
        int dup = 0;
        for (int q = 0; q < m; ++q) dup |= (out[q] == v);
        if (!dup) out[m++] = v;
    }
    return m;
}

static int64_t orc_row_cells(const orc_cells *g, const double *pos, const double *cell, double r2,
                             int i, int32_t *out)
{
    int c0[3], ox[3], oy[3], oz[3];
    for (int c = 0; c < 3; ++c) c0[c] = orc_cell_of(pos[3 * i + c], cell[c], g->nc[c]);
    int mx = orc_offsets(c0[0], g->nc[0], ox);
    int my = orc_offsets(c0[1], g->nc[1], oy);
    int mz = orc_offsets(c0[2], g->nc[2], oz);
    int64_t cnt = 0;
    for (int a = 0; a < mx; ++a)
        for (int b = 0; b < my; ++b)
            for (int c = 0; c < mz; ++c) {
                int id = (ox[a] * g->nc[1] + oy[b]) * g->nc[2] + oz[c];
                for (int q = g->head[id]; q < g->head[id + 1]; ++q) {
                    int j = g->atoms[q];
                    if (orc_dist2(pos + 3 * i, pos + 3 * j, cell) <= r2) {
                        if (out) out[cnt] = j;
                        ++cnt;
                    }
                }
            }
    if (out) qsort(out, (size_t)cnt, sizeof(int32_t), orc_cmp_int32);
    return cnt;
}

/* method 0 = brute force, 1 = cell list.  Writes per-row counts; returns nnzb. */
int64_t orc_neigh_count(int method, int n, const double *pos, const double *cell, double R,
                        int64_t *row_counts)
{
    double r2 = R * R;
    int64_t tot = 0;
    orc_cells g = {{0, 0, 0}, NULL, NULL};
    if (method == 1) orc_cells_build(n, pos, cell, R, &g);
    for (int i = 0; i < n; ++i) {
        int64_t c = method == 1 ? orc_row_cells(&g, pos, cell, r2, i, NULL)
                                : orc_row_brute(n, pos, cell, r2, i, NULL);
        row_counts[i] = c;
        tot += c;
    }
    free(g.head);
    free(g.atoms);
    return tot;
}

void orc_neigh_fill(int method, int n, const double *pos, const double *cell, double R,
                    const int64_t *row_ptr, int32_t *col)
{
    double r2 = R * R;
    orc_cells g = {{0, 0, 0}, NULL, NULL};
    if (method == 1) orc_cells_build(n, pos, cell, R, &g);
    for (int i = 0; i < n; ++i) {
        if (method == 1)
            orc_row_cells(&g, pos, cell, r2, i, col + row_ptr[i]);
        else
            orc_row_brute(n, pos, cell, r2, i, col + row_ptr[i]);
    }
    free(g.head);
    free(g.atoms);
}

/* ---- block-sparse algebra --------------------------------------------- */

/* Position of column j in row i of a pattern, or -1 (binary search). */
static int64_t orc_find(const int64_t *ptr, const int32_t *col, int i, int j)
{
    int64_t lo = ptr[i], hi = ptr[i + 1];
    while (lo < hi) {
        int64_t mid = lo + (hi - lo) / 2;
        if (col[mid] < j) lo = mid + 1;
        else hi = mid;
    }
    return (lo < ptr[i + 1] && col[lo] == j) ? lo : -1;
}

/*
 * Truncated product on the rows listed in 'rows' (all rows if rows == NULL):
 * C_ij = sum over k in row i of A, with (k, j) stored in B, of A_ik B_kj,
 * for every (i, j) stored in C.  Blocks of C with no contribution are zero.
 * Contributions are added in ascending k; within a block product the
 * b-term sum runs in ascending inner index.  Returns the number of block
 * triples (i, k, j) that contributed.
 */
/* One row i of the truncated product (the body of orc_bsr_matmul); slot[] is a scratch
 * map of n entries, all -1 on entry and on return.  Returns the row's block triples. */
static int64_t bsr_matmul_row(int b, int i,
                              const int64_t *a_ptr, const int32_t *a_col, const double *a_val,
                              const int64_t *b_ptr, const int32_t *b_col, const double *b_val,
                              const int64_t *c_ptr, const int32_t *c_col, double *c_val, int64_t *slot)
{
    int64_t bb = (int64_t)b * b;
    int64_t triples = 0;
    for (int64_t p = c_ptr[i]; p < c_ptr[i + 1]; ++p) {
        slot[c_col[p]] = p;
        memset(c_val + p * bb, 0, sizeof(double) * (size_t)bb);
    }
    for (int64_t pa = a_ptr[i]; pa < a_ptr[i + 1]; ++pa) {
        int k = a_col[pa];
        const double *ablk = a_val + pa * bb;
        for (int64_t pb = b_ptr[k]; pb < b_ptr[k + 1]; ++pb) {
            int64_t pc = slot[b_col[pb]];
            if (pc < 0) continue;
            const double *bblk = b_val + pb * bb;
            double *cblk = c_val + pc * bb;
            for (int x = 0; x < b; ++x)
                for (int y = 0; y < b; ++y) {
                    double acc = cblk[x * b + y];
                    for (int t = 0; t < b; ++t) {
                        double prod = ablk[x * b + t] * bblk[t * b + y];
                        acc = acc + prod;
                    }
                    cblk[x * b + y] = acc;
                }
            ++triples;
        }
    }
    for (int64_t p = c_ptr[i]; p < c_ptr[i + 1]; ++p) slot[c_col[p]] = -1;
    return triples;
}

int64_t orc_bsr_matmul(int b, int n,
                       const int64_t *a_ptr, const int32_t *a_col, const double *a_val,
                       const int64_t *b_ptr, const int32_t *b_col, const double *b_val,
                       const int64_t *c_ptr, const int32_t *c_col, double *c_val,
                       int nrows, const int32_t *rows)
{
    int64_t triples = 0;
    int nr = rows ? nrows : n;
    /* Rows are independent.  Built with OpenMP (only for the timed CPU baseline) the rows are
     * shared among threads, each with its own scratch map; every row is computed exactly as
     * in the single-threaded build. */
#ifdef _OPENMP
#pragma omp parallel reduction(+ : triples)
#endif
    {
        int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        for (int j = 0; j < n; ++j) slot[j] = -1;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 8)
#endif
        for (int r = 0; r < nr; ++r) {
            int i = rows ? rows[r] : r;
            triples += bsr_matmul_row(b, i, a_ptr, a_col, a_val, b_ptr, b_col, b_val, c_ptr, c_col, c_val, slot);
        }
        free(slot);
    }
    return triples;
}

/* Threads the products use: the OpenMP build sets and returns n (n <= 0: the default); the
 * plain build returns 1. */
int orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* Tr[X Y] = sum over stored (i, j) of X with (j, i) stored in Y of sum_rc X_ij[r][c] Y_ji[c][r]. */
double orc_trace_xy(int b, int n,
                    const int64_t *x_ptr, const int32_t *x_col, const double *x_val,
                    const int64_t *y_ptr, const int32_t *y_col, const double *y_val)
{
    int64_t bb = (int64_t)b * b;
    double tr = 0.0;
    for (int i = 0; i < n; ++i)
        for (int64_t p = x_ptr[i]; p < x_ptr[i + 1]; ++p) {
            int j = x_col[p];
            int64_t q = orc_find(y_ptr, y_col, j, i);
            if (q < 0) continue;
            const double *xb = x_val + p * bb;
            const double *yb = y_val + q * bb;
            for (int r = 0; r < b; ++r)
                for (int c = 0; c < b; ++c) {
                    double prod = xb[r * b + c] * yb[c * b + r];
                    tr = tr + prod;
                }
        }
    return tr;
}

/* out_ij = (X_ji)^T for every stored (i, j) of 'out'; zero where (j, i) is not stored in X. */
void orc_bsr_transpose(int b, int n,
                       const int64_t *x_ptr, const int32_t *x_col, const double *x_val,
                       const int64_t *o_ptr, const int32_t *o_col, double *o_val)
{
    int64_t bb = (int64_t)b * b;
    for (int i = 0; i < n; ++i)
        for (int64_t p = o_ptr[i]; p < o_ptr[i + 1]; ++p) {
            int j = o_col[p];
            int64_t q = orc_find(x_ptr, x_col, j, i);
            double *ob = o_val + p * bb;
            if (q < 0) {
                memset(ob, 0, sizeof(double) * (size_t)bb);
                continue;
            }
            const double *xb = x_val + q * bb;
            for (int r = 0; r < b; ++r)
                for (int c = 0; c < b; ++c) ob[r * b + c] = xb[c * b + r];
        }
}

/* out_ij = X_ij for every stored (i, j) of 'out'; zero where (i, j) is not stored in X. */
void orc_bsr_restrict(int b, int n,
                      const int64_t *x_ptr, const int32_t *x_col, const double *x_val,
                      const int64_t *o_ptr, const int32_t *o_col, double *o_val)
{
    int64_t bb = (int64_t)b * b;
    for (int i = 0; i < n; ++i)
        for (int64_t p = o_ptr[i]; p < o_ptr[i + 1]; ++p) {
            int64_t q = orc_find(x_ptr, x_col, i, o_col[p]);
            if (q < 0) memset(o_val + p * bb, 0, sizeof(double) * (size_t)bb);
            else memcpy(o_val + p * bb, x_val + q * bb, sizeof(double) * (size_t)bb);
        }
}
