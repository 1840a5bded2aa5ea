// Truncated atom-block products C = alpha op(A) op(B) + beta C on range patterns.
//
// Sec. 2.3.2 of the paper: every matrix of the linear-scaling method is
// sparse by range and every product is restricted to the range of its
// result, so C_ij = sum_k A_ik B_kj is evaluated only for the stored
// blocks (i, j) of C's pattern.  Two kernel forms cover the products of
// an LNV step with little wasted index work:
//
//  * MODE_ROWS ("row Gustavson"): a persistent block owns one row i of C
//    at a time, keeps a chunk of C_i's blocks in shared memory with a
//    shared atom -> slot map, and streams, for every k of row i of A, the
//    blocks B_kj of row k of B into the slots; each warp owns a disjoint
//    range of slots, so the accumulation needs no atomics.
//    Index work ~ sum_{k in A_i} |B_k|: ideal when C holds the natural
//    range of the product (L.S, LS.L, H'.LS).
//  * MODE_INNER: a block owns row i of C with an atom -> position map of
//    row i of A in shared memory; one warp per block (i, j) of C walks
//    column j of B (the pattern is symmetric, so row j of the pattern with
//    the transpose map), looks k up in the map and accumulates in
//    registers, then reduces across the warp.  Index work
//    ~ sum_{j in C_i} |B_j|: ideal when C is truncated well below the
//    natural range (LSL.SL|R_H, Q.LS|R_L).
//
// The plan picks the cheaper form from exact index counts and counts the
// block triples (i, k, j) once per geometry; 2 b^3 per triple is the
// algorithmic flop count.
#include <cuda_runtime.h>

#include <cstdio>
#include <cstdlib>
#include <cstring>

#include <algorithm>
#include <cstdint>
#include <string>

#include "lsq_internal.h"

namespace lsq {

// ---- 4 x 4 block helpers ---------------------------------------------------
__device__ __forceinline__ void ld_blk(const double *__restrict__ p, double (&x)[16]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double2 v = __ldg(q + k);
        x[2 * k] = v.x;
        x[2 * k + 1] = v.y;
    }
}
__device__ __forceinline__ void ld_blk(const float *__restrict__ p, float (&x)[16]) {
    const float4 *q = reinterpret_cast<const float4 *>(p);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        float4 v = __ldg(q + k);
        x[4 * k] = v.x;
        x[4 * k + 1] = v.y;
        x[4 * k + 2] = v.z;
        x[4 * k + 3] = v.w;
    }
}
template <bool TR, typename T>
__device__ __forceinline__ void ld_blk_t(const T *__restrict__ p, T (&x)[16]) {
    ld_blk(p, x);
    if (TR) {
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = r + 1; c < 4; ++c) {
                T t = x[r * 4 + c];
                x[r * 4 + c] = x[c * 4 + r];
                x[c * 4 + r] = t;
            }
    }
}

template <typename T>
__device__ __forceinline__ void warp_sum_u64(unsigned long long v, unsigned long long *out) {
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

struct MMArgs {
    int n;
    const int64_t *a_ptr;
    const int32_t *a_col;
    const int64_t *a_tm;
    const void *A;
    const int64_t *b_ptr;
    const int32_t *b_col;
    const int64_t *b_tm;
    const void *B;
    const int64_t *c_ptr;
    const int32_t *c_col;
    void *C;
    double alpha, beta;
    unsigned long long *triples;
};

// ---- MODE_ROWS, b = 4 --------------------------------------------------------
// First position q in [q0, q1) of a sorted column list with col[q] >= key (whole warp, two
// rounds of 32 probes for rows up to 1024 entries, repeated for longer rows).
__device__ __forceinline__ int64_t warp_lower_bound(const int32_t *__restrict__ col, int64_t q0,
                                                    int64_t q1, int key, int lane) {
    while (q1 - q0 > 32) {
        const int64_t len = q1 - q0;
        const int64_t step = (len + 31) >> 5;
        const int64_t last = q0 + min(len - 1, (int64_t)lane * step + step - 1);
        const bool below = ((int64_t)lane * step < len) && col[last] < key;
        const int nb = __popc(__ballot_sync(0xffffffffu, below));
        const int64_t nq0 = q0 + nb * step;
        q1 = min(q1, nq0 + step);
        q0 = nq0;
    }
    const int64_t pos = q0 + lane;
    const bool below = pos < q1 && col[pos] < key;
    return q0 + __popc(__ballot_sync(0xffffffffu, below));
}

// A persistent block owns row i of C (in chunks of C's blocks kept in shared memory).  Warp w
// owns a contiguous 1/nwarps share of the chunk's slots, i.e. a range [jlo, jhi] of atom
// indices; it walks every k of row i of op(A) and, for each, the segment of row k of op(B)
// inside its j-range, adding A_ik B_kj into its own slots.  Slots are private to a warp and
// distinct within one k, so plain shared-memory read-modify-write suffices (no atomics).
template <typename T, bool TA, bool TB, bool COUNT>
__global__ void __launch_bounds__(512) k_mm_rows_b4(MMArgs g, int chunk) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *acc = reinterpret_cast<T *>(smem_raw);                          // [chunk][16]
    short *map = reinterpret_cast<short *>(acc + (size_t)chunk * 16);  // [n]
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ B = static_cast<const T *>(g.B);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    unsigned long long cnt = 0;
    for (int j = tid; j < g.n; j += nth) map[j] = -1;
    __syncthreads();
    for (int i = blockIdx.x; i < g.n; i += gridDim.x) {
        const int64_t c0 = g.c_ptr[i], c1 = g.c_ptr[i + 1];
        const int64_t a0 = g.a_ptr[i], a1 = g.a_ptr[i + 1];
        for (int64_t s0 = c0; s0 < c1; s0 += chunk) {
            const int nch = (int)min((int64_t)chunk, c1 - s0);
            for (int s = tid; s < nch; s += nth) map[g.c_col[s0 + s]] = (short)s;
            if (!COUNT)
                for (int e = tid; e < nch * 16; e += nth) acc[e] = T(0);
            __syncthreads();
            const int lo = (int)(((int64_t)warp * nch) / nwarps);
            const int hi = (int)(((int64_t)(warp + 1) * nch) / nwarps);
            if (lo < hi) {
                const int jlo = g.c_col[s0 + lo], jhi = g.c_col[s0 + hi - 1];
                for (int64_t pa = a0; pa < a1; ++pa) {
                    const int k = g.a_col[pa];
                    const int64_t qb = g.b_ptr[k], qe = g.b_ptr[k + 1];
                    const int64_t q0 = warp_lower_bound(g.b_col, qb, qe, jlo, lane);
                    if (q0 >= qe || g.b_col[q0] > jhi) continue;
                    T a[16];
                    if (!COUNT) ld_blk_t<TA>(A + 16 * (TA ? g.a_tm[pa] : pa), a);
                    for (int64_t q = q0 + lane; q < qe; q += 32) {
                        const int j = g.b_col[q];
                        if (j > jhi) break;
                        const int slot = map[j];
                        if (slot < 0) continue;
                        if (COUNT) {
                            ++cnt;
                            continue;
                        }
                        T b[16];
                        ld_blk_t<TB>(B + 16 * (TB ? g.b_tm[q] : q), b);
                        T *dst = acc + 16 * slot;
#pragma unroll
                        for (int r = 0; r < 4; ++r)
#pragma unroll
                            for (int c = 0; c < 4; ++c) {
                                T v = dst[r * 4 + c];
                                v = fma(a[r * 4 + 0], b[0 * 4 + c], v);
                                v = fma(a[r * 4 + 1], b[1 * 4 + c], v);
                                v = fma(a[r * 4 + 2], b[2 * 4 + c], v);
                                v = fma(a[r * 4 + 3], b[3 * 4 + c], v);
                                dst[r * 4 + c] = v;
                            }
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            if (!COUNT) {
                const T al = (T)g.alpha, be = (T)g.beta;
                for (int e = tid; e < nch * 16; e += nth) {
                    T v = al * acc[e];
                    if (g.beta != 0.0) v = fma(be, C[16 * s0 + e], v);
                    C[16 * s0 + e] = v;
                }
            }
            for (int s = tid; s < nch; s += nth) map[g.c_col[s0 + s]] = -1;
            __syncthreads();
        }
    }
    if (COUNT) warp_sum_u64<T>(cnt, g.triples);
}

// ---- MODE_INNER, b = 4 -------------------------------------------------------
template <typename T, bool TA, bool TB, bool COUNT>
__global__ void __launch_bounds__(512) k_mm_inner_b4(MMArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *amap = reinterpret_cast<int *>(smem_raw);  // [n] offset in row i of A, or -1
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ B = static_cast<const T *>(g.B);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    unsigned long long cnt = 0;
    for (int j = tid; j < g.n; j += nth) amap[j] = -1;
    __syncthreads();
    for (int i = blockIdx.x; i < g.n; i += gridDim.x) {
        const int64_t a0 = g.a_ptr[i], a1 = g.a_ptr[i + 1];
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[g.a_col[p]] = (int)(p - a0);
        __syncthreads();
        for (int64_t s = g.c_ptr[i] + warp; s < g.c_ptr[i + 1]; s += nwarps) {
            const int j = g.c_col[s];
            T acc[16];
#pragma unroll
            for (int e = 0; e < 16; ++e) acc[e] = T(0);
            const int64_t q1 = g.b_ptr[j + 1];
            for (int64_t q = g.b_ptr[j] + lane; q < q1; q += 32) {
                const int k = g.b_col[q];
                const int off = amap[k];
                if (off < 0) continue;
                if (COUNT) {
                    ++cnt;
                    continue;
                }
                const int64_t pa = a0 + off;
                T a[16], b[16];
                ld_blk_t<TA>(A + 16 * (TA ? g.a_tm[pa] : pa), a);
                // (k, j) of op(B): for B it sits at the transpose position of (j, k);
                // for B^T it is (B_jk)^T, which sits at q itself.
                ld_blk_t<TB>(B + 16 * (TB ? q : g.b_tm[q]), b);
#pragma unroll
                for (int r = 0; r < 4; ++r)
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        T v = acc[r * 4 + c];
                        v = fma(a[r * 4 + 0], b[0 * 4 + c], v);
                        v = fma(a[r * 4 + 1], b[1 * 4 + c], v);
                        v = fma(a[r * 4 + 2], b[2 * 4 + c], v);
                        v = fma(a[r * 4 + 3], b[3 * 4 + c], v);
                        acc[r * 4 + c] = v;
                    }
            }
            if (!COUNT) {
#pragma unroll
                for (int e = 0; e < 16; ++e)
#pragma unroll
                    for (int off = 16; off > 0; off >>= 1)
                        acc[e] += __shfl_xor_sync(0xffffffffu, acc[e], off);
                T mine = acc[0];
#pragma unroll
                for (int e = 1; e < 16; ++e)
                    if (lane == e) mine = acc[e];
                if (lane < 16) {
                    T v = (T)g.alpha * mine;
                    if (g.beta != 0.0) v = fma((T)g.beta, C[16 * s + lane], v);
                    C[16 * s + lane] = v;
                }
            }
        }
        __syncthreads();
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[g.a_col[p]] = -1;
        __syncthreads();
    }
    if (COUNT) warp_sum_u64<T>(cnt, g.triples);
}

// ---- MODE_INNER, any b <= 16 (one warp per C block, elements over lanes) ----
template <typename T, bool TA, bool TB, bool COUNT>
__global__ void __launch_bounds__(256) k_mm_inner_gen(MMArgs g, int b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    int *amap = reinterpret_cast<int *>(smem_raw);
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ B = static_cast<const T *>(g.B);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    const int bb = b * b;
    unsigned long long cnt = 0;
    for (int j = tid; j < g.n; j += nth) amap[j] = -1;
    __syncthreads();
    for (int i = blockIdx.x; i < g.n; i += gridDim.x) {
        const int64_t a0 = g.a_ptr[i], a1 = g.a_ptr[i + 1];
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[g.a_col[p]] = (int)(p - a0);
        __syncthreads();
        for (int64_t s = g.c_ptr[i] + warp; s < g.c_ptr[i + 1]; s += nwarps) {
            const int j = g.c_col[s];
            T acc[8];
#pragma unroll
            for (int m = 0; m < 8; ++m) acc[m] = T(0);
            const int64_t q0 = g.b_ptr[j], q1 = g.b_ptr[j + 1];
            for (int64_t qb = q0; qb < q1; qb += 32) {
                const int64_t q = qb + lane;
                int off = -1;
                if (q < q1) off = amap[g.b_col[q]];
                unsigned mask = __ballot_sync(0xffffffffu, off >= 0);
                if (COUNT) {
                    if (lane == 0) cnt += __popc(mask);
                    continue;
                }
                while (mask) {
                    const int src = __ffs(mask) - 1;
                    mask &= mask - 1;
                    const int o = __shfl_sync(0xffffffffu, off, src);
                    const int64_t qq = qb + src;
                    const int64_t pa = a0 + o;
                    const T *ab = A + (size_t)bb * (TA ? g.a_tm[pa] : pa);
                    const T *bp = B + (size_t)bb * (TB ? qq : g.b_tm[qq]);
#pragma unroll
                    for (int m = 0; m < 8; ++m) {
                        const int e = lane + 32 * m;
                        if (e < bb) {
                            const int r = e / b, c = e % b;
                            T v = acc[m];
                            for (int t = 0; t < b; ++t) {
                                T x = TA ? ab[t * b + r] : ab[r * b + t];
                                T y = TB ? bp[c * b + t] : bp[t * b + c];
                                v = fma(x, y, v);
                            }
                            acc[m] = v;
                        }
                    }
                }
            }
            if (!COUNT) {
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int e = lane + 32 * m;
                    if (e < bb) {
                        T v = (T)g.alpha * acc[m];
                        if (g.beta != 0.0) v = fma((T)g.beta, C[(size_t)bb * s + e], v);
                        C[(size_t)bb * s + e] = v;
                    }
                }
            }
        }
        __syncthreads();
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[g.a_col[p]] = -1;
        __syncthreads();
    }
    if (COUNT) warp_sum_u64<T>(cnt, g.triples);
}

// out_ij = (X_ji)^T on one symmetric pattern (tm = transpose map of the pattern).
// B > 0 fixes the block size at compile time (index arithmetic by shifts for B = 4).
template <typename T, int B>
__global__ void k_transpose_pattern(int64_t nnzb, int b_rt, const int64_t *__restrict__ tm,
                                    const T *__restrict__ X, T *__restrict__ out) {
    const int b = B > 0 ? B : b_rt;
    const uint64_t bb = (uint64_t)(b * b);
    const uint64_t m = (uint64_t)nnzb * bb;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = e / bb;
        const int rc = (int)(e - p * bb);
        const int r = rc / b, c = rc - r * b;
        out[e] = X[tm[p] * (int64_t)bb + c * b + r];
    }
}

static int tgrid(int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 8192)); }

// X^T on pattern r (materialised so that later products read it row by row).
int transpose_on(lsq_geom g, int r, int b, int prec, const void *X, void *out,
                        cudaStream_t s) {
    LSQ_TRY(ensure_tmap(g, r, s));
    int64_t m = g->pats[r].nnzb * b * b;
    note_launch();
    auto go = [&](auto kern, auto *x, auto *o) { kern<<<tgrid(m), 256, 0, s>>>(g->pats[r].nnzb, b, g->pats[r].tmap.p, x, o); };
    if (prec == LSQ_F64) {
        if (b == 4) go(k_transpose_pattern<double, 4>, (const double *)X, (double *)out);
        else go(k_transpose_pattern<double, 0>, (const double *)X, (double *)out);
    } else {
        if (b == 4) go(k_transpose_pattern<float, 4>, (const float *)X, (float *)out);
        else go(k_transpose_pattern<float, 0>, (const float *)X, (float *)out);
    }
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

// out_ij = X_ij + (X_ji)^T on one symmetric pattern; element (r, c) and its mirror (c, r) of the
// mirrored block add the same two values (addition commutes), so out is symmetric to the last bit.
template <typename T, int B>
__global__ void k_sym_sum(int64_t nnzb, int b_rt, const int64_t *__restrict__ tm, const T *__restrict__ X,
                          T *__restrict__ out) {
    const int b = B > 0 ? B : b_rt;
    const uint64_t bb = (uint64_t)(b * b);
    const uint64_t m = (uint64_t)nnzb * bb;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t p = e / bb;
        const int rc = (int)(e - p * bb);
        const int r = rc / b, c = rc - r * b;
        out[e] = X[e] + X[tm[p] * (int64_t)bb + c * b + r];
    }
}

int sym_sum_on(lsq_geom g, int r, int b, int prec, const void *X, void *out, cudaStream_t s) {
    LSQ_TRY(ensure_tmap(g, r, s));
    int64_t m = g->pats[r].nnzb * b * b;
    note_launch();
    auto go = [&](auto kern, auto *x, auto *o) { kern<<<tgrid(m), 256, 0, s>>>(g->pats[r].nnzb, b, g->pats[r].tmap.p, x, o); };
    if (prec == LSQ_F64) {
        if (b == 4) go(k_sym_sum<double, 4>, (const double *)X, (double *)out);
        else go(k_sym_sum<double, 0>, (const double *)X, (double *)out);
    } else {
        if (b == 4) go(k_sym_sum<float, 4>, (const float *)X, (float *)out);
        else go(k_sym_sum<float, 0>, (const float *)X, (float *)out);
    }
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

// Diagonal blocks of a symmetric result formed as upper triangle + mirror: the lower element of
// each pair inside a diagonal block takes the upper one, so the whole matrix is symmetric to
// the last bit (the product computes the two elements of such a pair separately).
template <typename T>
__global__ void k_sym_diag_blocks(int64_t nnzb, int b, const int64_t *__restrict__ tm, T *__restrict__ U) {
    const int bb = b * b;
    const int64_t m = nnzb * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / bb;
        if (tm[p] != p) continue;
        const int rc = (int)(e - p * bb), r = rc / b, c = rc - r * b;
        if (r > c) U[e] = U[p * bb + c * b + r];
    }
}

int sym_diag_on(lsq_geom g, int r, int b, int prec, void *X, cudaStream_t s) {
    LSQ_TRY(ensure_tmap(g, r, s));
    const int64_t m = g->pats[r].nnzb * b * b;
    note_launch();
    if (prec == LSQ_F64)
        k_sym_diag_blocks<double><<<tgrid(m), 256, 0, s>>>(g->pats[r].nnzb, b, g->pats[r].tmap.p, (double *)X);
    else
        k_sym_diag_blocks<float><<<tgrid(m), 256, 0, s>>>(g->pats[r].nnzb, b, g->pats[r].tmap.p, (float *)X);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

// ---- index-cost estimate of the two forms ---------------------------------
__global__ void k_mm_cost(int n, const int64_t *__restrict__ a_ptr, const int32_t *__restrict__ a_col,
                          const int64_t *__restrict__ b_ptr, const int64_t *__restrict__ c_ptr,
                          const int32_t *__restrict__ c_col, int chunk,
                          unsigned long long *__restrict__ out) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    int i = warp;
    unsigned long long rows = 0, inner = 0;
    for (int64_t p = a_ptr[i] + lane; p < a_ptr[i + 1]; p += 32) {
        int k = a_col[p];
        rows += (unsigned long long)(b_ptr[k + 1] - b_ptr[k]);
    }
    for (int64_t s = c_ptr[i] + lane; s < c_ptr[i + 1]; s += 32) {
        int j = c_col[s];
        inner += (unsigned long long)(b_ptr[j + 1] - b_ptr[j]);
    }
    int64_t nchunks = (c_ptr[i + 1] - c_ptr[i] + chunk - 1) / chunk;
    rows *= (unsigned long long)(nchunks > 0 ? nchunks : 1);
    for (int off = 16; off > 0; off >>= 1) {
        rows += __shfl_xor_sync(0xffffffffu, rows, off);
        inner += __shfl_xor_sync(0xffffffffu, inner, off);
    }
    if (lane == 0) {
        atomicAdd(&out[0], rows);
        atomicAdd(&out[1], inner);
    }
}

template <typename K>
static int occupancy_grid(lsq_geom g, K kern, int threads, size_t smem) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    per_sm = std::max(per_sm, 1);
    return std::max(1, std::min(g->n, g->num_sms * per_sm));
}

static int rows_chunk(lsq_geom g, int dtype) {
    // shared memory: chunk * 16 * sizeof(T) + n * sizeof(short)
    size_t avail = g->smem_optin > 2048 ? g->smem_optin - 1024 : 0;
    size_t map = (size_t)g->n * sizeof(short);
    if (avail <= map) return 0;
    size_t c = (avail - map) / (16 * dtype_size(dtype));
    return (int)std::min<size_t>(c, 32767);
}

template <typename T, bool TA, bool TB, bool COUNT>
static int launch_typed(lsq_geom g, int b, int mode, int chunk, const MMArgs &a, cudaStream_t s) {
    if (b == 4 && mode == MODE_ROWS) {
        auto kern = k_mm_rows_b4<T, TA, TB, COUNT>;
        size_t smem = (size_t)chunk * 16 * sizeof(T) + (size_t)g->n * sizeof(short);
        LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int threads = 512;
        int grid = occupancy_grid(g, kern, threads, smem);
        note_launch();
        kern<<<grid, threads, smem, s>>>(a, chunk);
    } else if (b == 4) {
        auto kern = k_mm_inner_b4<T, TA, TB, COUNT>;
        size_t smem = (size_t)g->n * sizeof(int);
        LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int threads = 512;
        int grid = occupancy_grid(g, kern, threads, smem);
        note_launch();
        kern<<<grid, threads, smem, s>>>(a);
    } else {
        auto kern = k_mm_inner_gen<T, TA, TB, COUNT>;
        size_t smem = (size_t)g->n * sizeof(int);
        LSQ_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        int threads = 256;
        int grid = occupancy_grid(g, kern, threads, smem);
        note_launch();
        kern<<<grid, threads, smem, s>>>(a, b);
    }
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

template <typename T, bool COUNT>
static int launch_mm(lsq_geom g, int b, int mode, int chunk, int ta, int tb, const MMArgs &a,
                     cudaStream_t s) {
    if (ta && tb) return launch_typed<T, true, true, COUNT>(g, b, mode, chunk, a, s);
    if (ta) return launch_typed<T, true, false, COUNT>(g, b, mode, chunk, a, s);
    if (tb) return launch_typed<T, false, true, COUNT>(g, b, mode, chunk, a, s);
    return launch_typed<T, false, false, COUNT>(g, b, mode, chunk, a, s);
}

static int get_plan(lsq_geom g, int b, int dtype, int ra, int ta, int rb, int tb, int rc,
                    const MMArgs &base, Plan **out, cudaStream_t s) {
    auto key = std::make_tuple(ra, ta, rb, tb, rc, b, dtype);
    auto it = g->plans.find(key);
    if (it != g->plans.end()) {
        *out = &it->second;
        return LSQ_OK;
    }
    Plan p;
    const Pattern &PA = g->pats[ra], &PB = g->pats[rb], &PC = g->pats[rc];
    p.chunk = rows_chunk(g, dtype);
    DevBuf<unsigned long long> cnt;
    LSQ_TRY(cnt.alloc(3));
    LSQ_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, 3 * sizeof(unsigned long long), s));
    unsigned long long h[3] = {0, 0, 0};
    if (g->n > 0) {
        int threads = 256;
        int blocks = (int)(((int64_t)g->n * 32 + threads - 1) / threads);
        note_launch();
        k_mm_cost<<<blocks, threads, 0, s>>>(g->n, PA.row_ptr.p, PA.col.p, PB.row_ptr.p,
                                             PC.row_ptr.p, PC.col.p, std::max(p.chunk, 1), cnt.p);
        LSQ_CHECK_LAUNCH();
        LSQ_CUDA_TRY(cudaMemcpyAsync(h, cnt.p, 2 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    bool rows_ok = (b == 4) && p.chunk >= 64;
    p.mode = (rows_ok && h[0] <= h[1]) ? MODE_ROWS : MODE_INNER;
    if (p.mode == MODE_INNER && (size_t)g->n * sizeof(int) + 1024 > g->smem_optin)
        return set_error(LSQ_ERR_UNSUPPORTED, "too many atoms for the shared-memory atom map");
    if (p.mode == MODE_ROWS && PC.max_row > 0 && p.chunk < 1)
        return set_error(LSQ_ERR_UNSUPPORTED, "too many atoms for the shared-memory slot map");
    // exact triple count
    MMArgs a = base;
    a.triples = cnt.p + 2;
    if (g->n > 0) {
        int rc2 = dtype == LSQ_F64 ? launch_mm<double, true>(g, b, p.mode, p.chunk, ta, tb, a, s)
                                   : launch_mm<float, true>(g, b, p.mode, p.chunk, ta, tb, a, s);
        if (rc2) return rc2;
        LSQ_CUDA_TRY(cudaMemcpyAsync(&h[2], cnt.p + 2, sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    p.triples = (int64_t)h[2];
    *out = &g->plans.emplace(key, p).first->second;
    return LSQ_OK;
}

int mixed_choice(lsq_geom g, int ra, int rb, int rc, int sym, double beta) {
    const int upper = sym == 3 ? 2 : (sym == 2 || (sym == 1 && beta == 0.0) ? 1 : 0);
    auto ch = g->tc_choice.find(std::make_tuple(ra, rb, rc + 1000 * upper));
    return ch == g->tc_choice.end() ? -1 : ch->second.choice;
}

int block_matmul(lsq_geom g, int b, int dtype, int ra, int ta, const void *A, int rb, int tb,
                 const void *B, int rc, void *C, double alpha, double beta, int64_t *triples,
                 cudaStream_t s, int sym) {
    LSQ_TRY(geom_check(g, ra));
    LSQ_TRY(geom_check(g, rb));
    LSQ_TRY(geom_check(g, rc));
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (dtype != LSQ_F64 && dtype != LSQ_F32 && dtype != LSQ_TF32X3 && dtype != kMixedAuto)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64, LSQ_F32 or LSQ_TF32X3");
    if (dtype == kMixedAuto) {
        // the faster of the FP32 FMA schedules and the tensor-core kernel for this product,
        // timed on its first call with beta = 0 and remembered by g; the losing kernel's plan
        // is dropped (a later explicit call of that precision builds it again)
        if (b != 4 || g->n == 0) {
            dtype = LSQ_F32;
        } else {
            const int upper = sym == 3 ? 2 : (sym == 2 || (sym == 1 && beta == 0.0) ? 1 : 0);
            const auto key = std::make_tuple(ra, rb, rc + 1000 * upper);
            auto ch = g->tc_choice.find(key);
            if (ch == g->tc_choice.end()) {
                // a fixed choice instead of the timing (profiler runs, whose serialised launches
                // distort it): LSQ_TC_CHOICE="ra:rb:rc:tri=k,...,all=k", k = 1 tensor cores, 0 FMA,
                // tri the triangle code of the plans (0 all, 1 upper, 2 lower)
                if (const char *env = std::getenv("LSQ_TC_CHOICE")) {
                    int fixed = -1;
                    for (const char *q = env; *q;) {
                        int a0, a1, a2, a3, k;
                        if (std::sscanf(q, "%d:%d:%d:%d=%d", &a0, &a1, &a2, &a3, &k) == 5) {
                            if (a0 == ra && a1 == rb && a2 == rc && a3 == upper) fixed = k;
                        } else if (std::sscanf(q, "all=%d", &k) == 1) {
                            if (fixed < 0) fixed = k;
                        }
                        const char *c = std::strchr(q, ',');
                        if (!c) break;
                        q = c + 1;
                    }
                    if (fixed >= 0) ch = g->tc_choice.emplace(key, TcChoice{fixed ? 1 : 0, {0.f, 0.f}}).first;
                }
            }
            if (ch != g->tc_choice.end()) {
                dtype = ch->second.choice == 1 ? LSQ_TF32X3 : LSQ_F32;
            } else if (beta != 0.0) {
                dtype = LSQ_F32;  // no timing run on an accumulating call: FMA until timed
            } else {
                TcPlan *tp = nullptr;
                const int prc = tc_plan_get(g, ra, rb, rc, upper, &tp, s);
                if (prc == LSQ_ERR_OOM || prc == LSQ_ERR_UNSUPPORTED) {
                    (void)cudaGetLastError();
                    clear_error();
                    g->tc_choice[key] = TcChoice{0, {0.f, 0.f}};
                    dtype = LSQ_F32;
                } else if (prc != LSQ_OK) {
                    return prc;
                } else {
                    const int64_t tr = tp->triples;
                    // time each once more after its own first call (plan, tuning) has run
                    cudaEvent_t e0, e1;
                    LSQ_CUDA_TRY(cudaEventCreate(&e0));
                    LSQ_CUDA_TRY(cudaEventCreate(&e1));
                    float ms[2] = {0.f, 0.f};
                    for (int k = 0; k < 2; ++k) {
                        const int pk = k == 0 ? LSQ_F32 : LSQ_TF32X3;
                        LSQ_TRY(block_matmul(g, b, pk, ra, ta, A, rb, tb, B, rc, C, alpha, beta, nullptr, s, sym));
                        LSQ_CUDA_TRY(cudaEventRecord(e0, s));
                        LSQ_TRY(block_matmul(g, b, pk, ra, ta, A, rb, tb, B, rc, C, alpha, beta, nullptr, s, sym));
                        LSQ_CUDA_TRY(cudaEventRecord(e1, s));
                        LSQ_CUDA_TRY(cudaEventSynchronize(e1));
                        LSQ_CUDA_TRY(cudaEventElapsedTime(&ms[k], e0, e1));
                    }
                    cudaEventDestroy(e0);
                    cudaEventDestroy(e1);
                    const int choice = ms[1] < ms[0] ? 1 : 0;
                    g->tc_choice[key] = TcChoice{choice, {ms[0], ms[1]}};
                    if (std::getenv("LSQ_TUNE_LOG"))
                        std::fprintf(stderr, "lsq autotune: ranges (%g, %g, %g) tri %d: FP32 FMA %.3f ms, TF32X3 %.3f ms -> %s\n",
                                     g->pats[ra].R, g->pats[rb].R, g->pats[rc].R, upper, ms[0], ms[1],
                                     choice ? "tensor cores" : "FMA");
                    if (choice == 1)
                        g->pplans.erase(key);   // the FMA plan of this product is not needed any more
                    else
                        g->tcplans.erase(key);  // nor the tensor-core plan (tp is invalid from here)
                    if (triples) *triples = tr;
                    return LSQ_OK;  // C holds the product (both runs wrote the same result)
                }
            }
        }
    }
    if (g->n > 0 && (!A || !B || !C)) return set_error(LSQ_ERR_INVALID_ARG, "null matrix pointer");
    if (g->n > 0 && (C == A || C == B)) return set_error(LSQ_ERR_INVALID_ARG, "C must not alias A or B");
    if (dtype == LSQ_TF32X3) {
        // float32 storage; 4 x 4 blocks contract on the tensor cores in split TF32, other block
        // sizes on the float32 FMA kernels
        if (b == 4) {
            const int upper = sym == 3 ? 2 : (sym == 2 || (sym == 1 && beta == 0.0) ? 1 : 0);
            return tc_block_matmul(g, ra, ta, static_cast<const float *>(A), rb, tb, static_cast<const float *>(B),
                                   rc, static_cast<float *>(C), alpha, beta, upper, sym == 1, triples, s);
        }
        dtype = LSQ_F32;
    }
    // transposed operands and MODE_INNER read through transpose maps
    LSQ_TRY(ensure_tmap(g, ra, s));
    LSQ_TRY(ensure_tmap(g, rb, s));
    MMArgs a;
    a.n = g->n;
    a.a_ptr = g->pats[ra].row_ptr.p;
    a.a_col = g->pats[ra].col.p;
    a.a_tm = g->pats[ra].tmap.p;
    a.A = A;
    a.b_ptr = g->pats[rb].row_ptr.p;
    a.b_col = g->pats[rb].col.p;
    a.b_tm = g->pats[rb].tmap.p;
    a.B = B;
    a.c_ptr = g->pats[rc].row_ptr.p;
    a.c_col = g->pats[rc].col.p;
    a.C = C;
    a.alpha = alpha;
    a.beta = beta;
    a.triples = nullptr;
    // the 4 x 4 kernels read blocks in 16-byte vectors; other matrices take the general kernel
    const bool al16 = (reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B) |
                       reinterpret_cast<uintptr_t>(C)) % 16 == 0;
    if (b == 4 && al16) {
        // plan-driven form: op(A) rows and op(B)^T rows, transposing into scratch if needed
        ProductPlan *pp = nullptr;
        int prc = plan_build(g, ra, rb, rc, sym == 3 ? 2 : (sym == 2 || (sym == 1 && beta == 0.0) ? 1 : 0), &pp, s);
        if (prc == LSQ_OK) {
            if (triples) *triples = pp->triples;
            if (g->n == 0 || g->pats[rc].nnzb == 0) return LSQ_OK;
            const size_t es = 16 * dtype_size(dtype);
            const void *Aop = A, *X = B;
            if (ta) {
                size_t need = es * (size_t)g->pats[ra].nnzb;
                if (g->scratch_a.n < need) LSQ_TRY(g->scratch_a.alloc(need));
                LSQ_TRY(transpose_on(g, ra, b, dtype, A, g->scratch_a.p, s));
                Aop = g->scratch_a.p;
            }
            if (!tb) {
                size_t need = es * (size_t)g->pats[rb].nnzb;
                if (g->scratch_x.n < need) LSQ_TRY(g->scratch_x.alloc(need));
                LSQ_TRY(transpose_on(g, rb, b, dtype, B, g->scratch_x.p, s));
                X = g->scratch_x.p;
            }
            const int di = dtype == LSQ_F64 ? 0 : 1;
            if (pp->variant[di] < 0 && !g->schedule_hints.empty()) {
                // a schedule adopted from a geometry of the same ranges: no tuning run
                const int upper = sym == 3 ? 2 : (sym == 2 || (sym == 1 && beta == 0.0) ? 1 : 0);
                auto h = g->schedule_hints.find(std::make_tuple(ra, rb, rc + 1000 * upper));
                if (h != g->schedule_hints.end() && h->second[di] >= 0) {
                    pp->variant[di] = h->second[di];
                    pp->variant16[di] = h->second[2 + di];
                }
            }
            return plan_launch(g, dtype, *pp, ra, rb, rc, Aop, X, C, alpha, beta, s, sym == 1);
        }
        if (prc != LSQ_ERR_OOM && prc != LSQ_ERR_UNSUPPORTED) return prc;
        (void)cudaGetLastError();  // a failed allocation is not sticky; drop it
        clear_error();             // and fall back to the plan-free forms below
    } else {
        // any other block size (or unaligned 4 x 4 blocks): warp-per-block kernel, no scratch
        ProductPlan *pp = nullptr;
        int prc = plan_build(g, ra, rb, rc, sym == 3 ? 2 : (sym == 2 || (sym == 1 && beta == 0.0) ? 1 : 0), &pp, s);
        if (prc == LSQ_OK) {
            if (triples) *triples = pp->triples;
            if (g->n == 0 || g->pats[rc].nnzb == 0) return LSQ_OK;
            return plan_launch_gen(g, b, dtype, *pp, ra, ta, rb, tb, rc, A, B, C, alpha, beta, s, sym == 1);
        }
        if (prc != LSQ_ERR_OOM && prc != LSQ_ERR_UNSUPPORTED) return prc;
        (void)cudaGetLastError();
        clear_error();
    }
    if (b == 4 && !al16)
        return set_error(LSQ_ERR_OOM, "no device memory for a product plan, and the plan-free 4 x 4 "
                                      "kernels need 16-byte aligned matrices");
    Plan *p = nullptr;
    LSQ_TRY(get_plan(g, b, dtype, ra, ta, rb, tb, rc, a, &p, s));
    if (triples) *triples = p->triples;
    if (g->n == 0 || g->pats[rc].nnzb == 0) return LSQ_OK;
    return dtype == LSQ_F64 ? launch_mm<double, false>(g, b, p->mode, p->chunk, ta, tb, a, s)
                            : launch_mm<float, false>(g, b, p->mode, p->chunk, ta, tb, a, s);
}

// ---- reductions: traces and dots in float64 --------------------------------
constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

int reducer_ensure(lsq_geom g, int nslots) {
    if (g->red.partial.p && (int)g->red.scalars.n >= nslots) return LSQ_OK;
    LSQ_TRY(g->red.partial.alloc(kRedBlocks));
    LSQ_TRY(g->red.scalars.alloc(std::max(nslots, 16)));
    if (!g->red.host) {
        LSQ_CUDA_TRY(cudaMallocHost(&g->red.host, sizeof(double) * 64));
    }
    g->red.nblocks = kRedBlocks;
    return LSQ_OK;
}

__device__ __forceinline__ double block_sum(double v) {
    __shared__ double sh[32];
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x < 32) {
        r = threadIdx.x < (blockDim.x >> 5) ? sh[threadIdx.x] : 0.0;
        for (int off = 16; off > 0; off >>= 1) r += __shfl_xor_sync(0xffffffffu, r, off);
    }
    __syncthreads();
    return r;
}

// Tr[X Y]: sum over entries p of X with q = pm[p] >= 0 of sum_rc X_p[r][c] Y_q[c][r].
template <typename T>
__global__ void k_trace(int64_t nnzb, int b, const T *__restrict__ X, const T *__restrict__ Y,
                        const int64_t *__restrict__ pm, double *__restrict__ partial) {
    const int bb = b * b;
    double s = 0.0;
    int64_t total = nnzb * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = e / bb;
        int rc = (int)(e - p * bb);
        int64_t q = pm[p];
        if (q < 0) continue;
        int r = rc / b, c = rc - r * b;
        s += (double)X[e] * (double)Y[q * bb + c * b + r];
    }
    double t = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

template <typename T>
__global__ void k_dot(int64_t total, const T *__restrict__ X, const T *__restrict__ Y,
                      double *__restrict__ partial) {
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x)
        s += (double)X[e] * (double)Y[e];
    double t = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

// Float32 dot product accumulated without a float64 operation per element (the float64 pipe
// is 1/64 of the float32 one): each thread forms 8 products exactly as float pairs (TwoProduct
// with an FMA) and sums them with error-free TwoSum steps (Knuth; the Dot2 scheme of Ogita,
// Rump and Oishi, 2005), then adds the pair to a float64 accumulator.  Each group of 8 is
// summed as if in twice the float32 precision, so the result matches float64 accumulation of
// the exact products to well below float32 rounding.  X and Y must be 16-byte aligned.
__device__ __forceinline__ double dot8_exact(const float4 a0, const float4 a1, const float4 b0,
                                             const float4 b1) {
    const float x[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
    const float y[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    float s = 0.f, c = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) dot2_add(x[k], y[k], s, c);
    return (double)s + (double)c;
}

__global__ void k_dot_f32(int64_t total, const float *__restrict__ X, const float *__restrict__ Y,
                          double *__restrict__ partial) {
    double s = 0.0;
    const int64_t n8 = total / 8;
    const float4 *__restrict__ X4 = reinterpret_cast<const float4 *>(X);
    const float4 *__restrict__ Y4 = reinterpret_cast<const float4 *>(Y);
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n8;
         q += (int64_t)gridDim.x * blockDim.x)
        s += dot8_exact(__ldg(X4 + 2 * q), __ldg(X4 + 2 * q + 1), __ldg(Y4 + 2 * q), __ldg(Y4 + 2 * q + 1));
    // the last total % 8 values
    const int64_t e = n8 * 8 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < total) s += (double)X[e] * (double)Y[e];
    double t = block_sum(s);
    if (threadIdx.x == 0) partial[blockIdx.x] = t;
}

__global__ void k_finish(const double *__restrict__ partial, int m, double *__restrict__ out) {
    double s = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) s += partial[k];
    double t = block_sum(s);
    if (threadIdx.x == 0) *out = t;
}

int trace_into(lsq_geom g, int b, int dtype, int rx, const void *X, int ry, const void *Y, int slot,
               cudaStream_t s) {
    LSQ_TRY(reducer_ensure(g, slot + 1));
    const int64_t *pm = nullptr;
    LSQ_TRY(get_posmap(g, rx, ry, 1, &pm, s));
    int64_t nnzb = g->pats[rx].nnzb;
    if (dtype == LSQ_F64) {
        note_launch();
        k_trace<double><<<kRedBlocks, kRedThreads, 0, s>>>(nnzb, b, (const double *)X,
                                                           (const double *)Y, pm, g->red.partial.p);
    } else {
        note_launch();
        k_trace<float><<<kRedBlocks, kRedThreads, 0, s>>>(nnzb, b, (const float *)X,
                                                          (const float *)Y, pm, g->red.partial.p);
    }
    note_launch();
    k_finish<<<1, 1024, 0, s>>>(g->red.partial.p, kRedBlocks, g->red.scalars.p + slot);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

int dot_into(lsq_geom g, int b, int dtype, int r, const void *X, const void *Y, int slot,
             cudaStream_t s) {
    LSQ_TRY(reducer_ensure(g, slot + 1));
    int64_t total = g->pats[r].nnzb * b * b;
    if (dtype == LSQ_F64) {
        note_launch();
        k_dot<double><<<kRedBlocks, kRedThreads, 0, s>>>(total, (const double *)X, (const double *)Y,
                                                         g->red.partial.p);
    } else if ((reinterpret_cast<uintptr_t>(X) | reinterpret_cast<uintptr_t>(Y)) % 16 == 0) {
        note_launch();
        k_dot_f32<<<kRedBlocks, kRedThreads, 0, s>>>(total, (const float *)X, (const float *)Y,
                                                     g->red.partial.p);
    } else {
        note_launch();
        k_dot<float><<<kRedBlocks, kRedThreads, 0, s>>>(total, (const float *)X, (const float *)Y,
                                                        g->red.partial.p);
    }
    note_launch();
    k_finish<<<1, 1024, 0, s>>>(g->red.partial.p, kRedBlocks, g->red.scalars.p + slot);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

int sum_into(lsq_geom g, const double *x, int64_t m, int slot, cudaStream_t s) {
    LSQ_TRY(reducer_ensure(g, slot + 1));
    note_launch();
    k_finish<<<1, 1024, 0, s>>>(x, (int)m, g->red.scalars.p + slot);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

int fetch_scalars(lsq_geom g, int nslots, double *out, cudaStream_t s) {
    LSQ_CUDA_TRY(cudaMemcpyAsync(g->red.host, g->red.scalars.p, sizeof(double) * nslots,
                                 cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    for (int k = 0; k < nslots; ++k) out[k] = g->red.host[k];
    return LSQ_OK;
}

}  // namespace lsq

using namespace lsq;

extern "C" int lsq_block_matmul(lsq_geom g, int b, int precision, int range_a, int trans_a,
                                const void *A, int range_b, int trans_b, const void *B, int range_c,
                                void *C, double alpha, double beta, int64_t *n_triples,
                                void *stream) {
    clear_error();
    return block_matmul(g, b, precision, range_a, trans_a != 0, A, range_b, trans_b != 0, B, range_c,
                        C, alpha, beta, n_triples, (cudaStream_t)stream);
}

extern "C" int lsq_block_matmul_tri(lsq_geom g, int b, int precision, int range_a, int trans_a,
                                    const void *A, int range_b, int trans_b, const void *B, int range_c,
                                    void *C, double alpha, double beta, int triangle, int64_t *n_triples,
                                    void *stream) {
    clear_error();
    if (triangle < 0 || triangle > 3) return set_error(LSQ_ERR_INVALID_ARG, "triangle must be 0, 1, 2 or 3");
    if (triangle == 1 && beta != 0.0)
        return set_error(LSQ_ERR_INVALID_ARG, "triangle 1 (symmetric result) needs beta = 0");
    return block_matmul(g, b, precision, range_a, trans_a != 0, A, range_b, trans_b != 0, B, range_c,
                        C, alpha, beta, n_triples, (cudaStream_t)stream, triangle);
}

extern "C" int lsq_trace(lsq_geom g, int b, int precision, int range_x, const void *X, int range_y,
                         const void *Y, double *out, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g, range_x));
    LSQ_TRY(geom_check(g, range_y));
    if (!out) return set_error(LSQ_ERR_INVALID_ARG, "out is null");
    if (precision != LSQ_F64 && precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64 or LSQ_F32");
    cudaStream_t s = (cudaStream_t)stream;
    LSQ_TRY(trace_into(g, b, precision, range_x, X, range_y, Y, 0, s));
    return fetch_scalars(g, 1, out, s);
}

namespace lsq {

// out_ij = alpha (X_ji)^T where (j, i) is stored in X's pattern, else 0 (pm: transposed posmap).
template <typename T>
__global__ void k_transpose_into(int64_t nnzb, int b, const int64_t *__restrict__ pm, T alpha,
                                 const T *__restrict__ X, T *__restrict__ out) {
    const int bb = b * b;
    const int64_t m = nnzb * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / bb;
        const int rc = (int)(e - p * bb);
        const int r = rc / b, c = rc - r * b;
        const int64_t q = pm[p];
        out[e] = q >= 0 ? alpha * X[q * bb + c * b + r] : T(0);
    }
}

}  // namespace lsq

extern "C" int lsq_transpose(lsq_geom g, int b, int precision, int range_x, const void *X,
                             int range_out, void *out, double alpha, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g, range_x));
    LSQ_TRY(geom_check(g, range_out));
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (precision != LSQ_F64 && precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64 or LSQ_F32");
    if (g->n > 0 && (!X || !out)) return set_error(LSQ_ERR_INVALID_ARG, "null matrix pointer");
    if (X == out) return set_error(LSQ_ERR_INVALID_ARG, "out must not alias X");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t *pm = nullptr;
    LSQ_TRY(get_posmap(g, range_out, range_x, 1, &pm, s));
    const int64_t nnzb = g->pats[range_out].nnzb;
    if (nnzb == 0) return LSQ_OK;
    note_launch();
    if (precision == LSQ_F64)
        k_transpose_into<double><<<tgrid(nnzb * b * b), 256, 0, s>>>(nnzb, b, pm, alpha,
                                                                      (const double *)X, (double *)out);
    else
        k_transpose_into<float><<<tgrid(nnzb * b * b), 256, 0, s>>>(nnzb, b, pm, (float)alpha,
                                                                     (const float *)X, (float *)out);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

extern "C" int lsq_geom_adopt_schedules(lsq_geom g_to, lsq_geom g_from) {
    using namespace lsq;
    clear_error();
    if (!g_to || !g_from) return set_error(LSQ_ERR_INVALID_ARG, "null geometry handle");
    if (g_to == g_from) return LSQ_OK;
    if (g_to->n_ranges != g_from->n_ranges)
        return set_error(LSQ_ERR_INVALID_ARG, "the geometries hold different range lists");
    for (int r = 0; r < g_to->n_ranges; ++r)
        if (g_to->pats[r].R != g_from->pats[r].R)
            return set_error(LSQ_ERR_INVALID_ARG, "the geometries hold different range lists");
    // the source's own hints first, then its tuned plans (which take precedence)
    for (const auto &kv : g_from->schedule_hints) g_to->schedule_hints[kv.first] = kv.second;
    for (const auto &kv : g_from->pplans) {
        const ProductPlan &p = kv.second;
        std::array<int, 4> h = {p.variant[0], p.variant[1], p.variant16[0], p.variant16[1]};
        auto it = g_to->schedule_hints.find(kv.first);
        if (it != g_to->schedule_hints.end())
            for (int k = 0; k < 2; ++k)
                if (h[k] < 0) {
                    h[k] = it->second[k];
                    h[2 + k] = it->second[2 + k];
                }
        g_to->schedule_hints[kv.first] = h;
    }
    return LSQ_OK;
}
