// Plan-driven form of the truncated atom-block product (4 x 4 blocks).
//
// Sec. 2.3.2 of the paper: every product of the linear-scaling method is
// restricted to the range of its result, C_ij = sum_k A_ik B_kj over the
// stored blocks (i, j) of C.  The set of contributing k of each block of C
// depends only on the three range patterns, so it is found once per
// geometry (the symbolic product) and stored as a plan:
//
//   for each block s = (i, j) of C, the list of pairs (ao, xe) with
//   A_ik = A[a_ptr[i] + ao] and B_kj = (X_jk)^T, X_jk = X[x_ptr[j] + xe],
//   where X = B^T lives on B's (symmetric) pattern.
//
// The lists are stored back to back in the order of C's blocks (CSR over
// blocks of C).  The numeric kernel gives each block of C to a team of 16
// lanes, lane (r, c) owning C_ij[r][c]: per item it reads row r of A_ik
// and row c of X_jk (16 bytes each, the four lanes that share a row read
// the same 64-byte block), so every load instruction of a team touches
// one block of A and one of X.  All teams of a thread block work on the
// same row i of C, so row i of A is reused from L1; they take the row's
// blocks in an order sorted by list length, so the two teams of a warp
// run lists of similar length.  No index search is left in the kernel.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "lsq_internal.h"

namespace lsq {

// Triangle of C a plan covers: 0 every block, 1 the blocks with j >= i, 2 those with j <= i.
__device__ __forceinline__ bool tri_skip(int tri, int i, int j) {
    return tri == 1 ? j < i : (tri == 2 ? j > i : false);
}


constexpr int kMaxPlanRow = 8192;  // longest row of C a plan handles (shared-memory sort)
// The plan builder's atom map holds 16-bit positions within a row of A (plan items pack them in
// 16 bits too), so rows of A and B hold at most 65535 blocks and 0xffff marks an absent atom.
constexpr uint16_t kNoAtom = 0xffff;

// ---- symbolic product: item count of every block of C -----------------------
__global__ void __launch_bounds__(512) k_plan_count(int n, const int64_t *__restrict__ a_ptr,
                                                    const int32_t *__restrict__ a_col,
                                                    const int64_t *__restrict__ x_ptr,
                                                    const int32_t *__restrict__ x_col,
                                                    const int64_t *__restrict__ c_ptr,
                                                    const int32_t *__restrict__ c_col,
                                                    int upper, int32_t *__restrict__ cnt) {
    extern __shared__ uint16_t amap[];  // [n]: position of atom k in row i of A, kNoAtom if absent
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    for (int j = tid; j < n; j += nth) amap[j] = kNoAtom;
    __syncthreads();
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t a0 = a_ptr[i], a1 = a_ptr[i + 1];
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = (uint16_t)(p - a0);
        __syncthreads();
        for (int64_t s = c_ptr[i] + warp; s < c_ptr[i + 1]; s += nwarps) {
            const int j = c_col[s];
            int c = 0;
            if (!tri_skip(upper, i, j))
                for (int64_t q = x_ptr[j] + lane; q < x_ptr[j + 1]; q += 32) c += amap[x_col[q]] != kNoAtom;
            for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
            if (lane == 0) cnt[s] = c;
        }
        __syncthreads();
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = kNoAtom;
        __syncthreads();
    }
}

// ---- per row of C: order blocks by item count (descending), then index -----------
__global__ void __launch_bounds__(512) k_plan_sort(int n, const int64_t *__restrict__ c_ptr,
                                                   const int32_t *__restrict__ cnt,
                                                   int64_t *__restrict__ perm) {
    extern __shared__ unsigned long long key[];  // [next pow2 of the longest row]
    const int tid = threadIdx.x, nth = blockDim.x;
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t c0 = c_ptr[i];
        const int len = (int)(c_ptr[i + 1] - c0);
        int m = 1;
        while (m < len) m <<= 1;
        // key: (~count) in the high word sorts by count descending; the low word is the offset
        for (int e = tid; e < m; e += nth)
            key[e] = e < len ? ((unsigned long long)(~(unsigned)cnt[c0 + e]) << 32) | (unsigned)e
                             : ~0ull;
        __syncthreads();
        for (int size = 2; size <= m; size <<= 1)
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                for (int e = tid; e < m; e += nth) {
                    const int p = e ^ stride;
                    if (p > e) {
                        const bool up = (e & size) == 0;
                        const unsigned long long a = key[e], b = key[p];
                        if ((a > b) == up) {
                            key[e] = b;
                            key[p] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (int e = tid; e < len; e += nth) perm[c0 + e] = c0 + (int64_t)(key[e] & 0xffffffffu);
        __syncthreads();
    }
}

// Exclusive scan of int32 counts into int64 offsets (one block).
__global__ void k_scan_cnt(int64_t m, const int32_t *__restrict__ in, int64_t *__restrict__ out) {
    __shared__ int64_t part[1024];
    int t = threadIdx.x, nt = blockDim.x;
    int64_t seg = (m + nt - 1) / nt;
    int64_t b0 = t * seg, b1 = b0 + seg < m ? b0 + seg : m;
    int64_t s = 0;
    for (int64_t k = b0; k < b1; ++k) s += in[k];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        int64_t run = 0;
        for (int k = 0; k < nt; ++k) {
            int64_t v = part[k];
            part[k] = run;
            run += v;
        }
    }
    __syncthreads();
    int64_t run = part[t];
    for (int64_t k = b0; k < b1; ++k) {
        out[k] = run;
        run += in[k];
    }
    if (b1 == m && b0 < b1) out[m] = run;
    if (m == 0 && t == 0) out[0] = 0;
}

// ---- fill the item lists (one warp per block of C, ordered compaction) ---------
__global__ void __launch_bounds__(512) k_plan_fill(int n, const int64_t *__restrict__ a_ptr,
                                                   const int32_t *__restrict__ a_col,
                                                   const int64_t *__restrict__ x_ptr,
                                                   const int32_t *__restrict__ x_col,
                                                   const int64_t *__restrict__ c_ptr,
                                                   const int32_t *__restrict__ c_col,
                                                   const int64_t *__restrict__ item_ptr, int upper,
                                                   uint32_t *__restrict__ items) {
    extern __shared__ uint16_t amap[];  // as in k_plan_count
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    for (int j = tid; j < n; j += nth) amap[j] = kNoAtom;
    __syncthreads();
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t a0 = a_ptr[i], a1 = a_ptr[i + 1];
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = (uint16_t)(p - a0);
        __syncthreads();
        for (int64_t s = c_ptr[i] + warp; s < c_ptr[i + 1]; s += nwarps) {
            const int j = c_col[s];
            if (tri_skip(upper, i, j)) continue;
            const int64_t x0 = x_ptr[j], x1 = x_ptr[j + 1];
            int64_t w = item_ptr[s];
            for (int64_t qb = x0; qb < x1; qb += 32) {
                const int64_t q = qb + lane;
                const int ao = q < x1 ? (int)amap[x_col[q]] : (int)kNoAtom;
                const unsigned m = __ballot_sync(0xffffffffu, ao != kNoAtom);
                if (ao != kNoAtom)
                    items[w + __popc(m & ((1u << lane) - 1u))] = (uint32_t)ao | ((uint32_t)(q - x0) << 16);
                w += __popc(m);
            }
        }
        __syncthreads();
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = kNoAtom;
        __syncthreads();
    }
}

// ---- numeric product from a plan -------------------------------------------------
template <typename T> struct Row4;
template <> struct Row4<float> {
    static __device__ __forceinline__ void load(const float *__restrict__ p, float (&v)[4]) {
        float4 x = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
    }
};
template <> struct Row4<double> {
    static __device__ __forceinline__ void load(const double *__restrict__ p, double (&v)[4]) {
        double2 x = __ldg(reinterpret_cast<const double2 *>(p));
        double2 y = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        v[0] = x.x; v[1] = x.y; v[2] = y.x; v[3] = y.y;
    }
};

// Blocks of A staged in shared memory are stored with a padded stride (20 floats, 18 doubles:
// a multiple of 16 bytes) so that the lanes of a warp reading different blocks spread over
// the banks instead of colliding on the 16-value period.
template <typename T> struct SmemStride;
template <> struct SmemStride<float> { static constexpr int v = 20; };
template <> struct SmemStride<double> { static constexpr int v = 18; };

// N consecutive values from shared memory (16-byte vector loads through a generic pointer;
// the read-only global path must not be used on shared memory).
template <typename T, int N>
__device__ __forceinline__ void load_rows_shared(const T *p, T (&v)[N]) {
    constexpr int per = 16 / sizeof(T);
#pragma unroll
    for (int k = 0; k < N; k += per) {
        if (sizeof(T) == 4) {
            const float4 x = *reinterpret_cast<const float4 *>(p + k);
            reinterpret_cast<float *>(v)[k] = x.x;
            reinterpret_cast<float *>(v)[k + 1] = x.y;
            reinterpret_cast<float *>(v)[k + 2] = x.z;
            reinterpret_cast<float *>(v)[k + 3] = x.w;
        } else {
            const double2 x = *reinterpret_cast<const double2 *>(p + k);
            reinterpret_cast<double *>(v)[k] = x.x;
            reinterpret_cast<double *>(v)[k + 1] = x.y;
        }
    }
}

// Copies row i of A (na blocks of 16 values) into shared memory with the padded stride.
template <typename T>
__device__ __forceinline__ void stage_row(T *As, const T *__restrict__ A, int64_t a0, int64_t na) {
    constexpr int per = 16 / sizeof(T);   // values per 16-byte vector
    constexpr int vpb = 16 / per;         // vectors per block
    constexpr int svb = SmemStride<T>::v / per;
    for (int64_t e = threadIdx.x; e < na * vpb; e += blockDim.x) {
        const int64_t blk = e / vpb, q = e - blk * vpb;
        reinterpret_cast<float4 *>(As)[blk * svb + q] = reinterpret_cast<const float4 *>(A + 16 * a0)[e];
    }
}

struct PlanArgs {
    int n;                      // atoms (rows)
    int upper;                  // triangle of C computed: 0 all, 1 j >= i, 2 j <= i
    const int64_t *c_ptr;       // row pointers of C
    int64_t nblocks;            // blocks of C
    const int64_t *perm;        // blocks of C in processing order
    const int64_t *item_ptr;    // [nblocks + 1]
    const uint32_t *items;
    const int64_t *a_ptr;
    const int64_t *x_ptr;
    const int64_t *c_row;       // row of each block of C
    const int32_t *c_col;
    const void *A;  // op(A), rows contiguous
    const void *X;  // op(B)^T, rows contiguous
    void *C;
    double alpha, beta;
};

// Accumulates the items [q0, q1) of one block of C into acc (lane (r, c) of a 16-lane team).
// UNROLL items are fetched before any of their blocks is used, so each lane keeps
// 2 * UNROLL independent 16-byte loads in flight.
template <typename T, int UNROLL>
__device__ __forceinline__ T plan_items(const uint32_t *__restrict__ it, int nit,
                                        const T *__restrict__ arow, const T *__restrict__ xrow) {
    T acc[UNROLL];
#pragma unroll
    for (int u = 0; u < UNROLL; ++u) acc[u] = T(0);
    int q = 0;
    for (; q + UNROLL <= nit; q += UNROLL) {
        uint32_t w[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) w[u] = __ldg(it + q + u);
        T a[UNROLL][4], x[UNROLL][4];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            Row4<T>::load(arow + 16 * (w[u] & 0xffffu), a[u]);
            Row4<T>::load(xrow + 16 * (w[u] >> 16), x[u]);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t)
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) acc[u] = fma(a[u][t], x[u][t], acc[u]);
    }
    for (; q < nit; ++q) {
        const uint32_t w0 = __ldg(it + q);
        T a0[4], x0[4];
        Row4<T>::load(arow + 16 * (w0 & 0xffffu), a0);
        Row4<T>::load(xrow + 16 * (w0 >> 16), x0);
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[0] = fma(a0[t], x0[t], acc[0]);
    }
    T v = acc[0];
#pragma unroll
    for (int u = 1; u < UNROLL; ++u) v += acc[u];
    return v;
}

template <typename T>
__device__ __forceinline__ void plan_store(const PlanArgs &g, T *__restrict__ C, int64_t s, int sub, T v) {
    T *dst = C + 16 * s + sub;
    v = (T)g.alpha * v;
    *dst = g.beta != 0.0 ? fma((T)g.beta, *dst, v) : v;
}

// Blocks t0, t0 + step, ... (< t1) of C in the plan's order, one per team of 16 lanes (lane
// (r, c) = threadIdx.x % 16 accumulates C_ij[r][c]).
template <typename T, int UNROLL>
__device__ __forceinline__ void b4_blocks(const PlanArgs &g, int64_t t0, int64_t t1, int64_t step) {
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ X = static_cast<const T *>(g.X);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int sub = threadIdx.x & 15;
    const int r = sub >> 2, c = sub & 3;
    for (int64_t t = t0; t < t1; t += step) {
        const int64_t s = g.perm[t];
        const int i = (int)g.c_row[s];
        if (tri_skip(g.upper, i, g.c_col[s])) continue;
        const T *__restrict__ arow = A + 16 * g.a_ptr[i] + 4 * r;
        const T *__restrict__ xrow = X + 16 * g.x_ptr[g.c_col[s]] + 4 * c;
        const int64_t i0 = g.item_ptr[s];
        const T v = plan_items<T, UNROLL>(g.items + i0, (int)(g.item_ptr[s + 1] - i0), arow, xrow);
        plan_store(g, C, s, sub, v);
    }
}

// Two schedules of the same work (the plan's autotuner picks one per product):
//  ROWS = false: teams take blocks of C in the plan's order across the whole grid;
//  ROWS = true:  a thread block works on one row i of C at a time, so the row i of A it
//                reads stays in L1, and its teams share out that row's blocks.
// In both, a team of 16 lanes owns one block (i, j) of C, lane (r, c) accumulating
// C_ij[r][c] = sum over items of sum_t A_ik[r][t] X_jk[c][t]   (B_kj = X_jk^T).
template <typename T, bool ROWS, int UNROLL>
__global__ void __launch_bounds__(ROWS ? 1024 : 256) k_mm_plan_b4(PlanArgs g) {
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ X = static_cast<const T *>(g.X);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int sub = threadIdx.x & 15;
    const int r = sub >> 2, c = sub & 3;
    if (ROWS) {
        const int team = threadIdx.x >> 4, nteams = blockDim.x >> 4;
        for (int i = blockIdx.x; i < g.n; i += gridDim.x) {
            const T *__restrict__ arow = A + 16 * g.a_ptr[i] + 4 * r;
            for (int64_t e = g.c_ptr[i] + team; e < g.c_ptr[i + 1]; e += nteams) {
                const int64_t s = g.perm[e];
                if (tri_skip(g.upper, i, g.c_col[s])) continue;  // outside the triangle
                const T *__restrict__ xrow = X + 16 * g.x_ptr[g.c_col[s]] + 4 * c;
                const int64_t i0 = g.item_ptr[s];
                const T v = plan_items<T, UNROLL>(g.items + i0, (int)(g.item_ptr[s + 1] - i0), arow, xrow);
                plan_store(g, C, s, sub, v);
            }
        }
    } else {
        const int64_t team0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 4;
        const int64_t nteams = ((int64_t)gridDim.x * blockDim.x) >> 4;
        b4_blocks<T, UNROLL>(g, team0, g.nblocks, nteams);
    }
}

// Third schedule: one row i of C per thread block with row i of A copied once into shared
// memory, so that only the blocks of B^T come from L2 (needs 16 |row of A| values of smem).
template <typename T, int UNROLL>
__global__ void __launch_bounds__(1024) k_mm_plan_b4_smem(PlanArgs g) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ X = static_cast<const T *>(g.X);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int sub = threadIdx.x & 15;
    const int r = sub >> 2, c = sub & 3;
    const int team = threadIdx.x >> 4, nteams = blockDim.x >> 4;
    for (int i = blockIdx.x; i < g.n; i += gridDim.x) {
        __syncthreads();
        stage_row(As, A, g.a_ptr[i], g.a_ptr[i + 1] - g.a_ptr[i]);
        __syncthreads();
        constexpr int AS = SmemStride<T>::v;
        const T *arow = As + 4 * r;
        for (int64_t e = g.c_ptr[i] + team; e < g.c_ptr[i + 1]; e += nteams) {
            const int64_t s = g.perm[e];
            if (tri_skip(g.upper, i, g.c_col[s])) continue;
            const T *__restrict__ xrow = X + 16 * g.x_ptr[g.c_col[s]] + 4 * c;
            const int64_t i0 = g.item_ptr[s];
            const uint32_t *__restrict__ it = g.items + i0;
            const int nit = (int)(g.item_ptr[s + 1] - i0);
            T acc[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) acc[u] = T(0);
            int q = 0;
            for (; q + UNROLL <= nit; q += UNROLL) {
                uint32_t w[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) w[u] = __ldg(it + q + u);
                T a[UNROLL][4], x[UNROLL][4];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const T *ap = arow + AS * (w[u] & 0xffffu);
#pragma unroll
                    for (int t = 0; t < 4; ++t) a[u][t] = ap[t];
                    Row4<T>::load(xrow + 16 * (w[u] >> 16), x[u]);
                }
#pragma unroll
                for (int t = 0; t < 4; ++t)
#pragma unroll
                    for (int u = 0; u < UNROLL; ++u) acc[u] = fma(a[u][t], x[u][t], acc[u]);
            }
            for (; q < nit; ++q) {
                const uint32_t w0 = __ldg(it + q);
                const T *ap = arow + AS * (w0 & 0xffffu);
                T x0[4];
                Row4<T>::load(xrow + 16 * (w0 >> 16), x0);
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[0] = fma(ap[t], x0[t], acc[0]);
            }
            T v = acc[0];
#pragma unroll
            for (int u = 1; u < UNROLL; ++u) v += acc[u];
            plan_store(g, C, s, sub, v);
        }
    }
}

// Register-blocked schedule: a team of TEAM lanes per block (i, j) of C (TEAM = 4: each lane
// a 2 x 2 sub-block; TEAM = 2: a 2 x 4 sub-block), so each lane receives fewer bytes per FMA
// than with one element per lane (the 16-lane teams are bound by L1 register writeback).
template <typename T, int TEAM>
struct SubBlock {
    static constexpr int CT = TEAM == 4 ? 2 : 4;  // columns per lane
    static constexpr int RT = TEAM == 1 ? 4 : 2;  // rows per lane
};

// N consecutive values from global memory (read-only path).
template <typename T, int N>
__device__ __forceinline__ void load_rows(const T *__restrict__ p, T (&v)[N]) {
#pragma unroll
    for (int k = 0; k < N; k += 4) {
        T t[4];
        Row4<T>::load(p + k, t);
#pragma unroll
        for (int u = 0; u < 4; ++u) v[k + u] = t[u];
    }
}

// N consecutive values from global memory in 32-byte loads (read-only path; p must be
// 32-byte aligned).  Half as many load instructions as load_rows for the same bytes, so the
// lanes of a warp touch each cache line in half as many L1 wavefronts.
template <typename T, int N>
__device__ __forceinline__ void load_rows_256(const T *__restrict__ p, T (&v)[N]) {
    const size_t ga = __cvta_generic_to_global(p);
    if constexpr (sizeof(T) == 4) {
        static_assert(N % 8 == 0, "whole 32-byte vectors");
#pragma unroll
        for (int k = 0; k < N; k += 8)
            asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
                : "=f"(v[k]), "=f"(v[k + 1]), "=f"(v[k + 2]), "=f"(v[k + 3]), "=f"(v[k + 4]),
                  "=f"(v[k + 5]), "=f"(v[k + 6]), "=f"(v[k + 7])
                : "l"(ga + 4 * k));
    } else {
        static_assert(N % 4 == 0, "whole 32-byte vectors");
#pragma unroll
        for (int k = 0; k < N; k += 4)
            asm("ld.global.nc.v4.f64 {%0, %1, %2, %3}, [%4];"
                : "=d"(v[k]), "=d"(v[k + 1]), "=d"(v[k + 2]), "=d"(v[k + 3])
                : "l"(ga + 8 * k));
    }
}

template <bool W256, typename T, int N>
__device__ __forceinline__ void load_x(const T *p, T (&v)[N]) {
    if constexpr (W256)
        load_rows_256(p, v);
    else
        load_rows(p, v);
}

template <bool SMEM, typename T, int N, bool W256 = false>
__device__ __forceinline__ void load_a(const T *p, T (&v)[N]) {
    if constexpr (SMEM)
        load_rows_shared(p, v);
    else
        load_x<W256>(p, v);
}

// SPLIT > 1 (row schedule only): SPLIT consecutive teams share one block of C, each taking a
// contiguous part of its list, and combine with warp shuffles (for rows of C shorter than the
// number of teams of a thread block, e.g. products truncated to L's range).  With IL the teams
// take the list interleaved instead (team p items p, p + SPLIT, ...): a list is sorted by k, so
// the teams of a group then read neighbouring blocks of A (distinct shared-memory banks) and of
// B^T (shared cache lines).  THREADS fixes the block size, and with it the register budget.
// One block s = (i, j) of C for a team of TEAM lanes (a part of SPLIT teams sharing the
// block's items); As: row i of A staged in shared memory (SMEM), else unused.
template <typename T, int TEAM, bool SMEM, int SPLIT, bool IL, bool W256>
__device__ __forceinline__ void rb_work(const PlanArgs &g, const T *As, int64_t s, int i, int part) {
    constexpr int RT = SubBlock<T, TEAM>::RT, CT = SubBlock<T, TEAM>::CT;
    constexpr int NCB = 4 / CT;  // column blocks per row block
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ X = static_cast<const T *>(g.X);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int sub = threadIdx.x % TEAM;
    const int r0 = (sub / NCB) * RT, c0 = (sub % NCB) * CT;
    constexpr int AS = SMEM ? SmemStride<T>::v : 16;  // stride between blocks of A
    const T *arow = (SMEM ? As : A + 16 * g.a_ptr[i]) + 4 * r0;
    const T *__restrict__ xrow = X + 16 * g.x_ptr[g.c_col[s]] + 4 * c0;
    const int64_t i0 = g.item_ptr[s];
    const int ntot = (int)(g.item_ptr[s + 1] - i0);
    constexpr int STEP = IL ? SPLIT : 1;
    const int q0 = IL ? part : (SPLIT == 1 ? 0 : (int)((int64_t)ntot * part / SPLIT));
    const int nit = IL ? ntot : (SPLIT == 1 ? ntot : (int)((int64_t)ntot * (part + 1) / SPLIT));
    const uint32_t *__restrict__ it = g.items + i0;
    T acc[RT][CT];
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
        for (int c = 0; c < CT; ++c) acc[r][c] = T(0);
    int q = q0;
    // the next pair of item words is fetched while the current pair's blocks load, so a
    // pair costs one trip to L2 instead of two dependent ones
    uint32_t w0 = q < nit ? __ldg(it + q) : 0u, w1 = q + STEP < nit ? __ldg(it + q + STEP) : 0u;
    for (; q + STEP < nit; q += 2 * STEP) {
        const int qn = q + 2 * STEP;
        const uint32_t n0 = qn < nit ? __ldg(it + qn) : 0u;
        const uint32_t n1 = qn + STEP < nit ? __ldg(it + qn + STEP) : 0u;
        T a0[4 * RT], x0[4 * CT], a1[4 * RT], x1[4 * CT];
        load_a<SMEM, T, 4 * RT, W256>(arow + AS * (w0 & 0xffffu), a0);
        load_x<W256>(xrow + 16 * (w0 >> 16), x0);
        load_a<SMEM, T, 4 * RT, W256>(arow + AS * (w1 & 0xffffu), a1);
        load_x<W256>(xrow + 16 * (w1 >> 16), x1);
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
            for (int c = 0; c < CT; ++c)
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    acc[r][c] = fma(a0[4 * r + t], x0[4 * c + t], acc[r][c]);
                    acc[r][c] = fma(a1[4 * r + t], x1[4 * c + t], acc[r][c]);
                }
        w0 = n0;
        w1 = n1;
    }
    if (q < nit) {
        T a0[4 * RT], x0[4 * CT];
        load_a<SMEM, T, 4 * RT, W256>(arow + AS * (w0 & 0xffffu), a0);
        load_x<W256>(xrow + 16 * (w0 >> 16), x0);
#pragma unroll
        for (int r = 0; r < RT; ++r)
#pragma unroll
            for (int c = 0; c < CT; ++c)
#pragma unroll
                for (int t = 0; t < 4; ++t) acc[r][c] = fma(a0[4 * r + t], x0[4 * c + t], acc[r][c]);
    }
    if (SPLIT > 1) {
        const int lane = threadIdx.x & 31;
        const int gsz = TEAM * SPLIT;
        const unsigned gmask = gsz == 32 ? 0xffffffffu : (((1u << gsz) - 1u) << (lane / gsz * gsz));
#pragma unroll
        for (int off = TEAM; off < gsz; off <<= 1)
#pragma unroll
            for (int r = 0; r < RT; ++r)
#pragma unroll
                for (int c = 0; c < CT; ++c) acc[r][c] += __shfl_xor_sync(gmask, acc[r][c], off);
        if (part != 0) return;
    }
    T *dst = C + 16 * s;
#pragma unroll
    for (int r = 0; r < RT; ++r)
#pragma unroll
        for (int c = 0; c < CT; ++c) {
            const int e = (r0 + r) * 4 + c0 + c;
            const T v = (T)g.alpha * acc[r][c];
            dst[e] = g.beta != 0.0 ? fma((T)g.beta, dst[e], v) : v;
        }
}

// Blocks t0, t0 + step, ... (< t1) of C in the plan's order, one per team of TEAM lanes.
template <typename T, int TEAM>
__device__ __forceinline__ void rb_grid_blocks(const PlanArgs &g, int64_t t0, int64_t t1, int64_t step) {
    for (int64_t t = t0; t < t1; t += step) {
        const int64_t s = g.perm[t];
        const int i = (int)g.c_row[s];
        if (tri_skip(g.upper, i, g.c_col[s])) continue;
        rb_work<T, TEAM, false, 1, false, false>(g, nullptr, s, i, 0);
    }
}

template <typename T, bool ROWS, int TEAM, bool SMEM = false, int SPLIT = 1, bool IL = false,
          int THREADS = (ROWS ? 1024 : 256), bool W256 = false>
__global__ void __launch_bounds__(THREADS) k_mm_plan_b4_rb(PlanArgs g) {
    static_assert(TEAM * SPLIT <= 32, "a group of teams must fit in a warp");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *As = reinterpret_cast<T *>(smem_raw);  // row i of A (SMEM variant only)
    const T *__restrict__ A = static_cast<const T *>(g.A);
    auto work = [&](int64_t s, int i, int part) { rb_work<T, TEAM, SMEM, SPLIT, IL, W256>(g, As, s, i, part); };
    if (ROWS) {
        const int team = threadIdx.x / TEAM / SPLIT, nteams = blockDim.x / TEAM / SPLIT;
        const int part = (threadIdx.x / TEAM) % SPLIT;
        for (int i = blockIdx.x; i < g.n; i += gridDim.x) {
            if (SMEM) {
                __syncthreads();
                stage_row(As, A, g.a_ptr[i], g.a_ptr[i + 1] - g.a_ptr[i]);
                __syncthreads();
            }
            for (int64_t e = g.c_ptr[i] + team; e < g.c_ptr[i + 1]; e += nteams) {
                const int64_t s = g.perm[e];
                if (tri_skip(g.upper, i, g.c_col[s])) continue;
                work(s, i, part);
            }
        }
    } else {
        const int64_t team0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / TEAM;
        const int64_t nteams = ((int64_t)gridDim.x * blockDim.x) / TEAM;
        for (int64_t t = team0; t < g.nblocks; t += nteams) {
            const int64_t s = g.perm[t];
            const int i = (int)g.c_row[s];
            if (tri_skip(g.upper, i, g.c_col[s])) continue;
            work(s, i, 0);
        }
    }
}

// Any block size b <= 16: one warp per block of C.  Per item the warp stages op(A)_ik and
// X_jk = op(B)_kj^T in shared memory (transposing on the way when an operand is read through
// its transpose map), then lane l computes row l % b of C_ij over a slice of its columns.
struct PlanArgsGen {
    PlanArgs p;
    int b;
    const int64_t *a_tm;  // transpose map of A's pattern (TA)
    const int64_t *b_tm;  // transpose map of B's pattern (!TB)
};

// Blocks t0, t0 + step, ... (< t1) of C in the plan's order, one per warp; As and Xs are the
// warp's two b x b staging areas in shared memory.
template <typename T, bool TA, bool TB>
__device__ __forceinline__ void gen_blocks(const PlanArgsGen &ga, int64_t t0, int64_t t1, int64_t step, T *As,
                                           T *Xs) {
    const PlanArgs &g = ga.p;
    const int b = ga.b, bb = b * b;
    const int lane = threadIdx.x & 31;
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ X = static_cast<const T *>(g.X);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int nparts = 32 / b;                // lanes per row of C
    const int cw = (b + nparts - 1) / nparts;  // columns per lane (<= 8 for b <= 16)
    const int r = lane % b, part = lane / b;
    const bool active = part < nparts;
    const int cbeg = min(b, part * cw), cend = min(b, cbeg + cw);
    for (int64_t t = t0; t < t1; t += step) {
        const int64_t s = g.perm[t];
        const int i = (int)g.c_row[s];
        if (tri_skip(g.upper, i, g.c_col[s])) continue;
        const int j = g.c_col[s];
        const int64_t abase = g.a_ptr[i], xbase = g.x_ptr[j];
        const int64_t i0 = g.item_ptr[s], i1 = g.item_ptr[s + 1];
        T acc[8];
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[c] = T(0);
        for (int64_t q = i0; q < i1; ++q) {
            const uint32_t it = __ldg(g.items + q);
            const int64_t pa = abase + (it & 0xffffu), px = xbase + (it >> 16);
            const T *ab = A + (int64_t)bb * (TA ? ga.a_tm[pa] : pa);
            const T *xb = X + (int64_t)bb * (TB ? px : ga.b_tm[px]);
            __syncwarp();
            for (int e = lane; e < bb; e += 32) {
                const int u = e / b, v = e - u * b;
                As[e] = TA ? ab[v * b + u] : ab[e];  // As[u][v] = op(A)_ik[u][v]
                Xs[e] = TB ? xb[e] : xb[v * b + u];  // Xs[u][v] = X_jk[u][v] = op(B)_kj[v][u]
            }
            __syncwarp();
            if (active) {
                for (int tt = 0; tt < b; ++tt) {
                    const T a = As[r * b + tt];
#pragma unroll
                    for (int c = 0; c < 8; ++c)
                        if (cbeg + c < cend) acc[c] = fma(a, Xs[(cbeg + c) * b + tt], acc[c]);
                }
            }
        }
        if (active) {
            T *dst = C + (int64_t)bb * s + r * b;
#pragma unroll
            for (int c = 0; c < 8; ++c)
                if (cbeg + c < cend) {
                    const T v = (T)g.alpha * acc[c];
                    dst[cbeg + c] = g.beta != 0.0 ? fma((T)g.beta, dst[cbeg + c], v) : v;
                }
        }
    }
}

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_mm_plan_gen(PlanArgsGen ga) {
    __shared__ T stage[8][2][256];
    const int w = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    gen_blocks<T, TA, TB>(ga, w0, ga.p.nblocks, nw, stage[w][0], stage[w][1]);
}

// Lower blocks of a symmetric 4 x 4 result: C_ij = (C_ji)^T for j < i (tm: transpose map of C's
// pattern).  In a sorted symmetric pattern block (i, j) precedes (j, i) exactly when i < j, so
// the lower blocks are those with p > tm[p].
template <typename T>
__global__ void k_mirror_lower(int64_t nnzb, const int64_t *__restrict__ tm, T *__restrict__ C) {
    const uint64_t m = (uint64_t)nnzb * 16;
    for (uint64_t e = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const int64_t p = (int64_t)(e >> 4), t = tm[p];
        if (p <= t) continue;
        const int rc = (int)(e & 15);
        C[e] = C[t * 16 + (rc & 3) * 4 + (rc >> 2)];
    }
}

// Block sizes 9..16 (the 13-orbital model): one warp per block of C.  Per item, op(A)_ik and
// B^T_jk are staged transposed in shared memory (At[t][r] = op(A)_ik[r][t], Xt[t][c] =
// op(B)_kj[t][c]) inside a 16 x 16 frame, and lane l accumulates the 4 x 2 tile of C_ij at rows
// 4(l / 8) and columns 2(l % 8): per t one 4-vector of At and one 2-vector of Xt feed 8 FMAs.
// The next item's blocks are fetched into registers while the current one is multiplied.
// Frame entries beyond b are never initialised; they only reach accumulators that are not stored.
constexpr int kT16Stride = 20;  // frame row stride: 16-byte rows for float and double

// Blocks t0, t0 + step, ... (< t1) of C in the plan's order, one per warp; At and Xt are the
// warp's two 16 x kT16Stride frames in shared memory (16-byte aligned).
template <typename T, bool TA, bool TB>
__device__ __forceinline__ void t16_blocks(const PlanArgsGen &ga, int64_t t0, int64_t t1, int64_t step, T *At,
                                           T *Xt) {
    const PlanArgs &g = ga.p;
    const int b = ga.b, bb = b * b;
    constexpr int ST = kT16Stride;
    constexpr int PF = 8;   // values of a block per lane (256 / 32)
    const int lane = threadIdx.x & 31;
    const int r0 = 4 * (lane >> 3), c0 = 2 * (lane & 7);
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ X = static_cast<const T *>(g.X);
    T *__restrict__ C = static_cast<T *>(g.C);
    // frame offsets of the source elements e = lane + 32 k, fixed for the whole kernel
    int offA[PF], offX[PF];
#pragma unroll
    for (int k = 0; k < PF; ++k) {
        const int e = lane + 32 * k;
        const int u = e / b, v = e - u * b;  // element (u, v) of the source block
        offA[k] = TA ? u * ST + v : v * ST + u;
        offX[k] = TB ? v * ST + u : u * ST + v;
    }
    for (int64_t t = t0; t < t1; t += step) {
        const int64_t s = g.perm[t];
        const int i = (int)g.c_row[s];
        if (tri_skip(g.upper, i, g.c_col[s])) continue;
        const int j = g.c_col[s];
        const int64_t abase = g.a_ptr[i], xbase = g.x_ptr[j];
        const int64_t i0 = g.item_ptr[s], i1 = g.item_ptr[s + 1];
        T acc[4][2];
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r][0] = acc[r][1] = T(0);
        T pa[PF], px[PF];
        auto fetch = [&](int64_t q) {
            const uint32_t it = __ldg(g.items + q);
            const int64_t qa = abase + (it & 0xffffu), qx = xbase + (it >> 16);
            const T *ab = A + (int64_t)bb * (TA ? ga.a_tm[qa] : qa);
            const T *xb = X + (int64_t)bb * (TB ? qx : ga.b_tm[qx]);
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                const int e = lane + 32 * k;
                if (e < bb) {
                    pa[k] = __ldg(ab + e);
                    px[k] = __ldg(xb + e);
                }
            }
        };
        if (i0 < i1) fetch(i0);
        for (int64_t q = i0; q < i1; ++q) {
            __syncwarp();
#pragma unroll
            for (int k = 0; k < PF; ++k) {
                if (lane + 32 * k < bb) {
                    At[offA[k]] = pa[k];
                    Xt[offX[k]] = px[k];
                }
            }
            __syncwarp();
            if (q + 1 < i1) fetch(q + 1);
            for (int tt = 0; tt < b; ++tt) {
                T a[4], x[2];
                load_rows_shared(At + tt * ST + r0, a);
                if constexpr (sizeof(T) == 4) {
                    const float2 v = *reinterpret_cast<const float2 *>(Xt + tt * ST + c0);
                    x[0] = v.x;
                    x[1] = v.y;
                } else {
                    const double2 v = *reinterpret_cast<const double2 *>(Xt + tt * ST + c0);
                    x[0] = v.x;
                    x[1] = v.y;
                }
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    acc[r][0] = fma(a[r], x[0], acc[r][0]);
                    acc[r][1] = fma(a[r], x[1], acc[r][1]);
                }
            }
        }
        T *dst = C + (int64_t)bb * s;
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 2; ++c)
                if (r0 + r < b && c0 + c < b) {
                    const int e = (r0 + r) * b + c0 + c;
                    const T v = (T)g.alpha * acc[r][c];
                    dst[e] = g.beta != 0.0 ? fma((T)g.beta, dst[e], v) : v;
                }
    }
}

template <typename T, bool TA, bool TB>
__global__ void __launch_bounds__(256) k_mm_plan_t16(PlanArgsGen ga) {
    __shared__ __align__(16) T stage[8][2][16 * kT16Stride];
    const int w = threadIdx.x >> 5;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    t16_blocks<T, TA, TB>(ga, w0, ga.p.nblocks, nw, stage[w][0], stage[w][1]);
}

// Lower blocks of a symmetric result, any block size: one warp per block (lower blocks are
// those with p > tm[p], see k_mirror_lower).
template <typename T>
__global__ void k_mirror_lower_gen(int64_t nnzb, int b, const int64_t *__restrict__ tm, T *__restrict__ C) {
    const int lane = threadIdx.x & 31;
    const int bb = b * b;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < nnzb;
         p += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        const int64_t t = tm[p];
        if (p <= t) continue;
        for (int rc = lane; rc < bb; rc += 32) {
            const int r = rc / b, c = rc - r * b;
            C[p * bb + rc] = C[t * bb + c * b + r];
        }
    }
}

int mirror_lower_gen(lsq_geom g, int rc, int b, int dtype, void *C, cudaStream_t s) {
    LSQ_TRY(ensure_tmap(g, rc, s));
    const int64_t nnzb = g->pats[rc].nnzb;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nnzb * 32 + 255) / 256, (int64_t)g->num_sms * 16));
    note_launch();
    if (dtype == LSQ_F64)
        k_mirror_lower_gen<double><<<blocks, 256, 0, s>>>(nnzb, b, g->pats[rc].tmap.p, (double *)C);
    else
        k_mirror_lower_gen<float><<<blocks, 256, 0, s>>>(nnzb, b, g->pats[rc].tmap.p, (float *)C);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

__global__ void k_sum_cnt(int64_t m, const int32_t *__restrict__ cnt, unsigned long long *__restrict__ out) {
    unsigned long long s = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        s += (unsigned long long)cnt[e];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(out, s);
}

int plan_count_triples(lsq_geom g, int ra, int rb, int rc, int upper, int64_t *out, cudaStream_t s) {
    const Pattern &PA = g->pats[ra], &PB = g->pats[rb], &PC = g->pats[rc];
    const int n = g->n;
    *out = 0;
    if (n == 0 || PC.nnzb == 0) return LSQ_OK;
    auto it = g->pplans.find(std::make_tuple(ra, rb, rc + 1000 * upper));
    if (it != g->pplans.end()) {
        *out = it->second.triples;
        return LSQ_OK;
    }
    if (PA.max_row > 65535 || PB.max_row > 65535)
        return set_error(LSQ_ERR_UNSUPPORTED, "row too long for a product plan");
    if ((size_t)n * sizeof(uint16_t) + 1024 > g->smem_optin)
        return set_error(LSQ_ERR_UNSUPPORTED, "too many atoms for the shared-memory atom map");
    DevBuf<int32_t> cnt;
    DevBuf<unsigned long long> tot;
    LSQ_TRY(cnt.alloc(PC.nnzb));
    LSQ_TRY(tot.alloc(1));
    const size_t smem_map = (size_t)n * sizeof(uint16_t);
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_plan_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_map));
    int per_sm = 1;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_count, 512, smem_map);
    const int grid_rows = std::max(1, std::min(n, g->num_sms * std::max(per_sm, 1)));
    LSQ_CUDA_TRY(cudaMemsetAsync(tot.p, 0, sizeof(unsigned long long), s));
    note_launch();
    k_plan_count<<<grid_rows, 512, smem_map, s>>>(n, PA.row_ptr.p, PA.col.p, PB.row_ptr.p, PB.col.p,
                                                  PC.row_ptr.p, PC.col.p, upper, cnt.p);
    note_launch();
    k_sum_cnt<<<(int)std::min<int64_t>((PC.nnzb + 255) / 256, (int64_t)g->num_sms * 8), 256, 0, s>>>(
        PC.nnzb, cnt.p, tot.p);
    LSQ_CHECK_LAUNCH();
    unsigned long long h = 0;
    LSQ_CUDA_TRY(cudaMemcpyAsync(&h, tot.p, sizeof(h), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    *out = (int64_t)h;
    return LSQ_OK;
}

__global__ void k_rows_of(int n, const int64_t *__restrict__ c_ptr, int64_t *__restrict__ c_row) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    for (int64_t s = c_ptr[i]; s < c_ptr[i + 1]; ++s) c_row[s] = i;
}

int plan_build(lsq_geom g, int ra, int rb, int rc, int upper, ProductPlan **out, cudaStream_t s) {
    auto key = std::make_tuple(ra, rb, rc + 1000 * upper);
    auto it = g->pplans.find(key);
    if (it != g->pplans.end()) {
        *out = &it->second;
        return LSQ_OK;
    }
    const Pattern &PA = g->pats[ra], &PB = g->pats[rb], &PC = g->pats[rc];
    const int n = g->n;
    if (PA.max_row > 65535 || PB.max_row > 65535 || PC.max_row > kMaxPlanRow)
        return set_error(LSQ_ERR_UNSUPPORTED, "row too long for a product plan");
    if ((size_t)n * sizeof(uint16_t) + 1024 > g->smem_optin)
        return set_error(LSQ_ERR_UNSUPPORTED, "too many atoms for the shared-memory atom map");
    ProductPlan p;
    const int64_t nc = PC.nnzb;
    LSQ_TRY(p.cnt.alloc(nc));
    LSQ_TRY(p.perm.alloc(nc));
    LSQ_TRY(p.item_ptr.alloc((size_t)nc + 1));
    LSQ_TRY(p.c_row.alloc(nc));
    int per_sm = 1;
    size_t smem_map = (size_t)n * sizeof(uint16_t);
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_plan_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_map));
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_plan_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_map));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_count, 512, smem_map);
    const int grid_rows = std::max(1, std::min(n, g->num_sms * std::max(per_sm, 1)));
    int64_t nitems = 0;
    if (n > 0 && nc > 0) {
        note_launch();
        k_plan_count<<<grid_rows, 512, smem_map, s>>>(n, PA.row_ptr.p, PA.col.p, PB.row_ptr.p, PB.col.p,
                                                      PC.row_ptr.p, PC.col.p, upper, p.cnt.p);
        int m = 1;
        while (m < PC.max_row) m <<= 1;
        size_t smem_sort = sizeof(unsigned long long) * (size_t)std::max(m, 1);
        LSQ_CUDA_TRY(cudaFuncSetAttribute(k_plan_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sort));
        note_launch();
        k_plan_sort<<<std::min(n, g->num_sms * 2), 512, smem_sort, s>>>(n, PC.row_ptr.p, p.cnt.p, p.perm.p);
        note_launch();
        k_scan_cnt<<<1, 1024, 0, s>>>(nc, p.cnt.p, p.item_ptr.p);
        note_launch();
        k_rows_of<<<(n + 255) / 256, 256, 0, s>>>(n, PC.row_ptr.p, p.c_row.p);
        LSQ_CHECK_LAUNCH();
        LSQ_CUDA_TRY(cudaMemcpyAsync(&nitems, p.item_ptr.p + nc, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    } else if (nc >= 0) {
        LSQ_CUDA_TRY(cudaMemsetAsync(p.item_ptr.p, 0, sizeof(int64_t) * (nc + 1), s));
    }
    LSQ_TRY(p.items.alloc((size_t)std::max<int64_t>(nitems, 1)));
    if (nitems > 0) {
        note_launch();
        k_plan_fill<<<grid_rows, 512, smem_map, s>>>(n, PA.row_ptr.p, PA.col.p, PB.row_ptr.p, PB.col.p,
                                                     PC.row_ptr.p, PC.col.p, p.item_ptr.p, upper, p.items.p);
        LSQ_CHECK_LAUNCH();
    }
    p.triples = nitems;
    p.nitems = nitems;
    p.upper = upper;
    p.nblocks = nc;
    *out = &g->pplans.emplace(key, std::move(p)).first->second;
    return LSQ_OK;
}

namespace {
using PlanKernel = void (*)(PlanArgs);
struct Variant {
    PlanKernel k;
    bool rows;
    int threads;
    bool smem_a;  // stages the row of A in shared memory (16 values per block of the longest row)
    bool w256 = false;  // 32-byte global loads: A (unless staged) and B^T must be 32-byte aligned
};
template <typename T>
const Variant *variants(int *count) {
    static const Variant v[] = {
        {k_mm_plan_b4<T, false, 2>, false, 256, false}, {k_mm_plan_b4<T, false, 4>, false, 256, false},
        {k_mm_plan_b4<T, true, 2>, true, 1024, false},  {k_mm_plan_b4<T, true, 4>, true, 1024, false},
        {k_mm_plan_b4_smem<T, 2>, true, 1024, true},    {k_mm_plan_b4_smem<T, 4>, true, 1024, true},
        {k_mm_plan_b4_rb<T, false, 4>, false, 256, false}, {k_mm_plan_b4_rb<T, true, 4>, true, 1024, false},
        {k_mm_plan_b4_rb<T, false, 2>, false, 256, false}, {k_mm_plan_b4_rb<T, true, 2>, true, 1024, false},
        {k_mm_plan_b4_rb<T, true, 1>, true, 1024, false},
        {k_mm_plan_b4_rb<T, true, 4, true>, true, 1024, true}, {k_mm_plan_b4_rb<T, true, 2, true>, true, 1024, true},
        {k_mm_plan_b4_rb<T, true, 1, true>, true, 1024, true},
        {k_mm_plan_b4_rb<T, true, 4, true, 2>, true, 1024, true},
        {k_mm_plan_b4_rb<T, true, 4, true, 4>, true, 1024, true},
        {k_mm_plan_b4_rb<T, true, 4, false, 4>, true, 1024, false},
        {k_mm_plan_b4_rb<T, true, 4, true, 2, true>, true, 1024, true},
        {k_mm_plan_b4_rb<T, true, 4, true, 4, true>, true, 1024, true},
        {k_mm_plan_b4_rb<T, true, 2, true, 4, true, 512>, true, 512, true},
        {k_mm_plan_b4_rb<T, true, 1, true, 4, true, 256>, true, 256, true},
        {k_mm_plan_b4_rb<T, true, 1, true, 8, true, 256>, true, 256, true},
        {k_mm_plan_b4_rb<T, true, 1, false, 8, true, 256>, true, 256, false},
        {k_mm_plan_b4_rb<T, true, 4, true, 2, true, 1024, true>, true, 1024, true, true},
        {k_mm_plan_b4_rb<T, true, 4, true, 4, true, 1024, true>, true, 1024, true, true},
        {k_mm_plan_b4_rb<T, true, 4, true, 8, true, 1024, true>, true, 1024, true, true},
        {k_mm_plan_b4_rb<T, true, 2, true, 4, true, 512, true>, true, 512, true, true},
        {k_mm_plan_b4_rb<T, true, 1, true, 8, true, 256, true>, true, 256, true, true},
        {k_mm_plan_b4_rb<T, false, 4, false, 1, false, 256, true>, false, 256, false, true},
    };
    *count = 29;
    return v;
}

// Shared memory a variant needs for pattern ra (0 if none; -1 if it does not fit).
int64_t variant_smem(lsq_geom g, const Variant &v, int ra, size_t es) {
    if (!v.smem_a) return 0;
    const int64_t need = (int64_t)g->pats[ra].max_row * (es == 8 ? 18 : 20) * (int64_t)es;
    return need + 1024 <= (int64_t)g->smem_optin ? need : -1;
}

int run_variant(lsq_geom g, const Variant &v, const PlanArgs &a, int64_t nblocks, cudaStream_t s,
                int64_t smem = 0) {
    int per_sm = 1;
    if (smem > 0)
        LSQ_CUDA_TRY(cudaFuncSetAttribute((const void *)v.k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)smem));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, (const void *)v.k, v.threads, (size_t)smem);
    per_sm = std::max(per_sm, 1);
    int grid;
    if (v.rows)
        grid = std::max(1, std::min(g->n, g->num_sms * per_sm));
    else
        grid = (int)std::max<int64_t>(1, std::min<int64_t>((nblocks * 16 + v.threads - 1) / v.threads,
                                                           (int64_t)g->num_sms * per_sm));
    // (a grid-wide schedule never needs more threads than 16 per block of C)
    note_launch();
    v.k<<<grid, v.threads, (size_t)smem, s>>>(a);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}
}  // namespace

namespace {
int plan_launch_tuned(lsq_geom g, int dtype, ProductPlan &p, int ra, int rb, int rc, const PlanArgs &a,
                      cudaStream_t s);

GroupProduct group_product(const PlanArgs &a, int b, int dtype, int ta, int tb, const int64_t *a_tm,
                           const int64_t *b_tm) {
    GroupProduct q;
    q.b = b;
    q.dtype = dtype;
    q.ta = ta;
    q.tb = tb;
    q.upper = a.upper;
    q.n = a.n;
    q.nblocks = a.nblocks;
    q.c_ptr = a.c_ptr;
    q.perm = a.perm;
    q.item_ptr = a.item_ptr;
    q.a_ptr = a.a_ptr;
    q.x_ptr = a.x_ptr;
    q.c_row = a.c_row;
    q.a_tm = a_tm;
    q.b_tm = b_tm;
    q.items = a.items;
    q.c_col = a.c_col;
    q.A = a.A;
    q.X = a.X;
    q.C = a.C;
    q.alpha = a.alpha;
    q.beta = a.beta;
    return q;
}
}  // namespace

int plan_launch(lsq_geom g, int dtype, const ProductPlan &pc, int ra, int rb, int rc, const void *Aop,
                const void *X, void *C, double alpha, double beta, cudaStream_t s, bool mirror) {
    ProductPlan &p = const_cast<ProductPlan &>(pc);
    if (p.nblocks == 0) return LSQ_OK;
    PlanArgs a;
    a.n = g->n;
    a.upper = p.upper;
    a.c_ptr = g->pats[rc].row_ptr.p;
    a.nblocks = p.nblocks;
    a.perm = p.perm.p;
    a.item_ptr = p.item_ptr.p;
    a.items = p.items.p;
    a.a_ptr = g->pats[ra].row_ptr.p;
    a.x_ptr = g->pats[rb].row_ptr.p;
    a.c_row = p.c_row.p;
    a.c_col = g->pats[rc].col.p;
    a.A = Aop;
    a.X = X;
    a.C = C;
    a.alpha = alpha;
    a.beta = beta;
    if (g_group_rec) {
        // a step captured for a grouped launch: record the product, split the capture
        g_group_rec->products.push_back(group_product(a, 4, dtype, 0, 0, nullptr, nullptr));
        LSQ_TRY(g_group_rec->split(s));
    } else {
        LSQ_TRY(plan_launch_tuned(g, dtype, p, ra, rb, rc, a, s));
    }
    if (p.upper == 1 && mirror) {
        LSQ_TRY(ensure_tmap(g, rc, s));
        const int64_t m = g->pats[rc].nnzb * 16;
        const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, (int64_t)g->num_sms * 16));
        note_launch();
        if (dtype == LSQ_F64)
            k_mirror_lower<double><<<blocks, 256, 0, s>>>(g->pats[rc].nnzb, g->pats[rc].tmap.p, (double *)C);
        else
            k_mirror_lower<float><<<blocks, 256, 0, s>>>(g->pats[rc].nnzb, g->pats[rc].tmap.p, (float *)C);
        LSQ_CHECK_LAUNCH();
    }
    return LSQ_OK;
}

namespace {
// The product of plan_launch with the schedule tuned for it (timing every schedule on the
// first call).
int plan_launch_tuned(lsq_geom g, int dtype, ProductPlan &p, int ra, int rb, int rc, const PlanArgs &a,
                      cudaStream_t s) {
    const void *Aop = a.A, *X = a.X;
    const double beta = a.beta;
    int nv = 0;
    const Variant *v = dtype == LSQ_F64 ? variants<double>(&nv) : variants<float>(&nv);
    const int di = dtype == LSQ_F64 ? 0 : 1;
    int &choice = p.variant[di];
    // variants with 32-byte loads need 32-byte aligned operands (the blocks then are too)
    const bool al32 = reinterpret_cast<uintptr_t>(Aop) % 32 == 0 && reinterpret_cast<uintptr_t>(X) % 32 == 0;
    auto smem_for = [&](int k) -> int64_t {
        if (v[k].w256 && !al32) return -1;
        return variant_smem(g, v[k], ra, dtype_size(dtype));
    };
    if (const char *force = std::getenv("LSQ_PLAN_VARIANT")) {
        // a fixed schedule (tests exercise every variant this way)
        const int k = std::atoi(force);
        if (k >= 0 && k < nv && smem_for(k) >= 0) choice = k;
    }
    if (choice < 0) {
        // autotune: time every variant once on this product (each writes the same C), keep
        // the fastest for later calls.  Runs when beta == 0 so repeated runs are harmless.
        if (beta != 0.0) {
            choice = 0;
        } else {
            cudaEvent_t e0, e1;
            LSQ_CUDA_TRY(cudaEventCreate(&e0));
            LSQ_CUDA_TRY(cudaEventCreate(&e1));
            float best = 1e30f, best16 = 1e30f;
            int bi = 0, bi16 = 0;
            for (int k = 0; k < nv; ++k) {
                const int64_t sm = smem_for(k);
                if (sm < 0) continue;
                LSQ_CUDA_TRY(cudaEventRecord(e0, s));
                LSQ_TRY(run_variant(g, v[k], a, p.nblocks, s, sm));
                LSQ_CUDA_TRY(cudaEventRecord(e1, s));
                LSQ_CUDA_TRY(cudaEventSynchronize(e1));
                float ms = 0.f;
                LSQ_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
                if (ms < best) {
                    best = ms;
                    bi = k;
                }
                if (!v[k].w256 && ms < best16) {
                    best16 = ms;
                    bi16 = k;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            choice = bi;
            p.variant16[di] = bi16;
            p.tuned_ms[di] = best;
            if (std::getenv("LSQ_TUNE_LOG"))
                std::fprintf(stderr, "lsq autotune: ranges (%g, %g, %g)%s %s: variant %d, %.3f ms\n",
                             g->pats[ra].R, g->pats[rb].R, g->pats[rc].R, p.upper == 1 ? " upper" : (p.upper == 2 ? " lower" : ""),
                             dtype == LSQ_F64 ? "f64" : "f32", bi, best);
        }
    }
    // a later call may pass operands that the tuned variant cannot read
    const int use = smem_for(choice) >= 0 ? choice : std::max(p.variant16[di], 0);
    return run_variant(g, v[use], a, p.nblocks, s, smem_for(use));
}
}  // namespace

int plan_launch_gen(lsq_geom g, int b, int dtype, const ProductPlan &p, int ra, int ta, int rb, int tb, int rc,
                    const void *A, const void *B, void *C, double alpha, double beta, cudaStream_t s,
                    bool mirror) {
    if (p.nblocks == 0) return LSQ_OK;
    PlanArgsGen ga;
    PlanArgs &a = ga.p;
    a.n = g->n;
    a.upper = p.upper;
    a.c_ptr = g->pats[rc].row_ptr.p;
    a.nblocks = p.nblocks;
    a.perm = p.perm.p;
    a.item_ptr = p.item_ptr.p;
    a.items = p.items.p;
    a.a_ptr = g->pats[ra].row_ptr.p;
    a.x_ptr = g->pats[rb].row_ptr.p;
    a.c_row = p.c_row.p;
    a.c_col = g->pats[rc].col.p;
    a.A = A;
    a.X = B;
    a.C = C;
    a.alpha = alpha;
    a.beta = beta;
    ga.b = b;
    ga.a_tm = g->pats[ra].tmap.p;
    ga.b_tm = g->pats[rb].tmap.p;
    if (g_group_rec) {
        // a step captured for a grouped launch: record the product, split the capture
        g_group_rec->products.push_back(group_product(a, b, dtype, ta, tb, ga.a_tm, ga.b_tm));
        LSQ_TRY(g_group_rec->split(s));
        if (p.upper == 1 && mirror) LSQ_TRY(mirror_lower_gen(g, rc, b, dtype, C, s));
        return LSQ_OK;
    }
    const int threads = 256;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((p.nblocks + 7) / 8, (int64_t)g->num_sms * 8));
    note_launch();
    auto go = [&](auto kern) { kern<<<grid, threads, 0, s>>>(ga); };
    const bool t16 = b >= 9;  // 16 x 16 frames (4 x 2 tiles per lane); smaller blocks: row per lane
    if (dtype == LSQ_F64) {
        if (ta && tb) go(t16 ? k_mm_plan_t16<double, true, true> : k_mm_plan_gen<double, true, true>);
        else if (ta) go(t16 ? k_mm_plan_t16<double, true, false> : k_mm_plan_gen<double, true, false>);
        else if (tb) go(t16 ? k_mm_plan_t16<double, false, true> : k_mm_plan_gen<double, false, true>);
        else go(t16 ? k_mm_plan_t16<double, false, false> : k_mm_plan_gen<double, false, false>);
    } else {
        if (ta && tb) go(t16 ? k_mm_plan_t16<float, true, true> : k_mm_plan_gen<float, true, true>);
        else if (ta) go(t16 ? k_mm_plan_t16<float, true, false> : k_mm_plan_gen<float, true, false>);
        else if (tb) go(t16 ? k_mm_plan_t16<float, false, true> : k_mm_plan_gen<float, false, true>);
        else go(t16 ? k_mm_plan_t16<float, false, false> : k_mm_plan_gen<float, false, false>);
    }
    LSQ_CHECK_LAUNCH();
    if (p.upper == 1 && mirror) {
        // C_ij = (C_ji)^T for j < i, any block size
        LSQ_TRY(mirror_lower_gen(g, rc, b, dtype, C, s));
    }
    return LSQ_OK;
}

// ---- grouped products: one persistent launch over the products of several contexts -----
thread_local GroupRecorder *g_group_rec = nullptr;

int GroupRecorder::split(cudaStream_t s) {
    cudaGraph_t gr = nullptr;
    cudaError_t e = cudaStreamEndCapture(s, &gr);
    if (e != cudaSuccess) return set_error(LSQ_ERR_CUDA, std::string("ending a step segment: ") + cudaGetErrorString(e));
    segments.push_back(gr);
    LSQ_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    return LSQ_OK;
}

GroupRecorder::~GroupRecorder() {
    for (cudaGraph_t gr : segments)
        if (gr) cudaGraphDestroy(gr);
}

namespace {
// A product of a grouped launch, as the device sees it.
struct GroupDesc {
    PlanArgsGen ga;   // plan and operands; ga.b the block size
    int ta, tb;       // operands read through transpose maps (b != 4)
    int per_chunk;    // blocks of C per work item
    int64_t chunk0;   // first work item of this product in the launch's queue
};

// The two forms of a work item, kept out of line so that the kernel's registers are those of
// the larger form rather than of both together.
template <typename T>
__device__ __noinline__ void group_b4(const PlanArgs &a, int64_t t0, int64_t t1) {
    rb_grid_blocks<T, 4>(a, t0, t1, 64);
}

template <typename T, bool TA, bool TB>
__device__ __noinline__ void group_t16(const PlanArgsGen &ga, int64_t t0, int64_t t1, T *S0, T *S1) {
    t16_blocks<T, TA, TB>(ga, t0, t1, 8, S0, S1);
}

template <typename T, bool TA, bool TB>
__device__ __noinline__ void group_gen(const PlanArgsGen &ga, int64_t t0, int64_t t1, T *S0, T *S1) {
    gen_blocks<T, TA, TB>(ga, t0, t1, 8, S0, S1);
}

template <typename T>
__device__ __forceinline__ void group_frames(const GroupDesc &q, int64_t t0, int64_t t1, T *S0, T *S1) {
    if (q.ga.b >= 9) {
        if (q.ta && q.tb) group_t16<T, true, true>(q.ga, t0, t1, S0, S1);
        else if (q.ta) group_t16<T, true, false>(q.ga, t0, t1, S0, S1);
        else if (q.tb) group_t16<T, false, true>(q.ga, t0, t1, S0, S1);
        else group_t16<T, false, false>(q.ga, t0, t1, S0, S1);
    } else {
        if (q.ta && q.tb) group_gen<T, true, true>(q.ga, t0, t1, S0, S1);
        else if (q.ta) group_gen<T, true, false>(q.ga, t0, t1, S0, S1);
        else if (q.tb) group_gen<T, false, true>(q.ga, t0, t1, S0, S1);
        else group_gen<T, false, false>(q.ga, t0, t1, S0, S1);
    }
}

// Persistent: every thread block takes work items (per_chunk consecutive blocks of C, in the
// plan's order, of one product) from the queue counter until it runs past nchunks.  The
// blocks of an item are shared as in the stand-alone kernels: 4 lanes per 4 x 4 block (2 x 2
// values each, the register-blocked grid schedule), one warp per larger block (16 x 16
// frames for b >= 9).  Items only ever move forward, so no
// thread block waits on another.
// FR: the frame form of every product with b >= 9 in the launch, inlined: 0..3 = t16 with
// (TA, TB) = (FR / 2, FR % 2) (and b = 4 products), so that the kernel keeps the registers of
// one form (the occupancy of the stand-alone kernels); 4 = any mix, each form out of line.
template <typename T, int FR>
__global__ void __launch_bounds__(256, FR < 4 ? (sizeof(T) == 4 ? 3 : 2) : (sizeof(T) == 4 ? 2 : 1))
    k_mm_group(const GroupDesc *__restrict__ d, int nd, int64_t nchunks, unsigned long long *__restrict__ counter) {
    __shared__ __align__(16) T stage[8][2][16 * kT16Stride];
    __shared__ int64_t s_item;
    const int w = threadIdx.x >> 5;
    for (;;) {
        if (threadIdx.x == 0) s_item = (int64_t)atomicAdd(counter, 1ull);
        __syncthreads();
        const int64_t item = s_item;
        __syncthreads();
        if (item >= nchunks) break;
        int k = 0;
        while (k + 1 < nd && d[k + 1].chunk0 <= item) ++k;
        const GroupDesc &q = d[k];
        const int64_t t0 = (item - q.chunk0) * q.per_chunk;
        const int64_t t1 = min(t0 + (int64_t)q.per_chunk, q.ga.p.nblocks);
        const int b = q.ga.b;
        if constexpr (FR < 4) {
            if (b == 4) rb_grid_blocks<T, 4>(q.ga.p, t0 + (threadIdx.x >> 2), t1, 64);
            else t16_blocks<T, (FR >> 1) != 0, (FR & 1) != 0>(q.ga, t0 + w, t1, 8, stage[w][0], stage[w][1]);
        } else {
            if (b == 4) group_b4<T>(q.ga.p, t0 + (threadIdx.x >> 2), t1);
            else group_frames<T>(q, t0 + w, t1, stage[w][0], stage[w][1]);
        }
    }
}
}  // namespace

namespace {
const void *group_kernel(int dtype, int fr) {
    static const void *kf[5] = {(const void *)k_mm_group<float, 0>, (const void *)k_mm_group<float, 1>,
                                (const void *)k_mm_group<float, 2>, (const void *)k_mm_group<float, 3>,
                                (const void *)k_mm_group<float, 4>};
    static const void *kd[5] = {(const void *)k_mm_group<double, 0>, (const void *)k_mm_group<double, 1>,
                                (const void *)k_mm_group<double, 2>, (const void *)k_mm_group<double, 3>,
                                (const void *)k_mm_group<double, 4>};
    return dtype == LSQ_F64 ? kd[fr] : kf[fr];
}
}  // namespace

int group_prepare(const GroupProduct *products, int n, const lsq_geom g_any, GroupLaunch *out) {
    if (n < 1 || !g_any) return set_error(LSQ_ERR_INVALID_ARG, "empty product group");
    const int dtype = products[0].dtype;
    std::vector<int> order(n);
    for (int k = 0; k < n; ++k) {
        if (products[k].dtype != dtype) return set_error(LSQ_ERR_INVALID_ARG, "a product group mixes precisions");
        order[k] = k;
    }
    // the products with the costliest blocks first, so that the queue ends on short items
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return products[x].b > products[y].b; });
    std::vector<GroupDesc> d(n);
    int64_t chunks = 0;
    for (int k = 0; k < n; ++k) {
        const GroupProduct &q = products[order[k]];
        GroupDesc &e = d[k];
        PlanArgs &a = e.ga.p;
        a.n = q.n;
        a.upper = q.upper;
        a.c_ptr = q.c_ptr;
        a.nblocks = q.nblocks;
        a.perm = q.perm;
        a.item_ptr = q.item_ptr;
        a.items = q.items;
        a.a_ptr = q.a_ptr;
        a.x_ptr = q.x_ptr;
        a.c_row = q.c_row;
        a.c_col = q.c_col;
        a.A = q.A;
        a.X = q.X;
        a.C = q.C;
        a.alpha = q.alpha;
        a.beta = q.beta;
        e.ga.b = q.b;
        e.ga.a_tm = q.a_tm;
        e.ga.b_tm = q.b_tm;
        e.ta = q.ta;
        e.tb = q.tb;
        e.per_chunk = q.b == 4 ? 128 : 16;
        e.chunk0 = chunks;
        chunks += (q.nblocks + e.per_chunk - 1) / e.per_chunk;
    }
    void *dev = nullptr;
    LSQ_CUDA_TRY(cudaMalloc(&dev, sizeof(GroupDesc) * n));
    cudaError_t e = cudaMemcpy(dev, d.data(), sizeof(GroupDesc) * n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(dev);
        return set_error(LSQ_ERR_CUDA, std::string("uploading a product group: ") + cudaGetErrorString(e));
    }
    // one inlined frame form when every larger-block product is a t16 product with the same flags
    int fr = -1;
    for (int k = 0; k < n; ++k) {
        const GroupProduct &q = products[k];
        if (q.b == 4) continue;
        const int f = q.b >= 9 ? 2 * (q.ta != 0) + (q.tb != 0) : 4;
        fr = fr < 0 ? f : (fr == f ? fr : 4);
    }
    if (fr < 0) fr = 0;
    int per_sm = 1;
    const void *kern = group_kernel(dtype, fr);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0);
    out->desc = dev;
    out->nprod = n;
    out->dtype = dtype;
    out->form = fr;
    out->nchunks = chunks;
    out->grid = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, (int64_t)g_any->num_sms * std::max(per_sm, 1)));
    return LSQ_OK;
}

int group_launch(const GroupLaunch &gl, unsigned long long *counter, cudaStream_t s) {
    LSQ_CUDA_TRY(cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s));
    const GroupDesc *d = static_cast<const GroupDesc *>(gl.desc);
    int nd = gl.nprod;
    int64_t nch = gl.nchunks;
    void *args[] = {&d, &nd, &nch, &counter};
    note_launch();
    LSQ_CUDA_TRY(cudaLaunchKernel(group_kernel(gl.dtype, gl.form), dim3(gl.grid), dim3(256), args, 0, s));
    return LSQ_OK;
}

}  // namespace lsq
