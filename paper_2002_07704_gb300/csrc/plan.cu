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
// Blocks of C are grouped 32 to a warp within a row of C, sorted by list
// length so that the lanes of a warp run lists of similar length; the
// items of a group are interleaved (item t of lane l at off + 32 t + l) so
// that each step of the warp reads 128 contiguous bytes of plan.  The
// numeric kernel then does no index search at all: each lane streams its
// list, gathers A_ik from row i (shared by the warp, cache resident) and
// X_jk from row j, and accumulates C_ij in registers.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "lsq_internal.h"

namespace lsq {

constexpr int kMaxPlanRow = 8192;  // longest row of C a plan handles (shared-memory sort)

// ---- symbolic product: item count of every block of C -----------------------
__global__ void __launch_bounds__(512) k_plan_count(int n, const int64_t *__restrict__ a_ptr,
                                                    const int32_t *__restrict__ a_col,
                                                    const int64_t *__restrict__ x_ptr,
                                                    const int32_t *__restrict__ x_col,
                                                    const int64_t *__restrict__ c_ptr,
                                                    const int32_t *__restrict__ c_col,
                                                    int32_t *__restrict__ cnt) {
    extern __shared__ int amap[];  // [n]
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    for (int j = tid; j < n; j += nth) amap[j] = -1;
    __syncthreads();
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t a0 = a_ptr[i], a1 = a_ptr[i + 1];
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = (int)(p - a0);
        __syncthreads();
        for (int64_t s = c_ptr[i] + warp; s < c_ptr[i + 1]; s += nwarps) {
            const int j = c_col[s];
            int c = 0;
            for (int64_t q = x_ptr[j] + lane; q < x_ptr[j + 1]; q += 32) c += amap[x_col[q]] >= 0;
            for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
            if (lane == 0) cnt[s] = c;
        }
        __syncthreads();
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = -1;
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

// ---- groups of 32 blocks: row, first index, lanes in use, longest list ------------
__global__ void k_plan_groups(int n, const int64_t *__restrict__ c_ptr,
                              const int64_t *__restrict__ gbase, const int64_t *__restrict__ perm,
                              const int32_t *__restrict__ cnt, int32_t *__restrict__ g_row,
                              int64_t *__restrict__ g_first, int32_t *__restrict__ g_nvalid,
                              int64_t *__restrict__ g_size) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t c0 = c_ptr[i], len = c_ptr[i + 1] - c0;
    int64_t g = gbase[i];
    for (int64_t f = 0; f < len; f += 32, ++g) {
        g_row[g] = i;
        g_first[g] = c0 + f;
        g_nvalid[g] = (int)min((int64_t)32, len - f);
        g_size[g] = 32 * (int64_t)cnt[perm[c0 + f]];  // sorted: the first block has the longest list
    }
}

__global__ void k_rows_to_groups(int n, const int64_t *__restrict__ c_ptr, int64_t *__restrict__ ng) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ng[i] = (c_ptr[i + 1] - c_ptr[i] + 31) / 32;
}

// Exclusive scan of int64 (one block).
__global__ void k_scan64(int64_t m, const int64_t *__restrict__ in, int64_t *__restrict__ out) {
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

// ---- fill the interleaved items ------------------------------------------------
__global__ void __launch_bounds__(512) k_plan_fill(int n, const int64_t *__restrict__ a_ptr,
                                                   const int32_t *__restrict__ a_col,
                                                   const int64_t *__restrict__ x_ptr,
                                                   const int32_t *__restrict__ x_col,
                                                   const int32_t *__restrict__ c_col,
                                                   const int64_t *__restrict__ gbase,
                                                   const int64_t *__restrict__ g_first,
                                                   const int32_t *__restrict__ g_nvalid,
                                                   const int64_t *__restrict__ g_off,
                                                   const int64_t *__restrict__ perm,
                                                   uint32_t *__restrict__ items) {
    extern __shared__ int amap[];
    const int tid = threadIdx.x, nth = blockDim.x;
    const int lane = tid & 31, warp = tid >> 5, nwarps = nth >> 5;
    for (int j = tid; j < n; j += nth) amap[j] = -1;
    __syncthreads();
    for (int i = blockIdx.x; i < n; i += gridDim.x) {
        const int64_t a0 = a_ptr[i], a1 = a_ptr[i + 1];
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = (int)(p - a0);
        __syncthreads();
        for (int64_t g = gbase[i] + warp; g < gbase[i + 1]; g += nwarps) {
            if (lane < g_nvalid[g]) {
                const int64_t s = perm[g_first[g] + lane];
                const int j = c_col[s];
                const int64_t x0 = x_ptr[j];
                int64_t w = g_off[g] + lane;
                for (int64_t q = x0; q < x_ptr[j + 1]; ++q) {
                    const int ao = amap[x_col[q]];
                    if (ao >= 0) {
                        items[w] = (uint32_t)ao | ((uint32_t)(q - x0) << 16);
                        w += 32;
                    }
                }
            }
        }
        __syncthreads();
        for (int64_t p = a0 + tid; p < a1; p += nth) amap[a_col[p]] = -1;
        __syncthreads();
    }
}

// ---- numeric product from a plan -------------------------------------------------
__device__ __forceinline__ void ldb(const double *__restrict__ p, double (&x)[16]) {
    const double2 *q = reinterpret_cast<const double2 *>(p);
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        double2 v = __ldg(q + k);
        x[2 * k] = v.x;
        x[2 * k + 1] = v.y;
    }
}
__device__ __forceinline__ void ldb(const float *__restrict__ p, float (&x)[16]) {
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

struct PlanArgs {
    int64_t ngroups;
    const int32_t *g_row;
    const int64_t *g_first;
    const int32_t *g_nvalid;
    const int64_t *g_off;
    const int64_t *perm;
    const int32_t *cnt;
    const uint32_t *items;
    const int64_t *a_ptr;
    const int64_t *x_ptr;
    const int32_t *c_col;
    const void *A;  // op(A), rows contiguous
    const void *X;  // op(B)^T, rows contiguous
    void *C;
    double alpha, beta;
};

// One warp per group of 32 blocks of one row of C; lane l owns block perm[first + l].
template <typename T>
__global__ void __launch_bounds__(256) k_mm_plan_b4(PlanArgs g) {
    const T *__restrict__ A = static_cast<const T *>(g.A);
    const T *__restrict__ X = static_cast<const T *>(g.X);
    T *__restrict__ C = static_cast<T *>(g.C);
    const int lane = threadIdx.x & 31;
    const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t gi = warp0; gi < g.ngroups; gi += nw) {
        const bool valid = lane < g.g_nvalid[gi];
        if (!valid) continue;
        const int64_t s = g.perm[g.g_first[gi] + lane];
        const int j = g.c_col[s];
        const T *__restrict__ arow = A + 16 * g.a_ptr[g.g_row[gi]];
        const T *__restrict__ xrow = X + 16 * g.x_ptr[j];
        const uint32_t *__restrict__ it = g.items + g.g_off[gi] + lane;
        const int nit = g.cnt[s];
        T acc[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) acc[e] = T(0);
        uint32_t cur = nit > 0 ? __ldg(it) : 0u;
        for (int t = 0; t < nit; ++t) {
            const uint32_t nxt = (t + 1 < nit) ? __ldg(it + 32 * (t + 1)) : 0u;
            T a[16], x[16];
            ldb(arow + 16 * (cur & 0xffffu), a);
            ldb(xrow + 16 * (cur >> 16), x);
            // B_kj = (X_jk)^T:  acc[r][c] += sum_t a[r][t] x[c][t]
#pragma unroll
            for (int r = 0; r < 4; ++r)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                    T v = acc[r * 4 + c];
                    v = fma(a[r * 4 + 0], x[c * 4 + 0], v);
                    v = fma(a[r * 4 + 1], x[c * 4 + 1], v);
                    v = fma(a[r * 4 + 2], x[c * 4 + 2], v);
                    v = fma(a[r * 4 + 3], x[c * 4 + 3], v);
                    acc[r * 4 + c] = v;
                }
            cur = nxt;
        }
        T *dst = C + 16 * s;
        if (g.beta != 0.0) {
#pragma unroll
            for (int e = 0; e < 16; ++e) dst[e] = fma((T)g.beta, dst[e], (T)g.alpha * acc[e]);
        } else {
#pragma unroll
            for (int e = 0; e < 16; ++e) dst[e] = (T)g.alpha * acc[e];
        }
    }
}

static int grid64(int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 65535)); }

int plan_build(lsq_geom g, int ra, int rb, int rc, ProductPlan **out, cudaStream_t s) {
    auto key = std::make_tuple(ra, rb, rc);
    auto it = g->pplans.find(key);
    if (it != g->pplans.end()) {
        *out = &it->second;
        return LSQ_OK;
    }
    const Pattern &PA = g->pats[ra], &PB = g->pats[rb], &PC = g->pats[rc];
    const int n = g->n;
    if (PA.max_row > 65535 || PB.max_row > 65535 || PC.max_row > kMaxPlanRow)
        return set_error(LSQ_ERR_UNSUPPORTED, "row too long for a product plan");
    if ((size_t)n * sizeof(int) + 1024 > g->smem_optin)
        return set_error(LSQ_ERR_UNSUPPORTED, "too many atoms for the shared-memory atom map");
    ProductPlan p;
    const int64_t nc = PC.nnzb;
    DevBuf<int64_t> ng, gbase, gsize;
    LSQ_TRY(p.cnt.alloc(nc));
    LSQ_TRY(p.perm.alloc(nc));
    LSQ_TRY(ng.alloc((size_t)n + 1));
    LSQ_TRY(gbase.alloc((size_t)n + 1));
    int per_sm = 1;
    size_t smem_map = (size_t)n * sizeof(int);
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_plan_count, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_map));
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_plan_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_map));
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_plan_count, 512, smem_map);
    const int grid_rows = std::max(1, std::min(n, g->num_sms * std::max(per_sm, 1)));
    if (n > 0) {
        note_launch();
        k_plan_count<<<grid_rows, 512, smem_map, s>>>(n, PA.row_ptr.p, PA.col.p, PB.row_ptr.p, PB.col.p,
                                                      PC.row_ptr.p, PC.col.p, p.cnt.p);
        LSQ_CHECK_LAUNCH();
        int m = 1;
        while (m < PC.max_row) m <<= 1;
        size_t smem_sort = sizeof(unsigned long long) * (size_t)std::max(m, 1);
        LSQ_CUDA_TRY(cudaFuncSetAttribute(k_plan_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_sort));
        note_launch();
        k_plan_sort<<<std::min(n, g->num_sms * 2), 512, smem_sort, s>>>(n, PC.row_ptr.p, p.cnt.p, p.perm.p);
        note_launch();
        k_rows_to_groups<<<(n + 255) / 256, 256, 0, s>>>(n, PC.row_ptr.p, ng.p);
        note_launch();
        k_scan64<<<1, 1024, 0, s>>>(n, ng.p, gbase.p);
        LSQ_CHECK_LAUNCH();
    }
    int64_t ngroups = 0;
    if (n > 0) {
        LSQ_CUDA_TRY(cudaMemcpyAsync(&ngroups, gbase.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    p.ngroups = ngroups;
    LSQ_TRY(p.g_row.alloc(ngroups));
    LSQ_TRY(p.g_first.alloc(ngroups));
    LSQ_TRY(p.g_nvalid.alloc(ngroups));
    LSQ_TRY(p.g_off.alloc((size_t)ngroups + 1));
    LSQ_TRY(gsize.alloc(ngroups));
    int64_t nitems = 0;
    if (ngroups > 0) {
        note_launch();
        k_plan_groups<<<(n + 255) / 256, 256, 0, s>>>(n, PC.row_ptr.p, gbase.p, p.perm.p, p.cnt.p, p.g_row.p,
                                                      p.g_first.p, p.g_nvalid.p, gsize.p);
        note_launch();
        k_scan64<<<1, 1024, 0, s>>>(ngroups, gsize.p, p.g_off.p);
        LSQ_CHECK_LAUNCH();
        LSQ_CUDA_TRY(cudaMemcpyAsync(&nitems, p.g_off.p + ngroups, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    LSQ_TRY(p.items.alloc((size_t)std::max<int64_t>(nitems, 1)));
    if (ngroups > 0) {
        note_launch();
        k_plan_fill<<<grid_rows, 512, smem_map, s>>>(n, PA.row_ptr.p, PA.col.p, PB.row_ptr.p, PB.col.p,
                                                     PC.col.p, gbase.p, p.g_first.p, p.g_nvalid.p,
                                                     p.g_off.p, p.perm.p, p.items.p);
        LSQ_CHECK_LAUNCH();
    }
    // exact triple count = sum of list lengths
    {
        std::vector<int32_t> h((size_t)std::max<int64_t>(nc, 1));
        if (nc > 0) {
            LSQ_CUDA_TRY(cudaMemcpyAsync(h.data(), p.cnt.p, sizeof(int32_t) * nc, cudaMemcpyDeviceToHost, s));
            LSQ_CUDA_TRY(cudaStreamSynchronize(s));
        }
        int64_t t = 0;
        for (int64_t e = 0; e < nc; ++e) t += h[e];
        p.triples = t;
        p.nitems = nitems;
    }
    *out = &g->pplans.emplace(key, std::move(p)).first->second;
    return LSQ_OK;
}

int plan_launch(lsq_geom g, int dtype, const ProductPlan &p, int ra, int rb, int rc, const void *Aop,
                const void *X, void *C, double alpha, double beta, cudaStream_t s) {
    if (p.ngroups == 0) return LSQ_OK;
    PlanArgs a;
    a.ngroups = p.ngroups;
    a.g_row = p.g_row.p;
    a.g_first = p.g_first.p;
    a.g_nvalid = p.g_nvalid.p;
    a.g_off = p.g_off.p;
    a.perm = p.perm.p;
    a.cnt = p.cnt.p;
    a.items = p.items.p;
    a.a_ptr = g->pats[ra].row_ptr.p;
    a.x_ptr = g->pats[rb].row_ptr.p;
    a.c_col = g->pats[rc].col.p;
    a.A = Aop;
    a.X = X;
    a.C = C;
    a.alpha = alpha;
    a.beta = beta;
    const int threads = 256;
    const int64_t warps = p.ngroups;
    int grid = (int)std::min<int64_t>((warps * 32 + threads - 1) / threads, (int64_t)g->num_sms * 64);
    grid = std::max(grid, 1);
    note_launch();
    if (dtype == LSQ_F64)
        k_mm_plan_b4<double><<<grid, threads, 0, s>>>(a);
    else
        k_mm_plan_b4<float><<<grid, threads, 0, s>>>(a);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

}  // namespace lsq
