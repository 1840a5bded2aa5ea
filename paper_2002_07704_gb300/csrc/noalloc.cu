// Allocation-free variant of the trace Tr[X Y] (lsq_trace_static).
//
// lsq_trace keeps its per-block partial sums in device memory owned by
// the geometry and builds a position map on first use, so its first call
// allocates.  Some callers cannot allow that: code that owns all device
// memory through its own pool (a framework's caching allocator that has
// reserved HBM up front), or code that must not stall the device, since
// cudaMalloc and cudaFree can synchronise it.  This variant allocates
// nothing: it finds (j, i) in Y's pattern by binary search instead of a
// position map, and keeps one partial sum per atom row in a fixed,
// file-scope device array.
#include <cuda_runtime.h>

#include <string>

#include "lsq_internal.h"

namespace lsq {

// One float64 partial sum per atom row; 2 MiB, held by every device that loads the library.
constexpr int kStaticTraceRows = 262144;
static __device__ __align__(256) double g_trace_rows[kStaticTraceRows];

__device__ __forceinline__ int64_t find_col(const int64_t *__restrict__ ptr,
                                            const int32_t *__restrict__ col, int row, int key) {
    int64_t lo = ptr[row], hi = ptr[row + 1], end = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && col[lo] == key) ? lo : -1;
}

// One warp per atom row i of X: rows[i] = sum over (i, j) in X with (j, i) in Y of <X_ij, Y_ji^T>.
template <typename T>
__global__ void k_trace_rows(int n, int b, const int64_t *__restrict__ xp, const int32_t *__restrict__ xc,
                             const T *__restrict__ X, const int64_t *__restrict__ yp,
                             const int32_t *__restrict__ yc, const T *__restrict__ Y,
                             double *__restrict__ rows) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int i = warp, bb = b * b;
    double s = 0.0;
    for (int64_t p = xp[i]; p < xp[i + 1]; ++p) {
        const int64_t q = find_col(yp, yc, xc[p], i);
        if (q < 0) continue;
        for (int e = lane; e < bb; e += 32) {
            const int r = e / b, c = e - r * b;
            s += (double)X[p * bb + e] * (double)Y[q * bb + c * b + r];
        }
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) rows[i] = s;
}

// out = sum of rows[0..n), in a fixed order (one block).
__global__ void k_trace_rows_sum(int n, const double *__restrict__ rows, double *__restrict__ out) {
    __shared__ double sh[1024];
    double s = 0.0;
    for (int k = threadIdx.x; k < n; k += blockDim.x) s += rows[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0];
}

// Device address of g_trace_rows on the current device.  Looked up on every call: once the
// array's module is loaded on the device (by the geometry's creation, see noalloc_prime) the
// lookup neither allocates nor synchronises, and a reset device gets its new address.
static int static_rows_address(double **out) {
    void *p = nullptr;
    LSQ_CUDA_TRY(cudaGetSymbolAddress(&p, g_trace_rows));
    *out = static_cast<double *>(p);
    return LSQ_OK;
}

// Loads the array on the current device (the first symbol lookup does, allocating its 2 MiB),
// so that lsq_trace_static itself never does.  Called by lsq_build_neighbour_lists.
int noalloc_prime() {
    double *p = nullptr;
    return static_rows_address(&p);
}

}  // namespace lsq

using namespace lsq;

extern "C" int lsq_trace_static(lsq_geom g, int b, int precision, int range_x, const void *X,
                                int range_y, const void *Y, double *out_dev, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g, range_x));
    LSQ_TRY(geom_check(g, range_y));
    if (!out_dev) return set_error(LSQ_ERR_INVALID_ARG, "out_dev is null");
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (precision != LSQ_F64 && precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64 or LSQ_F32");
    if (g->n > kStaticTraceRows)
        return set_error(LSQ_ERR_UNSUPPORTED,
                         "lsq_trace_static handles at most 262144 atoms; the geometry has " +
                             std::to_string(g->n));
    if (g->n > 0 && (!X || !Y)) return set_error(LSQ_ERR_INVALID_ARG, "null matrix pointer");
    double *rows = nullptr;
    LSQ_TRY(static_rows_address(&rows));
    cudaStream_t s = (cudaStream_t)stream;
    const Pattern &PX = g->pats[range_x], &PY = g->pats[range_y];
    if (g->n > 0) {
        const int threads = 256;
        const int blocks = (int)(((int64_t)g->n * 32 + threads - 1) / threads);
        note_launch();
        if (precision == LSQ_F64)
            k_trace_rows<double><<<blocks, threads, 0, s>>>(g->n, b, PX.row_ptr.p, PX.col.p,
                                                            (const double *)X, PY.row_ptr.p,
                                                            PY.col.p, (const double *)Y, rows);
        else
            k_trace_rows<float><<<blocks, threads, 0, s>>>(g->n, b, PX.row_ptr.p, PX.col.p,
                                                           (const float *)X, PY.row_ptr.p, PY.col.p,
                                                           (const float *)Y, rows);
    }
    note_launch();
    k_trace_rows_sum<<<1, 1024, 0, s>>>(g->n, rows, out_dev);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}
