// Sparse approximate inverse overlap by the Hotelling iteration (Sec. 2.3.2, after Eq. 8:
// the LNV minimisation uses an approximate sparse inverse of S as its metric, found with the
// iterative Hotelling method).
//
//   X_{n+1} = 2 X_n - (X_n S) X_n,   X S on its natural range, X S X restricted to R_X,
//
// from X_0 = S / s^2 on R_X, s the largest absolute row sum of S (a Gershgorin bound on its
// largest eigenvalue, so the spectrum of I - X_0 S lies in [0, 1) and the iteration
// converges).  X S X is symmetric: it is formed on the upper triangle and mirrored, and X stays
// symmetric to the last bit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>

#include "lsq_internal.h"

namespace lsq {
namespace {

constexpr int kHotBlocks = 1024;
constexpr int kHotThreads = 256;

// rowabs[i b + r] = sum over the blocks (i, j) of S and c of |S_ij[r][c]| (thread per scalar row).
__global__ void k_row_abs(int n, int b, const int64_t *__restrict__ sp, const double *__restrict__ S,
                          double *__restrict__ rowabs) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * b) return;
    const int i = (int)(t / b), r = (int)(t - (int64_t)i * b);
    const int bb = b * b;
    double s = 0.0;
    for (int64_t p = sp[i]; p < sp[i + 1]; ++p)
        for (int c = 0; c < b; ++c) s += fabs(S[p * bb + r * b + c]);
    rowabs[t] = s;
}

// out[0] = max of x[0..m) (one block, fixed order).
__global__ void k_max(int64_t m, const double *__restrict__ x, double *__restrict__ out) {
    __shared__ double sh[1024];
    double v = 0.0;
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) v = fmax(v, x[k]);
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

// X = S / s^2 on X's pattern (pos: position of each block of X in S's pattern, or -1).
__global__ void k_scaled_start(int64_t nnzb, int bb, const int64_t *__restrict__ pos,
                               const double *__restrict__ S, const double *__restrict__ s_dev,
                               double *__restrict__ X) {
    const double s = s_dev[0];
    const double inv = 1.0 / (s * s);
    const int64_t m = nnzb * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / bb;
        const int rc = (int)(e - p * bb);
        const int64_t q = pos[p];
        X[e] = q >= 0 ? inv * S[q * bb + rc] : 0.0;
    }
}

__global__ void k_f64_to_f32(int64_t m, const double *__restrict__ x, float *__restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}

// X = 2 X - U elementwise (as X + (X - U)), with per-block partial sums of (X - U)^2.
template <typename T>
__global__ void k_hot_update(int64_t m, const T *__restrict__ U, double *__restrict__ X,
                             double *__restrict__ partial) {
    __shared__ double sh[kHotThreads];
    double s = 0.0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const double x = X[e];
        const double d = x - (double)U[e];
        X[e] = x + d;
        s = fma(d, d, s);
    }
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum_sqrt(int m, const double *__restrict__ partial, double *__restrict__ out) {
    __shared__ double sh[kHotBlocks];
    double s = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) s += partial[k];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(sh[0]);
}

int grid_of(int64_t m) { return (int)std::max<int64_t>(1, std::min<int64_t>((m + 255) / 256, 8192)); }

}  // namespace
}  // namespace lsq

using namespace lsq;

extern "C" int lsq_hotelling_inverse(lsq_geom g, int b, int precision, int range_s, const double *S,
                                     int range_x, int range_xs, double *X, int start, int n_iter,
                                     double *dx_host, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g, range_s));
    LSQ_TRY(geom_check(g, range_x));
    LSQ_TRY(geom_check(g, range_xs));
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (precision != LSQ_F64 && precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64 or LSQ_F32");
    if (n_iter < 0) return set_error(LSQ_ERR_INVALID_ARG, "n_iter must be >= 0");
    const Pattern &PS = g->pats[range_s], &PX = g->pats[range_x], &PXS = g->pats[range_xs];
    if (PXS.R < PX.R + PS.R - 1e-9)
        return set_error(LSQ_ERR_INVALID_ARG, "range_xs must cover the natural range R_X + R_S of X S");
    if (g->n > 0 && (!S || !X)) return set_error(LSQ_ERR_INVALID_ARG, "null matrix pointer");
    if (g->n == 0) return LSQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int bb = b * b;
    const int64_t mx = PX.nnzb * bb, ms = PS.nnzb * bb, mxs = PXS.nnzb * bb;
    const size_t es = dtype_size(precision);
    // workspace held by g, grown on demand (a later call of the same or smaller sizes allocates
    // nothing): partial sums and scalars, row sums of |S|, X S, (X S) X and float32 copies
    auto up = [](size_t v) { return (v + 255) / 256 * 256; };
    const size_t o_red = 0, o_row = up(sizeof(double) * (kHotBlocks + 2));
    const size_t o_T = o_row + up(sizeof(double) * (size_t)g->n * b);
    const size_t o_U = o_T + up(es * (size_t)mxs);
    const size_t o_Xc = o_U + up(es * (size_t)mx);
    const size_t o_Sc = o_Xc + (precision == LSQ_F32 ? up(es * (size_t)mx) : 0);
    const size_t need = o_Sc + (precision == LSQ_F32 ? up(es * (size_t)ms) : 0);
    if (g->hot_ws.n < need) LSQ_TRY(g->hot_ws.alloc(need));
    char *ws = g->hot_ws.p;
    double *red = reinterpret_cast<double *>(ws + o_red);  // [kHotBlocks] partial sums, then scalars
    void *T = ws + o_T, *U = ws + o_U;
    float *Xc = reinterpret_cast<float *>(ws + o_Xc), *Sc = reinterpret_cast<float *>(ws + o_Sc);
    if (start) {
        double *rowabs = reinterpret_cast<double *>(ws + o_row);
        const int64_t *pos = nullptr;
        LSQ_TRY(get_posmap(g, range_x, range_s, 0, &pos, s));
        note_launch();
        k_row_abs<<<(int)(((int64_t)g->n * b + 255) / 256), 256, 0, s>>>(g->n, b, PS.row_ptr.p, S, rowabs);
        note_launch();
        k_max<<<1, 1024, 0, s>>>((int64_t)g->n * b, rowabs, red + kHotBlocks);
        note_launch();
        k_scaled_start<<<grid_of(mx), 256, 0, s>>>(PX.nnzb, bb, pos, S, red + kHotBlocks, X);
        LSQ_CHECK_LAUNCH();
    }
    const void *Sop = S;
    if (precision == LSQ_F32) {
        note_launch();
        k_f64_to_f32<<<grid_of(ms), 256, 0, s>>>(ms, S, Sc);
        LSQ_CHECK_LAUNCH();
        Sop = Sc;
    }
    for (int it = 0; it < n_iter; ++it) {
        const void *Xop = X;
        if (precision == LSQ_F32) {
            note_launch();
            k_f64_to_f32<<<grid_of(mx), 256, 0, s>>>(mx, X, Xc);
            LSQ_CHECK_LAUNCH();
            Xop = Xc;
        }
        // T = X S (S symmetric: op(B) = S^T = S, read as rows), U = (T X)|R_X on the upper
        // triangle, mirrored (X symmetric)
        LSQ_TRY(block_matmul(g, b, precision, range_x, 0, Xop, range_s, 1, Sop, range_xs, T, 1.0, 0.0,
                             nullptr, s));
        LSQ_TRY(block_matmul(g, b, precision, range_xs, 0, T, range_x, 1, Xop, range_x, U, 1.0, 0.0,
                             nullptr, s, 1));
        // U exactly symmetric keeps X exactly symmetric.  (The second product reads X as X^T;
        // an antisymmetric part of X would double at every step.)
        LSQ_TRY(sym_diag_on(g, range_x, b, precision, U, s));
        note_launch();
        if (precision == LSQ_F64)
            k_hot_update<double><<<kHotBlocks, kHotThreads, 0, s>>>(mx, (const double *)U, X, red);
        else
            k_hot_update<float><<<kHotBlocks, kHotThreads, 0, s>>>(mx, (const float *)U, X, red);
        note_launch();
        k_sum_sqrt<<<1, kHotBlocks, 0, s>>>(kHotBlocks, red, red + kHotBlocks + 1);
        LSQ_CHECK_LAUNCH();
        if (dx_host) {
            LSQ_CUDA_TRY(cudaMemcpyAsync(dx_host + it, red + kHotBlocks + 1, sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
            LSQ_CUDA_TRY(cudaStreamSynchronize(s));
        }
    }
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    return LSQ_OK;
}
