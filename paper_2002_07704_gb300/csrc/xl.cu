// Extended-Lagrangian propagation of the density matrix between MD steps (Sec. 3.3).
//
// An auxiliary sparse matrix X, associated with L S, follows a harmonic potential centred on
// the ground state L(t) S(t).  Its Verlet step, with the dissipative sum the paper adds, is
//
//   X(t + dt) = 2 X(t) - X(t - dt) + kappa (L(t) S(t) - X(t)) + a sum_{m=0}^{M} c_m X(t - m dt),
//
// kappa = dt^2 w^2, and X S^-1 is the next step's initial L (here: its symmetric part on L's
// range).  When the atoms move, the matrices carried from one step to the next move to the
// new geometry's patterns block by block, matched by atom pair.
//
// Three entry points, each one or two kernels: the pattern move (index work, exact copies),
// the fused propagation (M + 3 reads and one write per value, bound by the FP64 pipe), and
// the initial L (one truncated product and an in-place symmetric part).
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <type_traits>

#include "lsq_internal.h"

namespace lsq {
namespace {

constexpr int kMaxHist = 10;

// Block (i, j) of the target pattern takes block (i, j) of the source pattern where the
// source stores it, else zero.  One warp per row: each lane finds one target block's source
// by binary search in the (ascending) source row, then the warp copies the chunk's blocks
// together, lane l taking values l, l + 32, ... of the chunk (coalesced writes; the reads are
// too wherever consecutive target blocks have consecutive sources).
template <typename T>
__global__ void k_remap_rows(int n, int bb, const int64_t *__restrict__ fp, const int32_t *__restrict__ fc,
                             const T *__restrict__ Xf, const int64_t *__restrict__ tp,
                             const int32_t *__restrict__ tc, T *__restrict__ Xt) {
    const int lane = threadIdx.x & 31;
    const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = w0; i < n; i += nw) {
        const int64_t f0 = fp[i], f1 = fp[i + 1], t1 = tp[i + 1];
        for (int64_t base = tp[i]; base < t1; base += 32) {
            const int64_t e = base + lane;
            int64_t src = -1;
            if (e < t1) {
                const int j = tc[e];
                int64_t lo = f0, hi = f1;  // first position with column >= j
                while (lo < hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    if (fc[mid] < j) lo = mid + 1;
                    else hi = mid;
                }
                if (lo < f1 && fc[lo] == j) src = lo;
            }
            // the chunk's nb blocks are contiguous in the target: lanes take consecutive values
            const int nv = (int)(t1 - base < 32 ? t1 - base : 32) * bb;
            T *dst = Xt + base * bb;
            for (int v0 = 0; v0 < nv; v0 += 32) {
                const int v = v0 + lane;
                const int t = (v < nv ? v : nv - 1) / bb;
                const int64_t s = __shfl_sync(0xffffffffu, src, t);
                if (v < nv) dst[v] = s >= 0 ? Xf[s * bb + (v - t * bb)] : T(0);
            }
        }
    }
}

struct XlArgs {
    const double *X[kMaxHist];  // X(t), X(t - dt), ...
    const double *LS;
    double w[kMaxHist];  // weight of each history entry
    int nh;              // history entries read (2 .. kMaxHist)
    double kappa;        // weight of L S
    double *out;
    int64_t m;
};

// The Verlet step with dissipation, its terms grouped by history entry,
//   X(t + dt) = kappa LS + (2 - kappa + a c_0) X(t) + (-1 + a c_1) X(t - dt) + sum_{m>=2} a c_m X(t - m dt),
// one FMA per entry.  The FP64 pipe, not HBM, bounds this kernel on this GPU (with six
// history entries, seven FP64 instructions per 64 bytes moved against a ridge near 0.08 per
// byte), so every FP64 instruction counts: the terms are grouped (about half the FP64
// instructions of the formula evaluated term by term) and the history length NH is a template
// argument (a loop unrolled to a fixed maximum and predicated still issues its idle FMAs).  All
// loads of a value issue together; V values per thread (16-byte loads for V = 2).  out may be
// one of the history arrays: each value is read before it is written, by the same thread.
template <int V, int NH>
__device__ __forceinline__ void xl_values(const XlArgs &a, int64_t e) {
    using VT = typename std::conditional<V == 2, double2, double>::type;
    auto ld = [&](const double *p) { return *reinterpret_cast<const VT *>(p + e); };
    auto part = [](const VT &x, int j) -> double {
        if constexpr (V == 2) return j == 0 ? x.x : x.y;
        else return x;
    };
    VT xk[NH];
    const VT ls = ld(a.LS);
#pragma unroll
    for (int k = 0; k < NH; ++k) xk[k] = ld(a.X[k]);
    double o[V];
#pragma unroll
    for (int j = 0; j < V; ++j) {
        double r = a.kappa * part(ls, j);
#pragma unroll
        for (int k = 0; k < NH; ++k) r = fma(a.w[k], part(xk[k], j), r);
        o[j] = r;
    }
    if constexpr (V == 2) *reinterpret_cast<double2 *>(a.out + e) = make_double2(o[0], o[1]);
    else a.out[e] = o[0];
}

template <int V, int NH>
__global__ void __launch_bounds__(256) k_xl_propagate(XlArgs a) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x * V;
    const int64_t mv = a.m / V * V;
    for (int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * V; e < mv; e += stride)
        xl_values<V, NH>(a, e);
    // the odd tail value (V = 2, m odd)
    if (V == 2 && blockIdx.x == 0 && threadIdx.x == 0 && mv < a.m) xl_values<1, NH>(a, mv);
}

template <int V>
void launch_propagate(const XlArgs &a, int grid, cudaStream_t s) {
    switch (a.nh) {
    case 2: k_xl_propagate<V, 2><<<grid, 256, 0, s>>>(a); break;
    case 3: k_xl_propagate<V, 3><<<grid, 256, 0, s>>>(a); break;
    case 4: k_xl_propagate<V, 4><<<grid, 256, 0, s>>>(a); break;
    case 5: k_xl_propagate<V, 5><<<grid, 256, 0, s>>>(a); break;
    case 6: k_xl_propagate<V, 6><<<grid, 256, 0, s>>>(a); break;
    case 7: k_xl_propagate<V, 7><<<grid, 256, 0, s>>>(a); break;
    case 8: k_xl_propagate<V, 8><<<grid, 256, 0, s>>>(a); break;
    case 9: k_xl_propagate<V, 9><<<grid, 256, 0, s>>>(a); break;
    default: k_xl_propagate<V, 10><<<grid, 256, 0, s>>>(a); break;
    }
}

// X = (X + X^T) / 2 in place on a symmetric pattern: the thread of the entry with p <= tm[p]
// reads both blocks of the pair and writes both, so the result is exactly symmetric.
__global__ void k_sym_part_inplace(int64_t nnzb, int b, const int64_t *__restrict__ tm, double *X) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int bb = b * b;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnzb; p += stride) {
        const int64_t q = tm[p];
        if (q < p) continue;
        double *P = X + p * bb, *Q = X + q * bb;
        if (q == p) {
            for (int r = 0; r < b; ++r)
                for (int c = r + 1; c < b; ++c) {
                    const double v = __dmul_rn(0.5, __dadd_rn(P[r * b + c], P[c * b + r]));
                    P[r * b + c] = v;
                    P[c * b + r] = v;
                }
        } else {
            for (int r = 0; r < b; ++r)
                for (int c = 0; c < b; ++c) {
                    const double v = __dmul_rn(0.5, __dadd_rn(P[r * b + c], Q[c * b + r]));
                    P[r * b + c] = v;
                    Q[c * b + r] = v;
                }
        }
    }
}

__global__ void k_to_f32(int64_t m, const double *__restrict__ x, float *__restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) y[e] = (float)x[e];
}

__global__ void k_to_f64(int64_t m, const float *__restrict__ x, double *__restrict__ y) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += stride) y[e] = (double)x[e];
}

int grid_of(int64_t m, int threads = 256) {
    return (int)std::max<int64_t>(1, std::min<int64_t>((m + threads - 1) / threads, 152 * 16));
}

}  // namespace
}  // namespace lsq

using namespace lsq;

extern "C" int lsq_pattern_remap(lsq_geom g_from, int range_from, lsq_geom g_to, int range_to, int b,
                                 int precision, const void *X_from, void *X_to, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g_from, range_from));
    LSQ_TRY(geom_check(g_to, range_to));
    if (g_from->n != g_to->n) return set_error(LSQ_ERR_INVALID_ARG, "the geometries hold different atom counts");
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (precision != LSQ_F64 && precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64 or LSQ_F32");
    const Pattern &F = g_from->pats[range_from], &T = g_to->pats[range_to];
    if (T.nnzb == 0 || g_to->n == 0) return LSQ_OK;
    if (!X_to || (F.nnzb > 0 && !X_from)) return set_error(LSQ_ERR_INVALID_ARG, "null matrix pointer");
    if (X_from == X_to) return set_error(LSQ_ERR_INVALID_ARG, "X_to must not alias X_from");
    cudaStream_t s = (cudaStream_t)stream;
    const int grid = grid_of((int64_t)g_to->n * 32);
    note_launch();
    if (precision == LSQ_F64)
        k_remap_rows<double><<<grid, 256, 0, s>>>(g_to->n, b * b, F.row_ptr.p, F.col.p, (const double *)X_from,
                                                  T.row_ptr.p, T.col.p, (double *)X_to);
    else
        k_remap_rows<float><<<grid, 256, 0, s>>>(g_to->n, b * b, F.row_ptr.p, F.col.p, (const float *)X_from,
                                                 T.row_ptr.p, T.col.p, (float *)X_to);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

extern "C" int lsq_xl_propagate(lsq_geom g, int b, int range_x, int n_hist, const double *const *X_hist,
                                const double *LS, double kappa, double alpha, const double *c, int n_c,
                                double *X_next, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g, range_x));
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (n_hist < 2 || n_hist > kMaxHist)
        return set_error(LSQ_ERR_INVALID_ARG, "n_hist must be in [2, " + std::to_string(kMaxHist) + "]");
    if (!X_hist) return set_error(LSQ_ERR_INVALID_ARG, "null history array");
    if (alpha != 0.0 && (!c || n_c < 1 || n_c > n_hist))
        return set_error(LSQ_ERR_INVALID_ARG, "dissipation needs 1 <= n_c <= n_hist coefficients");
    const int64_t m = g->pats[range_x].nnzb * (int64_t)(b * b);
    if (m == 0) return LSQ_OK;
    XlArgs a;
    for (int k = 0; k < n_hist; ++k) {
        if (!X_hist[k]) return set_error(LSQ_ERR_INVALID_ARG, "null history matrix");
        a.X[k] = X_hist[k];
    }
    if (!LS || !X_next) return set_error(LSQ_ERR_INVALID_ARG, "null matrix pointer");
    if (X_next == LS) return set_error(LSQ_ERR_INVALID_ARG, "X_next must not alias LS");
    // weights of the history entries: 2 - kappa and -1 from the Verlet step, a c_m from the
    // dissipation; entries beyond both are not read
    const int nc = alpha != 0.0 ? n_c : 0;
    a.nh = std::max(2, nc);
    for (int k = 0; k < a.nh; ++k) {
        double w = k == 0 ? 2.0 - kappa : (k == 1 ? -1.0 : 0.0);
        if (k < nc) w += alpha * c[k];
        a.w[k] = w;
    }
    a.LS = LS;
    a.kappa = kappa;
    a.out = X_next;
    a.m = m;
    bool al16 = reinterpret_cast<uintptr_t>(LS) % 16 == 0 && reinterpret_cast<uintptr_t>(X_next) % 16 == 0;
    for (int k = 0; k < a.nh; ++k) al16 = al16 && reinterpret_cast<uintptr_t>(X_hist[k]) % 16 == 0;
    note_launch();
    if (al16)
        launch_propagate<2>(a, grid_of((m + 1) / 2), (cudaStream_t)stream);
    else
        launch_propagate<1>(a, grid_of(m), (cudaStream_t)stream);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

extern "C" int lsq_xl_initial_L(lsq_geom g, int b, int precision, int range_x, const double *X, int range_sinv,
                                const double *Sinv, int range_l, double *L_out, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g, range_x));
    LSQ_TRY(geom_check(g, range_sinv));
    LSQ_TRY(geom_check(g, range_l));
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (precision != LSQ_F64 && precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64 or LSQ_F32");
    if (g->n > 0 && (!X || !Sinv || !L_out)) return set_error(LSQ_ERR_INVALID_ARG, "null matrix pointer");
    if ((const void *)L_out == (const void *)X || (const void *)L_out == (const void *)Sinv)
        return set_error(LSQ_ERR_INVALID_ARG, "L_out must not alias X or Sinv");
    if (g->n == 0) return LSQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t bb = (int64_t)b * b;
    const int64_t mx = g->pats[range_x].nnzb * bb, ms = g->pats[range_sinv].nnzb * bb;
    const int64_t ml = g->pats[range_l].nnzb * bb;
    if (precision == LSQ_F64) {
        LSQ_TRY(block_matmul(g, b, LSQ_F64, range_x, 0, X, range_sinv, 0, Sinv, range_l, L_out, 1.0, 0.0, nullptr,
                             s));
    } else {
        // float32 copies of the operands, the product in float32, the result widened
        auto up16 = [](int64_t m) { return (m * (int64_t)sizeof(float) + 255) / 256 * 256; };
        const size_t need = (size_t)(up16(mx) + up16(ms) + up16(ml));
        if (g->xl_scratch.n < need) {
            LSQ_CUDA_TRY(cudaStreamSynchronize(s));  // the old buffer may still be read
            LSQ_TRY(g->xl_scratch.alloc(need));
        }
        float *X32 = reinterpret_cast<float *>(g->xl_scratch.p);
        float *S32 = reinterpret_cast<float *>(g->xl_scratch.p + up16(mx));
        float *P32 = reinterpret_cast<float *>(g->xl_scratch.p + up16(mx) + up16(ms));
        note_launch();
        k_to_f32<<<grid_of(mx), 256, 0, s>>>(mx, X, X32);
        note_launch();
        k_to_f32<<<grid_of(ms), 256, 0, s>>>(ms, Sinv, S32);
        LSQ_CHECK_LAUNCH();
        LSQ_TRY(block_matmul(g, b, LSQ_F32, range_x, 0, X32, range_sinv, 0, S32, range_l, P32, 1.0, 0.0, nullptr,
                             s));
        note_launch();
        k_to_f64<<<grid_of(ml), 256, 0, s>>>(ml, P32, L_out);
        LSQ_CHECK_LAUNCH();
    }
    LSQ_TRY(ensure_tmap(g, range_l, s));
    const int64_t nnzb = g->pats[range_l].nnzb;
    note_launch();
    k_sym_part_inplace<<<grid_of(nnzb), 256, 0, s>>>(nnzb, b, g->pats[range_l].tmap.p, L_out);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}
