// LNV grand-potential minimisation on the GPU (Sec. 2.3.2 of the paper).
//
// K = 3LSL - 2LSLSL (the McWeeny form, Eq. 8) drives the density matrix
// towards weak idempotency; K has the range of H while L's range is
// restricted; E_band = 2 Tr[K H] is minimised with respect to L, the
// electron number held by a chemical potential mu.  With H' = H - mu S:
//
//   Omega = 2 Tr[K H'],  N_e = 2 Tr[K S]
//   G     = 2 [3 (Q + Q^T) - 2 (G1 + G1^T + G2)] on L's range,
//           Q = H'LS, G1 = Q.LS, G2 = Q^T.LS (= SLH'LS)
//
// Products per energy + gradient (ranges in brackets, R3 = R_H+R_L+R_S):
//   LS = L.S [R_L+R_S], LSL = (LS.L)|R3, Q = H'.LS [R3], and for the gradient one triangle
//   each on R_L of T1 = (Q + Q^T).LS (formed as its transpose SL.(Q + Q^T)) and T2 = SL.Q^T,
//   whose sum is the symmetric G1 + G1^T + G2;
//   Omega = 2 (3 Tr[H' LSL] - 2 <LSL, Q>), since Tr[LSLSLH'] = Tr[LSL (SLH')] and
//   SLH' = Q^T; N_e = 2 (3 Tr[S LSL] - 2 <LSL, SLS>) with SLS = S.LS [R3].
// When the gradient is formed, LSL is not needed: by the cyclic property,
//   Tr[LSLH'] = <L, Q> and Tr[LSLSLH'] = <L, G1> = <L, G1^T> = <L, G2> = <L, M> / 3
// over L's range, so Omega = 2 (3 <L, Q> - (2/3) <L, M>) comes out of the gradient's own
// data in the same pass as the combine.
// Exact line search along D: Omega(L + a D) = Omega + c1 a + c2 a^2 + c3 a^3,
//   c1 = <G, D>,  c2 = 2 (3 t2 - 2 (2 t3a + t3b)),  c3 = -4 t4, with
//   P = D.S, QD = H'.P, F = (P.D)|[R_H+R_L+R_S] (= DSD), Z = (QD^T.P)|R_L,
//   t2 = Tr[F H'] = Tr[DSDH'], t3a = <F, Q> = Tr[DSDSLH'] (= Tr[LSDSDH']),
//   t3b = <L, Z> = Tr[DSLSDH'], t4 = <D, Z> = Tr[DSDSDH'] (= <F, QD>),
// using the symmetry of S, H', L and D and the cyclic property of the trace.
// All matrices are symmetric; the CG keeps L exactly symmetric.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <memory>
#include <string>
#include <vector>

#include "lsq_internal.h"

namespace lsq {

constexpr double kHartreeEv = 27.211386245988;

// ---- elementwise kernels ---------------------------------------------------
__global__ void k_to_f32(int64_t m, const double *__restrict__ x, float *__restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (float)x[e];
}

__global__ void k_f32_to_f64(int64_t m, const float *__restrict__ x, double *__restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        y[e] = (double)x[e];
}

// H' = H - mu S_H and S_H (S placed on H's pattern; zero where S has no block).
__global__ void k_hprime(int64_t nnzb, int bb, const double *__restrict__ H,
                         const double *__restrict__ S, const int64_t *__restrict__ pos_s, double mu,
                         double *__restrict__ Hp, double *__restrict__ Sh) {
    int64_t m = nnzb * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x) {
        int64_t p = e / bb;
        int rc = (int)(e - p * bb);
        int64_t q = pos_s[p];
        double s = q >= 0 ? S[q * bb + rc] : 0.0;
        Sh[e] = s;
        Hp[e] = H[e] - mu * s;
    }
}

// The gradient from M = G1 + G1^T + G2 = (Q + Q^T).LS + SL.Q^T = T1 + T2, held as the lower
// triangle (j <= i) of T1^T = SL.(Q + Q^T) (array T1t) and the upper triangle (j >= i) of
// T2 = SL.Q^T:
//   G_ij[r][c] = spin (3 (Q_ij[r][c] + Q_ji[c][r]) - 2 M_ij[r][c]),
// M_ij = (T1t_ji)^T + T2_ij for j > i, its transpose for j < i, and the symmetric part for
// j = i.  A block (i, j) of the symmetric pattern precedes (j, i) exactly when i < j, so
// p < tmL[p] selects the upper blocks.  Every element of G and its mirror sum the same
// values in the same order: G is symmetric to the last bit.
// One warp per row i of L's pattern; the same pass forms the two energy terms of the row:
// row0[i] = sum_j <L_ij, Q_ij> and row1[i] = sum_j <L_ij, M_ij> / 3 (see the header), with L
// as the products read it (its float32 copy on the mixed path).
template <typename T, int B>
__global__ void k_grad_omega_rows(int n, int b_rt, double spin, const int64_t *__restrict__ rp,
                                  const int64_t *__restrict__ pq, const int64_t *__restrict__ pqt,
                                  const int64_t *__restrict__ tmL, const T *__restrict__ L,
                                  const T *__restrict__ Q, const T *__restrict__ T1t, const T *__restrict__ T2,
                                  double *__restrict__ G, double *__restrict__ row0, double *__restrict__ row1) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int b = B > 0 ? B : b_rt;
    const int bb = b * b;
    double s0 = 0.0, s1 = 0.0;
    const uint64_t e1 = (uint64_t)rp[warp + 1] * bb;
    for (uint64_t e = (uint64_t)rp[warp] * bb + lane; e < e1; e += 32) {
        const int64_t p = (int64_t)(e / (uint64_t)bb);
        const int rc = (int)(e - (uint64_t)p * bb);
        const int r = rc / b, c = rc - r * b;
        const int64_t tr = c * b + r;
        const int64_t a = pq[p], at = pqt[p], t = tmL[p];
        const double qd = a >= 0 ? (double)Q[a * bb + rc] : 0.0;
        const double q = qd + (at >= 0 ? (double)Q[at * bb + tr] : 0.0);
        double mv;
        if (p < t) {
            mv = (double)T1t[t * bb + tr] + (double)T2[p * bb + rc];
        } else if (p > t) {
            mv = (double)T1t[p * bb + rc] + (double)T2[t * bb + tr];
        } else {
            mv = 0.5 * (((double)T1t[p * bb + tr] + (double)T2[p * bb + rc]) +
                        ((double)T1t[p * bb + rc] + (double)T2[p * bb + tr]));
        }
        G[e] = spin * (3.0 * q - 2.0 * mv);
        const double l = (double)L[e];
        s0 = fma(l, qd, s0);
        s1 = fma(l, mv, s1);
    }
    for (int off = 16; off > 0; off >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, off);
        s1 += __shfl_xor_sync(0xffffffffu, s1, off);
    }
    if (lane == 0) {
        row0[warp] = s0;
        row1[warp] = s1 / 3.0;
    }
}

__global__ void k_cg_dir(int64_t m, double beta, const double *__restrict__ G, double *__restrict__ D) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        D[e] = beta == 0.0 ? -G[e] : -G[e] + beta * D[e];
}

__global__ void k_axpy_f32(int64_t m, double a, const float *__restrict__ x, float *__restrict__ y) {
    const float af = (float)a;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = fmaf(af, x[e], y[e]);
}

__global__ void k_axpy(int64_t m, double a, const double *__restrict__ x, double *__restrict__ y) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m;
         e += (int64_t)gridDim.x * blockDim.x)
        y[e] = y[e] + a * x[e];
}

// L_ii = (inv(S_ii) + inv(S_ii)^T) / 4, by Gauss-Jordan elimination with partial pivoting.
__global__ void k_onsite_inverse(int n, int b, const int64_t *__restrict__ sp,
                                 const int32_t *__restrict__ sc, const double *__restrict__ S,
                                 const int64_t *__restrict__ lp, const int32_t *__restrict__ lc,
                                 double *__restrict__ L, int *__restrict__ bad) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    auto find = [](const int64_t *ptr, const int32_t *col, int row, int key) -> int64_t {
        int64_t lo = ptr[row], hi = ptr[row + 1], end = hi;
        while (lo < hi) {
            int64_t mid = (lo + hi) >> 1;
            if (col[mid] < key) lo = mid + 1;
            else hi = mid;
        }
        return (lo < end && col[lo] == key) ? lo : -1;
    };
    int64_t ps = find(sp, sc, i, i), pl = find(lp, lc, i, i);
    if (ps < 0 || pl < 0) {
        atomicExch(bad, 1);
        return;
    }
    double a[16][32];
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < 2 * b; ++c)
            a[r][c] = c < b ? S[ps * b * b + r * b + c] : (c - b == r ? 1.0 : 0.0);
    for (int col = 0; col < b; ++col) {
        int piv = col;
        for (int r = col + 1; r < b; ++r)
            if (fabs(a[r][col]) > fabs(a[piv][col])) piv = r;
        if (a[piv][col] == 0.0) {
            atomicExch(bad, 1);
            return;
        }
        if (piv != col)
            for (int c = 0; c < 2 * b; ++c) {
                double t = a[col][c];
                a[col][c] = a[piv][c];
                a[piv][c] = t;
            }
        double inv = 1.0 / a[col][col];
        for (int c = 0; c < 2 * b; ++c) a[col][c] *= inv;
        for (int r = 0; r < b; ++r)
            if (r != col) {
                double f = a[r][col];
                if (f != 0.0)
                    for (int c = 0; c < 2 * b; ++c) a[r][c] -= f * a[col][c];
            }
    }
    for (int r = 0; r < b; ++r)
        for (int c = 0; c < b; ++c) L[pl * b * b + r * b + c] = 0.25 * (a[r][b + c] + a[c][b + r]);
}

// ============================================================================
// Batched minimisation: many independent systems held block-diagonally in one
// geometry (lsq_geom_concat).  Every product, trace and update of a CG step is
// one launch over all systems; the per-system scalars (Omega, the CG beta, the
// line coefficients and alpha) are reduced and computed on the device, so a
// whole step is captured once in a CUDA graph and replayed.
// ============================================================================
constexpr int kSlots = 16;

// warp per row: rowsum[i] = sum over the row's blocks of <X_p, Y_p>
template <typename T>
__global__ void k_rowdot(int n, int bb, const int64_t *__restrict__ rp, const T *__restrict__ X,
                         const T *__restrict__ Y, double *__restrict__ rowsum) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    double s = 0.0;
    for (int64_t e = rp[warp] * bb + lane; e < rp[warp + 1] * bb; e += 32) s += (double)X[e] * (double)Y[e];
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) rowsum[warp] = s;
}

// float32 operands: each lane sums groups of 8 products as float pairs (dot2_add) and adds
// each group to its float64 sum, so the float64 pipe sees one addition per 8 terms.
template <>
__global__ void k_rowdot<float>(int n, int bb, const int64_t *__restrict__ rp, const float *__restrict__ X,
                                const float *__restrict__ Y, double *__restrict__ rowsum) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    double acc = 0.0;
    float s = 0.f, c = 0.f;
    int k = 0;
    for (int64_t e = rp[warp] * bb + lane; e < rp[warp + 1] * bb; e += 32) {
        dot2_add(X[e], Y[e], s, c);
        if (++k == 8) {
            acc += (double)s + (double)c;
            s = c = 0.f;
            k = 0;
        }
    }
    acc += (double)s + (double)c;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) rowsum[warp] = acc;
}

// warp per row i of X: rowsum[i] = sum over (i, j) in X of <X_ij, (Y_ji)^T> (pm: posmap X -> Y^T)
template <typename T>
__global__ void k_rowtrace(int n, int b, const int64_t *__restrict__ xp, const int64_t *__restrict__ pm,
                           const T *__restrict__ X, const T *__restrict__ Y, double *__restrict__ rowsum) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const int bb = b * b;
    double s = 0.0;
    for (int64_t e = xp[warp] * bb + lane; e < xp[warp + 1] * bb; e += 32) {
        const int64_t p = e / bb;
        const int rc = (int)(e - p * bb);
        const int64_t q = pm[p];
        if (q < 0) continue;
        const int r = rc / b, c = rc - r * b;
        s += (double)X[e] * (double)Y[q * bb + c * b + r];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) rowsum[warp] = s;
}

// block per system: slots[sys * kSlots + slot] = sum of its rows' partial sums (fixed order)
__global__ void k_sys_sum(const int64_t *__restrict__ off, const double *__restrict__ rowsum,
                          double *__restrict__ slots, int slot) {
    __shared__ double sh[256];
    const int sys = blockIdx.x;
    double s = 0.0;
    for (int64_t i = off[sys] + threadIdx.x; i < off[sys + 1]; i += blockDim.x) s += rowsum[i];
    sh[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) slots[(int64_t)sys * kSlots + slot] = sh[0];
}

// H' = H - mu_sys S_H per row (mu of the row's system)
__global__ void k_hprime_rows(int n, int bb, const int64_t *__restrict__ hp, const int *__restrict__ atom_sys,
                              const double *__restrict__ mu, const double *__restrict__ H,
                              const double *__restrict__ S, const int64_t *__restrict__ pos_s,
                              double *__restrict__ Hp, double *__restrict__ Sh) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double m = mu[atom_sys ? atom_sys[warp] : 0];
    for (int64_t e = hp[warp] * bb + lane; e < hp[warp + 1] * bb; e += 32) {
        const int64_t p = e / bb;
        const int rc = (int)(e - p * bb);
        const int64_t q = pos_s[p];
        const double sv = q >= 0 ? S[q * bb + rc] : 0.0;
        Sh[e] = sv;
        Hp[e] = H[e] - m * sv;
    }
}

struct BatchDev {
    double *slots, *gg_prev, *beta, *alpha, *omega, *dom;
    int *status, *frozen, *reset, *iters, *natoms, *step;
};

// After the gradient: Omega and the Polak-Ribiere beta of every system.
__global__ void k_batch_beta(int nsys, double spin, int cg_reset, BatchDev d) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const double *sl = d.slots + (int64_t)s * kSlots;
    d.omega[s] = spin * (3.0 * sl[0] - 2.0 * sl[1]);
    const double gg = sl[10], ggp = sl[11];
    double b = 0.0;
    const int it = d.step[0];
    if (!d.reset[s] && it % cg_reset != 0 && d.gg_prev[s] > 0.0) b = fmax(0.0, (gg - ggp) / d.gg_prev[s]);
    d.reset[s] = 0;
    d.beta[s] = b;
    d.gg_prev[s] = gg;
}

// After the line products: alpha of every system (0 for frozen systems).
__global__ void k_batch_alpha(int nsys, double spin, double tol, BatchDev d) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s == 0) d.step[0] += 1;
    if (s >= nsys) return;
    const double *sl = d.slots + (int64_t)s * kSlots;
    d.alpha[s] = 0.0;
    if (d.frozen[s]) return;
    const double c1 = sl[4];
    const double c2 = spin * (3.0 * sl[5] - 2.0 * (2.0 * sl[6] + sl[7]));
    const double c3 = -2.0 * spin * sl[8];
    if (!(c1 < 0.0)) {  // not a descent direction: restart from -G next step
        d.reset[s] = 1;
        if (sl[10] == 0.0) d.frozen[s] = 1;  // exact stationary point
        return;
    }
    double a = 0.0;
    const double disc = c2 * c2 - 3.0 * c1 * c3;
    bool ok = false;
    if (disc >= 0.0) {
        const double den = c2 + sqrt(disc);
        if (den > 0.0) {
            a = -c1 / den;
            ok = true;
        }
    }
    if (!ok && c2 > 0.0) {
        a = -c1 / (2.0 * c2);
        ok = true;
    }
    if (!ok || !isfinite(a)) {
        d.status[s] = LSQ_ERR_UNSTABLE;
        d.frozen[s] = 1;
        return;
    }
    d.alpha[s] = a;
    const double dom = fabs(c1 * a + c2 * a * a + c3 * a * a * a) / kHartreeEv / max(d.natoms[s], 1);
    d.dom[s] = dom;
    d.iters[s] += 1;
    if (tol > 0.0 && dom < tol) {
        d.frozen[s] = 1;
        d.status[s] = LSQ_OK;
    }
}

// warp per row: D = -P + beta_sys D (P = G, or X G X in a metric)
__global__ void k_batch_dir(int n, int bb, const int64_t *__restrict__ rp, const int *__restrict__ atom_sys,
                            const double *__restrict__ beta, const double *__restrict__ G, double *__restrict__ D) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double b = beta[atom_sys ? atom_sys[warp] : 0];
    for (int64_t e = rp[warp] * bb + lane; e < rp[warp + 1] * bb; e += 32) D[e] = b == 0.0 ? -G[e] : -G[e] + b * D[e];
}

// warp per row: L += alpha_sys D ; Gp = G (with a metric the caller passes P and P_prev)
__global__ void k_batch_update(int n, int bb, const int64_t *__restrict__ rp, const int *__restrict__ atom_sys,
                               const double *__restrict__ alpha, const double *__restrict__ D,
                               double *__restrict__ L, const double *__restrict__ G, double *__restrict__ Gp) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double a = alpha[atom_sys ? atom_sys[warp] : 0];
    for (int64_t e = rp[warp] * bb + lane; e < rp[warp + 1] * bb; e += 32) {
        L[e] = L[e] + a * D[e];
        Gp[e] = G[e];
    }
}

// y += alpha_sys x on the rows of a pattern (alpha of the row's system): Q += a QD after the step.
template <typename T>
__global__ void k_batch_axpy_rows(int n, int bb, const int64_t *__restrict__ rp, const int *__restrict__ atom_sys,
                                  const double *__restrict__ alpha, const T *__restrict__ x, T *__restrict__ y) {
    const int warp = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= n) return;
    const double a = alpha[atom_sys ? atom_sys[warp] : 0];
    if (a == 0.0) return;
    const T at = (T)a;
    for (int64_t e = rp[warp] * bb + lane; e < rp[warp + 1] * bb; e += 32) y[e] = fma(at, x[e], y[e]);
}


static int grid_for(int64_t m) {
    int64_t g = (m + 255) / 256;
    return (int)std::max<int64_t>(1, std::min<int64_t>(g, 8192));
}



}  // namespace lsq

using namespace lsq;

struct lsq_lnv_s {
    lsq_geom g = nullptr;
    int b = 4;
    // product precision of the float32 path: LSQ_F32 (FMA kernels), or kMixedAuto when the
    // caller asked for LSQ_TF32X3 (per product the faster of those and the tensor-core kernel)
    int mm32 = LSQ_F32;
    int rS = -1, rH = -1, rL = -1, r1 = -1, r2 = -1, r3 = -1;
    // float64 working set
    DevBuf<double> Hp, Sh, G, Gp, D;
    // product buffers LS, SL, LSL, Q, QT, QD, G1, G2: sized for ws_es bytes per value (4 while
    // only float32 work has run, 8 once float64 work has), grown by ensure_ws at the entry
    // points; the float32 copies Lc, Dc, Hpc, Shc, Sc
    DevBuf<char> LS, SL, LSL, Q, QT, QD, G1, G2, Lc, Dc, Hpc, Shc, Sc;
    size_t ws_es = 0;
    DevBuf<double> om_rows;  // per-row energy terms formed with the gradient (2 x n)
    // metric of the CG (lsq_lnv_set_metric): X ~ S^-1 on range rX, X G on range rXG
    int rX = -1, rXG = -1;
    DevBuf<double> Xm, Pm, Pmp;   // X (float64), P = X G X and the previous P
    DevBuf<char> Xmc, XG, Pc;     // float32 copy of X, X G, P in the working precision
    const int64_t *pos_s_in_h = nullptr;
    // batched minimisation state (allocated by the first batch call)
    int b_nsys = 0;
    DevBuf<double> b_slots, b_rowsum, b_mu, b_gg_prev, b_beta, b_alpha, b_omega, b_dom;
    DevBuf<int> b_status, b_frozen, b_reset, b_iters, b_natoms, b_step;
    DevBuf<int64_t> b_off;
    // second stream of the line search (F = P.D beside QD = H'.P) and its two events
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    ~lsq_lnv_s() {
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (side) cudaStreamDestroy(side);
    }
};

static int64_t nvals(lsq_lnv c, int r) { return c->g->pats[r].nnzb * c->b * c->b; }

// Sizes the product buffers for values of the precision prec (grown, never shrunk; the
// contents do not survive a call).  Called by the entry points before any work is enqueued,
// with the widest precision the call may use, so that no buffer is reallocated inside a call.
static int ensure_ws(lsq_lnv c, int prec) {
    const size_t es = prec == LSQ_F64 ? 8 : 4;
    if (c->ws_es >= es) return LSQ_OK;
    const bool mat = c->b == 4;  // transposed operands materialised (see energy_gradient)
    const auto sz = [&](int r) { return es * (size_t)c->g->pats[r].nnzb * c->b * c->b; };
    c->ws_es = 0;
    LSQ_TRY(c->LS.alloc(sz(c->r1)));
    LSQ_TRY(c->LSL.alloc(sz(c->r3)));
    if (mat) {
        LSQ_TRY(c->SL.alloc(sz(c->r1)));
        LSQ_TRY(c->QT.alloc(sz(c->r3)));
    }
    LSQ_TRY(c->Q.alloc(sz(c->r3)));
    LSQ_TRY(c->QD.alloc(sz(c->r3)));
    LSQ_TRY(c->G1.alloc(sz(c->rL)));
    LSQ_TRY(c->G2.alloc(sz(c->rL)));
    c->ws_es = es;
    return LSQ_OK;
}

// The product buffers hold values of the precision prec (a guard of the internal functions).
static int need_ws(lsq_lnv c, int prec) {
    if (c->ws_es < (prec == LSQ_F64 ? 8u : 4u))
        return set_error(LSQ_ERR_INVALID_ARG, "internal: LNV workspace not sized for this precision");
    return LSQ_OK;
}

// Widest precision a minimisation with these options uses.
static int widest(const lsq_lnv_opts &o) {
    return (o.precision == LSQ_F64 || o.refine_iter > 0 || o.final_eval) ? LSQ_F64 : LSQ_F32;
}

// Precision handed to the products: the float32 path runs them as c->mm32.
static int mmp(lsq_lnv c, int prec) { return prec == LSQ_F32 ? c->mm32 : prec; }

// Accepts LSQ_F64, LSQ_F32 and LSQ_TF32X3; the latter runs the float32 path (float32 storage,
// float64 traces and CG) with the products chosen per product between the FP32 FMA schedules
// and the split-TF32 tensor-core kernel.  *prec becomes LSQ_F64 or LSQ_F32.
static int take_precision(lsq_lnv c, int *prec) {
    if (*prec != LSQ_F64 && *prec != LSQ_F32 && *prec != LSQ_TF32X3)
        return set_error(LSQ_ERR_INVALID_ARG, "precision must be LSQ_F64, LSQ_F32 or LSQ_TF32X3");
    c->mm32 = *prec == LSQ_TF32X3 ? kMixedAuto : LSQ_F32;
    if (*prec == LSQ_TF32X3) *prec = LSQ_F32;
    return LSQ_OK;
}

// Steps between fresh products Q = H'LS in the single-system CG (Q is updated along the line
// search in between).
constexpr int kQFresh = 10;

// Contexts of one grouped batch call.
constexpr int kMaxGroupContexts = 16;

extern "C" int lsq_lnv_default_opts(lsq_lnv_opts *o) {
    clear_error();
    if (!o) return set_error(LSQ_ERR_INVALID_ARG, "opts is null");
    o->max_iter = 100;
    o->tol_ha_per_atom = 0.0;
    o->cg_reset = 40;
    o->precision = LSQ_F64;
    o->refine_iter = 2;
    o->spin = 2.0;
    o->final_eval = 1;
    o->verbose = 0;
    o->graph = 1;
    return LSQ_OK;
}

extern "C" int lsq_lnv_required_ranges(double R_S, double R_H, double R_L, double *out) {
    clear_error();
    if (!out) return set_error(LSQ_ERR_INVALID_ARG, "out is null");
    out[0] = R_S;
    out[1] = R_H;
    out[2] = R_L;
    out[3] = R_L + R_S;
    out[4] = R_L + R_S + R_L;
    out[5] = R_H + R_L + R_S;
    return LSQ_OK;
}

extern "C" int lsq_lnv_create(lsq_geom g, int b, double R_S, double R_H, double R_L, lsq_lnv *out) {
    clear_error();
    if (!g || !out) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    *out = nullptr;
    if (b < 1 || b > 16) return set_error(LSQ_ERR_INVALID_ARG, "block size must be in [1, 16]");
    if (!(R_S <= R_H)) return set_error(LSQ_ERR_INVALID_ARG, "R_S must not exceed R_H");
    double need[6];
    lsq_lnv_required_ranges(R_S, R_H, R_L, need);
    int id[6];
    for (int k = 0; k < 6; ++k) {
        id[k] = find_range(g, need[k]);
        if (id[k] < 0)
            return set_error(LSQ_ERR_INVALID_ARG,
                             "geometry lacks range " + std::to_string(need[k]) +
                                 " (see lsq_lnv_required_ranges)");
    }
    lsq_lnv c = new lsq_lnv_s();
    c->g = g;
    c->b = b;
    c->rS = id[0];
    c->rH = id[1];
    c->rL = id[2];
    c->r1 = id[3];
    c->r2 = id[4];
    c->r3 = id[5];
    auto fail = [&](int rc) {
        delete c;
        return rc;
    };
    int rc;
    if ((rc = c->Hp.alloc(nvals(c, c->rH))) || (rc = c->Sh.alloc(nvals(c, c->rH))) ||
        (rc = c->G.alloc(nvals(c, c->rL))) || (rc = c->Gp.alloc(nvals(c, c->rL))) ||
        (rc = c->D.alloc(nvals(c, c->rL))) ||
        (rc = c->Lc.alloc(4 * nvals(c, c->rL))) || (rc = c->Dc.alloc(4 * nvals(c, c->rL))) ||
        (rc = c->Hpc.alloc(4 * nvals(c, c->rH))) || (rc = c->Shc.alloc(4 * nvals(c, c->rH))) ||
        (rc = c->Sc.alloc(4 * nvals(c, c->rS))))
        return fail(rc);
    if ((rc = get_posmap(g, c->rH, c->rS, 0, &c->pos_s_in_h, 0))) return fail(rc);
    if ((rc = ensure_tmap(g, c->rL, 0))) return fail(rc);
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess)
        return fail(set_error(LSQ_ERR_CUDA, "stream or event creation failed"));
    if (cudaDeviceSynchronize() != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, "sync failed"));
    *out = c;
    return LSQ_OK;
}

extern "C" int lsq_lnv_destroy(lsq_lnv c) {
    clear_error();
    if (!c) return LSQ_OK;
    cudaDeviceSynchronize();
    delete c;
    return LSQ_OK;
}

extern "C" int lsq_lnv_init_L(lsq_lnv c, const double *S, double *L, void *stream) {
    clear_error();
    if (!c || !S || !L) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    lsq_geom g = c->g;
    LSQ_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(double) * nvals(c, c->rL), s));
    DevBuf<int> bad;
    LSQ_TRY(bad.alloc(1));
    LSQ_CUDA_TRY(cudaMemsetAsync(bad.p, 0, sizeof(int), s));
    if (g->n > 0) {
        note_launch();
        k_onsite_inverse<<<(g->n + 127) / 128, 128, 0, s>>>(
            g->n, c->b, g->pats[c->rS].row_ptr.p, g->pats[c->rS].col.p, S,
            g->pats[c->rL].row_ptr.p, g->pats[c->rL].col.p, L, bad.p);
    }
    LSQ_CHECK_LAUNCH();
    int hbad = 0;
    LSQ_CUDA_TRY(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    if (hbad) return set_error(LSQ_ERR_INVALID_ARG, "an on-site block of S is singular or missing");
    return LSQ_OK;
}

namespace {

// Prepares H', S_H (float64) and the reduced-precision copies for 'prec'.
int prepare_hs(lsq_lnv c, const double *S, const double *H, double mu, int prec, cudaStream_t s) {
    int64_t nh = nvals(c, c->rH);
    note_launch();
    k_hprime<<<grid_for(nh), 256, 0, s>>>(c->g->pats[c->rH].nnzb, c->b * c->b, H, S, c->pos_s_in_h,
                                          mu, c->Hp.p, c->Sh.p);
    if (prec == LSQ_F32) {
        note_launch();
        k_to_f32<<<grid_for(nh), 256, 0, s>>>(nh, c->Hp.p, (float *)c->Hpc.p);
        note_launch();
        k_to_f32<<<grid_for(nh), 256, 0, s>>>(nh, c->Sh.p, (float *)c->Shc.p);
        int64_t ns = nvals(c, c->rS);
        note_launch();
        k_to_f32<<<grid_for(ns), 256, 0, s>>>(ns, S, (float *)c->Sc.p);
    }
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

struct Ops {
    const void *L, *S, *Hp, *Sh;
};

Ops operands(lsq_lnv c, const double *L, const double *S, int prec, cudaStream_t s) {
    Ops o;
    if (prec == LSQ_F32) {
        int64_t nl = nvals(c, c->rL);
        note_launch();
        k_to_f32<<<grid_for(nl), 256, 0, s>>>(nl, L, (float *)c->Lc.p);
        o.L = c->Lc.p;
        o.S = c->Sc.p;
        o.Hp = c->Hpc.p;
        o.Sh = c->Shc.p;
    } else {
        o.L = L;
        o.S = S;
        o.Hp = c->Hp.p;
        o.Sh = c->Sh.p;
    }
    return o;
}

// Per-system sums (batched geometries): slot k of every system.
int seg_dot(lsq_lnv c, int prec, int r, const void *X, const void *Y, int slot, cudaStream_t s) {
    lsq_geom g = c->g;
    const int n = g->n, bb = c->b * c->b;
    const int blocks = (int)(((int64_t)n * 32 + 255) / 256);
    note_launch();
    if (prec == LSQ_F64)
        k_rowdot<double><<<blocks, 256, 0, s>>>(n, bb, g->pats[r].row_ptr.p, (const double *)X,
                                                (const double *)Y, c->b_rowsum.p);
    else
        k_rowdot<float><<<blocks, 256, 0, s>>>(n, bb, g->pats[r].row_ptr.p, (const float *)X,
                                               (const float *)Y, c->b_rowsum.p);
    note_launch();
    k_sys_sum<<<c->b_nsys, 256, 0, s>>>(c->b_off.p, c->b_rowsum.p, c->b_slots.p, slot);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

int seg_trace(lsq_lnv c, int prec, int rx, const void *X, int ry, const void *Y, int slot, cudaStream_t s) {
    lsq_geom g = c->g;
    const int64_t *pm = nullptr;
    LSQ_TRY(get_posmap(g, rx, ry, 1, &pm, s));
    const int n = g->n;
    const int blocks = (int)(((int64_t)n * 32 + 255) / 256);
    note_launch();
    if (prec == LSQ_F64)
        k_rowtrace<double><<<blocks, 256, 0, s>>>(n, c->b, g->pats[rx].row_ptr.p, pm, (const double *)X,
                                                  (const double *)Y, c->b_rowsum.p);
    else
        k_rowtrace<float><<<blocks, 256, 0, s>>>(n, c->b, g->pats[rx].row_ptr.p, pm, (const float *)X,
                                                 (const float *)Y, c->b_rowsum.p);
    note_launch();
    k_sys_sum<<<c->b_nsys, 256, 0, s>>>(c->b_off.p, c->b_rowsum.p, c->b_slots.p, slot);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

// Omega, N_e (scalars slots 0..3 hold the four traces) and, if G != null, the gradient.
// seg: per-system sums into the batch slots, nothing fetched (omega, ne ignored).
// reuse_q: c->Q already holds H'LS for this L (updated along the line search), skip its product.
// s_as_h: S (on H's range) takes the place of H' everywhere, so that "Omega" is N_e and G is
// dN_e/dL (the canonical minimiser's electron-number gradient).
int energy_gradient(lsq_lnv c, const double *L, const double *S, double spin, int prec, double *G,
                    double *omega, double *ne, cudaStream_t s, bool seg = false, bool want_ne = false,
                    bool reuse_q = false, bool s_as_h = false) {
    LSQ_TRY(need_ws(c, prec));
    lsq_geom g = c->g;
    const int b = c->b;
    Ops o = operands(c, L, S, prec, s);
    if (s_as_h) o.Hp = o.Sh;
    // scalar slots: 0 = Tr[H' LSL], 1 = Tr[LSLSL H'] (= <LSL, Q>), 2 = Tr[S LSL], 3 = <LSL, SLS>.
    // With the gradient, slots 0 and 1 come from <L, Q> and <L, M> / 3 (see the header) and LSL
    // is formed only for N_e.
    const bool need_lsl = !G || ne || want_ne;
    LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rL, 0, o.L, c->rS, 1, o.S, c->r1, c->LS.p, 1.0, 0.0, nullptr, s));
    if (need_lsl)
        LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 0, c->LS.p, c->rL, 1, o.L, c->r3, c->LSL.p, 1.0, 0.0, nullptr, s, 1));
    // 4 x 4 blocks: transposed operands are materialised so the plan kernel reads rows; the
    // kernel for other block sizes reads transposes through the transpose map
    const bool mat = c->b == 4;
    const void *LSop = mat ? c->SL.p : c->LS.p;  // operand giving LS as op(B)
    const int tLS = mat ? 1 : 0;
    if (mat) LSQ_TRY(transpose_on(g, c->r1, b, prec, c->LS.p, c->SL.p, s));
    if (!reuse_q)
        LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rH, 0, o.Hp, c->r1, tLS, LSop, c->r3, c->Q.p, 1.0, 0.0, nullptr, s));
    auto tr = [&](int rx, const void *X, int ry, const void *Y, int slot) {
        return seg ? seg_trace(c, prec, rx, X, ry, Y, slot, s) : trace_into(g, b, prec, rx, X, ry, Y, slot, s);
    };
    auto dt = [&](int r, const void *X, const void *Y, int slot) {
        return seg ? seg_dot(c, prec, r, X, Y, slot, s) : dot_into(g, b, prec, r, X, Y, slot, s);
    };
    if (!G) {
        LSQ_TRY(tr(c->rH, o.Hp, c->r3, c->LSL.p, 0));
        LSQ_TRY(dt(c->r3, c->LSL.p, c->Q.p, 1));
    }
    if (ne || want_ne) {
        void *SLS = c->QD.p;
        LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rH, 0, o.Sh, c->r1, tLS, LSop, c->r3, SLS, 1.0, 0.0, nullptr, s, 1));
        LSQ_TRY(tr(c->rH, o.Sh, c->r3, c->LSL.p, 2));
        LSQ_TRY(dt(c->r3, c->LSL.p, SLS, 3));
    }
    if (G) {
        // M = G1 + G1^T + G2 (G1 = Q.LS, G2 = Q^T.LS) is symmetric and equals T1 + T2 with
        // T1 = (Q + Q^T).LS and T2 = SL.Q^T, so the upper triangles of T1 and T2 on L's range
        // give all of it: one full product's work instead of G1 in full plus G2's upper half.
        // Q + Q^T goes to QD's storage, free until the line search.  T1 is formed through its
        // transpose SL.(Q + Q^T), lower triangle (j <= i), so that the operand whose rows the
        // kernel walks is SL on L+S's range rather than Q + Q^T on R3: G1 holds T1's upper
        // blocks transposed.
        void *Qs = c->QD.p;
        // With the tensor-core kernel chosen for a product (LSQ_TF32X3), its split operand copy
        // is formed from Q + Q^T directly, and the split of SL is shared by T1 and T2.
        const bool tc1 = mat && mmp(c, prec) == kMixedAuto && mixed_choice(g, c->r1, c->r3, c->rL, 3, 0.0) == 1;
        const bool tc2 = mat && mmp(c, prec) == kMixedAuto && mixed_choice(g, c->r1, c->r3, c->rL, 2, 0.0) == 1;
        if (tc1) {
            LSQ_TRY(tc_block_matmul(g, c->r1, 0, (const float *)c->SL.p, c->r3, 1, (const float *)c->Q.p, c->rL,
                                    (float *)c->G1.p, 1.0, 0.0, 2, false, nullptr, s, true, false));
        } else {
            LSQ_TRY(sym_sum_on(g, c->r3, b, prec, c->Q.p, Qs, s));
            if (mat)
                LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 0, c->SL.p, c->r3, 1, Qs, c->rL, c->G1.p, 1.0, 0.0, nullptr, s, 3));
            else
                LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 1, c->LS.p, c->r3, 1, Qs, c->rL, c->G1.p, 1.0, 0.0, nullptr, s, 3));
        }
        // T2 = SL.Q^T: op(B) = Q^T, read as rows of Q; op(A) = SL (materialised for 4 x 4 blocks)
        if (tc2)
            LSQ_TRY(tc_block_matmul(g, c->r1, 0, (const float *)c->SL.p, c->r3, 1, (const float *)c->Q.p, c->rL,
                                    (float *)c->G2.p, 1.0, 0.0, 1, false, nullptr, s, false, tc1));
        else if (mat)
            LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 0, c->SL.p, c->r3, 1, c->Q.p, c->rL, c->G2.p, 1.0, 0.0, nullptr, s, 2));
        else
            LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 1, c->LS.p, c->r3, 1, c->Q.p, c->rL, c->G2.p, 1.0, 0.0, nullptr, s, 2));
        const int64_t *pq = nullptr, *pqt = nullptr;
        LSQ_TRY(get_posmap(g, c->rL, c->r3, 0, &pq, s));
        LSQ_TRY(get_posmap(g, c->rL, c->r3, 1, &pqt, s));
        LSQ_TRY(ensure_tmap(g, c->rL, s));
        const int n = g->n;
        if (c->om_rows.n < (size_t)2 * std::max(n, 1)) LSQ_TRY(c->om_rows.alloc((size_t)2 * std::max(n, 1)));
        double *row0 = c->om_rows.p, *row1 = c->om_rows.p + std::max(n, 1);
        const int blocks = (int)(((int64_t)n * 32 + 255) / 256);
        auto go = [&](auto kern, auto *l, auto *q, auto *t1, auto *t2) {
            if (n == 0) return;
            note_launch();
            kern<<<blocks, 256, 0, s>>>(n, b, spin, g->pats[c->rL].row_ptr.p, pq, pqt, g->pats[c->rL].tmap.p,
                                        l, q, t1, t2, G, row0, row1);
        };
        if (prec == LSQ_F64) {
            auto *l = (const double *)o.L, *q = (const double *)c->Q.p;
            auto *t1 = (const double *)c->G1.p, *t2 = (const double *)c->G2.p;
            if (b == 4) go(k_grad_omega_rows<double, 4>, l, q, t1, t2);
            else go(k_grad_omega_rows<double, 0>, l, q, t1, t2);
        } else {
            auto *l = (const float *)o.L, *q = (const float *)c->Q.p;
            auto *t1 = (const float *)c->G1.p, *t2 = (const float *)c->G2.p;
            if (b == 4) go(k_grad_omega_rows<float, 4>, l, q, t1, t2);
            else go(k_grad_omega_rows<float, 0>, l, q, t1, t2);
        }
        LSQ_CHECK_LAUNCH();
        if (seg) {
            note_launch();
            k_sys_sum<<<c->b_nsys, 256, 0, s>>>(c->b_off.p, row0, c->b_slots.p, 0);
            note_launch();
            k_sys_sum<<<c->b_nsys, 256, 0, s>>>(c->b_off.p, row1, c->b_slots.p, 1);
            LSQ_CHECK_LAUNCH();
        } else {
            LSQ_TRY(sum_into(g, row0, n, 0, s));
            LSQ_TRY(sum_into(g, row1, n, 1, s));
        }
    }
    if (!seg && (omega || ne)) {
        double t[4];
        LSQ_TRY(fetch_scalars(g, ne ? 4 : 2, t, s));
        if (omega) *omega = spin * (3.0 * t[0] - 2.0 * t[1]);
        if (ne) *ne = spin * (3.0 * t[2] - 2.0 * t[3]);
    }
    return LSQ_OK;
}

// c1 = <G, D> (float64), c2, c3 from the products listed at the top of the file.
int line_coeffs(lsq_lnv c, const double *L, const double *S, double spin, int prec, double *c123,
                cudaStream_t s, bool seg = false) {
    LSQ_TRY(need_ws(c, prec));
    lsq_geom g = c->g;
    const int b = c->b;
    Ops o = operands(c, L, S, prec, s);
    const void *D = c->D.p;
    if (prec == LSQ_F32) {
        int64_t nl = nvals(c, c->rL);
        note_launch();
        k_to_f32<<<grid_for(nl), 256, 0, s>>>(nl, c->D.p, (float *)c->Dc.p);
        D = c->Dc.p;
    }
    void *P = c->LS.p, *PT = c->SL.p, *F = c->LSL.p, *QDT = c->QT.p, *Z = c->G2.p;
    const bool mat = c->b == 4;  // see energy_gradient
    LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rL, 0, D, c->rS, 1, o.S, c->r1, P, 1.0, 0.0, nullptr, s));
    // F = P.D and QD = H'.P both need only P: outside stream capture, when both run on the FMA
    // kernels, F runs on the context's second stream beside QD so that the two share the SMs
    // (measured: the float32 step 22.15 -> 21.78 ms at 4096 atoms).  With F on the tensor
    // cores the overlap was slower (17.7 -> 18.1 ms), and two tensor-core products would share
    // g's split buffers, so then the products run in turn.  The transpose maps both may build
    // are built here first.
    const bool fma_both = mmp(c, prec) != kMixedAuto || (mixed_choice(g, c->rH, c->r1, c->r3, 0, 0.0) == 0 &&
                                                         mixed_choice(g, c->r1, c->rL, c->r3, 1, 0.0) == 0);
    const bool fork = !seg && c->side && fma_both;
    cudaStream_t sf = s;
    if (fork) {
        LSQ_TRY(ensure_tmap(g, c->r1, s));
        LSQ_TRY(ensure_tmap(g, c->rL, s));
        LSQ_TRY(ensure_tmap(g, c->r3, s));
        LSQ_CUDA_TRY(cudaEventRecord(c->ev_fork, s));
        LSQ_CUDA_TRY(cudaStreamWaitEvent(c->side, c->ev_fork, 0));
        sf = c->side;
    }
    LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 0, P, c->rL, 1, D, c->r3, F, 1.0, 0.0, nullptr, sf, 1));
    if (mat) {
        LSQ_TRY(transpose_on(g, c->r1, b, prec, P, PT, s));
        LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rH, 0, o.Hp, c->r1, 1, PT, c->r3, c->QD.p, 1.0, 0.0, nullptr, s));
    } else {
        LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rH, 0, o.Hp, c->r1, 0, P, c->r3, c->QD.p, 1.0, 0.0, nullptr, s));
    }
    if (fork) {
        LSQ_CUDA_TRY(cudaEventRecord(c->ev_join, sf));
        LSQ_CUDA_TRY(cudaStreamWaitEvent(s, c->ev_join, 0));
    }
    // Z = QD^T.P is symmetric, so it is formed as P^T.QD: the operand whose rows the kernel
    // walks (and stages in shared memory) is then P^T on L+S's range, not QD^T on R3
    if (mat && mmp(c, prec) == kMixedAuto && mixed_choice(g, c->r1, c->r3, c->rL, 1, 0.0) == 1) {
        // on the tensor cores: the split copy of QD^T is read through the transpose map, so QD^T
        // is not materialised
        LSQ_TRY(tc_block_matmul(g, c->r1, 0, (const float *)PT, c->r3, 0, (const float *)c->QD.p, c->rL,
                                (float *)Z, 1.0, 0.0, 1, true, nullptr, s));
    } else if (mat) {
        LSQ_TRY(transpose_on(g, c->r3, b, prec, c->QD.p, QDT, s));
        LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 0, PT, c->r3, 1, QDT, c->rL, Z, 1.0, 0.0, nullptr, s, 1));
    } else {
        LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->r1, 1, P, c->r3, 0, c->QD.p, c->rL, Z, 1.0, 0.0, nullptr, s, 1));
    }
    if (seg) {
        LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, c->G.p, c->D.p, 4, s));
        LSQ_TRY(seg_trace(c, prec, c->rH, o.Hp, c->r3, F, 5, s));
        LSQ_TRY(seg_dot(c, prec, c->r3, F, c->Q.p, 6, s));
        LSQ_TRY(seg_dot(c, prec, c->rL, o.L, Z, 7, s));
        LSQ_TRY(seg_dot(c, prec, c->rL, D, Z, 8, s));
        return LSQ_OK;
    }
    LSQ_TRY(dot_into(g, b, LSQ_F64, c->rL, c->G.p, c->D.p, 4, s));
    LSQ_TRY(trace_into(g, b, prec, c->rH, o.Hp, c->r3, F, 5, s));
    LSQ_TRY(dot_into(g, b, prec, c->r3, F, c->Q.p, 6, s));
    LSQ_TRY(dot_into(g, b, prec, c->rL, o.L, Z, 7, s));
    LSQ_TRY(dot_into(g, b, prec, c->rL, D, Z, 8, s));
    double t[9];
    LSQ_TRY(fetch_scalars(g, 9, t, s));
    c123[0] = t[4];
    c123[1] = spin * (3.0 * t[5] - 2.0 * (2.0 * t[6] + t[7]));
    c123[2] = -2.0 * spin * t[8];
    return LSQ_OK;
}

// Step a > 0 along a descent direction (c1 < 0): the local minimum of the cubic,
// a = -c1 / (c2 + sqrt(c2^2 - 3 c1 c3)); if the cubic has none but c2 > 0, the minimum of
// its quadratic part, -c1 / (2 c2); otherwise no step (false).
bool line_minimum(double c1, double c2, double c3, double *a) {
    double disc = c2 * c2 - 3.0 * c1 * c3;
    if (disc >= 0.0) {
        double den = c2 + std::sqrt(disc);
        if (den > 0.0) {
            *a = -c1 / den;
            return std::isfinite(*a);
        }
    }
    if (c2 > 0.0) {
        *a = -c1 / (2.0 * c2);
        return std::isfinite(*a);
    }
    return false;
}

}  // namespace

extern "C" int lsq_lnv_energy_gradient(lsq_lnv c, const double *L, const double *S, const double *H,
                                       double mu, double spin, int prec, double *omega, double *ne,
                                       double *G, void *stream) {
    clear_error();
    if (!c || !L || !S || !H) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    LSQ_TRY(take_precision(c, &prec));
    LSQ_TRY(ensure_ws(c, prec));
    cudaStream_t s = (cudaStream_t)stream;
    LSQ_TRY(prepare_hs(c, S, H, mu, prec, s));
    double om = 0, n_e = 0;
    LSQ_TRY(energy_gradient(c, L, S, spin, prec, G, &om, &n_e, s));
    if (omega) *omega = om;
    if (ne) *ne = n_e;
    return LSQ_OK;
}

extern "C" int lsq_lnv_set_metric(lsq_lnv c, int range_x, const double *X, int range_xg, void *stream) {
    clear_error();
    if (!c) return set_error(LSQ_ERR_INVALID_ARG, "null context");
    lsq_geom g = c->g;
    cudaStream_t s = (cudaStream_t)stream;
    if (!X) {
        c->rX = c->rXG = -1;
        c->Xm.release();
        c->Pm.release();
        c->Pmp.release();
        c->Xmc.release();
        c->XG.release();
        c->Pc.release();
        return LSQ_OK;
    }
    LSQ_TRY(geom_check(g, range_x));
    LSQ_TRY(geom_check(g, range_xg));
    if (g->pats[range_xg].R < g->pats[range_x].R + g->pats[c->rL].R - 1e-9)
        return set_error(LSQ_ERR_INVALID_ARG, "range_xg must cover the natural range R_X + R_L of X G");
    const int bb = c->b * c->b;
    const int64_t nx = g->pats[range_x].nnzb * bb, nxg = g->pats[range_xg].nnzb * bb, nl = nvals(c, c->rL);
    LSQ_TRY(c->Xm.alloc((size_t)std::max<int64_t>(nx, 1)));
    LSQ_TRY(c->Pm.alloc((size_t)std::max<int64_t>(nl, 1)));
    LSQ_TRY(c->Pmp.alloc((size_t)std::max<int64_t>(nl, 1)));
    LSQ_TRY(c->Xmc.alloc(4 * (size_t)std::max<int64_t>(nx, 1)));
    LSQ_TRY(c->XG.alloc(8 * (size_t)std::max<int64_t>(nxg, 1)));
    LSQ_TRY(c->Pc.alloc(8 * (size_t)std::max<int64_t>(nl, 1)));
    LSQ_CUDA_TRY(cudaMemcpyAsync(c->Xm.p, X, sizeof(double) * nx, cudaMemcpyDeviceToDevice, s));
    if (nx > 0) {
        note_launch();
        k_to_f32<<<grid_for(nx), 256, 0, s>>>(nx, c->Xm.p, (float *)c->Xmc.p);
        LSQ_CHECK_LAUNCH();
    }
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    c->rX = range_x;
    c->rXG = range_xg;
    return LSQ_OK;
}

namespace {

// Gershgorin discs of the scalar rows of XH (pattern rp/col): lo = d - r, hi = d + r with d the
// diagonal element and r the sum of the other absolute values of the row.
__global__ void k_gersh_rows(int n, int b, const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                             const double *__restrict__ XH, double *__restrict__ lo, double *__restrict__ hi) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)n * b) return;
    const int i = (int)(t / b), r = (int)(t - (int64_t)i * b);
    const int bb = b * b;
    double a = 0.0, d = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; ++p) {
        for (int c = 0; c < b; ++c) a += fabs(XH[p * bb + r * b + c]);
        if (col[p] == i) d = XH[p * bb + r * b + r];
    }
    const double rad = a - fabs(d);
    lo[t] = d - rad;
    hi[t] = d + rad;
}

// out[0] = min of lo, out[1] = max of hi (one block).
__global__ void k_minmax(int64_t m, const double *__restrict__ lo, const double *__restrict__ hi,
                         double *__restrict__ out) {
    __shared__ double a[1024], z[1024];
    double mn = 1e300, mx = -1e300;
    for (int64_t k = threadIdx.x; k < m; k += blockDim.x) {
        mn = fmin(mn, lo[k]);
        mx = fmax(mx, hi[k]);
    }
    a[threadIdx.x] = mn;
    z[threadIdx.x] = mx;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            a[threadIdx.x] = fmin(a[threadIdx.x], a[threadIdx.x + w]);
            z[threadIdx.x] = fmax(z[threadIdx.x], z[threadIdx.x + w]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = a[0];
        out[1] = z[0];
    }
}

// K_0 = (lam / 2) (mu X - X H X) + X / 2 on L's range (pos: blocks of L's pattern in X's).
__global__ void k_pm_start(int64_t nnzb, int bb, const int64_t *__restrict__ pos, const double *__restrict__ X,
                           const double *__restrict__ XHX, double half_lam, double mu, double *__restrict__ K) {
    const int64_t m = nnzb * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / bb;
        const int rc = (int)(e - p * bb);
        const double xl = pos[p] >= 0 ? X[pos[p] * bb + rc] : 0.0;
        K[e] = half_lam * (mu * xl - XHX[e]) + 0.5 * xl;
    }
}

// K = 3 B - (C + C^T) (the symmetric part of 3 B - 2 C; C = (K S)(K S K) is not symmetric once
// K S K is truncated) with per-block partial sums of the change squared; tm: L's transpose map.
template <typename T>
__global__ void k_pm_update(int64_t nnzb, int b, const int64_t *__restrict__ tm, const T *__restrict__ B,
                            const T *__restrict__ C, double *__restrict__ K, double *__restrict__ partial) {
    __shared__ double sh[256];
    double acc = 0.0;
    const int bb = b * b;
    const int64_t m = nnzb * bb;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e / bb;
        const int rc = (int)(e - p * bb), r = rc / b, c = rc - r * b;
        const double kn = 3.0 * (double)B[e] - ((double)C[e] + (double)C[tm[p] * bb + c * b + r]);
        const double d = kn - K[e];
        K[e] = kn;
        acc = fma(d, d, acc);
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = sh[0];
}

__global__ void k_sum_partial(int m, const double *__restrict__ partial, double *__restrict__ out) {
    __shared__ double sh[1024];
    double acc = 0.0;
    for (int k = threadIdx.x; k < m; k += blockDim.x) acc += partial[k];
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sqrt(sh[0]);
}

}  // namespace

extern "C" int lsq_lnv_init_purify(lsq_lnv c, const double *S, const double *H, double mu, int range_x,
                                   const double *X, int range_xh, int n_iter, int precision, double *L,
                                   double *dk_host, void *stream) {
    clear_error();
    if (!c || !S || !H || !X || !L) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    lsq_geom g = c->g;
    LSQ_TRY(geom_check(g, range_x));
    LSQ_TRY(geom_check(g, range_xh));
    LSQ_TRY(take_precision(c, &precision));
    LSQ_TRY(ensure_ws(c, LSQ_F64));  // X H and X H X are formed in float64 in any precision
    if (n_iter < 0) return set_error(LSQ_ERR_INVALID_ARG, "n_iter must be >= 0");
    if (g->pats[range_xh].R < g->pats[range_x].R + g->pats[c->rH].R - 1e-9)
        return set_error(LSQ_ERR_INVALID_ARG, "range_xh must cover the natural range R_X + R_H of X H");
    if (g->pats[range_xh].nnzb > g->pats[c->r3].nnzb)
        return set_error(LSQ_ERR_UNSUPPORTED, "range_xh is larger than the workspace's widest range");
    cudaStream_t s = (cudaStream_t)stream;
    const int b = c->b, bb = b * b;
    const int n = g->n;
    const int64_t nl = nvals(c, c->rL);
    if (n == 0) return LSQ_OK;
    // X H (the workspace's Q storage), its Gershgorin bounds, X H X on L's range (G1 storage)
    double *XH = reinterpret_cast<double *>(c->Q.p), *XHX = reinterpret_cast<double *>(c->G1.p);
    LSQ_TRY(block_matmul(g, b, LSQ_F64, range_x, 0, X, c->rH, 1, H, range_xh, XH, 1.0, 0.0, nullptr, s));
    DevBuf<double> lohi, red;
    LSQ_TRY(lohi.alloc((size_t)2 * n * b));
    LSQ_TRY(red.alloc(1024 + 4));
    note_launch();
    k_gersh_rows<<<(int)(((int64_t)n * b + 255) / 256), 256, 0, s>>>(n, b, g->pats[range_xh].row_ptr.p,
                                                                      g->pats[range_xh].col.p, XH, lohi.p,
                                                                      lohi.p + (int64_t)n * b);
    note_launch();
    k_minmax<<<1, 1024, 0, s>>>((int64_t)n * b, lohi.p, lohi.p + (int64_t)n * b, red.p + 1024);
    LSQ_CHECK_LAUNCH();
    double eb[2];
    LSQ_CUDA_TRY(cudaMemcpyAsync(eb, red.p + 1024, sizeof(eb), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    if (!(eb[1] > mu && mu > eb[0]))
        return set_error(LSQ_ERR_INVALID_ARG, "mu lies outside the spectral bounds of X H");
    const double lam = std::min(1.0 / (eb[1] - mu), 1.0 / (mu - eb[0]));
    LSQ_TRY(block_matmul(g, b, LSQ_F64, range_xh, 0, XH, range_x, 1, X, c->rL, XHX, 1.0, 0.0, nullptr, s, 1));
    LSQ_TRY(sym_diag_on(g, c->rL, b, LSQ_F64, XHX, s));
    const int64_t *pos = nullptr;
    LSQ_TRY(get_posmap(g, c->rL, range_x, 0, &pos, s));
    note_launch();
    k_pm_start<<<grid_for(nl), 256, 0, s>>>(g->pats[c->rL].nnzb, bb, pos, X, XHX, 0.5 * lam, mu, L);
    LSQ_CHECK_LAUNCH();
    // McWeeny steps: K S at its natural range (LS storage), (K S) K and (K S)(K S K) on L's range
    const void *Sop = S, *Kop = L;
    if (precision == LSQ_F32) {
        const int64_t ns = nvals(c, c->rS);
        note_launch();
        k_to_f32<<<grid_for(ns), 256, 0, s>>>(ns, S, (float *)c->Sc.p);
        LSQ_CHECK_LAUNCH();
        Sop = c->Sc.p;
        Kop = c->Lc.p;
    }
    void *KS = c->LS.p, *Bm = c->G1.p, *Cm = c->G2.p;
    for (int it = 0; it < n_iter; ++it) {
        if (precision == LSQ_F32) {
            note_launch();
            k_to_f32<<<grid_for(nl), 256, 0, s>>>(nl, L, (float *)c->Lc.p);
            LSQ_CHECK_LAUNCH();
        }
        LSQ_TRY(block_matmul(g, b, mmp(c, precision), c->rL, 0, Kop, c->rS, 1, Sop, c->r1, KS, 1.0, 0.0, nullptr, s));
        LSQ_TRY(block_matmul(g, b, mmp(c, precision), c->r1, 0, KS, c->rL, 1, Kop, c->rL, Bm, 1.0, 0.0, nullptr, s, 1));
        LSQ_TRY(sym_diag_on(g, c->rL, b, precision, Bm, s));
        // (K S)(K S K) on every block (truncated K S K makes it unsymmetric); the second factor
        // read as rows of its transpose, which it equals
        LSQ_TRY(block_matmul(g, b, mmp(c, precision), c->r1, 0, KS, c->rL, 1, Bm, c->rL, Cm, 1.0, 0.0, nullptr, s));
        const int64_t *tmL = g->pats[c->rL].tmap.p;
        note_launch();
        if (precision == LSQ_F64)
            k_pm_update<double><<<1024, 256, 0, s>>>(g->pats[c->rL].nnzb, b, tmL, (const double *)Bm,
                                                     (const double *)Cm, L, red.p);
        else
            k_pm_update<float><<<1024, 256, 0, s>>>(g->pats[c->rL].nnzb, b, tmL, (const float *)Bm,
                                                    (const float *)Cm, L, red.p);
        note_launch();
        k_sum_partial<<<1, 1024, 0, s>>>(1024, red.p, red.p + 1026);
        LSQ_CHECK_LAUNCH();
        if (dk_host) {
            LSQ_CUDA_TRY(cudaMemcpyAsync(dk_host + it, red.p + 1026, sizeof(double), cudaMemcpyDeviceToHost, s));
        }
    }
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    return LSQ_OK;
}

namespace {

// P = (X G X) on L's range, symmetric to the last bit, in float64 (into c->Pm): the gradient
// in the metric X.  G and X are symmetric, so both products read their second factor as rows.
int metric_apply(lsq_lnv c, int prec, const double *G, cudaStream_t s) {
    lsq_geom g = c->g;
    const int b = c->b;
    const int64_t nl = nvals(c, c->rL);
    const void *Gop = G, *Xop = c->Xm.p;
    if (prec == LSQ_F32) {
        note_launch();
        k_to_f32<<<grid_for(nl), 256, 0, s>>>(nl, G, (float *)c->Dc.p);  // D's float32 copy is free here
        LSQ_CHECK_LAUNCH();
        Gop = c->Dc.p;
        Xop = c->Xmc.p;
    }
    LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rX, 0, Xop, c->rL, 1, Gop, c->rXG, c->XG.p, 1.0, 0.0, nullptr, s));
    LSQ_TRY(block_matmul(g, b, mmp(c, prec), c->rXG, 0, c->XG.p, c->rX, 1, Xop, c->rL, c->Pc.p, 1.0, 0.0, nullptr, s, 1));
    LSQ_TRY(sym_diag_on(g, c->rL, b, prec, c->Pc.p, s));
    if (prec == LSQ_F64) {
        LSQ_CUDA_TRY(cudaMemcpyAsync(c->Pm.p, c->Pc.p, sizeof(double) * nl, cudaMemcpyDeviceToDevice, s));
    } else {
        note_launch();
        k_f32_to_f64<<<grid_for(nl), 256, 0, s>>>(nl, (const float *)c->Pc.p, c->Pm.p);
        LSQ_CHECK_LAUNCH();
    }
    return LSQ_OK;
}

}  // namespace

extern "C" int lsq_lnv_minimise(lsq_lnv c, double *L, const double *S, const double *H, double mu,
                                const lsq_lnv_opts *opts, lsq_lnv_report *rep, void *stream) {
    clear_error();
    if (!c || !L || !S || !H) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    lsq_lnv_opts o;
    lsq_lnv_default_opts(&o);
    if (opts) o = *opts;
    LSQ_TRY(take_precision(c, &o.precision));
    if (o.max_iter < 0 || o.cg_reset < 1 || o.refine_iter < 0)
        return set_error(LSQ_ERR_INVALID_ARG, "bad iteration options");
    LSQ_TRY(ensure_ws(c, widest(o)));
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const int n = c->g->n;
    const int64_t nl = nvals(c, c->rL);
    LSQ_TRY(prepare_hs(c, S, H, mu, LSQ_F64, s));
    if (o.precision == LSQ_F32) LSQ_TRY(prepare_hs(c, S, H, mu, LSQ_F32, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->Gp.p, 0, sizeof(double) * nl, s));
    if (c->rX >= 0) LSQ_CUDA_TRY(cudaMemsetAsync(c->Pmp.p, 0, sizeof(double) * nl, s));
    // Phase 0: the requested precision for max_iter steps (or until converged);
    // phase 1 (mixed path only): refine_iter float64 steps from a fresh direction.
    int status = (o.tol_ha_per_atom > 0.0) ? LSQ_ERR_NOT_CONVERGED : LSQ_OK;
    int iters = 0, iters64 = 0;
    double last_d = 0.0;
    const int nphase = o.precision == LSQ_F32 ? 2 : 1;
    double om_pred = 0.0, ne_last = std::nan("");
    bool converged0 = false;  // the first phase reached tol
    for (int phase = 0; phase < nphase && status != LSQ_ERR_UNSTABLE; ++phase) {
        const int prec = phase == 0 ? o.precision : LSQ_F64;
        const int budget = phase == 0 ? o.max_iter : o.refine_iter;
        double gg_prev = 0.0;
        bool converged = false;
        for (int it = 0; it < budget; ++it) {
            // Q = H'LS is linear in L: after L += a D it is Q + a H'DS, and H'DS is the line
            // search's QD.  It is updated that way between fresh products every kQFresh steps
            // (and at every CG restart and phase start), which saves one R3 product per step.
            const bool reuse_q = it % std::min(o.cg_reset, kQFresh) != 0;
            LSQ_TRY(energy_gradient(c, L, S, o.spin, prec, c->G.p, nullptr, nullptr, s, false, false, reuse_q));
            // search directions from P = X G X in the metric X (lsq_lnv_set_metric), else from G;
            // Polak-Ribiere with beta = <G, P - P_prev> / <G_prev, P_prev>
            const bool metric = c->rX >= 0;
            if (metric) LSQ_TRY(metric_apply(c, prec, c->G.p, s));
            const double *Pdir = metric ? c->Pm.p : c->G.p;
            LSQ_TRY(dot_into(c->g, c->b, LSQ_F64, c->rL, c->G.p, Pdir, 10, s));
            LSQ_TRY(dot_into(c->g, c->b, LSQ_F64, c->rL, c->G.p, metric ? c->Pmp.p : c->Gp.p, 11, s));
            double t[12];
            LSQ_TRY(fetch_scalars(c->g, 12, t, s));
            const double om = o.spin * (3.0 * t[0] - 2.0 * t[1]);
            const double gg = t[10], ggp = t[11];
            if (gg == 0.0) {  // exact stationary point
                converged = true;
                break;
            }
            double beta = 0.0;
            if (it % o.cg_reset != 0 && gg_prev > 0.0) beta = std::max(0.0, (gg - ggp) / gg_prev);
            note_launch();
            k_cg_dir<<<grid_for(nl), 256, 0, s>>>(nl, beta, Pdir, c->D.p);
            LSQ_CHECK_LAUNCH();
            double cc[3];
            LSQ_TRY(line_coeffs(c, L, S, o.spin, prec, cc, s));
            if (cc[0] >= 0.0 && beta != 0.0) {  // not a descent direction: restart
                note_launch();
                k_cg_dir<<<grid_for(nl), 256, 0, s>>>(nl, 0.0, Pdir, c->D.p);
                LSQ_CHECK_LAUNCH();
                LSQ_TRY(line_coeffs(c, L, S, o.spin, prec, cc, s));
            }
            double a = 0.0;
            if (!(cc[0] < 0.0) || !line_minimum(cc[0], cc[1], cc[2], &a)) {
                if (o.verbose)
                    std::fprintf(stderr, "lnv step %d: no local minimum, c1 %.6e c2 %.6e c3 %.6e\n", iters,
                                 cc[0], cc[1], cc[2]);
                status = LSQ_ERR_UNSTABLE;
                break;
            }
            note_launch();
            k_axpy<<<grid_for(nl), 256, 0, s>>>(nl, a, c->D.p, L);
            const int64_t n3 = nvals(c, c->r3);
            note_launch();
            if (prec == LSQ_F64)
                k_axpy<<<grid_for(n3), 256, 0, s>>>(n3, a, (const double *)c->QD.p, (double *)c->Q.p);
            else
                k_axpy_f32<<<grid_for(n3), 256, 0, s>>>(n3, a, (const float *)c->QD.p, (float *)c->Q.p);
            LSQ_CHECK_LAUNCH();
            std::swap(c->G.p, c->Gp.p);
            if (metric) std::swap(c->Pm.p, c->Pmp.p);
            gg_prev = gg;
            ++iters;
            if (prec == LSQ_F64) ++iters64;
            const double dom = cc[0] * a + cc[1] * a * a + cc[2] * a * a * a;
            if (o.verbose)
                std::fprintf(stderr,
                             "lnv step %d %s omega %.12e eV |G|^2 %.6e c1 %.6e c2 %.6e c3 %.6e "
                             "alpha %.6e beta %.6e\n",
                             iters - 1, prec == LSQ_F64 ? "f64" : "f32", om, gg, cc[0], cc[1], cc[2], a,
                             beta);
            last_d = std::fabs(dom) / kHartreeEv / std::max(n, 1);
            om_pred = om + dom;
            if (o.tol_ha_per_atom > 0.0 && last_d < o.tol_ha_per_atom) {
                converged = true;
                break;
            }
        }
        if (status == LSQ_ERR_UNSTABLE) break;
        if (phase == 0) converged0 = converged;
        if (phase == nphase - 1 && o.tol_ha_per_atom > 0.0) {
            // converged if the last phase converged, or (mixed path) the FP64 steps stayed below
            // tol, or no FP64 steps were asked for and the mixed ones converged
            if (converged || (nphase == 2 && iters64 > 0 && last_d < o.tol_ha_per_atom) ||
                (nphase == 2 && budget == 0 && converged0))
                status = LSQ_OK;
        }
    }
    double om = om_pred, ne = ne_last;
    if (o.final_eval) LSQ_TRY(energy_gradient(c, L, S, o.spin, LSQ_F64, nullptr, &om, &ne, s));
    auto t1 = std::chrono::steady_clock::now();
    if (rep) {
        rep->iterations = iters;
        rep->iterations_fp64 = iters64;
        rep->status = status;
        rep->omega_ev = om;
        rep->ne = ne;
        rep->omega_ha_per_atom = om / kHartreeEv / std::max(n, 1);
        rep->last_domega_ha_per_atom = last_d;
        rep->seconds = std::chrono::duration<double>(t1 - t0).count();
    }
    if (status == LSQ_ERR_UNSTABLE) return set_error(status, "no local minimum along the CG direction");
    if (status == LSQ_ERR_NOT_CONVERGED) return set_error(status, "iteration limit reached");
    return LSQ_OK;
}

extern "C" int lsq_lnv_minimise_canonical(lsq_lnv c, double *L, const double *S, const double *H,
                                          double n_electrons, const lsq_lnv_opts *opts, lsq_lnv_report *rep,
                                          double *lambda_out, void *stream) {
    clear_error();
    if (!c || !L || !S || !H) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    lsq_lnv_opts o;
    lsq_lnv_default_opts(&o);
    if (opts) o = *opts;
    LSQ_TRY(take_precision(c, &o.precision));
    if (o.max_iter < 0 || o.cg_reset < 1) return set_error(LSQ_ERR_INVALID_ARG, "bad iteration options");
    LSQ_TRY(ensure_ws(c, widest(o)));
    if (!(n_electrons > 0.0)) return set_error(LSQ_ERR_INVALID_ARG, "n_electrons must be positive");
    if (c->rX >= 0) return set_error(LSQ_ERR_UNSUPPORTED, "the canonical minimiser has no metric; clear it");
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    lsq_geom g = c->g;
    const int n = g->n, b = c->b;
    const int64_t nl = nvals(c, c->rL);
    const int prec = o.precision;
    const double tol_ne = (prec == LSQ_F64 ? 1e-9 : 1e-6) * n_electrons;
    const int max_correct = 5;
    // mu = 0: H' = H, so the grand potential of energy_gradient is E_band
    LSQ_TRY(prepare_hs(c, S, H, 0.0, LSQ_F64, s));
    if (prec == LSQ_F32) LSQ_TRY(prepare_hs(c, S, H, 0.0, LSQ_F32, s));
    DevBuf<double> GN;
    LSQ_TRY(GN.alloc((size_t)std::max<int64_t>(nl, 1)));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->Gp.p, 0, sizeof(double) * nl, s));
    int status = o.tol_ha_per_atom > 0.0 ? LSQ_ERR_NOT_CONVERGED : LSQ_OK;
    int iters = 0;
    double gg_prev = 0.0, E = 0.0, N = 0.0, lam = 0.0, last_d = 0.0;
    auto dot2 = [&](const double *x, const double *y, const double *u, const double *v, double *out) {
        LSQ_TRY(dot_into(g, b, LSQ_F64, c->rL, x, y, 10, s));
        LSQ_TRY(dot_into(g, b, LSQ_F64, c->rL, u, v, 11, s));
        double t[12];
        LSQ_TRY(fetch_scalars(g, 12, t, s));
        out[0] = t[10];
        out[1] = t[11];
        return LSQ_OK;
    };
    for (int it = 0; it < o.max_iter; ++it) {
        // restore N_e along dN_e/dL
        double gnn = 0.0;
        for (int corr = 0;; ++corr) {
            LSQ_TRY(energy_gradient(c, L, S, o.spin, prec, GN.p, &N, nullptr, s, false, false, false, true));
            double t2[2];
            LSQ_TRY(dot2(GN.p, GN.p, GN.p, GN.p, t2));
            gnn = t2[0];
            if (!(gnn > 0.0)) return set_error(LSQ_ERR_UNSTABLE, "the electron-number gradient vanished");
            if (std::fabs(N - n_electrons) <= tol_ne || corr == max_correct) break;
            note_launch();
            k_axpy<<<grid_for(nl), 256, 0, s>>>(nl, (n_electrons - N) / gnn, GN.p, L);
            LSQ_CHECK_LAUNCH();
        }
        // energy gradient, projected on constant N_e; lam is the chemical potential
        LSQ_TRY(energy_gradient(c, L, S, o.spin, prec, c->G.p, &E, nullptr, s));
        double t2[2];
        LSQ_TRY(dot2(c->G.p, GN.p, c->G.p, c->Gp.p, t2));
        lam = t2[0] / gnn;
        note_launch();
        k_axpy<<<grid_for(nl), 256, 0, s>>>(nl, -lam, GN.p, c->G.p);
        LSQ_CHECK_LAUNCH();
        LSQ_TRY(dot2(c->G.p, c->G.p, c->G.p, c->Gp.p, t2));
        const double gg = t2[0], ggp = t2[1];
        if (gg == 0.0) {
            status = LSQ_OK;
            break;
        }
        double beta = 0.0;
        if (it % o.cg_reset != 0 && gg_prev > 0.0) beta = std::max(0.0, (gg - ggp) / gg_prev);
        auto direction = [&](double bt) {
            note_launch();
            k_cg_dir<<<grid_for(nl), 256, 0, s>>>(nl, bt, c->G.p, c->D.p);
            LSQ_CHECK_LAUNCH();
            double d2[2];
            LSQ_TRY(dot2(c->D.p, GN.p, c->D.p, GN.p, d2));
            note_launch();
            k_axpy<<<grid_for(nl), 256, 0, s>>>(nl, -d2[0] / gnn, GN.p, c->D.p);
            LSQ_CHECK_LAUNCH();
            return LSQ_OK;
        };
        LSQ_TRY(direction(beta));
        double cc[3];
        LSQ_TRY(line_coeffs(c, L, S, o.spin, prec, cc, s));
        if (cc[0] >= 0.0 && beta != 0.0) {
            LSQ_TRY(direction(0.0));
            LSQ_TRY(line_coeffs(c, L, S, o.spin, prec, cc, s));
        }
        double a = 0.0;
        if (!(cc[0] < 0.0) || !line_minimum(cc[0], cc[1], cc[2], &a)) {
            status = LSQ_ERR_UNSTABLE;
            break;
        }
        note_launch();
        k_axpy<<<grid_for(nl), 256, 0, s>>>(nl, a, c->D.p, L);
        LSQ_CHECK_LAUNCH();
        std::swap(c->G.p, c->Gp.p);
        gg_prev = gg;
        ++iters;
        const double de = cc[0] * a + cc[1] * a * a + cc[2] * a * a * a;
        last_d = std::fabs(de) / kHartreeEv / std::max(n, 1);
        if (o.verbose)
            std::fprintf(stderr, "lnv canonical step %d E %.12e eV N_e %.12f lambda %.6f alpha %.6e\n", iters - 1, E,
                         N, lam, a);
        if (o.tol_ha_per_atom > 0.0 && last_d < o.tol_ha_per_atom) {
            status = LSQ_OK;
            break;
        }
    }
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    if (lambda_out) *lambda_out = lam;
    if (rep) {
        rep->iterations = iters;
        rep->iterations_fp64 = prec == LSQ_F64 ? iters : 0;
        rep->status = status;
        rep->omega_ev = E;
        rep->ne = N;
        rep->omega_ha_per_atom = E / kHartreeEv / std::max(n, 1);
        rep->last_domega_ha_per_atom = last_d;
        rep->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    if (status == LSQ_ERR_UNSTABLE) return set_error(status, "no local minimum along the CG direction");
    if (status == LSQ_ERR_NOT_CONVERGED) return set_error(status, "iteration limit reached");
    return LSQ_OK;
}


namespace {

int batch_alloc(lsq_lnv c) {
    lsq_geom g = c->g;
    const int ns = g->n_sys;
    if (c->b_nsys == ns && c->b_slots.p) return LSQ_OK;
    c->b_nsys = ns;
    LSQ_TRY(c->b_slots.alloc((size_t)ns * kSlots));
    LSQ_TRY(c->b_rowsum.alloc((size_t)std::max(g->n, 1)));
    LSQ_TRY(c->b_mu.alloc(ns));
    LSQ_TRY(c->b_gg_prev.alloc(ns));
    LSQ_TRY(c->b_beta.alloc(ns));
    LSQ_TRY(c->b_alpha.alloc(ns));
    LSQ_TRY(c->b_omega.alloc(ns));
    LSQ_TRY(c->b_dom.alloc(ns));
    LSQ_TRY(c->b_status.alloc(ns));
    LSQ_TRY(c->b_frozen.alloc(ns));
    LSQ_TRY(c->b_reset.alloc(ns));
    LSQ_TRY(c->b_iters.alloc(ns));
    LSQ_TRY(c->b_natoms.alloc(ns));
    LSQ_TRY(c->b_step.alloc(1));
    LSQ_TRY(c->b_off.alloc((size_t)ns + 1));
    std::vector<int> na(ns);
    for (int k = 0; k < ns; ++k) na[k] = (int)(g->sys_atom_off[k + 1] - g->sys_atom_off[k]);
    LSQ_CUDA_TRY(cudaMemcpy(c->b_natoms.p, na.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    LSQ_CUDA_TRY(cudaMemcpy(c->b_off.p, g->sys_atom_off.data(), sizeof(int64_t) * (ns + 1),
                            cudaMemcpyHostToDevice));
    return LSQ_OK;
}

BatchDev batch_dev(lsq_lnv c) {
    BatchDev d;
    d.slots = c->b_slots.p;
    d.gg_prev = c->b_gg_prev.p;
    d.beta = c->b_beta.p;
    d.alpha = c->b_alpha.p;
    d.omega = c->b_omega.p;
    d.dom = c->b_dom.p;
    d.status = c->b_status.p;
    d.frozen = c->b_frozen.p;
    d.reset = c->b_reset.p;
    d.iters = c->b_iters.p;
    d.natoms = c->b_natoms.p;
    d.step = c->b_step.p;
    return d;
}

// One CG step of every system, enqueued on s with no host synchronisation.
// reuse_q: Q was carried along the previous step's line search (see lsq_lnv_minimise).
int batch_step(lsq_lnv c, double *L, const double *S, double spin, int prec, double tol, int cg_reset,
               cudaStream_t s, bool reuse_q) {
    lsq_geom g = c->g;
    const int ns = g->n_sys, bb = c->b * c->b;
    const int rows = (int)(((int64_t)g->n * 32 + 255) / 256);
    const int *asys = g->n_sys > 1 ? g->atom_sys.p : nullptr;
    BatchDev d = batch_dev(c);
    LSQ_TRY(energy_gradient(c, L, S, spin, prec, c->G.p, nullptr, nullptr, s, true, false, reuse_q));
    // in a metric X the directions come from P = X G X (block diagonal over the systems, as X is)
    // and each system's Polak-Ribiere sums are <G, P> and <G, P_prev>
    const bool metric = c->rX >= 0;
    if (metric) LSQ_TRY(metric_apply(c, prec, c->G.p, s));
    double *Pdir = metric ? c->Pm.p : c->G.p, *Pprev = metric ? c->Pmp.p : c->Gp.p;
    LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, c->G.p, Pdir, 10, s));
    LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, c->G.p, Pprev, 11, s));
    note_launch();
    k_batch_beta<<<(ns + 127) / 128, 128, 0, s>>>(ns, spin, cg_reset, d);
    note_launch();
    k_batch_dir<<<rows, 256, 0, s>>>(g->n, bb, g->pats[c->rL].row_ptr.p, asys, c->b_beta.p, Pdir, c->D.p);
    LSQ_CHECK_LAUNCH();
    double unused[3];
    LSQ_TRY(line_coeffs(c, L, S, spin, prec, unused, s, true));
    note_launch();
    k_batch_alpha<<<(ns + 127) / 128, 128, 0, s>>>(ns, spin, tol, d);
    note_launch();
    k_batch_update<<<rows, 256, 0, s>>>(g->n, bb, g->pats[c->rL].row_ptr.p, asys, c->b_alpha.p, c->D.p, L,
                                        Pdir, Pprev);
    note_launch();
    if (prec == LSQ_F64)
        k_batch_axpy_rows<double><<<rows, 256, 0, s>>>(g->n, bb, g->pats[c->r3].row_ptr.p, asys, c->b_alpha.p,
                                                        (const double *)c->QD.p, (double *)c->Q.p);
    else
        k_batch_axpy_rows<float><<<rows, 256, 0, s>>>(g->n, bb, g->pats[c->r3].row_ptr.p, asys, c->b_alpha.p,
                                                       (const float *)c->QD.p, (float *)c->Q.p);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

int batch_prepare_hs(lsq_lnv c, const double *S, const double *H, int prec, cudaStream_t s) {
    lsq_geom g = c->g;
    const int bb = c->b * c->b;
    const int rows = (int)(((int64_t)g->n * 32 + 255) / 256);
    note_launch();
    k_hprime_rows<<<rows, 256, 0, s>>>(g->n, bb, g->pats[c->rH].row_ptr.p, g->n_sys > 1 ? g->atom_sys.p : nullptr,
                                       c->b_mu.p, H, S, c->pos_s_in_h, c->Hp.p, c->Sh.p);
    LSQ_CHECK_LAUNCH();
    if (prec == LSQ_F32) {
        int64_t nh = nvals(c, c->rH), ns = nvals(c, c->rS);
        note_launch();
        k_to_f32<<<grid_for(nh), 256, 0, s>>>(nh, c->Hp.p, (float *)c->Hpc.p);
        note_launch();
        k_to_f32<<<grid_for(nh), 256, 0, s>>>(nh, c->Sh.p, (float *)c->Shc.p);
        note_launch();
        k_to_f32<<<grid_for(ns), 256, 0, s>>>(ns, S, (float *)c->Sc.p);
        LSQ_CHECK_LAUNCH();
    }
    return LSQ_OK;
}

// Step graphs of one batch call: kind 0 forms Q = H'LS afresh, kind 1 carries it along the line
// search (every kQFresh-th step is fresh, as in the single-system minimiser).
struct StepGraphs {
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaGraph_t graph[2] = {nullptr, nullptr};
    std::vector<void *> dev;  // grouped launches' descriptors and queue counters
    ~StepGraphs() {
        for (int k = 0; k < 2; ++k) {
            if (exec[k]) cudaGraphExecDestroy(exec[k]);
            if (graph[k]) cudaGraphDestroy(graph[k]);
        }
        for (void *p : dev) cudaFree(p);
    }
};

// Adds a segment of a context's step to G after deps (an empty node for an empty segment).
int add_segment(cudaGraph_t G, const std::vector<cudaGraphNode_t> &deps, cudaGraph_t seg, cudaGraphNode_t *out) {
    size_t nn = 0;
    LSQ_CUDA_TRY(cudaGraphGetNodes(seg, nullptr, &nn));
    if (nn == 0)
        LSQ_CUDA_TRY(cudaGraphAddEmptyNode(out, G, deps.data(), deps.size()));
    else
        LSQ_CUDA_TRY(cudaGraphAddChildGraphNode(out, G, deps.data(), deps.size(), seg));
    return LSQ_OK;
}

// One CG step of every context as a single graph.  Each context's step is captured with its
// products split out (GroupRecorder): segment k of every context runs, then the k-th products of
// all contexts run as one grouped persistent launch (group_launch), then segment k + 1 of
// every context.  Contexts whose step has fewer products simply have fewer segments.
int capture_group_step(int nctx, lsq_lnv *cs, double **L, const double **S, double spin, int prec, double tol,
                       int cg_reset, cudaStream_t s, bool reuse_q, StepGraphs &sg, int kind) {
    std::vector<std::unique_ptr<GroupRecorder>> recs(nctx);
    for (int c = 0; c < nctx; ++c) {
        recs[c].reset(new GroupRecorder());
        LSQ_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        g_group_rec = recs[c].get();
        const int rc = batch_step(cs[c], L[c], S[c], spin, prec, tol, cg_reset, s, reuse_q);
        g_group_rec = nullptr;
        cudaGraph_t last = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(s, &last);
        if (last) recs[c]->segments.push_back(last);
        if (rc != LSQ_OK) return rc;
        if (ec != cudaSuccess) return set_error(LSQ_ERR_CUDA, std::string("step capture: ") + cudaGetErrorString(ec));
    }
    size_t nprod = 0;
    for (int c = 0; c < nctx; ++c) nprod = std::max(nprod, recs[c]->products.size());
    unsigned long long *counters = nullptr;
    LSQ_CUDA_TRY(cudaMalloc(&counters, sizeof(unsigned long long) * std::max<size_t>(nprod, 1)));
    sg.dev.push_back(counters);
    cudaGraph_t G = nullptr;
    LSQ_CUDA_TRY(cudaGraphCreate(&G, 0));
    sg.graph[kind] = G;
    cudaStream_t side = nullptr;
    LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking));
    struct SideStream {
        cudaStream_t s;
        ~SideStream() { cudaStreamDestroy(s); }
    } side_guard{side};
    std::vector<cudaGraphNode_t> prev;
    for (size_t k = 0; k <= nprod; ++k) {
        std::vector<cudaGraphNode_t> deps;
        for (int c = 0; c < nctx; ++c) {
            if (k >= recs[c]->segments.size()) continue;
            cudaGraphNode_t node;
            LSQ_TRY(add_segment(G, prev, recs[c]->segments[k], &node));
            deps.push_back(node);
        }
        if (k == nprod) break;
        std::vector<GroupProduct> prods;
        for (int c = 0; c < nctx; ++c)
            if (k < recs[c]->products.size()) prods.push_back(recs[c]->products[k]);
        GroupLaunch gl;
        LSQ_TRY(group_prepare(prods.data(), (int)prods.size(), cs[0]->g, &gl));
        sg.dev.push_back(gl.desc);
        // the launch (queue reset and kernel) as a small graph of its own
        LSQ_CUDA_TRY(cudaStreamBeginCapture(side, cudaStreamCaptureModeThreadLocal));
        const int rc = group_launch(gl, counters + k, side);
        cudaGraph_t pg = nullptr;
        const cudaError_t ec = cudaStreamEndCapture(side, &pg);
        if (rc != LSQ_OK) {
            if (pg) cudaGraphDestroy(pg);
            return rc;
        }
        if (ec != cudaSuccess) return set_error(LSQ_ERR_CUDA, std::string("product capture: ") + cudaGetErrorString(ec));
        cudaGraphNode_t node;
        const cudaError_t ea = cudaGraphAddChildGraphNode(&node, G, deps.data(), deps.size(), pg);
        cudaGraphDestroy(pg);
        if (ea != cudaSuccess) return set_error(LSQ_ERR_CUDA, std::string("product node: ") + cudaGetErrorString(ea));
        prev.assign(1, node);
    }
    LSQ_CUDA_TRY(cudaGraphInstantiate(&sg.exec[kind], G, 0));
    return LSQ_OK;
}

// The batched minimiser over nctx contexts (each on its own block-diagonal geometry, with its own
// block size).  grouped: the steps after the first run as graphs whose products are grouped
// launches over all contexts (capture_group_step); otherwise (one context) each step is captured
// as it runs, with the tuned product kernels.
int minimise_batch_impl(int nctx, lsq_lnv *cs, double **L, const double **S, const double **H,
                        const double **mu_host, const lsq_lnv_opts *opts, lsq_lnv_report **reps, cudaStream_t us,
                        bool grouped) {
    if (nctx < 1 || !cs || !L || !S || !H || !mu_host) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    for (int c = 0; c < nctx; ++c) {
        if (!cs[c] || !L[c] || !S[c] || !H[c] || !mu_host[c]) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
        if ((cs[c]->rX >= 0) != (cs[0]->rX >= 0))
            return set_error(LSQ_ERR_INVALID_ARG, "the contexts of a batch take a metric all or none");
        for (int d = 0; d < c; ++d)
            if (cs[d]->g == cs[c]->g)
                return set_error(LSQ_ERR_INVALID_ARG, "the contexts of a grouped batch need distinct geometries");
    }
    lsq_lnv_opts o;
    lsq_lnv_default_opts(&o);
    if (opts) o = *opts;
    if (grouped && o.precision != LSQ_F64 && o.precision != LSQ_F32)
        return set_error(LSQ_ERR_INVALID_ARG, "a grouped batch runs LSQ_F64 or LSQ_F32 products");
    for (int c = 0; c < nctx; ++c) {
        int pr = o.precision;
        LSQ_TRY(take_precision(cs[c], &pr));
        if (c == nctx - 1) o.precision = pr;
    }
    if (o.max_iter < 0 || o.cg_reset < 1 || o.refine_iter < 0)
        return set_error(LSQ_ERR_INVALID_ARG, "bad iteration options");
    auto t0 = std::chrono::steady_clock::now();
    for (int c = 0; c < nctx; ++c) {
        LSQ_TRY(ensure_ws(cs[c], widest(o)));
        LSQ_TRY(batch_alloc(cs[c]));
    }
    // Work runs on a private stream ordered after the caller's (a graph cannot be captured
    // from the legacy default stream); the caller's stream waits for it at the end.
    cudaStream_t s = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    LSQ_CUDA_TRY(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    LSQ_CUDA_TRY(cudaEventCreateWithFlags(&ev_in, cudaEventDisableTiming));
    LSQ_CUDA_TRY(cudaEventCreateWithFlags(&ev_out, cudaEventDisableTiming));
    struct Cleanup {
        cudaStream_t us, s;
        cudaEvent_t a, b;
        ~Cleanup() {
            g_group_rec = nullptr;
            if (b && s) {
                cudaEventRecord(b, s);
                cudaStreamWaitEvent(us, b, 0);
            }
            if (s) cudaStreamSynchronize(s);
            if (s) cudaStreamDestroy(s);
            if (a) cudaEventDestroy(a);
            if (b) cudaEventDestroy(b);
        }
    } cleanup{us, s, ev_in, ev_out};
    LSQ_CUDA_TRY(cudaEventRecord(ev_in, us));
    LSQ_CUDA_TRY(cudaStreamWaitEvent(s, ev_in, 0));
    std::vector<int> nsys(nctx);
    for (int c = 0; c < nctx; ++c) {
        lsq_lnv x = cs[c];
        const int ns = x->g->n_sys;
        nsys[c] = ns;
        const int64_t nl = nvals(x, x->rL);
        LSQ_CUDA_TRY(cudaMemcpyAsync(x->b_mu.p, mu_host[c], sizeof(double) * ns, cudaMemcpyHostToDevice, s));
        LSQ_TRY(batch_prepare_hs(x, S[c], H[c], LSQ_F64, s));
        if (o.precision == LSQ_F32) LSQ_TRY(batch_prepare_hs(x, S[c], H[c], LSQ_F32, s));
        LSQ_CUDA_TRY(cudaMemsetAsync(x->Gp.p, 0, sizeof(double) * nl, s));
        if (x->rX >= 0) LSQ_CUDA_TRY(cudaMemsetAsync(x->Pmp.p, 0, sizeof(double) * nl, s));
        LSQ_CUDA_TRY(cudaMemsetAsync(x->b_frozen.p, 0, sizeof(int) * ns, s));
        LSQ_CUDA_TRY(cudaMemsetAsync(x->b_iters.p, 0, sizeof(int) * ns, s));
        LSQ_CUDA_TRY(cudaMemsetAsync(x->b_gg_prev.p, 0, sizeof(double) * ns, s));
        LSQ_CUDA_TRY(cudaMemsetAsync(x->b_dom.p, 0, sizeof(double) * ns, s));
        std::vector<int> one(ns, 1), st(ns, o.tol_ha_per_atom > 0.0 ? LSQ_ERR_NOT_CONVERGED : LSQ_OK);
        LSQ_CUDA_TRY(cudaMemcpyAsync(x->b_reset.p, one.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        LSQ_CUDA_TRY(cudaMemcpyAsync(x->b_status.p, st.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    std::vector<std::vector<int>> iters64(nctx), frozen(nctx), status(nctx), it_before(nctx);
    for (int c = 0; c < nctx; ++c) {
        iters64[c].assign(nsys[c], 0);
        frozen[c].assign(nsys[c], 0);
        status[c].assign(nsys[c], 0);
        it_before[c].assign(nsys[c], 0);
    }
    const int nphase = o.precision == LSQ_F32 ? 2 : 1;
    const int check_every = 5;
    for (int phase = 0; phase < nphase; ++phase) {
        const int prec = phase == 0 ? o.precision : LSQ_F64;
        const int budget = phase == 0 ? o.max_iter : o.refine_iter;
        for (int c = 0; c < nctx; ++c) {
            lsq_lnv x = cs[c];
            const int ns = nsys[c];
            if (phase == 1) {
                // refinement: float64 steps from a fresh direction for every system that did not fail
                LSQ_CUDA_TRY(cudaMemcpy(status[c].data(), x->b_status.p, sizeof(int) * ns, cudaMemcpyDeviceToHost));
                LSQ_CUDA_TRY(cudaMemcpy(it_before[c].data(), x->b_iters.p, sizeof(int) * ns, cudaMemcpyDeviceToHost));
                for (int k = 0; k < ns; ++k) frozen[c][k] = status[c][k] == LSQ_ERR_UNSTABLE ? 1 : 0;
                std::vector<int> one(ns, 1);
                LSQ_CUDA_TRY(cudaMemcpy(x->b_frozen.p, frozen[c].data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
                LSQ_CUDA_TRY(cudaMemcpy(x->b_reset.p, one.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
            }
            LSQ_CUDA_TRY(cudaMemsetAsync(x->b_step.p, 0, sizeof(int), s));
        }
        // tol = 0 freezes nothing; the refinement uses tol = 0 (fixed number of steps)
        const double tol = phase == 0 ? o.tol_ha_per_atom : 0.0;
        StepGraphs sg;
        for (int it = 0; it < budget; ++it) {
            const int kind = it % std::min(o.cg_reset, kQFresh) != 0 ? 1 : 0;
            if (it >= 1 && (o.graph || grouped) && !sg.exec[kind]) {
                // plans, maps and autotuning exist after the first step: capture this kind of step
                if (grouped) {
                    LSQ_TRY(capture_group_step(nctx, cs, L, S, o.spin, prec, tol, o.cg_reset, s, kind == 1, sg,
                                               kind));
                } else {
                    LSQ_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
                    int rc = batch_step(cs[0], L[0], S[0], o.spin, prec, tol, o.cg_reset, s, kind == 1);
                    cudaError_t ec = cudaStreamEndCapture(s, &sg.graph[kind]);
                    if (rc != LSQ_OK) return rc;
                    if (ec != cudaSuccess) return set_error(LSQ_ERR_CUDA, cudaGetErrorString(ec));
                    LSQ_CUDA_TRY(cudaGraphInstantiate(&sg.exec[kind], sg.graph[kind], 0));
                }
            }
            if (sg.exec[kind]) {
                LSQ_CUDA_TRY(cudaGraphLaunch(sg.exec[kind], s));
            } else {
                for (int c = 0; c < nctx; ++c)
                    LSQ_TRY(batch_step(cs[c], L[c], S[c], o.spin, prec, tol, o.cg_reset, s, kind == 1));
            }
            if (tol > 0.0 && (it + 1) % check_every == 0) {
                bool all = true;
                for (int c = 0; c < nctx; ++c) {
                    LSQ_CUDA_TRY(cudaMemcpyAsync(frozen[c].data(), cs[c]->b_frozen.p, sizeof(int) * nsys[c],
                                                 cudaMemcpyDeviceToHost, s));
                    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
                    for (int k = 0; k < nsys[c]; ++k) all = all && frozen[c][k];
                }
                if (all) break;
            }
        }
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
        for (int c = 0; c < nctx; ++c) {
            const int ns = nsys[c];
            if (phase == 1) {
                std::vector<int> it_after(ns);
                LSQ_CUDA_TRY(cudaMemcpy(it_after.data(), cs[c]->b_iters.p, sizeof(int) * ns, cudaMemcpyDeviceToHost));
                for (int k = 0; k < ns; ++k) iters64[c][k] = it_after[k] - it_before[c][k];
            } else if (prec == LSQ_F64) {
                LSQ_CUDA_TRY(cudaMemcpy(iters64[c].data(), cs[c]->b_iters.p, sizeof(int) * ns, cudaMemcpyDeviceToHost));
            }
        }
    }
    // final float64 Omega and N_e of every system (without it the report keeps the Omega of the
    // last step's energy evaluation, in the working precision, and no N_e)
    if (o.final_eval)
        for (int c = 0; c < nctx; ++c)
            LSQ_TRY(energy_gradient(cs[c], L[c], S[c], o.spin, LSQ_F64, nullptr, nullptr, nullptr, s, true, true));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = LSQ_OK;
    for (int c = 0; c < nctx; ++c) {
        lsq_lnv x = cs[c];
        lsq_geom g = x->g;
        const int ns = nsys[c];
        std::vector<double> slots((size_t)ns * kSlots), dom(ns);
        std::vector<int> iters(ns);
        LSQ_CUDA_TRY(cudaMemcpyAsync(slots.data(), x->b_slots.p, sizeof(double) * ns * kSlots, cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaMemcpyAsync(dom.data(), x->b_dom.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaMemcpyAsync(iters.data(), x->b_iters.p, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaMemcpyAsync(status[c].data(), x->b_status.p, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
        for (int k = 0; k < ns; ++k) {
            const double *sl = slots.data() + (size_t)k * kSlots;
            const int na = (int)(g->sys_atom_off[k + 1] - g->sys_atom_off[k]);
            int st = status[c][k];
            if (nphase == 2 && st != LSQ_ERR_UNSTABLE && o.tol_ha_per_atom > 0.0 && iters64[c][k] > 0 &&
                dom[k] < o.tol_ha_per_atom)
                st = LSQ_OK;
            if (reps && reps[c]) {
                lsq_lnv_report &r = reps[c][k];
                r.iterations = iters[k];
                r.iterations_fp64 = iters64[c][k];
                r.status = st;
                r.omega_ev = o.spin * (3.0 * sl[0] - 2.0 * sl[1]);
                r.ne = o.final_eval ? o.spin * (3.0 * sl[2] - 2.0 * sl[3]) : std::nan("");
                r.omega_ha_per_atom = r.omega_ev / kHartreeEv / std::max(na, 1);
                r.last_domega_ha_per_atom = dom[k];
                r.seconds = sec;
            }
            if (st == LSQ_ERR_UNSTABLE) worst = LSQ_ERR_UNSTABLE;
            else if (st == LSQ_ERR_NOT_CONVERGED && worst == LSQ_OK) worst = LSQ_ERR_NOT_CONVERGED;
        }
    }
    if (worst == LSQ_ERR_UNSTABLE) return set_error(worst, "a system has no local minimum along its CG direction");
    if (worst == LSQ_ERR_NOT_CONVERGED) return set_error(worst, "iteration limit reached for a system");
    return LSQ_OK;
}

}  // namespace

extern "C" int lsq_lnv_minimise_batch(lsq_lnv c, double *L, const double *S, const double *H,
                                      const double *mu_host, const lsq_lnv_opts *opts,
                                      lsq_lnv_report *reps, void *stream) {
    clear_error();
    if (!c || !L || !S || !H || !mu_host) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    return minimise_batch_impl(1, &c, &L, &S, &H, &mu_host, opts, &reps, (cudaStream_t)stream, false);
}

extern "C" int lsq_lnv_minimise_batch_group(int n_ctx, lsq_lnv *ctx, double **L_dev, const double **S_dev,
                                            const double **H_dev, const double **mu_host,
                                            const lsq_lnv_opts *opts, lsq_lnv_report **reps, void *stream) {
    clear_error();
    if (n_ctx < 1 || n_ctx > kMaxGroupContexts)
        return set_error(LSQ_ERR_INVALID_ARG, "n_ctx must be in [1, " + std::to_string(kMaxGroupContexts) + "]");
    return minimise_batch_impl(n_ctx, ctx, L_dev, S_dev, H_dev, mu_host, opts, reps, (cudaStream_t)stream, true);
}

namespace {

// Canonical batch, after an evaluation with S in place of H' (slots 0, 1: N_e's traces; slot 10:
// <G_N, G_N>): N_e of every system, and the Newton move (N0 - N_e) / <G_N, G_N> along G_N for each
// system still off by more than tol_rel N0 (0 for the others, for frozen systems and on the last
// evaluation of a step).  pending counts the systems that move.
__global__ void k_bcan_ne(int nsys, double spin, const double *__restrict__ n0, double tol_rel, int last,
                          BatchDev d, double *__restrict__ ne, double *__restrict__ gnn, double *__restrict__ coef,
                          int *__restrict__ pending) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const double *sl = d.slots + (int64_t)s * kSlots;
    const double N = spin * (3.0 * sl[0] - 2.0 * sl[1]);
    double cf = 0.0;
    if (!d.frozen[s]) {
        ne[s] = N;
        gnn[s] = sl[10];
        if (!(sl[10] > 0.0)) {  // the electron-number gradient vanished
            d.status[s] = LSQ_ERR_UNSTABLE;
            d.frozen[s] = 1;
        } else if (!last && fabs(N - n0[s]) > tol_rel * n0[s]) {
            cf = (n0[s] - N) / sl[10];
            atomicAdd(pending, 1);
        }
    }
    coef[s] = cf;
}

// coef = -<X, G_N> / <G_N, G_N> of every system (slot 12 holds <X, G_N>); with lam != null the
// ratio itself is the system's multiplier lambda (X = the energy gradient).
__global__ void k_bcan_proj(int nsys, BatchDev d, const double *__restrict__ gnn, double *__restrict__ lam,
                            double *__restrict__ coef) {
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nsys) return;
    const double r = d.frozen[s] ? 0.0 : d.slots[(int64_t)s * kSlots + 12] / gnn[s];
    if (lam && !d.frozen[s]) lam[s] = r;
    coef[s] = -r;
}

}  // namespace

extern "C" int lsq_lnv_minimise_batch_canonical(lsq_lnv c, double *L, const double *S, const double *H,
                                                const double *n_electrons_host, const lsq_lnv_opts *opts,
                                                lsq_lnv_report *reps, double *lambda_host, void *stream) {
    clear_error();
    if (!c || !L || !S || !H || !n_electrons_host) return set_error(LSQ_ERR_INVALID_ARG, "null argument");
    lsq_lnv_opts o;
    lsq_lnv_default_opts(&o);
    if (opts) o = *opts;
    LSQ_TRY(take_precision(c, &o.precision));
    if (o.max_iter < 0 || o.cg_reset < 1) return set_error(LSQ_ERR_INVALID_ARG, "bad iteration options");
    if (c->rX >= 0) return set_error(LSQ_ERR_UNSUPPORTED, "the canonical minimiser has no metric; clear it");
    lsq_geom g = c->g;
    const int ns = g->n_sys, bb = c->b * c->b;
    for (int k = 0; k < ns; ++k)
        if (!(n_electrons_host[k] > 0.0)) return set_error(LSQ_ERR_INVALID_ARG, "n_electrons must be positive");
    LSQ_TRY(ensure_ws(c, widest(o)));
    LSQ_TRY(batch_alloc(c));
    cudaStream_t s = (cudaStream_t)stream;
    auto t0 = std::chrono::steady_clock::now();
    const int prec = o.precision;
    const double tol_ne = prec == LSQ_F64 ? 1e-9 : 1e-6;  // relative, as lsq_lnv_minimise_canonical
    const int max_correct = 5;
    const int64_t nl = nvals(c, c->rL);
    const int rows = (int)(((int64_t)g->n * 32 + 255) / 256);
    const int *asys = ns > 1 ? g->atom_sys.p : nullptr;
    const int64_t *rpL = g->pats[c->rL].row_ptr.p;
    DevBuf<double> GN, n0, ne, gnn, lam, coef;
    DevBuf<int> pending;
    LSQ_TRY(GN.alloc((size_t)std::max<int64_t>(nl, 1)));
    LSQ_TRY(n0.alloc(ns));
    LSQ_TRY(ne.alloc(ns));
    LSQ_TRY(gnn.alloc(ns));
    LSQ_TRY(lam.alloc(ns));
    LSQ_TRY(coef.alloc(ns));
    LSQ_TRY(pending.alloc(1));
    // mu = 0 for every system: H' = H, so the grand potential of an evaluation is E_band
    LSQ_CUDA_TRY(cudaMemsetAsync(c->b_mu.p, 0, sizeof(double) * ns, s));
    LSQ_TRY(batch_prepare_hs(c, S, H, LSQ_F64, s));
    if (prec == LSQ_F32) LSQ_TRY(batch_prepare_hs(c, S, H, LSQ_F32, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(n0.p, n_electrons_host, sizeof(double) * ns, cudaMemcpyHostToDevice, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->Gp.p, 0, sizeof(double) * nl, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->b_frozen.p, 0, sizeof(int) * ns, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->b_iters.p, 0, sizeof(int) * ns, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->b_gg_prev.p, 0, sizeof(double) * ns, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->b_dom.p, 0, sizeof(double) * ns, s));
    LSQ_CUDA_TRY(cudaMemsetAsync(c->b_step.p, 0, sizeof(int), s));
    LSQ_CUDA_TRY(cudaMemsetAsync(lam.p, 0, sizeof(double) * ns, s));
    {
        std::vector<int> one(ns, 1), st(ns, o.tol_ha_per_atom > 0.0 ? LSQ_ERR_NOT_CONVERGED : LSQ_OK);
        LSQ_CUDA_TRY(cudaMemcpyAsync(c->b_reset.p, one.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        LSQ_CUDA_TRY(cudaMemcpyAsync(c->b_status.p, st.data(), sizeof(int) * ns, cudaMemcpyHostToDevice, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    BatchDev d = batch_dev(c);
    std::vector<int> frozen(ns);
    const int sb = (ns + 127) / 128;
    for (int it = 0; it < o.max_iter; ++it) {
        // restore every system's N_e along its dN_e/dL (Newton moves, at most max_correct)
        for (int corr = 0; corr <= max_correct; ++corr) {
            LSQ_TRY(energy_gradient(c, L, S, o.spin, prec, GN.p, nullptr, nullptr, s, true, false, false, true));
            LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, GN.p, GN.p, 10, s));
            LSQ_CUDA_TRY(cudaMemsetAsync(pending.p, 0, sizeof(int), s));
            note_launch();
            k_bcan_ne<<<sb, 128, 0, s>>>(ns, o.spin, n0.p, tol_ne, corr == max_correct ? 1 : 0, d, ne.p, gnn.p,
                                         coef.p, pending.p);
            LSQ_CHECK_LAUNCH();
            int np = 0;
            LSQ_CUDA_TRY(cudaMemcpyAsync(&np, pending.p, sizeof(int), cudaMemcpyDeviceToHost, s));
            LSQ_CUDA_TRY(cudaStreamSynchronize(s));
            if (np == 0) break;
            note_launch();
            k_batch_axpy_rows<double><<<rows, 256, 0, s>>>(g->n, bb, rpL, asys, coef.p, GN.p, L);
            LSQ_CHECK_LAUNCH();
        }
        // the energy gradient projected on constant N_e (lambda = <G_E, G_N> / <G_N, G_N>, the
        // chemical potential), Polak-Ribiere directions projected the same way, the cubic step
        LSQ_TRY(energy_gradient(c, L, S, o.spin, prec, c->G.p, nullptr, nullptr, s, true));
        LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, c->G.p, GN.p, 12, s));
        note_launch();
        k_bcan_proj<<<sb, 128, 0, s>>>(ns, d, gnn.p, lam.p, coef.p);
        note_launch();
        k_batch_axpy_rows<double><<<rows, 256, 0, s>>>(g->n, bb, rpL, asys, coef.p, GN.p, c->G.p);
        LSQ_CHECK_LAUNCH();
        LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, c->G.p, c->G.p, 10, s));
        LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, c->G.p, c->Gp.p, 11, s));
        note_launch();
        k_batch_beta<<<sb, 128, 0, s>>>(ns, o.spin, o.cg_reset, d);
        note_launch();
        k_batch_dir<<<rows, 256, 0, s>>>(g->n, bb, rpL, asys, c->b_beta.p, c->G.p, c->D.p);
        LSQ_CHECK_LAUNCH();
        LSQ_TRY(seg_dot(c, LSQ_F64, c->rL, c->D.p, GN.p, 12, s));
        note_launch();
        k_bcan_proj<<<sb, 128, 0, s>>>(ns, d, gnn.p, nullptr, coef.p);
        note_launch();
        k_batch_axpy_rows<double><<<rows, 256, 0, s>>>(g->n, bb, rpL, asys, coef.p, GN.p, c->D.p);
        LSQ_CHECK_LAUNCH();
        double unused[3];
        LSQ_TRY(line_coeffs(c, L, S, o.spin, prec, unused, s, true));
        note_launch();
        k_batch_alpha<<<sb, 128, 0, s>>>(ns, o.spin, o.tol_ha_per_atom, d);
        note_launch();
        k_batch_update<<<rows, 256, 0, s>>>(g->n, bb, rpL, asys, c->b_alpha.p, c->D.p, L, c->G.p, c->Gp.p);
        LSQ_CHECK_LAUNCH();
        if (o.tol_ha_per_atom > 0.0) {
            LSQ_CUDA_TRY(cudaMemcpyAsync(frozen.data(), c->b_frozen.p, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
            LSQ_CUDA_TRY(cudaStreamSynchronize(s));
            bool all = true;
            for (int k = 0; k < ns; ++k) all = all && frozen[k];
            if (all) break;
        }
    }
    std::vector<double> om(ns), nev(ns), lv(ns), dom(ns);
    std::vector<int> iters(ns), status(ns);
    LSQ_CUDA_TRY(cudaMemcpyAsync(om.data(), c->b_omega.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(nev.data(), ne.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(lv.data(), lam.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(dom.data(), c->b_dom.p, sizeof(double) * ns, cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(iters.data(), c->b_iters.p, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaMemcpyAsync(status.data(), c->b_status.p, sizeof(int) * ns, cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    const double sec = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    int worst = LSQ_OK;
    for (int k = 0; k < ns; ++k) {
        const int na = (int)(g->sys_atom_off[k + 1] - g->sys_atom_off[k]);
        if (reps) {
            lsq_lnv_report &r = reps[k];
            r.iterations = iters[k];
            r.iterations_fp64 = prec == LSQ_F64 ? iters[k] : 0;
            r.status = status[k];
            r.omega_ev = om[k];
            r.ne = nev[k];
            r.omega_ha_per_atom = om[k] / kHartreeEv / std::max(na, 1);
            r.last_domega_ha_per_atom = dom[k];
            r.seconds = sec;
        }
        if (lambda_host) lambda_host[k] = lv[k];
        if (status[k] == LSQ_ERR_UNSTABLE) worst = LSQ_ERR_UNSTABLE;
        else if (status[k] != LSQ_OK && worst == LSQ_OK) worst = status[k];
    }
    if (worst == LSQ_ERR_UNSTABLE) return set_error(worst, "a system found no local minimum or lost dN_e/dL");
    if (worst == LSQ_ERR_NOT_CONVERGED) return set_error(worst, "iteration limit reached");
    return LSQ_OK;
}
