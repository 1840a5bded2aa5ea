// Range patterns of atom-pair matrices on the GPU (cell lists -> CSR of blocks).
//
// Sec. 2.3.2 of the paper: the range of a matrix is set by the distance
// R_ij between atoms i and j; elements with R_ij beyond the cutoff are zero.
// This file builds, for every requested cutoff R, the pattern
// {(i, j) : d_min_image(i, j)^2 <= R^2} as CSR (row_ptr int64, col int32
// sorted ascending), plus position maps between patterns.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lsq_internal.h"

namespace lsq {

std::atomic<long long> g_launch_count{0};
void note_launch() { g_launch_count.fetch_add(1, std::memory_order_relaxed); }

static thread_local int g_last_code = LSQ_OK;
static thread_local std::string g_last_msg;

int set_error(int code, const std::string &msg) {
    g_last_code = code;
    g_last_msg = msg;
    return code;
}
void clear_error() {
    g_last_code = LSQ_OK;
    g_last_msg.clear();
}

// Largest number of candidates (atoms within the largest range) of one row.
constexpr int kMaxRowCandidates = 8192;
constexpr int kMaxRanges = 16;

struct RangeSq {
    double r2[kMaxRanges];
};

// Minimum-image squared distance; every operation correctly rounded, none fused.
__device__ __forceinline__ double min_image_d2(const double *__restrict__ pos, int i, int j,
                                               double Lx, double Ly, double Lz) {
    double L[3] = {Lx, Ly, Lz};
    double d[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        double s = __dsub_rn(pos[3 * j + c], pos[3 * i + c]);
        double t = rint(__ddiv_rn(s, L[c]));
        double u = __dmul_rn(L[c], t);
        d[c] = __dsub_rn(s, u);
    }
    double xy = __dadd_rn(__dmul_rn(d[0], d[0]), __dmul_rn(d[1], d[1]));
    return __dadd_rn(xy, __dmul_rn(d[2], d[2]));
}

__device__ __forceinline__ int cell_coord(double x, double L, int nc) {
    double f = x / L;
    f = f - floor(f);
    int c = (int)(f * nc);
    return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

struct CellGrid {
    int nc[3];
    int noff[3];
    int off[3][3];
    double L[3];
};

__global__ void k_cell_ids(int n, const double *__restrict__ pos, CellGrid cg, int *__restrict__ cid,
                           int *__restrict__ ccount) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int cx = cell_coord(pos[3 * i + 0], cg.L[0], cg.nc[0]);
    int cy = cell_coord(pos[3 * i + 1], cg.L[1], cg.nc[1]);
    int cz = cell_coord(pos[3 * i + 2], cg.L[2], cg.nc[2]);
    int id = (cx * cg.nc[1] + cy) * cg.nc[2] + cz;
    cid[i] = id;
    atomicAdd(&ccount[id], 1);
}

// Exclusive scan of 'count' (length m) into 'out' (length m + 1), one block.
template <typename TI, typename TO>
__global__ void k_scan_single(int64_t m, const TI *__restrict__ count, TO *__restrict__ out) {
    __shared__ TO part[1024];
    int t = threadIdx.x, nt = blockDim.x;
    int64_t seg = (m + nt - 1) / nt;
    int64_t b0 = t * seg, b1 = b0 + seg < m ? b0 + seg : m;
    TO s = 0;
    for (int64_t k = b0; k < b1; ++k) s += (TO)count[k];
    part[t] = s;
    __syncthreads();
    if (t == 0) {
        TO run = 0;
        for (int k = 0; k < nt; ++k) {
            TO v = part[k];
            part[k] = run;
            run += v;
        }
    }
    __syncthreads();
    TO run = part[t];
    for (int64_t k = b0; k < b1; ++k) {
        out[k] = run;
        run += (TO)count[k];
    }
    if (b1 == m && b0 < b1) out[m] = run;
    if (m == 0 && t == 0) out[0] = 0;
}

__global__ void k_cell_fill(int n, const int *__restrict__ cid, int *__restrict__ cfill,
                            int *__restrict__ catoms) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int slot = atomicAdd(&cfill[cid[i]], 1);
    catoms[slot] = i;
}

// One warp per atom: count neighbours within each range (and within the largest).
__global__ void k_pair_count(int n, const double *__restrict__ pos, CellGrid cg,
                             const int *__restrict__ cstart, const int *__restrict__ catoms,
                             RangeSq rs, int nr, double r2max, int64_t *__restrict__ counts,
                             int *__restrict__ max_cand) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    int i = warp;
    int c0[3];
    for (int c = 0; c < 3; ++c) c0[c] = cell_coord(pos[3 * i + c], cg.L[c], cg.nc[c]);
    int cnt[kMaxRanges];
    for (int r = 0; r < nr; ++r) cnt[r] = 0;
    int cand = 0;
    for (int a = 0; a < cg.noff[0]; ++a)
        for (int b = 0; b < cg.noff[1]; ++b)
            for (int c = 0; c < cg.noff[2]; ++c) {
                int x = (c0[0] + cg.off[0][a] + cg.nc[0]) % cg.nc[0];
                int y = (c0[1] + cg.off[1][b] + cg.nc[1]) % cg.nc[1];
                int z = (c0[2] + cg.off[2][c] + cg.nc[2]) % cg.nc[2];
                int id = (x * cg.nc[1] + y) * cg.nc[2] + z;
                for (int q = cstart[id] + lane; q < cstart[id + 1]; q += 32) {
                    int j = catoms[q];
                    double d2 = min_image_d2(pos, i, j, cg.L[0], cg.L[1], cg.L[2]);
                    if (d2 <= r2max) ++cand;
                    for (int r = 0; r < nr; ++r) cnt[r] += (d2 <= rs.r2[r]);
                }
            }
    for (int off = 16; off > 0; off >>= 1) {
        cand += __shfl_xor_sync(0xffffffffu, cand, off);
        for (int r = 0; r < nr; ++r) cnt[r] += __shfl_xor_sync(0xffffffffu, cnt[r], off);
    }
    if (lane == 0) {
        for (int r = 0; r < nr; ++r) counts[(int64_t)r * n + i] = cnt[r];
        atomicMax(max_cand, cand);
    }
}

// One block per atom: gather candidates, sort by atom index, write each range's row.
__global__ void k_pair_fill(int n, const double *__restrict__ pos, CellGrid cg,
                            const int *__restrict__ cstart, const int *__restrict__ catoms,
                            RangeSq rs, int nr, double r2max, int64_t *const *__restrict__ row_ptrs,
                            int32_t *const *__restrict__ cols) {
    extern __shared__ int sj[];  // [kMaxRowCandidates]
    __shared__ int s_cnt;
    __shared__ int s_part[1024];
    int i = blockIdx.x;
    int t = threadIdx.x, nt = blockDim.x;
    if (t == 0) s_cnt = 0;
    __syncthreads();
    int c0[3];
    for (int c = 0; c < 3; ++c) c0[c] = cell_coord(pos[3 * i + c], cg.L[c], cg.nc[c]);
    for (int a = 0; a < cg.noff[0]; ++a)
        for (int b = 0; b < cg.noff[1]; ++b)
            for (int c = 0; c < cg.noff[2]; ++c) {
                int x = (c0[0] + cg.off[0][a] + cg.nc[0]) % cg.nc[0];
                int y = (c0[1] + cg.off[1][b] + cg.nc[1]) % cg.nc[1];
                int z = (c0[2] + cg.off[2][c] + cg.nc[2]) % cg.nc[2];
                int id = (x * cg.nc[1] + y) * cg.nc[2] + z;
                for (int q = cstart[id] + t; q < cstart[id + 1]; q += nt) {
                    int j = catoms[q];
                    double d2 = min_image_d2(pos, i, j, cg.L[0], cg.L[1], cg.L[2]);
                    if (d2 <= r2max) {
                        int k = atomicAdd(&s_cnt, 1);
                        if (k < kMaxRowCandidates) sj[k] = j;
                    }
                }
            }
    __syncthreads();
    int cnt = s_cnt < kMaxRowCandidates ? s_cnt : kMaxRowCandidates;
    int m = 1;
    while (m < cnt) m <<= 1;
    for (int k = cnt + t; k < m; k += nt) sj[k] = 0x7fffffff;
    __syncthreads();
    // bitonic sort of sj[0..m)
    for (int size = 2; size <= m; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int k = t; k < m; k += nt) {
                int p = k ^ stride;
                if (p > k) {
                    bool up = (k & size) == 0;
                    int a = sj[k], b = sj[p];
                    if ((a > b) == up) {
                        sj[k] = b;
                        sj[p] = a;
                    }
                }
            }
            __syncthreads();
        }
    }
    // ordered compaction for each range: contiguous segment per thread
    int seg = (cnt + nt - 1) / nt;
    int b0 = t * seg, b1 = min(cnt, b0 + seg);
    for (int r = 0; r < nr; ++r) {
        int local = 0;
        for (int k = b0; k < b1; ++k)
            local += min_image_d2(pos, i, sj[k], cg.L[0], cg.L[1], cg.L[2]) <= rs.r2[r];
        s_part[t] = local;
        __syncthreads();
        if (t == 0) {
            int run = 0;
            for (int k = 0; k < nt; ++k) {
                int v = s_part[k];
                s_part[k] = run;
                run += v;
            }
        }
        __syncthreads();
        int64_t w = row_ptrs[r][i] + s_part[t];
        for (int k = b0; k < b1; ++k) {
            int j = sj[k];
            if (min_image_d2(pos, i, j, cg.L[0], cg.L[1], cg.L[2]) <= rs.r2[r]) cols[r][w++] = j;
        }
        __syncthreads();
    }
}

// Position of column 'key' within row 'row' of a CSR pattern, or -1.
__device__ __forceinline__ int64_t find_in_row(const int64_t *__restrict__ ptr,
                                               const int32_t *__restrict__ col, int row, int key) {
    int64_t lo = ptr[row], hi = ptr[row + 1];
    int64_t end = hi;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return (lo < end && col[lo] == key) ? lo : -1;
}

// For every entry (i, j) of pattern p: position in pattern q of (i, j), or of (j, i) if transposed.
__global__ void k_posmap(int n, const int64_t *__restrict__ pp, const int32_t *__restrict__ pc,
                         const int64_t *__restrict__ qp, const int32_t *__restrict__ qc, int transposed,
                         int64_t *__restrict__ out) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    int i = warp;
    for (int64_t e = pp[i] + lane; e < pp[i + 1]; e += 32) {
        int j = pc[e];
        out[e] = transposed ? find_in_row(qp, qc, j, i) : find_in_row(qp, qc, i, j);
    }
}

int geom_check(lsq_geom g, int r) {
    if (!g) return set_error(LSQ_ERR_INVALID_ARG, "null geometry handle");
    if (r < 0 || r >= g->n_ranges)
        return set_error(LSQ_ERR_INVALID_ARG, "range id " + std::to_string(r) + " out of bounds");
    return LSQ_OK;
}

int find_range(lsq_geom g, double R) {
    for (int r = 0; r < g->n_ranges; ++r)
        if (g->pats[r].R == R) return r;
    return -1;
}

int get_posmap(lsq_geom g, int p, int q, int transposed, const int64_t **out, cudaStream_t s) {
    auto key = std::make_tuple(p, q, transposed);
    auto it = g->posmaps.find(key);
    if (it == g->posmaps.end()) {
        DevBuf<int64_t> buf;
        LSQ_TRY(buf.alloc((size_t)g->pats[p].nnzb));
        if (g->n > 0 && g->pats[p].nnzb > 0) {
            int threads = 256;
            int blocks = (int)(((int64_t)g->n * 32 + threads - 1) / threads);
            note_launch();
            k_posmap<<<blocks, threads, 0, s>>>(g->n, g->pats[p].row_ptr.p, g->pats[p].col.p,
                                                g->pats[q].row_ptr.p, g->pats[q].col.p, transposed,
                                                buf.p);
            LSQ_CHECK_LAUNCH();
        }
        it = g->posmaps.emplace(key, std::move(buf)).first;
    }
    *out = it->second.p;
    return LSQ_OK;
}

int ensure_tmap(lsq_geom g, int r, cudaStream_t s) {
    Pattern &P = g->pats[r];
    if (P.tmap.p) return LSQ_OK;
    LSQ_TRY(P.tmap.alloc((size_t)P.nnzb));
    if (g->n > 0 && P.nnzb > 0) {
        int threads = 256;
        int blocks = (int)(((int64_t)g->n * 32 + threads - 1) / threads);
        note_launch();
        k_posmap<<<blocks, threads, 0, s>>>(g->n, P.row_ptr.p, P.col.p, P.row_ptr.p, P.col.p, 1,
                                            P.tmap.p);
        LSQ_CHECK_LAUNCH();
    }
    return LSQ_OK;
}

}  // namespace lsq

using namespace lsq;

extern "C" int lsq_last_error(char *buf, size_t len) {
    if (buf && len > 0) {
        size_t m = std::min(len - 1, g_last_msg.size());
        std::memcpy(buf, g_last_msg.data(), m);
        buf[m] = '\0';
    }
    return g_last_code;
}

extern "C" int lsq_version(void) { return 100; }

extern "C" int lsq_launch_count(int64_t *out) {
    clear_error();
    if (!out) return set_error(LSQ_ERR_INVALID_ARG, "out is null");
    *out = (int64_t)g_launch_count.load();
    return LSQ_OK;
}

extern "C" int lsq_build_neighbour_lists(const double *pos_dev, int n, const double *cell,
                                         const double *ranges, int nr, lsq_geom *out,
                                         void *stream) {
    clear_error();
    if (!out) return set_error(LSQ_ERR_INVALID_ARG, "out is null");
    *out = nullptr;
    if (n < 0 || n > (1 << 30)) return set_error(LSQ_ERR_INVALID_ARG, "n_atoms out of range");
    if (n > 0 && !pos_dev) return set_error(LSQ_ERR_INVALID_ARG, "pos_dev is null");
    if (!cell || !ranges) return set_error(LSQ_ERR_INVALID_ARG, "cell or ranges is null");
    if (nr < 1 || nr > kMaxRanges)
        return set_error(LSQ_ERR_INVALID_ARG, "n_ranges must be in [1, 16]");
    for (int c = 0; c < 3; ++c)
        if (!(cell[c] > 0.0) || !std::isfinite(cell[c]))
            return set_error(LSQ_ERR_INVALID_ARG, "cell lengths must be positive");
    double rmax = 0.0;
    for (int r = 0; r < nr; ++r) {
        if (!(ranges[r] > 0.0) || !std::isfinite(ranges[r]))
            return set_error(LSQ_ERR_INVALID_ARG, "ranges must be positive");
        rmax = std::max(rmax, ranges[r]);
    }
    cudaStream_t s = (cudaStream_t)stream;
    lsq_geom g = new lsq_geom_s();
    auto fail = [&](int rc) {
        delete g;
        return rc;
    };
    g->n = n;
    g->n_ranges = nr;
    g->n_sys = 1;
    g->sys_atom_off = {0, (int64_t)n};
    for (int c = 0; c < 3; ++c) g->cell[c] = cell[c];
    if (cudaGetDevice(&g->device) != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, "no device"));
    cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, g->device);
    g->smem_optin = (size_t)optin;
    g->pats.resize(nr);
    // load lsq_trace_static's fixed scratch array on this device now (geometry creation
    // allocates anyway), so that the allocation-free call never triggers the module load
    {
        const int prc = noalloc_prime();
        if (prc != LSQ_OK) return fail(prc);
    }

    CellGrid cg;
    int ncell = 1;
    for (int c = 0; c < 3; ++c) {
        int k = (int)std::floor(cell[c] / (rmax * (1.0 + 1e-6)));
        k = std::max(1, std::min(k, 1024));
        cg.nc[c] = k;
        cg.L[c] = cell[c];
        ncell *= k;
        if (k == 1) {
            cg.noff[c] = 1;
            cg.off[c][0] = 0;
        } else if (k == 2) {
            cg.noff[c] = 2;
            cg.off[c][0] = 0;
            cg.off[c][1] = 1;
        } else {
            cg.noff[c] = 3;
            cg.off[c][0] = -1;
            cg.off[c][1] = 0;
            cg.off[c][2] = 1;
        }
    }
    if (ncell > (1 << 24)) return fail(set_error(LSQ_ERR_UNSUPPORTED, "too many cells"));
    RangeSq rs;
    for (int r = 0; r < nr; ++r) {
        rs.r2[r] = ranges[r] * ranges[r];
        g->pats[r].R = ranges[r];
    }
    double r2max = rmax * rmax;

    int rc = g->pos.alloc((size_t)3 * std::max(n, 1));
    if (rc) return fail(rc);
    if (n > 0) {
        cudaError_t e = cudaMemcpyAsync(g->pos.p, pos_dev, sizeof(double) * 3 * n,
                                        cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, cudaGetErrorString(e)));
    }
    DevBuf<int> cid, ccount, cstart, catoms, maxc;
    DevBuf<int64_t> counts;
    if ((rc = cid.alloc(n)) || (rc = ccount.alloc(ncell)) || (rc = cstart.alloc(ncell + 1)) ||
        (rc = catoms.alloc(n)) || (rc = maxc.alloc(1)) || (rc = counts.alloc((size_t)nr * n)))
        return fail(rc);
    for (int r = 0; r < nr; ++r)
        if ((rc = g->pats[r].row_ptr.alloc((size_t)n + 1))) return fail(rc);
    cudaMemsetAsync(ccount.p, 0, sizeof(int) * ncell, s);
    cudaMemsetAsync(maxc.p, 0, sizeof(int), s);
    if (n > 0) {
        note_launch();
        k_cell_ids<<<(n + 255) / 256, 256, 0, s>>>(n, g->pos.p, cg, cid.p, ccount.p);
        note_launch();
        k_scan_single<int, int><<<1, 1024, 0, s>>>(ncell, ccount.p, cstart.p);
        cudaMemcpyAsync(ccount.p, cstart.p, sizeof(int) * ncell, cudaMemcpyDeviceToDevice, s);
        note_launch();
        k_cell_fill<<<(n + 255) / 256, 256, 0, s>>>(n, cid.p, ccount.p, catoms.p);
        int threads = 256;
        int blocks = (int)(((int64_t)n * 32 + threads - 1) / threads);
        note_launch();
        k_pair_count<<<blocks, threads, 0, s>>>(n, g->pos.p, cg, cstart.p, catoms.p, rs, nr, r2max,
                                                counts.p, maxc.p);
        for (int r = 0; r < nr; ++r) {
            note_launch();
            k_scan_single<int64_t, int64_t>
                <<<1, 1024, 0, s>>>(n, counts.p + (int64_t)r * n, g->pats[r].row_ptr.p);
        }
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, cudaGetErrorString(e)));
    } else {
        for (int r = 0; r < nr; ++r) cudaMemsetAsync(g->pats[r].row_ptr.p, 0, sizeof(int64_t), s);
    }
    int hmax = 0;
    std::vector<int64_t> tot(nr, 0);
    cudaMemcpyAsync(&hmax, maxc.p, sizeof(int), cudaMemcpyDeviceToHost, s);
    for (int r = 0; r < nr; ++r)
        cudaMemcpyAsync(&tot[r], g->pats[r].row_ptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, cudaGetErrorString(e)));
    if (hmax > kMaxRowCandidates)
        return fail(set_error(LSQ_ERR_UNSUPPORTED,
                              "an atom has " + std::to_string(hmax) +
                                  " neighbours within the largest range; the limit is 8192"));
    for (int r = 0; r < nr; ++r) {
        g->pats[r].nnzb = tot[r];
        g->pats[r].max_row = 0;
        if ((rc = g->pats[r].col.alloc((size_t)tot[r]))) return fail(rc);
    }
    if (n > 0) {
        std::vector<int64_t *> hp(nr);
        std::vector<int32_t *> hc(nr);
        for (int r = 0; r < nr; ++r) {
            hp[r] = g->pats[r].row_ptr.p;
            hc[r] = g->pats[r].col.p;
        }
        DevBuf<int64_t *> dp;
        DevBuf<int32_t *> dc;
        if ((rc = dp.alloc(nr)) || (rc = dc.alloc(nr))) return fail(rc);
        cudaMemcpyAsync(dp.p, hp.data(), sizeof(int64_t *) * nr, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(dc.p, hc.data(), sizeof(int32_t *) * nr, cudaMemcpyHostToDevice, s);
        int threads = 256;
        int m = 1;
        while (m < hmax) m <<= 1;
        size_t smem = sizeof(int) * (size_t)std::max(m, 1);
        cudaFuncSetAttribute(k_pair_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(int) * kMaxRowCandidates));
        note_launch();
        k_pair_fill<<<n, threads, smem, s>>>(n, g->pos.p, cg, cstart.p, catoms.p, rs, nr, r2max,
                                              dp.p, dc.p);
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, cudaGetErrorString(e)));
        // row lengths: max per pattern (host needs them for kernel limits)
        std::vector<int64_t> rp((size_t)n + 1);
        for (int r = 0; r < nr; ++r) {
            cudaMemcpyAsync(rp.data(), g->pats[r].row_ptr.p, sizeof(int64_t) * (n + 1),
                            cudaMemcpyDeviceToHost, s);
            e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, cudaGetErrorString(e)));
            int64_t mr = 0;
            for (int i = 0; i < n; ++i) mr = std::max(mr, rp[i + 1] - rp[i]);
            g->pats[r].max_row = (int)mr;
        }
    }
    if ((rc = reducer_ensure(g, 16))) return fail(rc);
    *out = g;
    return LSQ_OK;
}

extern "C" int lsq_geom_destroy(lsq_geom g) {
    clear_error();
    if (!g) return LSQ_OK;
    cudaDeviceSynchronize();
    if (g->red.host) cudaFreeHost(g->red.host);
    delete g;
    return LSQ_OK;
}

extern "C" int lsq_geom_info(lsq_geom g, int *n_atoms, int *n_ranges) {
    clear_error();
    if (!g) return set_error(LSQ_ERR_INVALID_ARG, "null geometry handle");
    if (n_atoms) *n_atoms = g->n;
    if (n_ranges) *n_ranges = g->n_ranges;
    return LSQ_OK;
}

extern "C" int lsq_pattern(lsq_geom g, int r, const int64_t **row_ptr, const int32_t **col,
                           int64_t *nnzb) {
    clear_error();
    LSQ_TRY(geom_check(g, r));
    if (row_ptr) *row_ptr = g->pats[r].row_ptr.p;
    if (col) *col = g->pats[r].col.p;
    if (nnzb) *nnzb = g->pats[r].nnzb;
    return LSQ_OK;
}

extern "C" int lsq_pattern_copy(lsq_geom g, int r, int64_t *row_ptr, int32_t *col, void *stream) {
    clear_error();
    LSQ_TRY(geom_check(g, r));
    cudaStream_t s = (cudaStream_t)stream;
    if (!row_ptr || (!col && g->pats[r].nnzb > 0))
        return set_error(LSQ_ERR_INVALID_ARG, "null output pointer");
    LSQ_CUDA_TRY(cudaMemcpyAsync(row_ptr, g->pats[r].row_ptr.p, sizeof(int64_t) * (g->n + 1),
                                 cudaMemcpyDeviceToDevice, s));
    if (g->pats[r].nnzb > 0)
        LSQ_CUDA_TRY(cudaMemcpyAsync(col, g->pats[r].col.p, sizeof(int32_t) * g->pats[r].nnzb,
                                     cudaMemcpyDeviceToDevice, s));
    return LSQ_OK;
}

// ---- block-diagonal concatenation of independent systems --------------------
namespace lsq {

__global__ void k_concat_rows(int n, const int64_t *__restrict__ rp, int64_t row_off, int64_t nnz_off,
                              int64_t *__restrict__ out_rp) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out_rp[row_off + i] = rp[i] + nnz_off;
}

__global__ void k_concat_cols(int64_t m, const int32_t *__restrict__ col, int atom_off,
                              int32_t *__restrict__ out_col) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e < m) out_col[e] = col[e] + atom_off;
}

__global__ void k_fill_sys(int n, int sys, int *__restrict__ atom_sys) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atom_sys[i] = sys;
}

}  // namespace lsq

extern "C" int lsq_geom_concat(int n_sys, const lsq_geom *geoms, lsq_geom *out, void *stream) {
    clear_error();
    if (!out || !geoms || n_sys < 1) return set_error(LSQ_ERR_INVALID_ARG, "bad arguments");
    *out = nullptr;
    const int nr = geoms[0] ? geoms[0]->n_ranges : 0;
    int64_t ntot = 0;
    for (int k = 0; k < n_sys; ++k) {
        if (!geoms[k]) return set_error(LSQ_ERR_INVALID_ARG, "null geometry in the list");
        if (geoms[k]->n_ranges != nr)
            return set_error(LSQ_ERR_INVALID_ARG, "all geometries must have the same ranges");
        for (int r = 0; r < nr; ++r)
            if (geoms[k]->pats[r].R != geoms[0]->pats[r].R)
                return set_error(LSQ_ERR_INVALID_ARG, "all geometries must have the same ranges");
        ntot += geoms[k]->n;
    }
    if (ntot > (1 << 30)) return set_error(LSQ_ERR_INVALID_ARG, "too many atoms");
    cudaStream_t s = (cudaStream_t)stream;
    lsq_geom g = new lsq_geom_s();
    auto fail = [&](int rc) {
        delete g;
        return rc;
    };
    g->n = (int)ntot;
    g->n_ranges = nr;
    g->device = geoms[0]->device;
    g->num_sms = geoms[0]->num_sms;
    g->smem_optin = geoms[0]->smem_optin;
    g->pats.resize(nr);
    g->n_sys = n_sys;
    g->sys_atom_off.assign((size_t)n_sys + 1, 0);
    for (int k = 0; k < n_sys; ++k) g->sys_atom_off[k + 1] = g->sys_atom_off[k] + geoms[k]->n;
    int rc;
    if ((rc = g->atom_sys.alloc((size_t)std::max<int64_t>(ntot, 1)))) return fail(rc);
    if ((rc = g->pos.alloc((size_t)3 * std::max<int64_t>(ntot, 1)))) return fail(rc);
    for (int k = 0; k < n_sys; ++k) {
        const int nk = geoms[k]->n;
        if (nk == 0) continue;
        note_launch();
        k_fill_sys<<<(nk + 255) / 256, 256, 0, s>>>(nk, k, g->atom_sys.p + g->sys_atom_off[k]);
        cudaMemcpyAsync(g->pos.p + 3 * g->sys_atom_off[k], geoms[k]->pos.p, sizeof(double) * 3 * nk,
                        cudaMemcpyDeviceToDevice, s);
    }
    for (int r = 0; r < nr; ++r) {
        Pattern &P = g->pats[r];
        P.R = geoms[0]->pats[r].R;
        int64_t nnz = 0;
        int mr = 0;
        for (int k = 0; k < n_sys; ++k) {
            nnz += geoms[k]->pats[r].nnzb;
            mr = std::max(mr, geoms[k]->pats[r].max_row);
        }
        P.nnzb = nnz;
        P.max_row = mr;
        if ((rc = P.row_ptr.alloc((size_t)ntot + 1)) || (rc = P.col.alloc((size_t)std::max<int64_t>(nnz, 1))))
            return fail(rc);
        int64_t off = 0;
        for (int k = 0; k < n_sys; ++k) {
            const Pattern &Q = geoms[k]->pats[r];
            const int nk = geoms[k]->n;
            if (nk > 0) {
                note_launch();
                k_concat_rows<<<(nk + 255) / 256, 256, 0, s>>>(nk, Q.row_ptr.p, g->sys_atom_off[k], off,
                                                               P.row_ptr.p);
            }
            if (Q.nnzb > 0) {
                note_launch();
                k_concat_cols<<<(int)((Q.nnzb + 255) / 256), 256, 0, s>>>(Q.nnzb, Q.col.p,
                                                                          (int)g->sys_atom_off[k],
                                                                          P.col.p + off);
            }
            off += Q.nnzb;
        }
        cudaMemcpyAsync(P.row_ptr.p + ntot, &P.nnzb, sizeof(int64_t), cudaMemcpyHostToDevice, s);
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return fail(set_error(LSQ_ERR_CUDA, cudaGetErrorString(e)));
    if ((rc = reducer_ensure(g, 16))) return fail(rc);
    *out = g;
    return LSQ_OK;
}

extern "C" int lsq_geom_systems(lsq_geom g, int *n_sys, int64_t *atom_off_host) {
    clear_error();
    if (!g) return set_error(LSQ_ERR_INVALID_ARG, "null geometry handle");
    if (n_sys) *n_sys = g->n_sys;
    if (atom_off_host)
        for (int k = 0; k <= g->n_sys; ++k) atom_off_host[k] = g->sys_atom_off[k];
    return LSQ_OK;
}
