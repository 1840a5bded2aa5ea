// Tensor-core form of the truncated 4 x 4 block product (precision LSQ_TF32X3).
//
// Sec. 2.3.2 of the paper: every product of the linear-scaling method is restricted to the
// range of its result, C_ij = sum_k A_ik B_kj over the stored blocks (i, j) of C.  Here the
// 4 x 4 blocks are contracted on the tensor cores (tcgen05.mma, kind::tf32, FP32
// accumulation in tensor memory):
//
//  * Split TF32 operands.  Every float32 value v is held as hi = tf32(v) and
//    lo = tf32(v - hi), so hi + lo carries v to 22 bits.  A block is one 128-byte unit: the
//    4 x 4 hi values (row-major), then the 4 x 4 lo values.
//  * Tiles.  Atoms i are taken in groups of 8 (one diamond cell in cell-ordered systems).
//    The atoms j of the group's rows of C are cut into tiles of 16, and each tile has one
//    list of atoms k: the union of the group's rows of op(A), restricted to atoms that the
//    tile's rows of op(B)^T hold (padded to a multiple of 16).  A tile is one accumulator of
//    M = 128 rows (16 j x {hi, lo} x 4 rows c of X_jk = (B_kj)^T) by N = 64 columns
//    (8 i x {hi, lo} x 4 rows r of A_ik), and one MMA takes K = 8 (two atoms k x 4).  The
//    {hi, lo} x {hi, lo} cross terms land in separate rows and columns and are summed in the
//    epilogue: one pass gives hi.hi + hi.lo + lo.hi + lo.lo.
//  * Gathers.  The blocks of a stage (16 k of the list for the 16 rows j and the 8 rows i)
//    are copied into shared memory by 16-byte asynchronous copies (cp.async), eight lanes
//    per 128-byte block, so one warp instruction moves four whole cache lines; the lanes of
//    a block a row does not hold store zeros instead (no L2 request), so every stage lands
//    whole.  Each copying thread arrives on the stage's mbarrier twice: after its stores of
//    zeros (with a proxy fence, as the MMAs read through the async proxy) and when its copies
//    complete.  The block indices a CTA gathers are laid out by the plan as one stream of
//    stage records, read four stages ahead, so no copy waits on an index load.  The kernel
//    is bound by the rate of these gathers (about 10 TB/s of scattered 128-byte lines), not
//    by DRAM.  (Bulk copies of runs of consecutive blocks were measured first: at the ~4
//    blocks a run averages, their request rate, not the bytes, bounded the kernel.)
//  * Roles.  Six warps issue the copies through a ring of stages, one thread issues the
//    MMAs, four warps read the accumulator (tcgen05.ld) and write the blocks of C the plan
//    keeps.  The tensor core's float32 additions truncate, which biases long sums, so each
//    stage (8 MMAs) accumulates into a fresh accumulator of a ring of four in tensor memory
//    and the epilogue adds the stages in float32 with rounding to nearest.  Every wait on an
//    mbarrier is bounded: past the limit the kernel records an error code in a device word,
//    stops issuing work, waits (bounded) for its copies and MMAs in flight, frees its tensor
//    memory and returns.
//
// The plan (which blocks to gather, where to write) is built on the GPU once per geometry
// and product, like the FMA path's plan.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <vector>

#include "lsq_internal.h"

namespace lsq {
namespace {

constexpr int kG = 8;                         // atoms i per group
constexpr int kJT = 16;                       // atoms j per tile
constexpr int kKS = 16;                       // atoms k per pipeline stage
constexpr int kStages = 4;                    // stages in the ring
constexpr int kUnit = 128;                    // bytes of a split block (hi 64, lo 64)
constexpr int kRows = kJT + kG;               // gathered rows per stage
constexpr int kPanelX = kJT * kKS * kUnit;    // X rows of a stage (M side), 32 KB
constexpr int kStageBytes = kRows * kKS * kUnit;  // 48 KB
constexpr int kN = 8 * kG;                    // accumulator columns of a tile
constexpr int kPartials = 4;                  // ring of per-stage accumulators in tensor memory
constexpr int kTmemCols = kPartials * kN;
constexpr int kCopyWarps = 6;                 // warps 0-5 copy (4 rows of a stage each)
constexpr int kMmaWarp = 6;                   // one thread of warp 6 issues the MMAs
constexpr int kThreads = 352;                 // warps 7-10 read the accumulator
constexpr int kRec = kRows * kKS;             // entries of a stage record
constexpr uint16_t kAbsent = 0xffff;
constexpr unsigned long long kWaitNs = 1000000000ull;  // bound of every mbarrier wait (1 s)

// Index of (row r, block kk) in a stage record.  Rows come in six groups of four, one per
// copying warp; lane l of warp w loads entries 64 w + 2 l and 64 w + 2 l + 1 and, for copy
// instruction q (row 4 w + q / 4, block 4 (q % 4) + l / 8), finds its block index in lane
// 8 (l / 8) + q / 2, entry q % 2.
__host__ __device__ constexpr int rec_index(int r, int kk) {
    return 64 * (r >> 2) + 16 * (kk & 3) + 2 * ((4 * (r & 3) + (kk >> 2)) >> 1) + ((4 * (r & 3) + (kk >> 2)) & 1);
}

__device__ __forceinline__ bool tri_skip_tc(int tri, int i, int j) {
    return tri == 1 ? j < i : (tri == 2 ? j > i : false);
}

// ---- PTX wrappers ---------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity; false if the CTA aborted or the wait ran past
// its limit (which then records `code` in *err and raises the abort flag).
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int *abort_flag, int *err,
                                          int code, unsigned long long limit_ns) {
    const unsigned long long t0 = globaltimer();
    while (!mbar_try(bar, parity)) {
        if (*abort_flag) return false;
        if (globaltimer() - t0 > limit_ns) {
            atomicCAS(err, 0, code);
            *abort_flag = 1;
            return false;
        }
    }
    return true;
}
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
// Arrives on the mbarrier once every cp.async this thread issued before has completed
// (the arrival counts against the count the barrier was initialised with).
__device__ __forceinline__ void cp_async_arrive(uint32_t bar) {
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void st_shared_zero16(uint32_t dst) {
    asm volatile("st.shared.v4.u32 [%0], {%1, %1, %1, %1};" ::"r"(dst), "r"(0u) : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, K-major without swizzle: core matrices of 8 rows x 16
// bytes (rows 16 bytes apart); lbo = bytes between core matrices along K, sbo = bytes
// between groups of 8 rows along M (or N).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3fffu);
    d |= (uint64_t)((lbo >> 4) & 0x3fffu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3fffu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version of the tcgen05 family
    return d;                // base offset 0, no swizzle
}

// Instruction descriptor of kind::tf32: D float32, A and B tf32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
        "%14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// ---- split TF32 operands -------------------------------------------------------------
// Round to the nearest tf32 value (10 fraction bits), halfway cases away from zero: add
// half a unit of the 11th bit to the magnitude bits, then clear the 13 low bits.
__device__ __forceinline__ float tf32_round(float v) {
    return __uint_as_float((__float_as_uint(v) + 0x1000u) & 0xffffe000u);
}

// Unit p of out: hi and lo of block p of X (MODE 0), of X^T read through the transpose map tm
// (MODE 1; block (i, j) of X^T is (X_ji)^T), or of X + X^T (MODE 2, X on a symmetric pattern;
// the sum rounded once in float32, as a separate symmetric sum would).  v - hi is exact in
// float32.
template <int MODE>
__global__ void k_split_tf32(int64_t nnzb, const int64_t *__restrict__ tm, const float *__restrict__ X,
                             float *__restrict__ out) {
    const int64_t m = nnzb * 16;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t p = e >> 4;
        const int rc = (int)(e & 15);
        const float v = MODE == 0   ? X[e]
                        : MODE == 1 ? X[16 * tm[p] + (rc & 3) * 4 + (rc >> 2)]
                                    : X[e] + X[16 * tm[p] + (rc & 3) * 4 + (rc >> 2)];
        const float hi = tf32_round(v);
        const float lo = tf32_round(v - hi);
        out[32 * p + rc] = hi;
        out[32 * p + 16 + rc] = lo;
    }
}

// ---- plan ------------------------------------------------------------------------------
// Number of entries of pos[0, m) that name a block (>= 0).
__global__ void k_count_present(int64_t m, const int32_t *__restrict__ pos, unsigned long long *__restrict__ out) {
    unsigned long long c = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < m; e += (int64_t)gridDim.x * blockDim.x)
        c += pos[e] >= 0 ? 1ull : 0ull;
    for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

struct TcBuild {
    int n, ngroups, upper;
    const int64_t *a_ptr, *x_ptr, *c_ptr;
    const int32_t *a_col, *x_col, *c_col;
    const int32_t *g_toff;        // [ngroups + 1] first tile of each group
    int32_t *tile_j;              // [16 ntiles]
    int32_t *tile_nk;             // [ntiles]
    const int64_t *tile_posoff;   // [ntiles]
    const int64_t *tile_koff;     // [ntiles] start of the tile's k-list in klist
    int32_t *klist;               // scratch
    int32_t *pos;
    int32_t *cpos;
};

__device__ __forceinline__ void clear_bits(uint32_t *bm, int W) {
    for (int w = threadIdx.x; w < W; w += blockDim.x) bm[w] = 0u;
}

// bm |= the columns of row r (those within the triangle tri of row r when tri > 0).
__device__ __forceinline__ void or_row(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, int r,
                                       int tri, uint32_t *bm) {
    for (int64_t q = ptr[r] + threadIdx.x; q < ptr[r + 1]; q += blockDim.x) {
        const int c = col[q];
        if (!tri_skip_tc(tri, r, c)) atomicOr(&bm[c >> 5], 1u << (c & 31));
    }
}

// Sum of v over the block (every thread receives it).  sh: 32 ints of shared memory.
__device__ int block_sum(int v, int *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    int t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    __syncthreads();
    return t;
}

// Exclusive prefix sum of v over the block; *total receives the sum.  sh: 32 ints.
__device__ int block_scan_excl(int v, int *total, int *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    const int before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    *total = sh[nw - 1];
    __syncthreads();
    return before;
}

// Writes the set bits of bm[0..W) in ascending order to out[0..); returns their number.
__device__ int compact_bits(const uint32_t *bm, int W, int32_t *out, int *sh) {
    const int chunk = (W + (int)blockDim.x - 1) / (int)blockDim.x;
    const int w0 = min(W, (int)threadIdx.x * chunk), w1 = min(W, w0 + chunk);
    int v = 0;
    for (int w = w0; w < w1; ++w) v += __popc(bm[w]);
    int total;
    int r = block_scan_excl(v, &total, sh);
    for (int w = w0; w < w1; ++w) {
        uint32_t bits = bm[w];
        while (bits) {
            const int b = __ffs(bits) - 1;
            bits &= bits - 1u;
            out[r++] = 32 * w + b;
        }
    }
    return total;
}

// Pass 1: tiles of each group (its atoms j: the union of its rows of C within the triangle).
__global__ void __launch_bounds__(512) k_tc_groups(TcBuild a, int32_t *__restrict__ nt_out) {
    extern __shared__ __align__(16) uint32_t jb[];
    __shared__ int sh[32];
    const int W = (a.n + 31) >> 5;
    for (int g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
        clear_bits(jb, W);
        __syncthreads();
        for (int i = kG * g; i < min(kG * g + kG, a.n); ++i) or_row(a.c_ptr, a.c_col, i, a.upper, jb);
        __syncthreads();
        int c = 0;
        for (int w = threadIdx.x; w < W; w += blockDim.x) c += __popc(jb[w]);
        c = block_sum(c, sh);
        if (threadIdx.x == 0) nt_out[g] = (c + kJT - 1) / kJT;
        __syncthreads();
    }
}

// Pass 2: atoms j of each tile and the length of its k-list (a multiple of 16).
__global__ void __launch_bounds__(512) k_tc_tiles(TcBuild a) {
    extern __shared__ __align__(16) uint32_t bm[];
    __shared__ int sh[32];
    const int W = (a.n + 31) >> 5;
    uint32_t *kb = bm, *jb = bm + W, *tb = bm + 2 * W;
    for (int g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
        const int i0 = kG * g, i1 = min(i0 + kG, a.n);
        clear_bits(kb, 2 * W);
        __syncthreads();
        for (int i = i0; i < i1; ++i) {
            or_row(a.a_ptr, a.a_col, i, 0, kb);
            or_row(a.c_ptr, a.c_col, i, a.upper, jb);
        }
        __syncthreads();
        const int t0 = a.g_toff[g], nt = a.g_toff[g + 1] - t0;
        const int cj = compact_bits(jb, W, a.tile_j + (int64_t)kJT * t0, sh);
        for (int m = cj + threadIdx.x; m < kJT * nt; m += blockDim.x) a.tile_j[(int64_t)kJT * t0 + m] = -1;
        __syncthreads();
        for (int t = t0; t < t0 + nt; ++t) {
            clear_bits(tb, W);
            __syncthreads();
            for (int jj = 0; jj < kJT; ++jj) {
                const int j = a.tile_j[(int64_t)kJT * t + jj];
                if (j >= 0) or_row(a.x_ptr, a.x_col, j, 0, tb);
            }
            __syncthreads();
            int c = 0;
            for (int w = threadIdx.x; w < W; w += blockDim.x) c += __popc(tb[w] & kb[w]);
            c = block_sum(c, sh);
            if (threadIdx.x == 0) a.tile_nk[t] = max(kKS, (c + kKS - 1) / kKS * kKS);
            __syncthreads();
        }
    }
}

// map[col] = offset of col in row r (set) or kAbsent (unset), for one row at a time.
__device__ __forceinline__ void map_row(const int64_t *__restrict__ ptr, const int32_t *__restrict__ col, int r,
                                        uint16_t *map, bool set) {
    const int64_t p0 = ptr[r], p1 = ptr[r + 1];
    for (int64_t q = p0 + threadIdx.x; q < p1; q += blockDim.x) map[col[q]] = set ? (uint16_t)(q - p0) : kAbsent;
}

// Pass 3: each tile's k-list, the index of each listed block in the tile's 24 rows (stage
// records), and the positions in C of the blocks (i, j) the tile writes.
__global__ void __launch_bounds__(512) k_tc_fill(TcBuild a) {
    extern __shared__ __align__(16) uint32_t bm[];
    __shared__ int sh[32];
    const int W = (a.n + 31) >> 5;
    uint32_t *kb = bm, *tb = bm + W;
    uint16_t *map = reinterpret_cast<uint16_t *>(bm + 2 * W);
    for (int e = threadIdx.x; e < a.n; e += blockDim.x) map[e] = kAbsent;
    __syncthreads();
    for (int g = blockIdx.x; g < a.ngroups; g += gridDim.x) {
        const int i0 = kG * g, i1 = min(i0 + kG, a.n);
        const int t0 = a.g_toff[g], nt = a.g_toff[g + 1] - t0;
        clear_bits(kb, W);
        __syncthreads();
        for (int i = i0; i < i1; ++i) or_row(a.a_ptr, a.a_col, i, 0, kb);
        __syncthreads();
        for (int t = t0; t < t0 + nt; ++t) {
            clear_bits(tb, W);
            __syncthreads();
            for (int jj = 0; jj < kJT; ++jj) {
                const int j = a.tile_j[(int64_t)kJT * t + jj];
                if (j >= 0) or_row(a.x_ptr, a.x_col, j, 0, tb);
            }
            __syncthreads();
            for (int w = threadIdx.x; w < W; w += blockDim.x) tb[w] &= kb[w];
            __syncthreads();
            const int nk = a.tile_nk[t];
            const int64_t po = a.tile_posoff[t];
            int32_t *kl = a.klist + a.tile_koff[t];
            const int ck = compact_bits(tb, W, kl, sh);
            for (int m = ck + threadIdx.x; m < nk; m += blockDim.x) kl[m] = -1;
            __syncthreads();
            for (int r = 0; r < kRows; ++r) {
                int row;
                const int64_t *ptr;
                const int32_t *col;
                if (r < kJT) {
                    row = a.tile_j[(int64_t)kJT * t + r];
                    ptr = a.x_ptr;
                    col = a.x_col;
                } else {
                    row = i0 + r - kJT < a.n ? i0 + r - kJT : -1;
                    ptr = a.a_ptr;
                    col = a.a_col;
                }
                const int64_t row0 = row >= 0 ? ptr[row] : 0;
                if (row >= 0) map_row(ptr, col, row, map, true);
                __syncthreads();
                for (int m = threadIdx.x; m < nk; m += blockDim.x) {
                    const int k = kl[m];
                    const uint16_t o = (row >= 0 && k >= 0) ? map[k] : kAbsent;
                    a.pos[po + (int64_t)kRec * (m / kKS) + rec_index(r, m % kKS)] =
                        o == kAbsent ? -1 : (int32_t)(row0 + o);
                }
                __syncthreads();
                if (row >= 0) map_row(ptr, col, row, map, false);
                __syncthreads();
            }
        }
        for (int rr = 0; rr < kG; ++rr) {
            const int i = i0 + rr;
            if (i < i1) map_row(a.c_ptr, a.c_col, i, map, true);
            __syncthreads();
            for (int m = threadIdx.x; m < kJT * nt; m += blockDim.x) {
                const int t = t0 + m / kJT, jj = m % kJT;
                const int j = a.tile_j[(int64_t)kJT * t0 + m];
                int32_t v = -1;
                if (i < i1 && j >= 0 && !tri_skip_tc(a.upper, i, j) && map[j] != kAbsent)
                    v = (int32_t)(a.c_ptr[i] + map[j]);
                a.cpos[(int64_t)128 * t + kJT * rr + jj] = v;
            }
            __syncthreads();
            if (i < i1) map_row(a.c_ptr, a.c_col, i, map, false);
            __syncthreads();
        }
    }
}

// ---- the product -----------------------------------------------------------------------
struct TcArgs {
    int ntiles;
    const int32_t *tile_nk, *cpos, *cta_stages;
    const int64_t *tile_posoff;
    const int32_t *pos;
    const char *As, *Xs;  // split units of op(A) and of X = op(B)^T
    float *C;
    const int64_t *c_tm;  // transpose map of C's pattern: also write C_ji = C_ij^T (or null)
    float alpha, beta;
    int *err;
    unsigned long long wait_ns;  // bound of the pipeline waits (the final drain keeps kWaitNs)
};

__global__ void __launch_bounds__(kThreads, 1) k_tc_product(TcArgs p) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(smem + kStages * kStageBytes);
    // bars: full[kStages], empty[kStages], tfull[kPartials], tempty[kPartials], drain[1]
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(bars + 2 * kStages + 2 * kPartials + 1);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bar0 = smem_u32(bars);
    auto full = [&](int s) { return bar0 + 8u * s; };
    auto empty = [&](int s) { return bar0 + 8u * (kStages + s); };
    auto tfull = [&](int b) { return bar0 + 8u * (2 * kStages + b); };
    auto tempty = [&](int b) { return bar0 + 8u * (2 * kStages + kPartials + b); };
    const uint32_t drain = bar0 + 8u * (2 * kStages + 2 * kPartials);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            // per copying thread and stage: one arrival after its stores of zeros, one when its
            // copies have landed
            mbar_init(full(s), 2 * 32 * kCopyWarps);
            mbar_init(empty(s), 1);
        }
        for (int b = 0; b < kPartials; ++b) {
            mbar_init(tfull(b), 1);
            mbar_init(tempty(b), 4);
        }
        mbar_init(drain, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kCopyWarps) {
        // ---- copies.  Warp w fills rows 4w .. 4w + 3 of every stage (rows 0-15: atoms j of the
        // tile, rows of X; 16-23: atoms i of the group, rows of op(A)).  One instruction moves
        // four blocks: lane l copies 16-byte chunk l % 8 of block 4 (q % 4) + l / 8 of row
        // 4 w + q / 4 (q = 0..15).  The CTA's stage records are read four stages ahead.
        const char *arr = warp < 4 ? p.Xs : p.As;
        const int sub = lane >> 3;
        const int S = p.cta_stages[blockIdx.x];
        const int32_t *rec = p.pos + p.tile_posoff[blockIdx.x] + 64 * warp + 2 * lane;
        auto ld = [&](int st) -> int2 {
            return st < S ? *reinterpret_cast<const int2 *>(rec + (int64_t)kRec * st) : make_int2(-1, -1);
        };
        int2 p0 = ld(0), p1 = ld(1), p2 = ld(2), p3 = ld(3);
        const uint32_t dlane = (uint32_t)(4 * warp * kKS * kUnit + 16 * (lane & 7));
        for (int st = 0; st < S; ++st) {
            const int2 p4 = ld(st + 4);
            const int slot = st % kStages;
            const uint32_t ph = (uint32_t)(st / kStages) & 1u;
            bool ok = mbar_wait(empty(slot), ph ^ 1u, abort_flag, p.err, 1, p.wait_ns);
            ok = __all_sync(0xffffffffu, ok);
            if (!ok) break;
            const uint32_t dst0 = sbase + (uint32_t)slot * kStageBytes + dlane;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                const int v = __shfl_sync(0xffffffffu, (q & 1) ? p0.y : p0.x, 8 * sub + (q >> 1));
                const uint32_t dst = dst0 + (uint32_t)((q >> 2) * (kKS * kUnit) + (4 * (q & 3) + sub) * kUnit);
                if (v < 0)
                    st_shared_zero16(dst);  // a block the row does not hold
                else
                    cp_async16(dst, arr + (int64_t)kUnit * v + 16 * (lane & 7));
            }
            // the zeros are generic-proxy stores that the MMAs read through the async proxy
            fence_proxy_async();
            mbar_arrive(full(slot));
            cp_async_arrive(full(slot));
            p0 = p1;
            p1 = p2;
            p2 = p3;
            p3 = p4;
        }
        // every copy of this thread has landed before the CTA exits
        asm volatile("cp.async.wait_all;" ::: "memory");
    } else if (warp == kMmaWarp) {
        if (lane == 0) {
            // ---- MMAs: per stage 8 of M = 128, N = 64, K = 8 (two atoms k), into a fresh
            // accumulator of the ring (the tensor core's float32 additions truncate, so sums
            // are kept to one stage there and the stages are added by the epilogue)
            constexpr uint32_t idesc = idesc_tf32(128, kN);
            int it = 0;
            bool ok = true;
            for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
                const int nk = p.tile_nk[t];
                for (int k0 = 0; k0 < nk; k0 += kKS, ++it) {
                    const int buf = it % kPartials;
                    ok = mbar_wait(tempty(buf), ((uint32_t)(it / kPartials) & 1u) ^ 1u, abort_flag, p.err, 3, p.wait_ns);
                    if (!ok) break;
                    const int slot = it % kStages;
                    ok = mbar_wait(full(slot), (uint32_t)(it / kStages) & 1u, abort_flag, p.err, 2, p.wait_ns);
                    if (!ok) break;
                    // the stage was written by cp.async (generic proxy); the MMAs read it
                    // through the async proxy
                    fence_proxy_async();
                    tc_fence_after();
                    const uint32_t d = tmem + (uint32_t)(buf * kN);
                    const uint32_t sa = sbase + (uint32_t)slot * kStageBytes, sb = sa + kPanelX;
#pragma unroll
                    for (int kk = 0; kk < kKS; kk += 2) {
                        const uint64_t ad = sdesc(sa + kk * kUnit, kUnit, kKS * kUnit);
                        const uint64_t bd = sdesc(sb + kk * kUnit, kUnit, kKS * kUnit);
                        mma_tf32(d, ad, bd, idesc, kk > 0 ? 1u : 0u);
                    }
                    mma_commit(empty(slot));
                    mma_commit(tfull(buf));
                }
            }
            // every MMA issued has completed before tensor memory is released
            mma_commit(drain);
            const unsigned long long t0 = globaltimer();
            while (!mbar_try(drain, 0u))
                if (globaltimer() - t0 > kWaitNs) {
                    atomicCAS(p.err, 0, 6);
                    break;
                }
        }
    } else {
        // ---- epilogue: thread row m = 8 jj + 4 h + c of the accumulator.  The stages' partial
        // accumulators of a tile are added here in float32 (rounded to nearest), then the
        // {hi, lo} cross terms are combined and the blocks of C written.
        const int sub = warp & 3;
        const int m = 32 * sub + lane;
        const int jj = m >> 3, h = (m >> 2) & 1, c = m & 3;
        const uint32_t tlane = tmem + ((uint32_t)(32 * sub) << 16);
        int it = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < p.ntiles && ok; t += gridDim.x) {
            const int nst = p.tile_nk[t] / kKS;
            int32_t cp[kG];
#pragma unroll
            for (int ii = 0; ii < kG; ++ii) cp[ii] = p.cpos[(int64_t)128 * t + kJT * ii + jj];
            float acc[kN];
#pragma unroll
            for (int e = 0; e < kN; ++e) acc[e] = 0.f;
            for (int st = 0; st < nst; ++st, ++it) {
                const int buf = it % kPartials;
                ok = mbar_wait(tfull(buf), (uint32_t)(it / kPartials) & 1u, abort_flag, p.err, 4, p.wait_ns);
                ok = __all_sync(0xffffffffu, ok);
                if (!ok) break;
                tc_fence_after();
                // all four loads of the stage in flight before one wait
                uint32_t v[kN / 16][16];
#pragma unroll
                for (int q = 0; q < kN / 16; ++q) tmem_ld16(tlane + (uint32_t)(buf * kN + 16 * q), v[q]);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < kN / 16; ++q)
#pragma unroll
                    for (int e = 0; e < 16; ++e) acc[16 * q + e] += __uint_as_float(v[q][e]);
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(tempty(buf));
            }
            if (!ok) break;
            // columns 8 ii + 4 h' + r: atom i = ii, hi (h' = 0) or lo (h' = 1) rows r of A_ik
            float s[kG][4];
#pragma unroll
            for (int ii = 0; ii < kG; ++ii)
#pragma unroll
                for (int r = 0; r < 4; ++r) s[ii][r] = acc[8 * ii + r] + acc[8 * ii + 4 + r];
            // rows hi and lo of the same (j, c) are lanes l and l + 4
#pragma unroll
            for (int ii = 0; ii < kG; ++ii)
#pragma unroll
                for (int r = 0; r < 4; ++r) s[ii][r] += __shfl_down_sync(0xffffffffu, s[ii][r], 4);
            if (h == 0) {
#pragma unroll
                for (int ii = 0; ii < kG; ++ii) {
                    if (cp[ii] < 0) continue;
                    float *dst = p.C + 16 * (int64_t)cp[ii] + c;
                    float w[4];
#pragma unroll
                    for (int r = 0; r < 4; ++r) {
                        const float v = p.alpha * s[ii][r];
                        w[r] = p.beta != 0.f ? fmaf(p.beta, dst[4 * r], v) : v;
                        dst[4 * r] = w[r];
                    }
                    if (p.c_tm) {
                        // symmetric result: row c of the mirrored block C_ji is column c of C_ij
                        const int64_t q = p.c_tm[cp[ii]];
                        if (q != cp[ii]) {
                            float *m = p.C + 16 * q + 4 * c;
#pragma unroll
                            for (int r = 0; r < 4; ++r) m[r] = w[r];
                        }
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

constexpr size_t kSmemBytes = (size_t)kStages * kStageBytes + 256;

}  // namespace

int tc_plan_get(lsq_geom g, int ra, int rb, int rc, int upper, TcPlan **out, cudaStream_t s) {
    auto key = std::make_tuple(ra, rb, rc + 1000 * upper);
    auto f = g->tcplans.find(key);
    if (f != g->tcplans.end()) {
        *out = &f->second;
        return LSQ_OK;
    }
    const Pattern &PA = g->pats[ra], &PX = g->pats[rb], &PC = g->pats[rc];
    const int n = g->n;
    if (PA.max_row >= 65535 || PX.max_row >= 65535 || PC.max_row >= 65535)
        return set_error(LSQ_ERR_UNSUPPORTED, "row too long for a tensor-core plan");
    if (PC.nnzb >= ((int64_t)1 << 31) || PA.nnzb >= ((int64_t)1 << 31) || PX.nnzb >= ((int64_t)1 << 31))
        return set_error(LSQ_ERR_UNSUPPORTED, "matrix too large for a tensor-core plan (2^31 blocks)");
    const int W = (n + 31) / 32;
    const size_t smem_tiles = (size_t)3 * W * sizeof(uint32_t);
    const size_t smem_fill = (size_t)2 * W * sizeof(uint32_t) + (size_t)n * sizeof(uint16_t) + 16;
    if (std::max(smem_tiles, smem_fill) + 1024 > g->smem_optin)
        return set_error(LSQ_ERR_UNSUPPORTED, "too many atoms for the tensor-core plan builder");
    TcPlan p;
    p.upper = upper;
    p.ngroups = (n + kG - 1) / kG;
    const int ng = p.ngroups;
    TcBuild a{};
    a.n = n;
    a.ngroups = ng;
    a.upper = upper;
    a.a_ptr = PA.row_ptr.p;
    a.a_col = PA.col.p;
    a.x_ptr = PX.row_ptr.p;
    a.x_col = PX.col.p;
    a.c_ptr = PC.row_ptr.p;
    a.c_col = PC.col.p;
    const int grid = std::max(1, std::min(ng, g->num_sms * 2));
    // pass 1: tiles per group
    std::vector<int32_t> nt(std::max(ng, 1), 0), toff(ng + 1, 0);
    if (ng > 0) {
        DevBuf<int32_t> nt_d;
        LSQ_TRY(nt_d.alloc(ng));
        LSQ_CUDA_TRY(cudaFuncSetAttribute(k_tc_groups, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)(W * sizeof(uint32_t))));
        note_launch();
        k_tc_groups<<<grid, 512, W * sizeof(uint32_t), s>>>(a, nt_d.p);
        LSQ_CHECK_LAUNCH();
        LSQ_CUDA_TRY(cudaMemcpyAsync(nt.data(), nt_d.p, sizeof(int32_t) * ng, cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    }
    for (int q = 0; q < ng; ++q) toff[q + 1] = toff[q] + nt[q];
    p.ntiles = toff[ng];
    const int T = std::max(p.ntiles, 1);
    DevBuf<int32_t> toff_d, tile_j;
    LSQ_TRY(toff_d.alloc(ng + 1));
    LSQ_TRY(tile_j.alloc((size_t)kJT * T));
    LSQ_TRY(p.tile_nk.alloc(T));
    LSQ_TRY(p.tile_posoff.alloc(T));
    LSQ_TRY(p.cpos.alloc((size_t)128 * T));
    std::vector<int32_t> tnk(T, 0);
    std::vector<int64_t> tpo(T, 0), tko(T, 0);
    int64_t total = 0, klen = 0;
    p.grid = std::max(1, std::min(p.ntiles, g->num_sms));
    std::vector<int32_t> cst(p.grid, 0);
    if (p.ntiles > 0) {
        LSQ_CUDA_TRY(cudaMemcpyAsync(toff_d.p, toff.data(), sizeof(int32_t) * (ng + 1), cudaMemcpyHostToDevice, s));
        a.g_toff = toff_d.p;
        a.tile_j = tile_j.p;
        a.tile_nk = p.tile_nk.p;
        // pass 2: atoms j of the tiles, k-list lengths
        LSQ_CUDA_TRY(cudaFuncSetAttribute(k_tc_tiles, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_tiles));
        note_launch();
        k_tc_tiles<<<grid, 512, smem_tiles, s>>>(a);
        LSQ_CHECK_LAUNCH();
        LSQ_CUDA_TRY(cudaMemcpyAsync(tnk.data(), p.tile_nk.p, sizeof(int32_t) * p.ntiles, cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));
        // tile t runs on CTA t % grid, after the CTA's earlier tiles: its stage records follow
        // theirs in the CTA's stream
        for (int c = 0; c < p.grid; ++c)
            for (int t = c; t < p.ntiles; t += p.grid) {
                tpo[t] = total;
                total += (int64_t)kRec * (tnk[t] / kKS);
                cst[c] += tnk[t] / kKS;
            }
        for (int t = 0; t < p.ntiles; ++t) {
            tko[t] = klen;
            klen += tnk[t];
            p.units += (int64_t)kRows * tnk[t];
            p.dense_triples += (int64_t)kG * kJT * tnk[t];
        }
    }
    LSQ_TRY(p.pos.alloc(std::max<int64_t>(total, 16)));
    LSQ_TRY(p.cta_stages.alloc(p.grid));
    LSQ_CUDA_TRY(cudaMemcpyAsync(p.cta_stages.p, cst.data(), sizeof(int32_t) * p.grid, cudaMemcpyHostToDevice, s));
    if (p.ntiles > 0) {
        DevBuf<int32_t> klist;
        DevBuf<int64_t> tko_d;
        LSQ_TRY(klist.alloc(std::max<int64_t>(klen, 1)));
        LSQ_TRY(tko_d.alloc(p.ntiles));
        LSQ_CUDA_TRY(cudaMemcpyAsync(p.tile_posoff.p, tpo.data(), sizeof(int64_t) * p.ntiles, cudaMemcpyHostToDevice, s));
        LSQ_CUDA_TRY(cudaMemcpyAsync(tko_d.p, tko.data(), sizeof(int64_t) * p.ntiles, cudaMemcpyHostToDevice, s));
        a.tile_posoff = p.tile_posoff.p;
        a.tile_koff = tko_d.p;
        a.klist = klist.p;
        a.pos = p.pos.p;
        a.cpos = p.cpos.p;
        // pass 3: k-lists, block offsets, positions in C
        LSQ_CUDA_TRY(cudaFuncSetAttribute(k_tc_fill, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_fill));
        note_launch();
        k_tc_fill<<<grid, 512, smem_fill, s>>>(a);
        LSQ_CHECK_LAUNCH();
        // blocks the launches copy (the other slots are zeros stored in shared memory)
        DevBuf<unsigned long long> cnt;
        LSQ_TRY(cnt.alloc(1));
        LSQ_CUDA_TRY(cudaMemsetAsync(cnt.p, 0, sizeof(unsigned long long), s));
        note_launch();
        k_count_present<<<std::max(1, std::min<int>((int)((total + 255) / 256), g->num_sms * 8)), 256, 0, s>>>(
            total, p.pos.p, cnt.p);
        LSQ_CHECK_LAUNCH();
        unsigned long long h = 0;
        LSQ_CUDA_TRY(cudaMemcpyAsync(&h, cnt.p, sizeof(h), cudaMemcpyDeviceToHost, s));
        LSQ_CUDA_TRY(cudaStreamSynchronize(s));  // the scratch lists are freed on return
        p.present = (int64_t)h;
    }
    LSQ_TRY(plan_count_triples(g, ra, rb, rc, upper, &p.triples, s));
    if (std::getenv("LSQ_TC_LOG")) {
        const int smax = p.grid > 0 ? *std::max_element(cst.begin(), cst.end()) : 0;
        std::fprintf(stderr,
                     "lsq tc plan: ranges (%g, %g, %g) tri %d: %d tiles, %lld blocks gathered, %lld dense / %lld "
                     "triples (%.3f), %d CTAs, max %d stages per CTA, records %.1f MB\n",
                     PA.R, PX.R, PC.R, upper, p.ntiles, (long long)p.units, (long long)p.dense_triples,
                     (long long)p.triples, p.dense_triples ? (double)p.triples / p.dense_triples : 0.0, p.grid, smax,
                     4.0 * total / 1e6);
    }
    *out = &g->tcplans.emplace(key, std::move(p)).first->second;
    return LSQ_OK;
}

namespace {

// mode: 0 X, 1 X^T, 2 X + X^T (see k_split_tf32).
int split_operand(lsq_geom g, int r, int mode, const float *X, DevBuf<char> &buf, cudaStream_t s) {
    const int64_t nnzb = g->pats[r].nnzb;
    const size_t need = (size_t)kUnit * (size_t)std::max<int64_t>(nnzb, 1);
    if (buf.n < need) LSQ_TRY(buf.alloc(need));
    if (nnzb == 0) return LSQ_OK;
    const int blocks = (int)std::max<int64_t>(1, std::min<int64_t>((nnzb * 16 + 255) / 256, (int64_t)g->num_sms * 16));
    float *out = reinterpret_cast<float *>(buf.p);
    note_launch();
    if (mode == 1)
        k_split_tf32<1><<<blocks, 256, 0, s>>>(nnzb, g->pats[r].tmap.p, X, out);
    else if (mode == 2)
        k_split_tf32<2><<<blocks, 256, 0, s>>>(nnzb, g->pats[r].tmap.p, X, out);
    else
        k_split_tf32<0><<<blocks, 256, 0, s>>>(nnzb, nullptr, X, out);
    LSQ_CHECK_LAUNCH();
    return LSQ_OK;
}

}  // namespace

int dev_err_ptr(lsq_geom g, int **out) {
    if (!g->dev_err.p) {
        LSQ_TRY(g->dev_err.alloc(1));
        LSQ_CUDA_TRY(cudaMemset(g->dev_err.p, 0, sizeof(int)));
    }
    *out = g->dev_err.p;
    return LSQ_OK;
}

int tc_block_matmul(lsq_geom g, int ra, int ta, const float *A, int rb, int tb, const float *B, int rc, float *C,
                    double alpha, double beta, int upper, bool mirror, int64_t *triples, cudaStream_t s,
                    bool b_sym, bool reuse_a) {
    LSQ_TRY(ensure_tmap(g, ra, s));
    LSQ_TRY(ensure_tmap(g, rb, s));
    TcPlan *p = nullptr;
    LSQ_TRY(tc_plan_get(g, ra, rb, rc, upper, &p, s));
    if (triples) *triples = p->triples;
    if (g->n == 0 || g->pats[rc].nnzb == 0 || p->ntiles == 0) return LSQ_OK;
    if (!p->pos.p || !p->cpos.p || !p->tile_nk.p || !p->tile_posoff.p || !p->cta_stages.p)
        return set_error(LSQ_ERR_CUDA, "tensor-core plan without its records");
    // op(A) and X = op(B)^T (B's rows when trans_b, else B read through its transpose map; B +
    // B^T when b_sym) in split form, in buffers held by g.  The split of A is kept when the
    // caller says A is unchanged since the previous split of the same array.
    const bool keep = reuse_a && g->tc_a_src == A && g->tc_a_range == ra && g->tc_a_trans == (ta != 0);
    if (!keep) {
        g->tc_a_src = nullptr;
        LSQ_TRY(split_operand(g, ra, ta != 0 ? 1 : 0, A, g->tc_a, s));
        g->tc_a_src = A;
        g->tc_a_range = ra;
        g->tc_a_trans = ta != 0;
    }
    LSQ_TRY(split_operand(g, rb, b_sym ? 2 : (tb == 0 ? 1 : 0), B, g->tc_x, s));
    int *err = nullptr;
    LSQ_TRY(dev_err_ptr(g, &err));
    TcArgs a;
    a.ntiles = p->ntiles;
    a.tile_nk = p->tile_nk.p;
    a.cpos = p->cpos.p;
    a.tile_posoff = p->tile_posoff.p;
    a.cta_stages = p->cta_stages.p;
    a.pos = p->pos.p;
    a.As = g->tc_a.p;
    a.Xs = g->tc_x.p;
    a.C = C;
    a.c_tm = nullptr;
    if (upper == 1 && mirror) {
        LSQ_TRY(ensure_tmap(g, rc, s));
        a.c_tm = g->pats[rc].tmap.p;
    }
    a.alpha = (float)alpha;
    a.beta = (float)beta;
    a.err = err;
    // LSQ_TC_WAIT_NS lowers the bound of the pipeline waits (0: any wait that does not succeed at
    // once expires), so that a test can check the timeout path and its status; default 1 s
    a.wait_ns = kWaitNs;
    if (const char *w = std::getenv("LSQ_TC_WAIT_NS")) a.wait_ns = std::strtoull(w, nullptr, 10);
    LSQ_CUDA_TRY(cudaFuncSetAttribute(k_tc_product, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBytes));
    note_launch();
    k_tc_product<<<p->grid, kThreads, kSmemBytes, s>>>(a);
    LSQ_CHECK_LAUNCH();
    // (a symmetric result's lower blocks are written by the kernel itself, see c_tm)
    return LSQ_OK;
}

}  // namespace lsq

using namespace lsq;

extern "C" int lsq_product_plan_info(lsq_geom g, int range_a, int range_b, int range_c, int triangle,
                                     int64_t *info_host) {
    clear_error();
    LSQ_TRY(geom_check(g, range_a));
    LSQ_TRY(geom_check(g, range_b));
    LSQ_TRY(geom_check(g, range_c));
    if (!info_host) return set_error(LSQ_ERR_INVALID_ARG, "info_host is null");
    if (triangle < 0 || triangle > 3) return set_error(LSQ_ERR_INVALID_ARG, "triangle must be 0..3");
    const int upper = triangle == 3 ? 2 : (triangle >= 1 ? 1 : 0);
    const auto key = std::make_tuple(range_a, range_b, range_c + 1000 * upper);
    auto f = g->tcplans.find(key);
    auto ch = g->tc_choice.find(key);
    if (f == g->tcplans.end() && ch == g->tc_choice.end())
        return set_error(LSQ_ERR_INVALID_ARG, "no tensor-core plan or timing for these ranges yet");
    for (int k = 0; k < 6; ++k) info_host[k] = -1;
    if (f != g->tcplans.end()) {
        const TcPlan &p = f->second;
        info_host[0] = p.triples;
        info_host[1] = p.dense_triples;
        info_host[2] = p.units;
        info_host[3] = p.ntiles;
        info_host[5] = p.present;
    }
    info_host[4] = ch == g->tc_choice.end() ? -1 : ch->second.choice;
    return LSQ_OK;
}

extern "C" int lsq_device_status(lsq_geom g, void *stream) {
    clear_error();
    if (!g) return set_error(LSQ_ERR_INVALID_ARG, "null geometry");
    if (!g->dev_err.p) return LSQ_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int h = 0;
    LSQ_CUDA_TRY(cudaMemcpyAsync(&h, g->dev_err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    if (h == 0) return LSQ_OK;
    LSQ_CUDA_TRY(cudaMemsetAsync(g->dev_err.p, 0, sizeof(int), s));
    LSQ_CUDA_TRY(cudaStreamSynchronize(s));
    static const char *where[] = {"", "copy issue (stage free)", "MMA issue (stage full)", "MMA issue (accumulator free)",
                                  "epilogue (accumulator full)", "copies in flight at exit", "MMAs in flight at exit"};
    return set_error(LSQ_ERR_TIMEOUT, std::string("a bounded wait of the tensor-core product expired: ") +
                                          (h > 0 && h < 7 ? where[h] : "unknown"));
}
