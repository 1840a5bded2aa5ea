// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <atomic>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/lsq.h"

namespace lsq {

// ---- kernel launch counter (every launch site calls note_launch) -----------
extern std::atomic<long long> g_launch_count;
void note_launch();

// ---- errors -------------------------------------------------------------
int set_error(int code, const std::string &msg);
void clear_error();

#define LSQ_CUDA_TRY(expr)                                                              \
    do {                                                                                \
        cudaError_t e_ = (expr);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::lsq::set_error(e_ == cudaErrorMemoryAllocation ? LSQ_ERR_OOM       \
                                                                    : LSQ_ERR_CUDA,     \
                                    std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define LSQ_TRY(expr)                  \
    do {                               \
        int rc_ = (expr);              \
        if (rc_ != LSQ_OK) return rc_; \
    } while (0)

#define LSQ_CHECK_LAUNCH() LSQ_CUDA_TRY(cudaGetLastError())

// ---- device buffers owned by the library --------------------------------
template <typename T>
struct DevBuf {
    T *p = nullptr;
    size_t n = 0;
    int alloc(size_t count) {
        release();
        if (count == 0) count = 1;
        cudaError_t e = cudaMalloc(&p, count * sizeof(T));
        if (e != cudaSuccess) {
            p = nullptr;
            return set_error(LSQ_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
        }
        n = count;
        return LSQ_OK;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    DevBuf(DevBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
};

// One range pattern: CSR of atom blocks, plus lazily built position maps.
struct Pattern {
    double R = 0.0;
    int64_t nnzb = 0;
    int max_row = 0;
    DevBuf<int64_t> row_ptr;  // [n + 1]
    DevBuf<int32_t> col;      // [nnzb]
    DevBuf<int64_t> tmap;     // [nnzb] position of (j, i) for entry (i, j); built on demand
};

// Plan of a truncated product: the kernel mode and its exact triple count.
enum { MODE_ROWS = 0, MODE_INNER = 1 };
struct Plan {
    int mode = MODE_ROWS;
    int chunk = 0;
    int64_t triples = 0;
};

// Symbolic product stored as a plan (see plan.cu).
struct ProductPlan {
    int64_t triples = 0;   // block triples the plan executes
    int64_t nblocks = 0;
    int64_t nitems = 0;
    int upper = 0;         // triangle computed: 0 all blocks, 1 j >= i (rest mirrored), 2 j <= i
    int variant[2] = {-1, -1};      // kernel schedule picked by the autotuner (f64, f32)
    int variant16[2] = {-1, -1};    // the fastest of those needing only 16-byte alignment
    float tuned_ms[2] = {0.f, 0.f};
    DevBuf<int64_t> perm;      // blocks of C in processing order (sorted by list length per row)
    DevBuf<int32_t> cnt;       // list length per block of C
    DevBuf<int64_t> item_ptr;  // [nblocks + 1] start of each block's list
    DevBuf<int64_t> c_row;     // row of each block of C
    DevBuf<uint32_t> items;
    ProductPlan() = default;
    ProductPlan(ProductPlan &&) = default;
};

// Tensor-core plan of a truncated 4 x 4 product (see tc.cu): atoms i in groups of 8, the
// atoms j of each group's rows of C in tiles of 16, and per tile a list of atoms k (the
// union of the group's rows of op(A), restricted to atoms in the tile's rows of op(B)^T).
// Tile t runs on CTA t % grid; the block indices each CTA gathers form one stream of stage
// records (24 rows x 16 blocks, -1 for a block its row does not hold).
struct TcPlan {
    int ngroups = 0;
    int ntiles = 0;
    int grid = 0;                // CTAs the plan was laid out for
    int upper = 0;
    int64_t triples = 0;         // exact block triples of the computed blocks of C
    int64_t units = 0;           // operand block slots filled per launch (incl. zeros)
    int64_t present = 0;         // of those, blocks copied from op(A) or op(B)^T
    int64_t dense_triples = 0;   // block triples the MMAs execute (incl. zero blocks)
    DevBuf<int32_t> tile_nk;     // [ntiles] k-list length (a multiple of 16)
    DevBuf<int64_t> tile_posoff; // [ntiles] first stage record of the tile
    DevBuf<int32_t> cta_stages;  // [grid] stages of each CTA
    DevBuf<int32_t> pos;         // stage records: block indices in op(A) or op(B)^T, or -1
    DevBuf<int32_t> cpos;        // [128 ntiles]: block (i, j) of C, -1 if not computed
    TcPlan() = default;
    TcPlan(TcPlan &&) = default;
};

// Outcome of the timing of a kMixedAuto product: 0 the FP32 FMA schedule won, 1 the
// tensor-core kernel won; the two times (ms) of that comparison.
struct TcChoice {
    int choice = 0;
    float ms[2] = {0.f, 0.f};
};

struct Reducer {
    DevBuf<double> partial;   // per-block partial sums
    DevBuf<double> scalars;   // result slots
    double *host = nullptr;   // pinned mirror of scalars
    int nblocks = 0;
};

}  // namespace lsq

struct lsq_geom_s {
    int n = 0;
    int n_ranges = 0;
    double cell[3] = {0, 0, 0};
    int device = 0;
    int num_sms = 0;
    size_t smem_optin = 0;
    lsq::DevBuf<double> pos;
    std::vector<lsq::Pattern> pats;
    // independent systems held block-diagonally (1 for an ordinary geometry)
    int n_sys = 1;
    std::vector<int64_t> sys_atom_off;   // [n_sys + 1] first atom of each system
    lsq::DevBuf<int32_t> atom_sys;       // [n] system of each atom (batched geometries only)
    // key: (range_a, trans_a, range_b, trans_b, range_c, b, dtype)
    std::map<std::tuple<int, int, int, int, int, int, int>, lsq::Plan> plans;
    // key: (pattern p, pattern q, transposed): position in q of (i, j) or (j, i) for each entry of p
    std::map<std::tuple<int, int, int>, lsq::DevBuf<int64_t>> posmaps;
    // product plans keyed by (range_a, range_b, range_c)
    std::map<std::tuple<int, int, int>, lsq::ProductPlan> pplans;
    // schedules adopted from another geometry (lsq_geom_adopt_schedules), same keys:
    // {variant f64, variant f32, variant16 f64, variant16 f32}; used by a plan not yet tuned
    std::map<std::tuple<int, int, int>, std::array<int, 4>> schedule_hints;
    // scratch for transposed operands of lsq_block_matmul (grown on demand)
    lsq::DevBuf<char> scratch_a, scratch_x;
    // tensor-core plans keyed by (range_a, range_b, range_c + 1000 * triangle), the split
    // (hi, lo) operand copies they read (grown on demand), and the device error word of the
    // kernels with bounded waits (0: none)
    std::map<std::tuple<int, int, int>, lsq::TcPlan> tcplans;
    // the kernel each kMixedAuto product was timed to run on (same keys)
    std::map<std::tuple<int, int, int>, lsq::TcChoice> tc_choice;
    lsq::DevBuf<char> tc_a, tc_x;
    // what tc_a holds the split of (see tc_block_matmul's reuse_a)
    const void *tc_a_src = nullptr;
    int tc_a_range = -1;
    bool tc_a_trans = false;
    lsq::DevBuf<int> dev_err;
    // workspace of lsq_hotelling_inverse (grown on demand)
    lsq::DevBuf<char> hot_ws;
    // float32 operands and result of lsq_xl_initial_L (grown on demand)
    lsq::DevBuf<char> xl_scratch;
    lsq::Reducer red;
};

namespace lsq {

int geom_check(lsq_geom g, int range_id);
int ensure_tmap(lsq_geom g, int r, cudaStream_t s);
// Position map from pattern p to pattern q (see posmaps).  Returned pointer owned by g.
int get_posmap(lsq_geom g, int p, int q, int transposed, const int64_t **out, cudaStream_t s);
int find_range(lsq_geom g, double R);

// Truncated product C = alpha op(A) op(B) + beta C (see lsq_block_matmul).  sym = 1
// declares the result symmetric (C = C^T in exact arithmetic): only blocks with j >= i
// are computed and the others are their transposes.  sym = 2 computes the blocks with
// j >= i (for a caller that needs only the upper triangle of a product that is not itself
// symmetric); the other blocks of C are left unspecified.  sym = 3 likewise the blocks with
// j <= i.
int block_matmul(lsq_geom g, int b, int dtype, int ra, int ta, const void *A, int rb, int tb,
                 const void *B, int rc, void *C, double alpha, double beta, int64_t *triples,
                 cudaStream_t s, int sym = 0);

int plan_build(lsq_geom g, int ra, int rb, int rc, int upper, ProductPlan **out, cudaStream_t s);
// mirror: for an upper-triangle plan, fill the lower blocks with the transposes afterwards.
int plan_launch(lsq_geom g, int dtype, const ProductPlan &p, int ra, int rb, int rc, const void *Aop,
                const void *X, void *C, double alpha, double beta, cudaStream_t s, bool mirror = true);
// Plan-driven product for any block size; transposed operands read through transpose maps.
int plan_launch_gen(lsq_geom g, int b, int dtype, const ProductPlan &p, int ra, int ta, int rb, int tb, int rc,
                    const void *A, const void *B, void *C, double alpha, double beta, cudaStream_t s,
                    bool mirror = true);
// out = X^T on the (symmetric) pattern r: out_ij = (X_ji)^T.
int transpose_on(lsq_geom g, int r, int b, int dtype, const void *X, void *out, cudaStream_t s);
// Makes the diagonal blocks of X (pattern r) symmetric: X_ii[r][c] = X_ii[c][r] for r > c.
int sym_diag_on(lsq_geom g, int r, int b, int dtype, void *X, cudaStream_t s);
// out = X + X^T on the (symmetric) pattern r: out_ij = X_ij + (X_ji)^T.
int sym_sum_on(lsq_geom g, int r, int b, int dtype, const void *X, void *out, cudaStream_t s);

// Reductions into g->red.scalars[slot] (float64), enqueued on s.
int trace_into(lsq_geom g, int b, int dtype, int rx, const void *X, int ry, const void *Y, int slot,
               cudaStream_t s);
int dot_into(lsq_geom g, int b, int dtype, int r, const void *X, const void *Y, int slot,
             cudaStream_t s);
int reducer_ensure(lsq_geom g, int nslots);
// g->red.scalars[slot] = sum of x[0..m) (float64, fixed order; m < 2^31).
int sum_into(lsq_geom g, const double *x, int64_t m, int slot, cudaStream_t s);
int fetch_scalars(lsq_geom g, int nslots, double *out, cudaStream_t s);

inline size_t dtype_size(int dtype) { return dtype == LSQ_F64 ? 8 : 4; }

// ---- grouped products (the batched minimiser over several contexts) ----------
// One product as the plan kernels would have been launched with it.  For b = 4 the operands
// are op(A) and X = op(B)^T with rows contiguous (transposed into scratch beforehand); for
// other b, A and B as given, read through the transpose maps when ta / tb.
struct GroupProduct {
    int b = 0, dtype = 0, ta = 0, tb = 0, upper = 0, n = 0;
    int64_t nblocks = 0;
    const int64_t *c_ptr = nullptr, *perm = nullptr, *item_ptr = nullptr, *a_ptr = nullptr,
                  *x_ptr = nullptr, *c_row = nullptr, *a_tm = nullptr, *b_tm = nullptr;
    const uint32_t *items = nullptr;
    const int32_t *c_col = nullptr;
    const void *A = nullptr, *X = nullptr;
    void *C = nullptr;
    double alpha = 1.0, beta = 0.0;
};

// While a step is captured for a grouped launch, g_group_rec is set (per host thread): the plan
// launches then record their product and split the capture (the work before the product is
// one graph segment, the work after it starts the next) instead of launching a kernel.
// segments[k] precedes products[k]; the last segment follows the last product.
struct GroupRecorder {
    std::vector<cudaGraph_t> segments;
    std::vector<GroupProduct> products;
    int split(cudaStream_t s);
    ~GroupRecorder();
};
extern thread_local GroupRecorder *g_group_rec;

// Device descriptors of a grouped launch (uploaded once; see group_launch).
struct GroupLaunch {
    void *desc = nullptr;  // device copy of the products' descriptors
    int nprod = 0, dtype = 0;
    int form = 4;          // kernel variant (see k_mm_group)
    int64_t nchunks = 0;   // work items of the launch's queue
    int grid = 0;
};
// Uploads the descriptors of products (all of one dtype) into out->desc (device memory owned by
// the caller: free with cudaFree).  Synchronous; call it outside stream capture.
int group_prepare(const GroupProduct *products, int n, const lsq_geom g_any, GroupLaunch *out);
// The grouped product: one persistent launch whose thread blocks take work items (a chunk of
// blocks of C of one product) from a queue in device memory until it is empty.  counter is
// reset on s before the launch.
int group_launch(const GroupLaunch &gl, unsigned long long *counter, cudaStream_t s);

// Internal product precision (not part of the ABI): float32 storage, and per product the
// faster of the FP32 FMA schedules and the LSQ_TF32X3 tensor-core kernel, timed on the
// product's first call (with beta = 0).  The LNV path uses it when asked for LSQ_TF32X3.
constexpr int kMixedAuto = 100;

// The TF32X3 tensor-core plan of a product (built on first use; see tc.cu).
int tc_plan_get(lsq_geom g, int ra, int rb, int rc, int upper, TcPlan **out, cudaStream_t s);

// Exact block triples of a product restricted to a triangle (upper: 0 all, 1 j >= i, 2 j <= i).
int plan_count_triples(lsq_geom g, int ra, int rb, int rc, int upper, int64_t *out, cudaStream_t s);
// Loads the fixed scratch array of lsq_trace_static on the current device (noalloc.cu).
int noalloc_prime();
// Device error word of g (allocated and cleared on first use).
int dev_err_ptr(lsq_geom g, int **out);
// Tensor-core truncated 4 x 4 product in split TF32 (see tc.cu); float32 operands and result.
// b_sym: op(B) = B + B^T (B on a symmetric pattern; tb ignored), without forming the sum.
// reuse_a: A (same array, range and flag) is unchanged since the previous call split it.
int tc_block_matmul(lsq_geom g, int ra, int ta, const float *A, int rb, int tb, const float *B, int rc,
                    float *C, double alpha, double beta, int upper, bool mirror, int64_t *triples,
                    cudaStream_t s, bool b_sym = false, bool reuse_a = false);
// The kernel the kMixedAuto timing chose for this product (-1 not timed yet, 0 FP32 FMA, 1
// tensor cores); sym and beta as for block_matmul.
int mixed_choice(lsq_geom g, int ra, int rb, int rc, int sym, double beta);

#ifdef __CUDACC__
// Error-free float32 sum (Knuth's TwoSum): s = fl(a + b) and s + e = a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Adds x * y to the float pair (s, c) without losing the rounding errors of the product (an
// FMA recovers it exactly) or of the sum (TwoSum); s + c then carries about twice the float32
// precision.  Used to accumulate float32 dot products without a float64 operation per term.
__device__ __forceinline__ void dot2_add(float x, float y, float &s, float &c) {
    const float p = __fmul_rn(x, y);
    const float pe = __fmaf_rn(x, y, -p);
    float t, te;
    two_sum(s, p, t, te);
    s = t;
    c = __fadd_rn(c, __fadd_rn(te, pe));
}
#endif

}  // namespace lsq
