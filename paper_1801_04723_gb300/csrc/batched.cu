// spin_invert_batched: many independent inversions of uneven order in one call.
//
// Matrices are grouped by order into buckets.  Every matrix of a bucket has
// the same recursion tree (same splits, same leaves), so the bucket runs the
// recursion of Algorithm 1 once, in lockstep, with each launch covering the
// whole bucket: a batched product (grid.z = matrix) or a batched leaf
// (one thread-block cluster per matrix).  Buckets are independent and run
// concurrently on a pool of streams forked from the caller's stream.
//
// The launch sequence (all buckets, fork and join) is captured once into a
// CUDA graph and replayed while the caller passes the same arguments, so a
// batch of thousands of matrices costs one graph launch on the host.
//
// Mixed precision (SPIN_MIXED_BF16X3): the same lockstep recursion with the
// level products on the tensor cores, batched over the bucket (one launch
// per split and per product; the digit or BF16 planes of every matrix of the
// bucket sit in one arena, one problem after the other), FP64-class Schur
// complements at the top fp64_levels levels, then Newton-Schulz refinement
// of every matrix with FP64-class residuals (cached digit planes of A).  The
// refinement's stopping decisions are taken per matrix on the device
// (refine.cu): every round is part of the captured graph and a matrix that
// has converged is switched off, so a mixed batch is one graph replay too.
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "mixed.h"
#include "persistent.h"
#include "tc_gemm.h"

namespace spin {
namespace {

constexpr int kStreams = 8;

struct Bucket {
    int64_t n, leaf;
    int count;
    int first;             // offset of the bucket in the sorted order
    size_t ws_elems;       // per matrix
    size_t ws_offset;      // elements into the workspace block
    // mixed precision
    size_t scratch_per;    // split-plane bytes per matrix (products, residual, update)
    size_t cache_per;      // cached digit planes of A per matrix
    size_t arena_offset;   // bytes into the plan's arena
    int stream;            // pool stream the bucket runs on
    int sr, s0;            // mixed: digit slices of the certifying residuals and of the first one
    int tile_cap = 64;     // persistent schedule: largest product tile
};

// Residual slices of a bucket of order n (the single-matrix rule).
void set_slices(Bucket& b, const spin_opts& o) {
    b.sr = o.residual_slices > 0 ? o.residual_slices : residual_slices_for(b.n, o.tol);
    b.s0 = o.residual_slices > 0 ? o.residual_slices : first_residual_slices_for(b.n, o.tol, b.sr);
}

struct BatchPlan {
    std::vector<uint64_t> key;
    std::vector<Bucket> buckets;
    // device arrays in sorted (bucket) order
    const double** a_base = nullptr;
    int64_t* a_ld = nullptr;
    double** x_base = nullptr;
    double** w_base = nullptr;
    int* user_index = nullptr;
    int32_t* records = nullptr;  // [count][INFO_WORDS]
    double* ws = nullptr;
    size_t ws_bytes = 0;
    int count = 0;
    int kernels = 0;        // kernel launches of the latest call (graph + refinement)
    int graph_kernels = 0;  // kernel launches in the captured graph
    // mixed precision
    int precision = SPIN_FP64;
    int fp64_levels = 2, max_refine = 6;
    double tol = 1e-10;
    unsigned char* arena = nullptr;
    size_t arena_bytes = 0;
    double* norms = nullptr;       // device: [3][count] sums of squares of A, X, R (sorted order)
    int* active = nullptr;         // device: [count] refinement still running
    double* rel = nullptr;         // device: [count] latest relative residual
    int* iters = nullptr;          // device: [count] refinement steps taken
    int* err = nullptr;            // device: SPIN_ERR_TIMEOUT from a bounded wait
    const int* nvalid = nullptr;   // device, optional: [count] order of the matrix inside its identity padding
    // plain form on the persistent kernel (persistent.cu): stage list, task
    // starts, control block (done counters, task counter, error flag)
    bool persistent = false;
    PStage* pstages = nullptr;
    int64_t* pstart = nullptr;
    unsigned char* pctl = nullptr;
    size_t pctl_bytes = 0;
    int nstages = 0;
    int64_t ptasks = 0;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;  // private stream the launch sequence is captured on
    cudaStream_t streams[kStreams] = {};
    cudaEvent_t fork = nullptr, join[kStreams] = {};
};

std::mutex g_bmu;
std::map<cudaStream_t, BatchPlan> g_plans;

void free_plan(BatchPlan& p) {
    if (p.exec) cudaGraphExecDestroy(p.exec);
    cudaFree(p.arena);
    cudaFree(p.norms);
    cudaFree(p.active);
    cudaFree(p.rel);
    cudaFree(p.iters);
    cudaFree(p.err);
    p.arena = nullptr;
    p.arena_bytes = 0;
    p.norms = nullptr;
    p.active = nullptr;
    p.rel = nullptr;
    p.iters = nullptr;
    p.err = nullptr;
    cudaFree((void*)p.a_base);
    cudaFree(p.a_ld);
    cudaFree(p.x_base);
    cudaFree(p.w_base);
    cudaFree(p.user_index);
    cudaFree(p.records);
    cudaFree(p.ws);
    cudaFree(p.pstages);
    cudaFree(p.pstart);
    cudaFree(p.pctl);
    p.pstages = nullptr;
    p.pstart = nullptr;
    p.pctl = nullptr;
    p.pctl_bytes = 0;
    p.nstages = 0;
    p.ptasks = 0;
    p.persistent = false;
    p.exec = nullptr;
    p.a_base = nullptr;
    p.a_ld = nullptr;
    p.x_base = p.w_base = nullptr;
    p.user_index = nullptr;
    p.records = nullptr;
    p.ws = nullptr;
    p.ws_bytes = 0;
}

__global__ void scatter_status_kernel(const int32_t* records, const int* user_index, int count, int* info_dev) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) info_dev[user_index[i]] = records[(int64_t)i * INFO_WORDS + INFO_STATUS];
}

struct BRun {
    int* kernels;  // launch counter
    cudaStream_t s;
    int32_t* records;  // bucket's first record
    int leaf_counter;
    int64_t leaf;
    int count;
    double* ws_block;  // bucket's workspace block (count * ws_elems)
    int64_t ws_stride;
};

BatchView sub(BatchView v, int64_t dr, int64_t dc) {
    v.r0 += dr;
    v.c0 += dc;
    return v;
}

#define BRET(x)                       \
    do {                              \
        int _r = (x);                 \
        if (_r != SPIN_OK) return _r; \
    } while (0)

// Lockstep recursion for a bucket.  W is a view into each matrix's private
// workspace (linear offset in c0, uniform ld set per use).
int binv(BRun& r, BatchView A, BatchView X, const double* const* wbase, int64_t woff, int64_t n) {
    if (n <= r.leaf) {
        double* scratch = leaf_scratch_elems(n) ? r.ws_block + woff : nullptr;
        (*r.kernels)++;
        return launch_leaf_gj_batched(A, X, n, scratch, r.ws_stride, r.records, r.leaf_counter++, r.count, r.s);
    }
    *r.kernels += 6;
    const int64_t n1 = split_order(n), n2 = n - n1;
    BatchView A11 = A, A12 = sub(A, 0, n1), A21 = sub(A, n1, 0), A22 = sub(A, n1, n1);
    BatchView X11 = X, X12 = sub(X, 0, n1), X21 = sub(X, n1, 0), X22 = sub(X, n1, n1);
    BatchView T{wbase, nullptr, n2, 0, woff};                // n1 x n2
    BatchView S{wbase, nullptr, n2, 0, woff + n1 * n2};      // n2 x n2
    BatchView T2{wbase, nullptr, n1, 0, woff};               // n2 x n1 (II)
    const int64_t wsub = woff + n1 * n2 + n2 * n2;
    BatchView none{wbase, nullptr, 1, 0, 0};
    BRET(binv(r, A11, X11, wbase, woff, n1));
    BRET(launch_gemm_f64_batched(n1, n2, n1, 1.0, X11, A12, 0.0, none, T, r.count, r.s));
    BRET(launch_gemm_f64_batched(n2, n2, n1, -1.0, A21, T, 1.0, A22, S, r.count, r.s));
    BRET(binv(r, S, X22, wbase, wsub, n2));
    BRET(launch_gemm_f64_batched(n1, n2, n2, -1.0, T, X22, 0.0, none, X12, r.count, r.s));
    BRET(launch_gemm_f64_batched(n2, n1, n1, 1.0, A21, X11, 0.0, none, T2, r.count, r.s));
    BRET(launch_gemm_f64_batched(n2, n1, n2, -1.0, X22, T2, 0.0, none, X21, r.count, r.s));
    BRET(launch_gemm_f64_batched(n1, n1, n2, -1.0, X12, T2, 1.0, X11, X11, r.count, r.s));
    return SPIN_OK;
}

// ---- the plain form as one persistent launch ----

PView pview(int src, int64_t ld, int64_t r0, int64_t c0) {
    PView v;
    v.src = src;
    v.pad = 0;
    v.ld = ld;
    v.r0 = r0;
    v.c0 = c0;
    return v;
}

PView psub(PView v, int64_t dr, int64_t dc) {
    v.r0 += dr;
    v.c0 += dc;
    return v;
}

// Product tile of the persistent schedule: every bucket's tasks run side by
// side, so a product need not fill the GPU by itself.  The tile with the
// least CTA time: padded FMAs (one per clock for one of the two CTAs of an
// SM) plus a fixed cost per task (taking the task, its dependency check and
// its completion, about 3000 clocks).  The tile never changes a result bit.
int persist_tile(int64_t m, int64_t n, int64_t k, int cap) {
    const int forced = forced_f64_tile();
    if (forced) return forced;
    constexpr double kTaskClocks = 3000.0;
    int best = 0;
    double best_cost = 0.0;
    for (int tm : {64, 32, 16}) {
        if (tm > cap && tm != 16) continue;
        const double tiles = (double)((m + tm - 1) / tm) * (double)((n + tm - 1) / tm);
        const double cost = tiles * ((double)tm * tm * (double)k + kTaskClocks);
        if (best == 0 || cost < best_cost) {
            best = tm;
            best_cost = cost;
        }
    }
    return best;
}

// Stages of one bucket's recursion, in binv's order (the lockstep launches
// become stages; their tile choice and leaf numbering are binv's).
struct StageList {
    std::vector<PStage> st;
    int first = 0, count = 0;
    int64_t leaf = 0;
    int tile_cap = 64;
    int leaf_counter = 0;
    int32_t need = 0;

    PStage base(int kind) const {
        PStage x;
        memset(&x, 0, sizeof x);
        x.kind = kind;
        x.first = first;
        x.count = count;
        x.need = need;
        return x;
    }
    void leaf_inv(int64_t L, PView a, PView d) {
        PStage x = base(PSTAGE_LEAF);
        x.tiles = 1;
        x.tiles_n = 1;
        x.leaf_index = leaf_counter++;
        x.m = x.n = x.k = L;
        x.a = a;
        x.d = d;
        st.push_back(x);
        need += 1;
    }
    void product(int64_t m, int64_t n, int64_t k, double alpha, PView a, PView b, double beta, PView c, PView d) {
        if (m <= 0 || n <= 0) return;
        PStage x = base(PSTAGE_PRODUCT);
        x.tm = persist_tile(m, n, k, tile_cap);
        x.tiles_n = (int32_t)((n + x.tm - 1) / x.tm);
        x.tiles = (int32_t)((m + x.tm - 1) / x.tm) * x.tiles_n;
        x.m = m;
        x.n = n;
        x.k = k;
        x.alpha = alpha;
        x.beta = beta;
        x.a = a;
        x.b = b;
        x.c = c;
        x.d = d;
        st.push_back(x);
        need += x.tiles;
    }
};

// binv's recursion with the launches recorded as stages.
void pinv(StageList& L, PView A, PView X, int64_t woff, int64_t n) {
    if (n <= L.leaf) {
        L.leaf_inv(n, A, X);
        return;
    }
    const int64_t n1 = split_order(n), n2 = n - n1;
    PView A12 = psub(A, 0, n1), A21 = psub(A, n1, 0), A22 = psub(A, n1, n1);
    PView X11 = X, X12 = psub(X, 0, n1), X21 = psub(X, n1, 0), X22 = psub(X, n1, n1);
    PView T = pview(2, n2, 0, woff);             // n1 x n2
    PView S = pview(2, n2, 0, woff + n1 * n2);   // n2 x n2
    PView T2 = pview(2, n1, 0, woff);            // n2 x n1 (II)
    const int64_t wsub = woff + n1 * n2 + n2 * n2;
    PView none = pview(2, 1, 0, 0);
    pinv(L, A, X11, woff, n1);
    L.product(n1, n2, n1, 1.0, X11, A12, 0.0, none, T);
    L.product(n2, n2, n1, -1.0, A21, T, 1.0, A22, S);
    pinv(L, S, X22, wsub, n2);
    L.product(n1, n2, n2, -1.0, T, X22, 0.0, none, X12);
    L.product(n2, n1, n1, 1.0, A21, X11, 0.0, none, T2);
    L.product(n2, n1, n2, -1.0, X22, T2, 0.0, none, X21);
    L.product(n1, n1, n2, -1.0, X12, T2, 1.0, X11, X11);
}

// Task order of the whole batch: stage position first, larger orders first
// within a position (each bucket's stages stay in their order, so every
// task only depends on tasks before it).  start gets nstages + 1 entries.
// Starting the buckets 1 to 3 positions apart, so that a position mixes
// leaves and products, measured the same on the batching workload (709.8 to
// 710.2 ms against 710.2): the leaves' pivot steps already share the SMs
// with product tiles as the positions drift apart.
void order_stages(const std::vector<Bucket>& buckets, std::vector<PStage>& out, std::vector<int64_t>& start) {
    std::vector<StageList> lists(buckets.size());
    size_t longest = 0;
    for (size_t i = 0; i < buckets.size(); i++) {
        const Bucket& b = buckets[i];
        StageList& L = lists[i];
        L.first = b.first;
        L.count = b.count;
        L.leaf = b.leaf;
        L.tile_cap = b.tile_cap;
        pinv(L, pview(0, 0, 0, 0), pview(1, b.n, 0, 0), 0, b.n);
        for (PStage& x : L.st) x.bucket = (int32_t)i;
        longest = std::max(longest, L.st.size());
    }
    std::vector<size_t> by_order(buckets.size());
    std::iota(by_order.begin(), by_order.end(), 0);
    std::stable_sort(by_order.begin(), by_order.end(),
                     [&](size_t a, size_t b) { return buckets[a].n > buckets[b].n; });
    out.clear();
    start.assign(1, 0);
    for (size_t pos = 0; pos < longest; pos++)
        for (size_t i : by_order)
            if (pos < lists[i].st.size()) {
                const PStage& x = lists[i].st[pos];
                out.push_back(x);
                start.push_back(start.back() + (int64_t)x.count * x.tiles);
            }
}

// ---- mixed precision ----

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Smallest m, n and k a batched mixed product takes to the tensor cores
// (SPIN_TC_MIN_BATCHED overrides it, for measurement; read once).
int64_t tc_min_batched() {
    static int64_t v = -1;
    if (v < 0) {
        const char* e = getenv("SPIN_TC_MIN_BATCHED");
        const long long x = e ? atoll(e) : 0;
        v = x > 0 ? (int64_t)x : 32;
    }
    return v;
}

// Split-plane bytes per matrix for a bucket of order n: the largest level
// product (bf16x3 planes, or digit planes for the top Schur complements),
// the residual's digit planes of X and the update's three planes of X and R.
size_t mixed_scratch_per(int64_t n, int64_t leaf, int fp64_levels, int sr) {
    size_t need = 0;
    if (n > leaf) {
        const int64_t n1 = split_order(n);
        const size_t ld1 = (size_t)tc_ld(n1);
        need = std::max(need, 2 * 2 * (size_t)n1 * ld1 * 2);  // bf16x3: 2 planes of m and n rows
        if (fp64_levels > 0)
            need = std::max(need, (size_t)kSchurSlices * 2 * (size_t)n1 * ld1 * 2 + 2 * (size_t)n1 * 4 + 512);
    }
    const size_t ld = (size_t)tc_ld(n);
    need = std::max(need, (size_t)sr * (size_t)n * ld * 2 + (size_t)n * 4 + 512);  // residual: X digits
    need = std::max(need, 3 * 2 * (size_t)n * ld * 2);                             // update: X and R planes
    return align256(need);
}

size_t mixed_cache_per(int64_t n, int sr) {
    return align256((size_t)sr * (size_t)n * (size_t)tc_ld(n) * 2 + (size_t)n * 4 + 512);
}

struct BMix {
    unsigned char* scratch;  // bucket's split planes: count * scratch_per bytes
    int count;
    int fp64_levels;
    int* err;
    int* kernels;
    cudaStream_t s;
};

template <class T>
T* after(const void* p, size_t bytes) {
    return (T*)(((uintptr_t)p + bytes + 255) & ~(uintptr_t)255);
}

// D(z) = beta C(z) + alpha A(z) B(z) for every matrix z of the bucket, in
// the form the single-matrix mixed path uses for this product.
int bproduct(BMix& x, int depth, bool schur, int64_t m, int64_t n, int64_t k, double alpha, const BatchView& A,
             const BatchView& B, double beta, const BatchView& C, const BatchView& D) {
    // The batch's products are small and numerous: on the tensor cores a
    // 128 x 256 tile that a 32 x 32 product fills to 1/32 still outruns the
    // FP64 pipe (GB300's BF16 rate is ~1500x its FP64 rate), so only products
    // below 32 in some dimension stay in FP64 (64 measures the same, 128 and
    // 256 are 12 % and 72 % slower per batch).
    const int64_t tcm = tc_min_batched();
    if (m < tcm || n < tcm || k < tcm) {
        (*x.kernels)++;
        return launch_gemm_f64_batched(m, n, k, alpha, A, B, beta, C, D, x.count, x.s);
    }
    const int64_t ld = tc_ld(k);
    const int64_t cnt = x.count;
    TcGemmParams p = {};
    p.M = (int)m;
    p.N = (int)n;
    p.K = (int)k;
    p.alpha = alpha;
    p.beta = beta;
    p.err = x.err;
    p.batch = x.count;
    p.c_base = beta != 0.0 ? C.base : nullptr;
    p.c_lds = C.lds;
    p.c_ld = C.ld;
    p.c_r0 = C.r0;
    p.c_c0 = C.c0;
    p.d_base = const_cast<double* const*>(D.base);
    p.d_lds = D.lds;
    p.d_ld = D.ld;
    p.d_r0 = D.r0;
    p.d_c0 = D.c0;
    uint16_t* pa = (uint16_t*)x.scratch;
    if (schur && depth < x.fp64_levels) {
        const int sl = kSchurSlices;
        uint16_t* pb = pa + cnt * sl * m * ld;
        int* ea = after<int>(pb, (size_t)cnt * sl * n * ld * 2);
        int* eb = ea + cnt * m;
        *x.kernels += 2 * 3 + 1;
        BRET(launch_ozaki_split_batched(A, (int)m, (int)k, false, sl, ea, pa, ld, nullptr, x.count, x.s));
        BRET(launch_ozaki_split_batched(B, (int)k, (int)n, true, sl, eb, pb, ld, nullptr, x.count, x.s));
        tc_pairs_ozaki(p, sl);
        p.row_exp = ea;
        p.col_exp = eb;
        return launch_tc_gemm(TcOperand{pa, (int)m, sl, ld}, TcOperand{pb, (int)n, sl, ld}, p, x.s);
    }
    uint16_t* pb = pa + cnt * 2 * m * ld;
    *x.kernels += 3;
    BRET(launch_split_planes_batched(A, (int)m, (int)k, false, 2, pa, ld, x.count, x.s));
    BRET(launch_split_planes_batched(B, (int)k, (int)n, true, 2, pb, ld, x.count, x.s));
    tc_pairs_bf16x3(p);
    return launch_tc_gemm(TcOperand{pa, (int)m, 2, ld}, TcOperand{pb, (int)n, 2, ld}, p, x.s);
}

// Lockstep recursion of a bucket with tensor-core level products (binv's
// schedule; the Schur product is the one that forms S = -V).
int binv_mixed(BRun& r, BMix& x, int depth, BatchView A, BatchView X, const double* const* wbase, int64_t woff,
               int64_t n) {
    if (n <= r.leaf) {
        double* scratch = leaf_scratch_elems(n) ? r.ws_block + woff : nullptr;
        (*r.kernels)++;
        return launch_leaf_gj_batched(A, X, n, scratch, r.ws_stride, r.records, r.leaf_counter++, r.count, r.s);
    }
    const int64_t n1 = split_order(n), n2 = n - n1;
    BatchView A12 = sub(A, 0, n1), A21 = sub(A, n1, 0), A22 = sub(A, n1, n1);
    BatchView X11 = X, X12 = sub(X, 0, n1), X21 = sub(X, n1, 0), X22 = sub(X, n1, n1);
    BatchView T{wbase, nullptr, n2, 0, woff};
    BatchView S{wbase, nullptr, n2, 0, woff + n1 * n2};
    BatchView T2{wbase, nullptr, n1, 0, woff};
    const int64_t wsub = woff + n1 * n2 + n2 * n2;
    BatchView none{wbase, nullptr, 1, 0, 0};
    const int d = depth;
    BRET(binv_mixed(r, x, d + 1, A, X11, wbase, woff, n1));
    BRET(bproduct(x, d, false, n1, n2, n1, 1.0, X11, A12, 0.0, none, T));
    BRET(bproduct(x, d, true, n2, n2, n1, -1.0, A21, T, 1.0, A22, S));
    BRET(binv_mixed(r, x, d + 1, S, X22, wbase, wsub, n2));
    BRET(bproduct(x, d, false, n1, n2, n2, -1.0, T, X22, 0.0, none, X12));
    BRET(bproduct(x, d, false, n2, n1, n1, 1.0, A21, X11, 0.0, none, T2));
    BRET(bproduct(x, d, false, n2, n1, n2, -1.0, X22, T2, 0.0, none, X21));
    BRET(bproduct(x, d, false, n1, n1, n2, -1.0, X12, T2, 1.0, X11, X11));
    return SPIN_OK;
}

// Refinement of the matrices of one bucket, enqueued on s: residuals
// R(z) = I - A(z) X(z) FP64-class (digit planes, A's cached), X(z) <- X(z) +
// X(z) R(z) in the six-product BF16 form, rounds 0 .. max_refine all
// enqueued; each matrix's decision is taken on the device and a matrix that
// has converged (or failed) is switched off, its launches returning at once.
// R lives in each matrix's workspace.  Statuses go to the records (sorted
// order): SPIN_ERR_NOT_CONVERGED when the cap is reached above tol.
int bucket_refine(BatchPlan& p, const Bucket& b, cudaStream_t s) {
    const int count = p.count;
    const int sr = b.sr;
    BatchView Av{p.a_base + b.first, p.a_ld + b.first, 0, 0, 0};
    BatchView Xv{(const double* const*)(p.x_base + b.first), nullptr, b.n, 0, 0};
    BatchView Rv{(const double* const*)(p.w_base + b.first), nullptr, b.n, 0, 0};
    int* act = p.active + b.first;
    double* nA = p.norms + b.first;
    double* nX = p.norms + count + b.first;
    double* nR = p.norms + 2 * count + b.first;
    int32_t* rec = p.records + (int64_t)b.first * INFO_WORDS;
    const int64_t ld = tc_ld(b.n);
    unsigned char* scratch = p.arena + b.arena_offset;
    unsigned char* cache = scratch + (size_t)b.count * b.scratch_per;
    uint16_t* aplanes = (uint16_t*)cache;
    int* aex = after<int>(aplanes, (size_t)b.count * sr * b.n * ld * 2);
    uint16_t* xplanes = (uint16_t*)scratch;
    int* xex = after<int>(xplanes, (size_t)b.count * sr * b.n * ld * 2);
    uint16_t* xp = (uint16_t*)scratch;  // update: three planes of X, then of R
    uint16_t* rp = xp + (int64_t)b.count * 3 * b.n * ld;
    BRET(launch_refine_init(rec, b.count, act, p.rel + b.first, p.iters + b.first, s));
    SPIN_CUDA_TRY(cudaMemsetAsync(nA, 0, b.count * sizeof(double), s));
    p.kernels += 3;
    const int* nv = p.nvalid ? p.nvalid + b.first : nullptr;  // norms over the unpadded block
    BRET(launch_ozaki_split_batched(Av, (int)b.n, (int)b.n, false, sr, aex, aplanes, ld, nA, b.count, s, act, nv));
    for (int it = 0; it <= p.max_refine; it++) {
        SPIN_CUDA_TRY(cudaMemsetAsync(nX, 0, b.count * sizeof(double), s));
        SPIN_CUDA_TRY(cudaMemsetAsync(nR, 0, b.count * sizeof(double), s));
        BRET(launch_ozaki_split_batched(Xv, (int)b.n, (int)b.n, true, sr, xex, xplanes, ld, nX, b.count, s, act, nv));
        // the first residual only feeds the update: fewer slice pairs
        const int s_it = it == 0 ? b.s0 : sr;
        TcGemmParams q = {};
        q.M = q.N = q.K = (int)b.n;
        tc_pairs_ozaki(q, s_it);
        q.alpha = -1.0;
        q.beta = 0.0;
        q.add_identity = 1;
        q.sumsq = nR;
        q.err = p.err;
        q.active = act;
        q.sum_order = nv;
        q.row_exp = aex;
        q.col_exp = xex;
        q.batch = b.count;
        q.d_base = p.w_base + b.first;
        q.d_ld = b.n;
        BRET(launch_tc_gemm(TcOperand{aplanes, (int)b.n, sr, ld}, TcOperand{xplanes, (int)b.n, sr, ld}, q, s));
        BRET(launch_refine_decide(nA, nX, nR, b.count, p.tol, residual_error_model(b.n, s_it), it, p.max_refine, act,
                                  p.rel + b.first, p.iters + b.first, rec, s));
        p.kernels += 6;
        if (it == p.max_refine) break;
        BRET(launch_split_planes_batched(Xv, (int)b.n, (int)b.n, false, 3, xp, ld, b.count, s, act));
        BRET(launch_split_planes_batched(Rv, (int)b.n, (int)b.n, true, 3, rp, ld, b.count, s, act));
        TcGemmParams u = {};
        u.M = u.N = u.K = (int)b.n;
        tc_pairs_bf16x6(u);
        u.alpha = 1.0;
        u.beta = 1.0;
        u.err = p.err;
        u.active = act;
        u.batch = b.count;
        u.c_base = Xv.base;
        u.c_ld = b.n;
        u.d_base = p.x_base + b.first;
        u.d_ld = b.n;
        p.kernels += 3;
        BRET(launch_tc_gemm(TcOperand{xp, (int)b.n, 3, ld}, TcOperand{rp, (int)b.n, 3, ld}, u, s));
    }
    return SPIN_OK;
}

// Leaf of a bucket of order n: the caller's, else the one the batched
// autotuner recorded for (precision, n), else n for n <= 128 and 64 above.
std::mutex g_bleaf_mu;
std::map<std::pair<int, int64_t>, int64_t> g_bleaf;  // (precision, order) -> leaf
uint64_t g_bleaf_gen = 0;                           // bumped on every record (part of the plan key)

int64_t batched_leaf(int64_t n, int leaf_opt, int precision) {
    int64_t L = leaf_opt > 0 ? leaf_opt : 0;
    if (L == 0) {
        std::lock_guard<std::mutex> lk(g_bleaf_mu);
        auto it = g_bleaf.find(std::make_pair(precision, n));
        if (it != g_bleaf.end()) L = it->second;
    }
    if (L == 0) L = n <= 128 ? n : 64;
    return std::min<int64_t>(L, n);
}

// Largest product tile of a bucket of order n in the persistent schedule:
// the one spin_autotune_batched_persistent recorded, else 64.
std::map<int64_t, int> g_btile;  // order -> tile cap (guarded by g_bleaf_mu)

int persist_tile_cap(int64_t n) {
    std::lock_guard<std::mutex> lk(g_bleaf_mu);
    auto it = g_btile.find(n);
    return it == g_btile.end() ? 64 : it->second;
}

// Plain batches run on the persistent kernel unless the caller asks for the
// lockstep launches (opts.schedule 1) or passes a leaf above its limit.
bool use_persistent(const spin_opts& o) {
    if (o.precision != SPIN_FP64) return false;
    if (o.schedule == SPIN_SCHEDULE_LOCKSTEP) return false;
    return o.leaf <= kPersistMaxLeaf;
}

// Bound of one dependency wait of the persistent kernel: a whole batch of
// thousands of matrices takes under a second.
constexpr uint64_t kPersistWaitNs = 5000000000ull;

// The plain batch as one persistent launch: the stage list goes up once,
// and the captured graph is two memsets (records; done counters, task
// counter and error flag) and the kernel.
int capture_persistent(BatchPlan& p) {
    std::vector<PStage> stages;
    std::vector<int64_t> start;
    order_stages(p.buckets, stages, start);
    p.nstages = (int)stages.size();
    p.ptasks = start.back();
    int64_t max_leaf = 1;
    for (const Bucket& b : p.buckets) max_leaf = std::max(max_leaf, std::min(b.leaf, b.n));
    const size_t smem = persistent_smem_bytes(max_leaf);
    int grid = 0;
    BRET(persistent_grid(smem, p.ptasks, &grid));
    const size_t done_bytes = align256((size_t)p.count * sizeof(unsigned));
    p.pctl_bytes = done_bytes + 256;
    SPIN_CUDA_TRY(cudaMalloc(&p.pstages, std::max<size_t>(stages.size(), 1) * sizeof(PStage)));
    SPIN_CUDA_TRY(cudaMalloc(&p.pstart, start.size() * sizeof(int64_t)));
    SPIN_CUDA_TRY(cudaMalloc(&p.pctl, p.pctl_bytes));
    SPIN_CUDA_TRY(cudaMemcpy(p.pstages, stages.data(), stages.size() * sizeof(PStage), cudaMemcpyHostToDevice));
    SPIN_CUDA_TRY(cudaMemcpy(p.pstart, start.data(), start.size() * sizeof(int64_t), cudaMemcpyHostToDevice));
    PersistentArgs a;
    a.stages = p.pstages;
    a.start = p.pstart;
    a.nstages = p.nstages;
    a.a_base = p.a_base;
    a.a_ld = p.a_ld;
    a.x_base = p.x_base;
    a.w_base = p.w_base;
    a.records = p.records;
    a.done = (unsigned*)p.pctl;
    a.next = (unsigned long long*)(p.pctl + done_bytes);
    a.err = (int*)(p.pctl + done_bytes + 8);
    a.limit_ns = kPersistWaitNs;
    a.bucket_clocks = nullptr;
    cudaStream_t s = p.cap;
    cudaGraph_t graph = nullptr;
    SPIN_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = SPIN_OK;
    cudaError_t e = cudaMemsetAsync(p.records, 0, (size_t)p.count * INFO_WORDS * sizeof(int32_t), s);
    if (e == cudaSuccess) e = cudaMemsetAsync(p.pctl, 0, p.pctl_bytes, s);
    if (e != cudaSuccess) {
        record_cuda_error(e, "persistent batch memsets", __FILE__, __LINE__);
        rc = SPIN_ERR_CUDA;
    }
    if (rc == SPIN_OK) rc = launch_persistent_batch(a, smem, grid, s);
    cudaError_t ec = cudaStreamEndCapture(s, &graph);
    if (rc != SPIN_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    SPIN_CUDA_TRY(ec);
    cudaError_t ei = cudaGraphInstantiate(&p.exec, graph, 0);
    cudaGraphDestroy(graph);
    SPIN_CUDA_TRY(ei);
    p.kernels = p.graph_kernels = 1;
    return SPIN_OK;
}

int build_plan(BatchPlan& p, const double* const* A, const int64_t* lda, double* const* X, const int64_t* n,
               int count, const spin_opts& o, cudaStream_t s) {
    free_plan(p);
    const int leaf_opt = o.leaf;
    const bool mixed = o.precision != SPIN_FP64;
    p.persistent = use_persistent(o);
    p.count = count;
    p.kernels = 0;
    p.precision = o.precision;
    p.tol = o.tol;
    p.max_refine = o.max_refine;
    p.fp64_levels = o.fp64_levels;
    std::vector<int> order(count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return n[a] < n[b]; });
    p.buckets.clear();
    size_t ws_total = 0;
    for (int i = 0; i < count;) {
        int j = i;
        while (j < count && n[order[j]] == n[order[i]]) j++;
        Bucket b;
        b.n = n[order[i]];
        b.leaf = batched_leaf(b.n, leaf_opt, o.precision);
        if (p.persistent) {
            b.leaf = std::min(b.leaf, kPersistMaxLeaf);
            b.tile_cap = persist_tile_cap(b.n);
        }
        b.count = j - i;
        b.first = i;
        b.ws_elems = std::max<size_t>(fp64_workspace_elems(b.n, b.leaf), 1);
        if (mixed) b.ws_elems = std::max<size_t>(b.ws_elems, (size_t)b.n * (size_t)b.n);  // holds R
        b.ws_offset = ws_total;
        ws_total += b.ws_elems * (size_t)b.count;
        set_slices(b, o);
        b.scratch_per = mixed ? mixed_scratch_per(b.n, b.leaf, p.fp64_levels, b.sr) : 0;
        b.cache_per = mixed ? mixed_cache_per(b.n, b.sr) : 0;
        b.arena_offset = p.arena_bytes;
        p.arena_bytes += (size_t)b.count * (b.scratch_per + b.cache_per);
        b.stream = 0;
        p.buckets.push_back(b);
        i = j;
    }
    std::vector<const double*> ha(count);
    std::vector<int64_t> hl(count);
    std::vector<double*> hx(count), hw(count);
    std::vector<int> hu(count);
    if (cudaMalloc(&p.ws, ws_total * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        return SPIN_ERR_OOM;
    }
    if (mixed) {
        if (cudaMalloc(&p.arena, std::max<size_t>(p.arena_bytes, 256)) != cudaSuccess) {
            cudaGetLastError();
            return SPIN_ERR_OOM;
        }
        SPIN_CUDA_TRY(cudaMalloc(&p.norms, 3 * (size_t)count * sizeof(double)));
        SPIN_CUDA_TRY(cudaMalloc(&p.active, (size_t)count * sizeof(int)));
        SPIN_CUDA_TRY(cudaMalloc(&p.rel, (size_t)count * sizeof(double)));
        SPIN_CUDA_TRY(cudaMalloc(&p.iters, (size_t)count * sizeof(int)));
        SPIN_CUDA_TRY(cudaMalloc(&p.err, sizeof(int)));
    }
    p.ws_bytes = ws_total * sizeof(double);
    for (const Bucket& b : p.buckets)
        for (int z = 0; z < b.count; z++) {
            const int pos = b.first + z, u = order[pos];
            ha[pos] = A[u];
            hl[pos] = lda[u];
            hx[pos] = X[u];
            hw[pos] = p.ws + b.ws_offset + (size_t)z * b.ws_elems;
            hu[pos] = u;
        }
    SPIN_CUDA_TRY(cudaMalloc((void**)&p.a_base, count * sizeof(double*)));
    SPIN_CUDA_TRY(cudaMalloc(&p.a_ld, count * sizeof(int64_t)));
    SPIN_CUDA_TRY(cudaMalloc(&p.x_base, count * sizeof(double*)));
    SPIN_CUDA_TRY(cudaMalloc(&p.w_base, count * sizeof(double*)));
    SPIN_CUDA_TRY(cudaMalloc(&p.user_index, count * sizeof(int)));
    SPIN_CUDA_TRY(cudaMalloc(&p.records, (size_t)count * INFO_WORDS * sizeof(int32_t)));
    SPIN_CUDA_TRY(cudaMemcpy((void*)p.a_base, ha.data(), count * sizeof(double*), cudaMemcpyHostToDevice));
    SPIN_CUDA_TRY(cudaMemcpy(p.a_ld, hl.data(), count * sizeof(int64_t), cudaMemcpyHostToDevice));
    SPIN_CUDA_TRY(cudaMemcpy(p.x_base, hx.data(), count * sizeof(double*), cudaMemcpyHostToDevice));
    SPIN_CUDA_TRY(cudaMemcpy(p.w_base, hw.data(), count * sizeof(double*), cudaMemcpyHostToDevice));
    SPIN_CUDA_TRY(cudaMemcpy(p.user_index, hu.data(), count * sizeof(int), cudaMemcpyHostToDevice));
    for (int i = 0; i < kStreams; i++) {
        if (!p.streams[i]) SPIN_CUDA_TRY(cudaStreamCreateWithFlags(&p.streams[i], cudaStreamNonBlocking));
        if (!p.join[i]) SPIN_CUDA_TRY(cudaEventCreateWithFlags(&p.join[i], cudaEventDisableTiming));
    }
    if (!p.fork) SPIN_CUDA_TRY(cudaEventCreateWithFlags(&p.fork, cudaEventDisableTiming));
    if (!p.cap) SPIN_CUDA_TRY(cudaStreamCreateWithFlags(&p.cap, cudaStreamNonBlocking));

    if (p.persistent) return capture_persistent(p);

    // Capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the
    // caller's stream.  Order: memset records, fork, buckets (largest first,
    // least-loaded stream), join.  The statuses are scattered after it.
    cudaGraph_t graph = nullptr;
    s = p.cap;
    SPIN_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = SPIN_OK;
    cudaError_t e = cudaMemsetAsync(p.records, 0, (size_t)count * INFO_WORDS * sizeof(int32_t), s);
    if (e == cudaSuccess && mixed) e = cudaMemsetAsync(p.err, 0, sizeof(int), s);
    if (e == cudaSuccess) e = cudaEventRecord(p.fork, s);
    for (int i = 0; i < kStreams && e == cudaSuccess; i++) e = cudaStreamWaitEvent(p.streams[i], p.fork, 0);
    if (e != cudaSuccess) {
        record_cuda_error(e, "batched fork", __FILE__, __LINE__);
        rc = SPIN_ERR_CUDA;
    }
    std::vector<int> by_work(p.buckets.size());
    std::iota(by_work.begin(), by_work.end(), 0);
    std::sort(by_work.begin(), by_work.end(), [&](int a, int b) {
        const Bucket &x = p.buckets[a], &y = p.buckets[b];
        return (double)x.count * x.n * x.n * x.n > (double)y.count * y.n * y.n * y.n;
    });
    std::vector<double> load(kStreams, 0.0);
    for (int bi : by_work) {
        if (rc != SPIN_OK) break;
        Bucket& b = p.buckets[bi];
        const int si = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[si] += (double)b.count * b.n * b.n * b.n;
        b.stream = si;
        BRun r{&p.kernels, p.streams[si], p.records + (int64_t)b.first * INFO_WORDS, 0, b.leaf, b.count,
               p.ws + b.ws_offset, (int64_t)b.ws_elems};
        BatchView Av{p.a_base + b.first, p.a_ld + b.first, 0, 0, 0};
        BatchView Xv{(const double* const*)(p.x_base + b.first), nullptr, b.n, 0, 0};
        if (mixed) {
            BMix x{p.arena + b.arena_offset, b.count, p.fp64_levels, p.err, &p.kernels, p.streams[si]};
            rc = binv_mixed(r, x, 0, Av, Xv, (const double* const*)(p.w_base + b.first), 0, b.n);
            if (rc == SPIN_OK) rc = bucket_refine(p, b, p.streams[si]);
        } else {
            rc = binv(r, Av, Xv, (const double* const*)(p.w_base + b.first), 0, b.n);
        }
    }
    for (int i = 0; i < kStreams; i++) {
        cudaError_t e2 = cudaEventRecord(p.join[i], p.streams[i]);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, p.join[i], 0);
        if (e2 != cudaSuccess && rc == SPIN_OK) {
            record_cuda_error(e2, "batched join", __FILE__, __LINE__);
            rc = SPIN_ERR_CUDA;
        }
    }
    if (rc == SPIN_OK && mixed) {
        p.kernels++;
        rc = launch_refine_finish(p.err, p.records, count, s);
    }
    cudaError_t ec = cudaStreamEndCapture(s, &graph);
    if (rc != SPIN_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    SPIN_CUDA_TRY(ec);
    cudaError_t ei = cudaGraphInstantiate(&p.exec, graph, 0);
    cudaGraphDestroy(graph);
    SPIN_CUDA_TRY(ei);
    p.graph_kernels = p.kernels;
    return SPIN_OK;
}

std::vector<uint64_t> make_key(const double* const* A, const int64_t* lda, double* const* X, const int64_t* n,
                               int count, const spin_opts& o) {
    std::vector<uint64_t> k;
    k.reserve((size_t)count * 4 + 8);
    k.push_back((uint64_t)count);
    k.push_back((uint64_t)(int64_t)o.leaf);
    k.push_back((uint64_t)(int64_t)o.precision);
    uint64_t tb;
    memcpy(&tb, &o.tol, sizeof(tb));
    k.push_back(tb);
    k.push_back((uint64_t)(int64_t)o.max_refine);
    k.push_back((uint64_t)(int64_t)o.fp64_levels);
    k.push_back((uint64_t)(int64_t)o.residual_slices);
    k.push_back((uint64_t)(int64_t)o.schedule);
    {
        std::lock_guard<std::mutex> lk(g_bleaf_mu);
        k.push_back(g_bleaf_gen);  // a new autotuned leaf invalidates captured plans
    }
    int dev = 0;
    cudaGetDevice(&dev);
    k.push_back((uint64_t)dev);
    for (int i = 0; i < count; i++) {
        k.push_back((uint64_t)(uintptr_t)A[i]);
        k.push_back((uint64_t)lda[i]);
        k.push_back((uint64_t)(uintptr_t)X[i]);
        k.push_back((uint64_t)n[i]);
    }
    return k;
}

// Identity padding: Ap = [[A, 0], [0, I]] of order np >= n.
__global__ void pad_identity_kernel(const double* A, int64_t lda, int64_t n, double* Ap, int64_t np) {
    const int64_t total = np * np;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = i / np, c = i % np;
        Ap[i] = (r < n && c < n) ? A[r * lda + c] : (r == c ? 1.0 : 0.0);
    }
}

// Device layout of one bucket run directly (run_bucket), every part 256-byte
// aligned: upload block (a_base, a_ld, x_base, w_base: count 8-byte words
// each; nvalid: count ints), records, refinement control (active, rel,
// iters, norms [3][count], err), FP64 workspaces, mixed arena.
struct DirectLayout {
    size_t upload, records, active, rel, iters, norms, err, ws, arena, total;
    size_t ws_elems, scratch_per, cache_per;
    int64_t leaf;
    int sr, s0;
};

DirectLayout direct_layout(int64_t n, int count, const spin_opts& o) {
    DirectLayout L;
    const bool mixed = o.precision != SPIN_FP64;
    const size_t c = (size_t)count;
    L.leaf = batched_leaf(n, o.leaf, o.precision);
    Bucket probe;
    probe.n = n;
    set_slices(probe, o);
    L.sr = probe.sr;
    L.s0 = probe.s0;
    L.ws_elems = std::max<size_t>(fp64_workspace_elems(n, L.leaf), 1);
    if (mixed) L.ws_elems = std::max<size_t>(L.ws_elems, (size_t)n * (size_t)n);  // holds R
    L.scratch_per = mixed ? mixed_scratch_per(n, L.leaf, o.fp64_levels, L.sr) : 0;
    L.cache_per = mixed ? mixed_cache_per(n, L.sr) : 0;
    size_t off = 0;
    L.upload = off;
    off = align256(off + 32 * c + 4 * c);
    L.records = off;
    off = align256(off + c * INFO_WORDS * 4);
    L.active = off;
    off = align256(off + 4 * c);
    L.rel = off;
    off = align256(off + 8 * c);
    L.iters = off;
    off = align256(off + 4 * c);
    L.norms = off;
    off = align256(off + 24 * c);
    L.err = off;
    off = align256(off + 4);
    L.ws = off;
    off = align256(off + L.ws_elems * 8 * c);
    L.arena = off;
    off = align256(off + c * (L.scratch_per + L.cache_per));
    L.total = off;
    return L;
}

}  // namespace

size_t bucket_bytes(int64_t n, int count, const spin_opts& o) {
    if (n < 1 || count < 1) return 0;
    return direct_layout(n, count, o).total;
}

// Pinned host staging: upload block (36 bytes per matrix, padded to 40 so
// that the results start 8-byte aligned), then records, rel, iters.
size_t bucket_host_bytes(int count) { return 40 * (size_t)count + (size_t)count * (INFO_WORDS * 4 + 12); }

int launch_pad_identity(const double* A, int64_t lda, int64_t n, double* Ap, int64_t np, cudaStream_t s) {
    if (n < 1 || np < n) return SPIN_ERR_INVALID_ARG;
    const int64_t total = np * np;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 8);
    pad_identity_kernel<<<blocks, 256, 0, s>>>(A, lda, n, Ap, np);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

int run_bucket(const double* const* A, const int64_t* lda, double* const* X, const int* nvalid, int64_t n,
               int count, const spin_opts& o, void* ws, size_t ws_bytes, void* host_stage, cudaStream_t s) {
    if (n < 1 || count < 1 || count > 65535 || ws == nullptr || host_stage == nullptr) return SPIN_ERR_INVALID_ARG;
    if (o.precision != SPIN_FP64 && o.precision != SPIN_MIXED_BF16X3) return SPIN_ERR_NOT_IMPLEMENTED;
    const DirectLayout L = direct_layout(n, count, o);
    if (ws_bytes < L.total || ((uintptr_t)ws & 255u) != 0 || L.leaf > kMaxLeaf) return SPIN_ERR_INVALID_ARG;
    const bool mixed = o.precision != SPIN_FP64;
    unsigned char* base = (unsigned char*)ws;
    // pointer arrays: staged in pinned host memory, one copy up
    unsigned char* up = (unsigned char*)host_stage;
    const size_t c = (size_t)count;
    double* wsb = (double*)(base + L.ws);
    for (int z = 0; z < count; z++) {
        ((const double**)up)[z] = A[z];
        ((int64_t*)(up + 8 * c))[z] = lda[z];
        ((double**)(up + 16 * c))[z] = X[z];
        ((double**)(up + 24 * c))[z] = wsb + (size_t)z * L.ws_elems;
        ((int*)(up + 32 * c))[z] = nvalid ? nvalid[z] : (int)n;
    }
    SPIN_CUDA_TRY(cudaMemcpyAsync(base + L.upload, up, 36 * c, cudaMemcpyHostToDevice, s));
    BatchPlan p;
    p.count = count;
    p.precision = o.precision;
    p.tol = o.tol;
    p.max_refine = o.max_refine;
    p.fp64_levels = o.fp64_levels;
    p.a_base = (const double**)(base + L.upload);
    p.a_ld = (int64_t*)(base + L.upload + 8 * c);
    p.x_base = (double**)(base + L.upload + 16 * c);
    p.w_base = (double**)(base + L.upload + 24 * c);
    p.nvalid = nvalid ? (const int*)(base + L.upload + 32 * c) : nullptr;
    p.records = (int32_t*)(base + L.records);
    p.active = (int*)(base + L.active);
    p.rel = (double*)(base + L.rel);
    p.iters = (int*)(base + L.iters);
    p.norms = (double*)(base + L.norms);
    p.err = (int*)(base + L.err);
    p.ws = wsb;
    p.arena = base + L.arena;
    SPIN_CUDA_TRY(cudaMemsetAsync(p.records, 0, c * INFO_WORDS * 4, s));
    SPIN_CUDA_TRY(cudaMemsetAsync(p.err, 0, 4, s));
    Bucket b;
    b.n = n;
    b.leaf = L.leaf;
    b.count = count;
    b.first = 0;
    b.ws_elems = L.ws_elems;
    b.ws_offset = 0;
    b.scratch_per = L.scratch_per;
    b.cache_per = L.cache_per;
    b.arena_offset = 0;
    b.stream = 0;
    b.sr = L.sr;
    b.s0 = L.s0;
    BRun r{&p.kernels, s, p.records, 0, b.leaf, count, p.ws, (int64_t)b.ws_elems};
    BatchView Av{p.a_base, p.a_ld, 0, 0, 0};
    BatchView Xv{(const double* const*)p.x_base, nullptr, n, 0, 0};
    int rc;
    if (mixed) {
        BMix x{p.arena, count, p.fp64_levels, p.err, &p.kernels, s};
        rc = binv_mixed(r, x, 0, Av, Xv, (const double* const*)p.w_base, 0, n);
        if (rc == SPIN_OK) rc = bucket_refine(p, b, s);
        if (rc == SPIN_OK) rc = launch_refine_finish(p.err, p.records, count, s);
    } else {
        rc = binv(r, Av, Xv, (const double* const*)p.w_base, 0, n);
    }
    if (rc != SPIN_OK) return rc;
    // results down: records, rel, iters (read by bucket_result after the stream is synchronised)
    unsigned char* res = up + 40 * c;
    SPIN_CUDA_TRY(cudaMemcpyAsync(res, p.records, c * INFO_WORDS * 4, cudaMemcpyDeviceToHost, s));
    if (mixed) {
        SPIN_CUDA_TRY(cudaMemcpyAsync(res + c * INFO_WORDS * 4, p.rel, 8 * c, cudaMemcpyDeviceToHost, s));
        SPIN_CUDA_TRY(cudaMemcpyAsync(res + c * INFO_WORDS * 4 + 8 * c, p.iters, 4 * c, cudaMemcpyDeviceToHost, s));
    }
    return SPIN_OK;
}

void bucket_result(const void* host_stage, int count, int z, bool mixed, int32_t* status, double* rel, int* iters) {
    const unsigned char* res = (const unsigned char*)host_stage + 40 * (size_t)count;
    *status = ((const int32_t*)res)[(size_t)z * INFO_WORDS + INFO_STATUS];
    *rel = mixed ? ((const double*)(res + (size_t)count * INFO_WORDS * 4))[z] : -1.0;
    *iters = mixed ? ((const int*)(res + (size_t)count * INFO_WORDS * 4 + 8 * (size_t)count))[z] : 0;
}

}  // namespace spin

using namespace spin;

// Host-side description of the persistent schedule of a plain batch (no
// device work): stages, tasks, leaves, products and their flops, after
// checking the task order's invariants (each bucket's stages in recursion
// order, each stage's `need` equal to the tasks of the bucket's earlier
// stages, task starts the running sums of count x tiles).
// Test hook for the persistent kernel's bounded dependency waits: two
// matrices 2I of order 128 (leaf 64) whose first level product is made to
// wait for a task count nothing reaches, every wait limited to limit_ms.
// The wait runs out, the kernel records SPIN_ERR_TIMEOUT, every later task
// skips its work and the launch ends.  Writes both matrices' statuses.
extern "C" int spin_test_persistent_timeout(double limit_ms, int* status0, int* status1) {
    if (!(limit_ms > 0.0) || limit_ms > 4000.0 || status0 == nullptr || status1 == nullptr)
        return SPIN_ERR_INVALID_ARG;
    constexpr int64_t n = 128, leaf = 64;
    constexpr int count = 2;
    Bucket b;
    b.n = n;
    b.leaf = leaf;
    b.count = count;
    b.first = 0;
    std::vector<Bucket> buckets(1, b);
    std::vector<PStage> st;
    std::vector<int64_t> start;
    order_stages(buckets, st, start);
    if (st.size() < 2 || st[1].kind != PSTAGE_PRODUCT) return SPIN_ERR_CUDA;
    st[1].need += 1 << 30;  // the first product waits for a count nothing reaches
    const size_t nn = (size_t)n * n, ws = fp64_workspace_elems(n, leaf);
    const size_t done_bytes = align256(count * sizeof(unsigned));
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = align256(off + bytes);
        return o;
    };
    const size_t o_a = take(count * nn * 8), o_x = take(count * nn * 8), o_w = take(count * ws * 8),
                 o_ptr = take(4 * count * 8), o_rec = take(count * INFO_WORDS * 4), o_ctl = take(done_bytes + 256),
                 o_st = take(st.size() * sizeof(PStage)), o_start = take(start.size() * 8);
    unsigned char* d = nullptr;
    if (cudaMalloc(&d, off) != cudaSuccess) {
        cudaGetLastError();
        return SPIN_ERR_OOM;
    }
    int rc = SPIN_OK;
    {
        std::vector<double> A(count * nn, 0.0);
        for (int z = 0; z < count; z++)
            for (int64_t i = 0; i < n; i++) A[z * nn + (size_t)i * n + i] = 2.0;
        std::vector<uint64_t> ptr(4 * count);
        for (int z = 0; z < count; z++) {
            ptr[z] = (uint64_t)(uintptr_t)(d + o_a + z * nn * 8);
            ptr[count + z] = (uint64_t)n;
            ptr[2 * count + z] = (uint64_t)(uintptr_t)(d + o_x + z * nn * 8);
            ptr[3 * count + z] = (uint64_t)(uintptr_t)(d + o_w + z * ws * 8);
        }
        cudaError_t e = cudaMemcpy(d + o_a, A.data(), A.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d + o_ptr, ptr.data(), ptr.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d + o_st, st.data(), st.size() * sizeof(PStage), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(d + o_start, start.data(), start.size() * 8, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemset(d + o_rec, 0, count * INFO_WORDS * 4);
        if (e == cudaSuccess) e = cudaMemset(d + o_ctl, 0, done_bytes + 256);
        if (e != cudaSuccess) {
            record_cuda_error(e, "persistent timeout test set-up", __FILE__, __LINE__);
            cudaGetLastError();
            rc = SPIN_ERR_CUDA;
        }
    }
    if (rc == SPIN_OK) {
        PersistentArgs a;
        a.stages = (const PStage*)(d + o_st);
        a.start = (const int64_t*)(d + o_start);
        a.nstages = (int)st.size();
        a.a_base = (const double* const*)(d + o_ptr);
        a.a_ld = (const int64_t*)(d + o_ptr + count * 8);
        a.x_base = (double* const*)(d + o_ptr + 2 * count * 8);
        a.w_base = (double* const*)(d + o_ptr + 3 * count * 8);
        a.records = (int32_t*)(d + o_rec);
        a.done = (unsigned*)(d + o_ctl);
        a.next = (unsigned long long*)(d + o_ctl + done_bytes);
        a.err = (int*)(d + o_ctl + done_bytes + 8);
        a.limit_ns = (uint64_t)(limit_ms * 1e6);
        a.bucket_clocks = nullptr;
        const size_t smem = persistent_smem_bytes(leaf);
        int grid = 0;
        rc = persistent_grid(smem, start.back(), &grid);
        if (rc == SPIN_OK) rc = launch_persistent_batch(a, smem, std::min(grid, 4), 0);
        int32_t rec[count * INFO_WORDS] = {};
        if (rc == SPIN_OK) {
            cudaError_t e = cudaMemcpy(rec, d + o_rec, sizeof rec, cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) {
                record_cuda_error(e, "persistent timeout test result", __FILE__, __LINE__);
                cudaGetLastError();
                rc = SPIN_ERR_CUDA;
            }
        }
        *status0 = rec[INFO_STATUS];
        *status1 = rec[INFO_WORDS + INFO_STATUS];
    }
    cudaFree(d);
    return rc;
}

extern "C" int spin_batch_schedule_info(const int64_t* n, int count, int leaf, int64_t* stages, int64_t* tasks,
                                        int64_t* leaves, int64_t* products, double* flops) {
    if (n == nullptr || count < 1 || count > 65535 || leaf < 0 || leaf > kPersistMaxLeaf) return SPIN_ERR_INVALID_ARG;
    std::vector<int64_t> sorted(n, n + count);
    for (int64_t v : sorted)
        if (v < 1 || v > 65536) return SPIN_ERR_INVALID_ARG;
    std::stable_sort(sorted.begin(), sorted.end());
    std::vector<Bucket> buckets;
    for (int i = 0; i < count;) {
        int j = i;
        while (j < count && sorted[j] == sorted[i]) j++;
        Bucket b;
        b.n = sorted[i];
        b.leaf = std::min(batched_leaf(b.n, leaf, SPIN_FP64), kPersistMaxLeaf);
        b.tile_cap = persist_tile_cap(b.n);
        b.count = j - i;
        b.first = i;
        buckets.push_back(b);
        i = j;
    }
    std::vector<PStage> st;
    std::vector<int64_t> start;
    order_stages(buckets, st, start);
    std::map<int, int64_t> seen;  // bucket first -> tasks of its stages so far
    std::map<int, int> last_leaf;
    int64_t nl = 0, np = 0;
    double fl = 0.0;
    for (size_t i = 0; i < st.size(); i++) {
        const PStage& x = st[i];
        if (start[i + 1] - start[i] != (int64_t)x.count * x.tiles) return SPIN_ERR_CUDA;
        if (x.need != seen[x.first]) return SPIN_ERR_CUDA;
        seen[x.first] += x.tiles;
        if (x.kind == PSTAGE_LEAF) {
            if (x.m > kPersistMaxLeaf || x.leaf_index != last_leaf[x.first]) return SPIN_ERR_CUDA;
            last_leaf[x.first]++;
            nl += x.count;
            fl += 2.0 * (double)x.m * (double)x.m * (double)x.m * x.count;
        } else {
            np += x.count;
            fl += 2.0 * (double)x.m * (double)x.n * (double)x.k * x.count;
        }
    }
    if (stages) *stages = (int64_t)st.size();
    if (tasks) *tasks = start.back();
    if (leaves) *leaves = nl;
    if (products) *products = np;
    if (flops) *flops = fl;
    return SPIN_OK;
}

// The persistent task list itself, for host-side checks: per stage (task
// order) five int64 -- kind (0 leaf, 1 product), first matrix (sorted
// order), matrices, tasks per matrix, dependency count -- into out (5 *
// max_stages entries); *stages gets the stage count (SPIN_ERR_INVALID_ARG
// if above max_stages, with nothing written).
extern "C" int spin_batch_schedule_stages(const int64_t* n, int count, int leaf, int64_t* out, int64_t max_stages,
                                          int64_t* stages) {
    if (n == nullptr || out == nullptr || stages == nullptr || count < 1 || count > 65535 || leaf < 0 ||
        leaf > kPersistMaxLeaf)
        return SPIN_ERR_INVALID_ARG;
    std::vector<int64_t> sorted(n, n + count);
    for (int64_t v : sorted)
        if (v < 1 || v > 65536) return SPIN_ERR_INVALID_ARG;
    std::stable_sort(sorted.begin(), sorted.end());
    std::vector<Bucket> buckets;
    for (int i = 0; i < count;) {
        int j = i;
        while (j < count && sorted[j] == sorted[i]) j++;
        Bucket b;
        b.n = sorted[i];
        b.leaf = std::min(batched_leaf(b.n, leaf, SPIN_FP64), kPersistMaxLeaf);
        b.tile_cap = persist_tile_cap(b.n);
        b.count = j - i;
        b.first = i;
        buckets.push_back(b);
        i = j;
    }
    std::vector<PStage> st;
    std::vector<int64_t> start;
    order_stages(buckets, st, start);
    *stages = (int64_t)st.size();
    if ((int64_t)st.size() > max_stages) return SPIN_ERR_INVALID_ARG;
    for (size_t i = 0; i < st.size(); i++) {
        out[5 * i + 0] = st[i].kind;
        out[5 * i + 1] = st[i].first;
        out[5 * i + 2] = st[i].count;
        out[5 * i + 3] = st[i].tiles;
        out[5 * i + 4] = st[i].need;
    }
    return SPIN_OK;
}

extern "C" int spin_invert_batched(const double* const* A, const int64_t* lda, double* const* X, const int64_t* n,
                                   int count, const spin_opts* opts, int* info_dev, spin_stream_t stream) {
    if (count < 1 || A == nullptr || lda == nullptr || X == nullptr || n == nullptr) return SPIN_ERR_INVALID_ARG;
    spin_opts o = opts ? *opts : spin_opts_default();
    if (o.precision != SPIN_FP64 && o.precision != SPIN_MIXED_BF16X3) return SPIN_ERR_NOT_IMPLEMENTED;
    if (o.pretransform != 0) return SPIN_ERR_NOT_IMPLEMENTED;  // the batch has no butterfly transform
    const bool mixed = o.precision != SPIN_FP64;
    if (o.leaf < 0 || o.schedule < SPIN_SCHEDULE_DEFAULT || o.schedule > SPIN_SCHEDULE_PERSISTENT)
        return SPIN_ERR_INVALID_ARG;
    if (!mixed && o.schedule == SPIN_SCHEDULE_PERSISTENT && o.leaf > kPersistMaxLeaf) return SPIN_ERR_INVALID_ARG;
    if (mixed && (o.residual_slices < 0 || o.residual_slices > 7 || o.max_refine < 0 || !(o.tol > 0.0) ||
                  o.fp64_levels < 0))
        return SPIN_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++) {
        if (n[i] < 1 || n[i] > 65536 || lda[i] < n[i] || A[i] == nullptr || X[i] == nullptr) return SPIN_ERR_INVALID_ARG;
        if (((uintptr_t)A[i] & 7u) || ((uintptr_t)X[i] & 7u)) return SPIN_ERR_INVALID_ARG;
        if (batched_leaf(n[i], o.leaf, o.precision) > kMaxLeaf) return SPIN_ERR_INVALID_ARG;
    }
    if (count > 65535) return SPIN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchPlan& p = g_plans[s];
    std::vector<uint64_t> key = make_key(A, lda, X, n, count, o);
    if (p.exec == nullptr || key != p.key) {
        int rc = build_plan(p, A, lda, X, n, count, o, s);
        if (rc != SPIN_OK) {
            free_plan(p);
            p.key.clear();
            return rc;
        }
        p.key = key;
    }
    SPIN_CUDA_TRY(cudaGraphLaunch(p.exec, s));
    p.kernels = p.graph_kernels;
    // statuses go to the caller's array outside the graph, so that a new
    // info_dev does not force a new capture
    if (info_dev != nullptr) {
        p.kernels++;
        scatter_status_kernel<<<(count + 255) / 256, 256, 0, s>>>(p.records, p.user_index, count, info_dev);
        SPIN_CUDA_TRY(cudaGetLastError());
    }
    if (o.blocking) SPIN_CUDA_TRY(cudaStreamSynchronize(s));
    return SPIN_OK;
}

extern "C" int spin_batched_refine_info(spin_stream_t stream, int* refine_iters, double* worst_rel) {
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_plans.find((cudaStream_t)stream);
    if (it == g_plans.end() || it->second.exec == nullptr) return SPIN_ERR_INVALID_ARG;
    const BatchPlan& p = it->second;
    int most = 0;
    double worst = -1.0;
    if (p.precision != SPIN_FP64 && p.count > 0) {
        SPIN_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
        std::vector<double> rel(p.count);
        std::vector<int> its(p.count);
        SPIN_CUDA_TRY(cudaMemcpy(rel.data(), p.rel, p.count * sizeof(double), cudaMemcpyDeviceToHost));
        SPIN_CUDA_TRY(cudaMemcpy(its.data(), p.iters, p.count * sizeof(int), cudaMemcpyDeviceToHost));
        worst = 0.0;
        for (int z = 0; z < p.count; z++) {
            most = std::max(most, its[z]);
            if (rel[z] == rel[z]) worst = std::max(worst, rel[z]);  // NaN: a matrix whose leaf failed
        }
    }
    if (refine_iters) *refine_iters = most;
    if (worst_rel) *worst_rel = worst;
    return SPIN_OK;
}

extern "C" int spin_batched_stats(spin_stream_t stream, int* kernels, int* buckets) {
    std::lock_guard<std::mutex> lk(g_bmu);
    auto it = g_plans.find((cudaStream_t)stream);
    if (it == g_plans.end() || it->second.exec == nullptr) return SPIN_ERR_INVALID_ARG;
    if (kernels) *kernels = it->second.kernels;
    if (buckets) *buckets = (int)it->second.buckets.size();
    return SPIN_OK;
}

namespace spin {
namespace {

// Seeded strictly diagonally dominant matrices for the autotuner: entry
// (z, i, j) = U(-1, 1) from splitmix64 of its position, plus n on the diagonal.
__global__ void synth_batch_kernel(double* A, int64_t n, int64_t count, uint64_t seed) {
    const int64_t total = n * n * count;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t x = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;
        x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
        x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
        x ^= x >> 31;
        double v = 2.0 * (double)(x >> 11) * 0x1.0p-53 - 1.0;
        const int64_t e = i % (n * n);
        if (e / n == e % n) v += (double)n;
        A[i] = v;
    }
}

// A whole plain batch on the persistent kernel with given per-bucket leaves
// and tile caps (matrix z of the sorted order at A[z], result to X[z],
// leading dimension n), the device memory kept across runs; per-bucket SM
// clocks accumulate into clocks_dev when it is given.
struct PersistBatchRun {
    unsigned char* d = nullptr;
    size_t bytes = 0;
    ~PersistBatchRun() { cudaFree(d); }

    int run(const std::vector<Bucket>& buckets, const std::vector<const double*>& A, const std::vector<double*>& X,
            unsigned long long* clocks_dev, cudaStream_t s) {
        std::vector<PStage> st;
        std::vector<int64_t> start;
        order_stages(buckets, st, start);
        const size_t c = A.size();
        std::vector<size_t> wsoff(c);
        size_t ws_total = 0;
        int64_t max_leaf = 1;
        for (const Bucket& b : buckets) {
            const size_t w = std::max<size_t>(fp64_workspace_elems(b.n, b.leaf), 1);
            for (int z = 0; z < b.count; z++) {
                wsoff[b.first + z] = ws_total;
                ws_total += w;
            }
            max_leaf = std::max(max_leaf, std::min(b.leaf, b.n));
        }
        const size_t done_bytes = align256(c * sizeof(unsigned));
        size_t off = 0;
        auto take = [&](size_t by) {
            const size_t o = off;
            off = align256(off + by);
            return o;
        };
        const size_t o_w = take(ws_total * 8), o_ptr = take(4 * c * 8), o_rec = take(c * INFO_WORDS * 4),
                     o_ctl = take(done_bytes + 256), o_st = take(st.size() * sizeof(PStage)),
                     o_start = take(start.size() * 8);
        if (off > bytes) {
            cudaFree(d);
            d = nullptr;
            bytes = 0;
            if (cudaMalloc(&d, off) != cudaSuccess) {
                cudaGetLastError();
                return SPIN_ERR_OOM;
            }
            bytes = off;
        }
        std::vector<uint64_t> ptr(4 * c);
        for (size_t z = 0; z < c; z++) {
            ptr[z] = (uint64_t)(uintptr_t)A[z];
            ptr[2 * c + z] = (uint64_t)(uintptr_t)X[z];
            ptr[3 * c + z] = (uint64_t)(uintptr_t)(d + o_w + wsoff[z] * 8);
        }
        for (const Bucket& b : buckets)
            for (int z = 0; z < b.count; z++) ptr[c + b.first + z] = (uint64_t)b.n;
        SPIN_CUDA_TRY(cudaMemcpyAsync(d + o_ptr, ptr.data(), ptr.size() * 8, cudaMemcpyHostToDevice, s));
        SPIN_CUDA_TRY(cudaMemcpyAsync(d + o_st, st.data(), st.size() * sizeof(PStage), cudaMemcpyHostToDevice, s));
        SPIN_CUDA_TRY(cudaMemcpyAsync(d + o_start, start.data(), start.size() * 8, cudaMemcpyHostToDevice, s));
        SPIN_CUDA_TRY(cudaMemsetAsync(d + o_rec, 0, c * INFO_WORDS * 4, s));
        SPIN_CUDA_TRY(cudaMemsetAsync(d + o_ctl, 0, done_bytes + 256, s));
        SPIN_CUDA_TRY(cudaStreamSynchronize(s));  // the host vectors must outlive the copies
        PersistentArgs a;
        a.stages = (const PStage*)(d + o_st);
        a.start = (const int64_t*)(d + o_start);
        a.nstages = (int)st.size();
        a.a_base = (const double* const*)(d + o_ptr);
        a.a_ld = (const int64_t*)(d + o_ptr + c * 8);
        a.x_base = (double* const*)(d + o_ptr + 2 * c * 8);
        a.w_base = (double* const*)(d + o_ptr + 3 * c * 8);
        a.records = (int32_t*)(d + o_rec);
        a.done = (unsigned*)(d + o_ctl);
        a.next = (unsigned long long*)(d + o_ctl + done_bytes);
        a.err = (int*)(d + o_ctl + done_bytes + 8);
        a.limit_ns = kPersistWaitNs;
        a.bucket_clocks = clocks_dev;
        const size_t smem = persistent_smem_bytes(max_leaf);
        int grid = 0;
        BRET(persistent_grid(smem, start.back(), &grid));
        return launch_persistent_batch(a, smem, grid, s);
    }
};

}  // namespace
}  // namespace spin

// The autotuner of the persistent schedule (plain batches), per order
// bucket in the context of the whole batch: one batch of the given orders
// (seeded strictly diagonally dominant matrices) runs on the persistent
// kernel once per candidate pair of leaf (<= 64) and largest product tile
// (64, 32 or 16), the pair applied to every bucket, after a warm-up run;
// the kernel adds the SM clocks of each task to its bucket's counter, and
// each bucket takes the pair under which its tasks took the fewest clocks
// (the schedule's makespan is about the sum of the task times over the
// CTAs, so a bucket's task time is its share of it), if that beats the
// library's own pair (leaf 64, tile 64) by 2 %.  A bucket timed alone
// would instead favour small tiles that fill the GPU by themselves.
extern "C" int spin_autotune_batched_persistent(const int64_t* orders, int count, const int* leaves, int nleaf,
                                                const int* tiles, int ntile, int* leaf_out, int* tile_out,
                                                double* ms_out, spin_stream_t stream) {
    using namespace spin;
    if (orders == nullptr || count < 1 || count > 65535 || nleaf < 1 || ntile < 1 || leaves == nullptr ||
        tiles == nullptr || leaf_out == nullptr || tile_out == nullptr)
        return SPIN_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++)
        if (orders[i] < 1 || orders[i] > 65536) return SPIN_ERR_INVALID_ARG;
    for (int i = 0; i < nleaf; i++)
        if (leaves[i] < 1 || leaves[i] > kPersistMaxLeaf) return SPIN_ERR_INVALID_ARG;
    for (int i = 0; i < ntile; i++)
        if (tiles[i] != 16 && tiles[i] != 32 && tiles[i] != 64) return SPIN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::map<int64_t, int> mult;
    for (int i = 0; i < count; i++) mult[orders[i]]++;
    std::vector<Bucket> buckets;
    size_t elems = 0;
    int first = 0;
    for (const auto& kv : mult) {
        Bucket b;
        b.n = kv.first;
        b.count = kv.second;
        b.first = first;
        b.leaf = 1;
        first += kv.second;
        elems += (size_t)kv.second * (size_t)b.n * (size_t)b.n;
        buckets.push_back(b);
    }
    const size_t nb = buckets.size();
    double* A = nullptr;
    double* X = nullptr;
    unsigned long long* clk = nullptr;
    if (cudaMalloc(&A, elems * sizeof(double)) != cudaSuccess || cudaMalloc(&X, elems * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&clk, nb * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(A);
        cudaFree(X);
        return SPIN_ERR_OOM;
    }
    std::vector<const double*> ap(count);
    std::vector<double*> xp(count);
    {
        size_t off = 0;
        for (const Bucket& b : buckets) {
            const size_t nn = (size_t)b.n * (size_t)b.n;
            synth_batch_kernel<<<1024, 256, 0, s>>>(A + off, b.n, b.count, 0x5EEDBA7Cull + (uint64_t)b.n);
            for (int z = 0; z < b.count; z++) {
                ap[b.first + z] = A + off + z * nn;
                xp[b.first + z] = X + off + z * nn;
            }
            off += (size_t)b.count * nn;
        }
    }
    int rc = SPIN_OK;
    {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            record_cuda_error(e, "autotuner inputs", __FILE__, __LINE__);
            rc = SPIN_ERR_CUDA;
        }
    }
    std::vector<unsigned long long> best_clk(nb, ~0ull), ref_clk(nb, ~0ull), h(nb);
    std::vector<int64_t> best_leaf(nb, 0), ref_leaf(nb, 0);
    std::vector<int> best_tile(nb, 0), ref_tile(nb, 0);
    std::vector<std::pair<int, int>> tried;
    PersistBatchRun runner;
    for (int li = 0; li < nleaf && rc == SPIN_OK; li++)
        for (int ti = 0; ti < ntile && rc == SPIN_OK; ti++) {
            const std::pair<int, int> key(leaves[li], tiles[ti]);
            if (std::find(tried.begin(), tried.end(), key) != tried.end()) continue;
            tried.push_back(key);
            for (Bucket& b : buckets) {
                b.leaf = std::min<int64_t>(leaves[li], b.n);
                b.tile_cap = tiles[ti];
            }
            // a warm-up run, then two counted ones (each bucket keeps its smaller count)
            std::vector<unsigned long long> m(nb, ~0ull);
            for (int rep = 0; rep < 3 && rc == SPIN_OK; rep++) {
                if (cudaMemsetAsync(clk, 0, nb * sizeof(unsigned long long), s) != cudaSuccess) rc = SPIN_ERR_CUDA;
                if (rc == SPIN_OK) rc = runner.run(buckets, ap, xp, clk, s);
                if (rc == SPIN_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = SPIN_ERR_CUDA;
                if (rc == SPIN_OK && rep > 0) {
                    if (cudaMemcpy(h.data(), clk, nb * sizeof(unsigned long long), cudaMemcpyDeviceToHost) !=
                        cudaSuccess)
                        rc = SPIN_ERR_CUDA;
                    for (size_t i = 0; i < nb && rc == SPIN_OK; i++) m[i] = std::min(m[i], h[i]);
                }
            }
            if (rc != SPIN_OK) break;
            // the library's own pair (leaf 64, tile 64), or else the first one, is the
            // reference; another pair must beat it by 2 % (task clocks vary by about
            // 1 % between runs, as the buckets share the SMs)
            const bool is_ref = tried.size() == 1 || (leaves[li] == kPersistMaxLeaf && tiles[ti] == 64);
            for (size_t i = 0; i < nb; i++) {
                if (is_ref) {
                    ref_clk[i] = m[i];
                    ref_leaf[i] = buckets[i].leaf;
                    ref_tile[i] = tiles[ti];
                }
                if (m[i] < best_clk[i]) {
                    best_clk[i] = m[i];
                    best_leaf[i] = buckets[i].leaf;
                    best_tile[i] = tiles[ti];
                }
            }
        }
    for (size_t i = 0; i < nb && rc == SPIN_OK; i++)
        if (!((double)best_clk[i] < 0.98 * (double)ref_clk[i])) {
            best_clk[i] = ref_clk[i];
            best_leaf[i] = ref_leaf[i];
            best_tile[i] = ref_tile[i];
        }
    int dev = 0, khz = 0;
    if (rc == SPIN_OK && (cudaGetDevice(&dev) != cudaSuccess ||
                          cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0))
        rc = SPIN_ERR_CUDA;
    cudaFree(A);
    cudaFree(X);
    cudaFree(clk);
    if (rc != SPIN_OK) {
        cudaGetLastError();
        return rc;
    }
    std::map<int64_t, size_t> index;
    {
        std::lock_guard<std::mutex> lk(g_bleaf_mu);
        for (size_t i = 0; i < nb; i++) {
            index[buckets[i].n] = i;
            g_bleaf[std::make_pair((int)SPIN_FP64, buckets[i].n)] = best_leaf[i];
            g_btile[buckets[i].n] = best_tile[i];
        }
        g_bleaf_gen++;
    }
    for (int i = 0; i < count; i++) {
        const size_t b = index[orders[i]];
        leaf_out[i] = (int)best_leaf[b];
        tile_out[i] = best_tile[b];
        if (ms_out) ms_out[i] = (double)best_clk[b] / (double)khz;
    }
    return SPIN_OK;
}

// Batched leaf autotuning: for every distinct order of `orders` (with its
// multiplicity in the list, i.e. the bucket that order forms in a batch), one
// lockstep run of the bucket per candidate leaf on seeded diagonally
// dominant matrices, after a warm-up run; the fastest is recorded for
// (precision, order) and used by spin_invert_batched when opts.leaf is 0.
extern "C" int spin_autotune_batched_leaf(const int64_t* orders, int count, int precision, const int* candidates,
                                          int ncand, int* leaf_out, double* ms_out, spin_stream_t stream) {
    using namespace spin;
    if (orders == nullptr || count < 1 || ncand < 0 || (ncand > 0 && candidates == nullptr) || leaf_out == nullptr)
        return SPIN_ERR_INVALID_ARG;
    if (precision != SPIN_FP64 && precision != SPIN_MIXED_BF16X3) return SPIN_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++)
        if (orders[i] < 1 || orders[i] > 65536) return SPIN_ERR_INVALID_ARG;
    if (ncand == 0) {  // forget the records of these orders
        {
            std::lock_guard<std::mutex> lk(g_bleaf_mu);
            for (int i = 0; i < count; i++) {
                g_bleaf.erase(std::make_pair(precision, orders[i]));
                if (precision == SPIN_FP64) g_btile.erase(orders[i]);
            }
            g_bleaf_gen++;
        }
        for (int i = 0; i < count; i++) {
            leaf_out[i] = (int)batched_leaf(orders[i], 0, precision);
            if (ms_out) ms_out[i] = -1.0;
        }
        return SPIN_OK;
    }
    cudaStream_t s = (cudaStream_t)stream;
    std::map<int64_t, int> mult;
    for (int i = 0; i < count; i++) mult[orders[i]]++;
    spin_opts o = spin_opts_default();
    o.precision = precision;
    std::map<int64_t, std::pair<int64_t, double>> chosen;  // order -> (leaf, ms)
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    SPIN_CUDA_TRY(cudaEventCreate(&e0));
    SPIN_CUDA_TRY(cudaEventCreate(&e1));
    int rc = SPIN_OK;
    for (const auto& kv : mult) {
        const int64_t n = kv.first;
        const int k = std::min(kv.second, 65535);
        double* A = nullptr;
        double* X = nullptr;
        void* host = nullptr;
        const size_t nn = (size_t)n * (size_t)n;
        if (cudaMalloc(&A, nn * k * sizeof(double)) != cudaSuccess || cudaMalloc(&X, nn * k * sizeof(double)) != cudaSuccess ||
            cudaMallocHost(&host, bucket_host_bytes(k)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(A);
            cudaFree(X);
            rc = SPIN_ERR_OOM;
            break;
        }
        synth_batch_kernel<<<1024, 256, 0, s>>>(A, n, k, 0x5EEDBA7Cull + (uint64_t)n);
        std::vector<const double*> ap(k);
        std::vector<int64_t> ld(k, n);
        std::vector<double*> xp(k);
        for (int z = 0; z < k; z++) {
            ap[z] = A + (size_t)z * nn;
            xp[z] = X + (size_t)z * nn;
        }
        int64_t best = 0;
        double best_ms = 1e300;
        std::vector<int64_t> tried;
        for (int c = 0; c < ncand && rc == SPIN_OK; c++) {
            const int64_t L = std::min<int64_t>(candidates[c], n);
            if (candidates[c] < 1 || L > kMaxLeaf || std::find(tried.begin(), tried.end(), L) != tried.end()) continue;
            tried.push_back(L);
            o.leaf = (int)L;
            const size_t wsb = bucket_bytes(n, k, o);
            void* ws = nullptr;
            if (cudaMalloc(&ws, wsb) != cudaSuccess) {
                cudaGetLastError();
                rc = SPIN_ERR_OOM;
                break;
            }
            float ms = 0.f;
            for (int rep = 0; rep < 2 && rc == SPIN_OK; rep++) {  // warm-up, then timed
                if (rep == 1) cudaEventRecord(e0, s);
                rc = run_bucket(ap.data(), ld.data(), xp.data(), nullptr, n, k, o, ws, wsb, host, s);
                if (rep == 1) cudaEventRecord(e1, s);
                if (rc == SPIN_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = SPIN_ERR_CUDA;
            }
            if (rc == SPIN_OK) cudaEventElapsedTime(&ms, e0, e1);
            cudaFree(ws);
            if (rc == SPIN_OK && ms < best_ms) {
                best_ms = ms;
                best = L;
            }
        }
        cudaFree(A);
        cudaFree(X);
        cudaFreeHost(host);
        if (rc != SPIN_OK) break;
        if (best > 0) chosen[n] = std::make_pair(best, best_ms);
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != SPIN_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_bleaf_mu);
        for (const auto& kv : chosen) g_bleaf[std::make_pair(precision, kv.first)] = kv.second.first;
        g_bleaf_gen++;
    }
    for (int i = 0; i < count; i++) {
        auto it = chosen.find(orders[i]);
        leaf_out[i] = it == chosen.end() ? 0 : (int)it->second.first;
        if (ms_out) ms_out[i] = it == chosen.end() ? -1.0 : it->second.second;
    }
    return SPIN_OK;
}
