// C ABI and recursion driver (include/spin.h).
//
// The recursion of Algorithm 1 (Sec. 3.1) / Algorithm 2 (Sec. 3.3) is run
// on the host as a sequence of kernel launches over strided views of three
// device buffers: the read-only input A, the output X and a workspace W.
// The paper's breakMat / xy (Alg. 3, 4) become pointer arithmetic and its
// arrange (Alg. 6) disappears because every quadrant is written in place.
// Per internal node, with n1 = split(n), n2 = n - n1, T a n1 x n2 (later
// n2 x n1) slab of W and S a n2 x n2 slab after it:
//
//   X11 <- inv(A11)                       I                  (recursion)
//   T   <- X11 A12                        III = I A12
//   S   <- A22 - A21 T                    S = -V = A22 - IV  (subtract fused)
//   X22 <- inv(S)                         inv(-V) = -VI = C22 (scalarMul folded)
//   X12 <- -T X22                         C12 = III VI
//   T   <- A21 X11                        II = A21 I
//   X21 <- -X22 T                         C21 = VI II
//   X11 <- X11 - X12 T                    C11 = I - VII, VII = III C21 = C12 II
//
// so the six products and two subtractions of each level are six fused
// GEMM launches, and the only memory beyond A and X is W with
// ws(n) = max(ws(n1), n1 n2 + n2^2 + ws(n2)) elements (2n^2/3 for n = 2^p).
// For the plain method at orders up to 8192 the schedule is a small DAG
// instead of a sequence: II = A21 I (which needs only I) runs on a second
// stream beside III, S and the recursion on S, and C21, C11 wait for it;
// II then has its own slab of W (n^2 elements for n = 2^p).
#include <cuda_runtime.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "mixed.h"
#include "tc_gemm.h"

namespace spin {

static thread_local std::string g_last_error;


void record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
}

int64_t split_order(int64_t n) { return n > 64 ? 32 * ((n + 63) / 64) : (n + 1) / 2; }

// Workspace of the plain recursion: T (n1 x n2) and S (n2 x n2) per node,
// plus, in the overlapped schedule, II (n2 x n1) so that II = A21 I can run
// beside the recursion on S.
static size_t ws_fp64_elems(int64_t n, int64_t leaf, bool overlap = false) {
    if (n <= leaf) return leaf_scratch_elems(n);
    const int64_t n1 = split_order(n), n2 = n - n1;
    const size_t a = ws_fp64_elems(n1, leaf, overlap);
    const size_t b = (size_t)(n1 * n2 + n2 * n2) + (overlap ? (size_t)(n2 * n1) : 0) + ws_fp64_elems(n2, leaf, overlap);
    return a > b ? a : b;
}

// II = A21 I runs on a second stream, beside the recursion on S (which
// depends only on III = I A12), for problems up to these orders: there the
// leaves (one cluster of at most 16 SMs) and the small products leave SMs
// idle.  Above them the products fill the GPU and the schedule stays on one
// stream.  spin_opts.schedule 1 keeps every order on one stream, 2 takes
// the second stream at every order.
constexpr int64_t kOverlapMaxN = 8192;        // plain method
constexpr int64_t kOverlapMaxNMixed = 16384;  // mixed forms
bool overlap_schedule(int64_t n, int precision, int schedule) {
    if (schedule == SPIN_SCHEDULE_LOCKSTEP) return false;
    if (schedule == SPIN_SCHEDULE_PERSISTENT) return true;
    return n <= (precision == SPIN_FP64 ? kOverlapMaxN : kOverlapMaxNMixed);
}

namespace {

struct ProfEntry {
    spin_prof_record rec;
    cudaEvent_t start, stop;
    int gate_slot;  // >= 0: the launch ran only if flags[gate_slot] != 0
};

struct Profiler {
    bool on = false;
    int max_records = 0;
    std::vector<ProfEntry> entries;
    std::vector<cudaEvent_t> pool;
    // Refinement launches are gated on the device by a matrix's active flag;
    // a copy of the flag taken just before each gated launch (device int per
    // record) tells profile_stop which ones did the work they describe.
    int* flags = nullptr;
    int flags_cap = 0;

    cudaEvent_t event() {
        if (!pool.empty()) {
            cudaEvent_t e = pool.back();
            pool.pop_back();
            return e;
        }
        cudaEvent_t e = nullptr;
        cudaEventCreate(&e);
        return e;
    }
};

// Device status block of a stream (32 bytes, pinned mirror on the host):
// int32 info record [status, leaf, column, spare], then the refinement's
// active flag, iteration count and last relative residual.
constexpr int CTL_ACTIVE = INFO_WORDS, CTL_ITERS = INFO_WORDS + 1, CTL_REL = INFO_WORDS + 2;  // int32 offsets
constexpr size_t CTL_BYTES = 32;

struct StreamState {
    Profiler prof;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t side = nullptr;        // second stream of the overlapped schedule
    std::vector<cudaEvent_t> events;    // its fork / join events (one per use within a call)
    int32_t* info_dev = nullptr;   // CTL_BYTES: info record + refinement control
    int32_t* info_host = nullptr;  // pinned mirror
    double* hostA = nullptr;       // device staging for spin_invert_host
    double* hostX = nullptr;
    size_t host_elems = 0;
    int* err_dev = nullptr;        // device: tensor-core bounded-wait failures
    int last_mixed = 0;            // host: the latest call refined (mixed precision)
    int last_pretransformed = 0;   // host: the latest call went through the butterfly transform
    // The schedule as a CUDA graph: the previous call's arguments, and the
    // graph captured when a call repeated them (replayed while they repeat).
    std::vector<uint64_t> prev_key, graph_key;
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;    // private capture stream
    int graph_mixed = 0, graph_rbt = 0;
    int64_t graph_launches = 0;    // graph replays (host counter)
    int64_t graph_nodes = 0;       // nodes of the captured graph
    int* active() { return (int*)(info_dev + CTL_ACTIVE); }
    int* iters() { return (int*)(info_dev + CTL_ITERS); }
    double* rel() { return (double*)(info_dev + CTL_REL); }
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, StreamState> g_states;

int get_state(cudaStream_t s, StreamState** out) {
    int dev = 0;
    SPIN_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    StreamState& st = g_states[std::make_pair(dev, s)];
    if (st.info_dev == nullptr) {
        SPIN_CUDA_TRY(cudaMalloc(&st.info_dev, CTL_BYTES));
        SPIN_CUDA_TRY(cudaMemset(st.info_dev, 0, CTL_BYTES));
        SPIN_CUDA_TRY(cudaMallocHost(&st.info_host, CTL_BYTES));
        SPIN_CUDA_TRY(cudaMalloc(&st.err_dev, sizeof(int)));
        SPIN_CUDA_TRY(cudaMemset(st.err_dev, 0, sizeof(int)));
    }
    *out = &st;
    return SPIN_OK;
}

int ensure_ws(StreamState* st, size_t bytes) {
    if (bytes <= st->ws_bytes) return SPIN_OK;
    if (st->ws) {
        cudaFree(st->ws);
        st->ws = nullptr;
        st->ws_bytes = 0;
    }
    if (bytes == 0) return SPIN_OK;
    if (cudaMalloc(&st->ws, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SPIN_ERR_OOM;
    }
    st->ws_bytes = bytes;
    return SPIN_OK;
}

struct Run {
    cudaStream_t s;
    int32_t* info;
    int leaf_counter;
    int64_t leaf;
    Profiler* prof;  // nullptr when not recording
    // overlapped schedule: II and C21 on `side`, events from `events`
    cudaStream_t side = nullptr;
    std::vector<cudaEvent_t>* events = nullptr;
    size_t next_event = 0;
    // mixed precision only
    int precision = SPIN_FP64;
    int fp64_levels = 0;
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    void* side_scratch = nullptr;  // split arena of the side stream's products
    size_t side_scratch_bytes = 0;
    int* err = nullptr;
};


// Bracket one launch with events when the stream's profiler is on.  gate
// (optional, device int): the launch is gated on it; its value just before
// the launch is kept so that profile_stop can drop the flops and bytes of a
// launch that did nothing.
struct ProfScope {
    Profiler* p;
    cudaStream_t s;
    ProfEntry e;
    bool active;
    ProfScope(Profiler* prof, cudaStream_t st, int kind, int depth, int64_t m, int64_t n, int64_t k, double flops,
              double bytes, const int* gate = nullptr)
        : p(prof), s(st), active(prof != nullptr && prof->on && (int)prof->entries.size() < prof->max_records) {
        if (!active) return;
        e.rec = spin_prof_record{kind, depth, m, n, k, flops, bytes, 0.0};
        e.gate_slot = -1;
        if (gate != nullptr && p->flags != nullptr && (int)p->entries.size() < p->flags_cap) {
            e.gate_slot = (int)p->entries.size();
            cudaMemcpyAsync(p->flags + e.gate_slot, gate, sizeof(int), cudaMemcpyDeviceToDevice, s);
        }
        e.start = p->event();
        e.stop = p->event();
        cudaEventRecord(e.start, s);
    }
    ~ProfScope() {
        if (!active) return;
        cudaEventRecord(e.stop, s);
        p->entries.push_back(e);
    }
};

int gemm_f64_prof(Run& r, int depth, int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                  const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D, int64_t ldd) {
    const double flops = 2.0 * (double)m * (double)n * (double)k;
    const double bytes = 8.0 * ((double)m * k + (double)k * n + (double)m * n * (beta != 0.0 ? 2.0 : 1.0));
    ProfScope ps(r.prof, r.s, SPIN_KERNEL_GEMM_F64, depth, m, n, k, flops, bytes, nullptr);
    return launch_gemm_f64(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, r.s);
}

int leaf_prof(Run& r, int depth, const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, double* W) {
    ProfScope ps(r.prof, r.s, SPIN_KERNEL_LEAF, depth, n, n, 0, 2.0 * (double)n * n * n, 16.0 * (double)n * n);
    return launch_leaf_gj(A, lda, X, ldx, n, W, r.info, r.leaf_counter++, r.s);
}

#define RET(x)                        \
    do {                              \
        int _r = (x);                 \
        if (_r != SPIN_OK) return _r; \
    } while (0)

// One level product D = beta*C + alpha*(A B).  FP64 for the plain method
// (and for small products in mixed mode); in mixed mode bf16x3 on the
// tensor cores, or FP64-class digit slices for the Schur complement of the
// top fp64_levels levels.
// Smallest m and n a mixed-mode product takes to the tensor cores
// (SPIN_TC_MIN overrides it, for measurement; read once).
int64_t tc_min() {
    static int64_t v = -1;
    if (v < 0) {
        const char* e = getenv("SPIN_TC_MIN");
        const long long x = e ? atoll(e) : 0;
        v = x > 0 ? (int64_t)x : kTcMin;
    }
    return v;
}

int level_gemm(Run& r, int depth, bool schur, int64_t m, int64_t n, int64_t k, double alpha, const double* A,
               int64_t lda, const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D,
               int64_t ldd) {
    if (r.precision == SPIN_FP64 || m < tc_min() || n < tc_min() || k < 64)
        return gemm_f64_prof(r, depth, m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd);
    const double f = 2.0 * (double)m * (double)n * (double)k;
    SplitPlan sp;
    int rc;
    const bool fp64_schur = schur && depth < r.fp64_levels;
    if (fp64_schur || r.precision == SPIN_MIXED_DIGITS) {
        const int sl = fp64_schur ? kSchurSlices : kLevelSlices;
        RET(plan_ozaki(m, n, k, sl, r.scratch, r.scratch_bytes, &sp));
        {
            ProfScope ps(r.prof, r.s, SPIN_KERNEL_SPLIT, depth, m, k, 0, 0.0, 8.0 * m * k + 2.0 * sl * m * k);
            RET(split_a_ozaki(sp, A, lda, m, k, nullptr, r.s));
        }
        {
            ProfScope ps(r.prof, r.s, SPIN_KERNEL_SPLIT, depth, k, n, 0, 0.0, 8.0 * k * n + 2.0 * sl * k * n);
            RET(split_b_ozaki(sp, B, ldb, k, n, nullptr, r.s));
        }
        const int pairs = sl * (sl + 1) / 2;
        ProfScope ps(r.prof, r.s, SPIN_KERNEL_GEMM_TC, depth, m, n, k, pairs * f,
                     2.0 * sl * (m * k + k * n) + 8.0 * m * n * (beta != 0.0 ? 2 : 1));
        rc = product_ozaki(sp, m, n, k, alpha, beta, C, ldc, D, ldd, 0, nullptr, r.err, r.s);
        return rc;
    }
    RET(plan_bf16x3(m, n, k, r.scratch, r.scratch_bytes, &sp));
    {
        ProfScope ps(r.prof, r.s, SPIN_KERNEL_SPLIT, depth, m, k, 0, 0.0, 12.0 * m * k);
        RET(split_a_bf16x3(sp, A, lda, m, k, r.s));
    }
    {
        ProfScope ps(r.prof, r.s, SPIN_KERNEL_SPLIT, depth, k, n, 0, 0.0, 12.0 * k * n);
        RET(split_b_bf16x3(sp, B, ldb, k, n, r.s));
    }
    ProfScope ps(r.prof, r.s, SPIN_KERNEL_GEMM_TC, depth, m, n, k, 3.0 * f,
                 4.0 * (m * k + k * n) + 8.0 * m * n * (beta != 0.0 ? 2 : 1));
    return product_bf16x3(sp, m, n, k, alpha, beta, C, ldc, D, ldd, r.err, r.s);
}

// A fresh event for this call (created on first use, kept for later calls).
int take_event(Run& r, cudaEvent_t* e) {
    if (r.next_event == r.events->size()) {
        cudaEvent_t ne = nullptr;
        SPIN_CUDA_TRY(cudaEventCreateWithFlags(&ne, cudaEventDisableTiming));
        r.events->push_back(ne);
    }
    *e = (*r.events)[r.next_event++];
    return SPIN_OK;
}

int inv_rec(Run& r, int depth, const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, double* W) {
    if (n <= r.leaf) return leaf_prof(r, depth, A, lda, X, ldx, n, W);
    const int64_t n1 = split_order(n), n2 = n - n1;
    if (r.side != nullptr) {
        // Overlapped schedule: the same products on the same operands, so the
        // same values as the sequential one.  II = A21 I depends only on I:
        // it runs on the side stream from the moment I is done, beside
        // III, S and the whole recursion on S.  C21 = -C22 II needs C22 and
        // II only: it follows II on the side stream once C22 is done, beside
        // C12 and C11 (which write X12 and X11); the level ends when both
        // streams are through.
        const double* A11 = A;
        const double* A12 = A + n1;
        const double* A21 = A + n1 * lda;
        const double* A22 = A21 + n1;
        double* X11 = X;
        double* X12 = X + n1;
        double* X21 = X + n1 * ldx;
        double* X22 = X21 + n1;
        double* T = W;                  // III, n1 x n2
        double* S = W + n1 * n2;        // -V, n2 x n2
        double* II = S + n2 * n2;       // II, n2 x n1
        double* Wsub = II + n2 * n1;
        const int d = depth;
        RET(inv_rec(r, d + 1, A11, lda, X11, ldx, n1, W));                                          // I
        cudaEvent_t e_i = nullptr, e_ii = nullptr;
        RET(take_event(r, &e_i));
        RET(take_event(r, &e_ii));
        SPIN_CUDA_TRY(cudaEventRecord(e_i, r.s));
        SPIN_CUDA_TRY(cudaStreamWaitEvent(r.side, e_i, 0));
        {
            Run rs = r;  // II alone on the side stream (a product, no recursion)
            rs.s = r.side;
            rs.side = nullptr;
            rs.scratch = r.side_scratch;
            rs.scratch_bytes = r.side_scratch_bytes;
            RET(level_gemm(rs, d, false, n2, n1, n1, 1.0, A21, lda, X11, ldx, 0.0, nullptr, 0, II, n1));  // II
        }
        SPIN_CUDA_TRY(cudaEventRecord(e_ii, r.side));
        RET(level_gemm(r, d, false, n1, n2, n1, 1.0, X11, ldx, A12, lda, 0.0, nullptr, 0, T, n2));   // III
        RET(level_gemm(r, d, true, n2, n2, n1, -1.0, A21, lda, T, n2, 1.0, A22, lda, S, n2));       // -V
        RET(inv_rec(r, d + 1, S, n2, X22, ldx, n2, Wsub));                                        // C22
        cudaEvent_t e_c22 = nullptr, e_c21 = nullptr;
        RET(take_event(r, &e_c22));
        RET(take_event(r, &e_c21));
        SPIN_CUDA_TRY(cudaEventRecord(e_c22, r.s));
        SPIN_CUDA_TRY(cudaStreamWaitEvent(r.side, e_c22, 0));
        {
            Run rs = r;  // C21 on the side stream, after II
            rs.s = r.side;
            rs.side = nullptr;
            rs.scratch = r.side_scratch;
            rs.scratch_bytes = r.side_scratch_bytes;
            RET(level_gemm(rs, d, false, n2, n1, n2, -1.0, X22, ldx, II, n1, 0.0, nullptr, 0, X21, ldx));  // C21
        }
        SPIN_CUDA_TRY(cudaEventRecord(e_c21, r.side));
        RET(level_gemm(r, d, false, n1, n2, n2, -1.0, T, n2, X22, ldx, 0.0, nullptr, 0, X12, ldx)); // C12
        SPIN_CUDA_TRY(cudaStreamWaitEvent(r.s, e_ii, 0));
        RET(level_gemm(r, d, false, n1, n1, n2, -1.0, X12, ldx, II, n1, 1.0, X11, ldx, X11, ldx));  // C11
        SPIN_CUDA_TRY(cudaStreamWaitEvent(r.s, e_c21, 0));
        return SPIN_OK;
    }
    const double* A11 = A;
    const double* A12 = A + n1;
    const double* A21 = A + n1 * lda;
    const double* A22 = A21 + n1;
    double* X11 = X;
    double* X12 = X + n1;
    double* X21 = X + n1 * ldx;
    double* X22 = X21 + n1;
    double* T = W;
    double* S = W + n1 * n2;
    double* Wsub = S + n2 * n2;
    const int d = depth;
    RET(inv_rec(r, d + 1, A11, lda, X11, ldx, n1, W));                                         // I
    RET(level_gemm(r, d, false, n1, n2, n1, 1.0, X11, ldx, A12, lda, 0.0, nullptr, 0, T, n2));   // III
    RET(level_gemm(r, d, true, n2, n2, n1, -1.0, A21, lda, T, n2, 1.0, A22, lda, S, n2));       // -V
    RET(inv_rec(r, d + 1, S, n2, X22, ldx, n2, Wsub));                                        // C22
    RET(level_gemm(r, d, false, n1, n2, n2, -1.0, T, n2, X22, ldx, 0.0, nullptr, 0, X12, ldx)); // C12
    RET(level_gemm(r, d, false, n2, n1, n1, 1.0, A21, lda, X11, ldx, 0.0, nullptr, 0, T, n1));  // II
    RET(level_gemm(r, d, false, n2, n1, n2, -1.0, X22, ldx, T, n1, 0.0, nullptr, 0, X21, ldx)); // C21
    RET(level_gemm(r, d, false, n1, n1, n2, -1.0, X12, ldx, T, n1, 1.0, X11, ldx, X11, ldx));   // C11
    return SPIN_OK;
}

bool aligned8(const void* p) { return ((uintptr_t)p & 7u) == 0; }

bool overlaps(const double* a, int64_t lda, const double* x, int64_t ldx, int64_t n) {
    const char* a0 = (const char*)a;
    const char* a1 = (const char*)(a + (n - 1) * lda + n);
    const char* x0 = (const char*)x;
    const char* x1 = (const char*)(x + (n - 1) * ldx + n);
    return a0 < x1 && x0 < a1;
}

int64_t resolve_leaf(int64_t n, int leaf, int precision) {
    if (leaf < 0) return -1;
    int64_t L = leaf > 0 ? leaf : spin_default_leaf(n, precision);
    if (L > n) L = n;
    return L;
}

int check_common(const void* A, int64_t lda, const void* X, int64_t ldx, int64_t n, int64_t leaf) {
    if (n < 1 || lda < n || ldx < n) return SPIN_ERR_INVALID_ARG;
    if (A == nullptr || X == nullptr || !aligned8(A) || !aligned8(X)) return SPIN_ERR_INVALID_ARG;
    if (leaf < 1 || leaf > kMaxLeaf) return SPIN_ERR_INVALID_ARG;
    if (overlaps((const double*)A, lda, (const double*)X, ldx, n)) return SPIN_ERR_INVALID_ARG;
    return SPIN_OK;
}

int read_info(StreamState* st, cudaStream_t s, spin_info* info) {
    SPIN_CUDA_TRY(cudaMemcpyAsync(st->info_host, st->info_dev, CTL_BYTES, cudaMemcpyDeviceToHost, s));
    SPIN_CUDA_TRY(cudaStreamSynchronize(s));
    const int32_t* h = st->info_host;
    const int status = h[INFO_STATUS];
    if (info) {
        // a leaf's failure records the leaf and column; a refinement status -1, -1
        info->status = status;
        info->refine_iters = st->last_mixed ? h[CTL_ITERS] : 0;
        info->fail_leaf = status ? h[INFO_LEAF] : -1;
        info->fail_col = status ? h[INFO_COL] : -1;
        info->rel_residual = st->last_mixed ? *(const double*)(h + CTL_REL) : -1.0;
        info->pretransformed = st->last_pretransformed;
        info->reserved = 0;
    }
    return status;
}

// Workspace of the mixed-precision form: the FP64 recursion workspace (later
// reused for the residual R), the split arena, and the cached digit planes
// of A for the refinement residual.
struct MixLayout {
    size_t region0, scratch, apl, off_scratch, off_apl, off_norms, total;
    size_t side_scratch, off_side;  // split arena of the side stream (overlapped schedule), else 0
    int sr;  // digit slices of the certifying residuals (and of A's cached planes)
    int s0;  // slices of the first residual's pairs (<= sr)
};

size_t round256(size_t x) { return (x + 255) & ~(size_t)255; }

MixLayout mix_layout(int64_t n, int64_t leaf, const spin_opts& o) {
    MixLayout L;
    // 9-bit digits relative to the largest entry of each row (column): the
    // residual's error is ~0.6 sqrt(n) 2^-(9s-1) in the normalised measure
    // (residual_error_model); slices per round from that model
    L.sr = o.residual_slices > 0 ? o.residual_slices : residual_slices_for(n, o.tol);
    L.s0 = o.residual_slices > 0 ? o.residual_slices : first_residual_slices_for(n, o.tol, L.sr);
    const size_t nn = (size_t)n * (size_t)n;
    const bool overlap = n > leaf && overlap_schedule(n, o.precision, o.schedule);
    L.region0 = round256(std::max(ws_fp64_elems(n, leaf, overlap), nn) * sizeof(double));
    size_t sc = 0;
    if (n > leaf) {
        const int64_t n1 = split_order(n);
        sc = bf16x3_scratch_bytes(n1, n1, n1);
        if (o.fp64_levels > 0) sc = std::max(sc, ozaki_scratch_bytes(n1, n1, n1, kSchurSlices));
        if (o.precision == SPIN_MIXED_DIGITS) sc = std::max(sc, ozaki_scratch_bytes(n1, n1, n1, kLevelSlices));
    }
    sc = std::max(sc, ozaki_scratch_bytes(0, n, n, L.sr));
    sc = std::max(sc, bf16x6_scratch_bytes(n, n, n));
    L.scratch = round256(sc);
    L.apl = round256((size_t)L.sr * (size_t)n * (size_t)tc_ld(n) * 2 + (size_t)n * 4 + 512);
    // the side stream's products (II and C21 of every level: at most n2 x n1 x n1)
    size_t side = 0;
    if (overlap) {
        const int64_t n1 = split_order(n);
        side = bf16x3_scratch_bytes(n1, n1, n1);
        if (o.precision == SPIN_MIXED_DIGITS) side = std::max(side, ozaki_scratch_bytes(n1, n1, n1, kLevelSlices));
    }
    L.side_scratch = round256(side);
    L.off_scratch = L.region0;
    L.off_apl = L.off_scratch + L.scratch;
    L.off_norms = L.off_apl + L.apl;
    L.off_side = L.off_norms + 256;
    L.total = L.off_side + L.side_scratch;
    return L;
}

size_t inner_bytes(int64_t n, int64_t leaf, const spin_opts& o) {
    if (o.precision == SPIN_FP64)
        return ws_fp64_elems(n, leaf, n > leaf && overlap_schedule(n, o.precision, o.schedule)) * sizeof(double);
    return mix_layout(n, leaf, o).total;
}

// Butterfly transform: [diagonals | Ar (np x np) | Y (np x np) | the
// workspace of the recursion on order np (mixed: also the refinement's)].
struct RbtLayout {
    int64_t np;
    size_t off_ar, off_y, off_inner, total;
};

RbtLayout rbt_layout(int64_t n, int64_t leaf, const spin_opts& o) {
    RbtLayout R;
    R.np = rbt_padded_order(n, kRbtDepth);
    const size_t nn = (size_t)R.np * (size_t)R.np * sizeof(double);
    R.off_ar = round256(2 * (size_t)kRbtDepth * (size_t)R.np * sizeof(double));
    R.off_y = R.off_ar + round256(nn);
    R.off_inner = R.off_y + round256(nn);
    R.total = R.off_inner + inner_bytes(R.np, leaf, o);
    return R;
}

size_t workspace_bytes_for(int64_t n, int64_t leaf, const spin_opts& o) {
    if (o.pretransform == 1) return rbt_layout(n, leaf, o).total;
    if (o.pretransform == 2) return std::max(inner_bytes(n, leaf, o), rbt_layout(n, leaf, o).total);
    return inner_bytes(n, leaf, o);
}

// Newton-Schulz refinement X <- X + X (I - A X) (Bailey-style stabilisation
// of Strassen's inversion, cited in Sec. 2.1): every residual R = I - A X is
// FP64-class (digit slices of A, split once and cached, and of X), the
// correction X R is a six-product BF16 form.  Every residual is recomputed
// in full: after a step the true residual is dominated by the previous
// residual's own rounding error, which an update of the form R - A (dX)
// cannot see.  Stops when ||AX - I||_F / (||A||_F ||X||_F) <= tol.
//
// The stopping decision is taken on the device (refine.cu): rounds
// 0 .. max_refine are all enqueued, each gated on the stream's active flag,
// so the call never waits for the host between steps.
int refine(Run& r, StreamState* st, const double* A, int64_t lda, double* X, int64_t ldx, int64_t n,
           const spin_opts& o, const MixLayout& L, unsigned char* ws) {
    cudaStream_t s = r.s;
    double* R = (double*)ws;
    double* norms = (double*)(ws + L.off_norms);
    int* act = st->active();
    const int64_t ld = tc_ld(n);
    OzakiCachedA ca{(uint16_t*)(ws + L.off_apl), (int*)(ws + L.off_apl + (size_t)L.sr * n * ld * 2)};
    void* scratch = ws + L.off_scratch;
    // a leaf that failed leaves the matrix switched off: nothing below runs
    RET(launch_refine_init(st->info_dev, 1, act, st->rel(), st->iters(), s));
    SPIN_CUDA_TRY(cudaMemsetAsync(norms, 0, 3 * sizeof(double), s));
    {
        ProfScope ps(r.prof, s, SPIN_KERNEL_SPLIT, -1, n, n, 0, 0.0, 8.0 * n * n + 2.0 * L.sr * n * n, act);
        RET(ozaki_split_a(A, lda, n, n, L.sr, &ca, &norms[0], s, act));
    }
    const double f = 2.0 * (double)n * n * n;
    const int sr = L.sr;
    for (int it = 0; it <= o.max_refine; it++) {
        // the first residual only feeds the update: fewer slice pairs
        const int s_it = it == 0 ? L.s0 : sr;
        const int pairs = s_it * (s_it + 1) / 2;
        SPIN_CUDA_TRY(cudaMemsetAsync(norms + 1, 0, 2 * sizeof(double), s));
        SplitPlan sp;
        RET(plan_ozaki(0, n, n, sr, scratch, L.scratch, &sp));
        sp.a = ca.planes;
        sp.ea = ca.exps;
        {
            ProfScope ps(r.prof, s, SPIN_KERNEL_SPLIT, -1, n, n, 0, 0.0, 8.0 * n * n + 2.0 * sr * n * n, act);
            RET(split_b_ozaki(sp, X, ldx, n, n, &norms[1], s, act));
        }
        {
            ProfScope ps(r.prof, s, SPIN_KERNEL_RESIDUAL, -1, n, n, n, pairs * f, 2.0 * sr * 2.0 * n * n + 8.0 * n * n,
                         act);
            RET(product_ozaki(sp, n, n, n, -1.0, 0.0, nullptr, 0, R, n, 1, &norms[2], r.err, s, act, s_it));
        }
        RET(launch_refine_decide(norms, norms + 1, norms + 2, 1, o.tol, residual_error_model(n, s_it), it,
                                 o.max_refine, act, st->rel(), st->iters(), st->info_dev, s));
        if (it == o.max_refine) break;
        // X <- X + X R with three-plane BF16 splits and six products (~2^-22
        // relative): the correction's own error enters the next residual
        // amplified by ~kappa * rel, so it needs more than bf16x3's ~2^-16.
        SplitPlan up;
        RET(plan_bf16x6(n, n, n, scratch, L.scratch, &up));
        {
            ProfScope ps(r.prof, s, SPIN_KERNEL_SPLIT, -1, n, n, 0, 0.0, 28.0 * n * n, act);
            RET(split_a_bf16x6(up, X, ldx, n, n, s, act));
            RET(split_b_bf16x6(up, R, n, n, n, s, act));
        }
        ProfScope ps(r.prof, s, SPIN_KERNEL_UPDATE, -1, n, n, n, 6.0 * f, 12.0 * n * n + 16.0 * n * n, act);
        RET(product_bf16x6(up, n, n, n, 1.0, 1.0, X, ldx, X, ldx, r.err, s, act));
    }
    return launch_refine_finish(r.err, st->info_dev, 1, s);
}

// One attempt: the recursion on A (pretransform 0) or on U^T A V with the
// transform undone afterwards (pretransform 1); mixed modes then refine
// X against A itself.
int enqueue_once(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, int64_t leaf, const spin_opts& o,
                 bool rbt, StreamState* st, cudaStream_t s, unsigned char* ws) {
    const bool mixed = o.precision != SPIN_FP64;
    st->last_mixed = mixed ? 1 : 0;
    st->last_pretransformed = rbt ? 1 : 0;
    SPIN_CUDA_TRY(cudaMemsetAsync(st->info_dev, 0, INFO_WORDS * sizeof(int32_t), s));
    Run r{s, st->info_dev, 0, leaf, st->prof.on ? &st->prof : nullptr};
    // what the recursion inverts, where it writes, and its workspace
    const double* Ain = A;
    int64_t lda_in = lda, n_in = n;
    double* Xout = X;
    int64_t ldx_out = ldx;
    unsigned char* inner = ws;
    RbtLayout R{};
    if (rbt) {
        R = rbt_layout(n, leaf, o);
        double* diag = (double*)ws;
        double* Ar = (double*)(ws + R.off_ar);
        RET(launch_rbt_diagonals(o.rbt_seed, R.np, kRbtDepth, diag, s));
        RET(launch_rbt_forward(A, lda, n, Ar, R.np, kRbtDepth, diag, s));
        Ain = Ar;
        lda_in = n_in = R.np;
        Xout = (double*)(ws + R.off_y);
        ldx_out = R.np;
        inner = ws + R.off_inner;
    }
    if (!mixed) {
        if (overlap_schedule(n_in, o.precision, o.schedule) && n_in > leaf) {
            if (st->side == nullptr) SPIN_CUDA_TRY(cudaStreamCreateWithFlags(&st->side, cudaStreamNonBlocking));
            r.side = st->side;
            r.events = &st->events;
        }
        RET(inv_rec(r, 0, Ain, lda_in, Xout, ldx_out, n_in, (double*)inner));
        if (rbt) RET(launch_rbt_backward(Xout, R.np, kRbtDepth, (const double*)ws, X, ldx, n, s));
        return SPIN_OK;
    }
    const MixLayout Lin = mix_layout(n_in, leaf, o);
    r.precision = o.precision;
    r.fp64_levels = o.fp64_levels;
    r.scratch = inner + Lin.off_scratch;
    r.scratch_bytes = Lin.scratch;
    if (Lin.side_scratch > 0) {
        if (st->side == nullptr) SPIN_CUDA_TRY(cudaStreamCreateWithFlags(&st->side, cudaStreamNonBlocking));
        r.side = st->side;
        r.events = &st->events;
        r.side_scratch = inner + Lin.off_side;
        r.side_scratch_bytes = Lin.side_scratch;
    }
    r.err = st->err_dev;
    SPIN_CUDA_TRY(cudaMemsetAsync(st->err_dev, 0, sizeof(int), s));
    RET(inv_rec(r, 0, Ain, lda_in, Xout, ldx_out, n_in, (double*)inner));
    if (rbt) RET(launch_rbt_backward(Xout, R.np, kRbtDepth, (const double*)ws, X, ldx, n, s));
    // the refinement's layout for order n fits in the recursion's (order >= n)
    return refine(r, st, A, lda, X, ldx, n, o, mix_layout(n, leaf, o), inner);
}

// Whether repeated calls replay a captured graph (SPIN_GRAPH=0 turns it
// off, for measurement; read once).
bool graph_mode() {
    static int v = -1;
    if (v < 0) {
        const char* e = getenv("SPIN_GRAPH");
        v = (e && atoi(e) == 0) ? 0 : 1;
    }
    return v == 1;
}

uint64_t bits_of(double x) {
    uint64_t u;
    memcpy(&u, &x, sizeof u);
    return u;
}

// Every argument that shapes the launch sequence or its operands.
std::vector<uint64_t> call_key(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, int64_t leaf,
                               const spin_opts& o, const void* ws) {
    return {(uint64_t)(uintptr_t)A, (uint64_t)lda, (uint64_t)(uintptr_t)X, (uint64_t)ldx, (uint64_t)n,
            (uint64_t)leaf, (uint64_t)o.precision, bits_of(o.tol), (uint64_t)o.max_refine,
            (uint64_t)o.fp64_levels, (uint64_t)o.residual_slices, (uint64_t)o.pretransform, o.rbt_seed,
            (uint64_t)(int64_t)o.schedule,
            (uint64_t)(uintptr_t)ws};
}

// Capture the whole schedule of one call (every launch enqueue_once makes,
// on this stream and on the side stream) into a graph on a private stream.
int capture_schedule(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, int64_t leaf,
                     const spin_opts& o, StreamState* st, unsigned char* ws) {
    if (st->cap == nullptr) SPIN_CUDA_TRY(cudaStreamCreateWithFlags(&st->cap, cudaStreamNonBlocking));
    if (st->exec) {
        cudaGraphExecDestroy(st->exec);
        st->exec = nullptr;
        st->graph_key.clear();
    }
    SPIN_CUDA_TRY(cudaStreamBeginCapture(st->cap, cudaStreamCaptureModeThreadLocal));
    const int rc = enqueue_once(A, lda, X, ldx, n, leaf, o, o.pretransform == 1, st, st->cap, ws);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st->cap, &graph);
    if (rc != SPIN_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    SPIN_CUDA_TRY(ec);
    size_t nodes = 0;
    cudaGraphGetNodes(graph, nullptr, &nodes);
    st->graph_nodes = (int64_t)nodes;
    const cudaError_t ei = cudaGraphInstantiate(&st->exec, graph, 0);
    cudaGraphDestroy(graph);
    SPIN_CUDA_TRY(ei);
    st->graph_mixed = st->last_mixed;
    st->graph_rbt = st->last_pretransformed;
    return SPIN_OK;
}

int enqueue(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, const spin_opts& o,
            StreamState* st, cudaStream_t s) {
    const int64_t leaf = resolve_leaf(n, o.leaf, o.precision);
    RET(check_common(A, lda, X, ldx, n, leaf));
    if (!valid_precision(o.precision)) return SPIN_ERR_INVALID_ARG;
    const bool mixed = o.precision != SPIN_FP64;
    if (mixed && (o.residual_slices < 0 || o.residual_slices > 7 || o.max_refine < 0 || !(o.tol > 0.0)))
        return SPIN_ERR_INVALID_ARG;
    if (o.pretransform < 0 || o.pretransform > 2) return SPIN_ERR_INVALID_ARG;
    if (o.schedule < SPIN_SCHEDULE_DEFAULT || o.schedule > SPIN_SCHEDULE_PERSISTENT) return SPIN_ERR_INVALID_ARG;
    const size_t need = workspace_bytes_for(n, leaf, o);
    unsigned char* ws;
    if (o.workspace != nullptr) {
        if (o.workspace_bytes < need || ((uintptr_t)o.workspace & 255u) != 0) return SPIN_ERR_INVALID_ARG;
        ws = (unsigned char*)o.workspace;
    } else {
        RET(ensure_ws(st, need));
        ws = (unsigned char*)st->ws;
    }
    if (o.pretransform != 2) {
        if (!graph_mode() || st->prof.on) return enqueue_once(A, lda, X, ldx, n, leaf, o, o.pretransform == 1, st, s, ws);
        // The second call with the same arguments captures the schedule;
        // later ones replay it (one graph launch, dependencies resolved on
        // the device); any other call runs the launches directly.
        std::vector<uint64_t> key = call_key(A, lda, X, ldx, n, leaf, o, ws);
        if (st->exec == nullptr || key != st->graph_key) {
            if (key != st->prev_key) {
                st->prev_key = key;
                return enqueue_once(A, lda, X, ldx, n, leaf, o, o.pretransform == 1, st, s, ws);
            }
            RET(capture_schedule(A, lda, X, ldx, n, leaf, o, st, ws));
            st->graph_key = key;
        }
        st->last_mixed = st->graph_mixed;
        st->last_pretransformed = st->graph_rbt;
        SPIN_CUDA_TRY(cudaGraphLaunch(st->exec, s));
        st->graph_launches++;
        return SPIN_OK;
    }
    // plain first; a zero or non-finite pivot (A11 or a Schur complement
    // singular in working precision) sends the call through the transform
    RET(enqueue_once(A, lda, X, ldx, n, leaf, o, false, st, s, ws));
    SPIN_CUDA_TRY(cudaMemcpyAsync(st->info_host, st->info_dev, INFO_WORDS * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, s));
    SPIN_CUDA_TRY(cudaStreamSynchronize(s));
    if (st->info_host[INFO_STATUS] != SPIN_ERR_SINGULAR) return SPIN_OK;
    return enqueue_once(A, lda, X, ldx, n, leaf, o, true, st, s, ws);
}

// ---- leaf autotuning ----
std::mutex g_tune_mu;
std::map<std::pair<int, int>, int> g_tuned;  // (precision, ceil log2 n) -> leaf

int size_class(int64_t n) {
    int c = 0;
    while (((int64_t)1 << c) < n) c++;
    return c;
}

__global__ void synth_sdd_kernel(double* A, int64_t n, uint64_t seed) {
    const int64_t total = n * n;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        uint64_t z = seed + (uint64_t)(i + 1) * 0x9E3779B97F4A7C15ull;  // splitmix64 of the position
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        double v = 2.0 * (double)(z >> 11) * 0x1.0p-53 - 1.0;
        if (i / n == i % n) v += (double)n;
        A[i] = v;
    }
}

// ---- cost model of the plain FP64 path (Sec. 4's cost analysis restated
// for one GB300) ----
//
// The paper prices each step of Algorithm 1 on a Spark cluster (Table 2,
// Eq. (SPIN-cost)) and finds a U-shaped dependence on the partition size
// (Fig. 3).  On one GPU the two sides of the U are: products of the deep
// levels are too small to fill 152 SMs (left), and Gauss-Jordan leaves run on
// one cluster of at most 16 SMs at the FP64 rate plus a per-pivot latency
// (right).  Model, per recursion node: six products (n1, n2 split), each
//   t = launch + max(ceil(tiles / 152) * 2 * TM * TM * k / P_sm, 2 m n k / P_gpu)
// with the product kernel's TM x TM tiles (64, 32 or 16) and P_sm = 4 flops/clock at 2.07 GHz (P_gpu = 152 P_sm,
// 1.259 TFLOP/s, the measured DFMA rate); per leaf of order L on C = min(16,
// 2^ceil(log2 L)) CTAs with R = ceil(L / C) rows each, L pivot steps of
//   a + b L + R L / (2 FMA/clock)     (rows in shared memory)
//   a + b L + R L g                   (rows in L2-resident global memory)
// with a = 1.55 us, b = 5 ns for L <= 256 (candidate rows pushed to every
// CTA) and a = 1.8 us, b = 14 ns above (pivot row read from its owner), and
// g = 0.55 ns per element: per-step times of one leaf on its 16-CTA cluster
// (bench.py --leaf-times, L = 32 ... 2048).  It reproduces the measured sweeps at n = 1024,
// 4096 and 8192 (leaf 64 ... 2048) within 8 %.
constexpr double kModelClock = 2.07e9;
constexpr double kModelPsm = 4.0 * kModelClock;
constexpr double kModelPgpu = 152.0 * kModelPsm;
constexpr double kModelLaunch = 4e-6;
constexpr double kModelAPush = 1.85e-6, kModelBPush = 0.0, kModelAPull = 3.46e-6, kModelBPull = 6.4e-9;
constexpr double kModelG = 0.44e-9;

double model_gemm(int64_t m, int64_t n, int64_t k) {
    const int64_t tm = gemm_f64_tile_size(m, n, 1);
    const double tiles = (double)((m + tm - 1) / tm) * (double)((n + tm - 1) / tm);
    const double wave = std::ceil(tiles / 152.0) * 2.0 * (double)(tm * tm) * (double)k / kModelPsm;
    return kModelLaunch + std::max(wave, 2.0 * (double)m * (double)n * (double)k / kModelPgpu);
}

double model_leaf(int64_t L) {
    int64_t C = 1;
    while (C < 16 && C < L) C <<= 1;
    const int64_t R = (L + C - 1) / C;
    const double fma_time = (double)R * L / (2.0 * kModelClock);
    if (L <= 256) return (double)L * (kModelAPush + kModelBPush * (double)L + fma_time);
    const bool smem = (double)R * L * 8 + 16.0 * R + 64.0 * C + 16.0 * L <= 200.0 * 1024;
    return (double)L * (kModelAPull + kModelBPull * (double)L + (smem ? fma_time : (double)R * L * kModelG));
}

double model_fp64(int64_t n, int64_t leaf) {
    if (n <= leaf) return model_leaf(n);
    const int64_t n1 = split_order(n), n2 = n - n1;
    return model_fp64(n1, leaf) + model_fp64(n2, leaf) + model_gemm(n1, n2, n1) + model_gemm(n2, n2, n1) +
           model_gemm(n1, n2, n2) + model_gemm(n2, n1, n1) + model_gemm(n2, n1, n2) + model_gemm(n1, n1, n2);
}

int model_best_leaf(int64_t n) {
    static const int cands[] = {64, 128, 256, 512, 1024, 2048};
    int best = 64;
    double bt = 1e300;
    for (int L : cands) {
        if (L > n) break;
        const double t = model_fp64(n, L);
        if (t < bt) {
            bt = t;
            best = L;
        }
    }
    return best;
}

}  // namespace

int tuned_leaf(int64_t n, int precision) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned.find(std::make_pair(precision, size_class(n)));
    if (it == g_tuned.end()) {
        // a size class above the largest tuned one reuses that class's choice
        int best_c = -1, leaf = 0;
        for (auto& kv : g_tuned)
            if (kv.first.first == precision && kv.first.second <= size_class(n) && kv.first.second > best_c) {
                best_c = kv.first.second;
                leaf = kv.second;
            }
        return leaf;
    }
    return it->second;
}

// Internal entry for other translation units: the FP64 recursion over a
// caller-supplied workspace W (fp64_workspace_elems(n, leaf) doubles) and
// info record, no profiling, nothing allocated.
size_t fp64_workspace_elems(int64_t n, int64_t leaf) { return ws_fp64_elems(n, leaf); }

int run_fp64_inversion(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, int64_t leaf, double* W,
                       int32_t* info, cudaStream_t s) {
    Run r{s, info, 0, leaf, nullptr};
    return inv_rec(r, 0, A, lda, X, ldx, n, W);
}

}  // namespace spin

using namespace spin;

extern "C" {

spin_opts spin_opts_default(void) {
    spin_opts o;
    memset(&o, 0, sizeof o);
    o.precision = SPIN_FP64;
    o.leaf = 0;
    o.tol = 1e-10;
    o.max_refine = 6;
    o.fp64_levels = 2;
    o.blocking = 1;
    o.residual_slices = 0;
    return o;
}

double spin_model_seconds(int64_t n, int leaf, int precision) {
    if (n < 1 || leaf < 1 || precision != SPIN_FP64) return -1.0;
    return model_fp64(n, std::min<int64_t>(leaf, n));
}

int spin_default_leaf(int64_t n, int precision) {
    if (n <= 128) return (int)(n < 1 ? 1 : n);
    const int t = tuned_leaf(n, precision);
    if (t > 0) return (int)std::min<int64_t>(t, n);
    // untuned: the cost model's optimum for the plain path; the mixed path's
    // products are ~1000x cheaper, so its leaves stay small
    if (precision == SPIN_FP64) return model_best_leaf(n);
    return 128;
}

int spin_autotune_leaf(int64_t n, int precision, const int* candidates, int ncand, int* leaf_out, double* ms_out,
                       spin_stream_t stream) {
    if (n < 2 || ncand < 1 || candidates == nullptr || leaf_out == nullptr) return SPIN_ERR_INVALID_ARG;
    if (!valid_precision(precision)) return SPIN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    StreamState* st = nullptr;
    RET(get_state(s, &st));
    double* A = nullptr;
    double* X = nullptr;
    const size_t bytes = (size_t)n * (size_t)n * sizeof(double);
    if (cudaMalloc(&A, bytes) != cudaSuccess || cudaMalloc(&X, bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(A);
        return SPIN_ERR_OOM;
    }
    synth_sdd_kernel<<<1024, 256, 0, s>>>(A, n, 0x5EED5EEDull);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1, rc = SPIN_OK;
    float best_ms = 1e30f;
    for (int i = 0; i < ncand && rc == SPIN_OK; i++) {
        const int L = candidates[i];
        if (ms_out) ms_out[i] = -1.0;
        if (L < 1 || L > kMaxLeaf || L >= n) continue;
        spin_opts o = spin_opts_default();
        o.precision = precision;
        o.leaf = L;
        spin_info info;
        // warm: workspace and modules, then the captured schedule
        for (int w = 0; w < 2 && rc == SPIN_OK; w++) rc = spin_invert_ex(A, n, X, n, n, &o, &info, stream);
        if (rc != SPIN_OK) break;
        cudaEventRecord(e0, s);
        rc = spin_invert_ex(A, n, X, n, n, &o, &info, stream);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms_out) ms_out[i] = ms;
        if (rc == SPIN_OK && info.status == SPIN_OK && ms < best_ms) {
            best_ms = ms;
            best = L;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(A);
    cudaFree(X);
    if (rc != SPIN_OK) return rc;
    if (best < 0) return SPIN_ERR_INVALID_ARG;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tuned[std::make_pair(precision, size_class(n))] = best;
    }
    *leaf_out = best;
    return SPIN_OK;
}

size_t spin_workspace_bytes(int64_t n, const spin_opts* opts) {
    spin_opts o = opts ? *opts : spin_opts_default();
    if (n < 1) return 0;
    if (o.schedule < SPIN_SCHEDULE_DEFAULT || o.schedule > SPIN_SCHEDULE_PERSISTENT) return 0;
    const int64_t leaf = resolve_leaf(n, o.leaf, o.precision);
    if (leaf < 1 || leaf > kMaxLeaf) return 0;
    return workspace_bytes_for(n, leaf, o);
}

int spin_invert_ex(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, const spin_opts* opts,
                   spin_info* info, spin_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    spin_opts o = opts ? *opts : spin_opts_default();
    if (!valid_precision(o.precision)) return SPIN_ERR_INVALID_ARG;
    RET(check_common(A, lda, X, ldx, n, n >= 1 ? resolve_leaf(n, o.leaf, o.precision) : 1));
    StreamState* st = nullptr;
    RET(get_state(s, &st));
    int rc = enqueue(A, lda, X, ldx, n, o, st, s);
    if (rc != SPIN_OK) return rc;
    if (o.blocking || info != nullptr) return read_info(st, s, info);
    return SPIN_OK;
}

int spin_invert(const double* A, double* X, int64_t n, int64_t lda, int leaf, spin_stream_t stream) {
    spin_opts o = spin_opts_default();
    o.leaf = leaf;
    o.blocking = 1;
    return spin_invert_ex(A, lda, X, n, n, &o, nullptr, stream);
}

int spin_schedule_stats(spin_stream_t stream, int64_t* replays, int64_t* nodes) {
    cudaStream_t s = (cudaStream_t)stream;
    StreamState* st = nullptr;
    RET(get_state(s, &st));
    if (replays) *replays = st->graph_launches;
    if (nodes) *nodes = st->exec ? st->graph_nodes : 0;
    return SPIN_OK;
}

int spin_sync(spin_stream_t stream, spin_info* info) {
    cudaStream_t s = (cudaStream_t)stream;
    StreamState* st = nullptr;
    RET(get_state(s, &st));
    return read_info(st, s, info);
}

int spin_invert_host(const double* A_host, int64_t lda, double* X_host, int64_t ldx, int64_t n,
                     const spin_opts* opts, spin_info* info, spin_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (A_host == nullptr || X_host == nullptr || n < 1 || lda < n || ldx < n) return SPIN_ERR_INVALID_ARG;
    StreamState* st = nullptr;
    RET(get_state(s, &st));
    const size_t elems = (size_t)n * (size_t)n;
    if (st->host_elems < elems) {
        if (st->hostA) cudaFree(st->hostA);
        if (st->hostX) cudaFree(st->hostX);
        st->hostA = st->hostX = nullptr;
        st->host_elems = 0;
        if (cudaMalloc(&st->hostA, elems * sizeof(double)) != cudaSuccess ||
            cudaMalloc(&st->hostX, elems * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            return SPIN_ERR_OOM;
        }
        st->host_elems = elems;
    }
    SPIN_CUDA_TRY(cudaMemcpy2DAsync(st->hostA, n * sizeof(double), A_host, lda * sizeof(double),
                                    n * sizeof(double), n, cudaMemcpyHostToDevice, s));
    spin_opts o = opts ? *opts : spin_opts_default();
    o.blocking = 0;
    int rc = enqueue(st->hostA, n, st->hostX, n, n, o, st, s);
    if (rc != SPIN_OK) return rc;
    SPIN_CUDA_TRY(cudaMemcpy2DAsync(X_host, ldx * sizeof(double), st->hostX, n * sizeof(double),
                                    n * sizeof(double), n, cudaMemcpyDeviceToHost, s));
    return read_info(st, s, info);
}

const char* spin_status_string(int status) {
    switch (status) {
        case SPIN_OK: return "SPIN_OK";
        case SPIN_ERR_INVALID_ARG: return "SPIN_ERR_INVALID_ARG";
        case SPIN_ERR_SINGULAR: return "SPIN_ERR_SINGULAR";
        case SPIN_ERR_NOT_CONVERGED: return "SPIN_ERR_NOT_CONVERGED";
        case SPIN_ERR_OOM: return "SPIN_ERR_OOM";
        case SPIN_ERR_CUDA: return "SPIN_ERR_CUDA";
        case SPIN_ERR_TIMEOUT: return "SPIN_ERR_TIMEOUT";
        case SPIN_ERR_BUSY: return "SPIN_ERR_BUSY";
        case SPIN_ERR_NOT_IMPLEMENTED: return "SPIN_ERR_NOT_IMPLEMENTED";
        default: return "SPIN_ERR_UNKNOWN";
    }
}

int spin_version(void) { return 100; }

const char* spin_last_error(void) { return g_last_error.c_str(); }

int spin_leaf_inverse(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, int32_t* info_dev,
                      spin_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    if (n < 1 || n > kMaxLeaf || lda < n || ldx < n || !A || !X || !aligned8(A) || !aligned8(X))
        return SPIN_ERR_INVALID_ARG;
    StreamState* st = nullptr;
    RET(get_state(s, &st));
    double* scratch = nullptr;
    const size_t need = leaf_scratch_elems(n) * sizeof(double);
    if (need) {
        RET(ensure_ws(st, need));
        scratch = (double*)st->ws;
    }
    int32_t* info = info_dev ? info_dev : st->info_dev;
    if (!info_dev) SPIN_CUDA_TRY(cudaMemsetAsync(info, 0, INFO_WORDS * sizeof(int32_t), s));
    return launch_leaf_gj(A, lda, X, ldx, n, scratch, info, 0, s);
}

int spin_profile_start(spin_stream_t stream, int max_records) {
    if (max_records < 0) return SPIN_ERR_INVALID_ARG;
    StreamState* st = nullptr;
    RET(get_state((cudaStream_t)stream, &st));
    Profiler& p = st->prof;
    for (auto& e : p.entries) {
        p.pool.push_back(e.start);
        p.pool.push_back(e.stop);
    }
    p.entries.clear();
    p.max_records = max_records;
    // one device int per possible record for the gate copies (grown here,
    // outside the timed region of a caller that profiles)
    if (p.flags_cap < max_records) {
        if (p.flags) cudaFree(p.flags);
        p.flags = nullptr;
        p.flags_cap = 0;
        if (max_records > 0) {
            SPIN_CUDA_TRY(cudaMalloc(&p.flags, (size_t)max_records * sizeof(int)));
            p.flags_cap = max_records;
        }
    }
    p.on = true;
    return SPIN_OK;
}

int spin_profile_stop(spin_stream_t stream, spin_prof_record* out, int max, int* count) {
    cudaStream_t s = (cudaStream_t)stream;
    StreamState* st = nullptr;
    RET(get_state(s, &st));
    Profiler& p = st->prof;
    p.on = false;
    SPIN_CUDA_TRY(cudaStreamSynchronize(s));
    std::vector<int> gates;
    if (p.flags != nullptr && !p.entries.empty()) {
        gates.resize(std::min<size_t>(p.entries.size(), (size_t)p.flags_cap));
        SPIN_CUDA_TRY(cudaMemcpy(gates.data(), p.flags, gates.size() * sizeof(int), cudaMemcpyDeviceToHost));
    }
    int c = 0;
    for (auto& e : p.entries) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.start, e.stop);
        e.rec.ms = ms;
        if (e.gate_slot >= 0 && e.gate_slot < (int)gates.size() && gates[e.gate_slot] == 0) {
            // gated off on the device: the launch returned at once
            e.rec.kind = SPIN_KERNEL_OTHER;
            e.rec.flops = 0.0;
            e.rec.bytes = 0.0;
        }
        if (out != nullptr && c < max) out[c] = e.rec;
        c++;
        p.pool.push_back(e.start);
        p.pool.push_back(e.stop);
    }
    p.entries.clear();
    if (count) *count = c;
    return SPIN_OK;
}

int spin_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, const double* B,
                  int64_t ldb, double beta, const double* C, int64_t ldc, double* D, int64_t ldd,
                  spin_stream_t stream) {
    if (m < 0 || n < 0 || k < 0 || lda < k || ldb < n || ldd < n) return SPIN_ERR_INVALID_ARG;
    if (!(alpha == 1.0 || alpha == -1.0) || !(beta == 0.0 || beta == 1.0)) return SPIN_ERR_INVALID_ARG;
    if (beta != 0.0 && (C == nullptr || ldc < n)) return SPIN_ERR_INVALID_ARG;
    if ((m > 0 && n > 0) && (D == nullptr || (k > 0 && (A == nullptr || B == nullptr)))) return SPIN_ERR_INVALID_ARG;
    return launch_gemm_f64(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, (cudaStream_t)stream);
}

}  // extern "C"
