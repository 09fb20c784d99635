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
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"

namespace spin {

static thread_local std::string g_last_error;


void record_cuda_error(cudaError_t e, const char* what, const char* file, int line) {
    char buf[512];
    snprintf(buf, sizeof buf, "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
}

int64_t split_order(int64_t n) { return n > 64 ? 32 * ((n + 63) / 64) : (n + 1) / 2; }

static size_t ws_fp64_elems(int64_t n, int64_t leaf) {
    if (n <= leaf) return leaf_scratch_elems(n);
    const int64_t n1 = split_order(n), n2 = n - n1;
    const size_t a = ws_fp64_elems(n1, leaf);
    const size_t b = (size_t)(n1 * n2 + n2 * n2) + ws_fp64_elems(n2, leaf);
    return a > b ? a : b;
}

namespace {

struct ProfEntry {
    spin_prof_record rec;
    cudaEvent_t start, stop;
};

struct Profiler {
    bool on = false;
    int max_records = 0;
    std::vector<ProfEntry> entries;
    std::vector<cudaEvent_t> pool;

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

struct StreamState {
    Profiler prof;
    void* ws = nullptr;
    size_t ws_bytes = 0;
    int32_t* info_dev = nullptr;   // INFO_WORDS ints
    int32_t* info_host = nullptr;  // pinned mirror
    double* hostA = nullptr;       // device staging for spin_invert_host
    double* hostX = nullptr;
    size_t host_elems = 0;
};

std::mutex g_mu;
std::map<std::pair<int, cudaStream_t>, StreamState> g_states;

int get_state(cudaStream_t s, StreamState** out) {
    int dev = 0;
    SPIN_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    StreamState& st = g_states[std::make_pair(dev, s)];
    if (st.info_dev == nullptr) {
        SPIN_CUDA_TRY(cudaMalloc(&st.info_dev, INFO_WORDS * sizeof(int32_t)));
        SPIN_CUDA_TRY(cudaMallocHost(&st.info_host, INFO_WORDS * sizeof(int32_t)));
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
};

// Bracket one launch with events when the stream's profiler is on.
struct ProfScope {
    Profiler* p;
    cudaStream_t s;
    ProfEntry e;
    bool active;
    ProfScope(Profiler* prof, cudaStream_t st, int kind, int depth, int64_t m, int64_t n, int64_t k, double flops,
              double bytes)
        : p(prof), s(st), active(prof != nullptr && prof->on && (int)prof->entries.size() < prof->max_records) {
        if (!active) return;
        e.rec = spin_prof_record{kind, depth, m, n, k, flops, bytes, 0.0};
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
    ProfScope ps(r.prof, r.s, SPIN_KERNEL_GEMM_F64, depth, m, n, k, flops, bytes);
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

int inv_fp64(Run& r, int depth, const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, double* W) {
    if (n <= r.leaf) return leaf_prof(r, depth, A, lda, X, ldx, n, W);
    const int64_t n1 = split_order(n), n2 = n - n1;
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
    RET(inv_fp64(r, d + 1, A11, lda, X11, ldx, n1, W));                                      // I
    RET(gemm_f64_prof(r, d, n1, n2, n1, 1.0, X11, ldx, A12, lda, 0.0, nullptr, 0, T, n2));   // III
    RET(gemm_f64_prof(r, d, n2, n2, n1, -1.0, A21, lda, T, n2, 1.0, A22, lda, S, n2));      // -V
    RET(inv_fp64(r, d + 1, S, n2, X22, ldx, n2, Wsub));                                     // C22
    RET(gemm_f64_prof(r, d, n1, n2, n2, -1.0, T, n2, X22, ldx, 0.0, nullptr, 0, X12, ldx)); // C12
    RET(gemm_f64_prof(r, d, n2, n1, n1, 1.0, A21, lda, X11, ldx, 0.0, nullptr, 0, T, n1));  // II
    RET(gemm_f64_prof(r, d, n2, n1, n2, -1.0, X22, ldx, T, n1, 0.0, nullptr, 0, X21, ldx)); // C21
    RET(gemm_f64_prof(r, d, n1, n1, n2, -1.0, X12, ldx, T, n1, 1.0, X11, ldx, X11, ldx));   // C11
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
    SPIN_CUDA_TRY(cudaMemcpyAsync(st->info_host, st->info_dev, INFO_WORDS * sizeof(int32_t),
                                  cudaMemcpyDeviceToHost, s));
    SPIN_CUDA_TRY(cudaStreamSynchronize(s));
    const int32_t* h = st->info_host;
    if (info) {
        info->status = h[INFO_STATUS];
        info->refine_iters = 0;
        info->fail_leaf = h[INFO_STATUS] ? h[INFO_LEAF] : -1;
        info->fail_col = h[INFO_STATUS] ? h[INFO_COL] : -1;
        info->rel_residual = -1.0;
    }
    return h[INFO_STATUS];
}

int enqueue(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, const spin_opts& o,
            StreamState* st, cudaStream_t s) {
    const int64_t leaf = resolve_leaf(n, o.leaf, o.precision);
    RET(check_common(A, lda, X, ldx, n, leaf));
    if (o.precision != SPIN_FP64) return SPIN_ERR_NOT_IMPLEMENTED;
    const size_t need = ws_fp64_elems(n, leaf) * sizeof(double);
    double* W;
    if (o.workspace != nullptr) {
        if (o.workspace_bytes < need || !aligned8(o.workspace)) return SPIN_ERR_INVALID_ARG;
        W = (double*)o.workspace;
    } else {
        RET(ensure_ws(st, need));
        W = (double*)st->ws;
    }
    SPIN_CUDA_TRY(cudaMemsetAsync(st->info_dev, 0, INFO_WORDS * sizeof(int32_t), s));
    Run r{s, st->info_dev, 0, leaf, st->prof.on ? &st->prof : nullptr};
    return inv_fp64(r, 0, A, lda, X, ldx, n, W);
}

}  // namespace
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
    return o;
}

int spin_default_leaf(int64_t n, int precision) {
    (void)precision;
    if (n <= 128) return (int)(n < 1 ? 1 : n);
    return 128;
}

size_t spin_workspace_bytes(int64_t n, const spin_opts* opts) {
    spin_opts o = opts ? *opts : spin_opts_default();
    if (n < 1) return 0;
    const int64_t leaf = resolve_leaf(n, o.leaf, o.precision);
    if (leaf < 1 || leaf > kMaxLeaf) return 0;
    return ws_fp64_elems(n, leaf) * sizeof(double);
}

int spin_invert_ex(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, const spin_opts* opts,
                   spin_info* info, spin_stream_t stream) {
    cudaStream_t s = (cudaStream_t)stream;
    spin_opts o = opts ? *opts : spin_opts_default();
    if (o.precision < SPIN_FP64 || o.precision > SPIN_MIXED_TF32) return SPIN_ERR_INVALID_ARG;
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
    int c = 0;
    for (auto& e : p.entries) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e.start, e.stop);
        e.rec.ms = ms;
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
