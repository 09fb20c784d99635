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
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"

namespace spin {
namespace {

constexpr int kStreams = 8;

struct Bucket {
    int64_t n, leaf;
    int count;
    int first;             // offset of the bucket in the sorted order
    size_t ws_elems;       // per matrix
    size_t ws_offset;      // elements into the workspace block
};

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
    int kernels = 0;  // kernel launches in the captured graph
    cudaGraphExec_t exec = nullptr;
    cudaStream_t cap = nullptr;  // private stream the launch sequence is captured on
    cudaStream_t streams[kStreams] = {};
    cudaEvent_t fork = nullptr, join[kStreams] = {};
};

std::mutex g_bmu;
std::map<cudaStream_t, BatchPlan> g_plans;

void free_plan(BatchPlan& p) {
    if (p.exec) cudaGraphExecDestroy(p.exec);
    cudaFree((void*)p.a_base);
    cudaFree(p.a_ld);
    cudaFree(p.x_base);
    cudaFree(p.w_base);
    cudaFree(p.user_index);
    cudaFree(p.records);
    cudaFree(p.ws);
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

int64_t batched_leaf(int64_t n, int leaf_opt) {
    int64_t L = leaf_opt > 0 ? leaf_opt : (n <= 128 ? n : 64);
    return std::min<int64_t>(L, n);
}

int build_plan(BatchPlan& p, const double* const* A, const int64_t* lda, double* const* X, const int64_t* n,
               int count, int leaf_opt, int* info_dev, cudaStream_t s) {
    free_plan(p);
    p.count = count;
    p.kernels = 0;
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
        b.leaf = batched_leaf(b.n, leaf_opt);
        b.count = j - i;
        b.first = i;
        b.ws_elems = std::max<size_t>(fp64_workspace_elems(b.n, b.leaf), 1);
        b.ws_offset = ws_total;
        ws_total += b.ws_elems * (size_t)b.count;
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

    // Capture on a private stream (the caller's may be the legacy default
    // stream, which cannot be captured); the graph is launched on the
    // caller's stream.  Order: memset records, fork, buckets (largest first,
    // least-loaded stream), join, scatter statuses.
    cudaGraph_t graph = nullptr;
    s = p.cap;
    SPIN_CUDA_TRY(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    int rc = SPIN_OK;
    cudaError_t e = cudaMemsetAsync(p.records, 0, (size_t)count * INFO_WORDS * sizeof(int32_t), s);
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
        const Bucket& b = p.buckets[bi];
        const int si = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[si] += (double)b.count * b.n * b.n * b.n;
        BRun r{&p.kernels, p.streams[si], p.records + (int64_t)b.first * INFO_WORDS, 0, b.leaf, b.count,
               p.ws + b.ws_offset, (int64_t)b.ws_elems};
        BatchView Av{p.a_base + b.first, p.a_ld + b.first, 0, 0, 0};
        BatchView Xv{(const double* const*)(p.x_base + b.first), nullptr, b.n, 0, 0};
        rc = binv(r, Av, Xv, (const double* const*)(p.w_base + b.first), 0, b.n);
    }
    for (int i = 0; i < kStreams; i++) {
        cudaError_t e2 = cudaEventRecord(p.join[i], p.streams[i]);
        if (e2 == cudaSuccess) e2 = cudaStreamWaitEvent(s, p.join[i], 0);
        if (e2 != cudaSuccess && rc == SPIN_OK) {
            record_cuda_error(e2, "batched join", __FILE__, __LINE__);
            rc = SPIN_ERR_CUDA;
        }
    }
    if (rc == SPIN_OK && info_dev != nullptr) {
        p.kernels++;
        scatter_status_kernel<<<(count + 255) / 256, 256, 0, s>>>(p.records, p.user_index, count, info_dev);
        cudaError_t e3 = cudaGetLastError();
        if (e3 != cudaSuccess) {
            record_cuda_error(e3, "scatter", __FILE__, __LINE__);
            rc = SPIN_ERR_CUDA;
        }
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
    return SPIN_OK;
}

std::vector<uint64_t> make_key(const double* const* A, const int64_t* lda, double* const* X, const int64_t* n,
                               int count, int leaf, int* info_dev) {
    std::vector<uint64_t> k;
    k.reserve((size_t)count * 4 + 4);
    k.push_back((uint64_t)count);
    k.push_back((uint64_t)(int64_t)leaf);
    k.push_back((uint64_t)(uintptr_t)info_dev);
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

}  // namespace
}  // namespace spin

using namespace spin;

extern "C" int spin_invert_batched(const double* const* A, const int64_t* lda, double* const* X, const int64_t* n,
                                   int count, const spin_opts* opts, int* info_dev, spin_stream_t stream) {
    if (count < 1 || A == nullptr || lda == nullptr || X == nullptr || n == nullptr) return SPIN_ERR_INVALID_ARG;
    spin_opts o = opts ? *opts : spin_opts_default();
    if (o.precision != SPIN_FP64) return SPIN_ERR_NOT_IMPLEMENTED;
    if (o.leaf < 0) return SPIN_ERR_INVALID_ARG;
    for (int i = 0; i < count; i++) {
        if (n[i] < 1 || n[i] > 65536 || lda[i] < n[i] || A[i] == nullptr || X[i] == nullptr) return SPIN_ERR_INVALID_ARG;
        if (((uintptr_t)A[i] & 7u) || ((uintptr_t)X[i] & 7u)) return SPIN_ERR_INVALID_ARG;
        if (batched_leaf(n[i], o.leaf) > kMaxLeaf) return SPIN_ERR_INVALID_ARG;
    }
    if (count > 65535) return SPIN_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_bmu);
    BatchPlan& p = g_plans[s];
    std::vector<uint64_t> key = make_key(A, lda, X, n, count, o.leaf, info_dev);
    if (p.exec == nullptr || key != p.key) {
        int rc = build_plan(p, A, lda, X, n, count, o.leaf, info_dev, s);
        if (rc != SPIN_OK) {
            free_plan(p);
            p.key.clear();
            return rc;
        }
        p.key = key;
    }
    SPIN_CUDA_TRY(cudaGraphLaunch(p.exec, s));
    if (o.blocking) SPIN_CUDA_TRY(cudaStreamSynchronize(s));
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
