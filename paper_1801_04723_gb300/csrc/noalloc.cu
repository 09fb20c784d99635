// spin_invert_noalloc: the plain FP64 inversion for callers that must not
// allocate device memory.
//
// Some callers cannot let a library call cudaMalloc: a process whose device
// memory has been reserved up front by another allocator (cudaMalloc would
// fail or fragment it), or latency-sensitive code that cannot afford the
// device-wide synchronisation that cudaMalloc and cudaFree may cause.  This
// entry point runs exactly the recursion of spin_invert, but its workspace
// and its status record live in one fixed array in device global memory,
// declared below, instead of memory the library obtains at run time.  Every
// GPU that loads the library keeps that array (8 MB) until the process
// exits.
//
// Host code may not use the array's name as a device address (on the host
// it names a stand-in object); the address is looked up once per device with
// cudaGetSymbolAddress on the first call made with that device current.
#include <mutex>

#include "common.cuh"

namespace spin {
namespace {

constexpr size_t kNoAllocBytes = 8u << 20;        // 8 MB of scratch per device
constexpr size_t kNoAllocHeader = 256;            // status record at the front
constexpr size_t kNoAllocElems = (kNoAllocBytes - kNoAllocHeader) / sizeof(double);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
int noalloc_address(void** out) {
    int dev = 0;
    SPIN_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SPIN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_ptr[dev] == nullptr) {
        void* p = nullptr;
        SPIN_CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return SPIN_OK;
}

}  // namespace
}  // namespace spin

using namespace spin;

extern "C" int spin_invert_noalloc(const double* A, double* X, int64_t n, int64_t lda, int leaf,
                                   spin_stream_t stream) {
    if (n < 1 || lda < n || A == nullptr || X == nullptr || leaf < 0) return SPIN_ERR_INVALID_ARG;
    if (((uintptr_t)A & 7u) != 0 || ((uintptr_t)X & 7u) != 0) return SPIN_ERR_INVALID_ARG;
    int64_t L = leaf > 0 ? leaf : spin_default_leaf(n, SPIN_FP64);
    if (L > n) L = n;
    if (L > kMaxLeaf) return SPIN_ERR_INVALID_ARG;
    const char* a0 = (const char*)A;
    const char* a1 = (const char*)(A + (n - 1) * lda + n);
    const char* x0 = (const char*)X;
    const char* x1 = (const char*)(X + (n - 1) * n + n);
    if (a0 < x1 && x0 < a1) return SPIN_ERR_INVALID_ARG;
    if (fp64_workspace_elems(n, L) > kNoAllocElems) return SPIN_ERR_INVALID_ARG;  // beyond the fixed scratch
    void* base = nullptr;
    int rc = noalloc_address(&base);
    if (rc != SPIN_OK) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t* info = (int32_t*)base;
    double* W = (double*)((unsigned char*)base + kNoAllocHeader);
    // the status record keeps the previous call's contents: clear it first
    SPIN_CUDA_TRY(cudaMemsetAsync(info, 0, INFO_WORDS * sizeof(int32_t), s));
    rc = run_fp64_inversion(A, lda, X, n, n, L, W, info, s);
    if (rc != SPIN_OK) return rc;
    int32_t h[INFO_WORDS] = {0, 0, 0, 0};
    SPIN_CUDA_TRY(cudaMemcpyAsync(h, info, sizeof h, cudaMemcpyDeviceToHost, s));
    SPIN_CUDA_TRY(cudaStreamSynchronize(s));
    return h[INFO_STATUS];
}
