// Internal helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include <atomic>

#include "../../include/spin.h"

namespace spin {

// Device info record layout: int32[4] = {status, leaf_index, column, spare}.
enum { INFO_STATUS = 0, INFO_LEAF = 1, INFO_COL = 2, INFO_WORDS = 4 };

// On failure: remember the message, clear the runtime's last-error slot (so
// that a later, unrelated cudaGetLastError() check does not see it again)
// and return SPIN_ERR_CUDA.
#define SPIN_CUDA_TRY(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            spin::record_cuda_error(_e, #expr, __FILE__, __LINE__);                \
            cudaGetLastError();                                                    \
            return SPIN_ERR_CUDA;                                                  \
        }                                                                          \
    } while (0)

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// One-time set-up per device (cudaFuncSetAttribute applies to the current
// device only): run(f) calls f once for each device it is used on; threads
// that race on a new device may both call f, which is harmless for attribute
// setting.  Devices beyond 64 run f every time.
struct PerDeviceOnce {
    std::atomic<unsigned long long> done{0};
    template <class F>
    int run(F&& f) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) {
            cudaGetLastError();
            return f();
        }
        const unsigned long long bit = (dev >= 0 && dev < 64) ? (1ull << dev) : 0ull;
        if (bit && (done.load(std::memory_order_acquire) & bit)) return 0;
        const int rc = f();
        if (rc == 0 && bit) done.fetch_or(bit, std::memory_order_acq_rel);
        return rc;
    }
};

// The precisions of spin_precision (0, 1 and 3).
inline bool valid_precision(int p) { return p == SPIN_FP64 || p == SPIN_MIXED_BF16X3 || p == SPIN_MIXED_DIGITS; }

// First failure wins: status 0 -> code, then leaf and column are recorded.
__device__ __forceinline__ void record_failure(int32_t* info, int code, int leaf, int col) {
    if (info == nullptr) return;
    if (atomicCAS(&info[INFO_STATUS], 0, code) == 0) {
        info[INFO_LEAF] = leaf;
        info[INFO_COL] = col;
    }
}

// A strided view inside each matrix of a batch: problem z's view starts at
// base[z] + r0 * ld + c0, with ld = lds[z] when lds is given, else ld.
struct BatchView {
    const double* const* base;  // device array of per-problem base pointers
    const int64_t* lds;         // device array of per-problem leading dims, or nullptr
    int64_t ld;                 // uniform leading dim when lds == nullptr
    int64_t r0, c0;
    __device__ __forceinline__ int64_t ld_of(int z) const { return lds ? lds[z] : ld; }
    __device__ __forceinline__ const double* ptr(int z, int64_t l) const { return base[z] + r0 * l + c0; }
};

// ---- kernel launchers (host) ----
// FP64 product tile size (64, 32 or 16) for count m x n products side by side.
int gemm_f64_tile_size(int64_t m, int64_t n, int64_t count);
// The tile SPIN_F64_TILE forces (64, 32 or 16; for measurement), else 0.
int forced_f64_tile();
int launch_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D,
                    int64_t ldd, cudaStream_t s);

int launch_gemm_f64_batched(int64_t m, int64_t n, int64_t k, double alpha, const BatchView& a, const BatchView& b,
                            double beta, const BatchView& c, const BatchView& d, int count, cudaStream_t s);
// Batched leaf: problem z inverts view src(z) into dst(z); scratch(z) = scratch_base + z * scratch_stride
// (L*L doubles each when L > 256); info(z) = info + 4 z; leaf index reported = leaf_index.
int launch_leaf_gj_batched(const BatchView& src, const BatchView& dst, int64_t L, double* scratch_base,
                           int64_t scratch_stride, int32_t* info, int leaf_index, int count, cudaStream_t s);

// Leaf Gauss-Jordan: scratch (L*L doubles) is required when L > 256 (rows may spill to it).
int launch_leaf_gj(const double* A, int64_t lda, double* X, int64_t ldx, int64_t L, double* scratch,
                   int32_t* info, int leaf_index, cudaStream_t s);
size_t leaf_scratch_elems(int64_t L);

// Random butterfly transform (rbt.cu): depth, padded order (a multiple of
// 2^depth), diagonals (2 * depth * np doubles: U's levels, then V's),
// Ar = U^T pad(A) V, and X = crop(V Y U^T) (Y overwritten).
constexpr int kRbtDepth = 2;
int64_t rbt_padded_order(int64_t n, int depth);
int launch_rbt_diagonals(uint64_t seed, int64_t np, int depth, double* out, cudaStream_t s);
int launch_rbt_forward(const double* A, int64_t lda, int64_t n, double* Ar, int64_t np, int depth,
                       const double* diag, cudaStream_t s);
int launch_rbt_backward(double* Y, int64_t np, int depth, const double* diag, double* X, int64_t ldx, int64_t n,
                        cudaStream_t s);
constexpr int64_t kMaxLeaf = 4096;

// FP64 recursion over caller-supplied workspace and info record (api.cu).
size_t fp64_workspace_elems(int64_t n, int64_t leaf);
int run_fp64_inversion(const double* A, int64_t lda, double* X, int64_t ldx, int64_t n, int64_t leaf, double* W,
                       int32_t* info, cudaStream_t s);
int64_t split_order(int64_t n);

// One bucket of `count` matrices of order n inverted in lockstep directly on
// stream s, no graph, every byte of device memory from the caller (batched.cu):
//   bucket_bytes       device bytes run_bucket needs (ws, 256-byte aligned);
//   bucket_host_bytes  pinned host staging bytes (pointer upload, results);
//   run_bucket         A, lda, X: host arrays of device views (X ld = n);
//                      nvalid (host, optional): order of each matrix inside
//                      its identity padding (norms of the refinement cover
//                      that leading block); precision FP64 or BF16X3;
//   bucket_result      after the stream has finished: status, relative
//                      residual (-1 for FP64) and refinement steps of z.
size_t bucket_bytes(int64_t n, int count, const spin_opts& o);
size_t bucket_host_bytes(int count);
int run_bucket(const double* const* A, const int64_t* lda, double* const* X, const int* nvalid, int64_t n,
               int count, const spin_opts& o, void* ws, size_t ws_bytes, void* host_stage, cudaStream_t s);
void bucket_result(const void* host_stage, int count, int z, bool mixed, int32_t* status, double* rel, int* iters);
// Ap = [[A, 0], [0, I]] (np x np, leading dimension np).
int launch_pad_identity(const double* A, int64_t lda, int64_t n, double* Ap, int64_t np, cudaStream_t s);

}  // namespace spin
