// Internal helpers shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>

#include "../../include/spin.h"

namespace spin {

// Device info record layout: int32[4] = {status, leaf_index, column, spare}.
enum { INFO_STATUS = 0, INFO_LEAF = 1, INFO_COL = 2, INFO_WORDS = 4 };

#define SPIN_CUDA_TRY(expr)                                                        \
    do {                                                                           \
        cudaError_t _e = (expr);                                                   \
        if (_e != cudaSuccess) {                                                   \
            spin::record_cuda_error(_e, #expr, __FILE__, __LINE__);                \
            return SPIN_ERR_CUDA;                                                  \
        }                                                                          \
    } while (0)

void record_cuda_error(cudaError_t e, const char* what, const char* file, int line);

// First failure wins: status 0 -> code, then leaf and column are recorded.
__device__ __forceinline__ void record_failure(int32_t* info, int code, int leaf, int col) {
    if (info == nullptr) return;
    if (atomicCAS(&info[INFO_STATUS], 0, code) == 0) {
        info[INFO_LEAF] = leaf;
        info[INFO_COL] = col;
    }
}

// ---- kernel launchers (host) ----
int launch_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D,
                    int64_t ldd, cudaStream_t s);

// Leaf Gauss-Jordan: scratch (L*L doubles) is required only when L > 512.
int launch_leaf_gj(const double* A, int64_t lda, double* X, int64_t ldx, int64_t L, double* scratch,
                   int32_t* info, int leaf_index, cudaStream_t s);
size_t leaf_scratch_elems(int64_t L);
constexpr int64_t kMaxLeaf = 4096;

}  // namespace spin
