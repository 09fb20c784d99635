// Device-side control of the Newton-Schulz refinement X <- X + X (I - A X)
// (the iteration the paper cites as the stabiliser of Strassen's inversion,
// Sec. 2.1), for one matrix or for every matrix of a batch.
//
// Each matrix z has an active flag.  Every refinement round enqueues the same
// launches (split X, residual R = I - A X, decision, split X and R, update);
// the tensor-core products and the splits of a matrix whose flag is 0 return
// at once, so a round costs a matrix nothing once it has converged.  The
// decision kernel reads the round's sums of squares, computes
// rel = ||R||_F / (||A||_F ||X||_F) and switches the matrix off when
// rel + margin <= tol, margin being the model error of that round's residual
// (converged), when rel is not finite, or when the iteration cap is reached
// (both recorded as SPIN_ERR_NOT_CONVERGED, leaf and column -1, unless a
// status is already set).
// No host read happens between rounds: a mixed inversion is one stream of
// launches (and, batched, one CUDA graph), and the result of each matrix
// depends only on that matrix, not on what it is batched with.
#include <math.h>

#include "common.cuh"
#include "mixed.h"

namespace spin {
namespace {

// active = (no failure recorded by the recursion), rel = -1, iters = 0.
__global__ void refine_init_kernel(const int32_t* records, int count, int* active, double* rel, int* iters) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= count) return;
    active[z] = records[(int64_t)z * INFO_WORDS + INFO_STATUS] == 0 ? 1 : 0;
    rel[z] = -1.0;
    iters[z] = 0;
}

__global__ void refine_decide_kernel(const double* nA, const double* nX, const double* nR, int count, double tol,
                                     double margin, int it, int max_refine, int* active, double* rel, int* iters,
                                     int32_t* records) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= count || active[z] == 0) return;
    const double r = sqrt(nR[z]) / (sqrt(nA[z]) * sqrt(nX[z]));
    rel[z] = r;
    iters[z] = it;
    if (r + margin <= tol) {
        active[z] = 0;
    } else if (!(r == r) || it >= max_refine) {
        active[z] = 0;
        record_failure(records + (int64_t)z * INFO_WORDS, SPIN_ERR_NOT_CONVERGED, -1, -1);
    }
}

// A bounded wait of a tensor-core launch that gave up makes every result
// it could have touched suspect: record it for every matrix still at SPIN_OK.
__global__ void refine_finish_kernel(const int* err, int32_t* records, int count) {
    const int z = blockIdx.x * blockDim.x + threadIdx.x;
    if (z >= count) return;
    const int e = *err;
    if (e != 0) record_failure(records + (int64_t)z * INFO_WORDS, e, -1, -1);
}

unsigned blocks_for(int count) { return (unsigned)((count + 255) / 256); }

}  // namespace

int launch_refine_init(const int32_t* records, int count, int* active, double* rel, int* iters, cudaStream_t s) {
    if (count <= 0) return SPIN_OK;
    refine_init_kernel<<<blocks_for(count), 256, 0, s>>>(records, count, active, rel, iters);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

int launch_refine_decide(const double* nA, const double* nX, const double* nR, int count, double tol, double margin,
                         int it, int max_refine, int* active, double* rel, int* iters, int32_t* records,
                         cudaStream_t s) {
    if (count <= 0) return SPIN_OK;
    refine_decide_kernel<<<blocks_for(count), 256, 0, s>>>(nA, nX, nR, count, tol, margin, it, max_refine, active,
                                                           rel, iters, records);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

int launch_refine_finish(const int* err, int32_t* records, int count, cudaStream_t s) {
    if (count <= 0 || err == nullptr) return SPIN_OK;
    refine_finish_kernel<<<blocks_for(count), 256, 0, s>>>(err, records, count);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace spin
