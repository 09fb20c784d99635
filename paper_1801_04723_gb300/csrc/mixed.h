// Mixed-precision level products (mixed.cu).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "tc_gemm.h"

namespace spin {

constexpr int kSchurSlices = 7;  // digit slices of the FP64-class Schur complements (55 bits)
constexpr int kLevelSlices = 4;  // digit slices of the level products in SPIN_MIXED_DIGITS (31 bits)
constexpr int kMaxResidualSlices = 7;

// Digit slices of the refinement residual R = I - A X.  The error of the
// computed rel = ||R||_F / (||A||_F ||X||_F) is modelled as
// residual_error_model(n, s); a residual that certifies a result (a
// stopping decision) keeps it within 1 % of tol, the first residual, which
// only feeds the Newton-Schulz update (its error enters the next residual
// additively), within 20 %; each decision adds the model error of its own
// residual to rel before comparing with tol.
double residual_error_model(int64_t n, int s);
int residual_slices_for(int64_t n, double tol);
int first_residual_slices_for(int64_t n, double tol, int sr);
// Products smaller than this in m or n stay in FP64: below it a product has
// a handful of 128 x 256 tiles and a short K, so the tensor-core path (two
// operand splits and a launch that fills a few SMs) costs more than the FP64
// kernel, whose small tiles fill the SMs.  Measured single inversions, bf16x3
// to 1e-10: threshold 128 -> 384 took n = 512 / 1024 / 2048 / 4096 from
// 3.29 / 6.10 / 13.1 / 30.0 ms to 1.82 / 4.57 / 10.4 / 24.7 ms (512 gives the
// same times; 384 keeps orders like 777 on the tensor cores).
constexpr int64_t kTcMin = 384;

// Slice-pair schedules of the tensor-core product forms (fill pa, pb, pg,
// num_pairs and the exactness fields of p).
void tc_pairs_bf16x3(TcGemmParams& p);           // planes hi, lo: hi hi + hi lo + lo hi
void tc_pairs_bf16x6(TcGemmParams& p);           // planes hi, mid, lo: pairs of weight >= 2^-16
void tc_pairs_ozaki(TcGemmParams& p, int slices);  // digit pairs t + u < slices, exact runs of 1024

// A growable device arena for split planes.
struct MixScratch {
    void* base = nullptr;
    size_t cap = 0;
    int reserve(size_t bytes);
};

// Digit planes and row exponents of an A operand split once and reused
// (the refinement multiplies by the same A every iteration).
struct OzakiCachedA {
    uint16_t* planes;
    int* exps;
};

size_t bf16x3_scratch_bytes(int64_t m, int64_t n, int64_t k);
size_t bf16x6_scratch_bytes(int64_t m, int64_t n, int64_t k);
size_t ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices);

int gemm_bf16x3(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, const double* B,
                int64_t ldb, double beta, const double* C, int64_t ldc, double* D, int64_t ldd, void* scratch,
                size_t scratch_bytes, int* err, cudaStream_t s);

int gemm_ozaki(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, const double* B,
               int64_t ldb, double beta, const double* C, int64_t ldc, double* D, int64_t ldd, int slices,
               int add_identity, double* sumsq, double* sumsq_a, double* sumsq_b, void* scratch,
               size_t scratch_bytes, int* err, cudaStream_t s, const OzakiCachedA* cached_a);

// Split-then-multiply in two halves so callers can time them separately.
struct SplitPlan {
    uint16_t* a;    // A planes (rows of A, K-major)
    uint16_t* b;    // B planes (columns of B as rows, K-major)
    int* ea;        // ozaki: row exponents of A
    int* eb;        // ozaki: column exponents of B
    int64_t ld;
    int slices;     // ozaki slice count (bf16x3: 2 planes)
};
int plan_bf16x3(int64_t m, int64_t n, int64_t k, void* scratch, size_t bytes, SplitPlan* sp);
int plan_ozaki(int64_t m, int64_t n, int64_t k, int slices, void* scratch, size_t bytes, SplitPlan* sp);
int split_a_bf16x3(const SplitPlan& sp, const double* A, int64_t lda, int64_t m, int64_t k, cudaStream_t s);
int split_b_bf16x3(const SplitPlan& sp, const double* B, int64_t ldb, int64_t k, int64_t n, cudaStream_t s);
// active (optional, device int): the split / product runs only while *active != 0.
int split_a_ozaki(const SplitPlan& sp, const double* A, int64_t lda, int64_t m, int64_t k, double* sumsq,
                  cudaStream_t s);
int split_b_ozaki(const SplitPlan& sp, const double* B, int64_t ldb, int64_t k, int64_t n, double* sumsq,
                  cudaStream_t s, const int* active = nullptr);
int product_bf16x3(const SplitPlan& sp, int64_t m, int64_t n, int64_t k, double alpha, double beta, const double* C,
                   int64_t ldc, double* D, int64_t ldd, int* err, cudaStream_t s);
// Three-plane form (hi, mid, lo) with the six products of weight <= 2^-16.
int plan_bf16x6(int64_t m, int64_t n, int64_t k, void* scratch, size_t bytes, SplitPlan* sp);
int split_a_bf16x6(const SplitPlan& sp, const double* A, int64_t lda, int64_t m, int64_t k, cudaStream_t s,
                   const int* active = nullptr);
int split_b_bf16x6(const SplitPlan& sp, const double* B, int64_t ldb, int64_t k, int64_t n, cudaStream_t s,
                   const int* active = nullptr);
int product_bf16x6(const SplitPlan& sp, int64_t m, int64_t n, int64_t k, double alpha, double beta, const double* C,
                   int64_t ldc, double* D, int64_t ldd, int* err, cudaStream_t s, const int* active = nullptr);
// pair_slices (0: sp.slices): the pairs t + u < pair_slices of the first
// pair_slices planes of each operand's stack.
int product_ozaki(const SplitPlan& sp, int64_t m, int64_t n, int64_t k, double alpha, double beta, const double* C,
                  int64_t ldc, double* D, int64_t ldd, int add_identity, double* sumsq, int* err, cudaStream_t s,
                  const int* active = nullptr, int pair_slices = 0);

int ozaki_split_a(const double* A, int64_t lda, int64_t m, int64_t k, int slices, OzakiCachedA* out,
                  double* sumsq, cudaStream_t s, const int* active = nullptr);

// Device-side Newton-Schulz control (refine.cu) for `count` matrices whose
// info records (INFO_WORDS int32 each) start at `records`:
//   init    active[z] = (status of z == 0), rel[z] = -1, iters[z] = 0;
//   decide  for every active z: rel[z] = sqrt(nR[z]) / (sqrt(nA[z]) sqrt(nX[z])),
//           iters[z] = it; off when rel <= tol, or (recording
//           SPIN_ERR_NOT_CONVERGED) when rel is not finite or it >= max_refine;
//   finish  a nonzero *err (a bounded wait that gave up) becomes the status of
//           every matrix still at SPIN_OK.
int launch_refine_init(const int32_t* records, int count, int* active, double* rel, int* iters, cudaStream_t s);
// margin: the model error of this round's residual; converged when rel + margin <= tol.
int launch_refine_decide(const double* nA, const double* nX, const double* nR, int count, double tol, double margin,
                         int it, int max_refine, int* active, double* rel, int* iters, int32_t* records,
                         cudaStream_t s);
int launch_refine_finish(const int* err, int32_t* records, int count, cudaStream_t s);

}  // namespace spin
