// Host/device interface of the tensor-core product kernel (tc_gemm.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace spin {

constexpr int kTcMaxPairs = 32;
constexpr int kTcMaxGroups = 16;

// One operand as a stack of BF16 slices: slice s is a rows x K row-major
// (K-major) matrix at base + s * rows * ld; ld is a multiple of 8 elements.
struct TcOperand {
    const uint16_t* base;
    int rows;    // rows per slice: M for the A operand, N for the B operand (B stored transposed)
    int slices;
    int64_t ld;
};

// D = beta*C + alpha * sum over slice pairs (+ I when add_identity).
struct TcGemmParams {
    int M, N, K;
    int a_rows, b_rows;     // filled by launch_tc_gemm
    int num_pairs;
    int8_t pa[kTcMaxPairs];  // A slice of each pair
    int8_t pb[kTcMaxPairs];  // B slice of each pair
    int8_t pg[kTcMaxPairs];  // group of each pair (pairs sorted by group)
    int exact;               // 0: one FP32 accumulation of all pairs; 1: exact integer runs
    int chunk_kb;            // exact mode: 64-wide k-blocks per exact run
    int group_shift[kTcMaxGroups];  // exact mode: power-of-two weight of each group
    double alpha, beta;
    const double* C;
    int64_t ldc;
    double* D;
    int64_t ldd;
    const int* row_exp;      // exact mode: 2^row_exp[i] scales row i of A
    const int* col_exp;      // exact mode: 2^col_exp[j] scales column j of B
    int add_identity;
    double* sumsq;           // if set: += sum of squares of the final D values
    int* err;                // set to SPIN_ERR_TIMEOUT if a bounded wait gives up
    const int* active;       // if set: problem z runs only while active[z] != 0 (batch = 0: active[0])
    const int* sum_order;    // if set: sumsq covers rows and columns < sum_order[z] only
    // Batched launches (batch > 0): problem z = blockIdx.y.  The operand
    // planes of problem z follow those of problem z - 1 in the slice stack
    // (a_zrows = slices * rows of one problem, filled by launch_tc_gemm);
    // C and D of problem z are views base[z] + (r0 + i) * ld + c0 with ld =
    // lds[z] (or the uniform ld when lds is null); row_exp / col_exp hold M
    // (N) entries per problem; sumsq has one entry per problem.  C, ldc, D
    // and ldd are unused.
    int batch;
    int64_t a_zrows, b_zrows;
    const double* const* c_base;
    const int64_t* c_lds;
    int64_t c_ld, c_r0, c_c0;
    double* const* d_base;
    const int64_t* d_lds;
    int64_t d_ld, d_r0, d_c0;
};

int64_t tc_ld(int64_t k);
int launch_tc_gemm(const TcOperand& a, const TcOperand& b, const TcGemmParams& p, cudaStream_t s);
// FP64 view -> (hi, mid, lo) BF16 planes; transpose=true writes the cols x rows transpose.
// active (optional, device): split only while *active != 0.
int launch_split_bf16x3p(const double* src, int64_t lds, int rows, int cols, bool transpose, uint16_t* dst,
                         int64_t ldd, cudaStream_t s, const int* active = nullptr);
// FP64 view -> (hi, lo) BF16 planes; transpose=true writes the cols x rows transpose.
int launch_split_bf16x2(const double* src, int64_t lds, int rows, int cols, bool transpose, uint16_t* dst,
                        int64_t ldd, cudaStream_t s);
// FP64 view -> nslices fixed-point digit planes plus per-row (or, transposed,
// per-column) exponents in ex; sumsq (optional) += sum of squares of src.
int launch_ozaki_split(const double* src, int64_t lds, int rows, int cols, bool transpose, int nslices, int* ex,
                       uint16_t* dst, int64_t ldd, double* sumsq, cudaStream_t s, const int* active = nullptr);

// Batched forms: problem z's FP64 view is src(z); its planes start at
// dst + z * planes * (transpose ? cols : rows) * ldd (the slice stack a
// batched product expects), its exponents at ex + z * (rows or cols) and its
// sum of squares at sumsq[z] (sumsq optional); problem z is split only while
// active[z] != 0 (active optional, device); with valid (optional, device) the
// sum of squares of problem z covers its leading valid[z] x valid[z] block.
int launch_split_planes_batched(const BatchView& src, int rows, int cols, bool transpose, int planes,
                                uint16_t* dst, int64_t ldd, int count, cudaStream_t s, const int* active = nullptr);
int launch_ozaki_split_batched(const BatchView& src, int rows, int cols, bool transpose, int nslices, int* ex,
                               uint16_t* dst, int64_t ldd, double* sumsq, int count, cudaStream_t s,
                               const int* active = nullptr, const int* valid = nullptr);

}  // namespace spin
