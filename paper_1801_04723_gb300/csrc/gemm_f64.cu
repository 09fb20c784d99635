// FP64 level products of the plain method: D = beta*C + alpha*(A B).
//
// Algorithm 1's six products per recursion level (II, III, IV, C12, C21,
// VII; Sec. 3.1) and its two subtractions (V = IV - A22, C11 = I - VII) are
// one kernel here: the subtraction and the sign are the epilogue.
//
// On GB300 the FP64 pipe retires about 2 FMA per clock per SM (DFMA measured
// at ~1.2 TFLOP/s over 152 SMs; DMMA at ~1.05-1.10), so the kernel is
// bounded by the FP64 pipe at any reasonable tiling.  A 64x64 output tile
// per 256-thread CTA, 4x4 register tile per thread, k-step 16 staged through
// double-buffered shared memory, gives 16 independent FMAs per thread per
// k-slice and needs ~0.25 B of L2 traffic per FMA -- far under any memory
// roof.  Operands are arbitrary strided views (no alignment beyond 8 B).
#include "common.cuh"

namespace spin {
namespace {

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

__device__ __forceinline__ void gemm_f64_tile(int64_t m, int64_t n, int64_t k, double alpha,
                                              const double* __restrict__ A, int64_t lda,
                                              const double* __restrict__ B, int64_t ldb, double beta,
                                              const double* C, int64_t ldc, double* D, int64_t ldd) {
    __shared__ double As[2][BK][BM + 1];
    __shared__ double Bs[2][BK][BN];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;

    // load mapping: A tile (BM x BK): row = ty + 16*i, kk = tx; B tile (BK x BN): kr = tid/64 + 4*i, col = tid%64
    const int a_kk = tx;
    const int b_col = tid & 63, b_kr = tid >> 6;
    double ra[4], rb[4];

    auto load_regs = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            const int64_t r = m0 + ty + 16 * i, c = k0 + a_kk;
            ra[i] = (r < m && c < k) ? A[r * lda + c] : 0.0;
            const int64_t kr = k0 + b_kr + 4 * i, cc = n0 + b_col;
            rb[i] = (kr < k && cc < n) ? B[kr * ldb + cc] : 0.0;
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int i = 0; i < 4; i++) {
            As[buf][a_kk][ty + 16 * i] = ra[i];
            Bs[buf][b_kr + 4 * i][b_col] = rb[i];
        }
    };

    double acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int j = 0; j < 4; j++) acc[i][j] = 0.0;

    const int64_t ktiles = (k + BK - 1) / BK;
    if (ktiles > 0) {
        load_regs(0);
        store_smem(0);
        __syncthreads();
    }
    for (int64_t t = 0; t < ktiles; t++) {
        const int buf = (int)(t & 1);
        if (t + 1 < ktiles) load_regs((t + 1) * BK);
#pragma unroll
        for (int kk = 0; kk < BK; kk++) {
            double a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; i++) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < 4; j++) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; i++)
#pragma unroll
                for (int j = 0; j < 4; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (t + 1 < ktiles) {
            store_smem(buf ^ 1);
            __syncthreads();
        }
    }

#pragma unroll
    for (int i = 0; i < 4; i++) {
        const int64_t r = m0 + ty + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const int64_t c = n0 + tx + 16 * j;
            if (c >= n) continue;
            double v = alpha * acc[i][j];
            if (beta != 0.0) v = fma(beta, C[r * ldc + c], v);
            D[r * ldd + c] = v;
        }
    }
}

__global__ void __launch_bounds__(NT, 2)
gemm_f64_kernel(int64_t m, int64_t n, int64_t k, double alpha, const double* __restrict__ A, int64_t lda,
                const double* __restrict__ B, int64_t ldb, double beta, const double* C, int64_t ldc,
                double* D, int64_t ldd) {
    gemm_f64_tile(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd);
}

// Batched form: problem blockIdx.z uses the views described by the BatchView
// operands (same shape for every problem, per-problem base and leading dim).
__global__ void __launch_bounds__(NT, 2)
gemm_f64_batched_kernel(int64_t m, int64_t n, int64_t k, double alpha, BatchView a, BatchView b, double beta,
                        BatchView c, BatchView d) {
    const int z = blockIdx.z;
    const int64_t lda = a.ld_of(z), ldb = b.ld_of(z), ldd = d.ld_of(z);
    const double* A = a.ptr(z, lda);
    const double* B = b.ptr(z, ldb);
    const double* C = nullptr;
    int64_t ldc = 0;
    if (beta != 0.0) {
        ldc = c.ld_of(z);
        C = c.ptr(z, ldc);
    }
    gemm_f64_tile(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, const_cast<double*>(d.ptr(z, ldd)), ldd);
}

}  // namespace

int launch_gemm_f64_batched(int64_t m, int64_t n, int64_t k, double alpha, const BatchView& a, const BatchView& b,
                            double beta, const BatchView& c, const BatchView& d, int count, cudaStream_t s) {
    if (m <= 0 || n <= 0 || count <= 0) return SPIN_OK;
    dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM), (unsigned)count);
    if (grid.y > 65535u || grid.z > 65535u) return SPIN_ERR_INVALID_ARG;
    gemm_f64_batched_kernel<<<grid, NT, 0, s>>>(m, n, k, alpha, a, b, beta, c, d);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

int launch_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D,
                    int64_t ldd, cudaStream_t s) {
    if (m <= 0 || n <= 0) return SPIN_OK;
    dim3 grid((unsigned)((n + BN - 1) / BN), (unsigned)((m + BM - 1) / BM));
    if (grid.y > 65535u) return SPIN_ERR_INVALID_ARG;
    gemm_f64_kernel<<<grid, NT, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace spin
