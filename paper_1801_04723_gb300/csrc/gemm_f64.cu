// FP64 level products of the plain method: D = beta*C + alpha*(A B).
//
// Algorithm 1's six products per recursion level (II, III, IV, C12, C21,
// VII; Sec. 3.1) and its two subtractions (V = IV - A22, C11 = I - VII) are
// one kernel here: the subtraction and the sign are the epilogue.
//
// On GB300 the FP64 pipe retires about 2 FMA per clock per SM (DFMA measured
// at ~1.2 TFLOP/s over 152 SMs; DMMA at ~1.05-1.10), so the kernel is
// bounded by the FP64 pipe at any reasonable tiling, and a product runs at
// the rate of the SMs it occupies.  A 64x64 output tile per 256-thread CTA,
// 4x4 register tile per thread, k-step 16 staged through double-buffered
// shared memory, gives 16 independent FMAs per thread per k-slice and needs
// ~0.25 B of L2 traffic per FMA -- far under any memory roof.  Products too
// small to give every SM a 64x64 tile (the deep recursion levels: at n =
// 1024 the three levels have 64, 16 and 4 such tiles) take 32x32 or 16x16
// tiles instead.  Every output is one FMA chain over k in order, whatever
// the tile, so the tile size never changes a result bit.  Operands are
// arbitrary strided views (no alignment beyond 8 B).
#include <math.h>
#include <stdlib.h>

#include <cmath>

#include "common.cuh"

namespace spin {
namespace {

constexpr int BK = 16, NT = 256;
// Tile rows per group of the single-product tile order.  Measured on a
// 4096^3 product (ncu dram__bytes_read.sum + dram__bytes_write.sum, same
// duration every time): 3.87 GB in row-major order, 1.49 GB with groups of
// 8 tile rows, 1.03 GB with 16, against 0.40 GB of operands and result.
constexpr int kTileGroup = 16;

// One TM x TM output tile per 256-thread CTA: thread (tx, ty) of a 16 x 16
// grid owns a (TM/16) x (TM/16) register tile.
template <int TM>
__device__ __forceinline__ void gemm_f64_tile(int64_t m, int64_t n, int64_t k, double alpha,
                                              const double* __restrict__ A, int64_t lda,
                                              const double* __restrict__ B, int64_t ldb, double beta,
                                              const double* C, int64_t ldc, double* D, int64_t ldd,
                                              int64_t tile_m, int64_t tile_n) {
    constexpr int T = TM / 16;        // outputs per thread along each side
    constexpr int BR = NT / TM;       // B tile rows loaded per pass
    __shared__ double As[2][BK][TM + 1];
    __shared__ double Bs[2][BK][TM];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = tile_m * TM, n0 = tile_n * TM;

    // load mapping: A tile (TM x BK): row = ty + 16*i, kk = tx; B tile (BK x TM): kr = tid/TM + BR*i, col = tid%TM
    const int a_kk = tx;
    const int b_col = tid % TM, b_kr = tid / TM;
    double ra[T], rb[T];

    auto load_regs = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < T; i++) {
            const int64_t r = m0 + ty + 16 * i, c = k0 + a_kk;
            ra[i] = (r < m && c < k) ? A[r * lda + c] : 0.0;
            const int64_t kr = k0 + b_kr + BR * i, cc = n0 + b_col;
            rb[i] = (kr < k && cc < n) ? B[kr * ldb + cc] : 0.0;
        }
    };
    auto store_smem = [&](int buf) {
#pragma unroll
        for (int i = 0; i < T; i++) {
            As[buf][a_kk][ty + 16 * i] = ra[i];
            Bs[buf][b_kr + BR * i][b_col] = rb[i];
        }
    };

    double acc[T][T];
#pragma unroll
    for (int i = 0; i < T; i++)
#pragma unroll
        for (int j = 0; j < T; j++) acc[i][j] = 0.0;

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
            double a[T], b[T];
#pragma unroll
            for (int i = 0; i < T; i++) a[i] = As[buf][kk][ty + 16 * i];
#pragma unroll
            for (int j = 0; j < T; j++) b[j] = Bs[buf][kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < T; i++)
#pragma unroll
                for (int j = 0; j < T; j++) acc[i][j] = fma(a[i], b[j], acc[i][j]);
        }
        if (t + 1 < ktiles) {
            store_smem(buf ^ 1);
            __syncthreads();
        }
    }

#pragma unroll
    for (int i = 0; i < T; i++) {
        const int64_t r = m0 + ty + 16 * i;
        if (r >= m) continue;
#pragma unroll
        for (int j = 0; j < T; j++) {
            const int64_t c = n0 + tx + 16 * j;
            if (c >= n) continue;
            double v = alpha * acc[i][j];
            if (beta != 0.0) v = fma(beta, C[r * ldc + c], v);
            D[r * ldd + c] = v;
        }
    }
}

// Output tile of this CTA.  With group > 1 consecutive CTAs walk `group`
// tile rows down before moving one tile column right, so that the CTAs
// resident at once cover a squarer block of the output and share more of
// their A row panels and B column panels in L2; group <= 1 is row-major
// order.  A bijection of the grid either way (the last group may be short).
__device__ __forceinline__ void tile_of(int group, int64_t& tile_m, int64_t& tile_n) {
    if (group <= 1) {
        tile_m = blockIdx.y;
        tile_n = blockIdx.x;
        return;
    }
    const int64_t gx = gridDim.x, gy = gridDim.y;
    const int64_t pid = (int64_t)blockIdx.y * gx + blockIdx.x;
    const int64_t per = (int64_t)group * gx;
    const int64_t g = pid / per, first = g * group;
    const int64_t rows = gy - first < group ? gy - first : (int64_t)group;
    const int64_t local = pid - g * per;
    tile_m = first + local % rows;
    tile_n = local / rows;
}

template <int TM>
__global__ void __launch_bounds__(NT, 2)
gemm_f64_kernel(int64_t m, int64_t n, int64_t k, double alpha, const double* __restrict__ A, int64_t lda,
                const double* __restrict__ B, int64_t ldb, double beta, const double* C, int64_t ldc,
                double* D, int64_t ldd, int group) {
    int64_t tile_m, tile_n;
    tile_of(group, tile_m, tile_n);
    gemm_f64_tile<TM>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, tile_m, tile_n);
}

// Batched form: problem blockIdx.z uses the views described by the BatchView
// operands (same shape for every problem, per-problem base and leading dim).
template <int TM>
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
    gemm_f64_tile<TM>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, const_cast<double*>(d.ptr(z, ldd)), ldd,
                      blockIdx.y, blockIdx.x);
}

// SPIN_F64_TILE=64|32|16 forces a tile size (for measurement); read once.
int forced_tile() {
    static int t = -1;
    if (t < 0) {
        const char* e = getenv("SPIN_F64_TILE");
        const int v = e ? atoi(e) : 0;
        t = (v == 64 || v == 32 || v == 16) ? v : 0;
    }
    return t;
}

// Tile rows per group of the single-product tile order (SPIN_F64_GROUP
// overrides it, for measurement; read once).
int tile_group() {
    static int g = -1;
    if (g < 0) {
        const char* e = getenv("SPIN_F64_GROUP");
        const int v = e ? atoi(e) : 0;
        g = v > 0 ? v : kTileGroup;
    }
    return g;
}

}  // namespace

int forced_f64_tile() { return forced_tile(); }

// Tile size for an m x n product (count of them side by side): the one
// whose busiest SM has the fewest FMAs, ceil(tiles / 152) * TM^2 per
// k, larger tiles preferred unless a smaller one is at least 1.25x better
// (a smaller tile keeps fewer FMAs in flight per thread).
int gemm_f64_tile_size(int64_t m, int64_t n, int64_t count) {
    const int forced = forced_tile();
    if (forced) return forced;
    int best = 64;
    double best_cost = 0.0;
    for (int tm : {64, 32, 16}) {
        const double tiles = (double)((m + tm - 1) / tm) * (double)((n + tm - 1) / tm) * (double)count;
        const double cost = std::ceil(tiles / 152.0) * tm * tm;
        if (tm == 64 || cost * 1.25 <= best_cost) {
            best = tm;
            best_cost = cost;
        }
    }
    return best;
}

int launch_gemm_f64_batched(int64_t m, int64_t n, int64_t k, double alpha, const BatchView& a, const BatchView& b,
                            double beta, const BatchView& c, const BatchView& d, int count, cudaStream_t s) {
    if (m <= 0 || n <= 0 || count <= 0) return SPIN_OK;
    const int tm = gemm_f64_tile_size(m, n, count);
    dim3 grid((unsigned)((n + tm - 1) / tm), (unsigned)((m + tm - 1) / tm), (unsigned)count);
    if (grid.y > 65535u || grid.z > 65535u) return SPIN_ERR_INVALID_ARG;
    if (tm == 64)
        gemm_f64_batched_kernel<64><<<grid, NT, 0, s>>>(m, n, k, alpha, a, b, beta, c, d);
    else if (tm == 32)
        gemm_f64_batched_kernel<32><<<grid, NT, 0, s>>>(m, n, k, alpha, a, b, beta, c, d);
    else
        gemm_f64_batched_kernel<16><<<grid, NT, 0, s>>>(m, n, k, alpha, a, b, beta, c, d);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

int launch_gemm_f64(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                    const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D,
                    int64_t ldd, cudaStream_t s) {
    if (m <= 0 || n <= 0) return SPIN_OK;
    const int tm = gemm_f64_tile_size(m, n, 1);
    dim3 grid((unsigned)((n + tm - 1) / tm), (unsigned)((m + tm - 1) / tm));
    if (grid.y > 65535u) return SPIN_ERR_INVALID_ARG;
    if (tm == 64)
        gemm_f64_kernel<64><<<grid, NT, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, tile_group());
    else if (tm == 32)
        gemm_f64_kernel<32><<<grid, NT, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, tile_group());
    else
        gemm_f64_kernel<16><<<grid, NT, 0, s>>>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, tile_group());
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace spin
