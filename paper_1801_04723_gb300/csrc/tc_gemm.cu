// Tensor-core level products for the mixed-precision method.
//
// Algorithm 1's products (Sec. 3.1) dominate the method's cost (Table 3:
// "multiply" is the costliest step once b >= 4).  On GB300 FP64 runs at
// ~1.2 TFLOP/s while BF16 tcgen05 runs at ~1.9 PFLOP/s, so the mixed path
// evaluates an FP64 product A*B as a short sum of BF16 products:
//
//   float mode (bf16x3): a = a_hi + a_lo with a_hi = bf16(a),
//       a_lo = bf16(a - a_hi); A*B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi, all
//       three accumulated in one FP32 TMEM accumulator (~2^-16 relative).
//   exact mode (fixed-point digit slices, the Ozaki splitting): every row of
//       A is scaled by a power of two 2^e_i so that |a_ik| < 2^e_i, and the
//       scaled row is written as digits d_1 + 2^-8 d_2 + ... (|d| <= 128,
//       each an exact BF16 integer); likewise every column of B.  A product
//       of two digits is an integer of at most 2^14, so a run of 512 of them
//       sums exactly in the FP32 accumulator.  Each run is drained into int32
//       registers, and each group of slice pairs of equal weight
//       (t + u = const) is scaled by 2^(e_i + f_j + shift) and added into the
//       FP64 output: the result is exact up to the truncation of the digit
//       expansion, i.e. FP64-class for 5-7 slices.
//
// Kernel: one CTA per 128 x 256 output tile:
//   warp 0      TMA producer (one lane): 4-stage ring of (A 128x64, B 256x64)
//               BF16 tiles, 128-byte swizzled, mbarrier complete_tx.
//   warp 1      TMEM owner (512 columns = two 128 x 256 FP32 accumulators)
//               and MMA issuer (one lane): 4 tcgen05.mma (K = 16) per stage.
//   warps 2..   epilogue: warp w reads TMEM lanes 32*(w%4).. with tcgen05.ld.
//               Float mode uses 8 epilogue warps (128 columns each, no state);
//               exact mode uses 16 (64 columns each), so that the int32 run
//               sums of a thread (64) stay in registers.
// The two accumulators alternate between runs so that draining one overlaps
// the MMAs of the next.  Every wait is bounded (%globaltimer); on a timeout
// the kernel records SPIN_ERR_TIMEOUT, stops issuing, waits (bounded) for
// its own copies and MMAs, frees TMEM and returns.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "common.cuh"
#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace spin {
namespace {

using namespace tc;

constexpr int BM = 128, BK = 64;
#ifndef SPIN_EXACT_BN
#define SPIN_EXACT_BN 128
#define SPIN_EXACT_EPI_WARPS 8
#endif
constexpr int kExactBN = SPIN_EXACT_BN;             // exact-mode tile width
constexpr int kExactEpiWarps = SPIN_EXACT_EPI_WARPS;  // exact-mode epilogue warps
constexpr uint32_t A_TILE_BYTES = BM * BK * 2;  // 16 KB
constexpr int FLUSH_LIMIT = 96;  // exact runs summed in int32 before an FP64 flush (96 * 2^23 < 2^31)
constexpr uint64_t WAIT_LIMIT_NS = 10ull * 1000 * 1000 * 1000;

template <int BN>
struct Cfg {
    static constexpr uint32_t B_TILE_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE_BYTES = A_TILE_BYTES + B_TILE_BYTES;
    static constexpr int STAGES = (196608 / STAGE_BYTES) > 6 ? 6 : (196608 / STAGE_BYTES);  // ~192 KB ring
    static constexpr uint32_t TMEM_COLS = 2 * BN <= 256 ? 256 : 512;  // power of two >= 2 BN
    static constexpr size_t SMEM_BYTES = 1024 /*align slack*/ + STAGES * STAGE_BYTES + 256 /*barriers etc.*/;
};
constexpr int STAGES_MAX = 6;

struct SmemCtl {
    uint64_t full[STAGES_MAX];
    uint64_t empty[STAGES_MAX];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t final_bar;
    uint32_t tmem_base;
    int abort;
};

// 2^e for -1022 <= e <= 1023, built from the exponent bits (exact).
__device__ __forceinline__ double pow2(int e) { return __longlong_as_double((long long)(e + 1023) << 52); }

__device__ __forceinline__ void raise_timeout(SmemCtl* ctl, int* err) {
    ctl->abort = 1;
    if (err) atomicCAS(err, 0, SPIN_ERR_TIMEOUT);
}

template <int EPI_WARPS>
struct Epi {
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    // registers are granted per group of four warps: budget for the rounded-up count
    static constexpr int ALLOC_THREADS = (THREADS + 127) / 128 * 128;
    static constexpr int MAXREG = (65536 / ALLOC_THREADS) / 8 * 8 > 255 ? 248 : (65536 / ALLOC_THREADS) / 8 * 8;
};

template <int BN, bool EXACT, int EPI_WARPS>
__global__ void __maxnreg__(Epi<EPI_WARPS>::MAXREG)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const TcGemmParams p) {
    constexpr int STAGES = Cfg<BN>::STAGES;
    constexpr uint32_t B_TILE_BYTES = Cfg<BN>::B_TILE_BYTES;
    constexpr uint32_t STAGE_BYTES = Cfg<BN>::STAGE_BYTES;
    constexpr uint32_t TMEM_COLS = Cfg<BN>::TMEM_COLS;
    constexpr int HALF = BN / (EPI_WARPS / 4);  // columns per epilogue warp
    static_assert(EPI_WARPS % 4 == 0 && BN % (EPI_WARPS / 4) == 0 && HALF % 16 == 0, "epilogue split");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* smA = base;
    unsigned char* smB = base + STAGES * A_TILE_BYTES;
    SmemCtl* ctl = reinterpret_cast<SmemCtl*>(base + STAGES * STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
    const int KB = (p.K + BK - 1) / BK;
    const int chunk_kb = EXACT ? p.chunk_kb : KB;
    const int nchunks_per_pair = (KB + chunk_kb - 1) / chunk_kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(&ctl->full[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&ctl->tfull[b], 1);
            mbar_init(&ctl->tempty[b], EPI_WARPS);
        }
        mbar_init(&ctl->final_bar, 1);
        ctl->abort = 0;
        fence_mbar_init();
        prefetch_tensormap(&tmA);
        prefetch_tensormap(&tmB);
    }
    if (warp == 1) {
        tmem_alloc(&ctl->tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = ctl->tmem_base;
    volatile int* abort = &ctl->abort;

    if (warp == 0) {
        // ------------------------------------------------------ producer --
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            auto issue = [&](int pair, int kb) -> bool {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(&ctl->empty[s], ph ^ 1u, abort, WAIT_LIMIT_NS)) return false;
                mbar_arrive_expect_tx(&ctl->full[s], STAGE_BYTES);
                tma_load_2d(smA + s * A_TILE_BYTES, &tmA, kb * BK, p.pa[pair] * p.a_rows + m0, &ctl->full[s]);
                tma_load_2d(smB + s * B_TILE_BYTES, &tmB, kb * BK, p.pb[pair] * p.b_rows + n0, &ctl->full[s]);
                it++;
                return true;
            };
            if (!EXACT) {
                for (int kb = 0; kb < KB && ok; kb++)
                    for (int q = 0; q < p.num_pairs && ok; q++) ok = issue(q, kb);
            } else {
                for (int q = 0; q < p.num_pairs && ok; q++)
                    for (int c = 0; c < nchunks_per_pair && ok; c++) {
                        const int kb1 = min(KB, (c + 1) * chunk_kb);
                        for (int kb = c * chunk_kb; kb < kb1 && ok; kb++) ok = issue(q, kb);
                    }
            }
            if (!ok) raise_timeout(ctl, p.err);
            // own copies still in flight: the last min(STAGES, it) loads
            for (int j = max(0, it - STAGES); j < it; j++) {
                volatile int never = 0;
                mbar_wait(&ctl->full[j % STAGES], (uint32_t)((j / STAGES) & 1), &never, WAIT_LIMIT_NS);
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ----------------------------------------------------------- MMA --
        if (lane == 0) {
            const uint32_t idesc = idesc_bf16_f32(BM, BN);
            int it = 0, chunk = 0;
            bool ok = true;
            auto consume = [&](uint32_t d_tmem, bool first_in_chunk) -> bool {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(&ctl->full[s], ph, abort, WAIT_LIMIT_NS)) return false;
                tc_fence_after();
                const uint32_t a_addr = smem_u32(smA + s * A_TILE_BYTES);
                const uint32_t b_addr = smem_u32(smB + s * B_TILE_BYTES);
#pragma unroll
                for (int k = 0; k < BK / 16; k++) {
                    const uint64_t ad = sdesc_kmajor_sw128(a_addr + k * 32);
                    const uint64_t bd = sdesc_kmajor_sw128(b_addr + k * 32);
                    mma_bf16(d_tmem, ad, bd, idesc, (first_in_chunk && k == 0) ? 0u : 1u);
                }
                mma_commit(&ctl->empty[s]);  // frees the stage once these MMAs have read it
                it++;
                return true;
            };
            auto begin_chunk = [&](int& buf) -> bool {
                buf = chunk & 1;
                const uint32_t use = (uint32_t)(chunk >> 1);
                if (!mbar_wait(&ctl->tempty[buf], (use & 1u) ^ 1u, abort, WAIT_LIMIT_NS)) return false;
                tc_fence_after();
                return true;
            };
            if (!EXACT) {
                int buf = 0;
                ok = begin_chunk(buf);
                const uint32_t d = tmem_base + (uint32_t)(buf * BN);
                for (int kb = 0; kb < KB && ok; kb++)
                    for (int q = 0; q < p.num_pairs && ok; q++) ok = consume(d, kb == 0 && q == 0);
                if (ok) mma_commit(&ctl->tfull[buf]);
                chunk++;
            } else {
                for (int q = 0; q < p.num_pairs && ok; q++)
                    for (int c = 0; c < nchunks_per_pair && ok; c++) {
                        int buf = 0;
                        ok = begin_chunk(buf);
                        const uint32_t d = tmem_base + (uint32_t)(buf * BN);
                        const int kb0 = c * chunk_kb, kb1 = min(KB, (c + 1) * chunk_kb);
                        for (int kb = kb0; kb < kb1 && ok; kb++) ok = consume(d, kb == kb0);
                        if (ok) mma_commit(&ctl->tfull[buf]);
                        chunk++;
                    }
            }
            if (!ok) raise_timeout(ctl, p.err);
            // every MMA issued so far has completed once final_bar flips
            mma_commit(&ctl->final_bar);
            volatile int never = 0;
            mbar_wait(&ctl->final_bar, 0u, &never, WAIT_LIMIT_NS);
        }
        __syncwarp();
    } else {
        // ------------------------------------------------------ epilogue --
        const int e = warp - 2;         // 0 .. EPI_WARPS-1
        const int quarter = warp & 3;   // TMEM lane quarter this warp may access
        const int half = e >> 2;        // column group of the tile
        const int row = quarter * 32 + lane;
        const int grow = m0 + row;
        const bool row_ok = grow < p.M;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quarter * 32) << 16);
        const int col0 = n0 + half * HALF;
        double sumsq = 0.0;

        if (!EXACT) {
            bool ok = mbar_wait(&ctl->tfull[0], 0u, abort, WAIT_LIMIT_NS);
            if (!ok) raise_timeout(ctl, p.err);
            tc_fence_after();
            if (ok) {
#pragma unroll 1
                for (int cc = 0; cc < HALF; cc += 16) {
                    uint32_t v[16];
                    tmem_ld_32x32b_x16(lane_addr + (uint32_t)(half * HALF + cc), v);
                    tmem_ld_wait();
                    if (row_ok) {
                        const double* crow = p.C ? p.C + (int64_t)grow * p.ldc : nullptr;
                        double* drow = p.D + (int64_t)grow * p.ldd;
#pragma unroll
                        for (int j = 0; j < 16; j++) {
                            const int gcol = col0 + cc + j;
                            if (gcol < p.N) {
                                double val = p.alpha * (double)__uint_as_float(v[j]);
                                if (p.beta != 0.0) val = fma(p.beta, crow[gcol], val);
                                if (p.add_identity && gcol == grow) val += 1.0;
                                drow[gcol] = val;
                                sumsq = fma(val, val, sumsq);
                            }
                        }
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&ctl->tempty[0]);
        } else {
            int acc[HALF];
#pragma unroll
            for (int j = 0; j < HALF; j++) acc[j] = 0;
            int chunk = 0, since_flush = 0;
            bool first_flush = true, ok = true;
            const int erow = (p.row_exp && row_ok) ? p.row_exp[grow] : 0;
            for (int q = 0; q < p.num_pairs && ok; q++) {
                for (int c = 0; c < nchunks_per_pair && ok; c++) {
                    const int buf = chunk & 1;
                    const uint32_t use = (uint32_t)(chunk >> 1);
                    ok = mbar_wait(&ctl->tfull[buf], use & 1u, abort, WAIT_LIMIT_NS);
                    if (!ok) {
                        raise_timeout(ctl, p.err);
                        break;
                    }
                    tc_fence_after();
#pragma unroll
                    for (int cc = 0; cc < HALF; cc += 16) {
                        uint32_t v[16];
                        tmem_ld_32x32b_x16(lane_addr + (uint32_t)(buf * BN + half * HALF + cc), v);
                        tmem_ld_wait();
#pragma unroll
                        for (int j = 0; j < 16; j++) acc[cc + j] += __float2int_rn(__uint_as_float(v[j]));
                    }
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
                    chunk++;
                    since_flush++;
                    const bool group_end =
                        (c == nchunks_per_pair - 1) && (q == p.num_pairs - 1 || p.pg[q + 1] != p.pg[q]);
                    const bool last = (c == nchunks_per_pair - 1) && (q == p.num_pairs - 1);
                    if (group_end || since_flush >= FLUSH_LIMIT) {
                        if (row_ok) {
                            // exact powers of two: 2^(e_row + shift) * 2^(e_col) * integer
                            const int er = erow + p.group_shift[(int)p.pg[q]];
                            const bool fast = er >= -1000 && er <= 1000;
                            const double srow = fast ? pow2(er) : 0.0;
                            double* drow = p.D + (int64_t)grow * p.ldd;
                            const double* crow = p.C ? p.C + (int64_t)grow * p.ldc : nullptr;
#pragma unroll
                            for (int jj = 0; jj < HALF; jj += 16) {
                                // keep the compiler from hoisting every column's loads at once
                                asm volatile("" ::: "memory");
#pragma unroll
                                for (int j = jj; j < jj + 16; j++) {
                                    const int gcol = col0 + j;
                                    if (gcol < p.N) {
                                        const int ec = p.col_exp ? p.col_exp[gcol] : 0;
                                        double val;
                                        if (fast && ec >= -1000 && ec <= 1000)
                                            val = p.alpha * ((double)acc[j] * srow) * pow2(ec);
                                        else
                                            val = p.alpha * ldexp((double)acc[j], er + ec);
                                        if (first_flush) {
                                            if (p.beta != 0.0) val = fma(p.beta, crow[gcol], val);
                                            if (p.add_identity && gcol == grow) val += 1.0;
                                        } else {
                                            val += drow[gcol];
                                        }
                                        drow[gcol] = val;
                                        if (last) sumsq = fma(val, val, sumsq);
                                    }
                                    acc[j] = 0;
                                }
                            }
                        } else {
#pragma unroll
                            for (int j = 0; j < HALF; j++) acc[j] = 0;
                        }
                        first_flush = false;
                        since_flush = 0;
                    }
                }
            }
        }
        if (p.sumsq) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sumsq += __shfl_down_sync(0xffffffffu, sumsq, off);
            if (lane == 0 && sumsq != 0.0) atomicAdd(p.sumsq, sumsq);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ------------------------------------------------------------ splitting --

__device__ __forceinline__ uint16_t bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// hi = bf16(a) (round to nearest from FP64 via FP32 is not exact, so the
// rounding goes FP64 -> FP32 (RN) -> BF16 (RN); hi is *a* nearby BF16 value
// and lo = bf16(a - hi) captures the next 8 bits either way).
__device__ __forceinline__ void split2(double a, uint16_t& hi, uint16_t& lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn((float)a);
    const double r = a - (double)__bfloat162float(h);
    hi = __bfloat16_as_ushort(h);
    lo = bf16_bits((float)r);
}

// Row-major FP64 (rows x cols, lds) -> two BF16 planes [2][rows][ldd].
__global__ void split_bf16x2_rows_kernel(const double* __restrict__ src, int64_t lds, int rows, int cols,
                                         uint16_t* __restrict__ dst, int64_t ldd, int64_t plane) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / cols), c = (int)(idx % cols);
        uint16_t hi, lo;
        split2(src[(int64_t)r * lds + c], hi, lo);
        dst[(int64_t)r * ldd + c] = hi;
        dst[plane + (int64_t)r * ldd + c] = lo;
    }
}

// FP64 (rows=K x cols=N, lds) -> transposed BF16 planes [2][N][ldd] (N x K).
__global__ void split_bf16x2_cols_kernel(const double* __restrict__ src, int64_t lds, int rows, int cols,
                                         uint16_t* __restrict__ dst, int64_t ldd, int64_t plane) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(int64_t)r * lds + c] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;  // output row c (a column of src), output col r
        if (c < cols && r < rows) {
            uint16_t hi, lo;
            split2(tile[threadIdx.x][i], hi, lo);
            dst[(int64_t)c * ldd + r] = hi;
            dst[plane + (int64_t)c * ldd + r] = lo;
        }
    }
}

// Exponent e with max|x| < 2^e (frexp convention); rows/columns of zeros get
// a small exponent so that every digit is zero.
__device__ __forceinline__ int exp_of_max(double m) {
    if (!(m > 0.0)) return -1000;
    int e;
    frexp(m, &e);
    return e;
}

// Per-row max-exponent of an FP64 matrix (one warp per row) and optional
// sum of squares of all entries.
__global__ void row_exp_kernel(const double* __restrict__ src, int64_t lds, int rows, int cols, int* __restrict__ ex,
                               double* sumsq) {
    const int warps = blockDim.x >> 5;
    const int r = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    double m = 0.0, ss = 0.0;
    for (int c = lane; c < cols; c += 32) {
        const double v = src[(int64_t)r * lds + c];
        m = fmax(m, fabs(v));
        ss = fma(v, v, ss);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        m = fmax(m, __shfl_down_sync(0xffffffffu, m, off));
        ss += __shfl_down_sync(0xffffffffu, ss, off);
    }
    if (lane == 0) {
        ex[r] = exp_of_max(m);
        if (sumsq) atomicAdd(sumsq, ss);
    }
}

// Per-column max-exponent (exponents only grow: atomicMax on a -1000 start).
__global__ void col_exp_kernel(const double* __restrict__ src, int64_t lds, int rows, int cols, int rows_per_block,
                               int* __restrict__ ex, double* sumsq) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r0 = blockIdx.y * rows_per_block;
    const int r1 = min(rows, r0 + rows_per_block);
    double m = 0.0, ss = 0.0;
    if (c < cols)
        for (int r = r0; r < r1; r++) {
            const double v = src[(int64_t)r * lds + c];
            m = fmax(m, fabs(v));
            ss = fma(v, v, ss);
        }
    if (c < cols && m > 0.0) atomicMax(&ex[c], exp_of_max(m));
    if (sumsq) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
        if ((threadIdx.x & 31) == 0 && ss != 0.0) atomicAdd(sumsq, ss);
    }
}

__global__ void fill_int_kernel(int* p, int n, int v) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Digits of x * 2^-e: t = x * 2^(7-e); d_1 = rint(t); t = (t - d_1) * 2^8; ...
template <int MAXS>
__device__ __forceinline__ void digits(double x, int e, int nslices, uint16_t (&d)[MAXS]) {
    double t = ldexp(x, 7 - e);
#pragma unroll
    for (int s = 0; s < MAXS; s++) {
        if (s < nslices) {
            const double di = rint(t);
            d[s] = bf16_bits((float)di);  // |di| <= 128: exact in BF16
            t = (t - di) * 256.0;
        }
    }
}

constexpr int kMaxSlices = 8;

__global__ void ozaki_rows_kernel(const double* __restrict__ src, int64_t lds, int rows, int cols,
                                  const int* __restrict__ ex, int nslices, uint16_t* __restrict__ dst, int64_t ldd,
                                  int64_t plane) {
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / cols), c = (int)(idx % cols);
        uint16_t d[kMaxSlices];
        digits<kMaxSlices>(src[(int64_t)r * lds + c], ex[r], nslices, d);
        for (int s = 0; s < nslices; s++) dst[s * plane + (int64_t)r * ldd + c] = d[s];
    }
}

__global__ void ozaki_cols_kernel(const double* __restrict__ src, int64_t lds, int rows, int cols,
                                  const int* __restrict__ ex, int nslices, uint16_t* __restrict__ dst, int64_t ldd,
                                  int64_t plane) {
    __shared__ double tile[32][33];
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(int64_t)r * lds + c] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) {
            uint16_t d[kMaxSlices];
            digits<kMaxSlices>(tile[threadIdx.x][i], ex[c], nslices, d);
            for (int s = 0; s < nslices; s++) dst[s * plane + (int64_t)c * ldd + r] = d[s];
        }
    }
}

// ----------------------------------------------------------- tensor maps --

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (fn == nullptr) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

int make_map(CUtensorMap* m, const uint16_t* base, int64_t inner, int64_t outer, int64_t ld_elems, uint32_t box_rows) {
    auto fn = encode_fn();
    if (fn == nullptr) return SPIN_ERR_CUDA;
    if (((uintptr_t)base & 15u) != 0 || (ld_elems * 2) % 16 != 0) return SPIN_ERR_INVALID_ARG;
    cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
    cuuint64_t strides[1] = {(cuuint64_t)(ld_elems * 2)};
    cuuint32_t box[2] = {(cuuint32_t)BK, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, (void*)base, dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? SPIN_OK : SPIN_ERR_CUDA;
}

template <int BN, bool EXACT, int EPI_WARPS>
int launch_impl(const TcOperand& a, const TcOperand& b, const TcGemmParams& p, cudaStream_t s) {
    CUtensorMap ta, tb;
    int rc = make_map(&ta, a.base, p.K, (int64_t)a.rows * a.slices, a.ld, BM);
    if (rc) return rc;
    rc = make_map(&tb, b.base, p.K, (int64_t)b.rows * b.slices, b.ld, BN);
    if (rc) return rc;
    static bool attr = false;
    auto kern = tc_gemm_kernel<BN, EXACT, EPI_WARPS>;
    if (!attr) {
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg<BN>::SMEM_BYTES));
        attr = true;
    }
    dim3 grid((unsigned)((p.N + BN - 1) / BN), (unsigned)((p.M + BM - 1) / BM));
    kern<<<grid, Epi<EPI_WARPS>::THREADS, Cfg<BN>::SMEM_BYTES, s>>>(ta, tb, p);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace

int64_t tc_ld(int64_t k) { return (k + 7) / 8 * 8; }

int launch_tc_gemm(const TcOperand& a, const TcOperand& b, const TcGemmParams& prm, cudaStream_t s) {
    if (prm.M <= 0 || prm.N <= 0) return SPIN_OK;
    if (prm.K <= 0 || prm.num_pairs <= 0 || prm.num_pairs > kTcMaxPairs) return SPIN_ERR_INVALID_ARG;
    if (prm.exact && (prm.chunk_kb < 1 || prm.chunk_kb > 8)) return SPIN_ERR_INVALID_ARG;
    TcGemmParams p = prm;
    p.a_rows = a.rows;
    p.b_rows = b.rows;
    if (prm.exact) return launch_impl<kExactBN, true, kExactEpiWarps>(a, b, p, s);
    return launch_impl<256, false, 8>(a, b, p, s);
}

int launch_split_bf16x2(const double* src, int64_t lds, int rows, int cols, bool transpose, uint16_t* dst,
                        int64_t ldd, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return SPIN_OK;
    if (!transpose) {
        const int64_t plane = (int64_t)rows * ldd;
        const int64_t total = (int64_t)rows * cols;
        const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
        split_bf16x2_rows_kernel<<<blocks, 256, 0, s>>>(src, lds, rows, cols, dst, ldd, plane);
    } else {
        const int64_t plane = (int64_t)cols * ldd;
        dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
        split_bf16x2_cols_kernel<<<grid, dim3(32, 8), 0, s>>>(src, lds, rows, cols, dst, ldd, plane);
    }
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

int launch_ozaki_split(const double* src, int64_t lds, int rows, int cols, bool transpose, int nslices, int* ex,
                       uint16_t* dst, int64_t ldd, double* sumsq, cudaStream_t s) {
    if (rows <= 0 || cols <= 0) return SPIN_OK;
    if (nslices < 1 || nslices > kMaxSlices) return SPIN_ERR_INVALID_ARG;
    if (!transpose) {
        row_exp_kernel<<<(rows + 7) / 8, 256, 0, s>>>(src, lds, rows, cols, ex, sumsq);
        const int64_t plane = (int64_t)rows * ldd;
        const int64_t total = (int64_t)rows * cols;
        const int blocks = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
        ozaki_rows_kernel<<<blocks, 256, 0, s>>>(src, lds, rows, cols, ex, nslices, dst, ldd, plane);
    } else {
        fill_int_kernel<<<(cols + 255) / 256, 256, 0, s>>>(ex, cols, -1000);
        const int rpb = 256;
        dim3 g1((unsigned)((cols + 255) / 256), (unsigned)((rows + rpb - 1) / rpb));
        col_exp_kernel<<<g1, 256, 0, s>>>(src, lds, rows, cols, rpb, ex, sumsq);
        const int64_t plane = (int64_t)cols * ldd;
        dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32));
        ozaki_cols_kernel<<<grid, dim3(32, 8), 0, s>>>(src, lds, rows, cols, ex, nslices, dst, ldd, plane);
    }
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace spin
