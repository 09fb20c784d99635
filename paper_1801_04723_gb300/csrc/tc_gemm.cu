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
//       of two digits is an integer of at most 2^14, so a run of 1024 of them
//       sums exactly in the FP32 accumulator (every partial sum is an integer
//       of magnitude <= 2^24).  Each run is drained into int32
//       registers, and each group of slice pairs of equal weight
//       (t + u = const) is scaled by 2^(e_i + f_j + shift) and added into the
//       FP64 output: the result is exact up to the truncation of the digit
//       expansion (8 s - 1 bits for s slices), i.e. FP64-class for 6-7 slices.
//       Runs are as long as exactness allows because each run ends with one
//       FP32-to-int32 conversion per output, and conversions issue at about
//       16 per clock per SM: with 9-bit digits (|d| <= 256, runs of 256) a
//       128 x 128 tile needs that whole rate to keep up with the MMAs, and the
//       kernel measured 970 against 1265 TFLOP/s (n = 32768 residual).
//
// Kernel (tc_gemm_kernel): one CTA per output tile (float mode: one CTA per
// SM looping over the tiles, see use_persistent_tiles), warp-specialised:
//   warp 0      TMA producer (one lane): a ~192 KB ring of BF16 operand
//               stages, 128-byte swizzled, mbarrier complete_tx.  Float mode:
//               128 x 256 tiles, 4 stages of one 64-wide k-block; exact mode:
//               128 x 128 tiles, 3 stages of two k-blocks.
//   warp 1      TMEM owner and MMA issuer (one lane): tcgen05.mma kind::f16,
//               K = 16 per instruction, one commit per stage.
//   warps 2..9  epilogue: warp w reads TMEM lanes 32*(w%4).. (tcgen05.ld);
//               the two column halves of the tile go to warps 2-5 and 6-9.
// TMEM holds two FP32 accumulators that alternate between runs, so draining
// one overlaps the MMAs of the next; in exact mode it also holds each
// output's FP64 running sum (two 32-bit columns), so the slice-pair groups
// are summed without global-memory traffic and D is written once.  Every
// wait is bounded (%globaltimer); on a timeout the kernel records
// SPIN_ERR_TIMEOUT, stops issuing, waits (bounded) for its own copies and
// MMAs, frees TMEM and returns.  tc_gemm_pair_kernel is the exact mode on
// CTA pairs (tcgen05 cta_group::2, 256 x 128 tiles), selected by
// SPIN_TC_PAIR=1.
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <stdlib.h>

#include <algorithm>

#include "common.cuh"
#include "tc_gemm.h"
#include "tc_ptx.cuh"

namespace spin {
namespace {

using namespace tc;

constexpr int BM = 128, BK = 64;
constexpr int GROUP_M = 8;  // row blocks per rasterisation band
#ifndef SPIN_EXACT_BN
#define SPIN_EXACT_BN 128
#define SPIN_EXACT_EPI_WARPS 8
#endif
#ifndef SPIN_EXACT_WIDE_MIN_TILES
#define SPIN_EXACT_WIDE_MIN_TILES 608  // 4 waves of 152 SMs
#endif
#ifndef SPIN_FLOAT_BN
#define SPIN_FLOAT_BN 256
#endif
#ifndef SPIN_KSUB_EXACT
#define SPIN_KSUB_EXACT 2
#endif
#ifndef SPIN_KSUB_FLOAT
#define SPIN_KSUB_FLOAT 1
#endif
constexpr int kFloatBN = SPIN_FLOAT_BN;             // float-mode tile width
constexpr int kExactBN = SPIN_EXACT_BN;             // exact-mode tile width (small products)
constexpr int kExactEpiWarps = SPIN_EXACT_EPI_WARPS;  // exact-mode epilogue warps (small products)
// Large exact products use 128 x 256 tiles: an MMA of N = 256 per SM keeps
// the tensor pipe busier than N = 128 (1254 vs 1136 TFLOP/s at n = 8192);
// TMEM then holds only the two accumulators, the running FP64 sums go to D,
// and 16 epilogue warps hold the int32 run sums (64 columns each).  Below a
// few waves of tiles the narrower tiles win (more CTAs, no D traffic), and
// so they do for long K (the n = 32768 residual: ~10 read-modify-write
// passes over D per tile, and the wider tiles lower the clock under the
// power cap without raising the work per clock).
constexpr int64_t kExactWideMinTiles = SPIN_EXACT_WIDE_MIN_TILES;
constexpr int kExactWideMaxK = 16384;
constexpr uint32_t A_TILE_BYTES = BM * BK * 2;  // 16 KB
// 64-wide k-blocks per pipeline stage.  The MMA issuer's fixed cost per
// stage (barrier wait, commit) is spread over 4 * KSUB MMAs: two k-blocks
// for the 128-wide exact tiles (measured 1140 vs 970 TFLOP/s at n = 8192),
// one for the 256-wide float tiles, whose stages are already twice as long
// and which need the deeper ring (4 stages rather than 2).
constexpr int KSUB_EXACT = SPIN_KSUB_EXACT;
constexpr int KSUB_FLOAT = SPIN_KSUB_FLOAT;
constexpr int FLUSH_LIMIT = 96;  // exact runs summed in int32 before an FP64 flush (96 * 2^24 < 2^31)
constexpr uint64_t WAIT_LIMIT_NS = 10ull * 1000 * 1000 * 1000;

template <int BN, int KS>
struct Cfg {
    static constexpr uint32_t B_TILE_BYTES = BN * BK * 2;
    static constexpr uint32_t STAGE_BYTES = KS * (A_TILE_BYTES + B_TILE_BYTES);
    static constexpr int STAGES = (196608 / STAGE_BYTES) > 6 ? 6 : (196608 / STAGE_BYTES);  // ~192 KB ring
    static constexpr uint32_t TMEM_COLS = 2 * BN <= 256 ? 256 : 512;  // power of two >= 2 BN
    static constexpr size_t SMEM_BYTES = 1024 /*align slack*/ + STAGES * STAGE_BYTES + 256 /*barriers etc.*/;
};
constexpr int STAGES_MAX = 8;

struct SmemCtl {
    uint64_t full[STAGES_MAX];
    uint64_t empty[STAGES_MAX];
    uint64_t tfull[2];
    uint64_t tempty[2];
    uint64_t final_bar;
    uint32_t tmem_base;
    int abort;
    int issued;  // pair kernel: stage uses this CTA's producer issued
};

// x * 2^E exactly, for |x| < 2^31, from the bits: the leading one of |x|
// becomes the implicit bit and the rest the fraction.  Integer operations
// only (GB300's FP64 pipe is ~2 operations per clock per SM); ldexp when
// the result would not be a normal double.
__device__ __forceinline__ double scaled_int(int x, int E) {
    if (x == 0) return 0.0;
    const unsigned u = x < 0 ? 0u - (unsigned)x : (unsigned)x;
    const int lz = __clz(u);     // leading one at bit 31 - lz
    const int e = 31 - lz + E;   // exponent of the result
    if (e < -1022 || e > 1023) return ldexp((double)x, E);
    const unsigned long long frac = ((unsigned long long)u << (21 + lz)) & 0xFFFFFFFFFFFFFull;
    const unsigned long long bits =
        ((unsigned long long)(x < 0) << 63) | ((unsigned long long)(e + 1023) << 52) | frac;
    return __longlong_as_double((long long)bits);
}

static_assert(sizeof(SmemCtl) <= 256, "control block");

// Row grow of D (and of C, or null) for problem z.
__device__ __forceinline__ double* out_row(const TcGemmParams& p, int z, int grow) {
    if (!p.batch) return p.D + (int64_t)grow * p.ldd;
    const int64_t ld = p.d_lds ? p.d_lds[z] : p.d_ld;
    return p.d_base[z] + (p.d_r0 + grow) * ld + p.d_c0;
}
__device__ __forceinline__ const double* in_row(const TcGemmParams& p, int z, int grow) {
    if (!p.batch) return p.C ? p.C + (int64_t)grow * p.ldc : nullptr;
    if (!p.c_base) return nullptr;
    const int64_t ld = p.c_lds ? p.c_lds[z] : p.c_ld;
    return p.c_base[z] + (p.c_r0 + grow) * ld + p.c_c0;
}

__device__ __forceinline__ void raise_timeout(SmemCtl* ctl, int* err) {
    ctl->abort = 1;
    if (err) atomicCAS(err, 0, SPIN_ERR_TIMEOUT);
}
// CTA pair: stop both CTAs (the peer's waits read its own abort flag).
__device__ __forceinline__ void raise_pair_error(SmemCtl* ctl, int* err, int code) {
    ctl->abort = 1;
    st_cluster_u32(mapa_u32(smem_u32(&ctl->abort), cluster_ctarank() ^ 1u), 1u);
    if (err) atomicCAS(err, 0, code);
}
__device__ __forceinline__ void raise_timeout_pair(SmemCtl* ctl, int* err) {
    raise_pair_error(ctl, err, SPIN_ERR_TIMEOUT);
}

template <int EPI_WARPS>
struct Epi {
    static constexpr int THREADS = 64 + 32 * EPI_WARPS;
    // registers are granted per group of four warps: budget for the rounded-up count
    static constexpr int ALLOC_THREADS = (THREADS + 127) / 128 * 128;
    static constexpr int MAXREG = (65536 / ALLOC_THREADS) / 8 * 8 > 255 ? 248 : (65536 / ALLOC_THREADS) / 8 * 8;
};

// Exact-mode epilogue of one warp (HALF columns of one TMEM lane quarter):
// drains every exact run from TMEM into int32 sums and, at the end of each
// group of equal-weight slice pairs (or every FLUSH_LIMIT runs), adds the
// group's 2^(e_row + e_col + shift)-scaled sums into the FP64 output.
// Returns this thread's sum of squares of its final outputs.  PAIR: the
// accumulators belong to a CTA pair whose MMA issuer waits on the even
// CTA's tempty barriers (cluster addresses tempty_c0 / tempty_c1); the
// tfull barriers are this CTA's own (the issuer multicasts its commits).
template <int BN, int HALF, bool PAIR, bool TMEM_SUMS = true, int DRAIN = 32, bool PACK = false>
__device__ __forceinline__ double exact_epilogue(const TcGemmParams& p, SmemCtl* ctl, volatile int* abort,
                                                 uint32_t lane_addr, int half, int grow, int col0,
                                                 int nchunks_per_pair, int lane, uint32_t tempty_c0,
                                                 uint32_t tempty_c1, int z, int& chunk, int pack = 1) {
    const bool row_ok = grow < p.M;
    // the sum of squares covers the leading sum_order x sum_order block only
    const int so = p.sum_order ? p.sum_order[z] : 0x7fffffff;
    const bool sum_row = grow < so;
    double sumsq = 0.0;
    // alpha = +-1 (every product of the method) is a sign flip of the integer
    // sums (|sum| < 2^31, no overflow); anything else costs one FP64 multiply
    const int alpha_sign = p.alpha == -1.0 ? -1 : 1;
    const bool alpha_general = p.alpha != 1.0 && p.alpha != -1.0;
    int acc[HALF];
#pragma unroll
    for (int j = 0; j < HALF; j++) acc[j] = 0;
    int since_flush = 0;
    bool first_flush = true, ok = true;
    const int* col_exp = p.col_exp ? p.col_exp + (p.batch ? (int64_t)z * p.N : 0) : nullptr;
    const int erow = (p.row_exp && row_ok) ? p.row_exp[(p.batch ? (int64_t)z * p.M : 0) + grow] : 0;
    // a run covers chunk c of pairs q .. q1-1 (several pairs of one weight
    // when pack > 1: their products then share the run's exact sum)
    for (int q = 0, q1 = 1; q < p.num_pairs && ok; q = q1, q1 = q + 1) {
        if constexpr (PACK)
            while (q1 < p.num_pairs && q1 - q < pack && p.pg[q1] == p.pg[q]) q1++;
        for (int c = 0; c < nchunks_per_pair && ok; c++) {
            const int buf = chunk & 1;
            const uint32_t use = (uint32_t)(chunk >> 1);
            ok = PAIR ? mbar_wait_cluster(&ctl->tfull[buf], use & 1u, abort, WAIT_LIMIT_NS)
                      : mbar_wait(&ctl->tfull[buf], use & 1u, abort, WAIT_LIMIT_NS);
            if (!ok) {
                if (PAIR)
                    raise_timeout_pair(ctl, p.err);
                else
                    raise_timeout(ctl, p.err);
                break;
            }
            tc_fence_after();
            {
                // DRAIN columns per wait (x16 loads in flight), DRAIN registers
#pragma unroll
                for (int c0 = 0; c0 < HALF; c0 += DRAIN) {
                    uint32_t v[DRAIN];
#pragma unroll
                    for (int c1 = 0; c1 < DRAIN; c1 += 16)
                        tmem_ld_32x32b_x16(lane_addr + (uint32_t)(buf * BN + half * HALF + c0 + c1),
                                           *reinterpret_cast<uint32_t(*)[16]>(&v[c1]));
                    tmem_ld_wait();
#pragma unroll
                    for (int j = 0; j < DRAIN; j++) acc[c0 + j] += __float2int_rn(__uint_as_float(v[j]));
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                if (PAIR)
                    mbar_arrive_cluster(buf ? tempty_c1 : tempty_c0);
                else
                    mbar_arrive(&ctl->tempty[buf]);
            }
            chunk++;
            since_flush++;
            const bool group_end = (c == nchunks_per_pair - 1) && (q1 == p.num_pairs || p.pg[q1] != p.pg[q]);
            const bool last = (c == nchunks_per_pair - 1) && (q1 == p.num_pairs);
            if (group_end || since_flush >= FLUSH_LIMIT) {
                // acc * 2^(e_row + e_col + shift) is built from the integer's
                // bits (exact, no FP64 arithmetic); the running FP64 sum of
                // this thread's columns stays in TMEM until the last flush,
                // which writes D once.
                const int er = erow + p.group_shift[(int)p.pg[q]];
                double* drow = out_row(p, z, grow);
                const double* crow = in_row(p, z, grow);
                const uint32_t sum_addr = lane_addr + (uint32_t)(2 * BN + half * 2 * HALF);
                if constexpr (!TMEM_SUMS) {
                    // 256-wide tiles fill TMEM with the two accumulators: the
                    // running sums live in D itself (read-modify-write)
#pragma unroll
                    for (int j = 0; j < HALF; j++) {
                        const int gcol = col0 + j;
                        const bool ok_ij = row_ok && gcol < p.N;
                        if (ok_ij) {
                            const int ec = col_exp ? col_exp[gcol] : 0;
                            double val = scaled_int(alpha_sign * acc[j], er + ec);
                            if (alpha_general) val *= p.alpha;
                            if (first_flush) {
                                if (p.beta != 0.0) val = fma(p.beta, crow[gcol], val);
                                if (p.add_identity && gcol == grow) val += 1.0;
                            } else {
                                val += drow[gcol];
                            }
                            drow[gcol] = val;
                            if (last && sum_row && gcol < so) sumsq = fma(val, val, sumsq);
                        }
                        acc[j] = 0;
                    }
                } else {
#pragma unroll
                    for (int jj = 0; jj < HALF; jj += 8) {
                        uint32_t w[16];  // 8 FP64 running sums as (lo, hi) words
                        if (!first_flush) {
                            tmem_ld_32x32b_x16(sum_addr + (uint32_t)(2 * jj), w);
                            tmem_ld_wait();
                        }
#pragma unroll
                        for (int j = 0; j < 8; j++) {
                            const int gcol = col0 + jj + j;
                            const bool ok_ij = row_ok && gcol < p.N;
                            const int ec = (col_exp && ok_ij) ? col_exp[gcol] : 0;
                            double val = scaled_int(alpha_sign * acc[jj + j], er + ec);
                            if (alpha_general) val *= p.alpha;
                            if (first_flush) {
                                if (p.beta != 0.0 && ok_ij) val = fma(p.beta, crow[gcol], val);
                                if (p.add_identity && gcol == grow) val += 1.0;
                            } else {
                                val += __hiloint2double((int)w[2 * j + 1], (int)w[2 * j]);
                            }
                            if (last) {
                                if (ok_ij) {
                                    drow[gcol] = val;
                                    if (sum_row && gcol < so) sumsq = fma(val, val, sumsq);
                                }
                            } else {
                                w[2 * j] = (uint32_t)__double2loint(val);
                                w[2 * j + 1] = (uint32_t)__double2hiint(val);
                            }
                            acc[jj + j] = 0;
                        }
                        if (!last) tmem_st_32x32b_x16(sum_addr + (uint32_t)(2 * jj), w);
                    }
                    if (!last) tmem_st_wait();
                }
                first_flush = false;
                since_flush = 0;
            }
        }
    }
    return sumsq;
}

// PERSIST: one CTA per SM walks the output tiles of every problem
// (t = blockIdx.x, blockIdx.x + gridDim.x, ...), so that the epilogue of
// one tile overlaps the MMAs of the next in the other TMEM accumulator and
// the set-up (barriers, TMEM, tensor maps) is paid once per SM; otherwise
// one CTA per tile (blockIdx.x) and problem (blockIdx.y).
// PACK (exact mode, K within one run): consecutive slice pairs of one
// weight share a run while their products fit in it.
template <int BN, bool EXACT, int EPI_WARPS, bool PERSIST = false, bool PACK = false>
__global__ void __maxnreg__(Epi<EPI_WARPS>::MAXREG)
tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               const TcGemmParams p) {
    // a problem switched off by its active flag does nothing (every thread
    // of the CTA reads the same flag, before any barrier or TMEM is set up)
    if (!PERSIST && p.active != nullptr && p.active[p.batch ? blockIdx.y : 0] == 0) return;
    // k-blocks per stage (256-wide exact tiles: one, for a 4-stage ring)
    constexpr int KS = EXACT ? (BN >= 256 ? 1 : KSUB_EXACT) : KSUB_FLOAT;
    // exact mode keeps the FP64 running sums in TMEM when they fit beside the
    // two accumulators (128-wide tiles), else in D
    constexpr bool TMEM_SUMS = !EXACT || 4 * BN <= 512;
    using C = Cfg<BN, KS>;
    constexpr int STAGES = C::STAGES;
    constexpr uint32_t B_TILE_BYTES = C::B_TILE_BYTES;
    constexpr uint32_t STAGE_BYTES = C::STAGE_BYTES;
    // exact mode: two FP32 accumulators (+ the FP64 running sums, 2 columns each)
    constexpr uint32_t TMEM_COLS = EXACT ? (TMEM_SUMS ? 4 * BN : 2 * BN) : C::TMEM_COLS;
    static_assert(TMEM_COLS <= 512, "TMEM");
    constexpr int HALF = BN / (EPI_WARPS / 4);  // columns per epilogue warp
    static_assert(EPI_WARPS % 4 == 0 && BN % (EPI_WARPS / 4) == 0 && HALF % 16 == 0, "epilogue split");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* smA = base;                              // [stage][sub] A tiles
    unsigned char* smB = base + STAGES * KS * A_TILE_BYTES;  // [stage][sub] B tiles
    SmemCtl* ctl = reinterpret_cast<SmemCtl*>(base + STAGES * STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Tiles: t = z * tiles_pp + pid (problem z of a batched launch, tile pid
    // of it).  Grouped rasterisation: consecutive tiles sweep a band of
    // GROUP_M row blocks column by column, so the CTAs resident at one time
    // share a few B column blocks and a few A row blocks (L2 reuse) instead
    // of streaming every B block once per row block.
    const int num_m = (p.M + BM - 1) / BM, num_n = (p.N + BN - 1) / BN;
    const int64_t tiles_pp = (int64_t)num_m * num_n;
    const int64_t t_end = PERSIST ? tiles_pp * (p.batch ? p.batch : 1) : 1;
    const int64_t t_first = PERSIST ? (int64_t)blockIdx.x : 0, t_step = PERSIST ? (int64_t)gridDim.x : 1;
    // tile t: problem z, origin (m0, n0); false if its problem is switched off
    auto tile_of = [&](int64_t t, int& z, int& m0, int& n0) -> bool {
        int pid;
        if (PERSIST) {
            z = p.batch ? (int)(t / tiles_pp) : 0;
            pid = (int)(t - (int64_t)z * tiles_pp);
        } else {
            z = p.batch ? (int)blockIdx.y : 0;
            pid = (int)blockIdx.x;
        }
        const int per_group = GROUP_M * num_n;
        const int first_m = (pid / per_group) * GROUP_M;
        const int gsize = min(num_m - first_m, GROUP_M);
        const int in_group = pid % per_group;
        m0 = (first_m + in_group % gsize) * BM;
        n0 = (in_group / gsize) * BN;
        return !(PERSIST && p.active != nullptr && p.active[z] == 0);
    };
    const int KB = (p.K + BK - 1) / BK;
    const int chunk_kb = EXACT ? p.chunk_kb : KB;
    const int nchunks_per_pair = (KB + chunk_kb - 1) / chunk_kb;
    // exact mode, K within one run: consecutive pairs of one weight share a
    // run while the run holds at most chunk_kb k-blocks of products (the sum
    // stays an integer of magnitude <= 2^24), which divides the drains
    const int pack = (PACK && nchunks_per_pair == 1) ? max(1, chunk_kb / KB) : 1;

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
            int z = 0, m0 = 0, n0 = 0;
            // one stage = k-blocks kb .. kb + KS - 1 of one slice pair (past K: zero fill)
            auto issue = [&](int pair, int kb) -> bool {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(&ctl->empty[s], ph ^ 1u, abort, WAIT_LIMIT_NS)) return false;
                mbar_arrive_expect_tx(&ctl->full[s], STAGE_BYTES);
#pragma unroll
                for (int u = 0; u < KS; u++) {
                    tma_load_2d(smA + (s * KS + u) * A_TILE_BYTES, &tmA, (kb + u) * BK,
                                (int)(z * p.a_zrows) + p.pa[pair] * p.a_rows + m0, &ctl->full[s]);
                    tma_load_2d(smB + (s * KS + u) * B_TILE_BYTES, &tmB, (kb + u) * BK,
                                (int)(z * p.b_zrows) + p.pb[pair] * p.b_rows + n0, &ctl->full[s]);
                }
                it++;
                return true;
            };
            for (int64_t t = t_first; t < t_end && ok; t += t_step) {
                if (!tile_of(t, z, m0, n0)) continue;
                if (!EXACT) {
                    for (int kb = 0; kb < KB && ok; kb += KS)
                        for (int q = 0; q < p.num_pairs && ok; q++) ok = issue(q, kb);
                } else {
                    for (int q = 0; q < p.num_pairs && ok; q++)
                        for (int c = 0; c < nchunks_per_pair && ok; c++) {
                            const int kb1 = min(KB, (c + 1) * chunk_kb);
                            for (int kb = c * chunk_kb; kb < kb1 && ok; kb += KS) ok = issue(q, kb);
                        }
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
            // nsub valid k-blocks in this stage; descriptors advance by 32 B per K = 16
            auto consume = [&](uint32_t d_tmem, bool first_in_chunk, int nsub) -> bool {
                const int s = it % STAGES;
                const uint32_t ph = (uint32_t)((it / STAGES) & 1);
                if (!mbar_wait(&ctl->full[s], ph, abort, WAIT_LIMIT_NS)) return false;
                tc_fence_after();
                const uint64_t ad0 = sdesc_kmajor_sw128(smem_u32(smA + s * KS * A_TILE_BYTES));
                const uint64_t bd0 = sdesc_kmajor_sw128(smem_u32(smB + s * KS * B_TILE_BYTES));
#pragma unroll
                for (int u = 0; u < KS; u++) {
                    if (u < nsub) {
#pragma unroll
                        for (int k = 0; k < BK / 16; k++)
                            mma_bf16(d_tmem, ad0 + ((u * A_TILE_BYTES + k * 32) >> 4),
                                     bd0 + ((u * B_TILE_BYTES + k * 32) >> 4), idesc,
                                     (first_in_chunk && u == 0 && k == 0) ? 0u : 1u);
                    }
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
            int z = 0, m0 = 0, n0 = 0;
            for (int64_t t = t_first; t < t_end && ok; t += t_step) {
                if (!tile_of(t, z, m0, n0)) continue;
                if (!EXACT) {
                    int buf = 0;
                    ok = begin_chunk(buf);
                    const uint32_t d = tmem_base + (uint32_t)(buf * BN);
                    for (int kb = 0; kb < KB && ok; kb += KS)
                        for (int q = 0; q < p.num_pairs && ok; q++)
                            ok = consume(d, kb == 0 && q == 0, min(KS, KB - kb));
                    if (ok) mma_commit(&ctl->tfull[buf]);
                    chunk++;
                } else if constexpr (PACK) {
                    // pairs q .. q1-1 of one weight share a run (one chunk each: K fits a run)
                    for (int q = 0, q1 = 1; q < p.num_pairs && ok; q = q1, q1 = q + 1) {
                        while (q1 < p.num_pairs && q1 - q < pack && p.pg[q1] == p.pg[q]) q1++;
                        int buf = 0;
                        ok = begin_chunk(buf);
                        const uint32_t d = tmem_base + (uint32_t)(buf * BN);
                        for (int qq = q; qq < q1 && ok; qq++)
                            for (int kb = 0; kb < KB && ok; kb += KS) ok = consume(d, qq == q && kb == 0, min(KS, KB - kb));
                        if (ok) mma_commit(&ctl->tfull[buf]);
                        chunk++;
                    }
                } else {
                    for (int q = 0; q < p.num_pairs && ok; q++)
                        for (int c = 0; c < nchunks_per_pair && ok; c++) {
                            int buf = 0;
                            ok = begin_chunk(buf);
                            const uint32_t d = tmem_base + (uint32_t)(buf * BN);
                            const int kb0 = c * chunk_kb, kb1 = min(KB, (c + 1) * chunk_kb);
                            for (int kb = kb0; kb < kb1 && ok; kb += KS)
                                ok = consume(d, kb == kb0, min(KS, kb1 - kb));
                            if (ok) mma_commit(&ctl->tfull[buf]);
                            chunk++;
                        }
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
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quarter * 32) << 16);
        int chunk = 0;  // accumulator uses so far (buffer chunk & 1, parity (chunk >> 1) & 1)
        int z = 0, m0 = 0, n0 = 0;
        for (int64_t t = t_first; t < t_end; t += t_step) {
            if (*abort) break;
            if (!tile_of(t, z, m0, n0)) continue;
            const int grow = m0 + row;
            const bool row_ok = grow < p.M;
            const int col0 = n0 + half * HALF;
            double sumsq = 0.0;
            if (!EXACT) {
                const int so = p.sum_order ? p.sum_order[z] : 0x7fffffff;
                const int buf = chunk & 1;
                bool ok = mbar_wait(&ctl->tfull[buf], (uint32_t)((chunk >> 1) & 1), abort, WAIT_LIMIT_NS);
                if (!ok) raise_timeout(ctl, p.err);
                tc_fence_after();
                if (ok) {
#pragma unroll 1
                    for (int cc = 0; cc < HALF; cc += 16) {
                        uint32_t v[16];
                        tmem_ld_32x32b_x16(lane_addr + (uint32_t)(buf * BN + half * HALF + cc), v);
                        tmem_ld_wait();
                        if (row_ok) {
                            const double* crow = in_row(p, z, grow);
                            double* drow = out_row(p, z, grow);
#pragma unroll
                            for (int j = 0; j < 16; j++) {
                                const int gcol = col0 + cc + j;
                                if (gcol < p.N) {
                                    double val = p.alpha * (double)__uint_as_float(v[j]);
                                    if (p.beta != 0.0) val = fma(p.beta, crow[gcol], val);
                                    if (p.add_identity && gcol == grow) val += 1.0;
                                    drow[gcol] = val;
                                    if (grow < so && gcol < so) sumsq = fma(val, val, sumsq);
                                }
                            }
                        }
                    }
                }
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&ctl->tempty[buf]);
                chunk++;
                if (!ok) break;
            } else {
                sumsq = exact_epilogue<BN, HALF, false, TMEM_SUMS, (EPI_WARPS >= 16 ? 16 : 32), PACK>(
                    p, ctl, abort, lane_addr, half, grow, col0, nchunks_per_pair, lane, 0u, 0u, z, chunk, pack);
            }
            if (p.sumsq) {
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) sumsq += __shfl_down_sync(0xffffffffu, sumsq, off);
                if (lane == 0 && sumsq != 0.0) atomicAdd(p.sumsq + (p.batch ? z : 0), sumsq);
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, TMEM_COLS);
    }
}

// ------------------------------------------------ exact mode on CTA pairs --
// The two CTAs of a cluster share one 256 x 128 output tile through
// tcgen05.mma.cta_group::2 (M = 256).  Each CTA loads its own 128 rows of A
// and its own 64 rows of B (half of the tile's 128 columns) into an 8-stage
// ring, so per K-step of 16 a CTA's shared memory supplies 6 KB per MMA
// instead of the 8 KB of the single-CTA 128 x 128 form, and the deeper ring
// covers more copy latency.  Both CTAs' copies of a stage complete on the
// even CTA's full barrier (armed by the even CTA for the pair's bytes); lane
// 0 of warp 1 of the even CTA issues the pair's MMAs and multicasts its
// commits to both CTAs' empty / tfull barriers; each CTA drains its own 128
// TMEM lanes with the exact epilogue, whose tempty arrivals go to the even
// CTA.  At exit the even CTA accounts for every copy either CTA issued
// (arming or cancelling the expected bytes of uses that only one CTA
// issued) and waits for them, so no copy is in flight when the pair leaves.
template <int PBN>
struct PairCfg {
    static constexpr int BNH = PBN / 2;                                  // B rows per CTA
    static constexpr uint32_t B_BYTES = BNH * BK * 2;
    static constexpr uint32_t STAGE_BYTES = KSUB_EXACT * (A_TILE_BYTES + B_BYTES);  // per CTA
    static constexpr int STAGES = (196608 / STAGE_BYTES) > 8 ? 8 : (196608 / STAGE_BYTES);
    static constexpr bool TMEM_SUMS = 4 * PBN <= 512;  // FP64 running sums beside the accumulators
    static constexpr uint32_t TMEM_COLS = TMEM_SUMS ? 4 * PBN : 2 * PBN;
    static constexpr size_t SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + 256;
    static_assert(STAGES >= 2 && STAGES <= STAGES_MAX, "ring");
};

template <int PBN, int EPI_WARPS>
__global__ void __cluster_dims__(2, 1, 1) __maxnreg__(Epi<EPI_WARPS>::MAXREG)
tc_gemm_pair_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                    const TcGemmParams p) {
    // both CTAs of the pair read the same flag: the pair leaves together
    if (p.active != nullptr && p.active[p.batch ? blockIdx.y : 0] == 0) return;
    using C = PairCfg<PBN>;
    constexpr int HALF = PBN / (EPI_WARPS / 4);
    static_assert(EPI_WARPS % 4 == 0 && PBN % (EPI_WARPS / 4) == 0 && HALF % 16 == 0, "epilogue split");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    unsigned char* smA = base;                                    // [stage][sub] A tiles
    unsigned char* smB = base + C::STAGES * KSUB_EXACT * A_TILE_BYTES;  // [stage][sub] B tiles
    SmemCtl* ctl = reinterpret_cast<SmemCtl*>(base + C::STAGES * C::STAGE_BYTES);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t rank = cluster_ctarank();  // 0 issues the pair's MMAs
    const int z = p.batch ? (int)blockIdx.y : 0;
    int m0, n0;  // the pair's tile; grouped rasterisation as in tc_gemm_kernel
    {
        const int num_m = (p.M + 2 * BM - 1) / (2 * BM), num_n = (p.N + PBN - 1) / PBN;
        const int pid = (int)(blockIdx.x >> 1);
        const int per_group = GROUP_M * num_n;
        const int first_m = (pid / per_group) * GROUP_M;
        const int gsize = min(num_m - first_m, GROUP_M);
        const int in_group = pid % per_group;
        m0 = (first_m + in_group % gsize) * 2 * BM;
        n0 = (in_group / gsize) * PBN;
    }
    const int my_m0 = m0 + (int)rank * BM;        // this CTA's A rows = its TMEM lanes
    const int my_n0 = n0 + (int)rank * C::BNH;  // this CTA's B rows
    const int KB = (p.K + BK - 1) / BK;
    const int chunk_kb = p.chunk_kb;
    const int nchunks_per_pair = (KB + chunk_kb - 1) / chunk_kb;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; s++) {
            mbar_init(&ctl->full[s], 1);
            mbar_init(&ctl->empty[s], 1);
        }
        for (int b = 0; b < 2; b++) {
            mbar_init(&ctl->tfull[b], 1);
            mbar_init(&ctl->tempty[b], 2 * EPI_WARPS);
        }
        mbar_init(&ctl->final_bar, 1);
        ctl->abort = 0;
        ctl->issued = 0;
        fence_mbar_init();
        prefetch_tensormap(&tmA);
        prefetch_tensormap(&tmB);
    }
    if (warp == 1) {
        tmem_alloc_pair(&ctl->tmem_base, C::TMEM_COLS);
        tmem_relinquish_pair();
    }
    tc_fence_before();
    cluster_sync_all();  // barriers initialised and TMEM allocated in both CTAs
    tc_fence_after();
    const uint32_t tmem_base = ctl->tmem_base;
    volatile int* abort = &ctl->abort;

    if (warp == 0) {
        // ------------------------------------------ producer (both CTAs) --
        if (lane == 0) {
            int it = 0;
            bool ok = true;
            const uint32_t full0 = mapa_u32(smem_u32(&ctl->full[0]), 0u);  // even CTA's barriers
            for (int q = 0; q < p.num_pairs && ok; q++)
                for (int c = 0; c < nchunks_per_pair && ok; c++) {
                    const int kb1 = min(KB, (c + 1) * chunk_kb);
                    for (int kb = c * chunk_kb; kb < kb1; kb += KSUB_EXACT) {
                        const int s = it % C::STAGES;
                        const uint32_t ph = (uint32_t)((it / C::STAGES) & 1);
                        ok = mbar_wait_cluster(&ctl->empty[s], ph ^ 1u, abort, WAIT_LIMIT_NS) && !*abort;
                        if (!ok) break;
                        if (rank == 0) mbar_arrive_expect_tx(&ctl->full[s], 2 * C::STAGE_BYTES);
                        const uint32_t bar = full0 + (uint32_t)(s * sizeof(uint64_t));
#pragma unroll
                        for (int u = 0; u < KSUB_EXACT; u++) {
                            tma_load_2d_pair(smA + (s * KSUB_EXACT + u) * A_TILE_BYTES, &tmA, (kb + u) * BK,
                                             (int)(z * p.a_zrows) + p.pa[q] * p.a_rows + my_m0, bar);
                            tma_load_2d_pair(smB + (s * KSUB_EXACT + u) * C::B_BYTES, &tmB, (kb + u) * BK,
                                             (int)(z * p.b_zrows) + p.pb[q] * p.b_rows + my_n0, bar);
                        }
                        it++;
                    }
                }
            if (!ok) raise_timeout_pair(ctl, p.err);
            ctl->issued = it;
        }
        __syncwarp();
    } else if (warp == 1) {
        if (lane == 0 && rank == 0) {
            // --------------------------------- MMA issuer (even CTA), M = 256
            bool ok = ld_cluster_u32(mapa_u32(smem_u32(&ctl->tmem_base), 1u)) == tmem_base;
            if (!ok) raise_pair_error(ctl, p.err, SPIN_ERR_CUDA);  // both CTAs must hold the same columns
            const uint32_t idesc = idesc_bf16_f32(2 * BM, PBN);
            int it = 0, chunk = 0;
            for (int q = 0; q < p.num_pairs && ok; q++)
                for (int c = 0; c < nchunks_per_pair && ok; c++) {
                    const int buf = chunk & 1;
                    const uint32_t use = (uint32_t)(chunk >> 1);
                    ok = mbar_wait_cluster(&ctl->tempty[buf], (use & 1u) ^ 1u, abort, WAIT_LIMIT_NS);
                    if (!ok) break;
                    tc_fence_after();
                    const uint32_t d = tmem_base + (uint32_t)(buf * PBN);
                    const int kb0 = c * chunk_kb, kb1 = min(KB, (c + 1) * chunk_kb);
                    for (int kb = kb0; kb < kb1 && ok; kb += KSUB_EXACT) {
                        const int s = it % C::STAGES;
                        ok = mbar_wait_cluster(&ctl->full[s], (uint32_t)((it / C::STAGES) & 1), abort,
                                               WAIT_LIMIT_NS);
                        if (!ok) break;
                        tc_fence_after();
                        const uint64_t ad0 = sdesc_kmajor_sw128(smem_u32(smA + s * KSUB_EXACT * A_TILE_BYTES));
                        const uint64_t bd0 = sdesc_kmajor_sw128(smem_u32(smB + s * KSUB_EXACT * C::B_BYTES));
                        const int nsub = min(KSUB_EXACT, kb1 - kb);
#pragma unroll
                        for (int u = 0; u < KSUB_EXACT; u++) {
                            if (u < nsub) {
#pragma unroll
                                for (int k = 0; k < BK / 16; k++)
                                    mma_bf16_pair(d, ad0 + ((u * A_TILE_BYTES + k * 32) >> 4),
                                                  bd0 + ((u * C::B_BYTES + k * 32) >> 4), idesc,
                                                  (kb == kb0 && u == 0 && k == 0) ? 0u : 1u);
                            }
                        }
                        mma_commit_pair(&ctl->empty[s], (uint16_t)3);  // frees stage s in both CTAs
                        it++;
                    }
                    if (ok) mma_commit_pair(&ctl->tfull[buf], (uint16_t)3);
                    chunk++;
                }
            if (!ok) raise_timeout_pair(ctl, p.err);
            // every MMA issued so far has completed once final_bar flips
            mma_commit_pair(&ctl->final_bar, (uint16_t)1);
            volatile int never = 0;
            mbar_wait_cluster(&ctl->final_bar, 0u, &never, WAIT_LIMIT_NS);
        }
        __syncwarp();
    } else {
        // ------------------------------------------ epilogue (both CTAs) --
        const int e = warp - 2;
        const int quarter = warp & 3;
        const int half = e >> 2;
        const int grow = my_m0 + quarter * 32 + lane;
        const uint32_t lane_addr = tmem_base + ((uint32_t)(quarter * 32) << 16);
        int chunk = 0;
        double sumsq = exact_epilogue<PBN, HALF, true, C::TMEM_SUMS, (EPI_WARPS >= 16 ? 16 : 32)>(
            p, ctl, abort, lane_addr, half, grow, n0 + half * HALF, nchunks_per_pair, lane,
            mapa_u32(smem_u32(&ctl->tempty[0]), 0u), mapa_u32(smem_u32(&ctl->tempty[1]), 0u), z, chunk);
        if (p.sumsq) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) sumsq += __shfl_down_sync(0xffffffffu, sumsq, off);
            if (lane == 0 && sumsq != 0.0) atomicAdd(p.sumsq + (p.batch ? z : 0), sumsq);
        }
    }

    tc_fence_before();
    cluster_sync_all();  // both producers have stopped; no MMA of the pair is in flight
    if (rank == 0 && threadIdx.x == 0) {
        // Copies still in flight can only belong to the last C::STAGES uses
        // (a use is issued after the use C::STAGES earlier was consumed).
        const int own = ctl->issued;
        const int peer = (int)ld_cluster_u32(mapa_u32(smem_u32(&ctl->issued), 1u));
        const int hi = max(own, peer);
        for (int j = max(0, hi - C::STAGES); j < hi; j++) {
            uint64_t* bar = &ctl->full[j % C::STAGES];
            if (j >= own)
                mbar_arrive_expect_tx(bar, C::STAGE_BYTES);  // only the odd CTA issued this use
            else if (j >= peer)
                mbar_complete_tx(bar, C::STAGE_BYTES);  // the odd CTA's share will not come
            volatile int never = 0;
            mbar_wait_cluster(bar, (uint32_t)((j / C::STAGES) & 1), &never, WAIT_LIMIT_NS);
        }
    }
    cluster_sync_all();  // no copy into either CTA is in flight
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc_pair(tmem_base, C::TMEM_COLS);
    }
}

// ------------------------------------------------------------ splitting --

__device__ __forceinline__ uint16_t bf16_bits(float f) {
    return __bfloat16_as_ushort(__float2bfloat16_rn(f));
}

// hi = bf16(x), lo = bf16(x - hi), both computed from xf = fp32(x): one
// FP64 operation per element (GB300's FP64 rate would otherwise bound this
// memory-bound pass); xf differs from x by 2^-24 relative, far below what
// the three-product form keeps (~2^-16).
__device__ __forceinline__ void split2(double a, uint16_t& hi, uint16_t& lo) {
    const float xf = __double2float_rn(a);
    const __nv_bfloat16 h = __float2bfloat16_rn(xf);
    hi = __bfloat16_as_ushort(h);
    lo = bf16_bits(xf - __bfloat162float(h));  // exact in FP32
}

// hi, mid, lo planes: the same from xf with one more level.
__device__ __forceinline__ void split3(double a, uint16_t& hi, uint16_t& mid, uint16_t& lo) {
    const float xf = __double2float_rn(a);
    const __nv_bfloat16 h = __float2bfloat16_rn(xf);
    const float r1 = xf - __bfloat162float(h);  // exact in FP32
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    hi = __bfloat16_as_ushort(h);
    mid = __bfloat16_as_ushort(m);
    lo = bf16_bits(r1 - __bfloat162float(m));  // exact in FP32
}

// Operand source of a split: one FP64 view, or problem z's view of a batch.
// act (optional): problem z is split only while act[z] != 0.  nv
// (optional): the sum of squares of problem z covers only its leading
// nv[z] x nv[z] block (a matrix padded with the identity).
struct SrcOne {
    const double* p;
    int64_t ld;
    const int* act;
    __device__ __forceinline__ const double* row(int, int r) const { return p + (int64_t)r * ld; }
    __device__ __forceinline__ bool on(int) const { return act == nullptr || act[0] != 0; }
    __device__ __forceinline__ int valid(int) const { return 0x7fffffff; }
};
struct SrcMany {
    BatchView v;
    const int* act;
    const int* nv;
    __device__ __forceinline__ const double* row(int z, int r) const {
        const int64_t l = v.ld_of(z);
        return v.base[z] + (v.r0 + r) * l + v.c0;
    }
    __device__ __forceinline__ bool on(int z) const { return act == nullptr || act[z] != 0; }
    __device__ __forceinline__ int valid(int z) const { return nv ? nv[z] : 0x7fffffff; }
};

// Every split kernel handles problem z = blockIdx.z: its planes start at
// dst + z * dzs, its exponents at ex + z * exs, its sum of squares at
// sumsq[z * sss] (sss = 0: one shared sum).

template <class Src>
__global__ void split_bf16x3p_rows_kernel(Src src, int rows, int cols, uint16_t* __restrict__ dst, int64_t ldd,
                                          int64_t plane, int64_t dzs) {
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    dst += z * dzs;
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / cols), c = (int)(idx % cols);
        uint16_t hi, mid, lo;
        split3(src.row(z, r)[c], hi, mid, lo);
        const int64_t o = (int64_t)r * ldd + c;
        dst[o] = hi;
        dst[plane + o] = mid;
        dst[2 * plane + o] = lo;
    }
}

template <class Src>
__global__ void split_bf16x3p_cols_kernel(Src src, int rows, int cols, uint16_t* __restrict__ dst, int64_t ldd,
                                          int64_t plane, int64_t dzs) {
    __shared__ double tile[32][33];
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    dst += z * dzs;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src.row(z, r)[c] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) {
            uint16_t hi, mid, lo;
            split3(tile[threadIdx.x][i], hi, mid, lo);
            const int64_t o = (int64_t)c * ldd + r;
            dst[o] = hi;
            dst[plane + o] = mid;
            dst[2 * plane + o] = lo;
        }
    }
}

// Row-major FP64 (rows x cols) -> two BF16 planes [2][rows][ldd].
template <class Src>
__global__ void split_bf16x2_rows_kernel(Src src, int rows, int cols, uint16_t* __restrict__ dst, int64_t ldd,
                                         int64_t plane, int64_t dzs) {
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    dst += z * dzs;
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / cols), c = (int)(idx % cols);
        uint16_t hi, lo;
        split2(src.row(z, r)[c], hi, lo);
        dst[(int64_t)r * ldd + c] = hi;
        dst[plane + (int64_t)r * ldd + c] = lo;
    }
}

// FP64 (rows=K x cols=N) -> transposed BF16 planes [2][N][ldd] (N x K).
template <class Src>
__global__ void split_bf16x2_cols_kernel(Src src, int rows, int cols, uint16_t* __restrict__ dst, int64_t ldd,
                                         int64_t plane, int64_t dzs) {
    __shared__ double tile[32][33];
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    dst += z * dzs;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src.row(z, r)[c] : 0.0;
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

// Biased exponent field of x (0 for zero and subnormals).  The exponent e
// with max|x| < 2^e (frexp convention) of a row is max(field) - 1022: the
// largest magnitude has the largest field.  Integer work only.
__device__ __forceinline__ int exp_field(double x) {
    return (int)((unsigned long long)__double_as_longlong(x) >> 52) & 0x7FF;
}

// Per-row max exponent of an FP64 matrix (one warp per row) and optional
// sum of squares of all entries.
template <class Src>
__global__ void row_exp_kernel(Src src, int rows, int cols, int* __restrict__ ex, int64_t exs, double* sumsq,
                               int64_t sss) {
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    const int warps = blockDim.x >> 5;
    const int r = blockIdx.x * warps + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (r >= rows) return;
    const double* sr = src.row(z, r);
    const int nv = src.valid(z);
    const bool sum_row = sumsq != nullptr && r < nv;
    int m = 0;
    double ss = 0.0;
    for (int c = lane; c < cols; c += 32) {
        const double v = sr[c];
        m = max(m, exp_field(v));
        if (sum_row && c < nv) ss = fma(v, v, ss);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        m = max(m, __shfl_down_sync(0xffffffffu, m, off));
        ss += __shfl_down_sync(0xffffffffu, ss, off);
    }
    if (lane == 0) {
        ex[z * exs + r] = m - 1022;
        if (sumsq) atomicAdd(sumsq + z * sss, ss);
    }
}

// Per-column max exponent: atomicMax of exponent fields on a zero start,
// converted to the frexp convention by col_exp_finish_kernel.
template <class Src>
__global__ void col_exp_kernel(Src src, int rows, int cols, int rows_per_block, int* __restrict__ ex, int64_t exs,
                               double* sumsq, int64_t sss) {
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    const int r0 = blockIdx.y * rows_per_block;
    const int r1 = min(rows, r0 + rows_per_block);
    int m = 0;
    const int nv = src.valid(z);
    const bool sum_col = sumsq != nullptr && c < nv;
    double ss4[4] = {0.0, 0.0, 0.0, 0.0};  // four FMA chains: a dependent FP64 FMA takes 64+ cycles here
    if (c < cols) {
        int r = r0;
        for (; r + 3 < r1; r += 4) {
#pragma unroll
            for (int u = 0; u < 4; u++) {
                const double v = src.row(z, r + u)[c];
                m = max(m, exp_field(v));
                if (sum_col && r + u < nv) ss4[u] = fma(v, v, ss4[u]);
            }
        }
        for (; r < r1; r++) {
            const double v = src.row(z, r)[c];
            m = max(m, exp_field(v));
            if (sum_col && r < nv) ss4[0] = fma(v, v, ss4[0]);
        }
    }
    double ss = (ss4[0] + ss4[1]) + (ss4[2] + ss4[3]);
    if (c < cols && m > 0) atomicMax(&ex[z * exs + c], m);
    if (sumsq) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) ss += __shfl_down_sync(0xffffffffu, ss, off);
        if ((threadIdx.x & 31) == 0 && ss != 0.0) atomicAdd(sumsq + z * sss, ss);
    }
}

__global__ void col_exp_finish_kernel(int* ex, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) ex[i] -= 1022;
}

__global__ void fill_int_kernel(int* p, int64_t n, int v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// Fixed-point digits of x relative to 2^e (|x| < 2^e): with t = x 2^(7-e)
// (|t| < 128), N = round(|t| 2^(8(s-1))) is an integer below 2^(8s-1);
// its balanced base-256 digits (low digits in [-128, 127], the top one in
// [-128, 128]) are the slices, so x = 2^(e-7) sum_i d_i 2^(-8 i) to within
// half a unit of the last slice.  Integer arithmetic on the IEEE fields.
template <int MAXS>
__device__ __forceinline__ void digits(double x, int e, int nslices, uint16_t (&d)[MAXS]) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x);
    const bool neg = (b >> 63) != 0;
    int fe = (int)(b >> 52) & 0x7FF;
    unsigned long long m = b & ((1ull << 52) - 1);
    if (fe == 0)
        fe = 1;  // subnormal: no implicit bit
    else
        m |= 1ull << 52;
    const int sh = fe - 1075 + 7 - e + 8 * (nslices - 1);  // |x| 2^(7-e+8(s-1)) = m 2^sh
    unsigned long long N;
    if (sh >= 0)
        N = m << sh;  // < 2^(8 s - 1) because |t| < 128
    else if (sh > -64)
        N = (m + (1ull << (-sh - 1))) >> (-sh);
    else
        N = 0;
    int dig[MAXS];
#pragma unroll
    for (int i = MAXS - 1; i >= 1; i--) {
        if (i < nslices) {
            int v = (int)(N & 255u);
            N >>= 8;
            if (v >= 128) {
                v -= 256;
                N += 1;
            }
            dig[i] = v;
        }
    }
    dig[0] = (int)N;
#pragma unroll
    for (int i = 0; i < MAXS; i++)
        if (i < nslices) d[i] = bf16_bits((float)(neg ? -dig[i] : dig[i]));  // |d| <= 128: exact
}

constexpr int kMaxSlices = 8;

template <class Src>
__global__ void ozaki_rows_kernel(Src src, int rows, int cols, const int* __restrict__ ex, int64_t exs, int nslices,
                                  uint16_t* __restrict__ dst, int64_t ldd, int64_t plane, int64_t dzs) {
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    dst += z * dzs;
    ex += z * exs;
    const int64_t total = (int64_t)rows * cols;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(idx / cols), c = (int)(idx % cols);
        uint16_t d[kMaxSlices];
        digits<kMaxSlices>(src.row(z, r)[c], ex[r], nslices, d);
        for (int q = 0; q < nslices; q++) dst[q * plane + (int64_t)r * ldd + c] = d[q];
    }
}

template <class Src>
__global__ void ozaki_cols_kernel(Src src, int rows, int cols, const int* __restrict__ ex, int64_t exs, int nslices,
                                  uint16_t* __restrict__ dst, int64_t ldd, int64_t plane, int64_t dzs) {
    __shared__ double tile[32][33];
    const int z = blockIdx.z;
    if (!src.on(z)) return;
    dst += z * dzs;
    ex += z * exs;
    const int r0 = blockIdx.y * 32, c0 = blockIdx.x * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src.row(z, r)[c] : 0.0;
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) {
            uint16_t d[kMaxSlices];
            digits<kMaxSlices>(tile[threadIdx.x][i], ex[c], nslices, d);
            for (int q = 0; q < nslices; q++) dst[q * plane + (int64_t)c * ldd + r] = d[q];
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

// Float-mode products (bf16x3, bf16x6) run on persistent CTAs, one per SM
// looping over the tiles: a float tile drains its one accumulator after its
// last MMA, which the next tile's MMAs now overlap (n = 8192 bf16x3: 2.51
// against 2.86 ms).  Exact-mode tiles already overlap their many runs'
// drains within the tile and measured the same or 1 % slower persistent
// (n = 8192: 19.49 and 19.30 against 19.31 and 19.34 ms), so they keep one
// CTA per tile.  At n = 32768 the mixed inversion's level products went from
// 1314 to 1356 TFLOP/s and its update from 1499 to 1603 (3.18 -> 3.15 s).
// SPIN_TC_PERSIST=0 turns persistence off, =2 on for both modes (for
// measurement); read once.
int persistent_tiles_mode() {
    static const int v = [] {
        const char* e = getenv("SPIN_TC_PERSIST");
        if (e && e[0] == '0') return 0;
        if (e && e[0] == '2') return 2;
        return 1;
    }();
    return v;
}
bool use_persistent_tiles(bool exact) {
    const int m = persistent_tiles_mode();
    return m == 2 || (m == 1 && !exact);
}

int sm_count() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return 152;
    }
    return n > 0 ? n : 152;
}

template <int BN, bool EXACT, int EPI_WARPS>
int launch_impl(const TcOperand& a, const TcOperand& b, const TcGemmParams& p, cudaStream_t s) {
    CUtensorMap ta, tb;
    const int64_t nz = p.batch ? p.batch : 1;
    int rc = make_map(&ta, a.base, p.K, (int64_t)a.rows * a.slices * nz, a.ld, BM);
    if (rc) return rc;
    rc = make_map(&tb, b.base, p.K, (int64_t)b.rows * b.slices * nz, b.ld, BN);
    if (rc) return rc;
    constexpr size_t smem = Cfg<BN, EXACT ? (BN >= 256 ? 1 : KSUB_EXACT) : KSUB_FLOAT>::SMEM_BYTES;
    static PerDeviceOnce attrs;
    auto kern = tc_gemm_kernel<BN, EXACT, EPI_WARPS, false>;
    auto kern_p = tc_gemm_kernel<BN, EXACT, EPI_WARPS, true>;
    auto kern_k = tc_gemm_kernel<BN, EXACT, EPI_WARPS, false, EXACT>;
    rc = attrs.run([&]() -> int {
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern_p, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern_k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        return SPIN_OK;
    });
    if (rc) return rc;
    const int64_t tiles = (int64_t)((p.N + BN - 1) / BN) * ((p.M + BM - 1) / BM);
    if (tiles > INT32_MAX) return SPIN_ERR_INVALID_ARG;
    // exact products whose K fits one run take the packing form: two or more
    // slice pairs per run when K fits half a run, and one chunk per pair
    // without the chunk loop otherwise (the mixed batch of 4096 matrices:
    // 192.1 against 207.3 ms).  Longer K keeps the other form: the packing
    // form's registers spill more, and the n = 32768 residual ran 1.7x
    // slower in it.
    const int KB = (p.K + BK - 1) / BK;
    const bool pack = EXACT && KB <= p.chunk_kb;
    if (use_persistent_tiles(EXACT)) {
        // one CTA per SM (the ring takes most of the shared memory), each
        // walking every gridDim.x-th tile of all problems
        const int64_t grid = std::min<int64_t>(tiles * nz, sm_count());
        kern_p<<<dim3((unsigned)grid, 1), Epi<EPI_WARPS>::THREADS, smem, s>>>(ta, tb, p);
    } else if (pack) {
        kern_k<<<dim3((unsigned)tiles, (unsigned)nz), Epi<EPI_WARPS>::THREADS, smem, s>>>(ta, tb, p);
    } else {
        kern<<<dim3((unsigned)tiles, (unsigned)nz), Epi<EPI_WARPS>::THREADS, smem, s>>>(ta, tb, p);
    }
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

template <int PBN, int EPI_WARPS>
int launch_pair(const TcOperand& a, const TcOperand& b, const TcGemmParams& p, cudaStream_t s) {
    using C = PairCfg<PBN>;
    CUtensorMap ta, tb;
    const int64_t nz = p.batch ? p.batch : 1;
    int rc = make_map(&ta, a.base, p.K, (int64_t)a.rows * a.slices * nz, a.ld, BM);
    if (rc) return rc;
    rc = make_map(&tb, b.base, p.K, (int64_t)b.rows * b.slices * nz, b.ld, C::BNH);
    if (rc) return rc;
    static PerDeviceOnce attrs;
    auto kern = tc_gemm_pair_kernel<PBN, EPI_WARPS>;
    rc = attrs.run([&]() -> int {
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM_BYTES));
        return SPIN_OK;
    });
    if (rc) return rc;
    const int64_t tiles = (int64_t)((p.N + PBN - 1) / PBN) * ((p.M + 2 * BM - 1) / (2 * BM));
    if (2 * tiles > INT32_MAX) return SPIN_ERR_INVALID_ARG;
    kern<<<dim3((unsigned)(2 * tiles), (unsigned)nz), Epi<EPI_WARPS>::THREADS, C::SMEM_BYTES, s>>>(ta, tb, p);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

// Exact products run on single CTAs (measured 1140 vs 1109 TFLOP/s for the
// pair form at n = 8192); SPIN_TC_PAIR=1 selects the pair kernel.
bool use_pair_kernel() {
    static const int v = [] {
        const char* e = getenv("SPIN_TC_PAIR");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return v != 0;
}

// Large exact products use the 256-wide tiles unless SPIN_TC_WIDE=0
// (SPIN_TC_WIDE=2: at any K as well, for measurement).
int wide_exact_mode() {
    static const int v = [] {
        const char* e = getenv("SPIN_TC_WIDE");
        if (e && e[0] == '0') return 0;
        if (e && e[0] == '2') return 2;
        return 1;
    }();
    return v;
}
bool use_wide_exact() { return wide_exact_mode() != 0; }

}  // namespace

int64_t tc_ld(int64_t k) { return (k + 7) / 8 * 8; }

int launch_tc_gemm(const TcOperand& a, const TcOperand& b, const TcGemmParams& prm, cudaStream_t s) {
    if (prm.M <= 0 || prm.N <= 0) return SPIN_OK;
    if (prm.K <= 0 || prm.num_pairs <= 0 || prm.num_pairs > kTcMaxPairs) return SPIN_ERR_INVALID_ARG;
    // runs <= 1024 k (exactness: 1024 products of at most 2^14) made of whole pipeline stages
    if (prm.exact && (prm.chunk_kb < 1 || prm.chunk_kb > 16 || prm.chunk_kb % KSUB_EXACT != 0)) return SPIN_ERR_INVALID_ARG;
    if (prm.batch < 0 || prm.batch > 65535) return SPIN_ERR_INVALID_ARG;
    if (prm.batch && (int64_t)prm.batch * a.rows * a.slices > INT32_MAX) return SPIN_ERR_INVALID_ARG;
    if (prm.batch && (int64_t)prm.batch * b.rows * b.slices > INT32_MAX) return SPIN_ERR_INVALID_ARG;
    TcGemmParams p = prm;
    p.a_rows = a.rows;
    p.b_rows = b.rows;
    p.a_zrows = p.batch ? (int64_t)a.rows * a.slices : 0;
    p.b_zrows = p.batch ? (int64_t)b.rows * b.slices : 0;
    if (prm.exact) {
        // per problem: many small problems of a batch stay on the narrow tiles
        const int64_t wide_tiles = (int64_t)((p.M + BM - 1) / BM) * ((p.N + 255) / 256);
        if (use_pair_kernel()) {
            if (use_wide_exact() && wide_tiles >= 2 * kExactWideMinTiles)
                return launch_pair<256, 16>(a, b, p, s);
            return launch_pair<128, kExactEpiWarps>(a, b, p, s);
        }
        if (use_wide_exact() && wide_tiles >= kExactWideMinTiles && (p.K <= kExactWideMaxK || wide_exact_mode() == 2))
            return launch_impl<256, true, 16>(a, b, p, s);
        return launch_impl<kExactBN, true, kExactEpiWarps>(a, b, p, s);
    }
    return launch_impl<kFloatBN, false, 8>(a, b, p, s);
}

namespace {

// Grid of a row-wise split: blocks per problem so that the whole launch has
// about 16 blocks per SM.
dim3 rows_grid(int64_t total, int count) {
    const int64_t per = std::max<int64_t>(1, (152 * 16) / std::max(1, count));
    return dim3((unsigned)std::min<int64_t>((total + 255) / 256, per), 1, (unsigned)count);
}

template <class Src>
int split_planes(Src src, int rows, int cols, bool transpose, int planes, uint16_t* dst, int64_t ldd, int count,
                 cudaStream_t s) {
    if (rows <= 0 || cols <= 0 || count <= 0) return SPIN_OK;
    const int64_t plane = (int64_t)(transpose ? cols : rows) * ldd;
    const int64_t dzs = planes * plane;
    if (!transpose) {
        const dim3 g = rows_grid((int64_t)rows * cols, count);
        if (planes == 2)
            split_bf16x2_rows_kernel<Src><<<g, 256, 0, s>>>(src, rows, cols, dst, ldd, plane, dzs);
        else
            split_bf16x3p_rows_kernel<Src><<<g, 256, 0, s>>>(src, rows, cols, dst, ldd, plane, dzs);
    } else {
        const dim3 g((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32), (unsigned)count);
        if (planes == 2)
            split_bf16x2_cols_kernel<Src><<<g, dim3(32, 8), 0, s>>>(src, rows, cols, dst, ldd, plane, dzs);
        else
            split_bf16x3p_cols_kernel<Src><<<g, dim3(32, 8), 0, s>>>(src, rows, cols, dst, ldd, plane, dzs);
    }
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

template <class Src>
int split_digits(Src src, int rows, int cols, bool transpose, int nslices, int* ex, uint16_t* dst, int64_t ldd,
                 double* sumsq, int64_t sss, int count, cudaStream_t s) {
    if (rows <= 0 || cols <= 0 || count <= 0) return SPIN_OK;
    if (nslices < 1 || nslices > kMaxSlices) return SPIN_ERR_INVALID_ARG;
    if (!transpose) {
        const int64_t plane = (int64_t)rows * ldd, dzs = nslices * plane;
        row_exp_kernel<Src><<<dim3((unsigned)((rows + 7) / 8), 1, (unsigned)count), 256, 0, s>>>(
            src, rows, cols, ex, rows, sumsq, sss);
        ozaki_rows_kernel<Src><<<rows_grid((int64_t)rows * cols, count), 256, 0, s>>>(src, rows, cols, ex, rows,
                                                                                      nslices, dst, ldd, plane, dzs);
    } else {
        const int64_t plane = (int64_t)cols * ldd, dzs = nslices * plane, nex = (int64_t)cols * count;
        fill_int_kernel<<<(unsigned)((nex + 255) / 256), 256, 0, s>>>(ex, nex, 0);
        // rows per block: enough blocks to cover the SMs at small orders,
        // at most 256 (fewer atomics at large ones)
        const int64_t col_blocks = (int64_t)((cols + 255) / 256) * count;
        int rpb = (int)std::min<int64_t>(256, std::max<int64_t>(16, (int64_t)rows * col_blocks / 608));
        rpb = (rpb + 7) & ~7;
        const dim3 g1((unsigned)((cols + 255) / 256), (unsigned)((rows + rpb - 1) / rpb), (unsigned)count);
        col_exp_kernel<Src><<<g1, 256, 0, s>>>(src, rows, cols, rpb, ex, cols, sumsq, sss);
        col_exp_finish_kernel<<<(unsigned)((nex + 255) / 256), 256, 0, s>>>(ex, nex);
        const dim3 g((unsigned)((cols + 31) / 32), (unsigned)((rows + 31) / 32), (unsigned)count);
        ozaki_cols_kernel<Src><<<g, dim3(32, 8), 0, s>>>(src, rows, cols, ex, cols, nslices, dst, ldd, plane, dzs);
    }
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace

int launch_split_bf16x2(const double* src, int64_t lds, int rows, int cols, bool transpose, uint16_t* dst,
                        int64_t ldd, cudaStream_t s) {
    return split_planes(SrcOne{src, lds, nullptr}, rows, cols, transpose, 2, dst, ldd, 1, s);
}

int launch_split_bf16x3p(const double* src, int64_t lds, int rows, int cols, bool transpose, uint16_t* dst,
                         int64_t ldd, cudaStream_t s, const int* active) {
    return split_planes(SrcOne{src, lds, active}, rows, cols, transpose, 3, dst, ldd, 1, s);
}

int launch_ozaki_split(const double* src, int64_t lds, int rows, int cols, bool transpose, int nslices, int* ex,
                       uint16_t* dst, int64_t ldd, double* sumsq, cudaStream_t s, const int* active) {
    return split_digits(SrcOne{src, lds, active}, rows, cols, transpose, nslices, ex, dst, ldd, sumsq, 0, 1, s);
}

int launch_split_planes_batched(const BatchView& src, int rows, int cols, bool transpose, int planes,
                                uint16_t* dst, int64_t ldd, int count, cudaStream_t s, const int* active) {
    if (planes != 2 && planes != 3) return SPIN_ERR_INVALID_ARG;
    return split_planes(SrcMany{src, active, nullptr}, rows, cols, transpose, planes, dst, ldd, count, s);
}

int launch_ozaki_split_batched(const BatchView& src, int rows, int cols, bool transpose, int nslices, int* ex,
                               uint16_t* dst, int64_t ldd, double* sumsq, int count, cudaStream_t s,
                               const int* active, const int* valid) {
    return split_digits(SrcMany{src, active, valid}, rows, cols, transpose, nslices, ex, dst, ldd, sumsq, 1, count,
                        s);
}

}  // namespace spin
