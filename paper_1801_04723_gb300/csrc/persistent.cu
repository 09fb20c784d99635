// The plain batched inversion as ONE persistent launch over a device-side
// task list.
//
// spin_invert_batched groups matrices by order; every matrix of a bucket
// has the same recursion (Algorithm 1: leaves, and per node the six level
// products with the subtraction and the sign in their epilogues).  The host
// turns each bucket's recursion into a list of stages once (batched.cu),
// and the stages of all buckets into one global task order: stage position
// first (every bucket's first leaf, then every bucket's first product, ...),
// larger orders first within a position.  A task is one stage applied to
// one matrix and one output tile (a leaf is one task).
//
// Every CTA of this kernel loops: take the next task index from a global
// counter, wait until the matrix's earlier stages are done (a per-matrix
// counter of finished tasks reaches the stage's `need`), run the task, count
// it as finished.  Tasks are taken in list order and a task only waits for
// tasks before it in the list, which CTAs already running have taken, so
// the lowest unfinished task can always proceed: the schedule cannot
// deadlock, whatever the number of CTAs resident.  The waits are bounded
// all the same (a wait that runs out records SPIN_ERR_TIMEOUT, and every
// later task skips its work, so the launch drains).
//
// Against the lockstep form (one launch per stage and bucket, buckets on a
// pool of streams), the SMs never wait for the slowest matrix of a level:
// a leaf's latency-bound pivot steps share the SM with product tiles of
// other matrices, and a bucket's deep levels overlap other buckets' work.
//
// Arithmetic: the product tiles compute every output as one FMA chain over
// k in order, then alpha * acc (+ beta * C), and the leaves run the one-CTA
// Gauss-Jordan body -- the operations of the lockstep kernels, so the
// results are the same bit for bit.  Data written by one CTA is read by
// another during the launch, so operand loads go through L2 only
// (ld.global.cg): a non-coherent L1 line could otherwise hold a stale copy.
#include <algorithm>

#include "common.cuh"
#include "leaf_core.cuh"
#include "persistent.h"
#include "tc_ptx.cuh"

namespace spin {
namespace {

constexpr int PBK = 16;  // k-step of a product tile

template <int TM>
constexpr size_t ptile_smem() {
    return 2 * PBK * (TM + 1) * sizeof(double) + 2 * PBK * TM * sizeof(double);
}

// One TM x TM output tile of D = beta C + alpha A B (m x n, inner order k)
// by the 256 threads of the CTA: thread (tx, ty) of a 16 x 16 grid owns a
// (TM/16) x (TM/16) register tile; A and B go through double-buffered
// shared memory in k-steps of 16.
template <int TM>
__device__ __forceinline__ void ptile(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                                      const double* B, int64_t ldb, double beta, const double* C, int64_t ldc,
                                      double* D, int64_t ldd, int64_t tile_m, int64_t tile_n, unsigned char* smem) {
    constexpr int T = TM / 16;   // outputs per thread along each side
    constexpr int BR = NT / TM;  // B rows loaded per pass
    typedef double ATile[PBK][TM + 1];
    typedef double BTile[PBK][TM];
    ATile* As = reinterpret_cast<ATile*>(smem);
    BTile* Bs = reinterpret_cast<BTile*>(smem + 2 * sizeof(ATile));
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = tile_m * TM, n0 = tile_n * TM;
    const int a_kk = tx;
    const int b_col = tid % TM, b_kr = tid / TM;
    double ra[T], rb[T];

    auto load_regs = [&](int64_t k0) {
#pragma unroll
        for (int i = 0; i < T; i++) {
            const int64_t r = m0 + ty + 16 * i, c = k0 + a_kk;
            ra[i] = (r < m && c < k) ? __ldcg(A + r * lda + c) : 0.0;
            const int64_t kr = k0 + b_kr + BR * i, cc = n0 + b_col;
            rb[i] = (kr < k && cc < n) ? __ldcg(B + kr * ldb + cc) : 0.0;
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

    const int64_t ktiles = (k + PBK - 1) / PBK;
    if (ktiles > 0) {
        load_regs(0);
        store_smem(0);
        __syncthreads();
    }
    for (int64_t t = 0; t < ktiles; t++) {
        const int buf = (int)(t & 1);
        if (t + 1 < ktiles) load_regs((t + 1) * PBK);
#pragma unroll
        for (int kk = 0; kk < PBK; kk++) {
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
            if (beta != 0.0) v = fma(beta, __ldcg(C + r * ldc + c), v);
            D[r * ldd + c] = v;
        }
    }
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Start of view v inside matrix z, and its leading dimension.
__device__ __forceinline__ const double* view_ptr(const PView& v, const PersistentArgs& p, int z, int64_t& ld) {
    const double* base;
    if (v.src == 0) {
        base = p.a_base[z];
        ld = p.a_ld[z];
    } else if (v.src == 1) {
        base = p.x_base[z];
        ld = v.ld;
    } else {
        base = p.w_base[z];
        ld = v.ld;
    }
    return base + v.r0 * ld + v.c0;
}

constexpr int kStageWords = (int)(sizeof(PStage) / sizeof(uint64_t));
static_assert(sizeof(PStage) % sizeof(uint64_t) == 0, "PStage is copied as 8-byte words");

__global__ void __launch_bounds__(NT, 2) persistent_batch_kernel(PersistentArgs p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ PStage s_st;
    __shared__ long long s_local;
    __shared__ int s_stage, s_z, s_skip;
    const int tid = threadIdx.x;
    int cursor = 0;  // thread 0: the stage of this CTA's previous task (task indices only grow)
    // thread 0 takes the index of its next task while it runs the current
    // one (the atomic's latency hides behind the task); holding one task
    // ahead keeps the schedule free of deadlock: the lowest unfinished task
    // is either running or held by a CTA whose running task is finished
    unsigned long long t_next = 0;
    if (tid == 0) t_next = atomicAdd(p.next, 1ull);
    for (;;) {
        if (tid == 0) {
            const long long total = p.start[p.nstages];
            const long long t = (long long)t_next;
            if (t < total) t_next = atomicAdd(p.next, 1ull);
            int g = -1, z = 0, skip = 0;
            long long local = 0;
            if (t < total) {
                // the stage g with start[g] <= t < start[g + 1]: gallop from the cursor, then bisect
                int lo = cursor, hi = cursor + 1, step = 1;
                while (hi < p.nstages && p.start[hi] <= t) {
                    lo = hi;
                    hi = min(p.nstages, hi + step);
                    step <<= 1;
                }
                while (hi - lo > 1) {
                    const int mid = (lo + hi) >> 1;
                    if (p.start[mid] <= t)
                        lo = mid;
                    else
                        hi = mid;
                }
                g = cursor = lo;
                local = t - p.start[g];
                const uint64_t* src = reinterpret_cast<const uint64_t*>(p.stages + g);
                uint64_t* dst = reinterpret_cast<uint64_t*>(&s_st);
#pragma unroll
                for (int w = 0; w < kStageWords; w++) dst[w] = src[w];
                z = s_st.first + (int)(local / s_st.tiles);
                const unsigned need = (unsigned)s_st.need;
                if (ld_acquire_u32(p.done + z) < need) {
                    const uint64_t t0 = tc::globaltimer_ns();
                    for (unsigned spins = 1;; spins++) {
                        if (ld_acquire_u32(p.done + z) >= need) break;
                        if (*(volatile int*)p.err != 0) break;
                        __nanosleep(200);
                        if ((spins & 15u) == 0 && tc::globaltimer_ns() - t0 > p.limit_ns) {
                            atomicExch(p.err, (int)SPIN_ERR_TIMEOUT);
                            break;
                        }
                    }
                }
                skip = *(volatile int*)p.err != 0;
            }
            s_stage = g;
            s_local = local;
            s_z = z;
            s_skip = skip;
        }
        __syncthreads();
        if (s_stage < 0) break;
        const long long clk0 = (tid == 0 && p.bucket_clocks != nullptr) ? clock64() : 0;
        const int z = s_z;
        int32_t* info = p.records + (int64_t)z * INFO_WORDS;
        if (s_skip) {
            if (tid == 0) record_failure(info, SPIN_ERR_TIMEOUT, -1, -1);
        } else if (s_st.kind == PSTAGE_LEAF) {
            int64_t lds, ldd;
            const double* src = view_ptr(s_st.a, p, z, lds);
            double* dst = const_cast<double*>(view_ptr(s_st.d, p, z, ldd));
            leaf_gj_cta_body<true>(src, lds, dst, ldd, (int)s_st.m, info, s_st.leaf_index, smem);
        } else {
            const int64_t tile = s_local % s_st.tiles;
            const int64_t tile_m = tile / s_st.tiles_n, tile_n = tile % s_st.tiles_n;
            int64_t lda, ldb, ldc = 0, ldd;
            const double* A = view_ptr(s_st.a, p, z, lda);
            const double* B = view_ptr(s_st.b, p, z, ldb);
            const double* C = s_st.beta != 0.0 ? view_ptr(s_st.c, p, z, ldc) : nullptr;
            double* D = const_cast<double*>(view_ptr(s_st.d, p, z, ldd));
            if (s_st.tm == 64)
                ptile<64>(s_st.m, s_st.n, s_st.k, s_st.alpha, A, lda, B, ldb, s_st.beta, C, ldc, D, ldd, tile_m,
                          tile_n, smem);
            else if (s_st.tm == 32)
                ptile<32>(s_st.m, s_st.n, s_st.k, s_st.alpha, A, lda, B, ldb, s_st.beta, C, ldc, D, ldd, tile_m,
                          tile_n, smem);
            else
                ptile<16>(s_st.m, s_st.n, s_st.k, s_st.alpha, A, lda, B, ldb, s_st.beta, C, ldc, D, ldd, tile_m,
                          tile_n, smem);
        }
        // the task's writes are visible device-wide before it counts as finished
        __threadfence();
        __syncthreads();
        if (tid == 0) {
            atomicAdd(p.done + z, 1u);
            if (p.bucket_clocks != nullptr)
                atomicAdd(p.bucket_clocks + s_st.bucket, (unsigned long long)(clock64() - clk0));
        }
    }
}

}  // namespace

size_t persistent_smem_bytes(int64_t max_leaf) {
    const size_t leaf = cta_leaf_smem((int)std::max<int64_t>(1, std::min<int64_t>(max_leaf, kPersistMaxLeaf)));
    return std::max(leaf, ptile_smem<64>());
}

namespace {
PerDeviceOnce g_pattr;

int prepare_persistent() {
    return g_pattr.run([]() -> int {
        SPIN_CUDA_TRY(cudaFuncSetAttribute(persistent_batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)persistent_smem_bytes(kPersistMaxLeaf)));
        return SPIN_OK;
    });
}
}  // namespace

int persistent_grid(size_t smem, int64_t tasks, int* grid) {
    if (grid == nullptr || smem > persistent_smem_bytes(kPersistMaxLeaf)) return SPIN_ERR_INVALID_ARG;
    {
        const int rc = prepare_persistent();
        if (rc != SPIN_OK) return rc;
    }
    int dev = 0, sms = 0, per_sm = 0;
    SPIN_CUDA_TRY(cudaGetDevice(&dev));
    SPIN_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    SPIN_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_batch_kernel, NT, smem));
    if (per_sm < 1) return SPIN_ERR_INVALID_ARG;
    const int64_t g = std::min<int64_t>((int64_t)sms * per_sm, std::max<int64_t>(tasks, 1));
    *grid = (int)g;
    return SPIN_OK;
}

int launch_persistent_batch(const PersistentArgs& a, size_t smem, int grid, cudaStream_t s) {
    if (grid < 1 || a.nstages < 1 || smem > persistent_smem_bytes(kPersistMaxLeaf)) return SPIN_ERR_INVALID_ARG;
    {
        const int rc = prepare_persistent();
        if (rc != SPIN_OK) return rc;
    }
    persistent_batch_kernel<<<(unsigned)grid, NT, smem, s>>>(a);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace spin
