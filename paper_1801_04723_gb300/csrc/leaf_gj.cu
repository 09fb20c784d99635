// Leaf inversion: Gauss-Jordan with partial pivoting on one leaf block.
//
// Algorithm 1 inverts a block directly once its order reaches the threshold
// ("invert A in any approach"; Algorithm 2's locInverse).  This kernel
// computes the same in-place Gauss-Jordan as the CPU oracle's leaf: at step
// k choose the row (among positions >= k) with the largest |a_ik|, lowest
// position on ties; scale it by 1/pivot with the pivot slot receiving
// 1/pivot; subtract f_i times it from every other row, slot (i,k) receiving
// -f_i/pivot; at the end undo the row interchanges as column interchanges
// in reverse order.
//
// GB300 mapping.  FP64 runs at ~2 FMA/clock/SM, so one L x L leaf on one SM
// takes ~L^3 cycles; the leaf is spread over a thread-block cluster of C
// CTAs (C <= 16) whose rows stay put: every CTA owns R = ceil(L/C) rows in
// shared memory when they fit (global memory, L2-resident, otherwise).  Row interchanges
// are bookkeeping only (position <-> physical row tables replicated in every
// CTA), so no data moves between CTAs except the pivot row, read through
// distributed shared memory.  Per step: cluster barrier -> every CTA reduces
// the C published candidates identically -> all CTAs eliminate their rows
// with the pivot row read raw from its owner through distributed shared
// memory and scaled on the fly -> each CTA publishes its candidate for the
// next column.  One cluster barrier per step (a hardware barrier: no
// spin-wait anywhere); the owner scales the pivot row in place after the
// next barrier.
#include <cooperative_groups.h>
#include <limits.h>

#include "common.cuh"

namespace cg = cooperative_groups;

namespace spin {
namespace {

constexpr int NT = 256;

struct Cand {
    double key;   // |pivot| (NaN mapped to +inf so that it is chosen and rejected)
    double val;   // signed pivot value
    int pos;      // logical position of the row
    int phys;     // physical row
};

struct LeafSmemLayout {
    size_t m_off, fcol_off, cand_off, phys_off, lpos_off, piv_off, sig_off, total;
};

__host__ __device__ inline LeafSmemLayout leaf_layout(int L, int R, bool rows_in_smem) {
    LeafSmemLayout s;
    size_t off = 0;
    s.m_off = off;
    if (rows_in_smem) off += (size_t)R * L * sizeof(double);
    s.fcol_off = off; off += (size_t)R * sizeof(double);
    s.cand_off = off; off += 2 * sizeof(Cand);
    s.phys_off = off; off += (size_t)L * sizeof(int);
    s.lpos_off = off; off += (size_t)L * sizeof(int);
    s.piv_off = off; off += (size_t)L * sizeof(int);
    s.sig_off = off; off += (size_t)L * sizeof(int);
    s.total = (off + 15) & ~(size_t)15;
    return s;
}

__device__ __forceinline__ bool better(double k1, int p1, double k2, int p2) {
    return k1 > k2 || (k1 == k2 && p1 < p2);
}

// Block-wide search of this CTA's candidate for column k among its rows at
// positions >= k.  Result in *out (written by thread 0).
__device__ void local_candidate(const double* M, int L, int nrows, int r0, const int* lpos, int k, Cand* out,
                                Cand* warp_scratch) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double key = -1.0, val = 0.0;
    int pos = INT_MAX, phys = -1;
    if (k < L) {
        for (int r = tid; r < nrows; r += NT) {
            const int pr = r0 + r;
            const int lp = lpos[pr];
            if (lp < k) continue;
            const double a = M[(size_t)r * L + k];
            const double kk = isnan(a) ? INFINITY : fabs(a);
            if (better(kk, lp, key, pos)) { key = kk; val = a; pos = lp; phys = pr; }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const double ok = __shfl_down_sync(0xffffffffu, key, off);
        const double ov = __shfl_down_sync(0xffffffffu, val, off);
        const int op = __shfl_down_sync(0xffffffffu, pos, off);
        const int oph = __shfl_down_sync(0xffffffffu, phys, off);
        if (better(ok, op, key, pos)) { key = ok; val = ov; pos = op; phys = oph; }
    }
    if (lane == 0) warp_scratch[warp] = Cand{key, val, pos, phys};
    __syncthreads();
    if (warp == 0) {
        Cand c = (lane < NT / 32) ? warp_scratch[lane] : Cand{-1.0, 0.0, INT_MAX, -1};
        key = c.key; val = c.val; pos = c.pos; phys = c.phys;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const double ok = __shfl_down_sync(0xffffffffu, key, off);
            const double ov = __shfl_down_sync(0xffffffffu, val, off);
            const int op = __shfl_down_sync(0xffffffffu, pos, off);
            const int oph = __shfl_down_sync(0xffffffffu, phys, off);
            if (better(ok, op, key, pos)) { key = ok; val = ov; pos = op; phys = oph; }
        }
        if (lane == 0) *out = Cand{key, val, pos, phys};
    }
}

template <bool ROWS_IN_SMEM>
__device__ __forceinline__ void leaf_gj_body(const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                                             int64_t ldd, double* __restrict__ gwork, int L, int R, int32_t* info,
                                             int leaf_index) {
    cg::cluster_group cluster = cg::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LeafSmemLayout lay = leaf_layout(L, R, ROWS_IN_SMEM);
    double* M = ROWS_IN_SMEM ? reinterpret_cast<double*>(smem_raw + lay.m_off) : gwork + (size_t)rank * R * L;
    double* fcol = reinterpret_cast<double*>(smem_raw + lay.fcol_off);
    Cand* cand = reinterpret_cast<Cand*>(smem_raw + lay.cand_off);
    int* phys_at = reinterpret_cast<int*>(smem_raw + lay.phys_off);
    int* lpos = reinterpret_cast<int*>(smem_raw + lay.lpos_off);
    int* piv = reinterpret_cast<int*>(smem_raw + lay.piv_off);
    int* sigma = reinterpret_cast<int*>(smem_raw + lay.sig_off);
    __shared__ Cand warp_scratch[NT / 32];
    __shared__ Cand chosen;
    __shared__ int s_fail;

    const int r0 = rank * R;
    const int nrows = max(0, min(R, L - r0));
    const int col_threads = L < NT ? L : NT;  // elimination: threads per row
    const int row_groups = NT / col_threads;  // ... and rows handled at once
    const int tc = tid % col_threads, tr = tid / col_threads;

    for (size_t idx = tid; idx < (size_t)nrows * L; idx += NT) {
        const int r = (int)(idx / L), j = (int)(idx % L);
        M[idx] = src[(size_t)(r0 + r) * lds + j];
    }
    for (int q = tid; q < L; q += NT) { phys_at[q] = q; lpos[q] = q; }
    if (tid == 0) s_fail = 0;
    __syncthreads();
    local_candidate(M, L, nrows, r0, lpos, 0, &cand[0], warp_scratch);

    // One cluster barrier per step.  The pivot row of step k is read raw by
    // every CTA (and scaled on the fly); its owner scales it in place at the
    // start of step k+1, after the barrier, when nobody reads it any more and
    // before it is eliminated like every other row.  The candidates
    // alternate between two slots (step k reads slot k & 1): a CTA writes
    // step k+1's candidate before the next barrier, while others may still
    // be reading step k's; the slot it overwrites was last read in step k-1,
    // which every CTA finished before the barrier that opened step k.
    int steps_done = 0;
    int prev_p = -1;
    double prev_inv = 0.0;
    for (int k = 0; k < L; k++) {
        cluster.sync();  // candidates for column k published; step k-1 finished everywhere
        if (prev_p >= 0 && prev_p / R == rank) {
            double* rp = M + (size_t)(prev_p - r0) * L;
            for (int j = tid; j < L; j += NT) rp[j] = (j == k - 1) ? prev_inv : rp[j] * prev_inv;
        }
        if (tid < 32) {
            Cand c{-1.0, 0.0, INT_MAX, -1};
            if (tid < C) c = *cluster.map_shared_rank(&cand[k & 1], tid);
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const double ok = __shfl_down_sync(0xffffffffu, c.key, off);
                const double ov = __shfl_down_sync(0xffffffffu, c.val, off);
                const int op = __shfl_down_sync(0xffffffffu, c.pos, off);
                const int oph = __shfl_down_sync(0xffffffffu, c.phys, off);
                if (better(ok, op, c.key, c.pos)) { c.key = ok; c.val = ov; c.pos = op; c.phys = oph; }
            }
            if (tid == 0) {
                chosen = c;
                const bool bad = !(c.key > 0.0) || isinf(c.key) || c.phys < 0;
                s_fail = bad ? 1 : 0;
                if (!bad) {
                    const int a = phys_at[k];
                    phys_at[k] = c.phys;
                    phys_at[c.pos] = a;
                    lpos[c.phys] = k;
                    lpos[a] = c.pos;
                    piv[k] = c.pos;
                }
            }
        }
        __syncthreads();  // pivot decided; the deferred scaling of the previous pivot row is done
        if (s_fail) {  // identical decision in every CTA: all leave the loop together
            if (rank == 0 && tid == 0) record_failure(info, SPIN_ERR_SINGULAR, leaf_index, k);
            break;
        }
        const int p = chosen.phys;
        const double inv = 1.0 / chosen.val;
        const int owner = p / R;
        for (int r = tid; r < nrows; r += NT)
            if (r0 + r != p) fcol[r] = M[(size_t)r * L + k];
        __syncthreads();  // every multiplier is stashed before column k is overwritten
        // the owner's raw pivot row: its shared memory (through the cluster
        // window), or the L2-resident work rows when they live in global memory
        const double* rprow = ROWS_IN_SMEM ? cluster.map_shared_rank(M, owner) + (size_t)(p - owner * R) * L
                                           : gwork + (size_t)p * L;
        // threads tile the rows x columns block: tc columns apart along a
        // row (coalesced), tr row groups, so that narrow leaves (L < NT)
        // keep every thread busy; each thread reads a pivot-row entry once
        // per column it owns
        if (tr < row_groups) {
            for (int j = tc; j < L; j += col_threads) {
                const double pj = (j == k) ? inv : rprow[j] * inv;
                for (int r = tr; r < nrows; r += row_groups) {
                    if (r0 + r == p) continue;
                    const double f = fcol[r];
                    if (f == 0.0) continue;
                    double* mr = M + (size_t)r * L;
                    const double base = (j == k) ? 0.0 : mr[j];
                    mr[j] = fma(-f, pj, base);
                }
            }
        }
        __syncthreads();
        // next step's candidate goes to the other slot: a slower CTA may
        // still be reading this step's slot through the cluster window
        local_candidate(M, L, nrows, r0, lpos, k + 1, &cand[(k + 1) & 1], warp_scratch);
        prev_p = p;
        prev_inv = inv;
        steps_done = k + 1;
    }
    cluster.sync();  // no CTA still reads a peer's rows
    if (steps_done < L) return;  // failure already recorded; X is undefined
    if (prev_p >= 0 && prev_p / R == rank) {  // the last pivot row is still unscaled
        double* rp = M + (size_t)(prev_p - r0) * L;
        for (int j = tid; j < L; j += NT) rp[j] = (j == L - 1) ? prev_inv : rp[j] * prev_inv;
    }
    __syncthreads();

    if (tid == 0) {
        for (int q = 0; q < L; q++) sigma[q] = q;
        for (int k = L - 1; k >= 0; k--) {
            const int q = piv[k];
            const int t = sigma[k]; sigma[k] = sigma[q]; sigma[q] = t;
        }
    }
    __syncthreads();
    int nonfinite = 0;
    for (int r = 0; r < nrows; r++) {
        const int i = lpos[r0 + r];
        const double* mr = M + (size_t)r * L;
        double* out = dst + (size_t)i * ldd;
        for (int j = tid; j < L; j += NT) {
            const double v = mr[sigma[j]];
            nonfinite |= !isfinite(v);
            out[j] = v;
        }
    }
    if (__syncthreads_or(nonfinite) && tid == 0) record_failure(info, SPIN_ERR_SINGULAR, leaf_index, L);
}

template <bool ROWS_IN_SMEM>
__global__ void __launch_bounds__(NT, 1)
leaf_gj_kernel(const double* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd,
               double* __restrict__ gwork, int L, int R, int32_t* info, int leaf_index) {
    leaf_gj_body<ROWS_IN_SMEM>(src, lds, dst, ldd, gwork, L, R, info, leaf_index);
}

// Batched form: cluster blockIdx.y inverts problem z = blockIdx.y.
template <bool ROWS_IN_SMEM>
__global__ void __launch_bounds__(NT, 1)
leaf_gj_batched_kernel(BatchView src, BatchView dst, double* __restrict__ gwork, int64_t gwork_stride, int L, int R,
                       int32_t* info, int leaf_index) {
    const int z = blockIdx.y;
    const int64_t lds = src.ld_of(z), ldd = dst.ld_of(z);
    leaf_gj_body<ROWS_IN_SMEM>(src.ptr(z, lds), lds, const_cast<double*>(dst.ptr(z, ldd)), ldd,
                               ROWS_IN_SMEM ? nullptr : gwork + (int64_t)z * gwork_stride, L, R,
                               info + (int64_t)z * INFO_WORDS, leaf_index);
}

struct LeafConfig {
    int C, R;
    bool smem_rows;
    size_t smem;
};

constexpr size_t kSmemBudget = 200 * 1024;

// Largest cluster the GPU can co-schedule for this kernel (16 on GB300 when
// the non-portable size is allowed, else 8); queried once.
int max_cluster_size() {
    static int cached = 0;
    if (cached) return cached;
    cached = 8;
    auto kern = leaf_gj_kernel<true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return cached;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = leaf_layout(512, 32, true).total;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 16;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int clusters = 0;
    if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) == cudaSuccess && clusters > 0) cached = 16;
    cudaGetLastError();
    return cached;
}

// Cluster shape.  A pivot step costs a few microseconds of latency
// (barrier, DSMEM reads) plus R*L FMAs on each CTA at ~2 FP64 FMA/clock:
// measured per-step times at L = 128 are 17.4 / 10.6 / 7.2 / 5.6 / 5.0 us for
// 1 / 2 / 4 / 8 / 16 CTAs.  A single inversion waits on its leaves, so it
// takes the widest cluster (latency); a batch runs many leaves side by side,
// so it takes the narrowest that fits shared memory (SM time).
LeafConfig leaf_config(int64_t L, bool have_scratch, bool batched = false) {
    LeafConfig c;
    const int cmax = max_cluster_size();
    c.C = 1;
    if (batched) {
        while (c.C < cmax && leaf_layout((int)L, (int)((L + c.C - 1) / c.C), true).total > kSmemBudget) c.C <<= 1;
    } else {
        while (c.C < cmax && c.C < L) c.C <<= 1;
    }
    c.R = (int)((L + c.C - 1) / c.C);
    c.smem_rows = leaf_layout((int)L, c.R, true).total <= kSmemBudget;
    if (!c.smem_rows && !have_scratch) c.smem_rows = true;  // rejected by the caller's size check
    c.smem = leaf_layout((int)L, c.R, c.smem_rows).total;
    return c;
}

template <bool S>
int launch_leaf_impl(const double* A, int64_t lda, double* X, int64_t ldx, const LeafConfig& c, int64_t L,
                     double* scratch, int32_t* info, int leaf_index, cudaStream_t s) {
    static bool attr_done[2] = {false, false};
    auto kern = leaf_gj_kernel<S>;
    if (!attr_done[S ? 1 : 0]) {
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget));
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr_done[S ? 1 : 0] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c.C, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SPIN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, A, lda, X, ldx, scratch, (int)L, c.R, info, leaf_index));
    return SPIN_OK;
}

template <bool S>
int launch_leaf_batched_impl(const BatchView& src, const BatchView& dst, const LeafConfig& c, int64_t L,
                             double* scratch, int64_t stride, int32_t* info, int leaf_index, int count,
                             cudaStream_t s) {
    static bool attr_done[2] = {false, false};
    auto kern = leaf_gj_batched_kernel<S>;
    if (!attr_done[S ? 1 : 0]) {
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget));
        SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
        attr_done[S ? 1 : 0] = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c.C, (unsigned)count, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SPIN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, src, dst, scratch, stride, (int)L, c.R, info, leaf_index));
    return SPIN_OK;
}

}  // namespace

int launch_leaf_gj_batched(const BatchView& src, const BatchView& dst, int64_t L, double* scratch_base,
                           int64_t scratch_stride, int32_t* info, int leaf_index, int count, cudaStream_t s) {
    if (L <= 0 || count <= 0) return SPIN_OK;
    if (L > kMaxLeaf || count > 65535) return SPIN_ERR_INVALID_ARG;
    const LeafConfig c = leaf_config(L, scratch_base != nullptr, true);
    if (c.smem > kSmemBudget) return SPIN_ERR_INVALID_ARG;
    if (c.smem_rows)
        return launch_leaf_batched_impl<true>(src, dst, c, L, nullptr, 0, info, leaf_index, count, s);
    return launch_leaf_batched_impl<false>(src, dst, c, L, scratch_base, scratch_stride, info, leaf_index, count, s);
}

// Leaves above 256 may not fit shared memory on every cluster shape, so
// they always get an L x L scratch slab (used only when the rows spill).
size_t leaf_scratch_elems(int64_t L) { return L > 256 ? (size_t)L * (size_t)L : 0; }

int launch_leaf_gj(const double* A, int64_t lda, double* X, int64_t ldx, int64_t L, double* scratch,
                   int32_t* info, int leaf_index, cudaStream_t s) {
    if (L <= 0) return SPIN_OK;
    if (L > kMaxLeaf) return SPIN_ERR_INVALID_ARG;
    const LeafConfig c = leaf_config(L, scratch != nullptr);
    if (c.smem > kSmemBudget) return SPIN_ERR_INVALID_ARG;
    if (c.smem_rows) return launch_leaf_impl<true>(A, lda, X, ldx, c, L, nullptr, info, leaf_index, s);
    return launch_leaf_impl<false>(A, lda, X, ldx, c, L, scratch, info, leaf_index, s);
}

}  // namespace spin
