// Gauss-Jordan pieces shared by the leaf kernels (leaf_gj.cu) and the
// persistent batch kernel (persistent.cu): the pivot candidate and its
// warp-wide argmax, the elimination of one column, the shared end that
// unscrambles the columns and writes X, and the whole one-CTA leaf.
//
// The arithmetic is that of the oracle's leaf (Gauss-Jordan with partial
// pivoting, the direct leaf inversion that Algorithm 1 leaves open): at step
// k the row with the largest |a_ik| among positions >= k, lowest position on
// ties, is scaled by 1/pivot with the pivot slot receiving 1/pivot; f_i times
// it is subtracted from every other row, slot (i,k) receiving -f_i/pivot; the
// row interchanges are undone at the end as column interchanges in reverse
// order.
#pragma once
#include <limits.h>

#include "common.cuh"

namespace spin {
namespace {

constexpr int NT = 256;
constexpr unsigned FULL = 0xffffffffu;

// A pivot candidate.  The key is the bit pattern of |pivot| (NaN mapped to
// +inf, so that it is chosen and then rejected): for non-negative doubles
// the bit patterns order like the values, so every comparison is an
// integer one and the SM's FP64 pipe (~2 operations per clock on GB300)
// only does the elimination's FMAs.  No candidate: key 0, position INT_MAX.
struct Cand {
    uint64_t key;
    double val;  // signed pivot value
    double inv;  // 1 / val, computed once by the CTA that publishes the candidate
    int pos;     // logical position of the row
    int phys;    // physical row, -1: no candidate
};
constexpr uint64_t kInfBits = 0x7ff0000000000000ull;

// Warp-wide argmax by (key descending, position ascending); every lane gets
// the winner.  Three redux.sync steps replace a shuffle tree: the high word
// of the key, the low word among the lanes that hold the high maximum, the
// lowest position among the ties.
__device__ __forceinline__ Cand warp_argmax(uint64_t key, double val, double inv, int pos, int phys) {
    const unsigned hi = (unsigned)(key >> 32), lo = (unsigned)key;
    const unsigned mhi = __reduce_max_sync(FULL, hi);
    const unsigned mlo = __reduce_max_sync(FULL, hi == mhi ? lo : 0u);
    const bool tie = hi == mhi && lo == mlo;
    const unsigned mpos = __reduce_min_sync(FULL, tie ? (unsigned)pos : 0xffffffffu);
    const int src = __ffs(__ballot_sync(FULL, tie && (unsigned)pos == mpos)) - 1;
    Cand w;
    w.key = ((uint64_t)mhi << 32) | mlo;
    w.val = __shfl_sync(FULL, val, src);
    w.inv = __shfl_sync(FULL, inv, src);
    w.pos = __shfl_sync(FULL, pos, src);
    w.phys = __shfl_sync(FULL, phys, src);
    return w;
}

// 1 if f is +0 or -0.  Evaluated once per row and step, where the
// multiplier is produced, and kept beside it: tested per entry, the same
// test costs an FP64-pipe instruction per FMA (measured: the pipe ran twice
// the elimination's FMAs).
__device__ __forceinline__ int zero_flag(double f) { return ((uint64_t)__double_as_longlong(f) << 1) == 0; }

// Step k's update of one entry: pj is the pivot row's entry scaled by
// 1/pivot (1/pivot itself in the pivot column, jk), f the row's multiplier
// (fz: f is zero), b its current entry; a zero multiplier leaves the entry
// as it is.
__device__ __forceinline__ double elim_val(int fz, double f, double b, double pj, bool jk) {
    return fz ? (jk ? f : b) : fma(-f, pj, jk ? 0.0 : b);
}

// Column j of this thread's rows r, r + rg, ... (< nrows), in groups of U
// (U FMAs in flight per thread); rows skip1 and skip2 are computed but not
// stored.  Returns the first row not done.
template <int U>
__device__ __forceinline__ int elim_rows(double* M, int L, int j, const double* fk, const int* zk, double pj, bool jk,
                                         int r, int rg, int nrows, int skip1, int skip2) {
    while (r + (U - 1) * rg < nrows) {
        double f[U], b[U];
        int z[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            f[u] = fk[r + u * rg];
            z[u] = zk[r + u * rg];
            b[u] = M[(size_t)(r + u * rg) * L + j];
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const int rr = r + u * rg;
            const double nv = elim_val(z[u], f[u], b[u], pj, jk);
            if (rr != skip1 && rr != skip2) M[(size_t)rr * L + j] = nv;
        }
        r += U * rg;
    }
    return r;
}

template <int G = 8>
__device__ __forceinline__ void elim_column(double* M, int L, int j, const double* fk, const int* zk, double pj,
                                            bool jk, int r, int rg, int nrows, int skip1, int skip2) {
    if constexpr (G >= 8) r = elim_rows<8>(M, L, j, fk, zk, pj, jk, r, rg, nrows, skip1, skip2);
    r = elim_rows<4>(M, L, j, fk, zk, pj, jk, r, rg, nrows, skip1, skip2);
    r = elim_rows<2>(M, L, j, fk, zk, pj, jk, r, rg, nrows, skip1, skip2);
    elim_rows<1>(M, L, j, fk, zk, pj, jk, r, rg, nrows, skip1, skip2);
}

// Shared end: scale the last pivot row, undo the row interchanges as column
// interchanges, write X.  Called after a block barrier.
__device__ __forceinline__ void leaf_finish(double* M, int L, int R, int r0, int nrows, int rank, int prev_p,
                                            double prev_inv, const int* lpos, const int* piv, int* sigma,
                                            double* __restrict__ dst, int64_t ldd, int32_t* info, int leaf_index) {
    const int tid = threadIdx.x;
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

// Row-interchange bookkeeping, by the block's last thread (the first ones
// update column k+1 right after it).
__device__ __forceinline__ void apply_pivot(int k, const Cand& w, int* phys_at, int* lpos, int* piv) {
    if (threadIdx.x == NT - 1) {
        const int a = phys_at[k];
        phys_at[k] = w.phys;
        phys_at[w.pos] = a;
        lpos[w.phys] = k;
        lpos[a] = w.pos;
        piv[k] = w.pos;
    }
}

__device__ __forceinline__ bool bad_pivot(const Cand& w) {
    return w.key == 0 || w.key >= kInfBits || w.phys < 0;  // zero, infinite or NaN pivot, or none
}

// ---------------------------------------------------------------------------
// One CTA per leaf (the batched paths' leaves, L <= kCtaMaxL): the cluster
// forms' exchange machinery (slot barriers, async-proxy fences, the
// messenger's named barrier) costs every step several thousand cycles on a
// single CTA, against 2 L^2 / 4 cycles of FMAs per sub-partition.  Here a
// step is: winner (every warp combines the per-warp candidates of the last
// step's phase A) -> A: column k+1 of every row and this step's candidates
// -> barrier -> C: every other column of every row; meanwhile one lane
// computes the next pivot's reciprocal -> barrier.  The arithmetic, the
// pivot choice and the order of operations on every entry are those of the
// cluster forms, so the results are identical bit for bit.
constexpr int kCtaMaxL = 128;

__host__ __device__ inline size_t cta_leaf_smem(int L) {
    size_t off = (size_t)L * L * sizeof(double);              // M
    off += 2 * (size_t)L * sizeof(double);                    // fcol
    off += 2 * (size_t)L * sizeof(int);                       // zcol
    off = (off + 15) & ~(size_t)15;
    off += (size_t)(NT / 32) * sizeof(Cand);                  // parts
    off += 2 * sizeof(double);                                // sinv
    off += 4 * (size_t)L * sizeof(int);                       // phys_at, lpos, piv, sigma
    return (off + 15) & ~(size_t)15;
}

// Loads of the leaf block: through the read-only path, or (kCoherent)
// through L2 only, for a block that another SM wrote during the same launch
// (the persistent batch kernel).
template <bool kCoherent>
__device__ __forceinline__ double leaf_src_load(const double* p) {
    if constexpr (kCoherent)
        return __ldcg(p);
    else
        return *p;
}

// The one-CTA leaf: inverts src (L x L, leading dimension lds) into dst
// (leading dimension ldd), failures to info; smem_raw holds cta_leaf_smem(L)
// bytes (16-byte aligned).  Every thread of the 256-thread block calls it.
template <bool kCoherent>
__device__ __forceinline__ void leaf_gj_cta_body(const double* __restrict__ src, int64_t lds,
                                                 double* __restrict__ dst, int64_t ldd, int L, int32_t* info,
                                                 int leaf_index, unsigned char* smem_raw) {
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    double* M = reinterpret_cast<double*>(smem_raw);
    double* fcol = M + (size_t)L * L;                        // [2][L] multipliers
    int* zcol = reinterpret_cast<int*>(fcol + 2 * L);        // [2][L] their zero flags
    size_t off = ((size_t)L * L + 2 * L) * sizeof(double) + 2 * (size_t)L * sizeof(int);
    off = (off + 15) & ~(size_t)15;
    Cand* parts = reinterpret_cast<Cand*>(smem_raw + off);   // [NT / 32] phase A's candidates
    double* sinv = reinterpret_cast<double*>(parts + NT / 32);  // [2] next pivot's reciprocal
    int* phys_at = reinterpret_cast<int*>(sinv + 2);
    int* lpos = phys_at + L;
    int* piv = lpos + L;
    int* sigma = piv + L;

    const int row_groups = NT / L;  // thread (tr, j): column j, rows tr, tr + row_groups, ...
    const int j = tid % L, tr = tid / L;
    const bool active = tr < row_groups;
    const int nparts = (L + 31) / 32;

    for (int idx = tid; idx < L * L; idx += NT) {
        const int r = idx / L, c = idx % L;
        M[idx] = leaf_src_load<kCoherent>(src + (size_t)r * lds + c);
    }
    for (int r = tid; r < L; r += NT) {  // step 0's multipliers (column 0)
        fcol[r] = leaf_src_load<kCoherent>(src + (size_t)r * lds);
        zcol[r] = zero_flag(fcol[r]);
        phys_at[r] = r;
        lpos[r] = r;
    }
    __syncthreads();
    // step 0's winner: every warp scans column 0 (contiguous in fcol)
    Cand w;
    {
        uint64_t key = 0;
        double val = 0.0;
        int pos = INT_MAX, phys = -1;
        for (int r = lane; r < L; r += 32) {
            const double a = fcol[r];
            const uint64_t mag = (uint64_t)__double_as_longlong(a) & ~(1ull << 63);
            const uint64_t kk = mag > kInfBits ? kInfBits : mag;
            if (kk > key || (kk == key && r < pos)) { key = kk; val = a; pos = r; phys = r; }
        }
        w = warp_argmax(key, val, 0.0, pos, phys);
        w.inv = __drcp_rn(w.val);  // once per leaf, in every thread
    }
    int steps_done = 0;
    int prev_p = -1;
    double prev_inv = 0.0;
    for (int k = 0; k < L; k++) {
        if (bad_pivot(w)) {  // identical decision in every thread: the CTA leaves together
            if (tid == 0) record_failure(info, SPIN_ERR_SINGULAR, leaf_index, k);
            break;
        }
        apply_pivot(k, w, phys_at, lpos, piv);
        const int p = w.phys;  // the pivot row stays raw in step k
        const double inv = w.inv;
        const double* fk = fcol + (k & 1) * L;
        const int* zk = zcol + (k & 1) * L;
        double* fn = fcol + ((k + 1) & 1) * L;
        int* zn = zcol + ((k + 1) & 1) * L;
        const double pj = (j == k) ? inv : M[(size_t)p * L + j] * inv;
        // the previous pivot row is scaled by its 1/pivot (its multiplier is
        // already scaled), except column k+1, which A scales
        const int pr = prev_p;
        const double pinv = prev_inv;
        if (active && pr >= 0 && pr % row_groups == tr && j != k + 1) {
            double* rp = M + (size_t)pr * L + j;
            *rp = (j == k - 1) ? pinv : *rp * pinv;
        }
        prev_p = p;
        prev_inv = inv;
        steps_done = k + 1;
        if (k + 1 == L) {  // last step: no next column
            if (active) elim_column<4>(M, L, j, fk, zk, pj, j == k, tr, row_groups, L, p, p);
            break;
        }
        // A: column k+1, one row per thread, and this CTA's candidates for it
        // (eligible: not taken before step k, not p; the row that was at
        // position k moves to w.pos -- both values of its position entry,
        // which thread NT - 1 is rewriting, give the same answer)
        if (tid < nparts * 32) {
            uint64_t key = 0;
            double val = 0.0;
            int pos = INT_MAX, phys = -1;
            if (tid < L) {
                const double pjn = M[(size_t)p * L + k + 1] * inv;
                if (tid == p) {
                    fn[tid] = pjn;
                    zn[tid] = zero_flag(pjn);
                } else {
                    double b = M[(size_t)tid * L + k + 1];
                    if (tid == pr) b *= pinv;
                    const double nv = elim_val(zk[tid], fk[tid], b, pjn, false);
                    M[(size_t)tid * L + k + 1] = nv;
                    fn[tid] = nv;
                    zn[tid] = zero_flag(nv);
                    const int lp = lpos[tid];
                    if (lp >= k) {
                        const uint64_t mag = (uint64_t)__double_as_longlong(nv) & ~(1ull << 63);
                        key = mag > kInfBits ? kInfBits : mag;
                        val = nv;
                        pos = lp == k ? w.pos : lp;
                        phys = tid;
                    }
                }
            }
            const Cand wc = warp_argmax(key, val, 0.0, pos, phys);
            if (lane == 0) parts[warp] = wc;
        }
        __syncthreads();  // candidates, column k+1 and the position table are up to date
        Cand c;
        {
            Cand q{0, 0.0, 0.0, INT_MAX, -1};
            if (lane < nparts) q = parts[lane];
            c = warp_argmax(q.key, q.val, 0.0, q.pos, q.phys);
        }
        // the next pivot's reciprocal, by one lane while the others eliminate
        if (tid == NT - 32) sinv[(k + 1) & 1] = __drcp_rn(c.val);  // inf or NaN for no candidate: never used
        // C: every row but the pivot row, every column but k+1
        if (active && j != k + 1) elim_column<4>(M, L, j, fk, zk, pj, j == k, tr, row_groups, L, p, p);
        __syncthreads();  // M, the next reciprocal and the multipliers are up to date
        w = c;
        w.inv = sinv[(k + 1) & 1];
    }
    __syncthreads();
    if (steps_done < L) return;  // failure already recorded; X is undefined
    leaf_finish(M, L, L, 0, L, 0, prev_p, prev_inv, lpos, piv, sigma, dst, ldd, info, leaf_index);
}

}  // namespace
}  // namespace spin
