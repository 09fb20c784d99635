// Leaf inversion: Gauss-Jordan with partial pivoting on one leaf block.
//
// Algorithm 1 inverts a block directly, by a method it leaves open, once its
// order reaches the threshold (Algorithm 2's locInverse).  This kernel
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
// shared memory when they fit (global memory, L2-resident, otherwise).  Row
// interchanges are bookkeeping only (position <-> physical row tables
// replicated in every CTA).  A pivot step is latency-bound at these sizes:
// each SM sub-partition's FP64 unit takes one warp instruction per 64
// cycles, a dependent FP64 operation waits behind every one queued before
// it (~250 cycles in a step), so a step keeps remote reads, fences and FP64
// work off its critical path:
//  - the pivot search compares the bit patterns of |a_ik| as integers
//    (redux.sync argmax), and each candidate's reciprocal is computed once,
//    by the CTA that publishes it;
//  - every CTA publishes its candidate for the next column into every other
//    CTA's shared memory, double-buffered by step parity (a CTA writes step
//    k+1's slot while a slower one may still read step k's; the slot it
//    overwrites was last read in step k-1);
//  - the multipliers of step k+1 (column k+1 after step k) go to a second
//    buffer, written by the threads that compute them;
//  - the pivot row of step k is left raw; its scaling by 1/pivot is folded
//    into step k+1's update of that row.
// Two forms (leaf_gj_push_body, leaf_gj_pull_body below): for L <= 256 the
// candidate rows travel with the candidates (st.async and bulk copies that
// complete on per-slot mbarriers, with the bulk of each step overlapping the
// exchange); above, the pivot row is read from its owner and a step ends at
// a cluster barrier.
#include <cooperative_groups.h>
#include <limits.h>

#include <algorithm>
#include <vector>

#include "common.cuh"
#include "leaf_core.cuh"
#include "tc_ptx.cuh"

namespace cg = cooperative_groups;

namespace spin {
namespace {

constexpr int kPushMaxL = NT;  // rows are pushed when one thread per column covers the row
constexpr int kMessengers = 32;  // with pushed rows: one more warp that publishes the candidates

struct LeafSmemLayout {
    size_t bar_off, m_off, prow_off, fcol_off, zcol_off, info_off, part_off, phys_off, lpos_off, piv_off, sig_off, total;
};

// Candidate-row slots hold L doubles padded to an even count, so that every
// slot row starts on a 16-byte boundary (16-byte remote stores).
__host__ __device__ inline int slot_stride(int L) { return (L + 1) & ~1; }

__host__ __device__ inline LeafSmemLayout leaf_layout(int L, int R, int C, bool rows_in_smem, bool push) {
    LeafSmemLayout s;
    auto a16 = [](size_t v) { return (v + 15) & ~(size_t)15; };
    size_t off = 0;
    s.bar_off = off; off += 2 * sizeof(uint64_t);
    s.m_off = off;
    if (rows_in_smem) off += (size_t)R * L * sizeof(double);
    s.prow_off = off = a16(off);
    if (push) off += 2 * (size_t)C * slot_stride(L) * sizeof(double);
    s.fcol_off = off = a16(off); off += 2 * (size_t)R * sizeof(double);
    s.zcol_off = off; off += 2 * (size_t)R * sizeof(int);  // zero flags of the multipliers
    s.info_off = off = a16(off); off += 2 * (size_t)C * sizeof(Cand);
    s.part_off = off; if (push) off += (size_t)(NT / 32) * sizeof(Cand);  // per-warp candidates of phase A
    s.phys_off = off; off += (size_t)L * sizeof(int);
    s.lpos_off = off; off += (size_t)L * sizeof(int);
    s.piv_off = off; off += (size_t)L * sizeof(int);
    s.sig_off = off; off += (size_t)L * sizeof(int);
    s.total = (off + 15) & ~(size_t)15;
    return s;
}


// This CTA's candidate for column k among its rows at positions >= k,
// computed by the calling warp (every warp computes the same).
__device__ __forceinline__ Cand warp_candidate(const double* M, int L, int nrows, int r0, const int* lpos, int k) {
    const int lane = threadIdx.x & 31;
    uint64_t key = 0;
    double val = 0.0;
    int pos = INT_MAX, phys = -1;
    for (int r = lane; r < nrows; r += 32) {
        const int lp = lpos[r0 + r];
        if (lp < k) continue;
        const double a = M[(size_t)r * L + k];
        const uint64_t mag = (uint64_t)__double_as_longlong(a) & ~(1ull << 63);
        const uint64_t kk = mag > kInfBits ? kInfBits : mag;
        if (kk > key || (kk == key && lp < pos)) { key = kk; val = a; pos = lp; phys = r0 + r; }
    }
    return warp_argmax(key, val, 0.0, pos, phys);
}

// Bounded wait for a slot barrier (a step takes microseconds; the limit
// only turns a broken exchange into an error instead of a hang).
constexpr uint64_t kLeafWaitLimitNs = 4000000000ull;

// Exchange settings of the pushed-row form: the wait limit, and (tests
// only) a CTA that sends nothing, so that the others' waits run out.
struct LeafWait {
    uint64_t limit_ns = kLeafWaitLimitNs;
    int mute_rank = -1;
};

__device__ __forceinline__ bool slot_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (tc::mbar_try_wait_cluster(bar, parity)) return true;
    const uint64_t t0 = tc::globaltimer_ns();
    for (uint32_t spins = 1;; spins++) {
        if (tc::mbar_try_wait_cluster(bar, parity)) return true;
        if ((spins & 63u) == 0 && tc::globaltimer_ns() - t0 > limit_ns) return false;
    }
}



// Winner of step k among the C published candidates (every warp computes it).
__device__ __forceinline__ Cand cluster_winner(const Cand* slot, int C) {
    Cand w{0, 0.0, 0.0, INT_MAX, -1};
    if ((int)(threadIdx.x & 31) < C) w = slot[threadIdx.x & 31];
    return warp_argmax(w.key, w.val, w.inv, w.pos, w.phys);
}


// ---------------------------------------------------------------------------
// L > 256: the pivot row is read from its owner.  Per step: cluster barrier
// -> winner -> eliminate every row of this CTA (rows in shared memory or in
// L2-resident global memory) -> block barrier -> candidate for column k+1,
// published with plain cluster stores -> arrive.
template <bool ROWS_IN_SMEM>
__device__ __forceinline__ void leaf_gj_pull_body(const double* __restrict__ src, int64_t lds,
                                                  double* __restrict__ dst, int64_t ldd, double* __restrict__ gwork,
                                                  int L, int R, int32_t* info, int leaf_index) {
    const int C = (int)tc::cluster_nctarank();
    const int rank = (int)tc::cluster_ctarank();
    const int tid = threadIdx.x;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LeafSmemLayout lay = leaf_layout(L, R, C, ROWS_IN_SMEM, false);
    double* M = ROWS_IN_SMEM ? reinterpret_cast<double*>(smem_raw + lay.m_off) : gwork + (size_t)rank * R * L;
    double* fcol = reinterpret_cast<double*>(smem_raw + lay.fcol_off);  // [2][R] multipliers
    int* zcol = reinterpret_cast<int*>(smem_raw + lay.zcol_off);        // [2][R] their zero flags
    Cand* infos = reinterpret_cast<Cand*>(smem_raw + lay.info_off);     // [2][C] candidates
    int* phys_at = reinterpret_cast<int*>(smem_raw + lay.phys_off);
    int* lpos = reinterpret_cast<int*>(smem_raw + lay.lpos_off);
    int* piv = reinterpret_cast<int*>(smem_raw + lay.piv_off);
    int* sigma = reinterpret_cast<int*>(smem_raw + lay.sig_off);

    const int r0 = rank * R;
    const int nrows = max(0, min(R, L - r0));
    // elimination: tc columns apart along a row (coalesced), tr row groups
    const int col_threads = L < NT ? L : NT;
    const int row_groups = NT / col_threads;
    const int tc = tid % col_threads, tr = tid / col_threads;

    auto publish = [&](const Cand& c, int slot) {
        if (tid < C) {
            const uint32_t a = tc::mapa_u32(tc::smem_u32(&infos[slot * C + rank]), (uint32_t)tid);
            tc::st_cluster_u64(a, c.key);
            tc::st_cluster_f64(a + 8, c.val);
            tc::st_cluster_f64(a + 16, __drcp_rn(c.val));  // inf or NaN for no candidate: never used
            tc::st_cluster_u64(a + 24, ((uint64_t)(uint32_t)c.phys << 32) | (uint32_t)c.pos);
        }
    };

    for (size_t idx = tid; idx < (size_t)nrows * L; idx += NT) {
        const int r = (int)(idx / L), j = (int)(idx % L);
        M[idx] = src[(size_t)(r0 + r) * lds + j];
    }
    for (int r = tid; r < nrows; r += NT) {  // step 0's multipliers
        fcol[r] = src[(size_t)(r0 + r) * lds];
        zcol[r] = zero_flag(fcol[r]);
    }
    for (int q = tid; q < L; q += NT) { phys_at[q] = q; lpos[q] = q; }
    __syncthreads();
    tc::cluster_sync_all();  // every CTA of the cluster runs before the first remote write
    publish(warp_candidate(M, L, nrows, r0, lpos, 0), 0);
    tc::cluster_arrive_release();

    cg::cluster_group cluster = cg::this_cluster();
    int steps_done = 0;
    int prev_p = -1;
    double prev_inv = 0.0;
    for (int k = 0; k < L; k++) {
        tc::cluster_wait_acquire();  // every CTA's candidate for column k is in slot k & 1
        const Cand w = cluster_winner(infos + (k & 1) * C, C);
        if (bad_pivot(w)) {  // identical decision in every thread of every CTA: all leave together
            if (rank == 0 && tid == 0) record_failure(info, SPIN_ERR_SINGULAR, leaf_index, k);
            break;
        }
        apply_pivot(k, w, phys_at, lpos, piv);
        const int p = w.phys;
        const double inv = w.inv;
        const int owner = p / R;
        const double* prow = owner == rank ? M + (size_t)(p - r0) * L
                             : ROWS_IN_SMEM ? cluster.map_shared_rank(M, owner) + (size_t)(p - owner * R) * L
                                            : gwork + (size_t)p * L;
        if (tr < row_groups) {
            const double* fk = fcol + (k & 1) * R;
            const int* zk = zcol + (k & 1) * R;
            double* fn = fcol + ((k + 1) & 1) * R;
            int* zn = zcol + ((k + 1) & 1) * R;
            // the previous pivot row is scaled by its 1/pivot first, by the
            // threads that eliminate it (its multiplier is already scaled)
            const int pr = prev_p - r0;
            if (prev_p >= 0 && pr >= 0 && pr < nrows && pr % row_groups == tr) {
                double* rp = M + (size_t)pr * L;
                for (int j = tc; j < L; j += col_threads) rp[j] = (j == k - 1) ? prev_inv : rp[j] * prev_inv;
            }
            const int pl = p - r0;  // the pivot row stays raw
            for (int j = tc; j < L; j += col_threads) {
                const double pj = (j == k) ? inv : prow[j] * inv;
                const bool jk = j == k, jnext = j == k + 1;
                // column k+1 also gives step k+1's multipliers (the pivot
                // row's: its scaled entry)
                auto store = [&](int rr, double nv) {
                    if (rr == pl) {
                        if (jnext) {
                            fn[rr] = pj;
                            zn[rr] = zero_flag(pj);
                        }
                        return;
                    }
                    M[(size_t)rr * L + j] = nv;
                    if (jnext) {
                        fn[rr] = nv;
                        zn[rr] = zero_flag(nv);
                    }
                };
                // groups of four rows, the next group's loads issued before
                // this group's stores
                int r = tr;
                const int g4 = 4 * row_groups;
                if (r + g4 - row_groups < nrows) {
                    double f[4], b[4];
                    int z[4];
#pragma unroll
                    for (int u = 0; u < 4; u++) {
                        f[u] = fk[r + u * row_groups];
                        z[u] = zk[r + u * row_groups];
                        b[u] = M[(size_t)(r + u * row_groups) * L + j];
                    }
                    while (true) {
                        double nv[4];
#pragma unroll
                        for (int u = 0; u < 4; u++) nv[u] = elim_val(z[u], f[u], b[u], pj, jk);
                        const int rn = r + g4;
                        const bool more = rn + g4 - row_groups < nrows;
                        if (more) {
#pragma unroll
                            for (int u = 0; u < 4; u++) {
                                f[u] = fk[rn + u * row_groups];
                                z[u] = zk[rn + u * row_groups];
                                b[u] = M[(size_t)(rn + u * row_groups) * L + j];
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 4; u++) store(r + u * row_groups, nv[u]);
                        r = rn;
                        if (!more) break;
                    }
                }
                for (; r < nrows; r += row_groups) store(r, elim_val(zk[r], fk[r], M[(size_t)r * L + j], pj, jk));
            }
        }
        prev_p = p;
        prev_inv = inv;
        steps_done = k + 1;
        if (k + 1 == L) break;
        __syncthreads();  // column k+1 and the position table are up to date
        publish(warp_candidate(M, L, nrows, r0, lpos, k + 1), (k + 1) & 1);
        tc::cluster_arrive_release();
    }
    tc::cluster_sync_all();  // rows read in place by peers outlive their last step
    if (steps_done < L) return;  // failure already recorded; X is undefined
    leaf_finish(M, L, R, r0, nrows, rank, prev_p, prev_inv, lpos, piv, sigma, dst, ldd, info, leaf_index);
}

// ---------------------------------------------------------------------------
// L <= 256: every CTA sends its candidate for the next column, and that
// row, into every other CTA's shared memory, completing on the receiver's
// slot barrier (mbarrier transaction bytes: no fence, no cluster barrier),
// and the bulk of each step's elimination runs while the data is in flight.
// Step k, after slot k & 1's barrier:
//   winner -> A: column k+1 of every row of this CTA (the multipliers of
//   step k+1) -> block barrier -> candidate for column k+1 -> B: that row's
//   step-k update, into M and this CTA's own slot -> C: every other row,
//   every column but k+1.
// 256 compute threads own one column each (L <= 256); A gives rows to
// threads, one each.  A ninth warp, the messenger, computes the candidate's
// reciprocal pivot (a ~10-operation FP64 sequence) and sends the candidate
// (st.async), then, once the compute threads have written the row in B
// (named barrier: they arrive, it waits), one bulk copy of the row per peer
// (copy engine), so that neither the reciprocal nor the sending holds up C.
// A CTA sends step k+1's candidate only after it has received step k's from
// every CTA, so no CTA runs more than one step ahead: two slots suffice (the
// slot a sender overwrites was last read before the receiver sent its own
// step-k candidate), and a copy's source row, rewritten two steps later, is
// no longer being read.  A CTA without a candidate sends its slot's stale
// row, so that every step delivers the same byte count.
__device__ __forceinline__ void leaf_gj_push_body(const double* __restrict__ src, int64_t lds,
                                                  double* __restrict__ dst, int64_t ldd, int L, int R, int32_t* info,
                                                  int leaf_index, LeafWait lw) {
    const int C = (int)tc::cluster_nctarank();
    const int rank = (int)tc::cluster_ctarank();
    const int tid = threadIdx.x;
    const int mt = tid - NT;  // messenger lane, if >= 0

    extern __shared__ __align__(16) unsigned char smem_raw[];
    const LeafSmemLayout lay = leaf_layout(L, R, C, true, true);
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem_raw + lay.bar_off);    // [2] slot barriers
    double* M = reinterpret_cast<double*>(smem_raw + lay.m_off);             // [R][L] this CTA's rows
    double* slots = reinterpret_cast<double*>(smem_raw + lay.prow_off);      // [2][C][L] candidate rows
    double* fcol = reinterpret_cast<double*>(smem_raw + lay.fcol_off);       // [2][R] multipliers
    int* zcol = reinterpret_cast<int*>(smem_raw + lay.zcol_off);             // [2][R] their zero flags
    Cand* infos = reinterpret_cast<Cand*>(smem_raw + lay.info_off);          // [2][C] candidates
    Cand* parts = reinterpret_cast<Cand*>(smem_raw + lay.part_off);          // [NT / 32] phase A's
    int* phys_at = reinterpret_cast<int*>(smem_raw + lay.phys_off);
    int* lpos = reinterpret_cast<int*>(smem_raw + lay.lpos_off);
    int* piv = reinterpret_cast<int*>(smem_raw + lay.piv_off);
    int* sigma = reinterpret_cast<int*>(smem_raw + lay.sig_off);

    const int r0 = rank * R;
    const int nrows = max(0, min(R, L - r0));
    const int nparts = (nrows + 31) / 32;  // warps that hold rows in phase A
    const int row_groups = NT / L;  // thread (tr, j): column j, rows tr, tr + row_groups, ...
    const int j = tid % L, tr = tid / L;
    const bool active = mt < 0 && tr < row_groups;
    const int LS = slot_stride(L);
    const uint32_t row_bytes = (uint32_t)(LS * sizeof(double));  // a multiple of 16
    const uint32_t step_bytes = (uint32_t)(C - 1) * (uint32_t)(row_bytes + sizeof(Cand));

    // Send this CTA's candidate row (already in its own slot, written and
    // fenced for the copy engine by the compute threads before a barrier the
    // messenger has passed) to the other CTAs' slot s: one bulk copy per
    // peer, by the messenger lanes.
    const bool muted = rank == lw.mute_rank;
    auto send_row = [&](int s) {
        if (mt >= 0 && mt < C && mt != rank && !muted) {
            const uint32_t src_row = tc::smem_u32(slots + ((size_t)s * C + rank) * LS);
            tc::bulk_copy_to_peer(tc::mapa_u32(src_row, (uint32_t)mt), src_row, row_bytes,
                                  tc::mapa_u32(tc::smem_u32(&bars[s]), (uint32_t)mt));
        }
    };
    // Send this CTA's candidate to every CTA's slot s: messenger lanes.
    auto send_info = [&](const Cand& c, int s) {
        if (mt >= 0 && mt < C) {
            const double inv = __drcp_rn(c.val);  // inf or NaN for no candidate: never used
            if (mt == rank) {
                Cand& mine = infos[s * C + rank];
                mine.key = c.key;
                mine.val = c.val;
                mine.inv = inv;
                mine.pos = c.pos;
                mine.phys = c.phys;
            } else if (!muted) {
                const uint32_t a = tc::mapa_u32(tc::smem_u32(&infos[s * C + rank]), (uint32_t)mt);
                const uint32_t b = tc::mapa_u32(tc::smem_u32(&bars[s]), (uint32_t)mt);
                tc::st_async_v2_b64(a, c.key, (uint64_t)__double_as_longlong(c.val), b);
                tc::st_async_v2_b64(a + 16, (uint64_t)__double_as_longlong(inv),
                                    ((uint64_t)(uint32_t)c.phys << 32) | (uint32_t)c.pos, b);
            }
        }
    };

    if (mt < 0) {
        for (size_t idx = tid; idx < (size_t)nrows * L; idx += NT) {
            const int r = (int)(idx / L), jj = (int)(idx % L);
            M[idx] = src[(size_t)(r0 + r) * lds + jj];
        }
        for (int r = tid; r < nrows; r += NT) {  // step 0's multipliers
            fcol[r] = src[(size_t)(r0 + r) * lds];
            zcol[r] = zero_flag(fcol[r]);
        }
        for (int q = tid; q < L; q += NT) { phys_at[q] = q; lpos[q] = q; }
    }
    // slot s's barrier completes when the C - 1 other CTAs' candidates and
    // rows for the step using that slot have landed; armed for steps 0 and 1
    // here, re-armed for step k + 2 once step k's wait is over
    if (tid == 0) {
        tc::mbar_init(&bars[0], 1);
        tc::mbar_init(&bars[1], 1);
        tc::fence_mbar_init();
        tc::mbar_arrive_expect_tx(&bars[0], step_bytes);
        tc::mbar_arrive_expect_tx(&bars[1], step_bytes);
    }
    __syncthreads();
    tc::cluster_sync_all();  // every CTA runs, its barriers armed, before the first remote write
    {
        const Cand c = warp_candidate(M, L, nrows, r0, lpos, 0);
        if (active && tr == 0 && c.phys >= 0) {
            slots[(size_t)rank * LS + j] = M[(size_t)(c.phys - r0) * L + j];
            tc::fence_proxy_async_smem();
        }
        __syncthreads();
        send_row(0);
        send_info(c, 0);
    }

    int steps_done = 0;
    int prev_p = -1;
    double prev_inv = 0.0;
    for (int k = 0; k < L; k++) {
        const int s = k & 1;
        const bool ok = slot_wait(&bars[s], (uint32_t)(k >> 1) & 1u, lw.limit_ns);
        if (__syncthreads_or(!ok)) {  // also makes this CTA's own slot entries visible
            if (tid == 0) record_failure(info, SPIN_ERR_TIMEOUT, leaf_index, k);
            break;
        }
        if (tid == 0 && k + 2 < L) tc::mbar_arrive_expect_tx(&bars[s], step_bytes);
        const Cand w = cluster_winner(infos + s * C, C);
        if (bad_pivot(w)) {  // identical decision in every thread of every CTA: all leave together
            if (rank == 0 && tid == 0) record_failure(info, SPIN_ERR_SINGULAR, leaf_index, k);
            break;
        }
        apply_pivot(k, w, phys_at, lpos, piv);
        const int p = w.phys, pl = p - r0;  // the pivot row stays raw
        const double inv = w.inv;
        const double* prow = slots + ((size_t)s * C + p / R) * LS;
        const double* fk = fcol + s * R;
        const int* zk = zcol + s * R;
        double* fn = fcol + (s ^ 1) * R;
        int* zn = zcol + (s ^ 1) * R;
        const double pj = (j == k) ? inv : prow[j] * inv;
        // the previous pivot row is scaled by its 1/pivot (its multiplier is
        // already scaled); column k+1 is scaled in A by the thread that
        // updates it
        const int pr = prev_p - r0;
        const double pinv = prev_inv;
        if (active && prev_p >= 0 && pr >= 0 && pr < nrows && pr % row_groups == tr && j != k + 1) {
            double* rp = M + (size_t)pr * L + j;
            *rp = (j == k - 1) ? pinv : *rp * pinv;
        }
        prev_p = p;
        prev_inv = inv;
        steps_done = k + 1;
        if (k + 1 == L) {  // last step: no next candidate
            if (active) elim_column(M, L, j, fk, zk, pj, j == k, tr, row_groups, nrows, pl, pl);
            break;
        }
        // A: column k+1, one row per thread; the same values give this
        // CTA's candidate for column k+1, a warp argmax each.  A row is
        // eligible if no step before k took it (position >= k) and step k
        // did not (it is not p); the row that was at position k moves to
        // w.pos.  Thread NT - 1 rewrites the position table meanwhile, but
        // only for rows p and phys_at[k], and both values of the latter's
        // entry (k before, w.pos after) give the same answer here.
        if (tid < nparts * 32) {
            uint64_t key = 0;
            double val = 0.0;
            int pos = INT_MAX, phys = -1;
            if (tid < nrows) {
                const double pjn = prow[k + 1] * inv;
                if (tid == pl) {
                    fn[tid] = pjn;
                    zn[tid] = zero_flag(pjn);
                } else {
                    double b = M[(size_t)tid * L + k + 1];
                    if (tid == pr) b *= pinv;
                    const double nv = elim_val(zk[tid], fk[tid], b, pjn, false);
                    M[(size_t)tid * L + k + 1] = nv;
                    fn[tid] = nv;
                    zn[tid] = zero_flag(nv);
                    const int lp = lpos[r0 + tid];
                    if (lp >= k) {
                        const uint64_t mag = (uint64_t)__double_as_longlong(nv) & ~(1ull << 63);
                        key = mag > kInfBits ? kInfBits : mag;
                        val = nv;
                        pos = lp == k ? w.pos : lp;
                        phys = r0 + tid;
                    }
                }
            }
            const Cand wc = warp_argmax(key, val, 0.0, pos, phys);
            if ((tid & 31) == 0) parts[tid >> 5] = wc;
        }
        __syncthreads();  // column k+1, the position table and the warp candidates are up to date
        Cand c;
        {
            Cand q{0, 0.0, 0.0, INT_MAX, -1};
            if ((tid & 31) < nparts) q = parts[tid & 31];
            c = warp_argmax(q.key, q.val, 0.0, q.pos, q.phys);
        }
        if (mt >= 0) {  // the messenger: the candidate now, its row once B is done
            send_info(c, s ^ 1);
            asm volatile("bar.sync 1, %0;" ::"n"(NT + kMessengers) : "memory");
            send_row(s ^ 1);
            continue;
        }
        const int rc = c.phys - r0;  // this CTA's candidate row (never p or the previous pivot row)
        // B: the candidate row's step-k update, into M and into this CTA's own slot
        if (active && c.phys >= 0 && rc % row_groups == tr) {
            double v = M[(size_t)rc * L + j];
            if (j != k + 1) {
                v = elim_val(zk[rc], fk[rc], v, pj, j == k);
                M[(size_t)rc * L + j] = v;
            }
            slots[((size_t)(s ^ 1) * C + rank) * LS + j] = v;
            tc::fence_proxy_async_smem();
        }
        asm volatile("bar.arrive 1, %0;" ::"n"(NT + kMessengers) : "memory");  // own slot row written

        // C: every other row, every column but k+1
        if (active && j != k + 1) elim_column(M, L, j, fk, zk, pj, j == k, tr, row_groups, nrows, pl, rc);
    }
    __syncthreads();
    if (steps_done < L) return;  // failure already recorded; X is undefined
    leaf_finish(M, L, R, r0, nrows, rank, prev_p, prev_inv, lpos, piv, sigma, dst, ldd, info, leaf_index);
}


// One CTA per leaf of a batch (leaf_gj_cta_body): problem blockIdx.x.
__global__ void __launch_bounds__(NT, 3)
leaf_gj_cta_kernel(BatchView srcv, BatchView dstv, int L, int32_t* info_base, int leaf_index) {
    const int z = blockIdx.x;
    const int64_t lds = srcv.ld_of(z), ldd = dstv.ld_of(z);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    leaf_gj_cta_body<false>(srcv.ptr(z, lds), lds, const_cast<double*>(dstv.ptr(z, ldd)), ldd, L,
                            info_base + (int64_t)z * INFO_WORDS, leaf_index, smem_raw);
}

template <bool ROWS_IN_SMEM, bool PUSH>
__device__ __forceinline__ void leaf_gj_body(const double* __restrict__ src, int64_t lds, double* __restrict__ dst,
                                             int64_t ldd, double* __restrict__ gwork, int L, int R, int32_t* info,
                                             int leaf_index, LeafWait lw) {
    if constexpr (PUSH)
        leaf_gj_push_body(src, lds, dst, ldd, L, R, info, leaf_index, lw);
    else
        leaf_gj_pull_body<ROWS_IN_SMEM>(src, lds, dst, ldd, gwork, L, R, info, leaf_index);
}

template <bool ROWS_IN_SMEM, bool PUSH>
__global__ void __launch_bounds__(PUSH ? NT + kMessengers : NT, 1)
leaf_gj_kernel(const double* __restrict__ src, int64_t lds, double* __restrict__ dst, int64_t ldd,
               double* __restrict__ gwork, int L, int R, int32_t* info, int leaf_index, LeafWait lw) {
    leaf_gj_body<ROWS_IN_SMEM, PUSH>(src, lds, dst, ldd, gwork, L, R, info, leaf_index, lw);
}

// Batched form: cluster blockIdx.y inverts problem z = blockIdx.y.  Many
// small leaves share an SM, so the registers are held to two CTAs per SM
// (one leaf's step is latency-bound: a second CTA fills its gaps).
template <bool ROWS_IN_SMEM, bool PUSH>
__global__ void __launch_bounds__(PUSH ? NT + kMessengers : NT, 2)
leaf_gj_batched_kernel(BatchView src, BatchView dst, double* __restrict__ gwork, int64_t gwork_stride, int L, int R,
                       int32_t* info, int leaf_index, LeafWait lw) {
    const int z = blockIdx.y;
    const int64_t lds = src.ld_of(z), ldd = dst.ld_of(z);
    leaf_gj_body<ROWS_IN_SMEM, PUSH>(src.ptr(z, lds), lds, const_cast<double*>(dst.ptr(z, ldd)), ldd,
                                     ROWS_IN_SMEM ? nullptr : gwork + (int64_t)z * gwork_stride, L, R,
                                     info + (int64_t)z * INFO_WORDS, leaf_index, lw);
}

struct LeafConfig {
    int C, R;
    bool smem_rows, push;
    size_t smem;
};

constexpr size_t kSmemBudget = 200 * 1024;

// Largest cluster the GPU can co-schedule for this kernel (16 on GB300 when
// the non-portable size is allowed, else 8); queried once.
int max_cluster_size() {
    static int cached = 0;
    if (cached) return cached;
    cached = 8;
    auto kern = leaf_gj_kernel<true, false>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget) != cudaSuccess ||
        cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) {
        cudaGetLastError();
        return cached;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1, 1);
    cfg.blockDim = dim3(NT, 1, 1);
    cfg.dynamicSmemBytes = leaf_layout(512, 32, 16, true, false).total;
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

size_t leaf_smem_bytes(int64_t L, int C, bool rows, bool push) {
    return leaf_layout((int)L, (int)((L + C - 1) / C), C, rows, push).total;
}

// Cluster shape.  A pivot step costs a barrier's latency plus R*L FMAs on
// each CTA at ~2 FP64 FMA/clock: measured per-step times at L = 128 are
// 12.2 / 7.4 / 4.5 / 3.2 / 2.9 us on 1 / 2 / 4 / 8 / 16 CTAs, and 2.0 us at
// L = 32 on 16.  A single inversion waits on its leaves,
// so it takes the widest cluster (latency); a batch runs many leaves side
// by side, so it takes the narrowest that fits shared memory (SM time).
// Rows are pushed to every CTA when L <= 256 and the slots fit.
// SPIN_LEAF_CLUSTER_MAX caps the single inversions' cluster width (1..16,
// for measurement: a narrower cluster takes longer per leaf but holds fewer
// SMs while other work could use them); read once.
int leaf_cluster_cap() {
    static const int v = [] {
        const char* e = getenv("SPIN_LEAF_CLUSTER_MAX");
        const int x = e ? atoi(e) : 0;
        return (x >= 1 && x <= 16) ? x : 16;
    }();
    return v;
}

LeafConfig leaf_config(int64_t L, bool have_scratch, bool batched = false) {
    LeafConfig c;
    const int cmax = batched ? max_cluster_size() : std::min(max_cluster_size(), leaf_cluster_cap());
    const bool push_ok = L <= kPushMaxL;
    c.C = 1;
    if (batched) {
        while (c.C < cmax && leaf_smem_bytes(L, c.C, true, push_ok) > kSmemBudget) c.C <<= 1;
    } else {
        while (c.C < cmax && c.C < L) c.C <<= 1;
    }
    c.R = (int)((L + c.C - 1) / c.C);
    c.push = push_ok && leaf_smem_bytes(L, c.C, true, true) <= kSmemBudget;
    c.smem_rows = c.push || leaf_smem_bytes(L, c.C, true, false) <= kSmemBudget;
    if (!c.smem_rows && !have_scratch) c.smem_rows = true;  // rejected by the caller's size check
    c.smem = leaf_smem_bytes(L, c.C, c.smem_rows, c.push);
    return c;
}

// Batched leaves of order <= kCtaMaxL run on the one-CTA kernel unless
// SPIN_LEAF_CLUSTER_BATCH=1 (the cluster form on one CTA; for measurement).
bool use_cluster_leaf_for_batches() {
    static const int v = [] {
        const char* e = getenv("SPIN_LEAF_CLUSTER_BATCH");
        return (e && e[0] == '1') ? 1 : 0;
    }();
    return v != 0;
}

template <typename K>
int prepare_leaf_kernel(K kern) {
    SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBudget));
    SPIN_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
    return SPIN_OK;
}

template <bool S, bool P>
int launch_leaf_impl(const double* A, int64_t lda, double* X, int64_t ldx, const LeafConfig& c, int64_t L,
                     double* scratch, int32_t* info, int leaf_index, cudaStream_t s, LeafWait lw = LeafWait()) {
    static PerDeviceOnce attrs;
    auto kern = leaf_gj_kernel<S, P>;
    {
        const int rc = attrs.run([&] { return prepare_leaf_kernel(kern); });
        if (rc != SPIN_OK) return rc;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c.C, 1, 1);
    cfg.blockDim = dim3(P ? NT + kMessengers : NT, 1, 1);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SPIN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, A, lda, X, ldx, scratch, (int)L, c.R, info, leaf_index, lw));
    return SPIN_OK;
}

template <bool S, bool P>
int launch_leaf_batched_impl(const BatchView& src, const BatchView& dst, const LeafConfig& c, int64_t L,
                             double* scratch, int64_t stride, int32_t* info, int leaf_index, int count,
                             cudaStream_t s) {
    static PerDeviceOnce attrs;
    auto kern = leaf_gj_batched_kernel<S, P>;
    {
        const int rc = attrs.run([&] { return prepare_leaf_kernel(kern); });
        if (rc != SPIN_OK) return rc;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)c.C, (unsigned)count, 1);
    cfg.blockDim = dim3(P ? NT + kMessengers : NT, 1, 1);
    cfg.dynamicSmemBytes = c.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c.C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    SPIN_CUDA_TRY(cudaLaunchKernelEx(&cfg, kern, src, dst, scratch, stride, (int)L, c.R, info, leaf_index,
                                     LeafWait()));
    return SPIN_OK;
}

}  // namespace

int launch_leaf_gj_batched(const BatchView& src, const BatchView& dst, int64_t L, double* scratch_base,
                           int64_t scratch_stride, int32_t* info, int leaf_index, int count, cudaStream_t s) {
    if (L <= 0 || count <= 0) return SPIN_OK;
    if (L > kMaxLeaf || count > 65535) return SPIN_ERR_INVALID_ARG;
    if (L <= kCtaMaxL && !use_cluster_leaf_for_batches()) {
        static PerDeviceOnce attrs;
        const size_t smem = cta_leaf_smem((int)L);
        const int rc = attrs.run([&]() -> int {
            SPIN_CUDA_TRY(cudaFuncSetAttribute(leaf_gj_cta_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)cta_leaf_smem(kCtaMaxL)));
            return SPIN_OK;
        });
        if (rc != SPIN_OK) return rc;
        leaf_gj_cta_kernel<<<(unsigned)count, NT, smem, s>>>(src, dst, (int)L, info, leaf_index);
        SPIN_CUDA_TRY(cudaGetLastError());
        return SPIN_OK;
    }
    const LeafConfig c = leaf_config(L, scratch_base != nullptr, true);
    if (c.smem > kSmemBudget) return SPIN_ERR_INVALID_ARG;
    if (c.push) return launch_leaf_batched_impl<true, true>(src, dst, c, L, nullptr, 0, info, leaf_index, count, s);
    if (c.smem_rows)
        return launch_leaf_batched_impl<true, false>(src, dst, c, L, nullptr, 0, info, leaf_index, count, s);
    return launch_leaf_batched_impl<false, false>(src, dst, c, L, scratch_base, scratch_stride, info, leaf_index,
                                                  count, s);
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
    if (c.push) return launch_leaf_impl<true, true>(A, lda, X, ldx, c, L, nullptr, info, leaf_index, s);
    if (c.smem_rows) return launch_leaf_impl<true, false>(A, lda, X, ldx, c, L, nullptr, info, leaf_index, s);
    return launch_leaf_impl<false, false>(A, lda, X, ldx, c, L, scratch, info, leaf_index, s);
}

}  // namespace spin

// Test hook: the identity of order L (2 <= L <= 256, the pushed-row form, on
// its widest cluster) with the CTA of rank mute_rank sending nothing and the
// exchange waits limited to limit_ms.  The other CTAs' waits for step 0 run
// out, the muted CTA's wait for step 1 does, every CTA leaves, and the info
// record gets SPIN_ERR_TIMEOUT.  Remote writes happen only in the first
// exchange, while every CTA still waits.  Returns the recorded status.
extern "C" int spin_test_leaf_timeout(int64_t L, int mute_rank, double limit_ms) {
    using namespace spin;
    if (L < 2 || L > kPushMaxL || !(limit_ms > 0.0) || limit_ms > 4000.0) return SPIN_ERR_INVALID_ARG;
    const LeafConfig c = leaf_config(L, false);
    if (!c.push || mute_rank < 0 || mute_rank >= c.C) return SPIN_ERR_INVALID_ARG;
    double* A = nullptr;
    double* X = nullptr;
    int32_t* info = nullptr;
    const size_t bytes = (size_t)L * (size_t)L * sizeof(double);
    if (cudaMalloc(&A, bytes) != cudaSuccess || cudaMalloc(&X, bytes) != cudaSuccess ||
        cudaMalloc(&info, INFO_WORDS * sizeof(int32_t)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(A);
        cudaFree(X);
        return SPIN_ERR_OOM;
    }
    {  // the identity: the muted CTA gets past step 0 (a valid pivot) and waits at step 1
        std::vector<double> I((size_t)L * (size_t)L, 0.0);
        for (int64_t i = 0; i < L; i++) I[(size_t)i * (size_t)L + (size_t)i] = 1.0;
        cudaMemcpy(A, I.data(), bytes, cudaMemcpyHostToDevice);
    }
    cudaMemset(info, 0, INFO_WORDS * sizeof(int32_t));
    LeafWait lw;
    lw.limit_ns = (uint64_t)(limit_ms * 1e6);
    lw.mute_rank = mute_rank;
    int rc = launch_leaf_impl<true, true>(A, L, X, L, c, L, nullptr, info, 0, 0, lw);
    int32_t h[INFO_WORDS] = {0, 0, 0, 0};
    if (rc == SPIN_OK) {
        if (cudaMemcpy(h, info, sizeof h, cudaMemcpyDeviceToHost) != cudaSuccess) rc = SPIN_ERR_CUDA;
    }
    cudaFree(A);
    cudaFree(X);
    cudaFree(info);
    return rc == SPIN_OK ? h[INFO_STATUS] : rc;
}
