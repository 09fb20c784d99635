// The plain batched recursion as one persistent kernel over a device-side
// task list (persistent.cu; the list is built by batched.cu).
#pragma once
#include "common.cuh"

namespace spin {

// An operand of a stage, the same view inside every matrix of a bucket:
// src 0 = the input A (per-matrix base and leading dimension), 1 = the
// output X, 2 = the matrix's workspace (leading dimension ld for both);
// the view starts at row r0, column c0 (a workspace view keeps r0 = 0 and
// puts its linear offset in c0).
struct PView {
    int32_t src;
    int32_t pad;
    int64_t ld, r0, c0;
};

// One step of a bucket's recursion (Algorithm 1's leaf inversion, or one of
// its six level products with the subtraction and sign in the epilogue),
// the same for every matrix of the bucket.  Its tasks are (matrix, output
// tile): `tiles` per matrix, in matrix-major order.  A task of matrix z may
// start once z's earlier stages are done, i.e. once `need` of z's tasks
// have finished.
struct PStage {
    int32_t kind;        // 0: leaf (a -> d, order m), 1: product d = beta c + alpha a b
    int32_t first;       // sorted index of the bucket's first matrix
    int32_t count;       // matrices of the bucket
    int32_t tm;          // product tile order (64, 32 or 16)
    int32_t tiles_n;     // tile columns per matrix
    int32_t tiles;       // tasks per matrix (leaf: 1)
    int32_t need;        // tasks of the matrix's earlier stages
    int32_t leaf_index;  // leaf: index reported with a failure
    int32_t bucket;      // index of the bucket (per-bucket clock counters)
    int32_t pad;
    int64_t m, n, k;
    double alpha, beta;
    PView a, b, c, d;
};

enum { PSTAGE_LEAF = 0, PSTAGE_PRODUCT = 1 };

// Largest leaf the persistent kernel inverts (one CTA, the block in shared
// memory beside the product tiles' buffers).
constexpr int64_t kPersistMaxLeaf = 64;

struct PersistentArgs {
    const PStage* stages;    // device, nstages entries in task order
    const int64_t* start;    // device, nstages + 1 entries: first task of each stage, then the total
    int nstages;
    const double* const* a_base;
    const int64_t* a_ld;
    double* const* x_base;
    double* const* w_base;
    int32_t* records;        // [matrices][INFO_WORDS]
    unsigned* done;          // [matrices] finished tasks (zero before the launch)
    unsigned long long* next;  // task counter (zero before the launch)
    int* err;                // SPIN_ERR_TIMEOUT once a dependency wait ran out (zero before the launch)
    uint64_t limit_ns;       // bound of one dependency wait
    unsigned long long* bucket_clocks;  // optional: SM clocks spent on each bucket's tasks (autotuner)
};

// Dynamic shared memory of the kernel for leaves up to max_leaf.
size_t persistent_smem_bytes(int64_t max_leaf);
// CTAs of one launch: every CTA the GPU holds at once (occupancy x SMs),
// at most `tasks`.
int persistent_grid(size_t smem, int64_t tasks, int* grid);
int launch_persistent_batch(const PersistentArgs& a, size_t smem, int grid, cudaStream_t s);

}  // namespace spin
