// Mixed-precision level products: operand splitting, slice-pair schedules
// and the two tensor-core product forms (see tc_gemm.cu):
//
//   bf16x3   D = beta*C + alpha*(A_hi B_hi + A_hi B_lo + A_lo B_hi)
//   ozaki(s) D = beta*C + alpha*(A B) (+ I) with s fixed-point digit slices
//            per operand, pairs (t, u) with t + u < s, exact partial sums.
//
// The split planes live in a per-stream scratch arena owned by the caller
// (struct MixScratch), reused across calls.
#include <algorithm>
#include <cmath>
#include <mutex>

#include "common.cuh"
#include "mixed.h"
#include "tc_gemm.h"

namespace spin {

void tc_pairs_bf16x3(TcGemmParams& p) {
    const int8_t pa[3] = {0, 0, 1}, pb[3] = {0, 1, 0};
    p.num_pairs = 3;
    for (int i = 0; i < 3; i++) {
        p.pa[i] = pa[i];
        p.pb[i] = pb[i];
        p.pg[i] = 0;
    }
    p.exact = 0;
}

void tc_pairs_bf16x6(TcGemmParams& p) {
    // planes 0 = hi, 1 = mid, 2 = lo: pairs of combined weight >= 2^-16
    const int8_t pa[6] = {0, 0, 1, 0, 1, 2}, pb[6] = {0, 1, 0, 2, 1, 0};
    p.num_pairs = 6;
    for (int i = 0; i < 6; i++) {
        p.pa[i] = pa[i];
        p.pb[i] = pb[i];
        p.pg[i] = 0;
    }
    p.exact = 0;
}

void tc_pairs_ozaki(TcGemmParams& p, int slices) {
    int q = 0;
    for (int w = 0; w < slices; w++)  // group w: pairs (t, u) with t + u = w
        for (int t = 0; t <= w; t++) {
            p.pa[q] = (int8_t)t;
            p.pb[q] = (int8_t)(w - t);
            p.pg[q] = (int8_t)w;
            q++;
        }
    p.num_pairs = q;
    // x = 2^(e - 7) sum_t d_t 2^(-8 t): pair (t, u) weighs 2^(e_i + f_j - 14 - 8 (t + u))
    for (int w = 0; w < slices; w++) p.group_shift[w] = -14 - 8 * w;
    p.exact = 1;
    p.chunk_kb = 16;  // runs of 1024: every partial sum is an integer of magnitude <= 2^24, exact in FP32
}

// The digit-slice residual's error relative to ||A||_F ||X||_F with s 8-bit
// slices at order n.  An exact CPU simulation of the product (Householder
// SPD matrices of condition 1e3 and approximate inverses, n = 1024, every
// pair product exact, compared with an 80-bit reference) gives
// 0.62 sqrt(n) 2^-(8s-1) for s = 6 and 0.67 sqrt(n) 2^-(8s-1) for s = 7;
// the model takes 0.7.
double residual_error_model(int64_t n, int s) {
    return 0.7 * std::sqrt((double)n) * std::ldexp(1.0, -(8 * s - 1));
}

int residual_slices_for(int64_t n, double tol) {
    for (int s = 5; s < kMaxResidualSlices; s++)
        if (residual_error_model(n, s) <= 0.01 * tol) return s;
    return kMaxResidualSlices;
}

int first_residual_slices_for(int64_t n, double tol, int sr) {
    for (int s = 4; s < sr; s++)
        if (residual_error_model(n, s) <= 0.2 * tol) return s;
    return sr;
}

int MixScratch::reserve(size_t bytes) {
    if (bytes <= cap) return SPIN_OK;
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
    if (cudaMalloc(&base, bytes) != cudaSuccess) {
        cudaGetLastError();
        return SPIN_ERR_OOM;
    }
    cap = bytes;
    return SPIN_OK;
}

size_t bf16x3_scratch_bytes(int64_t m, int64_t n, int64_t k) {
    const int64_t ld = tc_ld(k);
    return (size_t)(2 * m * ld + 2 * n * ld) * 2 + 256;
}

size_t bf16x6_scratch_bytes(int64_t m, int64_t n, int64_t k) {
    const int64_t ld = tc_ld(k);
    return (size_t)(3 * m * ld + 3 * n * ld) * 2 + 256;
}

size_t ozaki_scratch_bytes(int64_t m, int64_t n, int64_t k, int slices) {
    const int64_t ld = tc_ld(k);
    return (size_t)(slices * m * ld + slices * n * ld) * 2 + (size_t)(m + n) * 4 + 1024;
}

static uintptr_t align_up(uintptr_t p, uintptr_t a) { return (p + a - 1) / a * a; }

int plan_bf16x3(int64_t m, int64_t n, int64_t k, void* scratch, size_t bytes, SplitPlan* sp) {
    if (bytes < bf16x3_scratch_bytes(m, n, k)) return SPIN_ERR_INVALID_ARG;
    sp->ld = tc_ld(k);
    sp->a = (uint16_t*)align_up((uintptr_t)scratch, 256);
    sp->b = sp->a + 2 * m * sp->ld;
    sp->ea = sp->eb = nullptr;
    sp->slices = 2;
    return SPIN_OK;
}

int plan_ozaki(int64_t m, int64_t n, int64_t k, int slices, void* scratch, size_t bytes, SplitPlan* sp) {
    if (slices < 1 || slices > 7) return SPIN_ERR_INVALID_ARG;
    if (bytes < ozaki_scratch_bytes(m, n, k, slices)) return SPIN_ERR_INVALID_ARG;
    sp->ld = tc_ld(k);
    sp->a = (uint16_t*)align_up((uintptr_t)scratch, 256);
    sp->b = sp->a + (int64_t)slices * m * sp->ld;
    sp->ea = (int*)align_up((uintptr_t)(sp->b + (int64_t)slices * n * sp->ld), 16);
    sp->eb = sp->ea + m;
    sp->slices = slices;
    return SPIN_OK;
}

int split_a_bf16x3(const SplitPlan& sp, const double* A, int64_t lda, int64_t m, int64_t k, cudaStream_t s) {
    return launch_split_bf16x2(A, lda, (int)m, (int)k, false, sp.a, sp.ld, s);
}
int split_b_bf16x3(const SplitPlan& sp, const double* B, int64_t ldb, int64_t k, int64_t n, cudaStream_t s) {
    return launch_split_bf16x2(B, ldb, (int)k, (int)n, true, sp.b, sp.ld, s);
}
int split_a_ozaki(const SplitPlan& sp, const double* A, int64_t lda, int64_t m, int64_t k, double* sumsq,
                  cudaStream_t s) {
    return launch_ozaki_split(A, lda, (int)m, (int)k, false, sp.slices, sp.ea, sp.a, sp.ld, sumsq, s);
}
int split_b_ozaki(const SplitPlan& sp, const double* B, int64_t ldb, int64_t k, int64_t n, double* sumsq,
                  cudaStream_t s, const int* active) {
    return launch_ozaki_split(B, ldb, (int)k, (int)n, true, sp.slices, sp.eb, sp.b, sp.ld, sumsq, s, active);
}

int product_bf16x3(const SplitPlan& sp, int64_t m, int64_t n, int64_t k, double alpha, double beta, const double* C,
                   int64_t ldc, double* D, int64_t ldd, int* err, cudaStream_t s) {
    TcGemmParams p = {};
    p.M = (int)m;
    p.N = (int)n;
    p.K = (int)k;
    tc_pairs_bf16x3(p);
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.D = D;
    p.ldd = ldd;
    p.err = err;
    TcOperand oa{sp.a, (int)m, 2, sp.ld}, ob{sp.b, (int)n, 2, sp.ld};
    return launch_tc_gemm(oa, ob, p, s);
}

int plan_bf16x6(int64_t m, int64_t n, int64_t k, void* scratch, size_t bytes, SplitPlan* sp) {
    if (bytes < bf16x6_scratch_bytes(m, n, k)) return SPIN_ERR_INVALID_ARG;
    sp->ld = tc_ld(k);
    sp->a = (uint16_t*)align_up((uintptr_t)scratch, 256);
    sp->b = sp->a + 3 * m * sp->ld;
    sp->ea = sp->eb = nullptr;
    sp->slices = 3;
    return SPIN_OK;
}

int split_a_bf16x6(const SplitPlan& sp, const double* A, int64_t lda, int64_t m, int64_t k, cudaStream_t s,
                   const int* active) {
    return launch_split_bf16x3p(A, lda, (int)m, (int)k, false, sp.a, sp.ld, s, active);
}
int split_b_bf16x6(const SplitPlan& sp, const double* B, int64_t ldb, int64_t k, int64_t n, cudaStream_t s,
                   const int* active) {
    return launch_split_bf16x3p(B, ldb, (int)k, (int)n, true, sp.b, sp.ld, s, active);
}

int product_bf16x6(const SplitPlan& sp, int64_t m, int64_t n, int64_t k, double alpha, double beta, const double* C,
                   int64_t ldc, double* D, int64_t ldd, int* err, cudaStream_t s, const int* active) {
    TcGemmParams p = {};
    p.M = (int)m;
    p.N = (int)n;
    p.K = (int)k;
    tc_pairs_bf16x6(p);
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.D = D;
    p.ldd = ldd;
    p.err = err;
    p.active = active;
    TcOperand oa{sp.a, (int)m, 3, sp.ld}, ob{sp.b, (int)n, 3, sp.ld};
    return launch_tc_gemm(oa, ob, p, s);
}

int product_ozaki(const SplitPlan& sp, int64_t m, int64_t n, int64_t k, double alpha, double beta, const double* C,
                  int64_t ldc, double* D, int64_t ldd, int add_identity, double* sumsq, int* err, cudaStream_t s,
                  const int* active, int pair_slices) {
    const int slices = sp.slices;
    if (pair_slices < 1 || pair_slices > slices) pair_slices = slices;
    TcGemmParams p = {};
    p.M = (int)m;
    p.N = (int)n;
    p.K = (int)k;
    tc_pairs_ozaki(p, pair_slices);
    p.alpha = alpha;
    p.beta = beta;
    p.C = C;
    p.ldc = ldc;
    p.D = D;
    p.ldd = ldd;
    p.row_exp = sp.ea;
    p.col_exp = sp.eb;
    p.add_identity = add_identity;
    p.sumsq = sumsq;
    p.err = err;
    p.active = active;
    TcOperand oa{sp.a, (int)m, slices, sp.ld}, ob{sp.b, (int)n, slices, sp.ld};
    return launch_tc_gemm(oa, ob, p, s);
}

int gemm_bf16x3(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, const double* B,
                int64_t ldb, double beta, const double* C, int64_t ldc, double* D, int64_t ldd, void* scratch,
                size_t scratch_bytes, int* err, cudaStream_t s) {
    if (m <= 0 || n <= 0) return SPIN_OK;
    if (k <= 0) return SPIN_ERR_INVALID_ARG;
    SplitPlan sp;
    int rc = plan_bf16x3(m, n, k, scratch, scratch_bytes, &sp);
    if (rc) return rc;
    if ((rc = split_a_bf16x3(sp, A, lda, m, k, s))) return rc;
    if ((rc = split_b_bf16x3(sp, B, ldb, k, n, s))) return rc;
    return product_bf16x3(sp, m, n, k, alpha, beta, C, ldc, D, ldd, err, s);
}

int gemm_ozaki(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda, const double* B,
               int64_t ldb, double beta, const double* C, int64_t ldc, double* D, int64_t ldd, int slices,
               int add_identity, double* sumsq, double* sumsq_a, double* sumsq_b, void* scratch,
               size_t scratch_bytes, int* err, cudaStream_t s, const OzakiCachedA* cached_a) {
    if (m <= 0 || n <= 0) return SPIN_OK;
    if (k <= 0) return SPIN_ERR_INVALID_ARG;
    SplitPlan sp;
    int rc = plan_ozaki(m, n, k, slices, scratch, scratch_bytes, &sp);
    if (rc) return rc;
    if (cached_a != nullptr) {
        sp.a = cached_a->planes;
        sp.ea = cached_a->exps;
    } else if ((rc = split_a_ozaki(sp, A, lda, m, k, sumsq_a, s))) {
        return rc;
    }
    if ((rc = split_b_ozaki(sp, B, ldb, k, n, sumsq_b, s))) return rc;
    return product_ozaki(sp, m, n, k, alpha, beta, C, ldc, D, ldd, add_identity, sumsq, err, s);
}

int ozaki_split_a(const double* A, int64_t lda, int64_t m, int64_t k, int slices, OzakiCachedA* out,
                  double* sumsq, cudaStream_t s, const int* active) {
    const int64_t ld = tc_ld(k);
    return launch_ozaki_split(A, lda, (int)m, (int)k, false, slices, out->exps, out->planes, ld, sumsq, s, active);
}

}  // namespace spin

// ---------------------------------------------------------------- C ABI --

using namespace spin;

namespace {
std::mutex g_mix_mu;
MixScratch g_test_scratch;  // building-block entry points only
int* g_test_err = nullptr;  // device word: first bounded wait that gave up

int ensure_test_err() {
    if (g_test_err) return SPIN_OK;
    if (cudaMalloc(&g_test_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return SPIN_ERR_OOM;
    }
    SPIN_CUDA_TRY(cudaMemset(g_test_err, 0, sizeof(int)));
    return SPIN_OK;
}
}  // namespace

extern "C" int spin_take_device_error(spin_stream_t stream) {
    std::lock_guard<std::mutex> lk(g_mix_mu);
    if (!g_test_err) return SPIN_OK;
    int h = 0;
    SPIN_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    SPIN_CUDA_TRY(cudaMemcpy(&h, g_test_err, sizeof(int), cudaMemcpyDeviceToHost));
    SPIN_CUDA_TRY(cudaMemset(g_test_err, 0, sizeof(int)));
    return h;
}

extern "C" int spin_gemm_bf16x3(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                                const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D,
                                int64_t ldd, spin_stream_t stream) {
    if (m < 0 || n < 0 || k < 1 || lda < k || ldb < n || ldd < n) return SPIN_ERR_INVALID_ARG;
    if (!(alpha == 1.0 || alpha == -1.0) || !(beta == 0.0 || beta == 1.0)) return SPIN_ERR_INVALID_ARG;
    if (beta != 0.0 && (C == nullptr || ldc < n)) return SPIN_ERR_INVALID_ARG;
    if (m > INT32_MAX / 8 || n > INT32_MAX / 8 || k > INT32_MAX / 8) return SPIN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mix_mu);
    int rc = ensure_test_err();
    if (rc) return rc;
    rc = g_test_scratch.reserve(bf16x3_scratch_bytes(m, n, k));
    if (rc) return rc;
    return gemm_bf16x3(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, g_test_scratch.base, g_test_scratch.cap,
                       g_test_err, (cudaStream_t)stream);
}

extern "C" int spin_gemm_ozaki(int64_t m, int64_t n, int64_t k, double alpha, const double* A, int64_t lda,
                               const double* B, int64_t ldb, double beta, const double* C, int64_t ldc, double* D,
                               int64_t ldd, int slices, int add_identity, double* sumsq_dev, spin_stream_t stream) {
    if (m < 0 || n < 0 || k < 1 || lda < k || ldb < n || ldd < n) return SPIN_ERR_INVALID_ARG;
    if (!(alpha == 1.0 || alpha == -1.0) || !(beta == 0.0 || beta == 1.0)) return SPIN_ERR_INVALID_ARG;
    if (beta != 0.0 && (C == nullptr || ldc < n)) return SPIN_ERR_INVALID_ARG;
    if (slices < 1 || slices > 7) return SPIN_ERR_INVALID_ARG;
    if (m > INT32_MAX / 8 || n > INT32_MAX / 8 || k > INT32_MAX / 8) return SPIN_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_mix_mu);
    int rc = ensure_test_err();
    if (rc) return rc;
    rc = g_test_scratch.reserve(ozaki_scratch_bytes(m, n, k, slices));
    if (rc) return rc;
    return gemm_ozaki(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, D, ldd, slices, add_identity, sumsq_dev, nullptr,
                      nullptr, g_test_scratch.base, g_test_scratch.cap, g_test_err, (cudaStream_t)stream, nullptr);
}
