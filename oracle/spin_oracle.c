/*
 * spin_oracle.c -- CPU FP64 oracle for Strassen's block-recursive matrix inversion.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call, link or
 * execute this file: only the tests, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It shares no code, header or constant with the
 * CUDA library.
 *
 * What it computes (Misra et al., "SPIN", ICDCN'18, arXiv 1801.04723):
 *   - oracle_strassen_inv: Algorithm 1 (Strassen's serial inversion), step by
 *     step in the paper's order and notation:
 *        I = A11^-1, II = A21.I, III = I.A12, IV = A21.III, V = IV - A22,
 *        VI = V^-1, C12 = III.VI, C21 = VI.II, VII = III.C21,
 *        C11 = I - VII, C22 = -VI,
 *     recursing until the block order reaches the leaf size, where the block
 *     is inverted directly (Algorithm 1 leaves the direct leaf method open,
 *     Sec. 3.1; this oracle uses Gauss-Jordan with partial pivoting, below).
 *   - oracle_gj_inv: Gauss-Jordan inversion with partial pivoting on the full
 *     matrix (the plain definition X = A^-1), used at the leaves and as an
 *     independent second oracle.
 *   - oracle_residual: rel_res = ||A X - I||_F / (||A||_F ||X||_F) with every
 *     dot product evaluated by compensated (error-free transformation)
 *     arithmetic, so the measure itself is accurate to about 2^-104 relative.
 *   - oracle_freivalds: ||(A X - I) v|| for given probe vectors v, O(k n^2).
 *
 * Readings of the paper taken here (each also listed in the design notes):
 *   - leaf test: a block is a leaf when its order n <= leaf (Alg. 1 stops when
 *     the order equals the threshold, Alg. 2 when one block of that order is
 *     left; the two agree on powers of 2);
 *   - split point for any n (the paper treats n = 2^p only, Sec. 4):
 *     n1 = 32*ceil(n/64) when n > 64, else ceil(n/2); n2 = n - n1;
 *   - leaf pivoting: the row with the largest |a_ik|, i >= k, lowest index on
 *     ties; a zero or non-finite pivot means "singular";
 *   - precision: FP64 (the paper's JBlas DoubleMatrix);
 *   - layout: row-major with a leading dimension (the paper's blocks are
 *     column-major; inversion commutes with transposition).
 *
 * All arithmetic is plain C doubles, naive i-k-j loops with ascending-k
 * summation; compile with -ffp-contract=off so no FMA contraction occurs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_OK 0
#define OR_SINGULAR 2
#define OR_NOMEM 4

/* ---- operation counters (Sec. 4, Table 2: per recursion level SPIN does
 *      4 xy, 6 multiplications, 2 subtractions, 1 scalarMul, 1 arrange) ---- */
typedef struct {
    int64_t leaves;        /* directly inverted blocks                        */
    int64_t internal;      /* internal recursion nodes                        */
    int64_t multiplies;    /* block matrix products                           */
    int64_t subtracts;     /* block subtractions                              */
    int64_t scalar_muls;   /* C22 = -VI                                       */
    int64_t mult_flops;    /* sum 2*m*k*n over products                       */
    int64_t leaf_flops;    /* sum 2*L^3 over leaves (nominal GJ count)        */
    int64_t max_depth;     /* deepest recursion level reached (root = 0)      */
    int64_t fail_leaf;     /* index (in execution order) of the failing leaf  */
    int64_t fail_col;      /* pivot column that failed inside that leaf       */
} oracle_counts;

static oracle_counts g_cnt;

void oracle_counts_reset(void) { memset(&g_cnt, 0, sizeof g_cnt); g_cnt.fail_leaf = -1; g_cnt.fail_col = -1; }
void oracle_counts_get(oracle_counts* out) { *out = g_cnt; }

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
void oracle_set_threads(int t) {
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* C (m x n, ldc) = A (m x k, lda) * B (k x n, ldb); naive, ascending k. */
static void mat_mul(const double* A, int64_t lda, const double* B, int64_t ldb,
                    double* C, int64_t ldc, int64_t m, int64_t k, int64_t n) {
    int64_t i;
#pragma omp parallel for schedule(static) if (m * k * n > 32768)
    for (i = 0; i < m; i++) {
        double* c = C + i * ldc;
        for (int64_t j = 0; j < n; j++) c[j] = 0.0;
        for (int64_t p = 0; p < k; p++) {
            const double a = A[i * lda + p];
            const double* b = B + p * ldb;
            for (int64_t j = 0; j < n; j++) c[j] = c[j] + a * b[j];
        }
    }
    g_cnt.multiplies++;
    g_cnt.mult_flops += 2 * m * k * n;
}

/* C = A - B, all m x n. */
static void mat_sub(const double* A, int64_t lda, const double* B, int64_t ldb,
                    double* C, int64_t ldc, int64_t m, int64_t n) {
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) C[i * ldc + j] = A[i * lda + j] - B[i * ldb + j];
    g_cnt.subtracts++;
}

/* C = s * A (Alg 5, scalarMul). */
static void mat_scale(const double* A, int64_t lda, double s, double* C, int64_t ldc,
                      int64_t m, int64_t n) {
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) C[i * ldc + j] = s * A[i * lda + j];
    g_cnt.scalar_muls++;
}

static void mat_copy(const double* A, int64_t lda, double* C, int64_t ldc, int64_t m, int64_t n) {
    for (int64_t i = 0; i < m; i++) memcpy(C + i * ldc, A + i * lda, (size_t)n * sizeof(double));
}

/*
 * In-place Gauss-Jordan inversion with partial pivoting of the n x n block
 * M (row-major, ld).  On return M holds M^-1.  Returns OR_OK, or OR_SINGULAR
 * with *bad_col set to the pivot column whose pivot was zero or non-finite.
 *
 * Step k: choose the pivot row p >= k maximising |m_pk| (lowest p on ties),
 * swap rows p and k, divide row k by the pivot (the pivot slot receives
 * 1/pivot), then for every other row i subtract f_i = m_ik times row k (the
 * slot m_ik receives -f_i/pivot).  The row interchanges act on the inverse
 * as column interchanges, undone at the end in reverse order.
 */
int oracle_gj_inv(double* M, int64_t ld, int64_t n, int64_t* bad_col) {
    int64_t* piv = (int64_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(int64_t));
    if (!piv) return OR_NOMEM;
    for (int64_t k = 0; k < n; k++) {
        int64_t p = k;
        double best = fabs(M[k * ld + k]);
        for (int64_t i = k + 1; i < n; i++) {
            double v = fabs(M[i * ld + k]);
            if (v > best) { best = v; p = i; }
        }
        const double pv = M[p * ld + k];
        if (pv == 0.0 || !isfinite(pv)) {
            if (bad_col) *bad_col = k;
            free(piv);
            return OR_SINGULAR;
        }
        piv[k] = p;
        if (p != k)
            for (int64_t j = 0; j < n; j++) {
                double t = M[k * ld + j]; M[k * ld + j] = M[p * ld + j]; M[p * ld + j] = t;
            }
        double* rk = M + k * ld;
        const double inv = 1.0 / pv;
        rk[k] = 1.0;
        for (int64_t j = 0; j < n; j++) rk[j] = rk[j] * inv;
        int64_t i;
#pragma omp parallel for schedule(static) if (n >= 256)
        for (i = 0; i < n; i++) {
            if (i == k) continue;
            double* ri = M + i * ld;
            const double f = ri[k];
            if (f == 0.0) continue;
            ri[k] = 0.0;
            for (int64_t j = 0; j < n; j++) ri[j] = ri[j] - f * rk[j];
        }
    }
    for (int64_t k = n - 1; k >= 0; k--) {
        const int64_t p = piv[k];
        if (p != k)
            for (int64_t i = 0; i < n; i++) {
                double t = M[i * ld + k]; M[i * ld + k] = M[i * ld + p]; M[i * ld + p] = t;
            }
    }
    free(piv);
    return OR_OK;
}

int64_t oracle_split(int64_t n) {
    if (n > 64) return 32 * ((n + 63) / 64);
    return (n + 1) / 2;
}

/* Algorithm 1 on the n x n block A (lda) into C (ldc). */
static int strassen_rec(const double* A, int64_t lda, double* C, int64_t ldc,
                        int64_t n, int64_t leaf, int64_t depth) {
    if (depth > g_cnt.max_depth) g_cnt.max_depth = depth;
    if (n <= leaf) {
        /* leaf: invert directly */
        mat_copy(A, lda, C, ldc, n, n);
        int64_t col = -1;
        int st = oracle_gj_inv(C, ldc, n, &col);
        if (st == OR_SINGULAR && g_cnt.fail_leaf < 0) { g_cnt.fail_leaf = g_cnt.leaves; g_cnt.fail_col = col; }
        g_cnt.leaves++;
        g_cnt.leaf_flops += 2 * n * n * n;
        return st;
    }
    g_cnt.internal++;
    const int64_t n1 = oracle_split(n), n2 = n - n1;
    /* breakMat / xy: the four quadrants of A are views (Alg 3, Alg 4). */
    const double* A11 = A;
    const double* A12 = A + n1;
    const double* A21 = A + n1 * lda;
    const double* A22 = A + n1 * lda + n1;

    double* I   = (double*)malloc((size_t)(n1 * n1) * sizeof(double));
    double* II  = (double*)malloc((size_t)(n2 * n1) * sizeof(double));
    double* III = (double*)malloc((size_t)(n1 * n2) * sizeof(double));
    double* IV  = (double*)malloc((size_t)(n2 * n2) * sizeof(double));
    double* V   = (double*)malloc((size_t)(n2 * n2) * sizeof(double));
    double* VI  = (double*)malloc((size_t)(n2 * n2) * sizeof(double));
    double* C12 = (double*)malloc((size_t)(n1 * n2) * sizeof(double));
    double* C21 = (double*)malloc((size_t)(n2 * n1) * sizeof(double));
    double* VII = (double*)malloc((size_t)(n1 * n1) * sizeof(double));
    double* C11 = (double*)malloc((size_t)(n1 * n1) * sizeof(double));
    double* C22 = (double*)malloc((size_t)(n2 * n2) * sizeof(double));
    int st = OR_OK;
    if (!I || !II || !III || !IV || !V || !VI || !C12 || !C21 || !VII || !C11 || !C22) { st = OR_NOMEM; goto done; }

    st = strassen_rec(A11, lda, I, n1, n1, leaf, depth + 1);     /* I   = A11^-1   */
    if (st) goto done;
    mat_mul(A21, lda, I, n1, II, n1, n2, n1, n1);                 /* II  = A21.I    */
    mat_mul(I, n1, A12, lda, III, n2, n1, n1, n2);                /* III = I.A12    */
    mat_mul(A21, lda, III, n2, IV, n2, n2, n1, n2);               /* IV  = A21.III  */
    mat_sub(IV, n2, A22, lda, V, n2, n2, n2);                     /* V   = IV - A22 */
    st = strassen_rec(V, n2, VI, n2, n2, leaf, depth + 1);        /* VI  = V^-1     */
    if (st) goto done;
    mat_mul(III, n2, VI, n2, C12, n2, n1, n2, n2);                /* C12 = III.VI   */
    mat_mul(VI, n2, II, n1, C21, n1, n2, n2, n1);                 /* C21 = VI.II    */
    mat_mul(III, n2, C21, n1, VII, n1, n1, n2, n1);               /* VII = III.C21  */
    mat_sub(I, n1, VII, n1, C11, n1, n1, n1);                     /* C11 = I - VII  */
    mat_scale(VI, n2, -1.0, C22, n2, n2, n2);                     /* C22 = -VI      */
    /* arrange (Alg 6): place the four quadrants of C. */
    mat_copy(C11, n1, C, ldc, n1, n1);
    mat_copy(C12, n2, C + n1, ldc, n1, n2);
    mat_copy(C21, n1, C + n1 * ldc, ldc, n2, n1);
    mat_copy(C22, n2, C + n1 * ldc + n1, ldc, n2, n2);
done:
    free(I); free(II); free(III); free(IV); free(V); free(VI);
    free(C12); free(C21); free(VII); free(C11); free(C22);
    return st;
}

/* Public entry: C (n x n, ldc) = A^-1 by Algorithm 1 with the given leaf order. */
int oracle_strassen_inv(const double* A, int64_t lda, double* C, int64_t ldc, int64_t n, int64_t leaf) {
    if (n < 1 || leaf < 1 || lda < n || ldc < n) return 1;
    return strassen_rec(A, lda, C, ldc, n, leaf, 0);
}

/* ---- compensated arithmetic (Ogita, Rump, Oishi 2005: TwoSum, TwoProduct
 *      by Dekker splitting, Dot2) -- no FMA is used anywhere. ---- */
static inline void two_sum(double a, double b, double* s, double* e) {
    double x = a + b;
    double z = x - a;
    *e = (a - (x - z)) + (b - z);
    *s = x;
}
static inline void split(double a, double* hi, double* lo) {
    const double factor = 134217729.0; /* 2^27 + 1 */
    double c = factor * a;
    double h = c - (c - a);
    *hi = h;
    *lo = a - h;
}
static inline void two_prod(double a, double b, double* p, double* e) {
    double x = a * b;
    double ah, al, bh, bl;
    split(a, &ah, &al);
    split(b, &bh, &bl);
    *e = al * bl - (((x - ah * bh) - al * bh) - ah * bl);
    *p = x;
}

/*
 * rel_res = ||A X - I||_F / (||A||_F ||X||_F); R_ij = sum_k a_ik x_kj - d_ij
 * evaluated with Dot2 (the -d_ij enters as one more compensated term).
 * If R (optional, n x n) is given it receives the residual matrix.
 * Returns the relative residual; *abs_out (optional) receives ||AX - I||_F.
 */
double oracle_residual(const double* A, int64_t lda, const double* X, int64_t ldx, int64_t n,
                       double* R, double* abs_out) {
    double ss_r = 0.0, ss_a = 0.0, ss_x = 0.0;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : ss_r, ss_a, ss_x)
    for (i = 0; i < n; i++) {
        double* acc_s = (double*)calloc((size_t)n, sizeof(double));
        double* acc_c = (double*)calloc((size_t)n, sizeof(double));
        for (int64_t k = 0; k < n; k++) {
            const double a = A[i * lda + k];
            ss_a += a * a;
            const double* xr = X + k * ldx;
            for (int64_t j = 0; j < n; j++) {
                double p, ep, s, es;
                two_prod(a, xr[j], &p, &ep);
                two_sum(acc_s[j], p, &s, &es);
                acc_s[j] = s;
                acc_c[j] += ep + es;
            }
        }
        for (int64_t j = 0; j < n; j++) {
            double s, es;
            two_sum(acc_s[j], (i == j) ? -1.0 : 0.0, &s, &es);
            const double r = s + (acc_c[j] + es);
            if (R) R[i * n + j] = r;
            ss_r += r * r;
            const double x = X[i * ldx + j];
            ss_x += x * x;
        }
        free(acc_s);
        free(acc_c);
    }
    if (abs_out) *abs_out = sqrt(ss_r);
    const double den = sqrt(ss_a) * sqrt(ss_x);
    return sqrt(ss_r) / den;
}

/*
 * Freivalds-style probes: for each of the k columns v of V (n x k, row-major),
 * out[c] = ||A (X v) - v||_2, with both matrix-vector products in compensated
 * arithmetic.  O(k n^2) work: usable at orders where AX is out of reach.
 */
void oracle_freivalds(const double* A, int64_t lda, const double* X, int64_t ldx, int64_t n,
                      const double* V, int64_t k, double* out) {
    double* y = (double*)malloc((size_t)n * sizeof(double));
    for (int64_t c = 0; c < k; c++) {
        int64_t i;
#pragma omp parallel for schedule(static)
        for (i = 0; i < n; i++) {
            double s = 0.0, comp = 0.0;
            for (int64_t j = 0; j < n; j++) {
                double p, ep, t, et;
                two_prod(X[i * ldx + j], V[j * k + c], &p, &ep);
                two_sum(s, p, &t, &et);
                s = t;
                comp += ep + et;
            }
            y[i] = s + comp;
        }
        double ss = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : ss)
        for (i = 0; i < n; i++) {
            double s = 0.0, comp = 0.0;
            for (int64_t j = 0; j < n; j++) {
                double p, ep, t, et;
                two_prod(A[i * lda + j], y[j], &p, &ep);
                two_sum(s, p, &t, &et);
                s = t;
                comp += ep + et;
            }
            double t, et;
            two_sum(s, -V[i * k + c], &t, &et);
            const double r = t + (comp + et);
            ss += r * r;
        }
        out[c] = sqrt(ss);
    }
    free(y);
}

/* Relative Frobenius difference ||X - Y||_F / ||Y||_F. */
double oracle_rel_diff(const double* X, int64_t ldx, const double* Y, int64_t ldy, int64_t m, int64_t n) {
    double num = 0.0, den = 0.0;
    for (int64_t i = 0; i < m; i++)
        for (int64_t j = 0; j < n; j++) {
            const double d = X[i * ldx + j] - Y[i * ldy + j];
            num += d * d;
            den += Y[i * ldy + j] * Y[i * ldy + j];
        }
    return den > 0 ? sqrt(num / den) : sqrt(num);
}
