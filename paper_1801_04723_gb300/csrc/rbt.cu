// Random butterfly transform (RBT) around the recursion, for matrices whose
// leading blocks may be singular.
//
// Algorithm 1 inverts A11 and the Schur complement V without pivoting
// across blocks, so the paper restricts itself to matrices for which they
// are invertible (Sec. 2.1: positive definite).  A random butterfly
// transform (Parker, 1995; in the recursive form of Baboulin, Dongarra,
// Herrmann and Tomov, 2013) makes every leading block of U^T A V
// nonsingular with probability one for a nonsingular A, and
// A^-1 = V (U^T A V)^-1 U^T.
//
// A butterfly of order m (m even, h = m/2) is B = [[R, S], [R, -S]] / sqrt(2)
// with R, S random diagonal h x h matrices, diagonal entries exp(rho / 10),
// rho uniform in [-1/2, 1/2].  The recursive butterfly of depth d for order
// n (a multiple of 2^d) is W = L_d ... L_1 with L_k block diagonal: 2^(k-1)
// butterflies of order n / 2^(k-1).  Applying one level to a matrix touches
// every entry once (pairs of rows or pairs of columns), so the transform
// and its inverse cost 4d passes over n^2 entries: HBM-bound and small next
// to the 2 n^3 of the inversion.
//
// The random diagonals are drawn from splitmix64 (Steele, Lea and Flood,
// 2014) at counter (b * d + k) * n + i for butterfly b (0: U, 1: V), level
// k (0-based, L_{k+1}) and entry i (R of block j at j*m + [0, h), S at
// j*m + [h, m)), as a 53-bit uniform u, rho = u - 1/2.
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace spin {
namespace {

__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t c) {
    uint64_t z = seed + (c + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__global__ void rbt_diag_kernel(uint64_t seed, int64_t count, double* __restrict__ out) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < count; c += (int64_t)gridDim.x * blockDim.x) {
        const double u = (double)(splitmix64_at(seed, (uint64_t)c) >> 11) * 0x1.0p-53;
        out[c] = exp((u - 0.5) / 10.0);
    }
}

// Ar (np x np) = A (n x n, lda) padded with the identity.
__global__ void pad_identity_kernel(const double* __restrict__ A, int64_t lda, int64_t n, double* __restrict__ Ar,
                                    int64_t np) {
    const int64_t total = np * np;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / np, j = idx % np;
        Ar[idx] = (i < n && j < n) ? A[i * lda + j] : (i == j ? 1.0 : 0.0);
    }
}

// X (n x n, ldx) = top-left block of Y (np x np).
__global__ void crop_kernel(const double* __restrict__ Y, int64_t np, double* __restrict__ X, int64_t ldx,
                            int64_t n) {
    const int64_t total = n * n;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = idx / n, j = idx % n;
        X[i * ldx + j] = Y[i * np + j];
    }
}

// One level of butterflies of order m on M (np x np, ld), in place.  The
// level's diagonal entries are d[0 .. np): block j has R = d[j*m .. j*m+h)
// and S = d[j*m+h .. j*m+m).  Modes (x_i, x_{i+h}) -> (y_i, y_{i+h}):
//   0  left,  B:   ((r x_i + s x_{i+h}), (r x_i - s x_{i+h})) / sqrt 2  on rows
//   1  left,  B^T: (r (x_i + x_{i+h}), s (x_i - x_{i+h})) / sqrt 2      on rows
//   2  right, B:   (r (x_j + x_{j+h}), s (x_j - x_{j+h})) / sqrt 2      on columns
//   3  right, B^T: ((r x_j + s x_{j+h}), (r x_j - s x_{j+h})) / sqrt 2  on columns
__global__ void butterfly_level_kernel(double* __restrict__ M, int64_t ld, int64_t np, int64_t m,
                                       const double* __restrict__ d, int mode) {
    const int64_t h = m / 2;
    const int64_t pairs = np / 2 * np;  // (pair index, other coordinate)
    const double c = 0.70710678118654752440;  // 1 / sqrt(2), rounded to nearest
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < pairs;
         idx += (int64_t)gridDim.x * blockDim.x) {
        // consecutive threads take consecutive columns (rows) of a row pair
        // (column pair), so every access is coalesced
        const int64_t p = mode < 2 ? idx / np : idx % (np / 2);  // pair p of np/2
        const int64_t o = mode < 2 ? idx % np : idx / (np / 2);  // the other coordinate
        const int64_t blk = p / h, i = p % h;
        const int64_t a = blk * m + i, b = a + h;      // the paired rows (left) or columns (right)
        const double r = d[a], s = d[b];
        double* xa = mode < 2 ? M + a * ld + o : M + o * ld + a;
        double* xb = mode < 2 ? M + b * ld + o : M + o * ld + b;
        const double u = *xa, v = *xb;
        double ya, yb;
        if (mode == 0 || mode == 3) {
            ya = (r * u + s * v) * c;
            yb = (r * u - s * v) * c;
        } else {
            ya = r * (u + v) * c;
            yb = s * (u - v) * c;
        }
        *xa = ya;
        *xb = yb;
    }
}

int grid_for(int64_t work) { return (int)std::min<int64_t>((work + 255) / 256, 152 * 16); }

}  // namespace

int64_t rbt_padded_order(int64_t n, int depth) {
    const int64_t q = (int64_t)1 << depth;
    return (n + q - 1) / q * q;
}

int launch_rbt_diagonals(uint64_t seed, int64_t np, int depth, double* out, cudaStream_t s) {
    const int64_t count = 2 * (int64_t)depth * np;
    rbt_diag_kernel<<<grid_for(count), 256, 0, s>>>(seed, count, out);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

// Ar = U^T pad(A) V: U^T = L1^T ... Ld^T (Ld^T applied first), V = Ld ... L1
// on the right (Ld applied first).
int launch_rbt_forward(const double* A, int64_t lda, int64_t n, double* Ar, int64_t np, int depth,
                       const double* diag, cudaStream_t s) {
    pad_identity_kernel<<<grid_for(np * np), 256, 0, s>>>(A, lda, n, Ar, np);
    const int64_t half = np / 2 * np;
    for (int k = depth; k >= 1; k--) {  // left: U^T
        const int64_t m = np >> (k - 1);
        butterfly_level_kernel<<<grid_for(half), 256, 0, s>>>(Ar, np, np, m, diag + (int64_t)(k - 1) * np, 1);
    }
    for (int k = depth; k >= 1; k--) {  // right: V
        const int64_t m = np >> (k - 1);
        butterfly_level_kernel<<<grid_for(half), 256, 0, s>>>(Ar, np, np, m,
                                                              diag + (int64_t)(depth + k - 1) * np, 2);
    }
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

// X = crop(V Y U^T): V = Ld ... L1 on the left (L1 applied first), U^T =
// L1^T ... Ld^T on the right (L1^T applied first); Y is overwritten.
int launch_rbt_backward(double* Y, int64_t np, int depth, const double* diag, double* X, int64_t ldx, int64_t n,
                        cudaStream_t s) {
    const int64_t half = np / 2 * np;
    for (int k = 1; k <= depth; k++) {  // left: V
        const int64_t m = np >> (k - 1);
        butterfly_level_kernel<<<grid_for(half), 256, 0, s>>>(Y, np, np, m, diag + (int64_t)(depth + k - 1) * np,
                                                              0);
    }
    for (int k = 1; k <= depth; k++) {  // right: U^T
        const int64_t m = np >> (k - 1);
        butterfly_level_kernel<<<grid_for(half), 256, 0, s>>>(Y, np, np, m, diag + (int64_t)(k - 1) * np, 3);
    }
    crop_kernel<<<grid_for(n * n), 256, 0, s>>>(Y, np, X, ldx, n);
    SPIN_CUDA_TRY(cudaGetLastError());
    return SPIN_OK;
}

}  // namespace spin

extern "C" int spin_rbt_diagonals(uint64_t seed, int64_t n, int depth, double* out_dev, spin_stream_t stream) {
    if (n < 1 || depth < 1 || depth > 8 || out_dev == nullptr) return SPIN_ERR_INVALID_ARG;
    const int64_t np = spin::rbt_padded_order(n, depth);
    return spin::launch_rbt_diagonals(seed, np, depth, out_dev, (cudaStream_t)stream);
}
