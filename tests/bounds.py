"""Element-wise error bound shared by the parity tests.

First-order perturbation of an inverse: (A + dA)^-1 = X - X dA X + O(dA^2),
so a computation whose every step perturbs the data by at most eps relative
to |A| leaves element (i, j) within eps (|X| |A| |X|)_ij of the exact
inverse (the componentwise condition of inversion).  Two FP64 inversions of
order n that differ only in rounding order then agree element by element to

    |X - X_ref|_ij <= c * n * u * (|X_ref| |A| |X_ref|)_ij,   u = 2^-53,

with c = 4 here.  The oracle against LAPACK on the seeded families of the
parity tests (orders 65 ... 1500) stays below c = 0.1; a wrong entry in one
small block of the result, which a Frobenius norm over the whole matrix can
hide, does not pass (tests/test_oracle_pins.py plants one)."""
import numpy as np

U = 2.0 ** -53


def componentwise_ratio(X, ref, A) -> float:
    """max_ij |X - ref|_ij / (n u (|ref| |A| |ref|)_ij)."""
    n = A.shape[0]
    B = np.abs(ref) @ (np.abs(A) @ np.abs(ref))
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.abs(X - ref) / (n * U * B)
    r[(B == 0) & (X == ref)] = 0.0
    return float(np.nanmax(np.where(np.isnan(r), np.inf, r)))


def elementwise_ok(X, ref, A, c: float = 4.0) -> bool:
    return componentwise_ratio(X, ref, A) <= c
