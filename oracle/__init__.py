"""CPU FP64 oracle for Strassen's block-recursive matrix inversion (SPIN).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports, links or runs anything here, and this package shares no code
with it.

The arithmetic lives in ``spin_oracle.c`` (plain C, FP64, no FMA contraction);
this module compiles it with gcc on first use and wraps it with ctypes and
numpy.  Functions:

* :func:`strassen_inv` -- Algorithm 1 of Misra et al. (Sec. 3.1), steps
  I..VII, C11..C22 in the paper's order, leaf inverted directly.
* :func:`gj_inv` -- Gauss-Jordan with partial pivoting on the whole matrix:
  the plain definition of A^-1 (also the leaf method of the above).
* :func:`residual` -- ||AX - I||_F / (||A||_F ||X||_F) with compensated dot
  products (Ogita-Rump-Oishi Dot2).
* :func:`freivalds` -- ||(AX - I) v|| for given probe vectors, O(k n^2).
* :func:`counts` -- operation counters of the last :func:`strassen_inv` call
  (leaves, internal nodes, products, subtractions, scalar multiplications,
  product flops), which pin the recursion against Sec. 4 / Table 2.
* :func:`rbt_inv` -- the random butterfly transform around Algorithm 1 for
  matrices whose leading blocks are singular (dense definition; the
  uniforms are passed in).

Pins (tests under ``tests/test_oracle_*.py``): the 2x2 closed form, exact
rational inverses by Cramer's rule for n <= 6, permutation and power-of-two
diagonal matrices (exact), block-diagonal inputs, 2^k scaling, Householder
matrices of known inverse, numpy/LAPACK inversion, and the operation counts;
for the butterfly transform: the order-2 closed form, |det W| = the product
of its diagonal entries, orthogonality when every entry is 1, LAPACK's
inverse, and a matrix with a singular leading block.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "spin_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libspin_oracle.so")
_lock = threading.Lock()
_lib = None

OK = 0
SINGULAR = 2


class Counts(ctypes.Structure):
    _fields_ = [
        ("leaves", ctypes.c_int64),
        ("internal", ctypes.c_int64),
        ("multiplies", ctypes.c_int64),
        ("subtracts", ctypes.c_int64),
        ("scalar_muls", ctypes.c_int64),
        ("mult_flops", ctypes.c_int64),
        ("leaf_flops", ctypes.c_int64),
        ("max_depth", ctypes.c_int64),
        ("fail_leaf", ctypes.c_int64),
        ("fail_col", ctypes.c_int64),
    ]

    def as_dict(self) -> dict:
        return {name: int(getattr(self, name)) for name, _ in self._fields_}


def build(force: bool = False) -> str:
    """Compile ``spin_oracle.c`` into ``_build/libspin_oracle.so`` (gcc, -O2,
    OpenMP, -ffp-contract=off).  Returns the library path."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp",
           "-ffp-contract=off", "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def bind(path: str):
    """Load an oracle library built from ``spin_oracle.c`` (or a modified copy
    of it, as the mutation tests do) and declare its signatures."""
    lib = ctypes.CDLL(path)
    _declare(lib)
    return lib


def _load(lib=None):
    global _lib
    if lib is not None:
        return lib
    with _lock:
        if _lib is not None:
            return _lib
        _lib = bind(build())
        return _lib


def _declare(lib) -> None:
    if True:  # one block so the declarations read as a table
        i64, dp, vp = ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p
        lib.oracle_strassen_inv.argtypes = [vp, i64, vp, i64, i64, i64]
        lib.oracle_strassen_inv.restype = ctypes.c_int
        lib.oracle_gj_inv.argtypes = [vp, i64, i64, ctypes.POINTER(i64)]
        lib.oracle_gj_inv.restype = ctypes.c_int
        lib.oracle_residual.argtypes = [vp, i64, vp, i64, i64, vp, dp]
        lib.oracle_residual.restype = ctypes.c_double
        lib.oracle_freivalds.argtypes = [vp, i64, vp, i64, i64, vp, i64, vp]
        lib.oracle_freivalds.restype = None
        lib.oracle_rel_diff.argtypes = [vp, i64, vp, i64, i64, i64]
        lib.oracle_rel_diff.restype = ctypes.c_double
        lib.oracle_split.argtypes = [i64]
        lib.oracle_split.restype = i64
        lib.oracle_counts_reset.argtypes = []
        lib.oracle_counts_get.argtypes = [ctypes.POINTER(Counts)]
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]


def _f64(a: np.ndarray) -> np.ndarray:
    a = np.asarray(a, dtype=np.float64)
    if not a.flags.c_contiguous:
        a = np.ascontiguousarray(a)
    return a


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


class SingularError(ArithmeticError):
    """A leaf pivot (or a Schur complement leaf pivot) was zero or non-finite."""


def strassen_inv(A: np.ndarray, leaf: int, *, raise_on_singular: bool = True, lib=None):
    """X = A^-1 by Algorithm 1 (Sec. 3.1) with leaves of order <= ``leaf``.

    Returns ``(X, status)``; raises :class:`SingularError` on a singular leaf
    when ``raise_on_singular``."""
    A = _f64(A)
    n = A.shape[0]
    if A.ndim != 2 or A.shape[1] != n:
        raise ValueError("A must be square")
    X = np.empty_like(A)
    lib = _load(lib)
    lib.oracle_counts_reset()
    st = lib.oracle_strassen_inv(_ptr(A), n, _ptr(X), n, n, int(leaf))
    if st == 1:
        raise ValueError("invalid arguments")
    if st == SINGULAR and raise_on_singular:
        c = counts(lib)
        raise SingularError(f"zero or non-finite pivot in leaf {c['fail_leaf']} column {c['fail_col']}")
    return X, st


def gj_inv(A: np.ndarray, *, raise_on_singular: bool = True, lib=None):
    """X = A^-1 by Gauss-Jordan with partial pivoting (lowest row on ties)."""
    M = _f64(A).copy()
    n = M.shape[0]
    bad = ctypes.c_int64(-1)
    st = _load(lib).oracle_gj_inv(_ptr(M), n, n, ctypes.byref(bad))
    if st == SINGULAR and raise_on_singular:
        raise SingularError(f"zero or non-finite pivot in column {bad.value}")
    return M, st


def residual(A: np.ndarray, X: np.ndarray, *, return_matrix: bool = False, lib=None):
    """Relative residual ||AX - I||_F / (||A||_F ||X||_F), compensated.

    Returns ``(rel, abs)`` or ``(rel, abs, R)`` with ``return_matrix``."""
    A, X = _f64(A), _f64(X)
    n = A.shape[0]
    R = np.empty_like(A) if return_matrix else None
    ab = ctypes.c_double(0.0)
    rel = _load(lib).oracle_residual(_ptr(A), n, _ptr(X), n, n,
                                  _ptr(R) if R is not None else None, ctypes.byref(ab))
    return (rel, ab.value, R) if return_matrix else (rel, ab.value)


def freivalds(A: np.ndarray, X: np.ndarray, V: np.ndarray) -> np.ndarray:
    """For each column v of V (n x k): ||A (X v) - v||_2, compensated."""
    A, X, V = _f64(A), _f64(X), _f64(V)
    if V.ndim == 1:
        V = V[:, None].copy()
    n, k = V.shape
    out = np.empty(k)
    _load().oracle_freivalds(_ptr(A), A.shape[1], _ptr(X), X.shape[1], n, _ptr(V), k, _ptr(out))
    return out


def rel_diff(X: np.ndarray, Y: np.ndarray) -> float:
    """||X - Y||_F / ||Y||_F."""
    X, Y = _f64(X), _f64(Y)
    return _load().oracle_rel_diff(_ptr(X), X.shape[1], _ptr(Y), Y.shape[1], X.shape[0], X.shape[1])


# ------------------------------------------------ random butterfly transform --
#
# The recursion (Algorithm 1) does not pivot across blocks; a matrix whose
# leading block or Schur complement is singular breaks it.  The random
# butterfly transform of Parker (1995), recursive form of Baboulin, Dongarra,
# Herrmann and Tomov (2013): a butterfly of order m (h = m/2) is
# B = [[R, S], [R, -S]] / sqrt(2) with R, S random diagonal h x h matrices;
# the recursive butterfly of depth d is W = L_d ... L_1 where level k is
# block diagonal with 2^(k-1) butterflies of order n / 2^(k-1); with U, V two
# such matrices, A^-1 = V (U^T A V)^-1 U^T.  Diagonal entries exp(rho/10),
# rho = u - 1/2 for uniforms u passed in (the caller draws them).
# Everything below is the definition written out with dense matrices.

def rbt_padded_order(n: int, depth: int = 2) -> int:
    q = 2 ** depth
    return -(-n // q) * q


def rbt_butterfly(diag_levels: np.ndarray) -> np.ndarray:
    """W = L_d ... L_1 from the level diagonals (d x np): level k (1-based,
    row k-1) has blocks of order m = np / 2^(k-1), block j using R =
    diag[j*m : j*m+h] and S = diag[j*m+h : (j+1)*m]."""
    d, np_ = diag_levels.shape
    W = np.eye(np_)
    c = 1.0 / math.sqrt(2.0)
    for k in range(1, d + 1):
        m = np_ >> (k - 1)
        h = m // 2
        L = np.zeros((np_, np_))
        for j in range(np_ // m):
            b = j * m
            for i in range(h):
                r, s_ = diag_levels[k - 1, b + i], diag_levels[k - 1, b + h + i]
                L[b + i, b + i] = r * c
                L[b + i, b + h + i] = s_ * c
                L[b + h + i, b + i] = r * c
                L[b + h + i, b + h + i] = -s_ * c
        W = L @ W
    return W


def rbt_inv(A: np.ndarray, leaf: int, u: np.ndarray, depth: int = 2):
    """A^-1 = V (U^T pad(A) V)^-1 U^T, cropped to n x n, the middle inverse by
    Algorithm 1 (:func:`strassen_inv`).  ``u``: 2 * depth * np uniforms in
    [0, 1) (U's levels, then V's).  Returns (X, status, U, V)."""
    A = _f64(A)
    n = A.shape[0]
    np_ = rbt_padded_order(n, depth)
    diag = np.exp((np.asarray(u, dtype=np.float64).reshape(2, depth, np_) - 0.5) / 10.0)
    U = rbt_butterfly(diag[0])
    V = rbt_butterfly(diag[1])
    Ap = np.eye(np_)
    Ap[:n, :n] = A
    Ar = U.T @ Ap @ V
    Y, st = strassen_inv(Ar, leaf)
    X = V @ Y @ U.T
    return X[:n, :n].copy(), st, U, V


def split(n: int) -> int:
    """Order n1 of the leading block when an n x n block is split."""
    return int(_load().oracle_split(int(n)))


def counts(lib=None) -> dict:
    c = Counts()
    _load(lib).oracle_counts_get(ctypes.byref(c))
    return c.as_dict()


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))
