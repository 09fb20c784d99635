"""Seeded synthetic inputs shared by the CUDA path's tests, the benchmark and
the oracle checks.

This module holds no step of the inversion method: it only draws matrices.
Every draw is a pure function of (seed, position) through splitmix64
(Steele, Lea, Flood, "Fast splittable pseudorandom number generators",
OOPSLA 2014; the finaliser constants are the published ones), so the same
bytes come out on any machine and any device.

Workloads (the paper draws its test matrices with java.util.Random and an
unstated distribution, n = 16 ... 16384, Sec. 5.1; these seeded families
stand in for them):

* :func:`sdd` -- a_ij ~ U(-1, 1), a_ii += n: strictly diagonally dominant,
  so every leading block and every Schur complement is nonsingular.
* :func:`spd_gram` -- A = G G^T / n + alpha I with g_ij ~ N(0, 1):
  symmetric positive definite, eigenvalues in about [alpha, 4 + alpha].
* :func:`householder_spd` -- A = Q diag(d) Q^T with Q the product of
  ``reflectors`` seeded Householder reflectors and d log-uniform in
  [1, cond]; its inverse is known in closed form (:func:`householder_apply`).
* :func:`batch_orders`, :func:`serve_trace` -- order mixes for many-matrix
  workloads (log-uniform orders; Poisson arrivals).
"""
from __future__ import annotations

import math

import numpy as np

try:  # torch is optional here: only the large on-device draws need it
    import torch
except Exception:  # pragma: no cover
    torch = None

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_TWO53 = 2.0 ** -53

SEED_BASE = 0x5EED0000


def splitmix64(seed: int, counters: np.ndarray) -> np.ndarray:
    """The (c+1)-th splitmix64 output of a generator started at ``seed``,
    for every counter c (uint64 array)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + (counters.astype(np.uint64) + np.uint64(1)) * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, counters: np.ndarray) -> np.ndarray:
    """53-bit uniform doubles in [0, 1)."""
    return (splitmix64(seed, counters) >> np.uint64(11)).astype(np.float64) * _TWO53


def uniform(seed: int, shape, lo: float = -1.0, hi: float = 1.0, offset: int = 0) -> np.ndarray:
    cnt = np.arange(offset, offset + int(np.prod(shape)), dtype=np.uint64)
    return (lo + (hi - lo) * uniform01(seed, cnt)).reshape(shape)


def normal(seed: int, shape, offset: int = 0) -> np.ndarray:
    """N(0, 1) by Box-Muller on consecutive counter pairs (2c, 2c+1)."""
    m = int(np.prod(shape))
    c = np.arange(offset, offset + m, dtype=np.uint64) * np.uint64(2)
    u1 = uniform01(seed, c)
    u2 = uniform01(seed, c + np.uint64(1))
    r = np.sqrt(-2.0 * np.log1p(-u1))
    return (r * np.cos(2.0 * math.pi * u2)).reshape(shape)


# --------------------------------------------------------------------------
# matrix families
# --------------------------------------------------------------------------

def sdd(n: int, seed: int = SEED_BASE) -> np.ndarray:
    """a_ij ~ U(-1,1) from the seed, then n added to every diagonal entry."""
    A = uniform(seed, (n, n))
    A[np.diag_indices(n)] += float(n)
    return A


def spd_gram(n: int, seed: int = SEED_BASE + 1, alpha: float = 1.0) -> np.ndarray:
    """A = G G^T / n + alpha I (FP64 on the host), symmetrised exactly."""
    G = normal(seed, (n, n))
    A = (G @ G.T) / float(n)
    A = 0.5 * (A + A.T)
    A[np.diag_indices(n)] += alpha
    return A


# ---- the same counter-based draws with torch (any device, same bits) ----

def _i64(c: int) -> int:
    """A uint64 constant as the int64 with the same bits."""
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(z, s: int):
    """Logical right shift of int64 tensors (torch's >> is arithmetic)."""
    return (z >> s) & ((1 << (64 - s)) - 1)


def splitmix64_torch(seed: int, counters):
    """Same as :func:`splitmix64` on an int64 torch tensor of counters
    (int64 arithmetic wraps modulo 2^64, so the bits agree)."""
    z = counters + 1
    z = z * _i64(0x9E3779B97F4A7C15) + _i64(seed & 0xFFFFFFFFFFFFFFFF)
    z = (z ^ _srl(z, 30)) * _i64(0xBF58476D1CE4E5B9)
    z = (z ^ _srl(z, 27)) * _i64(0x94D049BB133111EB)
    return z ^ _srl(z, 31)


def uniform01_torch(seed: int, counters):
    return _srl(splitmix64_torch(seed, counters), 11).to(torch.float64) * _TWO53


def normal_torch(seed: int, rows: int, cols: int, row0: int, device, dtype=None):
    """N(0,1) block of rows [row0, row0+rows) of an n x cols matrix drawn as
    :func:`normal` draws it (Box-Muller on counters 2c, 2c+1, c = i*cols+j).
    The transcendental functions are torch's, so values may differ from the
    numpy draw in the last bits; the device inputs are only ever drawn here."""
    c = torch.arange(row0 * cols, (row0 + rows) * cols, dtype=torch.int64, device=device) * 2
    u1 = uniform01_torch(seed, c)
    u2 = uniform01_torch(seed, c + 1)
    g = torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)
    g = g.reshape(rows, cols)
    return g if dtype is None else g.to(dtype)


def sdd_device(n: int, seed: int, device):
    """:func:`sdd` drawn on the device (bit-identical to the host draw)."""
    A = torch.empty((n, n), dtype=torch.float64, device=device)
    step = max(1, (1 << 24) // max(n, 1))
    for r0 in range(0, n, step):
        r1 = min(n, r0 + step)
        c = torch.arange(r0 * n, r1 * n, dtype=torch.int64, device=device)
        A[r0:r1] = (-1.0 + 2.0 * uniform01_torch(seed, c)).reshape(r1 - r0, n)
    A.diagonal().add_(float(n))
    return A


def spd_gram_device(n: int, seed: int, device, alpha: float = 1.0, chunk_rows: int = 2048):
    """Large-n form of :func:`spd_gram`: G is drawn on the device, the
    product G G^T is formed there with torch in FP32 (input preparation only;
    the inversion never runs here), symmetrised, shifted by alpha I and
    stored as FP64.  The returned device tensor is the input; host-side
    checks read its bytes back rather than recomputing it."""
    if torch is None:
        raise RuntimeError("torch is required for device-side input generation")
    G = torch.empty((n, n), dtype=torch.float32, device=device)
    for r0 in range(0, n, chunk_rows):
        r1 = min(n, r0 + chunk_rows)
        G[r0:r1] = normal_torch(seed, r1 - r0, n, r0, device, torch.float32)
    prev = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        A = torch.empty((n, n), dtype=torch.float64, device=device)
        for r0 in range(0, n, chunk_rows):
            r1 = min(n, r0 + chunk_rows)
            A[r0:r1] = (G[r0:r1] @ G.T).double() / float(n)
    finally:
        torch.backends.cuda.matmul.allow_tf32 = prev
    del G
    for r0 in range(0, n, chunk_rows):  # symmetrise block by block
        r1 = min(n, r0 + chunk_rows)
        for c0 in range(r0, n, chunk_rows):
            c1 = min(n, c0 + chunk_rows)
            blk = 0.5 * (A[r0:r1, c0:c1] + A[c0:c1, r0:r1].T)
            A[r0:r1, c0:c1] = blk
            A[c0:c1, r0:r1] = blk.T
    A.diagonal().add_(alpha)
    return A


def householder_vectors(n: int, reflectors: int, seed: int) -> np.ndarray:
    """The ``reflectors`` x n matrix whose rows are the unnormalised
    Householder vectors v (N(0,1) entries)."""
    return normal(seed, (reflectors, n))


def log_uniform(seed: int, m: int, lo: float, hi: float, offset: int = 0) -> np.ndarray:
    u = uniform01(seed, np.arange(offset, offset + m, dtype=np.uint64))
    return np.exp(math.log(lo) + (math.log(hi) - math.log(lo)) * u)


def householder_spd(n: int, seed: int = SEED_BASE + 2, reflectors: int = 64, cond: float = 1e3):
    """A = Q diag(d) Q^T, Q = H_1 H_2 ... H_r, H = I - 2 v v^T / (v^T v),
    d log-uniform in [1, cond].  Returns (A, V, d) so that the inverse
    Q diag(1/d) Q^T can be applied with :func:`householder_apply`."""
    V = householder_vectors(n, reflectors, seed)
    d = log_uniform(seed ^ 0xD1A6, n, 1.0, cond)
    M = np.diag(d)
    for t in range(reflectors - 1, -1, -1):  # innermost reflector first
        v = V[t]
        beta = 2.0 / float(v @ v)
        w = M @ v
        M = M - beta * np.outer(v, v @ M) - beta * np.outer(w, v) + (beta * beta * float(v @ w)) * np.outer(v, v)
    M = 0.5 * (M + M.T)
    return M, V, d


def householder_apply(V: np.ndarray, dvals: np.ndarray, Y: np.ndarray) -> np.ndarray:
    """Q diag(dvals) Q^T Y for the Q of :func:`householder_spd` (Y: n or n x k)."""
    Z = np.array(Y, dtype=np.float64, copy=True)
    vec = Z.ndim == 1
    if vec:
        Z = Z[:, None]
    for t in range(V.shape[0]):  # Q^T = H_r ... H_1: apply H_1 first
        v = V[t]
        Z = Z - np.outer(v, (2.0 / float(v @ v)) * (v @ Z))
    Z = dvals[:, None] * Z
    for t in range(V.shape[0] - 1, -1, -1):  # Q = H_1 ... H_r: apply H_r first
        v = V[t]
        Z = Z - np.outer(v, (2.0 / float(v @ v)) * (v @ Z))
    return Z[:, 0] if vec else Z


def householder_spd_device(n: int, seed: int, device, reflectors: int = 64, cond: float = 1e3):
    """Large-n form of :func:`householder_spd`, built on the device with
    torch in FP64 by rank-2 updates (O(reflectors n^2)); returns (A, V, d)
    with V and d on the host."""
    if torch is None:
        raise RuntimeError("torch is required for device-side input generation")
    V = householder_vectors(n, reflectors, seed)
    d = log_uniform(seed ^ 0xD1A6, n, 1.0, cond)
    A = torch.diag(torch.from_numpy(d).to(device))
    for t in range(reflectors - 1, -1, -1):
        v = torch.from_numpy(V[t]).to(device)
        beta = 2.0 / float(V[t] @ V[t])
        w = A @ v
        u = v @ A
        s = beta * beta * float(v @ w)
        A.addr_(v, u, alpha=-beta)
        A.addr_(w, v, alpha=-beta)
        A.addr_(v, v, alpha=s)
    A = 0.5 * (A + A.T)
    return A.contiguous(), V, d


def batch_orders(count: int, seed: int, lo: int = 32, hi: int = 1024, multiple: int = 32) -> np.ndarray:
    """Orders log-uniform in [lo, hi], rounded to a multiple of ``multiple``."""
    x = log_uniform(seed, count, lo, hi)
    return np.clip(np.rint(x / multiple).astype(np.int64) * multiple, lo, hi)


def serve_trace(seed: int, rate: float, duration: float, lo: int = 64, hi: int = 8192):
    """Poisson arrivals at ``rate``/s for ``duration`` s.  Returns a list of
    (t_arrival, n, alpha, mixed) with n log-uniform in [lo, hi], alpha
    uniform in [0.1, 1] and mixed alternating False/True."""
    out = []
    t = 0.0
    j = 0
    while True:
        u = float(uniform01(seed, np.array([3 * j], dtype=np.uint64))[0])
        t += -math.log1p(-u) / rate
        if t >= duration:
            break
        n = int(round(float(log_uniform(seed, 1, lo, hi, offset=3 * j + 1)[0])))
        a = 0.1 + 0.9 * float(uniform01(seed, np.array([3 * j + 2], dtype=np.uint64))[0])
        out.append((t, n, a, bool(j % 2)))
        j += 1
    return out


def probes(n: int, k: int, seed: int = SEED_BASE + 77) -> np.ndarray:
    """n x k probe vectors with U(-1,1) entries (Freivalds checks)."""
    return uniform(seed, (n, k))
