"""Tensor-core (tcgen05) level products of the mixed method, through the C ABI.

Exact mode is checked bit for bit: on integer operands whose digits the
slices hold exactly, every digit product, every FP32 run and every int32
sum is exact, so D must equal the integer product A @ B exactly (compared in
int64).  FP64 inputs are checked against correctly rounded dot products
(math.fsum of error-free products) on sampled entries.  The bf16x3 form is
checked against the FP64 product with the bound of its error model:
|D - AB|_ij <= (2^-14 + k 2^-23) (|A||B|)_ij (dropped lo*lo terms and the
hi/lo representation error, plus FP32 accumulation).
"""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def spin():
    import paper_1801_04723_gb300 as s

    s.build()
    s.lib()
    return s


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A, dtype=np.float64)).to("cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def int_case(m, n, k, lim, seed):
    rng = np.random.default_rng(seed)
    A = rng.integers(-lim, lim + 1, size=(m, k)).astype(np.int64)
    B = rng.integers(-lim, lim + 1, size=(k, n)).astype(np.int64)
    return A, B


def test_ozaki_single_tile_exact(spin):
    A, B = int_case(128, 128, 64, 100, 1)
    D = host(spin.gemm_ozaki(dev(A), dev(B), slices=2))
    assert spin.take_device_error() == 0
    np.testing.assert_array_equal(D.astype(np.int64), A @ B)


@pytest.mark.parametrize("m,n,k,slices", [(300, 200, 1000, 3), (129, 257, 65, 2), (1, 1, 1, 1), (513, 130, 700, 4)])
def test_ozaki_ragged_exact(spin, m, n, k, slices):
    A, B = int_case(m, n, k, 120, m + n + k)
    C = np.random.default_rng(0).integers(-50, 50, size=(m, n)).astype(np.int64)
    D = host(spin.gemm_ozaki(dev(A), dev(B), slices=slices, alpha=-1.0, beta=1.0, C=dev(C), add_identity=True))
    assert spin.take_device_error() == 0
    want = C - A @ B
    want[np.arange(min(m, n)), np.arange(min(m, n))] += 1
    np.testing.assert_array_equal(D.astype(np.int64), want)


def test_ozaki_long_k_flushes_exact(spin):
    # runs of 1024: 49 per slice pair, 147 in the group t + u = 2, which
    # crosses the int32 flush limit (96 runs) once
    A, B = int_case(128, 128, 50000, 1000, 7)
    D = host(spin.gemm_ozaki(dev(A), dev(B), slices=3))
    assert spin.take_device_error() == 0
    np.testing.assert_array_equal(D.astype(np.int64), A @ B)


def exact_dot(a, b):
    """Correctly rounded sum of a_k b_k: Dekker two-product, then fsum."""
    terms = []
    for x, y in zip(a.tolist(), b.tolist()):
        p = x * y
        # error of the product via splitting (no FMA in Python floats)
        f = 134217729.0
        c = f * x; xh = c - (c - x); xl = x - xh
        c = f * y; yh = c - (c - y); yl = y - yh
        e = ((xh * yh - p) + xh * yl + xl * yh) + xl * yl
        terms += [p, e]
    return math.fsum(terms)


@pytest.mark.parametrize("slices,bound", [(7, 2.0 ** -50), (6, 2.0 ** -42), (5, 2.0 ** -34)])
def test_ozaki_fp64_class(spin, slices, bound):
    rng = np.random.default_rng(slices)
    m, n, k = 400, 300, 1500
    A = rng.uniform(-1, 1, (m, k)) * np.exp(rng.uniform(-3, 3, (m, 1)))  # rows of different scales
    B = rng.standard_normal((k, n))
    D = host(spin.gemm_ozaki(dev(A), dev(B), slices=slices))
    assert spin.take_device_error() == 0
    absAB = np.abs(A) @ np.abs(B)
    idx = rng.integers(0, m * n, size=150)
    for t in idx:
        i, j = divmod(int(t), n)
        ex = exact_dot(A[i], B[:, j])
        assert abs(D[i, j] - ex) <= bound * absAB[i, j] + 1e-300


@pytest.mark.parametrize("m,n,k", [(128, 256, 64), (700, 500, 1200), (33, 1000, 17), (1024, 1024, 1024)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 1.0)])
def test_bf16x3_error_model(spin, m, n, k, alpha, beta):
    rng = np.random.default_rng(m + n + k)
    A = rng.uniform(-1, 1, (m, k))
    B = rng.uniform(-1, 1, (k, n))
    C = rng.uniform(-1, 1, (m, n))
    D = host(spin.gemm_bf16x3(dev(A), dev(B), alpha=alpha, beta=beta, C=dev(C) if beta else None))
    assert spin.take_device_error() == 0
    want = alpha * (A @ B) + (beta * C if beta else 0.0)
    bound = (2.0 ** -14 + k * 2.0 ** -23) * (np.abs(A) @ np.abs(B)) + 1e-15 * np.abs(C)
    assert np.all(np.abs(D - want) <= bound)
    # and it is far better than plain BF16 would be on average
    assert np.sqrt(np.mean((D - want) ** 2)) < 2.0 ** -12 * np.sqrt(np.mean(want ** 2))


def test_bf16x3_in_place_strided(spin):
    rng = np.random.default_rng(3)
    big = dev(rng.uniform(-1, 1, (600, 700)))
    A = big[0:200, 0:300]
    B = big[200:500, 100:356]
    D = big[500:600, 400:656][:100]
    C0 = host(D).copy()
    Ah, Bh = host(A)[:100], host(B)
    spin.gemm_bf16x3(A[:100], B, alpha=-1.0, beta=1.0, C=D, out=D)
    got = host(D)
    want = C0 - Ah @ Bh
    assert np.max(np.abs(got - want)) < (2.0 ** -14 + 300 * 2.0 ** -23) * np.max(np.abs(Ah) @ np.abs(Bh))


PAIR_SCRIPT = r"""
import numpy as np, torch
import paper_1801_04723_gb300 as s
s.lib()
for (m, n, k, sl, seed) in [(300, 200, 1000, 3, 1), (513, 130, 700, 4, 2), (256, 128, 50000, 3, 3), (1, 1, 1, 1, 4)]:
    rng = np.random.default_rng(seed)
    lim = 1000 if k > 10000 else 120
    A = rng.integers(-lim, lim + 1, size=(m, k)).astype(np.int64)
    B = rng.integers(-lim, lim + 1, size=(k, n)).astype(np.int64)
    C = rng.integers(-50, 50, size=(m, n)).astype(np.int64)
    d = lambda X: torch.from_numpy(X.astype(np.float64)).to("cuda:0")
    D = s.gemm_ozaki(d(A), d(B), slices=sl, alpha=-1.0, beta=1.0, C=d(C))
    torch.cuda.synchronize()
    assert s.take_device_error() == 0
    assert (D.cpu().numpy().astype(np.int64) == C - A @ B).all(), (m, n, k, sl)
print("PAIR-OK")
"""


def test_pair_kernel_exact():
    """The CTA-pair form of the exact kernel (SPIN_TC_PAIR=1, read once per
    process) gives the same exact integer products, ragged and long-K."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SPIN_TC_PAIR="1")
    r = subprocess.run([sys.executable, "-c", PAIR_SCRIPT], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "PAIR-OK" in r.stdout, r.stdout + r.stderr


def test_ozaki_wide_tiles_exact(spin):
    # enough 128 x 256 tiles (20 x 32 = 640) for the wide exact kernel, whose
    # running sums go through D; ragged K, beta C and the identity
    m, n, k = 2560, 8192, 200
    rng = np.random.default_rng(5)
    A = rng.integers(-120, 121, size=(m, k)).astype(np.float64)
    B = rng.integers(-120, 121, size=(k, n)).astype(np.float64)
    C = rng.integers(-50, 50, size=(m, n)).astype(np.float64)
    D = host(spin.gemm_ozaki(dev(A), dev(B), slices=3, alpha=-1.0, beta=1.0, C=dev(C), add_identity=True))
    assert spin.take_device_error() == 0
    want = C - A @ B  # integers below 2^22: exact in FP64
    want[np.arange(m), np.arange(m)] += 1
    np.testing.assert_array_equal(D, want)
