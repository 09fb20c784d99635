"""Parity of the CUDA plain (FP64) path with the CPU oracle.

Every case runs the library through the C ABI on seeded synthetic inputs and
compares element by element with the oracle on the same bytes.

Tolerance.  Both sides compute in FP64 and differ only in summation order
and FMA contraction (the oracle never contracts).  For an inversion with
condition number kappa a perturbation of relative size ~u per operation
moves the result by ~c * n * kappa * u in relative norm; the tests use
    ||X_gpu - X_oracle||_F / ||X_oracle||_F <= 64 * n * kappa * u,  u = 2^-53
(about 1e-11 at n = 1024, kappa = 1.5); element by element (tests/bounds.py)
    |X_gpu - X_oracle|_ij <= 4 n u (|X_oracle| |A| |X_oracle|)_ij,
so that an error confined to one small block cannot hide under the norm;
and on top of both the method's own target: relative residual
||AX - I||_F / (||A||_F ||X||_F) <= 1e-13, measured by the oracle's
compensated residual.  Results that are exact in
floating point (permutations, power-of-two diagonals, block-diagonal and
2^k-scaled inputs) are compared bit for bit.
"""
import numpy as np
import pytest

import bounds
import oracle
from paper_1801_04723_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

U = 2.0 ** -53


@pytest.fixture(scope="module")
def spin():
    import paper_1801_04723_gb300 as s

    s.build()
    s.lib()
    return s


def dev(A):
    return torch.from_numpy(np.ascontiguousarray(A)).to("cuda:0")


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def tol(A):
    n = A.shape[0]
    return 64 * n * np.linalg.cond(A) * U


def rel(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


# ------------------------------------------------------------------ GEMM --

@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 64), (100, 37, 250), (513, 129, 1000), (7, 300, 65)])
@pytest.mark.parametrize("alpha,beta", [(1.0, 0.0), (-1.0, 0.0), (-1.0, 1.0), (1.0, 1.0)])
def test_gemm_f64(spin, m, n, k, alpha, beta):
    rng = np.random.default_rng(m * 1000 + n + k)
    A = rng.uniform(-1, 1, (m, k))
    B = rng.uniform(-1, 1, (k, n))
    C = rng.uniform(-1, 1, (m, n))
    D = host(spin.gemm_f64(dev(A), dev(B), alpha=alpha, beta=beta, C=dev(C) if beta else None))
    want = alpha * (A @ B) + (beta * C if beta else 0.0)
    bound = 4 * (k + 2) * U * (np.abs(A) @ np.abs(B) + np.abs(C))
    assert np.all(np.abs(D - want) <= bound)


def test_gemm_f64_in_place_and_strided(spin):
    rng = np.random.default_rng(5)
    big = dev(rng.uniform(-1, 1, (300, 400)))
    A = big[10:110, 20:220]   # 100 x 200, lda 400
    B = big[50:250, 1:81]     # 200 x 80
    Cref = host(big[200:300, 300:380]).copy()
    D = big[200:300, 300:380]  # in place: D = C - A B
    spin.gemm_f64(A, B, alpha=-1.0, beta=1.0, C=D, out=D)
    got = host(D)
    want = Cref - host(A) @ host(B)
    assert np.max(np.abs(got - want)) < 1e-13


def test_fp64_probes(spin):
    """Both FP64 forms of this GPU measured live: the DFMA probe (the plain
    path's roofline denominator) and the DMMA (mma.sync f64) probe."""
    dfma = spin.probe_fp64_peak()
    dmma = spin.probe_fp64_mma_peak()
    assert 0.3 < dfma < 100.0 and 0.3 < dmma < 100.0


# ------------------------------------------------------------- leaf (GJ) --

@pytest.mark.parametrize("L", [1, 2, 3, 5, 31, 32, 33, 64, 96, 100, 128, 200, 256, 300, 512, 513, 700, 1024])
def test_leaf_gj_matches_oracle(spin, L):
    rng = np.random.default_rng(L)
    A = rng.uniform(-1, 1, (L, L))  # no diagonal dominance: partial pivoting is exercised
    X = host(spin.leaf_inverse(dev(A)))
    G, st = oracle.gj_inv(A)
    assert st == 0
    assert rel(X, G) <= tol(A)
    assert oracle.residual(A, X)[0] < 1e-13


@pytest.mark.parametrize("L", [1, 2, 17, 64, 128, 200, 512, 600])
def test_leaf_permutation_exact(spin, L):
    P = np.eye(L)[np.random.default_rng(L).permutation(L)]
    X = host(spin.leaf_inverse(dev(P)))
    np.testing.assert_array_equal(X, P.T)


@pytest.mark.parametrize("L", [8, 100, 512])
def test_leaf_power_of_two_diagonal_exact(spin, L):
    rng = np.random.default_rng(L)
    d = 2.0 ** rng.integers(-30, 30, size=L) * np.where(rng.random(L) < 0.5, -1.0, 1.0)
    X = host(spin.leaf_inverse(dev(np.diag(d))))
    np.testing.assert_array_equal(X, np.diag(1.0 / d))


@pytest.mark.parametrize("L", [16, 33, 64, 100, 256])
def test_leaf_concurrent_streams_deterministic(spin, L):
    """Many leaves on eight streams at once (wide clusters, few rows per CTA:
    the fastest CTA of a cluster runs ahead of the slowest by up to one
    step): every result must equal the first bit for bit, and the oracle's
    Gauss-Jordan to rounding."""
    A = np.random.default_rng(100 + L).uniform(-1, 1, (L, L))
    Ad = dev(A)
    torch.cuda.synchronize()
    streams = [torch.cuda.Stream() for _ in range(8)]
    outs = []
    for i in range(96):
        st = streams[i % 8]
        with torch.cuda.stream(st):
            outs.append(spin.leaf_inverse(Ad, stream=st))
    torch.cuda.synchronize()
    first = outs[0].cpu().numpy()
    for o in outs[1:]:
        np.testing.assert_array_equal(o.cpu().numpy(), first)
    G, st = oracle.gj_inv(A)
    assert st == 0 and rel(first, G) <= tol(A)


@pytest.mark.parametrize("L,mute", [(128, 0), (128, 7), (64, 15), (200, 3)])
def test_leaf_exchange_timeout(spin, L, mute):
    """A CTA of a pushed-row leaf that sends nothing: the other CTAs' bounded
    waits (50 ms here) run out, every CTA leaves without a fault or a hang,
    the status is SPIN_ERR_TIMEOUT, and the context stays usable (a leaf run
    right after is right)."""
    assert spin.leaf_exchange_timeout(L, mute, 50.0) == 6
    A = np.random.default_rng(L).uniform(-1, 1, (L, L))
    X = host(spin.leaf_inverse(dev(A)))
    assert oracle.residual(A, X)[0] < 1e-13


def test_leaf_singular_reports_column(spin):
    # a zero column c stays exactly zero under row operations, so the pivot
    # search fails exactly at step c (the oracle agrees)
    A = np.random.default_rng(1).uniform(-1, 1, (40, 40))
    A[:, 17] = 0.0
    info = torch.zeros(4, dtype=torch.int32, device="cuda:0")
    spin.leaf_inverse(dev(A), info_dev=info)
    st, leaf, col, _ = host(info).tolist()
    assert (st, leaf, col) == (2, 0, 17)
    with pytest.raises(oracle.SingularError, match="column 17"):
        oracle.gj_inv(A)


# ------------------------------------------------------- full inversion --

def test_config0_n1024_leaf128(spin):
    """Plain method, one FP64 matrix n = 1024 (U(-1,1) + n on the diagonal),
    leaf 128: three recursion levels."""
    A = inputs.sdd(1024, seed=inputs.SEED_BASE)
    X, info = spin.invert(dev(A), leaf=128)
    X = host(X)
    ref, _ = oracle.strassen_inv(A, 128)
    assert info["status"] == 0
    assert rel(X, ref) <= tol(A)
    assert np.max(np.abs(X - ref)) <= 64 * 1024 * U * np.max(np.abs(ref))
    assert bounds.elementwise_ok(X, ref, A)
    assert oracle.residual(A, X)[0] <= 1e-13


@pytest.mark.parametrize("n,leaf", [(1, 1), (2, 1), (3, 1), (5, 2), (65, 8), (96, 32), (100, 16), (257, 64),
                                    (777, 100), (1000, 128), (1500, 512), (2048, 1024), (1100, 600)])
@pytest.mark.parametrize("family", ["sdd", "spd"])
def test_invert_ragged(spin, n, leaf, family):
    A = inputs.sdd(n, seed=11 + n) if family == "sdd" else inputs.spd_gram(n, seed=13 + n)
    X, info = spin.invert(dev(A), leaf=leaf)
    X = host(X)
    ref, _ = oracle.strassen_inv(A, leaf)
    assert info["status"] == 0
    assert rel(X, ref) <= tol(A)
    assert bounds.elementwise_ok(X, ref, A)
    assert oracle.residual(A, X)[0] <= 1e-13


@pytest.mark.parametrize("leaf", [0, 32, 64, 256])
def test_leaf_choice_changes_rounding_only(spin, leaf):
    A = inputs.spd_gram(512, seed=21)
    X, _ = spin.invert(dev(A), leaf=leaf)
    assert rel(host(X), np.linalg.inv(A)) < 1e-12


def test_singular_leading_block(spin):
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    X, info = spin.invert(dev(A), leaf=1, check=False)
    assert info["status"] == 2 and info["fail_leaf"] == 0 and info["fail_col"] == 0
    X, info = spin.invert(dev(A), leaf=2)
    np.testing.assert_array_equal(host(X), A)


def test_singular_schur_complement(spin):
    A = np.array([[1.0, 1.0], [1.0, 1.0]])
    _, info = spin.invert(dev(A), leaf=1, check=False)
    assert info["status"] == 2 and info["fail_leaf"] == 1


def test_singular_deep_leaf_index_matches_oracle(spin):
    # order 64, leaf 16: inside A11 (order 32) the blocks are [[I, B], [I, B]]
    # with B integer, so its Schur complement B - I I^-1 B is exactly zero and
    # the second leaf (index 1) fails at its first column on both sides
    A = inputs.sdd(64, seed=3)
    B = np.random.default_rng(2).integers(-3, 4, size=(16, 16)).astype(float)
    A[:32, :32] = np.block([[np.eye(16), B], [np.eye(16), B]])
    _, info = spin.invert(dev(A), leaf=16, check=False)
    _, st = oracle.strassen_inv(A, 16, raise_on_singular=False)
    c = oracle.counts()
    assert st == 2 and info["status"] == 2
    assert info["fail_leaf"] == c["fail_leaf"] == 1
    assert info["fail_col"] == c["fail_col"] == 0


@pytest.mark.parametrize("n,leaf", [(128, 32), (96, 64), (300, 64)])
def test_block_diagonal_bitwise(spin, n, leaf):
    n1 = oracle.split(n)
    A = inputs.sdd(n, seed=42)
    A[:n1, n1:] = 0.0
    A[n1:, :n1] = 0.0
    X = host(spin.invert(dev(A), leaf=leaf)[0])
    np.testing.assert_array_equal(X[:n1, n1:], 0.0)
    np.testing.assert_array_equal(X[n1:, :n1], 0.0)
    np.testing.assert_array_equal(X[:n1, :n1], host(spin.invert(dev(A[:n1, :n1]), leaf=leaf)[0]))
    np.testing.assert_array_equal(X[n1:, n1:], host(spin.invert(dev(A[n1:, n1:]), leaf=leaf)[0]))


@pytest.mark.parametrize("k", [-9, 5])
def test_power_of_two_scaling_bitwise(spin, k):
    A = inputs.sdd(300, seed=8)
    X = host(spin.invert(dev(A), leaf=64)[0])
    Xs = host(spin.invert(dev(A * 2.0 ** k), leaf=64)[0])
    np.testing.assert_array_equal(Xs, X * 2.0 ** -k)


def test_deterministic(spin):
    A = dev(inputs.spd_gram(700, seed=99))
    X1 = host(spin.invert(A, leaf=100)[0])
    X2 = host(spin.invert(A, leaf=100)[0])
    np.testing.assert_array_equal(X1, X2)


def test_leading_dimensions_and_transpose(spin):
    A = inputs.sdd(257, seed=4)
    big = torch.zeros((300, 320), dtype=torch.float64, device="cuda:0")
    big[5:262, 7:264] = dev(A)
    Aview = big[5:262, 7:264]
    outbig = torch.full((400, 290), 7.0, dtype=torch.float64, device="cuda:0")
    Xview = outbig[3:260, 11:268]
    spin.invert(Aview, leaf=64, out=Xview)
    X = host(Xview)
    ref, _ = oracle.strassen_inv(A, 64)
    assert rel(X, ref) <= tol(A)
    assert bounds.elementwise_ok(X, ref, A)
    # the frame around the output view is untouched
    ob = host(outbig)
    assert np.all(ob[:3] == 7.0) and np.all(ob[260:] == 7.0) and np.all(ob[:, :11] == 7.0)
    # column-major reading: inv(A^T) = inv(A)^T
    XT = host(spin.invert(dev(A.T.copy()), leaf=64)[0])
    assert rel(XT.T, ref) <= tol(A)


def test_host_buffers_and_caller_workspace(spin):
    A = inputs.sdd(600, seed=12)
    Xh, info = spin.invert_host(A, leaf=128)
    ref, _ = oracle.strassen_inv(A, 128)
    assert rel(Xh, ref) <= tol(A)
    assert bounds.elementwise_ok(Xh, ref, A)
    ws = torch.empty(spin.workspace_bytes(600, leaf=128) // 8 + 1, dtype=torch.float64, device="cuda:0")
    Xd = host(spin.invert(dev(A), leaf=128, workspace=ws)[0])
    np.testing.assert_array_equal(Xd, Xh)


def test_householder_known_inverse(spin):
    A, V, d = inputs.householder_spd(1024, seed=inputs.SEED_BASE + 2, reflectors=64, cond=1e3)
    X = host(spin.invert(dev(A), leaf=128)[0])
    ref = inputs.householder_apply(V, 1.0 / d, np.eye(1024))
    assert rel(X, ref) < 1e-11
    assert oracle.residual(A, X)[0] <= 1e-13


def test_autotune_leaf_records_choice(spin):
    best, ms = spin.autotune_leaf(1024, "fp64", candidates=(64, 128, 256, 2048))
    assert best in (64, 128, 256) and set(ms) == {64, 128, 256}  # 2048 >= n is skipped
    assert best == min(ms, key=ms.get)
    assert spin.default_leaf(1024) == best
    assert spin.default_leaf(1500) == best  # a larger size class reuses the largest tuned one
    A = inputs.sdd(1024, seed=77)
    X, info = spin.invert(dev(A))  # leaf 0 -> the tuned leaf
    ref, _ = oracle.strassen_inv(A, best)
    assert rel(host(X), ref) <= tol(A)


def test_cost_model_against_measured_sweep(spin):
    """The cost model's leaf choice for n = 4096 is within 5 % of the fastest
    measured leaf, and its times within 25 % of the measured ones (the model
    was calibrated on n = 8192 and the leaf microbenchmark, not on this)."""
    n = 4096
    cands = (128, 256, 512, 1024)
    best, ms = spin.autotune_leaf(n, "fp64", candidates=cands)
    pick = min(cands, key=lambda L: spin.model_seconds(n, L))
    assert ms[pick] <= 1.05 * ms[best]
    for L in cands:
        assert abs(spin.model_seconds(n, L) * 1e3 / ms[L] - 1.0) < 0.25, (L, ms[L])


TILE_SCRIPT = r"""
import sys
import numpy as np, torch
import paper_1801_04723_gb300 as s
from paper_1801_04723_gb300 import inputs
s.lib()
out = {}
for n, leaf in [(700, 64), (1024, 128), (333, 32)]:
    A = torch.from_numpy(inputs.sdd(n, seed=n)).to("cuda:0")
    X, info = s.invert(A, leaf=leaf)
    torch.cuda.synchronize()
    assert info["status"] == 0
    out[f"{n}_{leaf}"] = X.cpu().numpy()
np.savez(sys.argv[1], **out)
print("TILE-OK")
"""


def test_product_tile_size_changes_no_bit(spin, tmp_path):
    """The FP64 products choose 64-, 32- or 16-row tiles by how well they
    fill the SMs (SPIN_F64_TILE forces one, read once per process); every
    output is one FMA chain over k in order, so inversions are bit-identical
    whichever tile runs."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    results = {}
    for tile in ("", "64", "32", "16"):
        env = dict(os.environ, SPIN_F64_TILE=tile)
        path = str(tmp_path / f"x{tile or 'auto'}.npz")
        r = subprocess.run([sys.executable, "-c", TILE_SCRIPT, path], cwd=root, env=env, capture_output=True,
                           text=True, timeout=600)
        assert r.returncode == 0 and "TILE-OK" in r.stdout, r.stdout + r.stderr
        results[tile] = dict(np.load(path))
    for tile in ("64", "32", "16"):
        for key, X in results[""].items():
            np.testing.assert_array_equal(results[tile][key], X, err_msg=f"tile {tile}, {key}")
