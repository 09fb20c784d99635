"""Random butterfly transform around the recursion (spin_opts.pretransform)
for matrices whose leading block or a Schur complement is singular, where
Algorithm 1 (no pivoting across blocks) breaks down.  Checked against the
oracle's dense form of the transform (same uniforms, drawn by the shared
splitmix64 generator), LAPACK's inverse and the compensated residual."""
import math

import numpy as np
import pytest

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


def uniforms(seed, n, depth=2):
    np_ = oracle.rbt_padded_order(n, depth)
    return inputs.uniform01(seed, np.arange(2 * depth * np_, dtype=np.uint64))


def swapped_blocks(n, seed, scale=0.1):
    """[[0, I + E], [I + F, D]] (h = n/2, E, F, D ~ scale U(-1,1)): A11 = 0,
    Algorithm 1 fails at once."""
    h = n // 2
    A = scale * inputs.uniform(seed, (n, n))
    A[:h, :h] = 0.0
    A[:h, h:2 * h] += np.eye(h)
    A[h:2 * h, :h] += np.eye(h)
    if n > 2 * h:
        A[-1, -1] += 1.0
    return A


def test_diagonals_match_the_generator(spin):
    seed = inputs.SEED_BASE + 90
    for n in (8, 203, 1000):
        d = host(spin.rbt_diagonals(seed, n))
        want = np.exp((uniforms(seed, n) - 0.5) / 10.0)
        np.testing.assert_allclose(d, want, rtol=4 * U, atol=0)


@pytest.mark.parametrize("n,leaf", [(200, 32), (203, 32), (512, 128)])
def test_plain_fails_transform_succeeds(spin, n, leaf):
    A = swapped_blocks(n, inputs.SEED_BASE + 91 + n)
    _, info = spin.invert(dev(A), leaf=leaf, check=False)
    assert info["status"] == 2 and info["pretransformed"] == 0
    seed = inputs.SEED_BASE + 95
    X, info = spin.invert(dev(A), leaf=leaf, pretransform=1, rbt_seed=seed)
    X = host(X)
    assert info["status"] == 0 and info["pretransformed"] == 1
    ref, st, _, _ = oracle.rbt_inv(A, leaf, uniforms(seed, n))
    assert st == 0
    kappa = np.linalg.cond(A)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e4 * kappa * n * U
    inv = np.linalg.inv(A)
    assert np.linalg.norm(X - inv) / np.linalg.norm(inv) <= 1e4 * kappa * n * U
    # no pivoting across blocks: the residual depends on how well the
    # transformed leading blocks are conditioned for this draw; the oracle
    # runs the same transform, so the GPU result is held to its residual
    assert oracle.residual(A, X)[0] <= max(1e-12, 10 * oracle.residual(A, ref)[0])


def test_auto_mode(spin):
    # a safe matrix stays on the plain path, bit for bit
    S = inputs.spd_gram(300, seed=11)
    Xp, _ = spin.invert(dev(S), leaf=64)
    Xa, info = spin.invert(dev(S), leaf=64, pretransform=2, rbt_seed=5)
    assert info["pretransformed"] == 0
    np.testing.assert_array_equal(host(Xa), host(Xp))
    # a breakdown reruns through the transform
    A = swapped_blocks(256, inputs.SEED_BASE + 97)
    X, info = spin.invert(dev(A), leaf=64, pretransform=2, rbt_seed=5)
    assert info["status"] == 0 and info["pretransformed"] == 1
    assert oracle.residual(A, host(X))[0] <= 1e-12


def test_transform_with_mixed_precision(spin):
    # tensor-core recursion on U^T A V, refinement against A itself; the
    # perturbation is scaled so that A (kappa ~ 2) and the transformed
    # blocks (kappa ~ 1.7) are well conditioned: BF16 level products carry
    # ~2^-16 relative error times the blocks' conditioning
    A = swapped_blocks(1024, inputs.SEED_BASE + 98, scale=0.5 / math.sqrt(1024))
    X, info = spin.invert(dev(A), leaf=128, precision="bf16x3", pretransform=1, rbt_seed=7)
    X = host(X)
    assert info["status"] == 0 and info["pretransformed"] == 1
    assert 0 < info["rel_residual"] <= 1e-10
    assert oracle.residual(A, X)[0] <= 1e-10
    inv = np.linalg.inv(A)
    assert np.linalg.norm(X - inv) / np.linalg.norm(inv) <= np.linalg.cond(A) * 10 * 1e-10
