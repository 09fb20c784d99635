"""Mixed-precision form: BF16 tensor-core level products, FP64 leaves,
FP64-class Schur complements at the top levels, Newton-Schulz refinement.

The library reports the relative residual ||AX - I||_F / (||A||_F ||X||_F)
it reached; the tests recompute it with the oracle's compensated residual
(independent code, FP64 with error-free transformations) and require both to
be <= the requested tolerance (1e-10 unless stated), compare the result with
the oracle's FP64 Strassen inverse and, for Householder-built matrices, with
the known inverse.  Forward-error tolerance: kappa * 10 * tol.
"""
import numpy as np
import pytest

import oracle
from paper_1801_04723_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


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


def rel(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


@pytest.mark.parametrize("n,leaf", [(1024, 128), (1536, 256), (777, 100)])
def test_householder_cond1e3(spin, n, leaf):
    A, V, d = inputs.householder_spd(n, seed=inputs.SEED_BASE + 2, reflectors=64, cond=1e3)
    X, info = spin.invert(dev(A), leaf=leaf, precision="bf16x3")
    X = host(X)
    assert info["status"] == 0, info
    assert 0 < info["rel_residual"] <= 1e-10
    res = oracle.residual(A, X)[0]
    assert res <= 1e-10
    assert abs(res - info["rel_residual"]) <= 0.05 * res + 1e-16  # the library's figure is the true one
    ref = inputs.householder_apply(V, 1.0 / d, np.eye(n))
    assert rel(X, ref) <= 1e3 * 10 * 1e-10


@pytest.mark.parametrize("family,n,leaf", [("sdd", 1000, 128), ("spd", 1024, 128), ("spd", 640, 64)])
def test_against_oracle(spin, family, n, leaf):
    A = inputs.sdd(n, seed=31 + n) if family == "sdd" else inputs.spd_gram(n, seed=37 + n)
    X, info = spin.invert(dev(A), leaf=leaf, precision="bf16x3")
    X = host(X)
    ref, _ = oracle.strassen_inv(A, leaf)
    assert info["status"] == 0
    assert oracle.residual(A, X)[0] <= 1e-10
    assert rel(X, ref) <= np.linalg.cond(A) * 10 * 1e-10


@pytest.mark.parametrize("fp64_levels", [0, 1, 3])
def test_fp64_levels_option(spin, fp64_levels):
    A, _, _ = inputs.householder_spd(1024, seed=5, reflectors=32, cond=1e2)
    X, info = spin.invert(dev(A), leaf=128, precision="bf16x3", fp64_levels=fp64_levels)
    assert info["status"] == 0 and oracle.residual(A, host(X))[0] <= 1e-10


def test_tighter_tolerance(spin):
    A = inputs.spd_gram(1024, seed=41)
    X, info = spin.invert(dev(A), leaf=128, precision="bf16x3", tol=1e-13)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-13
    assert oracle.residual(A, host(X))[0] <= 1e-13


def test_refinement_is_decided_on_the_device(spin):
    """A non-blocking mixed call only enqueues: the Newton-Schulz rounds and
    their stopping decision run on the device, and spin_sync reads the
    status, steps and residual afterwards."""
    A = inputs.householder_spd(1024, seed=inputs.SEED_BASE + 2, reflectors=16, cond=1e3)[0]
    Ad = dev(A)
    X, none = spin.invert(Ad, leaf=128, precision="bf16x3", tol=1e-10, blocking=False)
    assert none is None
    info = spin.sync()
    assert info["status"] == 0 and info["refine_iters"] >= 1 and 0 < info["rel_residual"] <= 1e-10
    assert info["fail_leaf"] == -1
    Xb, infob = spin.invert(Ad, leaf=128, precision="bf16x3", tol=1e-10)
    np.testing.assert_array_equal(X.cpu().numpy(), Xb.cpu().numpy())
    # the sums of squares behind the residual are atomic adds: same X, last bits may differ
    assert abs(infob["rel_residual"] - info["rel_residual"]) <= 1e-12 * info["rel_residual"]
    assert oracle.residual(A, X.cpu().numpy())[0] <= 1e-10


def test_not_converged_status(spin):
    A, _, _ = inputs.householder_spd(512, seed=9, reflectors=16, cond=1e3)
    X, info = spin.invert(dev(A), leaf=64, precision="bf16x3", tol=1e-30, max_refine=1, check=False)
    assert info["status"] == 3 and info["refine_iters"] == 1
    assert info["fail_leaf"] == -1 and info["fail_col"] == -1  # a refinement status, not a leaf's
    assert info["rel_residual"] > 0


def test_small_orders_and_singular(spin):
    for n in (1, 2, 7, 100):
        A = inputs.sdd(n, seed=n)
        X, info = spin.invert(dev(A), leaf=16, precision="bf16x3")
        assert info["status"] == 0
        assert oracle.residual(A, host(X))[0] <= 1e-10
    _, info = spin.invert(dev(np.array([[0.0, 1.0], [1.0, 0.0]])), leaf=1, precision="bf16x3", check=False)
    assert info["status"] == 2 and info["fail_leaf"] == 0


def test_deterministic(spin):
    A = dev(inputs.spd_gram(900, seed=43))
    X1 = host(spin.invert(A, leaf=128, precision="bf16x3")[0])
    X2 = host(spin.invert(A, leaf=128, precision="bf16x3")[0])
    np.testing.assert_array_equal(X1, X2)


@pytest.mark.parametrize("n,leaf", [(1024, 128), (777, 100)])
def test_digit_level_products(spin, n, leaf):
    """SPIN_MIXED_DIGITS: 4-slice digit level products; same residual target."""
    A, V, d = inputs.householder_spd(n, seed=inputs.SEED_BASE + 2, reflectors=64, cond=1e3)
    X, info = spin.invert(dev(A), leaf=leaf, precision="digits")
    X = host(X)
    assert info["status"] == 0 and info["rel_residual"] <= 1e-10
    assert oracle.residual(A, X)[0] <= 1e-10
    ref = inputs.householder_apply(V, 1.0 / d, np.eye(n))
    assert rel(X, ref) <= 1e3 * 10 * 1e-10
