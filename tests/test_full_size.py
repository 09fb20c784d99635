"""The full-size workloads, in the configuration bench.py times: one plain
FP64 inversion of order 32768 (A = G G^T/n + I, leaf 512) and one mixed
precision inversion of order 32768 (A = Q diag(d) Q^T, kappa = 1e3, leaf
128).  The oracle cannot invert these, so the checks are what holds at any
size: the oracle's compensated Freivalds residual on probe vectors (host
copies of A and X), the known inverse on sampled columns (mixed), and the
symmetry of the inverse of a symmetric matrix."""
import math

import numpy as np
import pytest

import oracle
from paper_1801_04723_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N = 32768
SEED = inputs.SEED_BASE


@pytest.fixture(scope="module")
def spin():
    import paper_1801_04723_gb300 as s

    s.build()
    s.lib()
    return s


def oracle_rel_residual(A, X, k=2):
    """sqrt(mean_k ||(AX - I) v||^2) / (||A||_F ||X||_F) with the oracle's
    compensated products on host copies; v ~ U(-1, 1) scaled to unit RMS."""
    Ah = A.cpu().numpy()
    Xh = X.cpu().numpy()
    V = inputs.probes(Ah.shape[0], k) * math.sqrt(3.0)
    r = oracle.freivalds(Ah, Xh, V)
    return math.sqrt(float(np.mean(r * r))) / (np.linalg.norm(Ah) * np.linalg.norm(Xh))


def test_config1_plain_fp64_full_size(spin):
    A = inputs.spd_gram_device(N, SEED + 1, "cuda:0")
    X, info = spin.invert(A, leaf=512)
    torch.cuda.synchronize()
    assert info["status"] == 0
    assert oracle_rel_residual(A, X) <= 1e-15
    # the inverse of a symmetric matrix is symmetric (up to the recursion's rounding)
    asym = float(torch.linalg.norm(X - X.T) / torch.linalg.norm(X))
    assert asym <= 1e-13


def test_config2_mixed_full_size(spin):
    A, V, d = inputs.householder_spd_device(N, SEED + 2, "cuda:0", reflectors=64, cond=1e3)
    X, info = spin.invert(A, leaf=128, precision="bf16x3", tol=1e-10)
    torch.cuda.synchronize()
    assert info["status"] == 0 and 0 < info["rel_residual"] <= 1e-10
    assert oracle_rel_residual(A, X) <= 2e-10  # k = 2 probes estimate ||AX - I||_F
    js = np.linspace(0, N - 1, 8).astype(int)
    E = np.zeros((N, 8))
    E[js, np.arange(8)] = 1.0
    ref = inputs.householder_apply(V, 1.0 / d, E)
    got = X[:, js].cpu().numpy()
    err = np.linalg.norm(got - ref, axis=0) / np.linalg.norm(ref, axis=0)
    # X - A^-1 = -A^-1 R: normwise, ||X - A^-1|| / ||A^-1|| <= kappa * (||A||_F /
    # ||A||_2) * rel_residual, and ||A||_F / ||A||_2 <= sqrt(n)
    bound = 1e3 * math.sqrt(N) * 1e-10
    assert math.sqrt(float(np.mean(err * err))) <= bound and float(err.max()) <= 4 * bound
