"""Pins for the CPU oracle against facts fixed by the paper and by mathematics.

The oracle follows Algorithm 1 of the SPIN paper (Sec. 3.1); these tests tie
it to things other than itself: the 2x2 closed form, exact rational inverses
(Cramer's rule with a Leibniz determinant) on small integer matrices,
matrices whose inverse is exact in floating point (permutations, power-of-two
diagonals), the block-diagonal special case (II = III = 0), exact 2^k
scaling, Householder-built matrices of known inverse, LAPACK's inverse, and
the operation counts of Sec. 4 / Table 2 (6 products, 2 subtractions and one
scalar multiplication per internal node; 2^i nodes at level i; n/b leaves).
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import bounds
import oracle
from paper_1801_04723_gb300 import inputs

U = 2.0 ** -53


# ---------------------------------------------------------------- helpers --

def leibniz_det(M):
    n = len(M)
    total = Fraction(0)
    for perm in itertools.permutations(range(n)):
        inv = sum(1 for i in range(n) for j in range(i + 1, n) if perm[i] > perm[j])
        p = Fraction(1)
        for i in range(n):
            p *= M[i][perm[i]]
            if p == 0:
                break
        total += -p if inv % 2 else p
    return total


def exact_inverse(A):
    """A^-1 as Fractions by Cramer's rule: (A^-1)_ij = (-1)^(i+j) det(M_ji) / det(A)."""
    n = len(A)
    M = [[Fraction(x) if isinstance(x, Fraction) else Fraction(int(x)) for x in row] for row in A]
    det = leibniz_det(M)
    assert det != 0
    inv = [[None] * n for _ in range(n)]
    for i in range(n):
        for j in range(n):
            minor = [[M[r][c] for c in range(n) if c != i] for r in range(n) if r != j]
            inv[i][j] = (-1) ** (i + j) * (leibniz_det(minor) if minor else Fraction(1)) / det
    return inv


def leading_blocks_ok(A_int, leaf):
    """True when every block Algorithm 1 inverts at this leaf size (A11 and
    the Schur complement V, recursively) is nonsingular: the method has no
    pivoting across blocks (Sec. 2.1 restricts it to PD matrices)."""

    def rec(M):
        n = len(M)
        if leibniz_det(M) == 0:
            return False
        if n <= leaf:
            return True
        n1 = oracle.split(n)
        A11 = [r[:n1] for r in M[:n1]]
        if not rec(A11):
            return False
        inv11 = exact_inverse(A11)
        A12 = [r[n1:] for r in M[:n1]]
        A21 = [r[:n1] for r in M[n1:]]
        A22 = [r[n1:] for r in M[n1:]]
        n2 = n - n1
        T = [[sum(inv11[k][l] * A12[l][j] for l in range(n1)) for j in range(n2)] for k in range(n1)]
        S = [[A22[i][j] - sum(A21[i][k] * T[k][j] for k in range(n1)) for j in range(n2)] for i in range(n2)]
        return rec(S)

    return rec([[Fraction(int(x)) for x in row] for row in A_int])


def rel_err(X, Y):
    return float(np.linalg.norm(X - Y) / np.linalg.norm(Y))


# ------------------------------------------------------------------ tests --

def test_split_rule():
    # powers of two split in half; other orders keep a multiple of 32 on top
    assert oracle.split(2) == 1 and oracle.split(3) == 2 and oracle.split(64) == 32
    assert oracle.split(128) == 64 and oracle.split(1024) == 512 and oracle.split(32768) == 16384
    assert oracle.split(96) == 64 and oracle.split(100) == 64 and oracle.split(1000) == 512
    for n in range(2, 3000):
        n1 = oracle.split(n)
        assert 1 <= n1 < n and n1 >= n - n1


def test_2x2_closed_form_exact():
    # dyadic entries: every step of Algorithm 1 is exact, so the result equals
    # [[d, -b], [-c, a]] / (ad - bc) bit for bit
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    X, st = oracle.strassen_inv(A, 1)
    assert st == 0
    np.testing.assert_array_equal(X, np.array([[-2.0, 1.0], [1.5, -0.5]]))
    # Gauss-Jordan pivots on 3 here (1/3 rounds), so only close to it
    G, _ = oracle.gj_inv(A)
    assert rel_err(G, X) < 4 * U
    # a matrix whose pivots (4, then -1/2) keep every Gauss-Jordan step exact
    A = np.array([[4.0, 3.0], [2.0, 1.0]])
    want = np.array([[-0.5, 1.5], [1.0, -2.0]])
    np.testing.assert_array_equal(oracle.strassen_inv(A, 1)[0], want)
    np.testing.assert_array_equal(oracle.gj_inv(A)[0], want)


@pytest.mark.parametrize("seed", range(20))
def test_2x2_closed_form_random(seed):
    rng = np.random.default_rng(seed)
    a, b, c, d = rng.uniform(-1, 1, 4)
    a += 3.0 * np.sign(a)  # keep A11 and the Schur complement away from 0
    d += 3.0 * np.sign(d)
    A = np.array([[a, b], [c, d]])
    det = a * d - b * c
    ref = np.array([[d, -b], [-c, a]]) / det
    X, _ = oracle.strassen_inv(A, 1)
    assert rel_err(X, ref) < 8 * U


@pytest.mark.parametrize("n,leaf,seed", [(3, 1, 0), (4, 1, 1), (4, 2, 2), (5, 1, 3), (5, 2, 4),
                                         (5, 3, 5), (6, 1, 6), (6, 2, 7), (6, 3, 8), (6, 4, 9)])
def test_exact_rational_inverse(n, leaf, seed):
    """Brute force: Cramer's rule in exact rationals on random integer matrices."""
    rng = np.random.default_rng(1000 + seed)
    for _ in range(50):
        A = rng.integers(-9, 10, size=(n, n))
        A[np.diag_indices(n)] += 12 * np.where(rng.random(n) < 0.5, -1, 1)
        if leading_blocks_ok(A, leaf):
            break
    ex = exact_inverse(A)
    ref = np.array([[float(x) for x in row] for row in ex])
    X, st = oracle.strassen_inv(A.astype(float), leaf)
    assert st == 0
    kappa = np.linalg.cond(A.astype(float))
    assert rel_err(X, ref) < 50 * n * kappa * U
    G, _ = oracle.gj_inv(A.astype(float))
    assert rel_err(G, ref) < 50 * n * kappa * U


def test_exact_rational_inverse_nonsymmetric_blocks():
    # an integer matrix with an integer inverse (unimodular) exercises every
    # product with distinct, nonzero, asymmetric blocks; all steps are exact
    L = np.array([[1, 0, 0, 0], [2, 1, 0, 0], [-1, 3, 1, 0], [4, -2, 5, 1]])
    Uu = np.array([[1, 3, -1, 2], [0, 1, 2, -3], [0, 0, 1, 4], [0, 0, 0, 1]])
    A = (L @ Uu).astype(float)
    ex = exact_inverse(L @ Uu)
    ref = np.array([[float(x) for x in row] for row in ex])
    assert all(x.denominator == 1 for row in ex for x in row)
    for leaf in (1, 2):
        X, st = oracle.strassen_inv(A, leaf)
        assert st == 0
        np.testing.assert_allclose(X, ref, rtol=0, atol=1e-9)


@pytest.mark.parametrize("n", [1, 2, 5, 16, 33])
def test_permutation_exact(n):
    rng = np.random.default_rng(n)
    P = np.eye(n)[rng.permutation(n)]
    G, st = oracle.gj_inv(P)
    assert st == 0
    np.testing.assert_array_equal(G, P.T)


@pytest.mark.parametrize("n,leaf", [(8, 1), (16, 4), (64, 8), (100, 16)])
def test_power_of_two_diagonal_exact(n, leaf):
    rng = np.random.default_rng(n)
    d = 2.0 ** rng.integers(-20, 20, size=n) * np.where(rng.random(n) < 0.5, -1.0, 1.0)
    X, st = oracle.strassen_inv(np.diag(d), leaf)
    assert st == 0
    np.testing.assert_array_equal(X, np.diag(1.0 / d))


@pytest.mark.parametrize("n,leaf", [(64, 32), (128, 64), (96, 64)])
def test_block_diagonal_bitwise(n, leaf):
    """A12 = A21 = 0: II = III = IV = 0, V = -A22, so C11 = inv(A11) and
    C22 = -inv(-A22) = inv(A22) exactly; C12 = C21 = 0."""
    n1 = oracle.split(n)
    A = inputs.sdd(n, seed=42)
    A[:n1, n1:] = 0.0
    A[n1:, :n1] = 0.0
    X, st = oracle.strassen_inv(A, leaf)
    assert st == 0
    np.testing.assert_array_equal(X[:n1, n1:], 0.0)
    np.testing.assert_array_equal(X[n1:, :n1], 0.0)
    np.testing.assert_array_equal(X[:n1, :n1], oracle.strassen_inv(A[:n1, :n1].copy(), leaf)[0])
    np.testing.assert_array_equal(X[n1:, n1:], oracle.strassen_inv(A[n1:, n1:].copy(), leaf)[0])


@pytest.mark.parametrize("k", [-7, 3, 20])
def test_power_of_two_scaling_bitwise(k):
    A = inputs.sdd(96, seed=7)
    X, _ = oracle.strassen_inv(A, 16)
    Xs, _ = oracle.strassen_inv(A * 2.0 ** k, 16)
    np.testing.assert_array_equal(Xs, X * 2.0 ** -k)


@pytest.mark.parametrize("n,leaf", [(64, 8), (256, 32), (200, 32)])
def test_householder_known_inverse(n, leaf):
    A, V, d = inputs.householder_spd(n, seed=inputs.SEED_BASE + 2, reflectors=16, cond=1e3)
    ref = inputs.householder_apply(V, 1.0 / d, np.eye(n))
    X, st = oracle.strassen_inv(A, leaf)
    assert st == 0
    # forward error bound ~ c * kappa * u (kappa = 1e3)
    assert rel_err(X, ref) < 1e-11
    assert oracle.residual(A, X)[0] < 1e-14


@pytest.mark.parametrize("n,leaf", [(128, 16), (300, 64), (512, 128)])
def test_matches_lapack(n, leaf):
    A = inputs.sdd(n, seed=inputs.SEED_BASE + n)
    X, _ = oracle.strassen_inv(A, leaf)
    assert rel_err(X, np.linalg.inv(A)) < 1e-14
    G, _ = oracle.gj_inv(A)
    assert rel_err(G, np.linalg.inv(A)) < 1e-14


@pytest.mark.parametrize("n,leaf,family", [(65, 8, "sdd"), (257, 64, "spd"), (777, 100, "sdd"), (1100, 600, "spd")])
def test_matches_lapack_elementwise(n, leaf, family):
    """Element by element, within the componentwise bound the GPU parity
    tests use (|X - X_ref|_ij <= 4 n u (|X_ref||A||X_ref|)_ij)."""
    A = inputs.sdd(n, seed=11 + n) if family == "sdd" else inputs.spd_gram(n, seed=13 + n)
    X, _ = oracle.strassen_inv(A, leaf)
    assert bounds.elementwise_ok(X, np.linalg.inv(A), A)


def test_elementwise_bound_sees_a_local_error():
    """One deep leaf's block of the result off by 1e-11 relative: the
    Frobenius comparison of the parity tests (64 n kappa u) lets it through,
    the element-wise bound does not."""
    n, leaf = 1024, 128
    A = inputs.sdd(n, seed=inputs.SEED_BASE)
    ref, _ = oracle.strassen_inv(A, leaf)
    bad = ref.copy()
    bad[:32, :32] *= 1.0 + 1e-11  # inside the first leaf's block
    assert rel_err(bad, ref) <= 64 * n * np.linalg.cond(A) * U
    assert bounds.elementwise_ok(ref, np.linalg.inv(A), A)
    assert not bounds.elementwise_ok(bad, np.linalg.inv(A), A)


def test_transpose_and_leaf_invariance():
    A = inputs.spd_gram(256, seed=inputs.SEED_BASE + 1)
    A[0, 5] += 0.3  # break symmetry
    X16, _ = oracle.strassen_inv(A, 16)
    X64, _ = oracle.strassen_inv(A, 64)
    XT, _ = oracle.strassen_inv(A.T.copy(), 32)
    assert rel_err(X16, X64) < 1e-13
    assert rel_err(XT.T, X16) < 1e-13


def test_inverse_of_inverse():
    A = inputs.sdd(128, seed=5)
    X, _ = oracle.strassen_inv(A, 32)
    Y, _ = oracle.strassen_inv(X, 32)
    assert rel_err(Y, A) < 1e-14


def golden_counts():
    """Per-node operation counts as the paper states them (tests/golden)."""
    import os

    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "spin_op_counts.txt")
    out = {}
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                name, value = line.split()
                out[name] = int(value)
    return out


def test_golden_counts_fixture():
    assert golden_counts() == {"xy": 4, "multiplies": 6, "subtracts": 2, "scalar_muls": 1}


@pytest.mark.parametrize("p,q", [(10, 7), (10, 3), (9, 9), (12, 0)])
def test_operation_counts(p, q):
    """Sec. 4: 2^i nodes at level i, 2^(p-q) leaves; Table 2 / Sec. 4: per
    internal node 6 multiplications, 2 subtractions, 1 scalarMul.  The
    product flops 6 * 2 h^3 per node plus 2 L^3 per leaf sum to 2 n^3."""
    n, L = 2 ** p, 2 ** q
    A = inputs.sdd(n, seed=3) if n <= 1024 else None
    if A is None:
        pytest.skip("too large")
    per_node = golden_counts()
    oracle.strassen_inv(A, L)
    c = oracle.counts()
    b = n // L
    assert c["leaves"] == b
    assert c["internal"] == b - 1
    assert c["multiplies"] == per_node["multiplies"] * (b - 1)
    assert c["subtracts"] == per_node["subtracts"] * (b - 1)
    assert c["scalar_muls"] == per_node["scalar_muls"] * (b - 1)
    assert c["max_depth"] == p - q
    assert c["mult_flops"] + c["leaf_flops"] == 2 * n ** 3
    # Eq. (multiply): sum_i 2^i (n/2^(i+1))^3 = n^3 (b^2 - 1) / (6 b^2) per product type
    per_product = sum(2 ** i * (n // 2 ** (i + 1)) ** 3 for i in range(p - q))
    assert per_product * 6 * b * b == n ** 3 * (b * b - 1)
    assert c["mult_flops"] == 12 * per_product


def test_singular_leading_block():
    A = np.array([[0.0, 1.0], [1.0, 0.0]])
    with pytest.raises(oracle.SingularError):
        oracle.strassen_inv(A, 1)
    c = oracle.counts()
    assert c["fail_leaf"] == 0 and c["fail_col"] == 0
    X, st = oracle.strassen_inv(A, 2)  # the leaf pivots, so the whole matrix inverts
    assert st == 0
    np.testing.assert_array_equal(X, A)


def test_singular_schur_complement():
    # A11 = 1 is fine, but V = A21 A11^-1 A12 - A22 = 1 - 1 = 0
    A = np.array([[1.0, 1.0], [1.0, 1.0]])
    X, st = oracle.strassen_inv(A, 1, raise_on_singular=False)
    assert st == oracle.SINGULAR
    assert oracle.counts()["fail_leaf"] == 1


def test_residual_exact_cases():
    # exact inverse -> residual exactly 0
    L = np.array([[1, 0, 0], [2, 1, 0], [-1, 3, 1]], dtype=float)
    Li = np.array([[1, 0, 0], [-2, 1, 0], [7, -3, 1]], dtype=float)
    assert oracle.residual(L, Li)[1] == 0.0
    # A = I, X = (1 + e) I: R = e I
    n, e = 7, 2.0 ** -30
    rel, ab = oracle.residual(np.eye(n), (1 + e) * np.eye(n))
    assert ab == pytest.approx(e * math.sqrt(n), rel=1e-15)
    assert rel == pytest.approx(e / (math.sqrt(n) * (1 + e)), rel=1e-15)


def test_residual_is_compensated():
    # row [2^60, 1, -2^60] against a column of ones: the true product is 1;
    # naive FP64 summation returns 0.  The exact residual entry R_00 = 1 - 1 = 0.
    A = np.array([[2.0 ** 60, 1.0, -(2.0 ** 60)], [0, 1, 0], [0, 0, 1]])
    X = np.array([[1.0, 0, 0], [1.0, 1, 0], [1.0, 0, 1]])
    _, _, R = oracle.residual(A, X, return_matrix=True)
    # exact: AX = [[1, 1, -2^60], [1, 1, 0], [1, 0, 1]]
    exact = np.array([[1.0, 1.0, -(2.0 ** 60)], [1.0, 1.0, 0.0], [1.0, 0.0, 1.0]]) - np.eye(3)
    np.testing.assert_array_equal(R, exact)


def test_freivalds_exact_rational():
    rng = np.random.default_rng(9)
    A = rng.integers(-5, 6, size=(6, 6)).astype(float)
    X = rng.integers(-5, 6, size=(6, 6)).astype(float)
    V = rng.integers(-3, 4, size=(6, 3)).astype(float)
    got = oracle.freivalds(A, X, V)
    R = A @ X - np.eye(6)  # small integers: exact in FP64
    want = np.linalg.norm(R @ V, axis=0)
    np.testing.assert_allclose(got, want, rtol=1e-15)


def test_generators_deterministic():
    a = inputs.sdd(64, seed=1)
    b = inputs.sdd(64, seed=1)
    np.testing.assert_array_equal(a, b)
    assert np.all(np.abs(np.diag(a)) > np.sum(np.abs(a), axis=1) - np.abs(np.diag(a)))
    # splitmix64 reference outputs for seed 0 (Vigna's splitmix64.c, first three draws)
    z = inputs.splitmix64(0, np.arange(3, dtype=np.uint64))
    assert [int(x) for x in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


# ------------------------------------------------- random butterfly transform --

def _u(seed, n, depth=2):
    np_ = oracle.rbt_padded_order(n, depth)
    return inputs.uniform01(seed, np.arange(2 * depth * np_, dtype=np.uint64))


def test_rbt_order2_closed_form():
    # one butterfly of order 2: [[r, s], [r, -s]] / sqrt(2)
    r, s = 1.03, 0.97
    W = oracle.rbt_butterfly(np.array([[r, s]]))
    want = np.array([[r, s], [r, -s]]) / math.sqrt(2.0)
    np.testing.assert_allclose(W, want, rtol=0, atol=4 * U)


def test_rbt_determinant_is_product_of_diagonals():
    # each block of order m has |det| = prod(r) prod(s) (the 1/sqrt(2)^m and
    # the 2^(m/2) of [[R, S], [R, -S]] cancel); levels multiply
    rng = np.random.default_rng(3)
    for depth, np_ in ((1, 8), (2, 8), (3, 16), (2, 12)):
        d = np.exp((rng.random((depth, np_)) - 0.5) / 10.0)
        W = oracle.rbt_butterfly(d)
        assert abs(abs(np.linalg.det(W)) - np.prod(d)) <= 1e-12 * np.prod(d)


def test_rbt_unit_diagonals_are_orthogonal():
    # R = S = I: every block is the orthogonal Haar butterfly, so W is orthogonal
    W = oracle.rbt_butterfly(np.ones((2, 16)))
    np.testing.assert_allclose(W @ W.T, np.eye(16), atol=1e-15)


@pytest.mark.parametrize("n,leaf", [(50, 8), (64, 16), (33, 33)])
def test_rbt_inverse_matches_lapack(n, leaf):
    # nonsymmetric, moderately conditioned (the block recursion has no
    # pivoting: its error grows with the conditioning of the leading blocks)
    A = inputs.uniform(inputs.SEED_BASE + 60 + n, (n, n)) + 2.0 * math.sqrt(n) * np.eye(n)
    X, st, U_, V_ = oracle.rbt_inv(A, leaf, _u(inputs.SEED_BASE + 70, n))
    assert st == 0
    ref = np.linalg.inv(A)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e3 * np.linalg.cond(A) * U
    assert oracle.residual(A, X)[0] <= 1e-13


def test_rbt_handles_a_singular_leading_block():
    # [[0, I], [I, 0]] blocks: A11 = 0, so Algorithm 1 fails at its first
    # leaf; the transformed matrix's leading blocks are nonsingular
    n = 40
    A = np.zeros((n, n))
    A[:20, 20:] = np.eye(20)
    A[20:, :20] = np.eye(20)
    A += 0.1 * inputs.uniform(inputs.SEED_BASE + 80, (n, n))
    A[:20, :20] = 0.0
    with pytest.raises(oracle.SingularError):
        oracle.strassen_inv(A, 8)
    X, st, _, _ = oracle.rbt_inv(A, 8, _u(inputs.SEED_BASE + 81, n))
    assert st == 0
    ref = np.linalg.inv(A)
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e4 * np.linalg.cond(A) * U
