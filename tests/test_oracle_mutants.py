"""The oracle's pins have teeth: plant one plausible mistake at a time in a
copy of the oracle's C source (a flipped sign, a transposed operand, a
dropped factor, a wrong quadrant, a missing un-permutation), build it, and
check that the pins of ``test_oracle_pins.py`` reject it.  The mutants are
built and run on the CPU only."""
import os
import subprocess

import numpy as np
import pytest

import oracle
from paper_1801_04723_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "spin_oracle.c")

MUTANTS = {
    "c22_sign": ("mat_scale(VI, n2, -1.0, C22", "mat_scale(VI, n2, 1.0, C22"),
    "c12_operand_order": ("mat_mul(III, n2, VI, n2, C12, n2, n1, n2, n2)",
                          "mat_mul(VI, n2, III, n2, C12, n2, n1, n2, n2)"),
    "v_sign": ("mat_sub(IV, n2, A22, lda, V, n2, n2, n2)", "mat_sub(A22, lda, IV, n2, V, n2, n2, n2)"),
    "vii_drops_vi": ("mat_mul(III, n2, C21, n1, VII, n1, n1, n2, n1)",
                     "mat_mul(III, n2, II, n1, VII, n1, n1, n2, n1)"),
    "a12_a21_swapped": ("const double* A12 = A + n1;", "const double* A12 = A + n1 * lda;"),
    "ii_transposed": ("mat_mul(A21, lda, I, n1, II, n1, n2, n1, n1)",
                      "mat_mul(I, n1, A21, lda, II, n1, n2, n1, n1)"),
    "gj_no_unpermute": ("if (p != k)\n            for (int64_t i = 0; i < n; i++) {",
                        "if (0)\n            for (int64_t i = 0; i < n; i++) {"),
    "gj_pivot_slot": ("rk[k] = 1.0;", "rk[k] = rk[k];"),
    "gj_tie_or_max": ("if (v > best) { best = v; p = i; }", "if (v < best) { best = v; p = i; }"),
    "residual_drops_identity": ("(i == j) ? -1.0 : 0.0", "0.0"),
}


def build_mutant(tmp_path, name):
    old, new = MUTANTS[name]
    text = open(SRC).read()
    assert text.count(old) == 1, f"mutation site for {name} not unique"
    path = tmp_path / f"m_{name}.c"
    path.write_text(text.replace(old, new))
    so = tmp_path / f"m_{name}.so"
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
                    "-o", str(so), str(path), "-lm"], check=True)
    return oracle.bind(str(so))


def pins_pass(lib) -> bool:
    """A compact subset of the pins; True only if every one holds."""
    try:
        # 2x2 closed form (dyadic, exact)
        X, _ = oracle.strassen_inv(np.array([[4.0, 3.0], [2.0, 1.0]]), 1, lib=lib)
        if not np.array_equal(X, np.array([[-0.5, 1.5], [1.0, -2.0]])):
            return False
        # LAPACK agreement on SDD and nonsymmetric inputs, several leaf sizes
        for n, leaf in ((64, 8), (96, 16), (128, 32)):
            A = inputs.sdd(n, seed=11 + n)
            A[: n // 3, :] *= 1.7  # make it clearly nonsymmetric
            ref = np.linalg.inv(A)
            X, st = oracle.strassen_inv(A, leaf, lib=lib, raise_on_singular=False)
            if st != 0 or np.linalg.norm(X - ref) / np.linalg.norm(ref) > 1e-13:
                return False
            G, st = oracle.gj_inv(A, lib=lib, raise_on_singular=False)
            if st != 0 or np.linalg.norm(G - ref) / np.linalg.norm(ref) > 1e-13:
                return False
        # permutation (exact) and the residual of an exact inverse
        P = np.eye(9)[np.random.default_rng(3).permutation(9)]
        G, _ = oracle.gj_inv(P, lib=lib)
        if not np.array_equal(G, P.T):
            return False
        rel, ab = oracle.residual(np.eye(5), np.eye(5), lib=lib)
        if ab != 0.0:
            return False
        return True
    except (oracle.SingularError, ValueError, FloatingPointError):
        return False


def test_unmutated_oracle_passes():
    assert pins_pass(oracle._load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    lib = build_mutant(tmp_path, name)
    assert not pins_pass(lib), f"mutant {name} survived the pins"
