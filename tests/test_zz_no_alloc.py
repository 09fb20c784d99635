"""spin_invert_noalloc: the plain inversion with its workspace in a fixed
device array, for callers that cannot let the library allocate device
memory.  Its results must match spin_invert's (same kernels, same order of
operations) within the plain path's tolerance, on two calls in a row (the
second call finds the array holding the first call's data), and sizes whose
workspace does not fit the array must be refused before any work.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

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


def test_noalloc_matches_invert_twice(spin):
    for n, leaf, seed in ((700, 100, 1), (1024, 128, 2)):
        A = inputs.sdd(n, seed=seed) if seed == 1 else inputs.spd_gram(n, seed=seed)
        Ad = dev(A)
        want, info = spin.invert(Ad, leaf=leaf)
        torch.cuda.synchronize()
        tol = 64 * n * np.linalg.cond(A) * U
        for _ in range(2):
            X, status = spin.invert_noalloc(Ad, leaf=leaf)
            torch.cuda.synchronize()
            assert status == 0
            err = float(torch.linalg.norm(X - want) / torch.linalg.norm(want))
            assert err <= tol


def test_noalloc_reports_singular_and_refuses_large(spin):
    _, status = spin.invert_noalloc(dev(np.array([[0.0, 1.0], [1.0, 0.0]])), leaf=1)
    assert status == 2
    X, status = spin.invert_noalloc(dev(inputs.sdd(8, seed=3)), leaf=4)  # status record was cleared
    assert status == 0
    big = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda:0")
    _, status = spin.invert_noalloc(big, leaf=128)
    assert status == 1  # SPIN_ERR_INVALID_ARG: workspace beyond the fixed array
