"""spin_invert_noalloc: the plain inversion with its workspace in a fixed
device array, for callers that cannot let the library allocate device
memory (device memory reserved up front by another allocator, or code that
cannot afford the device-wide synchronisation of cudaMalloc / cudaFree).

It runs the same kernels in the same order as spin_invert, so its result
must be bit-identical to spin_invert's, on two calls in a row (the second
call finds the array holding the first call's data), and within the
oracle's element-wise bound; after a first call the device's free memory
must not change across further calls; sizes whose workspace does not fit
the array must be refused before any work.

This file is named so that pytest collects it last."""
import numpy as np
import pytest

import bounds
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


@pytest.mark.parametrize("n,leaf,family", [(700, 100, "sdd"), (1024, 128, "spd")])
def test_noalloc_matches_invert_twice(spin, n, leaf, family):
    A = inputs.sdd(n, seed=1) if family == "sdd" else inputs.spd_gram(n, seed=2)
    Ad = dev(A)
    want, info = spin.invert(Ad, leaf=leaf)
    torch.cuda.synchronize()
    assert info["status"] == 0
    want = want.cpu().numpy()
    ref, _ = oracle.strassen_inv(A, leaf)
    for _ in range(2):
        X, status = spin.invert_noalloc(Ad, leaf=leaf)
        torch.cuda.synchronize()
        assert status == 0
        got = X.cpu().numpy()
        np.testing.assert_array_equal(got, want)
        assert bounds.elementwise_ok(got, ref, A)


def test_noalloc_leaves_device_memory_alone(spin):
    n, leaf = 1024, 128
    Ad = dev(inputs.sdd(n, seed=5))
    X1 = torch.empty_like(Ad)
    X2 = torch.empty_like(Ad)
    _, status = spin.invert_noalloc(Ad, leaf=leaf, out=X1)  # first call on this device: module and array placed
    torch.cuda.synchronize()
    assert status == 0
    free0, _ = torch.cuda.mem_get_info()
    for out in (X2, X1, X2):
        _, status = spin.invert_noalloc(Ad, leaf=leaf, out=out)
        assert status == 0
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.equal(X1, X2)


def test_noalloc_reports_singular_and_refuses_large(spin):
    _, status = spin.invert_noalloc(dev(np.array([[0.0, 1.0], [1.0, 0.0]])), leaf=1)
    assert status == 2
    X, status = spin.invert_noalloc(dev(inputs.sdd(8, seed=3)), leaf=4)  # status record was cleared
    assert status == 0
    big = torch.zeros((2048, 2048), dtype=torch.float64, device="cuda:0")
    _, status = spin.invert_noalloc(big, leaf=128)
    assert status == 1  # SPIN_ERR_INVALID_ARG: workspace beyond the fixed array
