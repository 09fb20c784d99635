"""Host-side checks of the persistent schedule of a plain batch (no GPU):
the task list spin_invert_batched's persistent kernel walks is built from
each order bucket's recursion, so its leaf inversions and level products
must be those of Algorithm 1 as the oracle counts them, at the same leaf
sizes, and its flops must sum to 2 n^3 per matrix (Sec. 4: six products of
order n/2 per node plus 2 L^3 per leaf).  The library also checks the task
order's invariants itself (each bucket's stages in recursion order, every
dependency count equal to the tasks before it)."""
import ctypes

import numpy as np
import pytest

import oracle
import paper_1801_04723_gb300 as spin
from paper_1801_04723_gb300 import binding, inputs

MAX_LEAF = 64


@pytest.fixture(scope="module")
def L():
    spin.build()
    lib = binding.lib()
    i64p = ctypes.POINTER(ctypes.c_int64)
    lib.spin_batch_schedule_info.argtypes = [i64p, ctypes.c_int, ctypes.c_int, i64p, i64p, i64p, i64p,
                                             ctypes.POINTER(ctypes.c_double)]
    lib.spin_batch_schedule_info.restype = ctypes.c_int
    return lib


def info(L, orders, leaf):
    arr = (ctypes.c_int64 * len(orders))(*[int(v) for v in orders])
    out = [ctypes.c_int64() for _ in range(4)]
    fl = ctypes.c_double()
    rc = L.spin_batch_schedule_info(arr, len(orders), leaf, *[ctypes.byref(v) for v in out], ctypes.byref(fl))
    return rc, {"stages": out[0].value, "tasks": out[1].value, "leaves": out[2].value, "products": out[3].value,
                "flops": fl.value}


def effective_leaf(n, leaf):
    base = leaf if leaf > 0 else (n if n <= 128 else 64)
    return min(base, MAX_LEAF, n)


def oracle_counts(n, leaf):
    A = np.eye(n) * 2.0
    oracle.strassen_inv(A, leaf)
    return oracle.counts()


@pytest.mark.parametrize("leaf", [0, 32, 17])
def test_schedule_matches_algorithm1_counts(L, leaf):
    orders = [1, 5, 32, 33, 64, 96, 96, 130, 200, 300, 300, 300]
    rc, got = info(L, orders, leaf)
    assert rc == 0
    leaves = products = 0
    for n in orders:
        c = oracle_counts(n, effective_leaf(n, leaf))
        leaves += c["leaves"]
        products += c["multiplies"]
    assert got["leaves"] == leaves
    assert got["products"] == products
    assert got["flops"] == sum(2.0 * n ** 3 for n in orders)
    # one stage per leaf and per product of each bucket; tasks at least one per stage and matrix
    assert got["tasks"] >= got["leaves"] + got["products"]


def test_schedule_of_the_batching_workload(L):
    orders = inputs.batch_orders(4096, seed=inputs.SEED_BASE + 3)
    for leaf in (0, 32, 64):
        rc, got = info(L, orders, leaf)
        assert rc == 0
        assert got["flops"] == float(sum(2 * int(n) ** 3 for n in orders))
        assert got["tasks"] > got["leaves"] + got["products"] > 0


def test_schedule_rejects_bad_arguments(L):
    rc, _ = info(L, [64, 128], MAX_LEAF + 1)
    assert rc == 1
    rc, _ = info(L, [0, 128], 0)
    assert rc == 1
    rc, _ = info(L, [70000], 0)
    assert rc == 1
