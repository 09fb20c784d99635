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


def stages_of(L, orders, leaf):
    arr = (ctypes.c_int64 * len(orders))(*[int(v) for v in orders])
    cnt = ctypes.c_int64()
    L.spin_batch_schedule_stages.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.c_int, ctypes.c_int,
                                             ctypes.POINTER(ctypes.c_int64), ctypes.c_int64,
                                             ctypes.POINTER(ctypes.c_int64)]
    probe = (ctypes.c_int64 * 5)()
    L.spin_batch_schedule_stages(arr, len(orders), leaf, probe, 0, ctypes.byref(cnt))
    out = (ctypes.c_int64 * (5 * cnt.value))()
    assert L.spin_batch_schedule_stages(arr, len(orders), leaf, out, cnt.value, ctypes.byref(cnt)) == 0
    return np.array(out, dtype=np.int64).reshape(-1, 5)


def simulate(st, workers, seed):
    """The persistent kernel's protocol with `workers` CTAs: each holds the
    task it runs and the index of the next one (taken when it starts the
    current task, before its dependency wait); a task of matrix z starts once
    z's finished-task counter reaches its stage's dependency count.  Random
    task durations.  Returns the finished-task counter per matrix; raises if
    at some point no CTA can run while tasks remain (a deadlock)."""
    import heapq

    rng = np.random.default_rng(seed)
    starts = np.concatenate([[0], np.cumsum(st[:, 2] * st[:, 3])])
    total = int(starts[-1])
    nmat = int((st[:, 1] + st[:, 2]).max())
    done = np.zeros(nmat, dtype=np.int64)
    nxt = 0

    def task(t):
        g = int(np.searchsorted(starts, t, side="right") - 1)
        z = int(st[g, 1] + (t - starts[g]) // st[g, 3])
        return z, int(st[g, 4])

    # per worker: [current task, prefetched task]; waiting set; running heap
    held = []
    for _ in range(workers):
        held.append([nxt, None])
        nxt += 1
    waiting = set()
    for w in range(workers):
        if held[w][0] < total:
            held[w][1] = nxt  # taken as the worker starts on its first task
            nxt += 1
            waiting.add(w)
    running = []  # (end time, worker, z)
    now = 0.0
    finished = 0
    while finished < total:
        started = False
        for w in sorted(waiting):
            z, need = task(held[w][0])
            if done[z] >= need:
                heapq.heappush(running, (now + float(rng.exponential(1.0)), w, z))
                waiting.discard(w)
                started = True
        if not running:
            raise AssertionError(f"deadlock with {len(waiting)} CTAs waiting, {finished} of {total} tasks done")
        if started:
            continue
        now, w, z = heapq.heappop(running)
        done[z] += 1
        finished += 1
        t = held[w][1]
        held[w] = [t, None]
        if t < total:
            held[w][1] = nxt
            nxt += 1
            waiting.add(w)
    return done


@pytest.mark.parametrize("workers", [1, 3, 16, 64])
def test_persistent_protocol_completes(L, workers):
    """Every task only depends on tasks before it in the list, and the
    kernel's take-one-ahead protocol finishes the whole list for any number
    of CTAs (no deadlock), each matrix ending with all its tasks counted."""
    orders = [int(v) for v in inputs.batch_orders(120, seed=inputs.SEED_BASE + 31, lo=32, hi=512)] + [1, 5, 33]
    st = stages_of(L, orders, 0)
    # dependency counts are the matrix's tasks of earlier stages of its bucket,
    # all of which come earlier in the list
    seen = {}
    for kind, first, count, tiles, need in st:
        assert need == seen.get(first, 0)
        seen[first] = seen.get(first, 0) + tiles
    done = simulate(st, workers, seed=workers)
    per_matrix = {}
    for kind, first, count, tiles, need in st:
        for z in range(first, first + count):
            per_matrix[z] = per_matrix.get(z, 0) + tiles
    assert all(done[z] == v for z, v in per_matrix.items())
    assert len(per_matrix) == len(orders)


def test_protocol_simulation_catches_a_bad_order(L):
    """The simulation is not vacuous: a list whose second stage of a bucket
    comes before its first (a task waiting on tasks after it) deadlocks."""
    st = stages_of(L, [96, 96, 200], 0)
    bad = st.copy()
    first_rows = [i for i in range(len(bad)) if bad[i, 1] == bad[0, 1]]
    i0, i1 = first_rows[0], first_rows[1]
    bad[[i0, i1]] = bad[[i1, i0]]
    with pytest.raises(AssertionError, match="deadlock"):
        simulate(bad, 1, seed=0)
