"""Serving: requests of mixed orders and precisions submitted while others
run, batched as they arrive; every result must equal the same request served
alone, bit for bit (every decision of both paths is per matrix and the
kernels are deterministic), be within tolerance of the single-matrix library
call and within the requested residual, and admission must respect the
memory budget."""
import time

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


def serve_alone(spin, A, prec, tol, **cfg):
    """The same request through a server of its own, alone."""
    srv = spin.Server(hbm_budget_bytes=16 << 30, max_slots=1, **cfg)
    t = srv.submit(A, precision=prec, tol=tol)
    deadline = time.time() + 300
    while (got := srv.poll(t)) is None and time.time() < deadline:
        time.sleep(0.001)
    srv.close()
    assert got is not None
    return got


@pytest.mark.parametrize("priority_order", [0, 512])
def test_serve_mix_equals_alone(spin, priority_order):
    """Requests of mixed orders and precisions arriving while others run:
    each result equals the same request served alone, bit for bit (plain and
    mixed: every decision of the batched path is per matrix), and is within
    tolerance of the single-matrix library call."""
    trace = inputs.serve_trace(inputs.SEED_BASE + 4004, rate=400.0, duration=0.08, lo=64, hi=1400)
    assert len(trace) >= 20
    srv = spin.Server(hbm_budget_bytes=16 << 30, max_slots=4, priority_order=priority_order)
    reqs = []
    t0 = time.perf_counter()
    for j, (t_arr, n, alpha, mixed) in enumerate(trace):
        A = inputs.spd_gram(n, seed=inputs.SEED_BASE + 4000 + j, alpha=alpha)
        src = torch.from_numpy(A).cuda() if j % 3 else A  # device and host submissions
        prec, tol = ("bf16x3", 1e-10) if mixed else ("fp64", 1e-13)
        while time.perf_counter() - t0 < t_arr:
            time.sleep(0.001)
        reqs.append((srv.submit(src, precision=prec, tol=tol), A, prec, tol))
    results = {}
    deadline = time.time() + 300
    while len(results) < len(reqs) and time.time() < deadline:
        for t, A, prec, tol in reqs:
            if t in results:
                continue
            got = srv.poll(t)
            if got is not None:
                results[t] = got
        time.sleep(0.002)
    st = srv.stats()
    srv.close()
    assert len(results) == len(reqs)
    assert st["completed"] == st["submitted"] == len(reqs) and st["rejected"] == 0
    for t, A, prec, tol in reqs:
        X, r = results[t]
        assert r["status"] == 0, r
        Xa, ra = serve_alone(spin, A, prec, tol)
        assert ra["status"] == 0 and ra["batch"] == (1 if A.shape[0] <= 1024 else 0)  # orders above 1024: single path
        np.testing.assert_array_equal(X, Xa)
        lib, info = spin.invert(torch.from_numpy(A).cuda(), precision=prec, tol=tol)
        lib = lib.cpu().numpy()
        if prec == "fp64":
            assert oracle.residual(A, X)[0] <= 1e-13
            assert np.linalg.norm(X - lib) / np.linalg.norm(lib) <= 64 * A.shape[0] * np.linalg.cond(A) * 2.0 ** -53
        else:
            assert r["rel_residual"] <= tol and oracle.residual(A, X)[0] <= tol
            assert np.linalg.norm(X - lib) / np.linalg.norm(lib) <= np.linalg.cond(A) * 10 * tol
        assert r["latency_ms"] >= r["run_ms"] > 0


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-13), ("bf16x3", 1e-10)])
def test_serve_batches_same_order_requests(spin, prec, tol):
    """Requests queued behind a busy slot whose orders pad to the same
    multiple of 32 (449 ... 480 -> 480) run as one batched launch group: each
    reports the group's size, the server counts one group, and every result
    equals the request served alone, bit for bit."""
    orders = [449, 480, 463, 470, 455, 477]
    mats = [inputs.spd_gram(n, seed=inputs.SEED_BASE + 500 + i, alpha=0.5) for i, n in enumerate(orders)]
    srcs = [a if i % 2 else torch.from_numpy(a).cuda() for i, a in enumerate(mats)]  # host and device
    big = torch.from_numpy(inputs.sdd(4096, seed=3)).cuda()
    torch.cuda.synchronize()
    srv = spin.Server(hbm_budget_bytes=16 << 30, max_slots=1)
    tb = srv.submit(big, precision="fp64")  # keeps the only slot busy (~0.1 s)
    for _ in range(5000):  # bounded wait until it runs
        if srv.stats()["running"] == 1:
            break
        time.sleep(0.001)
    tickets = [srv.submit(a, precision=prec, tol=tol) for a in srcs]
    assert srv.stats()["running"] == 1  # all six queued behind it
    got = {}
    deadline = time.time() + 300
    while len(got) < len(tickets) and time.time() < deadline:
        for t in tickets:
            if t not in got and (g := srv.poll(t)) is not None:
                got[t] = g
        time.sleep(0.001)
    while srv.poll(tb, discard=True) is None:
        time.sleep(0.001)
    st = srv.stats()
    srv.close()
    assert len(got) == len(tickets)
    assert st["groups"] >= 1 and st["max_group"] == len(orders), st
    for t, A in zip(tickets, mats):
        X, r = got[t]
        assert r["status"] == 0 and r["batch"] == len(orders), r
        Xa, _ = serve_alone(spin, A, prec, tol)
        np.testing.assert_array_equal(X, Xa)
        lim = 1e-13 if prec == "fp64" else tol
        assert oracle.residual(A, X)[0] <= lim
        if prec != "fp64":
            assert r["rel_residual"] <= tol and r["refine_iters"] >= 1


def test_serve_batching_off_uses_the_single_path(spin):
    A = inputs.spd_gram(300, seed=9, alpha=0.5)
    X, r = serve_alone(spin, A, "fp64", 1e-13, max_batch=1)
    lib, _ = spin.invert(torch.from_numpy(A).cuda())
    np.testing.assert_array_equal(X, lib.cpu().numpy())
    assert r["batch"] == 0  # not a launch group


def test_serve_budget_and_errors(spin):
    srv = spin.Server(hbm_budget_bytes=16 << 20, max_slots=2)
    A = torch.from_numpy(inputs.sdd(2048, seed=1)).cuda()  # X alone is 32 MB > 16 MB
    with pytest.raises(spin.SpinError):
        srv.submit(A, precision="fp64")
    assert srv.stats()["rejected"] == 1
    small = inputs.sdd(200, seed=2)  # ~0.7 MB: fits
    t = srv.submit(small, precision="fp64")
    while (got := srv.poll(t)) is None:
        time.sleep(0.001)
    X, r = got
    assert r["status"] == 0
    assert oracle.residual(small, X)[0] <= 1e-13
    with pytest.raises(spin.SpinError):
        srv.poll(t)  # already collected
    srv.close()


def test_serve_load_shedding(spin):
    """max_queued_bytes bounds the A bytes of queued (not yet admitted)
    requests: with the only slot busy and room for two 256 x 256 requests,
    the third and later submits are shed (None) and counted; the queued
    ones still run and are right."""
    nbytes = 256 * 256 * 8
    srv = spin.Server(hbm_budget_bytes=1 << 30, max_slots=1, max_queued_bytes=2 * nbytes)
    big = torch.from_numpy(inputs.sdd(2048, seed=3)).cuda()
    tb = srv.submit(big, precision="fp64")
    assert tb is not None
    for _ in range(5000):  # the slot has taken the big request (bounded wait)
        if srv.stats()["running"] == 1:
            break
        time.sleep(0.001)
    assert srv.stats()["running"] == 1
    smalls = [inputs.sdd(256, seed=10 + i) for i in range(5)]
    tickets = [srv.submit(a, precision="fp64") for a in smalls]
    assert [t is None for t in tickets] == [False, False, True, True, True]
    assert srv.stats()["shed"] == 3
    for a, t in zip(smalls[:2], tickets[:2]):
        while (got := srv.poll(t)) is None:
            time.sleep(0.001)
        assert got[1]["status"] == 0 and oracle.residual(a, got[0])[0] <= 1e-13
    while srv.poll(tb, discard=True) is None:
        time.sleep(0.001)
    srv.close()


DEFER_SCRIPT = r"""
import time
import numpy as np, torch
import paper_1801_04723_gb300 as s
from paper_1801_04723_gb300 import inputs
s.lib()
srv = s.Server(hbm_budget_bytes=4 << 30, max_slots=2)
big = torch.from_numpy(inputs.sdd(4096, seed=1)).cuda()
small = inputs.sdd(300, seed=2)
torch.cuda.synchronize()
t1 = srv.submit(big, precision="fp64")  # ticket 1: ~0.1 s of work
for _ in range(5000):  # bounded wait until it runs
    if srv.stats()["running"] == 1:
        break
    time.sleep(0.001)
t2 = srv.submit(small, precision="fp64")  # ticket 2: its first two allocation attempts fail
assert (t1, t2) == (1, 2)
out = {}
for t in (t1, t2):
    for _ in range(600000):
        got = srv.poll(t, discard=(t == t1))
        if got is not None:
            break
        time.sleep(0.0005)
    out[t] = got
st = srv.stats()
srv.close()
assert out[t1][1]["status"] == 0 and out[t2][1]["status"] == 0, (out[t1][1], out[t2][1])
assert st["deferred"] == 1, st
srv2 = s.Server(hbm_budget_bytes=4 << 30, max_slots=1)  # the same request alone
t = srv2.submit(small, precision="fp64")
for _ in range(600000):
    alone = srv2.poll(t)
    if alone is not None:
        break
    time.sleep(0.0005)
srv2.close()
np.testing.assert_array_equal(out[t2][0], alone[0])
print("DEFER-OK")
"""


def test_serve_defers_on_allocation_failure(spin):
    """A request whose device memory cannot be allocated while another one
    runs is put back at the head of the queue and admitted again when that
    one completes, instead of failing.  The allocation failures are made on
    the host (SPIN_SERVE_INJECT_OOM=ticket:count makes the first count
    attempts of that ticket fail); the result equals the request served
    alone."""
    import os
    import subprocess
    import sys

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, SPIN_SERVE_INJECT_OOM="2:2")
    r = subprocess.run([sys.executable, "-c", DEFER_SCRIPT], cwd=root, env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0 and "DEFER-OK" in r.stdout, r.stdout + r.stderr
