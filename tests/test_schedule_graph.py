"""The recursion's schedule as a CUDA graph: a call that repeats the previous
call's arguments captures the DAG of product and leaf launches (Algorithm 2's
driver), later ones replay it.  A replay runs the same kernels on the same
operands, so it is bitwise the direct launch sequence; it reads A's current
contents; and it is checked against the oracle's Algorithm 1."""
import numpy as np
import pytest

import bounds
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


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda:0")


@pytest.mark.parametrize("n,leaf", [(1024, 128), (1500, 200), (300, 64)])
def test_replay_bitwise_and_against_oracle(spin, n, leaf):
    A_h = inputs.sdd(n, seed=inputs.SEED_BASE + 40 + n)
    A = dev(A_h)
    X = torch.empty_like(A)
    before = spin.schedule_stats()["replays"]
    outs = []
    for _ in range(4):  # direct, capture + replay, replay, replay
        spin.invert(A, leaf=leaf, out=X)
        outs.append(X.cpu().numpy().copy())
    st = spin.schedule_stats()
    assert st["replays"] - before == 3
    assert st["nodes"] > 0
    for x in outs[1:]:
        np.testing.assert_array_equal(x, outs[0])
    ref, _ = oracle.strassen_inv(A_h, leaf)
    assert np.linalg.norm(outs[0] - ref) / np.linalg.norm(ref) <= 64 * n * np.linalg.cond(A_h) * U
    assert bounds.elementwise_ok(outs[0], ref, A_h)
    # the replay reads A as it is now: scaling by 2^-3 scales X by 2^3 exactly
    A.mul_(0.125)
    spin.invert(A, leaf=leaf, out=X)
    assert spin.schedule_stats()["replays"] - before == 4
    np.testing.assert_array_equal(X.cpu().numpy(), outs[0] * 8.0)


def test_replay_reports_status(spin):
    """A singular leading block found during a replay is reported as in a
    direct call (leaf and column of the failing pivot)."""
    n, leaf = 512, 128
    A_h = inputs.sdd(n, seed=inputs.SEED_BASE + 41)
    A = dev(A_h)
    X = torch.empty_like(A)
    for _ in range(3):
        _, info = spin.invert(A, leaf=leaf, out=X)
        assert info["status"] == 0
    A[:, 5] = 0.0  # column 5 of the first leaf is zero
    _, info = spin.invert(A, leaf=leaf, out=X, check=False)
    assert info["status"] != 0 and info["fail_leaf"] == 0 and info["fail_col"] == 5
    A.copy_(dev(A_h))
    _, info = spin.invert(A, leaf=leaf, out=X)
    assert info["status"] == 0


def test_mixed_replay_matches_direct(spin):
    """The mixed form (tensor-core products, device-decided refinement) as a
    captured schedule: the same result and the same refinement record."""
    n = 2048
    A = inputs.spd_gram_device(n, inputs.SEED_BASE + 42, "cuda:0", alpha=1.0)
    X = torch.empty_like(A)
    res = []
    for _ in range(3):
        _, info = spin.invert(A, precision="bf16x3", out=X)
        res.append((X.cpu().numpy().copy(), info["refine_iters"], info["rel_residual"]))
    for x, it, r in res[1:]:
        assert it == res[0][1]
        assert abs(r - res[0][2]) <= 1e-12 * res[0][2]  # norm sums use atomics
        assert np.max(np.abs(x - res[0][0])) <= 1e-13 * np.max(np.abs(res[0][0]))
    A_h = A.cpu().numpy()
    assert oracle.residual(A_h, res[-1][0])[0] <= 1e-10


def test_other_arguments_launch_directly(spin):
    """A call with other arguments runs directly and keeps the captured
    graph's count of replays unchanged."""
    A = dev(inputs.sdd(256, seed=inputs.SEED_BASE + 43))
    X1 = torch.empty_like(A)
    X2 = torch.empty_like(A)
    before = spin.schedule_stats()["replays"]
    for i in range(6):  # alternating outputs: no call repeats the previous one
        spin.invert(A, leaf=64, out=X1 if i % 2 == 0 else X2)
    assert spin.schedule_stats()["replays"] == before
    np.testing.assert_array_equal(X1.cpu().numpy(), X2.cpu().numpy())


@pytest.mark.parametrize("precision,n,leaf", [("fp64", 1500, 128), ("fp64", 700, 64), ("bf16x3", 1500, 128),
                                              ("bf16x3", 2048, 128), ("digits", 1024, 128)])
def test_second_stream_schedule_matches_one_stream(spin, precision, n, leaf):
    """Each level's II and C21 on a second stream (the default up to order
    8192 plain, 16384 mixed; schedule "persistent" forces it) against the
    one-stream order of Algorithm 1 (schedule "lockstep"): the same products
    on the same operands, so the same inverse -- bit for bit in FP64; in the
    mixed forms the same refinement steps and the same X up to the order of
    the atomically summed norms that decide them."""
    A = inputs.spd_gram_device(n, inputs.SEED_BASE + 77 + n, "cuda:0", alpha=1.0)
    out = {}
    for sched in ("lockstep", "default", "persistent"):
        X, info = spin.invert(A, precision=precision, leaf=leaf, schedule=sched)
        torch.cuda.synchronize()
        assert info["status"] == 0
        out[sched] = (X.cpu().numpy(), info["refine_iters"])
        assert spin.workspace_bytes(n, leaf=leaf, precision=precision, schedule=sched) > 0
    ref, it = out["lockstep"]
    for sched in ("default", "persistent"):
        x, it2 = out[sched]
        if precision == "fp64":
            np.testing.assert_array_equal(x, ref)
        else:
            assert it2 == it
            assert np.max(np.abs(x - ref)) <= 1e-13 * np.max(np.abs(ref))
    A_h = A.cpu().numpy()
    assert oracle.residual(A_h, out["default"][0])[0] <= (1e-13 if precision == "fp64" else 1e-10)
    # the second stream needs more workspace than one stream
    assert spin.workspace_bytes(n, leaf=leaf, precision=precision, schedule="persistent") > \
        spin.workspace_bytes(n, leaf=leaf, precision=precision, schedule="lockstep")
