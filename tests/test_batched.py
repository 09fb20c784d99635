"""spin_invert_batched against the oracle: a batch of matrices of uneven
orders (log-uniform, multiples of 32, as in the batching workload), each
result compared with the oracle's Algorithm 1 at the same leaf size."""
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


PERSIST_MAX_LEAF = 64


def leaf_rule(n, leaf=0):
    """Leaf of a bucket of order n in the lockstep form (and the library's
    default leaf)."""
    return min(leaf if leaf > 0 else (n if n <= 128 else 64), n)


def persistent_leaf(n, leaf=0):
    """Leaf of a bucket in the plain form's default, persistent schedule."""
    return min(leaf_rule(n, leaf), PERSIST_MAX_LEAF)


def check(A, X, leaf):
    ref, _ = oracle.strassen_inv(A, leaf)
    n = A.shape[0]
    tol = 64 * n * np.linalg.cond(A) * U
    assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= tol
    assert bounds.elementwise_ok(X, ref, A)
    assert oracle.residual(A, X)[0] <= 1e-13


def test_batch_uneven_orders(spin):
    orders = inputs.batch_orders(48, seed=inputs.SEED_BASE + 3)
    orders = np.concatenate([orders, [32, 32, 1024, 96, 1, 5, 130]])
    mats = [inputs.sdd(int(n), seed=1000 + i) for i, n in enumerate(orders)]
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, info = spin.invert_batched(As)
    torch.cuda.synchronize()
    assert int(info.abs().sum()) == 0
    for i in range(0, len(mats), 5):  # oracle on a sample of the batch
        check(mats[i], Xs[i].cpu().numpy(), persistent_leaf(len(mats[i])))


def test_batch_replay_strided_and_singular(spin):
    big = torch.zeros((700, 900), dtype=torch.float64, device="cuda:0")
    a0 = inputs.spd_gram(300, seed=5)
    big[10:310, 20:320] = torch.from_numpy(a0).cuda()
    sing = torch.tensor([[0.0, 1.0], [1.0, 0.0]], dtype=torch.float64, device="cuda:0")
    a2 = torch.from_numpy(inputs.sdd(64, seed=6)).cuda()
    As = [big[10:310, 20:320], sing, a2]
    Xs, info = spin.invert_batched(As)
    torch.cuda.synchronize()
    st = info.cpu().tolist()
    assert st[0] == 0 and st[2] == 0
    # order 2 with leaf 2 (n <= 128: the whole matrix is the leaf) pivots: not singular
    assert st[1] == 0
    np.testing.assert_array_equal(Xs[1].cpu().numpy(), sing.cpu().numpy())
    check(a0, Xs[0].cpu().numpy(), 64)
    first = [x.clone() for x in Xs]
    Xs2, info2 = spin.invert_batched(As, outs=Xs)  # same arguments: graph replay
    torch.cuda.synchronize()
    for a, b in zip(first, Xs2):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    # leaf 1 on the 2x2 permutation: A11 = 0 is singular
    Xs3, info3 = spin.invert_batched([sing, a2], leaf=1)
    torch.cuda.synchronize()
    assert info3.cpu().tolist()[0] == 2 and info3.cpu().tolist()[1] == 0


def test_batch_matches_single_calls(spin):
    mats = [inputs.spd_gram(n, seed=n) for n in (256, 256, 512, 320)]
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, info = spin.invert_batched(As, leaf=64)
    for a, x in zip(As, Xs):
        xs, _ = spin.invert(a, leaf=64)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(x.cpu().numpy(), xs.cpu().numpy())


def test_batch_mixed_precision(spin):
    """Mixed form: tensor-core level products (orders >= 256 reach them),
    FP64-class Schur complements and residuals, Newton-Schulz to 1e-10 for
    every matrix; residuals re-checked by the oracle and against each
    matrix's known inverse where it has one."""
    orders = [32, 96, 200, 256, 300, 512, 640, 1024, 1024, 384]
    mats, known = [], []
    for i, n in enumerate(orders):
        if i % 3 == 2:
            A, V, d = inputs.householder_spd(n, seed=inputs.SEED_BASE + 40 + i, reflectors=16, cond=1e3)
            mats.append(A)
            known.append((V, d))
        else:
            mats.append(inputs.sdd(n, seed=2000 + i))
            known.append(None)
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, info = spin.invert_batched(As, precision="bf16x3", tol=1e-10)
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0] * len(orders)
    ri = spin.batched_refine_info()
    assert 0 < ri["worst_rel_residual"] <= 1e-10
    for A, X, kn in zip(mats, Xs, known):
        X = X.cpu().numpy()
        assert oracle.residual(A, X)[0] <= 1e-10
        if kn is not None:
            ref = inputs.householder_apply(kn[0], 1.0 / kn[1], np.eye(A.shape[0]))
            assert np.linalg.norm(X - ref) / np.linalg.norm(ref) <= 1e3 * 10 * 1e-10


def test_batch_mixed_refinement_in_the_graph(spin):
    """The mixed batch is one graph replay: its kernel count includes every
    refinement round of every order bucket (3 launches to split A, then per
    round 6 for the residual and decision and 3 for the update, the last
    round without one), a non-blocking call only enqueues, and the results
    equal those of a blocking call bit for bit."""
    orders = [96, 300, 300, 512]
    mats = [inputs.sdd(n, seed=3000 + i) for i, n in enumerate(orders)]
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, info = spin.invert_batched(As, precision="bf16x3", tol=1e-10, blocking=False)
    torch.cuda.synchronize()
    st = spin.batched_stats()
    assert st["buckets"] == 3
    per_bucket = 3 + 7 * 6 + 6 * 3
    assert st["kernels"] >= st["buckets"] * per_bucket
    assert info.cpu().tolist() == [0] * len(orders)
    first = [x.cpu().numpy() for x in Xs]
    Xs2, _ = spin.invert_batched(As, precision="bf16x3", tol=1e-10)
    for a, x1, x2 in zip(mats, first, Xs2):
        np.testing.assert_array_equal(x1, x2.cpu().numpy())
        assert oracle.residual(a, x1)[0] <= 1e-10
    ri = spin.batched_refine_info()
    assert ri["refine_iters"] >= 1 and 0 < ri["worst_rel_residual"] <= 1e-10


def test_batch_mixed_result_independent_of_batch(spin):
    """Per-matrix decisions: a matrix inverted in a batch equals the same
    matrix inverted in a batch of its own, bit for bit."""
    mats = [inputs.householder_spd(384, seed=inputs.SEED_BASE + 60 + i, reflectors=16, cond=1e3)[0]
            for i in range(3)]
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, _ = spin.invert_batched(As, precision="bf16x3", tol=1e-10)
    together = [x.cpu().numpy() for x in Xs]
    for a, xt in zip(As, together):
        alone, _ = spin.invert_batched([a], precision="bf16x3", tol=1e-10)
        np.testing.assert_array_equal(alone[0].cpu().numpy(), xt)


def test_batch_mixed_strided_singular_and_replay(spin):
    big = torch.zeros((700, 900), dtype=torch.float64, device="cuda:0")
    a0 = inputs.spd_gram(300, seed=7)
    big[10:310, 20:320] = torch.from_numpy(a0).cuda()
    sing = np.eye(256)
    sing[:, 100] = 0.0  # a zero column: the leaf holding it fails
    a2 = inputs.sdd(512, seed=8)
    As = [big[10:310, 20:320], torch.from_numpy(sing).cuda(), torch.from_numpy(a2).cuda()]
    for _ in range(2):  # the second call replays the captured recursion
        Xs, info = spin.invert_batched(As, precision="bf16x3", tol=1e-10)
        torch.cuda.synchronize()
        st = info.cpu().tolist()
        assert st[0] == 0 and st[1] == 2 and st[2] == 0
        assert oracle.residual(a0, Xs[0].cpu().numpy())[0] <= 1e-10
        assert oracle.residual(a2, Xs[2].cpu().numpy())[0] <= 1e-10


def test_batch_autotuned_leaf(spin):
    """The batched autotuner picks each order bucket's leaf among the
    candidates; a batch with leaf 0 then runs every bucket at its recorded
    leaf (bitwise the same results as that leaf given explicitly, and the
    oracle's Algorithm 1 at that leaf), until the records are forgotten."""
    orders = [64] * 6 + [300] * 3 + [1024] * 2
    cands = (32, 64, 128)
    try:
        rec = spin.autotune_batched_leaf(orders, "fp64", candidates=cands)
        for o in set(orders):
            leaf, ms = rec[o]
            assert leaf in {min(c, o) for c in cands}
            assert ms > 0.0
        As = [inputs.sdd(o, seed=inputs.SEED_BASE + 700 + i) for i, o in enumerate(orders)]
        dev = [torch.from_numpy(a).cuda() for a in As]
        for schedule, cap in (("lockstep", None), ("default", PERSIST_MAX_LEAF)):
            X0, info = spin.invert_batched(dev, leaf=0, schedule=schedule)
            assert int(info.abs().sum()) == 0
            for o in set(orders):
                idx = [i for i, v in enumerate(orders) if v == o]
                want = rec[o][0] if cap is None else min(rec[o][0], cap)
                X1, info1 = spin.invert_batched([dev[i] for i in idx], leaf=want, schedule=schedule)
                assert int(info1.abs().sum()) == 0
                for i, x in zip(idx, X1):
                    assert torch.equal(X0[i], x)
            for i in (0, 6, 9):
                want = rec[orders[i]][0] if cap is None else min(rec[orders[i]][0], cap)
                check(As[i], X0[i].cpu().numpy(), want)
    finally:
        back = spin.autotune_batched_leaf(sorted(set(orders)), "fp64", candidates=())
    for o, (leaf, ms) in back.items():
        assert leaf == leaf_rule(o) and ms == -1.0


def test_batch_persistent_matches_lockstep(spin):
    """The plain batch as one persistent launch (a device-side task list of
    leaf inversions and product tiles, dependencies counted per matrix)
    against the lockstep launches: the same operations on every entry, so
    the same results bit for bit, at ragged orders, several leaves, strided
    inputs and a graph replay; a sample is checked against the oracle."""
    orders = [1, 5, 31, 33, 64, 96, 100, 130, 255, 300, 300, 511, 700, 1024]
    mats = [inputs.sdd(n, seed=3000 + i) if i % 2 else inputs.spd_gram(n, seed=3000 + i)
            for i, n in enumerate(orders)]
    big = torch.zeros((1100, 1300), dtype=torch.float64, device="cuda:0")
    big[3:703, 7:707] = torch.from_numpy(mats[12]).cuda()  # a strided view
    As = [torch.from_numpy(a).cuda() for a in mats]
    As[12] = big[3:703, 7:707]
    for leaf in (64, 32, 7):
        Xp, ip = spin.invert_batched(As, leaf=leaf, schedule="persistent")
        assert spin.batched_stats()["kernels"] == 2  # the persistent kernel and the status scatter
        Xl, il = spin.invert_batched(As, leaf=leaf, schedule="lockstep")
        torch.cuda.synchronize()
        assert ip.cpu().tolist() == [0] * len(orders) and il.cpu().tolist() == [0] * len(orders)
        for a, b in zip(Xp, Xl):
            assert torch.equal(a, b)
        first = [x.clone() for x in Xp]
        Xp2, _ = spin.invert_batched(As, leaf=leaf, schedule="persistent", outs=Xp)  # graph replay
        torch.cuda.synchronize()
        for a, b in zip(first, Xp2):
            assert torch.equal(a, b)
        for i in (0, 3, 7, 12, 13):
            check(mats[i], Xp[i].cpu().numpy(), min(leaf, orders[i]))


def test_batch_persistent_singular_matrix_only(spin):
    """A singular leaf in one matrix of a persistent batch is reported for
    that matrix alone (the others finish and are right)."""
    sing = inputs.sdd(200, seed=11)
    sing[40:80, :] = 0.0
    sing[:, 40:80] = 0.0  # A11 (leaf 64) has a zero column block: a zero pivot
    mats = [inputs.sdd(300, seed=12), sing, inputs.spd_gram(150, seed=13)]
    As = [torch.from_numpy(a).cuda() for a in mats]
    Xs, info = spin.invert_batched(As, leaf=64, schedule="persistent")
    torch.cuda.synchronize()
    st = info.cpu().tolist()
    assert st == [0, 2, 0]
    check(mats[0], Xs[0].cpu().numpy(), 64)
    check(mats[2], Xs[2].cpu().numpy(), 64)


def test_batch_persistent_wait_timeout(spin):
    """A dependency wait of the persistent kernel that runs out (a count
    that nothing reaches, 50 ms limit) ends the launch with
    SPIN_ERR_TIMEOUT for the matrices it left undone, without a fault or a
    hang; a persistent batch right after it is right."""
    assert spin.persistent_wait_timeout(50.0) == (6, 6)
    mats = [inputs.sdd(200, seed=21), inputs.spd_gram(96, seed=22)]
    Xs, info = spin.invert_batched([torch.from_numpy(a).cuda() for a in mats], schedule="persistent")
    torch.cuda.synchronize()
    assert info.cpu().tolist() == [0, 0]
    for a, x in zip(mats, Xs):
        check(a, x.cpu().numpy(), persistent_leaf(a.shape[0]))


def test_batch_persistent_autotuner(spin):
    """The persistent schedule's autotuner picks, per order bucket, a leaf
    and a largest product tile among the candidates; a plain batch with leaf
    0 then runs every bucket with them (bitwise the results of that leaf
    given explicitly: the tile never changes a bit), until forgotten."""
    orders = [64] * 6 + [300] * 3 + [1024] * 2
    try:
        rec = spin.autotune_batched_persistent(orders, leaves=(32, 64), tiles=(64, 32, 16))
        for o in set(orders):
            leaf, tile, ms = rec[o]
            assert leaf in {min(c, o) for c in (32, 64)} and tile in (16, 32, 64) and ms > 0.0
        As = [inputs.sdd(o, seed=inputs.SEED_BASE + 900 + i) for i, o in enumerate(orders)]
        dev = [torch.from_numpy(a).cuda() for a in As]
        X0, info = spin.invert_batched(dev, leaf=0, schedule="persistent")
        assert int(info.abs().sum()) == 0
        for o in set(orders):
            idx = [i for i, v in enumerate(orders) if v == o]
            X1, info1 = spin.invert_batched([dev[i] for i in idx], leaf=rec[o][0], schedule="lockstep")
            assert int(info1.abs().sum()) == 0
            for i, x in zip(idx, X1):
                assert torch.equal(X0[i], x)
        for i in (0, 6, 9):
            check(As[i], X0[i].cpu().numpy(), rec[orders[i]][0])
    finally:
        spin.autotune_batched_leaf(sorted(set(orders)), "fp64", candidates=())
