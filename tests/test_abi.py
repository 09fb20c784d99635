"""Host-side checks of the C ABI (no GPU needed): the library builds for
sm_103a, loads, exports every function ``include/spin.h`` declares, and its
host logic (defaults, workspace sizing, argument validation) behaves."""
import ctypes
import os
import re

import pytest

import paper_1801_04723_gb300 as spin
from paper_1801_04723_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    spin.build()
    return binding.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "spin.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(spin_[a-z0-9_]+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_entry_points():
    names = declared_functions()
    for must in ("spin_invert", "spin_invert_ex", "spin_workspace_bytes", "spin_leaf_inverse", "spin_gemm_f64",
                 "spin_invert_host", "spin_status_string"):
        assert must in names


def test_every_declared_symbol_is_exported(L):
    missing = [n for n in declared_functions() if not hasattr(L, n)]
    assert not missing, missing


def test_defaults(L):
    o = L.spin_opts_default()
    assert o.precision == 0 and o.leaf == 0 and o.tol == 1e-10 and o.max_refine == 6
    assert o.fp64_levels == 2 and o.blocking == 1 and o.workspace is None
    assert L.spin_version() >= 100
    assert L.spin_status_string(0) == b"SPIN_OK"
    assert L.spin_status_string(2) == b"SPIN_ERR_SINGULAR"


def split(n):
    return 32 * ((n + 63) // 64) if n > 64 else (n + 1) // 2


def ws_elems(n, leaf, overlap=False):
    # per node T (n1 x n2) and S (n2 x n2); the overlapped schedule (plain
    # method, orders up to 8192) adds II (n2 x n1)
    if n <= leaf:
        return n * n if n > 256 else 0
    n1 = split(n)
    n2 = n - n1
    return max(ws_elems(n1, leaf, overlap), n1 * n2 + n2 * n2 + (n2 * n1 if overlap else 0) + ws_elems(n2, leaf, overlap))


@pytest.mark.parametrize("n,leaf", [(1, 1), (2, 1), (1024, 128), (1000, 64), (777, 100), (32768, 512),
                                    (8192, 2048), (4096, 4096), (65, 8), (8193, 512)])
def test_workspace_bytes(L, n, leaf):
    assert spin.workspace_bytes(n, leaf=leaf) == 8 * ws_elems(n, leaf, overlap=n <= 8192)


def test_workspace_power_of_two_is_two_thirds_n2(L):
    n, leaf = 1 << 14, 1 << 7  # above 8192: the sequential schedule, 2 n^2 / 3
    assert abs(spin.workspace_bytes(n, leaf=leaf) / 8 - 2 * n * n / 3) < n * n / 1000
    n = 1 << 13  # the overlapped schedule: n^2
    assert abs(spin.workspace_bytes(n, leaf=leaf) / 8 - n * n) < n * n / 1000


def test_invalid_arguments_rejected_on_host(L):
    o = binding.make_opts()
    info = binding.Info()
    vp = ctypes.c_void_p
    buf = (ctypes.c_double * 64)()
    a = vp(ctypes.addressof(buf))
    x = vp(ctypes.addressof(buf) + 8 * 32)
    # n < 1, lda < n, NULL pointers, misaligned pointer, negative leaf, overlap, bad precision
    assert L.spin_invert_ex(a, 4, x, 4, 0, ctypes.byref(o), ctypes.byref(info), None) == 1
    assert L.spin_invert_ex(a, 3, x, 4, 4, ctypes.byref(o), ctypes.byref(info), None) == 1
    assert L.spin_invert_ex(None, 4, x, 4, 4, ctypes.byref(o), ctypes.byref(info), None) == 1
    assert L.spin_invert_ex(vp(ctypes.addressof(buf) + 4), 4, x, 4, 4, ctypes.byref(o), ctypes.byref(info), None) == 1
    assert L.spin_invert_ex(a, 4, vp(ctypes.addressof(buf) + 8), 4, 4, ctypes.byref(o), ctypes.byref(info), None) == 1
    o.leaf = -3
    assert L.spin_invert_ex(a, 4, x, 4, 4, ctypes.byref(o), ctypes.byref(info), None) == 1
    o.leaf = 0
    o.precision = 9
    assert L.spin_invert_ex(a, 4, x, 4, 4, ctypes.byref(o), ctypes.byref(info), None) == 1
    o.precision = 2  # not a precision of spin_precision
    assert L.spin_invert_ex(a, 4, x, 4, 4, ctypes.byref(o), ctypes.byref(info), None) == 1
    # gemm: alpha/beta outside {+-1} x {0,1}
    assert L.spin_gemm_f64(4, 4, 4, 2.0, a, 4, a, 4, 0.0, None, 0, x, 4, None) == 1
    assert L.spin_gemm_f64(4, 4, 4, 1.0, a, 4, a, 4, 1.0, None, 0, x, 4, None) == 1
    # leaf order above the supported maximum
    assert L.spin_leaf_inverse(a, 5000, x, 5000, 5000, None, None) == 1
    # batched: a schedule outside 0..2, or the persistent schedule with a leaf above 64
    ptrs = (ctypes.c_void_p * 1)(ctypes.addressof(buf))
    outs = (ctypes.c_void_p * 1)(ctypes.addressof(buf) + 8 * 32)
    lds = (ctypes.c_int64 * 1)(4)
    ns = (ctypes.c_int64 * 1)(4)
    ob = binding.make_opts(schedule=3)
    assert L.spin_invert_batched(ptrs, lds, outs, ns, 1, ctypes.byref(ob), None, None) == 1
    ob = binding.make_opts(schedule="persistent", leaf=128)
    assert L.spin_invert_batched(ptrs, lds, outs, ns, 1, ctypes.byref(ob), None, None) == 1
    # leaf exchange timeout hook: order outside 2..256, limit outside (0, 4000] ms
    L.spin_test_leaf_timeout.argtypes = [ctypes.c_int64, ctypes.c_int, ctypes.c_double]
    assert L.spin_test_leaf_timeout(1, 0, 50.0) == 1
    assert L.spin_test_leaf_timeout(300, 0, 50.0) == 1
    assert L.spin_test_leaf_timeout(128, 0, 0.0) == 1
    assert L.spin_test_leaf_timeout(128, 0, 5000.0) == 1
    # persistent batch timeout hook: limit outside (0, 4000] ms, NULL outputs
    s0, s1 = ctypes.c_int(), ctypes.c_int()
    assert L.spin_test_persistent_timeout(0.0, ctypes.byref(s0), ctypes.byref(s1)) == 1
    assert L.spin_test_persistent_timeout(5000.0, ctypes.byref(s0), ctypes.byref(s1)) == 1
    assert L.spin_test_persistent_timeout(50.0, None, ctypes.byref(s1)) == 1
    # persistent autotuner: a leaf above 64, a tile that is not 16, 32 or 64, no candidates
    orders = (ctypes.c_int64 * 2)(64, 128)
    lo, to, ms = (ctypes.c_int * 2)(), (ctypes.c_int * 2)(), (ctypes.c_double * 2)()
    for leaves, tiles in (((65,), (64,)), ((32,), (48,)), ((0,), (64,))):
        la = (ctypes.c_int * 1)(*leaves)
        ta = (ctypes.c_int * 1)(*tiles)
        assert L.spin_autotune_batched_persistent(orders, 2, la, 1, ta, 1, lo, to, ms, None) == 1
    la = (ctypes.c_int * 1)(32)
    ta = (ctypes.c_int * 1)(64)
    assert L.spin_autotune_batched_persistent(orders, 2, la, 0, ta, 1, lo, to, ms, None) == 1


def test_pretransform_workspace(L):
    # the butterfly transform adds its diagonals, U^T A V and the inverse of
    # it (order padded to a multiple of 4) to the recursion's workspace
    n = 1001
    np_ = 1004
    plain = spin.workspace_bytes(n, leaf=64)
    rbt = spin.workspace_bytes(n, leaf=64, pretransform=1)
    assert rbt >= 2 * np_ * np_ * 8 + 4 * np_ * 8 + spin.workspace_bytes(np_, leaf=64)
    assert spin.workspace_bytes(n, leaf=64, pretransform=2) == max(plain, rbt)


def test_cost_model_shape(L):
    """The model of the plain path (spin_model_seconds): never faster than the
    FP64 peak allows, U-shaped in the leaf order with the optimum of the
    measured sweeps (a flat bottom at 64-128 at n = 4096 and 8192, within 1 %
    of each other), growing like n^3, and the untuned default leaf is its
    optimum."""
    peak = 152 * 4 * 2.07e9
    for n in (8192, 16384):
        t = {Lf: spin.model_seconds(n, Lf) for Lf in (64, 128, 256, 512, 1024, 2048)}
        assert all(v >= 2.0 * n ** 3 / peak for v in t.values())
        best = min(t, key=t.get)
        assert best in (64, 128)
        assert t[best] < t[256] < t[512] < t[1024] < t[2048]
        assert spin.default_leaf(n) == best
    r = spin.model_seconds(16384, 256) / spin.model_seconds(8192, 256)
    assert 7.0 < r < 8.0
    assert spin.model_seconds(100, 64, precision="bf16x3") == -1.0


def test_workspace_follows_the_schedule(L):
    """Workspace sizing per schedule (host logic): one stream needs T and S
    per level, n1 n2 + n2^2 = n^2 / 2 for n = 2^p, i.e. n^2 (1/2)(1 + 1/4 +
    ...) down to the leaf; the two-stream schedule adds II (n2 n1) per level,
    3 n^2 / 4.  The plain method takes the second stream up to order 8192
    by default, the mixed forms up to 16384, and everywhere when forced."""
    n, leaf = 1024, 128
    levels = [n, n // 2, n // 4]  # orders above the leaf
    one = 8 * sum(m * m // 2 for m in levels)
    two = 8 * sum(3 * m * m // 4 for m in levels)
    assert spin.workspace_bytes(n, leaf=leaf, schedule="lockstep") == one
    assert spin.workspace_bytes(n, leaf=leaf, schedule="default") == two
    assert spin.workspace_bytes(n, leaf=leaf, schedule="persistent") == two
    big = 16384
    assert spin.workspace_bytes(big, leaf=leaf, schedule="default") == \
        spin.workspace_bytes(big, leaf=leaf, schedule="lockstep")
    assert spin.workspace_bytes(big, leaf=leaf, schedule="persistent") > \
        spin.workspace_bytes(big, leaf=leaf, schedule="lockstep")
    for m in (1024, 16384):
        mixed = {s: spin.workspace_bytes(m, leaf=leaf, precision="bf16x3", schedule=s)
                 for s in ("lockstep", "default", "persistent")}
        assert mixed["default"] == mixed["persistent"] > mixed["lockstep"]
    assert spin.workspace_bytes(32768, leaf=leaf, precision="bf16x3", schedule="default") == \
        spin.workspace_bytes(32768, leaf=leaf, precision="bf16x3", schedule="lockstep")
    # a schedule outside 0..2 is refused: no workspace size
    o = binding.make_opts(schedule=3)
    assert L.spin_workspace_bytes(1024, ctypes.byref(o)) == 0
