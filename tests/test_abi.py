"""C-ABI library: loads, exports what include/swept.h declares, validates
configurations, and its swept schedule passes the host-side symbolic check
(no GPU work in this file)."""
import ctypes
import os
import re

import pytest

from paper_1612_02495_gb300 import build as libbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def S():
    libbuild.build()
    from paper_1612_02495_gb300 import swept

    return swept


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"^\s*(?:swept_status|void)\s+(\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol(S):
    names = declared_functions()
    assert "swept_init" in names and "classic_step_n" in names and len(names) >= 12
    lib = ctypes.CDLL(S.LIB_PATH)
    for n in names:
        assert hasattr(lib, n), n


def test_binding_names_match_header(S):
    for n in declared_functions():
        assert hasattr(S, n), n


def cfg(S, scheme=None, **kw):
    base = dict(scheme=S.KS if scheme is None else scheme, dtype=S.F64, n=1024, dx=0.785, dt=0.005, param0=1.0)
    base.update(kw)
    return S.make_config(**base)


@pytest.mark.parametrize("bad", [
    dict(n=0), dict(n=-5), dict(dx=0.0), dict(dt=-1.0), dict(tile_w=12), dict(tile_w=4096),
    dict(tile_w=1000), dict(threads=48), dict(threads=2048), dict(dtype=7), dict(scheme=9),
    dict(bc=1),  # KS is periodic only
    dict(warp_tiles=2),
    dict(warp_tiles=1, tile_w=96), dict(warp_tiles=1, tile_w=512),  # W / 32 must be 1, 2, 4 or 8
    dict(warp_tiles=1, tile_w=64, threads=64), dict(warp_tiles=1, tile_w=64, chunk=3),
    dict(warp_tiles=1, scheme=2, tile_w=64, param0=1.4, bc=1),  # Euler keeps its tiers in shared memory
    dict(chunk=3, scheme=2, tile_w=64, param0=1.4, bc=1),  # Euler: one or two threads per face
    dict(chunk=3), dict(chunk=5),  # heat/KS: one or two points a trip
])
def test_init_rejects_invalid_configs(S, bad):
    if bad.get("scheme") == 2:
        bad = dict(bad, scheme=S.EULER)
    c = cfg(S, **bad)
    h = ctypes.c_void_p()
    assert S.swept_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_EINVAL
    assert not h.value


def test_init_rejects_null(S):
    h = ctypes.c_void_p()
    assert S.swept_init(None, ctypes.byref(h)) == S.SWEPT_EINVAL


def test_plan_report(S):
    h = S.init(cfg(S, n=1 << 20))
    p = S.plan(h)
    assert p["radius"] == 2 and p["stages"] == 2 and p["components"] == 1
    assert p["half_cycle"] * 2 * p["radius"] == p["tile_w"]
    assert p["tiles"] * p["tile_w"] == 1 << 20
    assert p["smem_bytes"] == 2 * (p["tile_w"] + 4) * 8
    S.swept_free(h)


def test_heat_config_plan(S):
    h = S.init(S.make_config(S.HEAT, S.F64, 1024, 0.006, 1e-5, 1.0, tile_w=64))
    p = S.plan(h)
    assert p["tile_w"] == 64 and p["half_cycle"] == 32 and p["tiles"] == 16
    S.swept_free(h)


def test_compute_calls_fail_without_workspace(S):
    h = S.init(cfg(S))
    buf = ctypes.c_void_p(0x1000)
    assert S.swept_step_n(h, buf, 10, None) == S.SWEPT_ENOWORKSPACE
    assert S.classic_step_n(h, None, 10, None) == S.SWEPT_EINVAL
    assert S.swept_step_n(h, buf, -1, None) == S.SWEPT_EINVAL
    S.swept_free(h)


def test_free_null_is_noop(S):
    S.swept_free(None)


SCHED = [
    # scheme, bc, W, tiles
    (0, 0, 4, 2), (0, 0, 8, 3), (0, 0, 16, 5), (0, 1, 4, 2), (0, 1, 8, 3), (0, 1, 32, 4),
    (1, 0, 8, 2), (1, 0, 16, 3), (1, 0, 32, 5),
    (2, 0, 8, 2), (2, 1, 8, 3), (2, 1, 16, 5), (2, 1, 32, 2),
]


@pytest.mark.parametrize("scheme,bc,W,nt", SCHED)
def test_schedule_symbolic_replay(S, scheme, bc, W, nt):
    """Every (point, sub-timestep) is computed once, after its stencil inputs,
    with no race between blocks, for full passes, remainders and both BCs."""
    n = W * nt
    h = S.init(S.make_config(scheme, S.F64, n, 0.1, 1e-3, 1.4 if scheme == 2 else 1.0, bc=bc, tile_w=W))
    Sst = 1 if scheme == 0 else 2
    rr = 1 if scheme == 0 else 2
    hh = W // (2 * rr)
    for nsteps in sorted({0, 1, 2, 3, hh // Sst, hh // Sst + 1, 2 * hh // Sst + 1, 7 * hh // Sst + 3, 45}):
        assert S.check_schedule(h, nsteps) == n * nsteps * Sst
    S.swept_free(h)


def test_schedule_large_pass_count(S):
    """Enough passes to use the chunked graph path (head + repeated body + tail)."""
    h = S.init(S.make_config(S.HEAT, S.F64, 64, 0.1, 1e-3, 1.0, tile_w=16))
    assert S.check_schedule(h, 8 * 1100 + 5) == 64 * (8 * 1100 + 5)
    S.swept_free(h)


def test_batch_plan_layout_on_host(S):
    from paper_1612_02495_gb300 import inputs

    probs = inputs.batch_instances(inputs.batch_problems(count=16, seed=9, log2_hi=13, steps_lo=1, steps_hi=60))
    arr = (S.swept_batch_problem * len(probs))()
    for i, q in enumerate(probs):
        a = arr[i]
        a.scheme, a.n, a.nsteps, a.dx, a.dt, a.param = q["scheme"], q["n"], q["nsteps"], q["dx"], q["dt"], q["param"]
    h = ctypes.c_void_p()
    assert S.swept_batch_plan(arr, len(probs), S.F64, 0, ctypes.byref(h)) == S.SWEPT_OK
    offs = (ctypes.c_int64 * len(probs))()
    sv, wb, items = ctypes.c_int64(), ctypes.c_size_t(), ctypes.c_int64()
    assert S.swept_batch_sizes(h, offs, ctypes.byref(sv), ctypes.byref(wb), ctypes.byref(items)) == S.SWEPT_OK
    offs = list(offs)
    # states are disjoint, ordered, 64-value aligned and cover the layout
    for i, q in enumerate(probs):
        assert offs[i] % 64 == 0
        if i:
            assert offs[i] >= offs[i - 1] + probs[i - 1]["n"]
    assert sv.value >= offs[-1] + probs[-1]["n"]
    # items = sum over problems of tiles x passes (default tile 512)
    want = 0
    for q in probs:
        R, Sst = (1, 1) if q["scheme"] == 0 else (2, 2)
        W = 512
        hh = W // (2 * R)
        n_sub = q["nsteps"] * Sst
        npass = (n_sub // hh + 1 if n_sub // hh else 0) + (2 if n_sub % hh else 0)
        want += (q["n"] // W) * npass
    assert items.value == want
    S.swept_batch_free(h)


@pytest.mark.parametrize("bad", [dict(n=1002), dict(scheme=2), dict(nsteps=-1), dict(tile_w=24), dict(dt=0.0)])
def test_batch_plan_rejects_invalid(S, bad):
    q = dict(scheme=1, tile_w=0, n=2048, nsteps=10, dx=0.785, dt=0.005, param=1.0)
    q.update(bad)
    arr = (S.swept_batch_problem * 1)()
    a = arr[0]
    a.scheme, a.tile_w, a.n, a.nsteps, a.dx, a.dt, a.param = (q["scheme"], q["tile_w"], q["n"], q["nsteps"],
                                                              q["dx"], q["dt"], q["param"])
    h = ctypes.c_void_p()
    assert S.swept_batch_plan(arr, 1, S.F64, 0, ctypes.byref(h)) == S.SWEPT_EINVAL


def test_autotune_tile_candidates(S):
    from paper_1612_02495_gb300 import autotune

    c = autotune.tile_candidates(S.KS, 1 << 20)
    assert c == [64, 128, 256, 512, 1024]
    assert autotune.tile_candidates(S.HEAT, 1024) == [32, 64, 128, 256, 512]
    assert autotune.tile_candidates(S.KS, 64) == [32]
    # a non-power-of-two size keeps its legal divisors (multiples of 4r, >= 2 tiles)
    c = autotune.tile_candidates(S.KS, 3 * 1000)
    assert c and all(3000 % w == 0 and w % 8 == 0 and 3000 // w >= 2 for w in c)
    # with no divisor, the powers of two that leave at least two tiles
    assert autotune.tile_candidates(S.KS, 65537) == [64, 128, 256, 512, 1024]
    assert autotune.tile_candidates(S.HEAT, 1009) == [32, 64, 128, 256]


@pytest.mark.parametrize("scheme,W", [("heat", 32), ("heat", 64), ("heat", 256), ("ks", 64), ("ks", 128), ("ks", 256)])
def test_warp_tiles_plan(S, scheme, W):
    sc = S.HEAT if scheme == "heat" else S.KS
    c = cfg(S, scheme=sc, n=8 * W, tile_w=W, warp_tiles=1)
    h = ctypes.c_void_p()
    assert S.swept_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_OK
    p = S.plan(h.value)
    assert p["warp_tiles"] == 1 and p["threads"] == 32 and p["tile_w"] == W
    # the schedule itself is unchanged: the host replay still covers every point once
    assert S.check_schedule(h.value, 3 * W + 5) == 8 * W * (3 * W + 5) * (1 if scheme == "heat" else 2)
    S.swept_free(h.value)


def test_integer_minmod_rule_matches_comparison_form():
    """The kernels' minmod and wave-speed maximum select by IEEE bit patterns;
    check that rule against the comparison form (the oracle's) on special
    values and random doubles and floats of every magnitude."""
    import numpy as np

    def ref(a, b):
        if a > 0 and b > 0:
            return a if a <= b else b
        if a < 0 and b < 0:
            return a if a >= b else b
        return 0.0

    def bits_rule(a, b, itype, mag):
        ia, ib = np.array([a]).view(itype)[0], np.array([b]).view(itype)[0]
        same = ((ia ^ ib) >= 0) and (ia & mag) != 0 and (ib & mag) != 0
        return (a if ia <= ib else b) if same else 0.0

    g = np.random.default_rng(3)
    for ftype, itype, mag in ((np.float64, np.int64, np.int64(0x7fffffffffffffff)),
                              (np.float32, np.int32, np.int32(0x7fffffff))):
        fi = np.finfo(ftype)
        special = [0.0, -0.0, fi.tiny, -fi.tiny, fi.tiny / 4, -fi.tiny / 4, 1.0, -1.0, fi.max, -fi.max, np.inf, -np.inf]
        rand = list(g.standard_normal(400) * np.exp(g.uniform(-30, 30, 400)))
        vals = [ftype(v) for v in special + rand]
        for a in vals[:60]:
            for b in vals:
                r = ftype(ref(a, b))
                got = ftype(bits_rule(a, b, itype, mag))
                assert r.tobytes() == got.tobytes(), (a, b, r, got)
        for a in vals:
            for b in vals[:40]:
                if a >= 0 and b >= 0 and not np.signbit(a) and not np.signbit(b):
                    want = a if a >= b else b
                    ia, ib = np.array([a]).view(itype)[0], np.array([b]).view(itype)[0]
                    assert (a if ia >= ib else b) == want


def test_schedule_replay_random_configurations(S):
    """Seeded sweep of the 1D host replay over random schemes, boundary conditions,
    tile widths, tile counts and step counts (including remainders and a single
    full pass)."""
    import numpy as np

    g = np.random.default_rng(20161208)
    for _ in range(60):
        scheme = int(g.integers(0, 3))
        R = 1 if scheme == S.HEAT else 2
        W = 4 * R * int(g.integers(1, 9))
        nt = int(g.integers(2, 7))
        bc = 0 if scheme == S.KS else int(g.integers(0, 2))
        S_ = 1 if scheme == S.HEAT else 2
        h = W // (2 * R)
        nsteps = int(g.choice([1, max(1, h // S_), int(g.integers(1, 4 * h))]))
        param = 1.4 if scheme == S.EULER else 1.0
        c = cfg(S, scheme=scheme, n=nt * W, tile_w=W, bc=bc, param0=param)
        h_ = ctypes.c_void_p()
        assert S.swept_init(ctypes.byref(c), ctypes.byref(h_)) == S.SWEPT_OK
        assert S.check_schedule(h_.value, nsteps) == nt * W * nsteps * S_, (scheme, W, nt, bc, nsteps)
        S.swept_free(h_.value)


def test_schedule_replay_ragged_grids(S):
    """Grids that are not a multiple of the tile width (the last tile wider by
    X = n mod W, its flat top handed from pass to pass): seeded sweep of both
    replays (launch sequence and persistent queue) over schemes, boundaries,
    tile widths, X in [1, W), tile counts and step counts."""
    import numpy as np

    g = np.random.default_rng(1009)
    for _ in range(80):
        scheme = int(g.integers(0, 3))
        R = 1 if scheme == S.HEAT else 2
        W = 4 * R * int(g.integers(1, 7))
        nt = int(g.integers(2, 8))
        X = int(g.integers(1, W))
        n = nt * W + X
        bc = 0 if scheme == S.KS else int(g.integers(0, 2))
        S_ = 1 if scheme == S.HEAT else 2
        h = W // (2 * R)
        nsteps = int(g.choice([1, max(1, h // S_), int(g.integers(1, 5 * h))]))
        for persistent in (0, 1):
            c = cfg(S, scheme=scheme, n=n, tile_w=W, bc=bc, param0=1.4 if scheme == S.EULER else 1.0,
                    persistent=persistent)
            hh = ctypes.c_void_p()
            assert S.swept_init(ctypes.byref(c), ctypes.byref(hh)) == S.SWEPT_OK
            p = S.plan(hh.value)
            assert (p["tiles"], p["last_tile_extra"]) == (nt, X)
            k = ctypes.c_int64()
            st = S.swept_check_schedule(hh.value, nsteps, ctypes.byref(k))
            assert st == S.SWEPT_OK, (S.last_error(hh.value), scheme, W, nt, X, bc, nsteps, persistent)
            assert k.value == n * nsteps * S_
            S.swept_free(hh.value)


@pytest.mark.parametrize("n", [1009, 4099, 65537])
@pytest.mark.parametrize("scheme,bc", [("heat", 0), ("heat", 1), ("ks", 0), ("euler", 0), ("euler", 1)])
def test_schedule_replay_prime_grids(S, n, scheme, bc):
    """The ragged sizes of the GPU parity tests, with the library's default
    tile and with a 64-point tile in the persistent queue: both replays pass."""
    sc = {"heat": S.HEAT, "ks": S.KS, "euler": S.EULER}[scheme]
    S_ = 1 if sc == S.HEAT else 2
    param = 1.4 if sc == S.EULER else 1.0
    for W, persistent, nsteps in ((0, 0, 77), (64, 0, 203), (64 if n < 5000 else 1024, 1, 41)):
        h = S.init(cfg(S, scheme=sc, n=n, tile_w=W, bc=bc, param0=param, persistent=persistent))
        p = S.plan(h)
        assert p["tiles"] * p["tile_w"] + p["last_tile_extra"] == n and p["last_tile_extra"] > 0
        assert S.check_schedule(h, nsteps) == n * nsteps * S_
        S.swept_free(h)


def test_default_tile_prefers_a_divisor(S):
    """The library keeps a tile that divides n when one exists (no wide tile)."""
    for n in (1 << 14, 3 * 1000, 1 << 20):
        p = S.plan(S.init(cfg(S, n=n)))
        assert p["last_tile_extra"] == 0 and n % p["tile_w"] == 0


@pytest.mark.parametrize("scheme,n", [("heat", 3), ("heat", 7), ("ks", 5), ("ks", 15), ("euler", 5), ("euler", 15)])
def test_tiny_grids_get_a_classic_only_handle(S, scheme, n):
    """Any n >= 2r + 1 is a valid problem; below two tiles of 4r points the
    handle exists for classic_step_n, and the swept calls say so."""
    sc = {"heat": S.HEAT, "ks": S.KS, "euler": S.EULER}[scheme]
    c = cfg(S, scheme=sc, n=n, param0=1.4 if sc == S.EULER else 1.0, bc=1 if sc == S.EULER else 0)
    h = S.init(c)
    assert S.plan(h)["tiles"] == 0
    assert S.swept_check_schedule(h, 3, None) == S.SWEPT_EUNSUPPORTED
    S.swept_free(h)
    bad = cfg(S, scheme=sc, n=2 * (1 if sc == S.HEAT else 2), param0=1.4 if sc == S.EULER else 1.0)
    hb = ctypes.c_void_p()
    assert S.swept_init(ctypes.byref(bad), ctypes.byref(hb)) == S.SWEPT_EINVAL
    for extra in (dict(persistent=1), dict(cluster=1), dict(tile_w=8 if sc == S.HEAT else 16)):
        c2 = cfg(S, scheme=sc, n=n, param0=1.4 if sc == S.EULER else 1.0, **extra)
        assert S.swept_init(ctypes.byref(c2), ctypes.byref(hb)) == S.SWEPT_EINVAL, extra


def test_ragged_grids_refuse_cluster_and_warp_tiles(S):
    for extra in (dict(cluster=1, tile_w=64), dict(warp_tiles=1, tile_w=64)):
        c = cfg(S, n=3 * 64 + 8, **extra)
        h = ctypes.c_void_p()
        assert S.swept_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_EINVAL, extra


@pytest.mark.parametrize("option,value", [(0, 5), (3, 1), (1, 0), (1, 1 << 33), (2, -1)])
def test_set_option_rejects_invalid(S, option, value):
    c = cfg(S, n=1024, tile_w=64, persistent=1)
    h = ctypes.c_void_p()
    assert S.swept_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_OK
    assert S.swept_set_option(h.value, option, value) == S.SWEPT_EINVAL
    assert S.swept_set_option(h.value, S.SWEPT_OPT_SPIN_LIMIT, 5000) == S.SWEPT_OK
    assert S.swept_set_option(h.value, S.SWEPT_OPT_START_ITEM, 3) == S.SWEPT_OK
    S.swept_free(h.value)


def test_persistent_schedule_replay(S):
    """For a persistent handle swept_check_schedule replays the persistent kernel's
    item queue and checks the happens-before order its waits create (every read
    after its writer; every overwrite after the previous writer and its readers),
    besides the value flow.  Seeded sweep over schemes, boundaries, tile counts and
    step counts (full passes, remainders, remainder only)."""
    import numpy as np

    g = np.random.default_rng(1208)
    for _ in range(40):
        scheme = int(g.integers(0, 3))
        R = 1 if scheme == S.HEAT else 2
        W = 4 * R * int(g.integers(1, 6))
        nt = int(g.integers(2, 9))
        bc = 0 if scheme == S.KS else int(g.integers(0, 2))
        S_ = 1 if scheme == S.HEAT else 2
        h = W // (2 * R)
        nsteps = int(g.choice([1, max(1, h // S_), int(g.integers(1, 5 * h))]))
        c = cfg(S, scheme=scheme, n=nt * W, tile_w=W, bc=bc, param0=1.4 if scheme == S.EULER else 1.0, persistent=1)
        hh = ctypes.c_void_p()
        assert S.swept_init(ctypes.byref(c), ctypes.byref(hh)) == S.SWEPT_OK
        n = ctypes.c_int64()
        st = S.swept_check_schedule(hh.value, nsteps, ctypes.byref(n))
        assert st == S.SWEPT_OK, S.last_error(hh.value)
        assert n.value == nt * W * nsteps * S_
        S.swept_free(hh.value)
