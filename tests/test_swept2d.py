"""2D swept decomposition (include/swept2d.h).

CPU (no GPU work): the configuration checks, and the host-side symbolic replay of
the 2D launch sequence over full half cycles, the final write-back, remainders,
non-square grids and every tile width: each point of each level computed once,
after its five inputs, with no race between the blocks of a launch.  The same
for the persistent queue, whose replay checks happens-before through the waits
(and finds the race that dropping a needed wait opens).

GPU: swept2d_step_n == classic2d_step_n == the CPU oracle (oracle.heat2d) bit for
bit, FP64 and FP32, over the same kinds of cases plus runs long enough to use
the cached body graph.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_1612_02495_gb300 import build as libbuild
from paper_1612_02495_gb300 import inputs


@pytest.fixture(scope="module")
def S():
    libbuild.build()
    from paper_1612_02495_gb300 import swept

    return swept


@pytest.mark.parametrize("bad", [
    dict(nx=100), dict(ny=20), dict(tile_w=12), dict(tile_w=6), dict(tile_w=128),  # 128 > 64 for FP64
    dict(nx=64, tile_w=64), dict(threads=48), dict(dx=0.0), dict(dt=-1.0), dict(alpha=0.0), dict(bc=2),
    dict(dtype=5), dict(ny=70000, nx=64, tile_w=8), dict(persistent=2), dict(persistent=-1),
])
def test_init2d_rejects_invalid(S, bad):
    kw = dict(dtype=S.F64, nx=256, ny=128, dx=0.1, dt=0.002, alpha=1.0, tile_w=32, threads=0, bc=0, persistent=0)
    kw.update(bad)
    c = S.make_config2d(kw["dtype"], kw["nx"], kw["ny"], kw["dx"], kw["dt"], kw["alpha"], kw["tile_w"], kw["threads"],
                        kw["bc"], kw["persistent"])
    h = ctypes.c_void_p()
    assert S.swept2d_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_EINVAL
    assert not h.value


def test_init2d_plan_and_workspace(S):
    c = S.make_config2d(S.F32, 512, 256, 0.1, 0.002, 1.0, 0)
    h = ctypes.c_void_p()
    assert S.swept2d_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_OK
    p = S.swept2d_plan_info()
    assert S.swept2d_get_plan(h.value, ctypes.byref(p)) == S.SWEPT_OK
    assert (p.tile_w, p.half_cycle, p.tiles_x, p.tiles_y, p.threads) == (32, 16, 16, 8, 256)
    assert p.smem_bytes == 2 * 34 * 34 * 4
    sz = ctypes.c_size_t()
    assert S.swept2d_workspace_size(h.value, ctypes.byref(sz)) == S.SWEPT_OK
    # per tile: two strip buffers of 2 W^2 + 4 W values and bands of 2 W^2 - 4 W; plus the classic second array
    W, tiles = 32, 16 * 8
    assert sz.value >= 4 * (tiles * (2 * (2 * W * W + 4 * W) + (2 * W * W - 4 * W)) + 512 * 256)
    S.swept2d_free(h.value)


def test_init2d_rejects_nonzero_reserved(S):
    c = S.make_config2d(S.F64, 256, 128, 0.1, 0.002, 1.0, 32)
    c.reserved[1] = 1
    h = ctypes.c_void_p()
    assert S.swept2d_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_EINVAL


def test_persistent2d_plan_workspace_and_options(S):
    """A persistent handle reports it in its plan, adds a second band buffer and
    3 counters per tile to the workspace, and validates its options."""
    sizes = {}
    for pers in (0, 1):
        c = S.make_config2d(S.F32, 512, 256, 0.1, 0.002, 1.0, 32, persistent=pers)
        h = ctypes.c_void_p()
        assert S.swept2d_init(ctypes.byref(c), ctypes.byref(h)) == S.SWEPT_OK
        p = S.swept2d_plan_info()
        assert S.swept2d_get_plan(h.value, ctypes.byref(p)) == S.SWEPT_OK
        assert p.persistent == pers
        sz = ctypes.c_size_t()
        assert S.swept2d_workspace_size(h.value, ctypes.byref(sz)) == S.SWEPT_OK
        sizes[pers] = sz.value
        assert S.swept2d_set_option(h.value, S.SWEPT_OPT_SPIN_LIMIT, 0) == S.SWEPT_EINVAL
        assert S.swept2d_set_option(h.value, S.SWEPT_OPT_SPIN_LIMIT, 1 << 32) == S.SWEPT_EINVAL
        assert S.swept2d_set_option(h.value, S.SWEPT_OPT_START_ITEM, -1) == S.SWEPT_EINVAL
        assert S.swept2d_set_option(h.value, S.SWEPT2D_OPT_CHECK_DROP_WAIT, -2) == S.SWEPT_EINVAL
        assert S.swept2d_set_option(h.value, 99, 0) == S.SWEPT_EINVAL
        assert S.swept2d_set_option(h.value, S.SWEPT_OPT_SPIN_LIMIT, 1000) == S.SWEPT_OK
        assert S.swept2d_set_option(h.value, S.SWEPT_OPT_START_ITEM, 3) == S.SWEPT_OK
        S.swept2d_free(h.value)
    W, tiles = 32, 16 * 8
    assert sizes[1] - sizes[0] >= 4 * tiles * (2 * W * W - 4 * W) + 4 * 3 * tiles


SCHEDULES = [
    # nx, ny, W, nsteps
    (16, 16, 8, 4), (16, 16, 8, 3), (16, 16, 8, 13), (32, 32, 8, 9), (48, 32, 8, 13), (32, 48, 8, 21),
    (64, 64, 16, 40), (64, 48, 16, 37), (96, 64, 32, 100), (64, 64, 8, 3), (128, 128, 64, 70), (64, 64, 32, 16),
    (64, 32, 16, 0),
]


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny,W,nsteps", SCHEDULES)
def test_schedule2d_replay(S, nx, ny, W, nsteps, bc):
    assert S.check_schedule2d(S.F64, nx, ny, W, nsteps, bc=bc) == nx * ny * nsteps


def test_schedule2d_long_run_with_cached_body(S):
    # W = 8: h = 4, so 1,100 steps are 275 half cycles: head + one 256-cycle body + tail
    assert S.check_schedule2d(S.F32, 16, 16, 8, 1100) == 16 * 16 * 1100


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("nx,ny,W,nsteps", SCHEDULES)
def test_schedule2d_persistent_replay(S, nx, ny, W, nsteps, bc):
    """The persistent queue, replayed item by item in queue order: every access
    ordered after the write it reads (and every write after the reads of the
    value it replaces) through the transitive closure of the waits alone."""
    assert S.check_schedule2d(S.F64, nx, ny, W, nsteps, bc=bc, persistent=1) == nx * ny * nsteps


def test_schedule2d_persistent_replay_random_configurations(S):
    g = np.random.default_rng(1612)
    for _ in range(25):
        W = int(g.choice([8, 12, 16, 20, 24]))
        ntx, nty = int(g.integers(2, 6)), int(g.integers(2, 6))
        h = W // 2
        nsteps = int(g.choice([int(g.integers(1, h)), h, int(g.integers(h + 1, 6 * h))]))
        bc = int(g.integers(0, 2))
        assert S.check_schedule2d(S.F32, ntx * W, nty * W, W, nsteps, bc=bc, persistent=1) == ntx * W * nty * W * nsteps


def test_schedule2d_persistent_too_large(S):
    with pytest.raises(S.SweptError) as e:
        S.check_schedule2d(S.F64, 256, 256, 8, 400, persistent=1)
    assert e.value.status == S.SWEPT_EINVAL


@pytest.mark.parametrize("nx,ny,W,nsteps,bc", [(32, 32, 8, 13, 0), (32, 32, 8, 14, 1), (24, 16, 8, 9, 0),
                                               (32, 24, 8, 16, 1), (48, 32, 16, 19, 0)])
def test_schedule2d_persistent_replay_finds_dropped_waits(S, nx, ny, W, nsteps, bc):
    """Plant a mistake in the wait rule (the replay drops the last wait of one item)
    and check that the replay reports a race, for every item whose last wait is
    needed: each bridge and octahedron of a full half cycle, each remainder
    bridge, the remainder pyramids after an odd number of half cycles (after an
    even number only the first of their four waits is needed) and the remainder
    octahedra of more than one level (with one, the x-bridges' waits already
    cover its four tiles)."""
    h = W // 2
    T = (nx // W) * (ny // W)
    q, rem = divmod(nsteps, h)
    main = T + q * 3 * T if q else 0
    items = main + (4 * T if rem else 0)
    expected = []
    for it in range(T, items):
        if it >= main:
            r = it - main
            if r < T and q % 2 == 0:
                continue
            if r >= 3 * T and rem == 1:
                continue
        expected.append(it)
    assert expected
    for it in expected:
        with pytest.raises(S.SweptError) as e:
            S.check_schedule2d(S.F64, nx, ny, W, nsteps, bc=bc, persistent=1, drop_wait=it)
        assert e.value.status == S.SWEPT_EDEVICE
        assert "wait" in str(e.value) or "level" in str(e.value)


# --------------------------------------------------------------------------- GPU parity
GPU_CASES = [
    # nx, ny, W, nsteps, threads
    (64, 64, 8, 100, 0),
    (64, 48, 16, 37, 0),        # non-square, remainder
    (96, 64, 32, 100, 128),
    (128, 128, 32, 1000, 0),
    (128, 128, 64, 70, 512),
    (32, 32, 16, 7, 64),        # remainder only
    (16, 16, 8, 1100, 32),      # head + cached body + tail
    (1024, 1024, 32, 40, 0),    # the 2^20-point workload
    (4096, 4096, 128, 70, 1024),  # the 2^24-point workload, tuned FP32 plan (FP64 caps W at 64)
    (4096, 4096, 64, 37, 256),
]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("nx,ny,W,nsteps,threads", GPU_CASES)
def test_swept2d_parity(S, dtype, nx, ny, W, nsteps, threads):
    import torch

    if dtype == np.float64 and W > 64:
        pytest.skip("FP64 tiles are at most 64 wide (shared memory)")

    p = inputs.heat2d_problem(nx=nx, ny=ny, dtype=dtype)
    code = S.F64 if dtype == np.float64 else S.F32
    sol = S.Solver2D(code, nx, ny, p["dx"], p["dt"], p["alpha"], tile_w=W, threads=threads)
    u = torch.from_numpy(p["u0"]).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    assert np.array_equal(got, v.cpu().numpy()), "swept2d != classic2d"
    ref = oracle.heat2d(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, threads=8)
    assert np.array_equal(got, ref), "swept2d != oracle"
    sol.close()


MIRROR_CASES = [
    # nx, ny, W, nsteps
    (64, 48, 16, 37), (96, 64, 32, 100), (16, 16, 8, 1100), (1024, 1024, 32, 40), (128, 128, 64, 70),
]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("nx,ny,W,nsteps", MIRROR_CASES)
def test_swept2d_insulated_parity(S, dtype, nx, ny, W, nsteps):
    """Insulated (mirror) walls on both axes: swept2d == classic2d == the oracle bit for bit."""
    import torch

    p = inputs.heat2d_problem(nx=nx, ny=ny, dtype=dtype)
    code = S.F64 if dtype == np.float64 else S.F32
    sol = S.Solver2D(code, nx, ny, p["dx"], p["dt"], p["alpha"], tile_w=W, bc=S.BC_REFLECTIVE)
    u = torch.from_numpy(p["u0"]).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    assert np.array_equal(got, v.cpu().numpy()), "swept2d != classic2d"
    ref = oracle.heat2d(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, bc=oracle.BC_MIRROR, threads=8)
    assert np.array_equal(got, ref), "swept2d != oracle"
    sol.close()


@pytest.mark.gpu
def test_swept2d_repeated_calls_and_zero_steps(S):
    """Cached graphs are reused across calls; 0 steps is a no-op; results still equal the oracle."""
    import torch

    p = inputs.heat2d_problem(nx=64, ny=64)
    sol = S.Solver2D(S.F64, 64, 64, p["dx"], p["dt"], p["alpha"], tile_w=16)
    u = torch.from_numpy(p["u0"]).cuda()
    for _ in range(3):
        sol.step(u, 25)
    sol.step(u, 0)
    torch.cuda.synchronize()
    ref = oracle.heat2d(p["u0"], p["dx"], p["dt"], p["alpha"], 75)
    assert np.array_equal(u.cpu().numpy(), ref)
    sol.close()


PERSIST_CASES = [
    # nx, ny, W, nsteps, threads, bc
    (64, 64, 8, 100, 0, 0),
    (64, 48, 16, 37, 0, 1),         # non-square, remainder, walls
    (96, 64, 32, 100, 128, 0),
    (128, 128, 32, 1000, 0, 1),
    (32, 32, 16, 7, 64, 0),         # remainder only
    (16, 16, 8, 1100, 32, 0),       # many half cycles on 4 tiles
    (1024, 1024, 32, 40, 0, 0),     # the 2^20-point workload
    (1024, 1024, 32, 41, 0, 1),
    (4096, 4096, 64, 37, 256, 0),   # the 2^24-point workload
    (4096, 4096, 128, 70, 1024, 0),
]


@pytest.mark.gpu
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("nx,ny,W,nsteps,threads,bc", PERSIST_CASES)
def test_swept2d_persistent_parity(S, dtype, nx, ny, W, nsteps, threads, bc):
    """The persistent queue kernel: swept2d (persistent) == classic2d == the oracle bit for bit."""
    import torch

    if dtype == np.float64 and W > 64:
        pytest.skip("FP64 tiles are at most 64 wide (shared memory)")
    p = inputs.heat2d_problem(nx=nx, ny=ny, dtype=dtype)
    code = S.F64 if dtype == np.float64 else S.F32
    sol = S.Solver2D(code, nx, ny, p["dx"], p["dt"], p["alpha"], tile_w=W, threads=threads, bc=bc, persistent=1)
    assert sol.plan["persistent"] == 1
    u = torch.from_numpy(p["u0"]).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    got = u.cpu().numpy()
    assert np.array_equal(got, v.cpu().numpy()), "persistent swept2d != classic2d"
    ref = oracle.heat2d(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, bc=oracle.BC_MIRROR if bc else 0, threads=8)
    assert np.array_equal(got, ref), "persistent swept2d != oracle"
    sol.close()


@pytest.mark.gpu
def test_swept2d_persistent_timeout_path(S):
    """Failure detection without a GPU fault: the queue starts after the first
    pyramids, so the first bridges wait for tiles no block computes.  Each bounded
    wait gives up, SWEPT_ETIMEOUT reaches the host through swept2d_sync_status,
    and the context stays usable: a normal solve right after equals classic."""
    import torch

    nx = ny = 256
    p = inputs.heat2d_problem(nx=nx, ny=ny)
    sol = S.Solver2D(S.F64, nx, ny, p["dx"], p["dt"], p["alpha"], tile_w=32, persistent=1)
    u0 = torch.from_numpy(p["u0"]).cuda()
    u = u0.clone()
    sol.set_option(S.SWEPT_OPT_SPIN_LIMIT, 1000)
    sol.set_option(S.SWEPT_OPT_START_ITEM, (nx // 32) * (ny // 32))
    sol.step(u, 100)
    with pytest.raises(S.SweptError) as e:
        sol.sync_status()
    assert e.value.status == S.SWEPT_ETIMEOUT
    sol.set_option(S.SWEPT_OPT_START_ITEM, 0)
    sol.set_option(S.SWEPT_OPT_SPIN_LIMIT, 1 << 24)
    u.copy_(u0)
    v = u0.clone()
    sol.step(u, 100)
    sol.classic(v, 100)
    torch.cuda.synchronize()
    sol.sync_status()
    assert torch.equal(u, v)
    sol.close()


def test_small_divmod_argument_is_exact():
    """The 2D level mapping divides thread indices (<= 1024) by rectangle widths
    (<= 256) with one single-precision multiply by an approximate reciprocal
    (within 2 ulp of 1/b).  The quotient (a + 1/2) / b stays at least 1/(2b)
    from an integer; check that this margin exceeds the worst error of the
    product (3 ulp of 1/b carried through, plus the product's rounding) over the
    whole range, and that truncation is exact with the rounded reciprocal."""
    a = np.arange(0, 1025, dtype=np.float64)
    for b in range(1, 257):
        exact = (a + 0.5) / b
        margin = np.min(np.abs(exact - np.round(exact)))
        worst = exact.max() * (3 * 2.0 ** -23) + 2.0 ** -13  # reciprocal error + product rounding
        assert margin > worst, b
        rb = np.float32(1.0) / np.float32(b)
        q = ((a.astype(np.float32) + np.float32(0.5)) * rb).astype(np.int64)
        assert np.array_equal(q, np.arange(0, 1025) // b), b


def test_schedule2d_replay_random_configurations(S):
    """Seeded sweep of the 2D host replay over random grids (tile counts 2..5 per axis),
    tile widths 8..32 and step counts (full half cycles, remainders, both)."""
    g = np.random.default_rng(20161208)
    for _ in range(25):
        W = int(g.choice([8, 12, 16, 20, 24, 32]))
        ntx, nty = int(g.integers(2, 6)), int(g.integers(2, 6))
        h = W // 2
        nsteps = int(g.choice([int(g.integers(1, h)), h, int(g.integers(h + 1, 5 * h))]))
        bc = int(g.integers(0, 2))
        assert S.check_schedule2d(S.F64, ntx * W, nty * W, W, nsteps, bc=bc) == ntx * W * nty * W * nsteps
