"""GPU parity: the swept path and the classic path, called through the C ABI,
against the CPU oracle on the same seeded inputs.

Bar: the kernels evaluate every point with the oracle's operation order, so
swept == classic == oracle bit for bit (which is within the stated bounds of
1e-12 relative in FP64 and 1e-5 in FP32).  Cases span several tiles, odd tile
counts, ragged step counts (a remainder of sub-timesteps after the last full
pass), both boundary conditions, the minimum grid (two tiles) and the full
workload sizes.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1612_02495_gb300 import inputs

pytestmark = pytest.mark.gpu

THREADS = max(1, min(32, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def S():
    from paper_1612_02495_gb300 import build as libbuild

    libbuild.build()
    from paper_1612_02495_gb300 import swept

    return swept


def relerr(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


def run_gpu(S, scheme, dtype, u0, dx, dt, p0, nsteps, bc=0, tile_w=0, threads=0):
    import torch

    n = u0.shape[-1]
    sol = S.Solver(scheme, dtype, n, dx, dt, p0, bc=bc, tile_w=tile_w, threads=threads)
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    out = u.cpu().numpy(), v.cpu().numpy(), sol.plan
    sol.close()
    return out


def tol(dtype):
    return 1e-12 if dtype == np.float64 else 1e-5


# --------------------------------------------------------------------------- heat
HEAT_CASES = [
    # n, W, nsteps, bc
    (1024, 64, 10000, 0),   # the full heat workload (N=1024, r=0.25, 10,000 steps, W=64)
    (96, 16, 37, 0),        # ragged remainder
    (40, 20, 0, 0),         # no-op
    (40, 20, 1, 0),
    (8 * 24, 8, 101, 1),    # insulated ends
    (5 * 64, 64, 333, 1),   # odd tile count, insulated
    (2 * 128, 128, 64 + 7, 0),  # minimum grid (two tiles)
]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("n,W,nsteps,bc", HEAT_CASES)
def test_heat_parity(S, dtype, n, W, nsteps, bc):
    p = inputs.heat_problem(n=n, dtype=dtype)
    sw, cl, _ = run_gpu(S, S.HEAT, S.F64 if dtype == np.float64 else S.F32, p["u0"], p["dx"], p["dt"],
                        p["alpha"], nsteps, bc=bc, tile_w=W)
    ref = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, bc=bc)
    assert sw.dtype == dtype
    assert np.array_equal(sw, cl), "swept != classic"
    assert relerr(sw, ref) <= tol(dtype)
    assert np.array_equal(sw, ref), "swept != oracle bitwise (relerr %g)" % relerr(sw, ref)


# --------------------------------------------------------------------------- KS
KS_CASES = [
    # n, W, nsteps
    (2048, 64, 1003),
    (3 * 128, 128, 257),
    (2 * 32, 32, 75),
    (1 << 14, 0, 50000),    # the KS workload at N=2^14: full 50,000 steps, default plan
    (1 << 16, 256, 2001),
    (1 << 16, 1024, 600),   # largest tile
]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("n,W,nsteps", KS_CASES)
def test_ks_parity(S, dtype, n, W, nsteps):
    p = inputs.ks_problem(n=n, dtype=dtype)
    sw, cl, plan = run_gpu(S, S.KS, S.F64 if dtype == np.float64 else S.F32, p["u0"], p["dx"], p["dt"], p["nu"],
                           nsteps, tile_w=W)
    ref = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], nsteps, threads=THREADS)
    assert np.array_equal(sw, cl), "swept != classic"
    assert relerr(sw, ref) <= tol(dtype)
    assert np.array_equal(sw, ref), "swept != oracle bitwise (relerr %g)" % relerr(sw, ref)


@pytest.mark.parametrize("threads", [32, 64, 128, 256, 512])
def test_ks_thread_counts(S, threads):
    p = inputs.ks_problem(n=4096)
    sw, cl, plan = run_gpu(S, S.KS, S.F64, p["u0"], p["dx"], p["dt"], p["nu"], 377, tile_w=512, threads=threads)
    assert plan["threads"] == threads
    ref = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], 377, threads=THREADS)
    assert np.array_equal(sw, cl) and np.array_equal(sw, ref)


# --------------------------------------------------------------------------- Euler
EULER_CASES = [
    # n, W, nsteps, bc
    (1024, 64, 300, 1),
    (1024, 64, 300, 0),
    (3 * 32, 32, 77, 1),
    (2 * 8, 8, 13, 1),       # minimum tile and grid
    (1 << 16, 0, 1000, 1),   # the Sod workload at N=2^16, 1,000-step window, default plan
]


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("n,W,nsteps,bc", EULER_CASES)
def test_euler_parity(S, dtype, n, W, nsteps, bc):
    pr = inputs.euler_problem(n=n, dtype=dtype)
    U0 = pr["U0"]
    if bc == 0:  # periodic: a smooth travelling state instead of the tube
        x = (np.arange(n) + 0.5) / n
        rho = 1 + 0.2 * np.sin(2 * np.pi * x)
        u = 0.3 + 0.1 * np.cos(2 * np.pi * x)
        p = 1 + 0.1 * np.sin(4 * np.pi * x)
        U0 = np.stack([rho, rho * u, p / 0.4 + 0.5 * rho * u * u]).astype(dtype)
    sw, cl, _ = run_gpu(S, S.EULER, S.F64 if dtype == np.float64 else S.F32, U0, pr["dx"], pr["dt"], pr["gamma"],
                        nsteps, bc=bc, tile_w=W)
    ref = oracle.euler(U0, pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=bc, threads=THREADS)
    assert np.array_equal(sw, cl), "swept != classic"
    assert relerr(sw, ref) <= tol(dtype)
    assert np.array_equal(sw, ref), "swept != oracle bitwise (relerr %g)" % relerr(sw, ref)


# --------------------------------------------------------------------------- full size, bench launch config
def test_ks_full_size_sampled(S):
    """KS N=2^20 FP64, 50,000 steps, the library's default plan:
    swept == classic bit for bit; the mean is conserved; the whole field after
    the first 100 steps equals the oracle; and sampled points of the final
    state equal the oracle advanced 100 steps from the GPU state at 49,900
    steps on a window covering their domain of dependence."""
    import torch

    n, total, tail = 1 << 20, 50000, 100
    p = inputs.ks_problem(n=n)
    sol = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"])
    u = torch.from_numpy(p["u0"]).cuda()
    v, w = u.clone(), u.clone()
    sol.step(u, total)
    sol.classic(v, total)
    sol.step(w, total - tail)
    torch.cuda.synchronize()
    sol.sync_status()
    fin, fin_c, mid = u.cpu().numpy(), v.cpu().numpy(), w.cpu().numpy()
    assert np.array_equal(fin, fin_c)
    assert abs(fin.sum() - p["u0"].sum()) <= 1e-11 * np.abs(p["u0"]).sum()
    # first 100 steps, full field
    a = torch.from_numpy(p["u0"]).cuda()
    sol.step(a, tail)
    torch.cuda.synchronize()
    assert np.array_equal(a.cpu().numpy(), oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], tail, threads=THREADS))
    # sampled final points: domain of dependence of 100 steps is 2 stages * 2 * 100 points per side
    reach = 2 * 2 * tail
    rng = inputs.rng(99)
    for c in rng.integers(0, n, size=8):
        idx = (np.arange(c - reach - 8, c + reach + 9)) % n
        loc = oracle.ks(mid[idx], p["dx"], p["dt"], p["nu"], tail)  # periodic on the window; edges are garbage
        k = reach + 8
        assert loc[k] == fin[c], (c, loc[k], fin[c])
    sol.close()


@pytest.mark.parametrize("chunk", [1, 2])
@pytest.mark.parametrize("scheme,dtype", [("ks", np.float64), ("ks", np.float32), ("heat", np.float64),
                                          ("heat", np.float32)])
def test_chunked_tiers_parity(S, chunk, scheme, dtype):
    """One point a thread per trip (paired in FP32 KS) and two strided points a
    trip give the same bits as the oracle (tile 96/192, 32 threads: tiers wider
    than the block, ragged trip counts)."""
    code = S.F64 if dtype == np.float64 else S.F32
    if scheme == "ks":
        p = inputs.ks_problem(n=192 * 8, dtype=dtype)
        sw, cl, plan = None, None, None
        import torch

        sol = S.Solver(S.KS, code, p["u0"].size, p["dx"], p["dt"], p["nu"], tile_w=192, threads=32, chunk=chunk)
        ref = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], 333)
    else:
        p = inputs.heat_problem(n=96 * 10, dtype=dtype)
        import torch

        sol = S.Solver(S.HEAT, code, p["u0"].size, p["dx"], p["dt"], p["alpha"], tile_w=96, threads=32, chunk=chunk)
        ref = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], 333)
    assert sol.plan["chunk"] == chunk
    u = torch.from_numpy(p["u0"]).cuda()
    sol.step(u, 333)
    torch.cuda.synchronize()
    sol.sync_status()
    assert np.array_equal(u.cpu().numpy(), ref)
    sol.close()


PERSIST_CASES = [
    # scheme, dtype, n, W, threads, nsteps, bc
    ("heat", np.float64, 1024, 64, 64, 10000, 0),
    ("heat", np.float32, 8 * 24, 8, 32, 101, 1),
    ("ks", np.float64, 2048, 64, 64, 1003, 0),
    ("ks", np.float32, 3 * 128, 128, 128, 257, 0),
    ("ks", np.float64, 1 << 16, 512, 128, 701, 0),
    ("ks", np.float64, 2 * 32, 32, 32, 3, 0),       # remainder only
    ("euler", np.float64, 1024, 64, 64, 300, 1),
    ("euler", np.float64, 1024, 64, 64, 300, 0),
    ("euler", np.float32, 3 * 32, 32, 32, 77, 1),
]


@pytest.mark.parametrize("scheme,dtype,n,W,threads,nsteps,bc", PERSIST_CASES)
def test_persistent_mode_parity(S, scheme, dtype, n, W, threads, nsteps, bc):
    """swept_step_n with the persistent kernel (one queue of pass x tile items)
    equals the per-pass launches, classic and the oracle bit for bit."""
    import torch

    code = S.F64 if dtype == np.float64 else S.F32
    if scheme == "heat":
        p = inputs.heat_problem(n=n, dtype=dtype)
        u0, args, sc = p["u0"], (p["dx"], p["dt"], p["alpha"]), S.HEAT
        ref = oracle.heat(u0, p["dx"], p["dt"], p["alpha"], nsteps, bc=bc)
    elif scheme == "ks":
        p = inputs.ks_problem(n=n, dtype=dtype)
        u0, args, sc = p["u0"], (p["dx"], p["dt"], p["nu"]), S.KS
        ref = oracle.ks(u0, p["dx"], p["dt"], p["nu"], nsteps, threads=THREADS)
    else:
        pr = inputs.euler_problem(n=n, dtype=dtype)
        u0 = pr["U0"]
        if bc == 0:
            x = (np.arange(n) + 0.5) / n
            rho = 1 + 0.2 * np.sin(2 * np.pi * x)
            uu = 0.3 + 0.1 * np.cos(2 * np.pi * x)
            pp = 1 + 0.1 * np.sin(4 * np.pi * x)
            u0 = np.stack([rho, rho * uu, pp / 0.4 + 0.5 * rho * uu * uu]).astype(dtype)
        args, sc = (pr["dx"], pr["dt"], pr["gamma"]), S.EULER
        ref = oracle.euler(u0, pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=bc, threads=THREADS)
    sol = S.Solver(sc, code, n, *args, bc=bc, tile_w=W, threads=threads, persistent=1)
    assert sol.plan["persistent"] == 1
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    assert np.array_equal(u.cpu().numpy(), v.cpu().numpy())
    assert np.array_equal(u.cpu().numpy(), ref)
    # a second call continues from the state (graph replay, counters reset)
    sol.step(u, 7)
    sol.classic(v, 7)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), v.cpu().numpy())
    sol.close()


def test_ks_full_size_in_the_bench_plan(S):
    """KS N=2^20 FP64, 50,000 steps in the launch configuration bench.py times (the
    autotuner's plan, from the same tune_single call): swept == classic bit for
    bit, the mean is conserved, and sampled final points equal the oracle
    advanced 100 steps from the GPU state at 49,900 steps on windows covering
    their domain of dependence."""
    import torch

    from paper_1612_02495_gb300 import autotune

    n, total, tail = 1 << 20, 50000, 100
    plan = autotune.tune_single(S.KS, S.F64, n, probe_steps=4000)
    p = inputs.ks_problem(n=n)
    sol = autotune.solver_from_plan(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], plan)
    u = torch.from_numpy(p["u0"]).cuda()
    v, w = u.clone(), u.clone()
    sol.step(u, total)
    sol.classic(v, total)
    sol.step(w, total - tail)
    torch.cuda.synchronize()
    sol.sync_status()
    fin, mid = u.cpu().numpy(), w.cpu().numpy()
    assert np.array_equal(fin, v.cpu().numpy()), plan
    assert abs(fin.sum() - p["u0"].sum()) <= 1e-11 * np.abs(p["u0"]).sum()
    reach = 2 * 2 * tail
    rng = inputs.rng(98)
    for c in rng.integers(0, n, size=8):
        idx = (np.arange(c - reach - 8, c + reach + 9)) % n
        loc = oracle.ks(mid[idx], p["dx"], p["dt"], p["nu"], tail)
        assert loc[reach + 8] == fin[c], (plan, c, loc[reach + 8], fin[c])
    sol.close()


def test_persistent_full_size_ks(S):
    """KS N=2^20 FP64, 50,000 steps in the persistent kernel equals the per-pass path."""
    import torch

    n = 1 << 20
    p = inputs.ks_problem(n=n)
    a = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], tile_w=512, threads=128, persistent=1)
    b = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], tile_w=1024, threads=32)
    u = torch.from_numpy(p["u0"]).cuda()
    v = u.clone()
    a.step(u, 50000)
    b.step(v, 50000)
    torch.cuda.synchronize()
    a.sync_status()
    assert np.array_equal(u.cpu().numpy(), v.cpu().numpy())
    a.close()
    b.close()


CLUSTER_CASES = [
    # scheme, dtype, n, W, threads, nsteps, bc
    ("heat", np.float64, 1024, 64, 64, 10000, 0),    # the heat workload: 16 tiles = one 16-block cluster
    ("heat", np.float32, 1024, 64, 64, 333, 1),      # insulated ends
    ("heat", np.float64, 3 * 32, 32, 32, 101, 0),    # cluster of 3
    ("ks", np.float64, 1 << 14, 1024, 256, 2001, 0),  # KS 2^14 as 16 tiles of 1024
    ("ks", np.float32, 2 * 64, 64, 64, 77, 0),       # cluster of 2
    ("ks", np.float64, 5 * 128, 128, 128, 3, 0),     # remainder only
    ("euler", np.float64, 4 * 64, 64, 64, 300, 1),   # reflective walls at the split block
    ("euler", np.float32, 8 * 32, 32, 32, 41, 0),
]


@pytest.mark.parametrize("scheme,dtype,n,W,threads,nsteps,bc", CLUSTER_CASES)
def test_cluster_mode_parity(S, scheme, dtype, n, W, threads, nsteps, bc):
    """All tiles in one thread-block cluster, edges through distributed shared
    memory: equal to classic and the oracle bit for bit."""
    import torch

    code = S.F64 if dtype == np.float64 else S.F32
    if scheme == "heat":
        p = inputs.heat_problem(n=n, dtype=dtype)
        u0, args, sc = p["u0"], (p["dx"], p["dt"], p["alpha"]), S.HEAT
        ref = oracle.heat(u0, p["dx"], p["dt"], p["alpha"], nsteps, bc=bc)
    elif scheme == "ks":
        p = inputs.ks_problem(n=n, dtype=dtype)
        u0, args, sc = p["u0"], (p["dx"], p["dt"], p["nu"]), S.KS
        ref = oracle.ks(u0, p["dx"], p["dt"], p["nu"], nsteps, threads=THREADS)
    else:
        pr = inputs.euler_problem(n=n, dtype=dtype)
        u0 = pr["U0"]
        if bc == 0:
            x = (np.arange(n) + 0.5) / n
            rho = 1 + 0.2 * np.sin(2 * np.pi * x)
            uu = 0.3 + 0.1 * np.cos(2 * np.pi * x)
            pp = 1 + 0.1 * np.sin(4 * np.pi * x)
            u0 = np.stack([rho, rho * uu, pp / 0.4 + 0.5 * rho * uu * uu]).astype(dtype)
        args, sc = (pr["dx"], pr["dt"], pr["gamma"]), S.EULER
        ref = oracle.euler(u0, pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=bc, threads=THREADS)
    sol = S.Solver(sc, code, n, *args, bc=bc, tile_w=W, threads=threads, cluster=1)
    assert sol.plan["cluster"] == 1
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    assert np.array_equal(u.cpu().numpy(), v.cpu().numpy())
    assert np.array_equal(u.cpu().numpy(), ref)
    sol.close()


def test_cluster_mode_rejects_more_than_16_tiles(S):
    with pytest.raises(S.SweptError):
        S.Solver(S.KS, S.F64, 17 * 64, 0.785, 0.005, 1.0, tile_w=64, cluster=1)


WARP_CASES = [
    # scheme, dtype, n, W (= 32 P), nsteps, bc, mode (0 per pass, 1 persistent, 2 cluster)
    ("heat", np.float64, 1024, 64, 10000, 0, 0),   # the heat workload, P = 2
    ("heat", np.float32, 1024, 64, 10000, 0, 0),
    ("heat", np.float64, 7 * 32, 32, 333, 1, 0),   # P = 1, insulated ends, remainder
    ("heat", np.float32, 5 * 128, 128, 1001, 1, 1),
    ("heat", np.float64, 3 * 256, 256, 700, 0, 2),  # P = 8 in one cluster of 3
    ("heat", np.float32, 16 * 64, 64, 2049, 1, 2),
    ("ks", np.float64, 1 << 14, 64, 1001, 0, 0),   # P = 2
    ("ks", np.float32, 1 << 14, 128, 2000, 0, 0),  # P = 4
    ("ks", np.float64, 1 << 14, 256, 999, 0, 1),   # P = 8 persistent
    ("ks", np.float32, 12 * 64, 64, 77, 0, 1),
    ("ks", np.float64, 16 * 128, 128, 555, 0, 2),
    ("ks", np.float64, 2 * 64, 64, 7, 0, 0),       # two tiles, remainder only
    # KS with P = 1 < r: the 32-point register node (8 sub-steps = 4 timesteps a pass), halo
    # points from lanes two away and from the window's halo at both warp ends
    ("ks", np.float64, 64 * 32, 32, 1003, 0, 0),
    ("ks", np.float32, 2 * 32, 32, 301, 0, 0),
    ("ks", np.float64, 128 * 32, 32, 777, 0, 1),
    ("ks", np.float32, 9 * 32, 32, 203, 0, 2),
    ("ks", np.float64, 3 * 32, 32, 3, 0, 0),       # remainder only
]


@pytest.mark.parametrize("scheme,dtype,n,W,nsteps,bc,mode", WARP_CASES)
def test_warp_tiles_parity(S, scheme, dtype, n, W, nsteps, bc, mode):
    """Tier rows in registers with warp-shuffle neighbour reads: equal to the
    shared-memory swept path, classic and the oracle bit for bit."""
    import torch

    code = S.F64 if dtype == np.float64 else S.F32
    if scheme == "heat":
        p = inputs.heat_problem(n=n, dtype=dtype)
        args, sc = (p["dx"], p["dt"], p["alpha"]), S.HEAT
        ref = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, bc=bc)
    else:
        p = inputs.ks_problem(n=n, dtype=dtype)
        args, sc = (p["dx"], p["dt"], p["nu"]), S.KS
        ref = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], nsteps, threads=THREADS)
    sol = S.Solver(sc, code, n, *args, bc=bc, tile_w=W, warp_tiles=1, persistent=int(mode == 1),
                   cluster=int(mode == 2))
    assert sol.plan["warp_tiles"] == 1 and sol.plan["threads"] == 32
    smem = S.Solver(sc, code, n, *args, bc=bc, tile_w=W)
    u = torch.from_numpy(p["u0"]).cuda()
    v, w = u.clone(), u.clone()
    sol.step(u, nsteps)
    smem.step(v, nsteps)
    sol.classic(w, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    got = u.cpu().numpy()
    assert np.array_equal(got, v.cpu().numpy())
    assert np.array_equal(got, w.cpu().numpy())
    assert np.array_equal(got, ref)
    sol.close()
    smem.close()


EULER_PAIR_CASES = [
    # dtype, n, W, threads, nsteps, bc, mode (0 per pass, 1 persistent, 2 cluster)
    (np.float64, 1024, 64, 64, 300, 1, 0),
    (np.float32, 1024, 64, 128, 300, 0, 0),
    (np.float64, 3 * 32, 32, 32, 77, 1, 0),    # the wall face inside a 32-thread block
    (np.float64, 2 * 8, 8, 32, 13, 1, 0),      # minimum tile and grid
    (np.float64, 1 << 16, 256, 128, 300, 1, 0),
    (np.float64, 1 << 16, 256, 256, 301, 1, 1),
    (np.float32, 8 * 128, 128, 64, 99, 1, 2),
]


@pytest.mark.parametrize("dtype,n,W,threads,nsteps,bc,mode", EULER_PAIR_CASES)
def test_euler_pair_flux_parity(S, dtype, n, W, threads, nsteps, bc, mode):
    """Euler with two threads per face in the flux phase (chunk 2): equal to
    one thread per face, classic and the oracle bit for bit."""
    import torch

    pr = inputs.euler_problem(n=n, dtype=dtype)
    U0 = pr["U0"]
    if bc == 0:
        x = (np.arange(n) + 0.5) / n
        rho = 1 + 0.2 * np.sin(2 * np.pi * x)
        u = 0.3 + 0.1 * np.cos(2 * np.pi * x)
        p = 1 + 0.1 * np.sin(4 * np.pi * x)
        U0 = np.stack([rho, rho * u, p / 0.4 + 0.5 * rho * u * u]).astype(dtype)
    code = S.F64 if dtype == np.float64 else S.F32
    args = (pr["dx"], pr["dt"], pr["gamma"])
    pair = S.Solver(S.EULER, code, n, *args, bc=bc, tile_w=W, threads=threads, chunk=2, persistent=int(mode == 1),
                    cluster=int(mode == 2))
    one = S.Solver(S.EULER, code, n, *args, bc=bc, tile_w=W, threads=threads)
    a = torch.from_numpy(np.ascontiguousarray(U0)).cuda()
    b, c = a.clone(), a.clone()
    pair.step(a, nsteps)
    one.step(b, nsteps)
    one.classic(c, nsteps)
    torch.cuda.synchronize()
    pair.sync_status()
    got = a.cpu().numpy()
    assert np.array_equal(got, b.cpu().numpy())
    assert np.array_equal(got, c.cpu().numpy())
    ref = oracle.euler(U0, pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=bc, threads=THREADS)
    assert np.array_equal(got, ref)
    pair.close()
    one.close()


def test_euler_large_persistent(S):
    """Euler Sod at 2^20 cells with the tuned persistent plan (tile 512): equal to
    classic and the oracle bit for bit after 60 steps."""
    import torch

    n, nsteps = 1 << 20, 60
    pr = inputs.euler_problem(n=n)
    sol = S.Solver(S.EULER, S.F64, n, pr["dx"], pr["dt"], pr["gamma"], bc=1, tile_w=512, threads=128, persistent=1)
    u = torch.from_numpy(pr["U0"]).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    got = u.cpu().numpy()
    assert np.array_equal(got, v.cpu().numpy())
    ref = oracle.euler(pr["U0"], pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=1, threads=THREADS)
    assert np.array_equal(got, ref)
    sol.close()


def test_persistent_timeout_path(S):
    """Failure detection without a GPU fault: the persistent kernel's queue starts
    one pass layer late, so every item waits for tiles no block computes.  Each
    bounded wait gives up, SWEPT_ETIMEOUT reaches the host through
    swept_sync_status, and the context stays usable: a normal solve right after
    equals classic bit for bit."""
    import torch

    n, W = 1 << 14, 256
    p = inputs.ks_problem(n=n)
    sol = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], tile_w=W, threads=128, persistent=1)
    u0 = torch.from_numpy(p["u0"]).cuda()
    u = u0.clone()
    sol.set_option(S.SWEPT_OPT_SPIN_LIMIT, 1000)
    sol.set_option(S.SWEPT_OPT_START_ITEM, n // W)
    sol.step(u, 200)
    with pytest.raises(S.SweptError) as e:
        sol.sync_status()
    assert e.value.status == S.SWEPT_ETIMEOUT
    sol.set_option(S.SWEPT_OPT_START_ITEM, 0)
    sol.set_option(S.SWEPT_OPT_SPIN_LIMIT, 1 << 24)
    u.copy_(u0)
    v = u0.clone()
    sol.step(u, 200)
    sol.classic(v, 200)
    torch.cuda.synchronize()
    sol.sync_status()
    assert torch.equal(u, v)
    sol.close()
