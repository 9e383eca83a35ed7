"""GPU parity on grids of any size.  The problem statement is a grid of n
points, a stencil, a step count and a boundary condition (Section "Test
cases"); nothing ties n to the tile width.  When the tile width W does not
divide n, the last tile is wider by X = n mod W and hands its flat top from
pass to pass.  Swept (per pass and persistent) == classic == oracle bit for
bit at prime-like sizes, both boundary conditions, FP64 and FP32, ragged step
counts; the adjoint on such grids equals the oracle's reverse mode; grids too
small for a tiling run classic only.
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


def smooth_euler(n, dtype):
    x = (np.arange(n) + 0.5) / n
    rho = 1 + 0.2 * np.sin(2 * np.pi * x)
    u = 0.3 + 0.1 * np.cos(2 * np.pi * x)
    p = 1 + 0.1 * np.sin(4 * np.pi * x)
    return np.stack([rho, rho * u, p / 0.4 + 0.5 * rho * u * u]).astype(dtype)


def problem(S, scheme, n, dtype, bc):
    """(scheme code, u0, (dx, dt, param), oracle function of (u0, nsteps))."""
    if scheme == "heat":
        p = inputs.heat_problem(n=n, dtype=dtype)
        args = (p["dx"], p["dt"], p["alpha"])
        return S.HEAT, p["u0"], args, lambda u, k: oracle.heat(u, *args, k, bc=bc, threads=THREADS)
    if scheme == "ks":
        p = inputs.ks_problem(n=n, dtype=dtype)
        args = (p["dx"], p["dt"], p["nu"])
        return S.KS, p["u0"], args, lambda u, k: oracle.ks(u, *args, k, threads=THREADS)
    pr = inputs.euler_problem(n=n, dtype=dtype)
    U0 = pr["U0"] if bc == 1 else smooth_euler(n, dtype)
    args = (pr["dx"], pr["dt"], pr["gamma"])
    return S.EULER, U0, args, lambda u, k: oracle.euler(u, *args, k, bc=bc, threads=THREADS)


CASES = [
    # scheme, n, bc, dtype, tile_w (0 = library default), threads, persistent, nsteps
    ("heat", 1009, 0, np.float64, 0, 0, 0, 3001),
    ("heat", 1009, 1, np.float64, 64, 64, 0, 777),
    ("heat", 1009, 1, np.float32, 32, 32, 1, 1001),
    ("heat", 4099, 0, np.float32, 128, 128, 0, 555),
    ("heat", 4099, 1, np.float64, 256, 256, 1, 2003),
    ("heat", 65537, 0, np.float64, 0, 0, 0, 1500),
    ("heat", 65537, 1, np.float64, 1024, 256, 1, 1500),
    ("ks", 1009, 0, np.float64, 0, 0, 0, 1003),
    ("ks", 1009, 0, np.float32, 64, 64, 1, 333),
    ("ks", 4099, 0, np.float64, 512, 128, 0, 777),
    ("ks", 4099, 0, np.float64, 256, 256, 1, 1001),
    ("ks", 65537, 0, np.float64, 0, 0, 0, 600),
    ("ks", 65537, 0, np.float32, 1024, 512, 1, 701),
    ("ks", 3 * 1024 + 1023, 0, np.float64, 1024, 256, 0, 300),  # X = W - 1
    ("euler", 1009, 1, np.float64, 0, 0, 0, 300),
    ("euler", 1009, 0, np.float64, 64, 64, 1, 211),
    ("euler", 4099, 1, np.float32, 128, 128, 0, 257),
    ("euler", 4099, 0, np.float64, 256, 128, 1, 301),
    ("euler", 65537, 1, np.float64, 0, 0, 1, 101),
    ("euler", 65537, 1, np.float64, 512, 128, 0, 120),
    ("euler", 2 * 64 + 1, 1, np.float64, 64, 64, 0, 57),  # two tiles, X = 1 (the wall beside the flat top)
]


@pytest.mark.parametrize("scheme,n,bc,dtype,W,threads,persistent,nsteps", CASES)
def test_ragged_grid_parity(S, scheme, n, bc, dtype, W, threads, persistent, nsteps):
    import torch

    code = S.F64 if dtype == np.float64 else S.F32
    sc, u0, args, ref_fn = problem(S, scheme, n, dtype, bc)
    sol = S.Solver(sc, code, n, *args, bc=bc, tile_w=W, threads=threads, persistent=persistent)
    assert sol.plan["last_tile_extra"] == n % sol.plan["tile_w"] > 0
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    got = u.cpu().numpy()
    assert np.array_equal(got, v.cpu().numpy()), "swept != classic"
    assert np.array_equal(got, ref_fn(u0, nsteps)), "swept != oracle"
    # a second call continues from the state (cached graphs, counters reset)
    sol.step(u, 13)
    sol.classic(v, 13)
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), v.cpu().numpy())
    sol.close()


@pytest.mark.parametrize("scheme,n,bc", [("heat", 1009, 0), ("heat", 1009, 1), ("ks", 1009, 0), ("ks", 4099, 0)])
def test_ragged_grid_adjoint(S, scheme, n, bc):
    """The adjoint sweep runs the same phases, wide tile included: dL/du0 equals the
    oracle's reverse mode bit for bit, dL/dparam within the condition bound."""
    import torch

    eps = 2.0 ** -52
    W = 64
    if scheme == "ks":
        p = inputs.ks_problem(n=n, seed=61)
        args, sc, nsteps = (p["dx"], p["dt"], 1.0), S.KS, 203
    else:
        p = inputs.heat_problem(n=n, seed=63)
        args, sc, nsteps = (p["dx"], p["dt"], p["alpha"]), S.HEAT, 301
    gT = inputs.rng(62).standard_normal(n)
    sol = S.Solver(sc, S.F64, n, *args, bc=bc, tile_w=W)
    assert sol.plan["last_tile_extra"] > 0
    ck = torch.empty(sol.ckpt_size(nsteps), dtype=torch.uint8, device="cuda")
    g, gp = sol.adjoint(torch.from_numpy(gT).cuda(), nsteps, ck, u0=torch.from_numpy(p["u0"]).cuda())
    torch.cuda.synchronize()
    sol.sync_status()
    sol.close()
    if scheme == "ks":
        ref, ref_p, cond = oracle.ks_adjoint(p["u0"], *args, nsteps, gT, with_condition=True, threads=THREADS)
    else:
        ref, ref_p, cond = oracle.heat_adjoint(p["u0"], *args, nsteps, gT, bc=bc, with_condition=True)
    assert np.array_equal(g.cpu().numpy(), ref)
    gp = float(gp.cpu().numpy()[0])
    assert abs(gp - ref_p) <= 1e-12 * abs(ref_p) + 8 * eps * cond, (gp, ref_p, cond)


@pytest.mark.parametrize("scheme,n,bc", [("heat", 3, 0), ("heat", 3, 1), ("heat", 7, 0), ("ks", 5, 0), ("ks", 15, 0),
                                         ("euler", 5, 1), ("euler", 5, 0), ("euler", 15, 1)])
def test_tiny_grids_classic_only(S, scheme, n, bc):
    """n = 2r + 1 and other grids below two tiles of 4r points: classic_step_n
    equals the oracle bit for bit; swept_step_n returns SWEPT_EUNSUPPORTED."""
    import torch

    dtype = np.float64
    sc, u0, args, ref_fn = problem(S, scheme, n, dtype, bc)
    sol = S.Solver(sc, S.F64, n, *args, bc=bc)
    assert sol.plan["tiles"] == 0
    v = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    sol.classic(v, 101)
    torch.cuda.synchronize()
    assert np.array_equal(v.cpu().numpy(), ref_fn(u0, 101))
    with pytest.raises(S.SweptError) as e:
        sol.step(v, 3)
    assert e.value.status == S.SWEPT_EUNSUPPORTED
    sol.close()


def test_ragged_grid_host_buffers(S):
    """swept_run_host (host in, host out) on a ragged grid equals the oracle."""
    import torch

    n, nsteps = 4099, 400
    p = inputs.ks_problem(n=n)
    sol = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], tile_w=256)
    h_in = torch.from_numpy(p["u0"]).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    d = torch.empty(n, dtype=torch.float64, device="cuda")
    sol.run_host(h_in, h_out, d, nsteps)
    sol.close()
    assert np.array_equal(h_out.numpy(), oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], nsteps, threads=THREADS))
