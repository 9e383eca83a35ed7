"""Seeded random launch configurations on the GPU: scheme, precision, boundary
condition, grid size (tile multiples and ragged), tile width, threads, chunk,
execution mode (per pass, persistent, cluster, warp tiles) and step count are
drawn together, so that combinations no hand-written case names still run.
Every draw must give swept == classic == oracle bit for bit: the swept rule
changes only where and when each (point, sub-timestep) is evaluated, never
its arithmetic (Section "Related work").  Run with SWEPT_DEBUG=1 (the debug
build, device-side index checks) each draw must also leave the checks clean."""
import os
import random

import numpy as np
import pytest

import oracle
from paper_1612_02495_gb300 import inputs

pytestmark = pytest.mark.gpu

THREADS = max(1, min(32, os.cpu_count() or 1))
DRAWS = 60


@pytest.fixture(scope="module")
def S():
    from paper_1612_02495_gb300 import build as libbuild

    libbuild.build(debug=os.environ.get("SWEPT_DEBUG", "0") == "1")
    from paper_1612_02495_gb300 import swept

    return swept


def smooth_euler(n, dtype):
    x = (np.arange(n) + 0.5) / n
    rho = 1 + 0.2 * np.sin(2 * np.pi * x)
    u = 0.3 + 0.1 * np.cos(2 * np.pi * x)
    p = 1 + 0.1 * np.sin(4 * np.pi * x)
    return np.stack([rho, rho * u, p / 0.4 + 0.5 * rho * u * u]).astype(dtype)


def draw(rnd, S):
    scheme = rnd.choice(["heat", "ks", "euler"])
    R = 1 if scheme == "heat" else 2
    dtype = rnd.choice([np.float64, np.float32])
    bc = 0 if scheme == "ks" else rnd.choice([0, 1])
    W = 4 * R * rnd.choice([2, 4, 8, 16, 32, 64])
    mode = rnd.choice(["pass", "pass", "persistent", "cluster", "warp"])
    if mode == "warp":
        P = rnd.choice([1, 2, 4, 8])
        W = 32 * P
        if scheme == "euler":
            mode = "pass"
    nt = rnd.randint(2, 16 if mode == "cluster" else 40)
    ragged = mode in ("pass", "persistent") and rnd.random() < 0.4
    n = nt * W + (rnd.randint(1, W - 1) if ragged else 0)
    threads = 32 if mode == "warp" else rnd.choice([t for t in (32, 64, 128, 256, 512) if t <= max(32, 2 * W)])
    chunk = rnd.choice([1, 1, 2]) if mode != "warp" else 1
    nsteps = rnd.randint(1, 400)
    return dict(scheme=scheme, dtype=dtype, bc=bc, W=W, mode=mode, n=n, threads=threads, chunk=chunk, nsteps=nsteps)


CASES = [draw(random.Random(20161208 + i), None) for i in range(DRAWS)]


@pytest.mark.parametrize("case", CASES, ids=["%s-%s-n%d-W%d-%s-t%d-c%d-bc%d-s%d" % (
    c["scheme"], "f64" if c["dtype"] == np.float64 else "f32", c["n"], c["W"], c["mode"], c["threads"], c["chunk"],
    c["bc"], c["nsteps"]) for c in CASES])
def test_random_configuration(S, case):
    import torch

    c = case
    code = S.F64 if c["dtype"] == np.float64 else S.F32
    if c["scheme"] == "heat":
        p = inputs.heat_problem(n=c["n"], dtype=c["dtype"])
        u0, args, sc = p["u0"], (p["dx"], p["dt"], p["alpha"]), S.HEAT
        ref = oracle.heat(u0, *args, c["nsteps"], bc=c["bc"], threads=THREADS)
    elif c["scheme"] == "ks":
        p = inputs.ks_problem(n=c["n"], dtype=c["dtype"])
        u0, args, sc = p["u0"], (p["dx"], p["dt"], p["nu"]), S.KS
        ref = oracle.ks(u0, *args, c["nsteps"], threads=THREADS)
    else:
        pr = inputs.euler_problem(n=c["n"], dtype=c["dtype"])
        u0 = pr["U0"] if c["bc"] == 1 else smooth_euler(c["n"], c["dtype"])
        args, sc = (pr["dx"], pr["dt"], pr["gamma"]), S.EULER
        ref = oracle.euler(u0, *args, c["nsteps"], bc=c["bc"], threads=THREADS)
    sol = S.Solver(sc, code, c["n"], *args, bc=c["bc"], tile_w=c["W"], threads=c["threads"], chunk=c["chunk"],
                   persistent=int(c["mode"] == "persistent"), cluster=int(c["mode"] == "cluster"),
                   warp_tiles=int(c["mode"] == "warp"))
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    v = u.clone()
    sol.step(u, c["nsteps"])
    sol.classic(v, c["nsteps"])
    torch.cuda.synchronize()
    sol.sync_status()
    sol.close()
    if S.DEBUG_BUILD:
        enabled, rec = S.debug_status()
        assert enabled and rec is None, rec
    got = u.cpu().numpy()
    assert np.array_equal(got, v.cpu().numpy()), "swept != classic"
    assert np.array_equal(got, ref), "swept != oracle"


# --- the 2D decomposition ---------------------------------------------------------------------

def draw2d(rnd):
    dtype = rnd.choice([np.float64, np.float32])
    W = rnd.choice([8, 12, 16, 20, 24, 32, 48, 64] + ([96, 128] if dtype == np.float32 else []))
    nx, ny = W * rnd.randint(2, 9), W * rnd.randint(2, 9)
    threads = rnd.choice([32, 64, 128, 256, 512, 1024])
    return dict(dtype=dtype, W=W, nx=nx, ny=ny, threads=threads, bc=rnd.choice([0, 1]),
                persistent=rnd.choice([0, 1]), nsteps=rnd.randint(1, 3 * W))


CASES2D = [draw2d(random.Random(20161209 + i)) for i in range(30)]


@pytest.mark.parametrize("case", CASES2D, ids=["%s-%dx%d-W%d-t%d-bc%d-p%d-s%d" % (
    "f64" if c["dtype"] == np.float64 else "f32", c["nx"], c["ny"], c["W"], c["threads"], c["bc"], c["persistent"],
    c["nsteps"]) for c in CASES2D])
def test_random_configuration_2d(S, case):
    import torch

    c = case
    code = S.F64 if c["dtype"] == np.float64 else S.F32
    q = inputs.heat2d_problem(nx=c["nx"], ny=c["ny"], dtype=c["dtype"])
    sol = S.Solver2D(code, c["nx"], c["ny"], q["dx"], q["dt"], q["alpha"], tile_w=c["W"], threads=c["threads"],
                     bc=c["bc"], persistent=c["persistent"])
    u = torch.from_numpy(q["u0"]).cuda()
    v = u.clone()
    sol.step(u, c["nsteps"])
    sol.classic(v, c["nsteps"])
    torch.cuda.synchronize()
    sol.sync_status()
    sol.close()
    if S.DEBUG_BUILD:
        enabled, rec = S.debug_status()
        assert enabled and rec is None, rec
    ref = oracle.heat2d(q["u0"], q["dx"], q["dt"], q["alpha"], c["nsteps"], bc=c["bc"], threads=THREADS)
    assert np.array_equal(u.cpu().numpy(), v.cpu().numpy()), "2D swept != classic"
    assert np.array_equal(u.cpu().numpy(), ref), "2D swept != oracle"
