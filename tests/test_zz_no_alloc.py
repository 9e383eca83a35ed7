"""swept_step_n_static: the entry point that allocates nothing.

It serves callers that cannot call cudaMalloc (their device memory is owned by
an outside memory manager, or a cudaMalloc would synchronise a loop that must
not stall): the edge buffers live in a fixed 8 MiB array inside the library.
This test calls it through the C ABI twice in a row on the same state and
checks each result against swept_step_n, the entry point with bound
workspace, advanced the same way.  It must pass alone in a fresh process and
after every other test (the array keeps the previous call's contents).
"""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_1612_02495_gb300 import inputs

pytestmark = pytest.mark.gpu


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def scratch_bytes():
    """SWEPT_STATIC_SCRATCH_BYTES as include/swept.h defines it."""
    text = open(os.path.join(ROOT, "include", "swept.h")).read()
    m = re.search(r"#define\s+SWEPT_STATIC_SCRATCH_BYTES\s+\((\d+)u\s*<<\s*(\d+)\)", text)
    return int(m.group(1)) << int(m.group(2))


def largest_fp64_ks_grid():
    """The largest power-of-two FP64 KS grid whose two edge buffers (2 n values each) fit the array."""
    n = 1
    while 4 * (2 * n) * 8 <= scratch_bytes():
        n *= 2
    return n


@pytest.fixture(scope="module")
def S():
    from paper_1612_02495_gb300 import build as libbuild

    libbuild.build()
    from paper_1612_02495_gb300 import swept

    return swept


CASES = [
    # scheme, dtype, n, tile_w, (steps of call 1, steps of call 2)
    ("ks", "f64", 1 << 14, 256, (777, 1234)),
    ("ks", "f32", 1 << 12, 64, (300, 41)),
    ("heat", "f64", 1024, 64, (1001, 333)),
    ("euler", "f64", 1024, 32, (120, 77)),
]


def problem(S, kind, dtype, n):
    npd = np.float64 if dtype == "f64" else np.float32
    if kind == "ks":
        p = inputs.ks_problem(n=n, dtype=npd)
        return S.KS, p["u0"], p["dx"], p["dt"], p["nu"], S.BC_PERIODIC
    if kind == "heat":
        p = inputs.heat_problem(n=n, dtype=npd)
        return S.HEAT, p["u0"], p["dx"], p["dt"], p["alpha"], S.BC_PERIODIC
    p = inputs.euler_problem(n=n, dtype=npd)
    return S.EULER, p["U0"], p["dx"], p["dt"], p["gamma"], S.BC_REFLECTIVE


@pytest.mark.parametrize("kind,dtype,n,W,calls", CASES)
def test_static_scratch_matches_workspace_entry(S, kind, dtype, n, W, calls):
    import torch

    scheme, u0, dx, dt, p0, bc = problem(S, kind, dtype, n)
    dt_code = S.F64 if dtype == "f64" else S.F32
    ref = S.Solver(scheme, dt_code, n, dx, dt, p0, bc=bc, tile_w=W)
    cfg = S.make_config(scheme, dt_code, n, dx, dt, p0, bc=bc, tile_w=W)
    a = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    b = a.clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    tol = 1e-12 if dtype == "f64" else 1e-5
    for nsteps in calls:
        st = S.swept_step_n_static(ctypes.byref(cfg), ctypes.c_void_p(a.data_ptr()), nsteps, stream)
        assert st == S.SWEPT_OK, S.STATUS_NAMES.get(st, st)
        ref.step(b, nsteps)
        torch.cuda.synchronize()
        x, y = a.cpu().numpy().astype(np.float64), b.cpu().numpy().astype(np.float64)
        assert np.max(np.abs(x - y)) <= tol * np.max(np.abs(y))
        assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())
    ref.close()


def test_static_scratch_accepts_the_largest_grid_that_fits(S):
    """n = 2^18 FP64 KS needs 4 * n * 8 bytes = the whole array: accepted, and
    equal to swept_step_n."""
    import torch

    n = largest_fp64_ks_grid()
    assert 4 * n * 8 == scratch_bytes()
    p = inputs.ks_problem(n=n)
    cfg = S.make_config(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], tile_w=1024)
    a = torch.from_numpy(p["u0"]).cuda()
    b = a.clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert S.swept_step_n_static(ctypes.byref(cfg), ctypes.c_void_p(a.data_ptr()), 300, stream) == S.SWEPT_OK
    ref = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], tile_w=1024)
    ref.step(b, 300)
    torch.cuda.synchronize()
    ref.close()
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def test_static_scratch_large_tile_keeps_a_handles_opt_in(S):
    """A static call whose tile needs more than 48 KB of shared memory (Euler
    FP64, tile 512: about 50 KB), made between two solves of a handle with a
    larger tile (tile 1024: about 99 KB), must not lower the kernels' opt-in
    limit: the handle's next solve (a fresh graph capture) still succeeds and
    every result equals classic."""
    import torch

    n = 1 << 16
    p = inputs.euler_problem(n=n)
    big = S.Solver(S.EULER, S.F64, n, p["dx"], p["dt"], p["gamma"], bc=S.BC_REFLECTIVE, tile_w=1024)
    assert big.plan["smem_bytes"] > 96 * 1024
    a = torch.from_numpy(p["U0"]).cuda()
    ref = a.clone()
    big.step(a, 40)
    big.classic(ref, 40)
    cfg = S.make_config(S.EULER, S.F64, n, p["dx"], p["dt"], p["gamma"], bc=S.BC_REFLECTIVE, tile_w=512)
    c = torch.from_numpy(p["U0"]).cuda()
    c_ref = c.clone()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert S.swept_step_n_static(ctypes.byref(cfg), ctypes.c_void_p(c.data_ptr()), 57, stream) == S.SWEPT_OK
    big.classic(c_ref, 57)
    big.step(a, 23)  # a new step count: a new capture of the 99 KB kernels
    big.classic(ref, 23)
    torch.cuda.synchronize()
    big.sync_status()
    big.close()
    assert np.array_equal(c.cpu().numpy(), c_ref.cpu().numpy())
    assert np.array_equal(a.cpu().numpy(), ref.cpu().numpy())


def test_static_scratch_rejects_grids_beyond_its_size(S):
    import torch

    n = 2 * largest_fp64_ks_grid()  # FP64 KS needs 4 * n * 8 bytes = twice the array
    p = inputs.ks_problem(n=n)
    cfg = S.make_config(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"], tile_w=1024)
    u = torch.from_numpy(p["u0"]).cuda()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    st = S.swept_step_n_static(ctypes.byref(cfg), ctypes.c_void_p(u.data_ptr()), 10, stream)
    assert st == S.SWEPT_ENOMEM_WORKSPACE
    torch.cuda.synchronize()
    assert np.array_equal(u.cpu().numpy(), p["u0"])  # nothing ran


def test_static_scratch_requires_tile_width(S):
    cfg = S.make_config(S.KS, S.F64, 1024, 0.785, 0.005, 1.0, tile_w=0)
    assert S.swept_step_n_static(ctypes.byref(cfg), ctypes.c_void_p(0x1000), 10, None) == S.SWEPT_EINVAL
