"""A grid split over several ranks, on the GPU (include/swept_slab.h).

All ranks of the partition run in this one process on one GPU and one stream
(run_slabs_local): launch i of every rank, then the transfers after it as
device copies, so no kernel ever waits on another.  The gathered result must
equal the whole-grid swept solve (swept_step_n), the classic path and the
oracle bit for bit: the partition changes where each (point, sub-timestep) is
computed, never how (Section "Related work"; the swept rule of Section
"First-order" with the edges of Fig. collection traded between ranks, the
multi-GPU solver of Section "Conclusion").
"""
import os

import numpy as np
import pytest
import torch

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


def problem(S, scheme, n, dtype, bc):
    if scheme == "heat":
        p = inputs.heat_problem(n=n, dtype=dtype)
        args = (p["dx"], p["dt"], p["alpha"])
        return S.HEAT, p["u0"], args, lambda u, k: oracle.heat(u, *args, k, bc=bc, threads=THREADS)
    if scheme == "ks":
        p = inputs.ks_problem(n=n, dtype=dtype)
        args = (p["dx"], p["dt"], p["nu"])
        return S.KS, p["u0"], args, lambda u, k: oracle.ks(u, *args, k, threads=THREADS)
    pr = inputs.euler_problem(n=n, dtype=dtype)
    args = (pr["dx"], pr["dt"], pr["gamma"])
    return S.EULER, pr["U0"], args, lambda u, k: oracle.euler(u, *args, k, bc=bc, threads=THREADS)


CASES = [
    # scheme, n, bc, dtype, tile_w, threads, warp_tiles, nranks, nsteps
    ("heat", 1024, 0, np.float64, 64, 64, 0, 1, 1001),
    ("heat", 1024, 0, np.float64, 64, 64, 0, 2, 1001),
    ("heat", 1024, 1, np.float64, 64, 64, 0, 3, 777),
    ("heat", 1009, 1, np.float32, 32, 32, 0, 5, 501),     # ragged grid: wide last tile
    ("heat", 65536, 0, np.float32, 1024, 256, 0, 4, 3000),
    ("heat", 4096, 0, np.float64, 64, 32, 1, 3, 999),     # warp tiles
    ("ks", 1 << 14, 0, np.float64, 256, 256, 0, 2, 601),
    ("ks", 1 << 14, 0, np.float32, 512, 256, 0, 7, 433),
    ("ks", 4099, 0, np.float64, 128, 128, 0, 3, 257),
    ("ks", 1 << 16, 0, np.float64, 1024, 512, 0, 8, 300),
    ("euler", 4096, 1, np.float64, 128, 128, 0, 3, 301),
    ("euler", 1009, 1, np.float64, 64, 64, 0, 4, 123),
    ("euler", 1 << 16, 1, np.float64, 512, 128, 0, 6, 97),
]


def solve_split(S, code, u0, args, n, dtype, bc, W, threads, warp, nranks, nsteps):
    slabs = [S.Slab(code, S.F32 if dtype == np.float32 else S.F64, n, *args, r, nranks, bc=bc, tile_w=W,
                    threads=threads, warp_tiles=warp) for r in range(nranks)]
    ug = torch.from_numpy(np.ascontiguousarray(u0))
    states = [s.local_state(ug) for s in slabs]
    S.run_slabs_local(slabs, states, nsteps)
    torch.cuda.synchronize()
    C = 3 if code == S.EULER else 1
    out = np.concatenate([s.owned(u).cpu().numpy() for s, u in zip(slabs, states)], axis=1)
    for s in slabs:
        s.close()
    return out.reshape(C * n) if C > 1 else out.reshape(n)


@pytest.mark.parametrize("scheme,n,bc,dtype,W,threads,warp,nranks,nsteps", CASES)
def test_split_grid_equals_whole_grid_and_oracle(S, scheme, n, bc, dtype, W, threads, warp, nranks, nsteps):
    code, u0, args, ref_fn = problem(S, scheme, n, dtype, bc)
    got = solve_split(S, code, u0, args, n, dtype, bc, W, threads, warp, nranks, nsteps)
    sol = S.Solver(code, S.F32 if dtype == np.float32 else S.F64, n, *args, bc=bc, tile_w=W, threads=threads,
                   warp_tiles=warp)
    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    sol.close()
    whole = u.cpu().numpy().reshape(-1)
    assert np.array_equal(got.reshape(-1), whole), "split grid differs from the whole-grid swept solve"
    assert np.array_equal(whole, v.cpu().numpy().reshape(-1)), "swept and classic differ"
    ref = ref_fn(u0, nsteps)
    assert np.array_equal(got.reshape(-1), np.asarray(ref).reshape(-1)), "split grid differs from the oracle"


def test_split_grid_two_solves_in_a_row(S):
    """The rank keeps owning [x0, x1) after a solve, so a second solve continues from it."""
    code, u0, args, ref_fn = problem(S, "ks", 4096, np.float64, 0)
    slabs = [S.Slab(code, S.F64, 4096, *args, r, 3, tile_w=256, threads=128) for r in range(3)]
    states = [s.local_state(torch.from_numpy(u0)) for s in slabs]
    S.run_slabs_local(slabs, states, 133)   # odd number of full passes and a remainder
    S.run_slabs_local(slabs, states, 200)
    torch.cuda.synchronize()
    got = np.concatenate([s.owned(u).cpu().numpy() for s, u in zip(slabs, states)], axis=1).reshape(-1)
    assert np.array_equal(got, ref_fn(u0, 333))
    for s in slabs:
        s.close()


# --- ranks as processes, one GPU, messages through host memory --------------------------------

def _free_port():
    import socket

    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _gpu_rank(rank, world, port, case, q):
    try:
        from datetime import timedelta

        import torch.distributed as dist

        os.environ["MASTER_ADDR"] = "127.0.0.1"
        os.environ["MASTER_PORT"] = str(port)
        torch.cuda.set_device(0)
        dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=120))
        from paper_1612_02495_gb300 import swept as S

        scheme, n, bc, W, nsteps = case
        code, u0, args, ref_fn = problem(S, scheme, n, np.float64, bc)
        slab = S.Slab(code, S.F64, n, *args, rank, world, bc=bc, tile_w=W)
        u = slab.local_state(torch.from_numpy(np.ascontiguousarray(u0)))
        slab.step(u, nsteps, S.dist_transport(stage_on_host=True))
        torch.cuda.synchronize()
        got = slab.owned(u).cpu().numpy()
        x0, x1 = slab.layout["x0"], slab.layout["x1"]
        ref = np.asarray(ref_fn(u0, nsteps)).reshape(-1, n)[:, x0:x1]
        ok = bool(np.array_equal(got, ref))
        slab.close()
        dist.destroy_process_group()
        q.put((rank, ok, "" if ok else "max abs diff %g" % float(np.max(np.abs(got - ref)))))
    except Exception as e:  # reported to the parent
        q.put((rank, False, repr(e)))


@pytest.mark.parametrize("world,case", [
    (2, ("ks", 1 << 14, 0, 256, 601)),
    (3, ("heat", 1024, 1, 64, 333)),
    (2, ("euler", 4096, 1, 128, 201)),
])
def test_ranks_as_processes_on_one_gpu(S, world, case):
    """Each rank is its own process with its own CUDA context on the one GPU; the ranks trade
    through a gloo process group with the messages staged in host memory (dist_transport), so
    no kernel waits on another rank's kernel.  Every rank's points equal the oracle's."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_gpu_rank, args=(r, world, port, case, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=600) for _ in ps]
    for p in ps:
        p.join(timeout=120)
    for rank, ok, msg in res:
        assert ok, (rank, msg)
