"""Run one solve of a configuration through the C ABI and print its time.

  python -m paper_1612_02495_gb300.run_case --scheme ks|heat|euler|heat2d --dtype f64 --n 1048576 \\
      --nsteps 600 [--path swept|classic] [--tile 0] [--threads 0] [--chunk 0] [--persistent 0] [--cluster 0] [--warp-tiles 0] [--repeat 1]
  python -m paper_1612_02495_gb300.run_case --scheme batch --dtype f32 --count 4096 [--tile 0] [--threads 0]
      (the batched workload: count heat/KS problems, N = 2^U(10,18) rounded to 1024, 1,000-20,000 steps)
  python -m paper_1612_02495_gb300.run_case --scheme ks --adjoint 1 --n 262144 --nsteps 5000
      (FP64 heat / KS: the checkpointing forward solve, then the reverse sweep; times both)
  python -m paper_1612_02495_gb300.run_case --scheme ks --slab 2 --n 1048576 --nsteps 1000 --tile 1024
      (the grid split over --slab ranks, all in this process on one GPU: every rank's launch i, then
      the transfers after it as device copies; checks the gathered result against swept_step_n)
  python -m torch.distributed.run --nproc-per-node 8 --master-addr 127.0.0.1 -m paper_1612_02495_gb300.run_case \
      --scheme ks --slab-dist 1 --grid 8388608 --nsteps 2000 --tile 1024
      (one rank per process: rank r runs its slab on GPU LOCAL_RANK and trades edges over NCCL; with
      --slab-host 1 every rank uses GPU 0 and the messages go through host memory over gloo; rank 0
      gathers the grid and checks it against a whole-grid swept_step_n on its GPU)

Used to profile a single kernel on a chosen size (e.g. under ncu).  One
untimed warm-up solve precedes the timed repeats.
"""
import argparse
import json
import sys

import numpy as np


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--scheme", default="ks", choices=["heat", "ks", "euler", "heat2d", "batch"])
    ap.add_argument("--dtype", default="f64", choices=["f32", "f64"])
    # --grid is the same option, for launchers whose own options --n would abbreviate (torch.distributed.run)
    ap.add_argument("--n", "--grid", dest="n", type=int, default=1 << 20)
    ap.add_argument("--nsteps", type=int, default=600)
    ap.add_argument("--path", default="swept", choices=["swept", "classic"])
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--threads", type=int, default=0)
    ap.add_argument("--chunk", type=int, default=0)
    ap.add_argument("--persistent", type=int, default=0)
    ap.add_argument("--cluster", type=int, default=0)
    ap.add_argument("--warp-tiles", type=int, default=0)
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--count", type=int, default=4096, help="batch: number of problems")
    ap.add_argument("--adjoint", type=int, default=0, help="heat / KS FP64: time the adjoint sweep")
    ap.add_argument("--slab", type=int, default=0, help="split the grid over this many ranks (one process)")
    ap.add_argument("--slab-dist", type=int, default=0, help="split the grid over the torch.distributed ranks")
    ap.add_argument("--slab-host", type=int, default=0,
                    help="with --slab-dist: all ranks on GPU 0, messages staged through host memory over gloo")
    a = ap.parse_args(argv)

    import torch

    from . import inputs
    from . import swept as S

    npd = np.float64 if a.dtype == "f64" else np.float32
    dt_code = S.F64 if a.dtype == "f64" else S.F32
    if a.scheme == "heat2d":
        return run_heat2d(a, S, inputs, torch, npd, dt_code)
    if a.scheme == "batch":
        return run_batch(a, S, inputs, torch, npd, dt_code)
    if a.adjoint:
        return run_adjoint(a, S, inputs, torch)
    if a.scheme == "heat":
        p = inputs.heat_problem(n=a.n, dtype=npd)
        args = (S.HEAT, dt_code, a.n, p["dx"], p["dt"], p["alpha"], S.BC_PERIODIC)
        u0 = p["u0"]
    elif a.scheme == "ks":
        p = inputs.ks_problem(n=a.n, dtype=npd)
        args = (S.KS, dt_code, a.n, p["dx"], p["dt"], p["nu"], S.BC_PERIODIC)
        u0 = p["u0"]
    else:
        p = inputs.euler_problem(n=a.n, dtype=npd)
        args = (S.EULER, dt_code, a.n, p["dx"], p["dt"], p["gamma"], S.BC_REFLECTIVE)
        u0 = p["U0"]
    if a.slab_dist:
        return run_slab_dist(a, S, torch, args, u0)
    if a.slab:
        return run_slab(a, S, torch, args, u0)
    sol = S.Solver(*args, tile_w=a.tile, threads=a.threads, chunk=a.chunk, persistent=a.persistent,
                   cluster=a.cluster, warp_tiles=a.warp_tiles)
    u_init = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    u = u_init.clone()
    run = sol.step if a.path == "swept" else sol.classic
    run(u, a.nsteps)
    torch.cuda.synchronize()
    times = []
    for _ in range(a.repeat):
        u.copy_(u_init)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(u, a.nsteps)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    sol.sync_status()
    ms = float(np.median(times))
    print(json.dumps({"scheme": a.scheme, "dtype": a.dtype, "n": a.n, "nsteps": a.nsteps, "path": a.path,
                      "plan": sol.plan, "ms": ms,
                      "cell_updates_per_s": a.n * a.nsteps / (ms * 1e-3)}))
    sol.close()
    return 0


def run_slab(a, S, torch, args, u0):
    """The grid split over a.slab ranks in one process, against the whole-grid per-pass solve."""
    scheme, dt_code, n, dx, dt, p0, bc = args
    slabs = [S.Slab(scheme, dt_code, n, dx, dt, p0, r, a.slab, bc=bc, tile_w=a.tile, threads=a.threads,
                    chunk=a.chunk, warp_tiles=a.warp_tiles) for r in range(a.slab)]
    ug = torch.from_numpy(np.ascontiguousarray(u0))
    states = [s.local_state(ug) for s in slabs]
    init = [u.clone() for u in states]
    S.run_slabs_local(slabs, states, a.nsteps)
    torch.cuda.synchronize()

    def solve():
        for u, v in zip(states, init):
            u.copy_(v)
        S.run_slabs_local(slabs, states, a.nsteps)

    ms = _event_ms(torch, solve, a.repeat)
    got = torch.cat([s.owned(u) for s, u in zip(slabs, states)], dim=1).reshape(-1)
    sol = S.Solver(scheme, dt_code, n, dx, dt, p0, bc, tile_w=a.tile, threads=a.threads, chunk=a.chunk,
                   warp_tiles=a.warp_tiles)
    u = ug.cuda()
    whole_ms = _event_ms(torch, lambda: (u.copy_(ug.cuda()), sol.step(u, a.nsteps)), a.repeat)
    torch.cuda.synchronize()
    same = bool(torch.equal(got, u.reshape(-1)))
    print(json.dumps({"scheme": a.scheme, "dtype": a.dtype, "n": n, "nsteps": a.nsteps, "ranks": a.slab,
                      "layout": [s.layout for s in slabs], "ms": ms, "whole_grid_ms": whole_ms,
                      "launches_per_rank": slabs[0].launch_count(a.nsteps), "equal_to_whole_grid": same,
                      "cell_updates_per_s": n * a.nsteps / (ms * 1e-3)}))
    for s in slabs:
        s.close()
    sol.close()
    return 0 if same else 1


def run_slab_dist(a, S, torch, args, u0):
    """The grid split over the ranks of a torch.distributed job, one slab per process."""
    import os

    import torch.distributed as dist

    rank, world = int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    torch.cuda.set_device(0 if a.slab_host else local)
    dist.init_process_group("gloo" if a.slab_host else "nccl", rank=rank, world_size=world)
    scheme, dt_code, n, dx, dt, p0, bc = args
    slab = S.Slab(scheme, dt_code, n, dx, dt, p0, rank, world, bc=bc, tile_w=a.tile, threads=a.threads,
                  chunk=a.chunk, warp_tiles=a.warp_tiles)
    ug = torch.from_numpy(np.ascontiguousarray(u0))
    u = slab.local_state(ug)
    init = u.clone()
    transport = S.dist_transport(stage_on_host=bool(a.slab_host))
    slab.step(u, a.nsteps, transport)  # warm-up
    torch.cuda.synchronize()
    times = []
    for _ in range(a.repeat):
        u.copy_(init)
        dist.barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        slab.step(u, a.nsteps, transport)
        e1.record()
        torch.cuda.synchronize()
        dist.barrier()
        times.append(e0.elapsed_time(e1))
    t = torch.tensor([float(np.median(times))], dtype=torch.float64, device="cpu" if a.slab_host else "cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)  # the slowest rank
    owned = slab.owned(u).cpu()
    parts = [None] * world
    dist.all_gather_object(parts, (slab.layout["x0"], owned.numpy()))
    same = None
    if rank == 0:
        got = np.concatenate([p[1] for p in sorted(parts, key=lambda q: q[0])], axis=1).reshape(-1)
        sol = S.Solver(scheme, dt_code, n, dx, dt, p0, bc, tile_w=a.tile, threads=a.threads, chunk=a.chunk,
                       warp_tiles=a.warp_tiles)
        w = ug.cuda()
        sol.step(w, a.nsteps)
        torch.cuda.synchronize()
        same = bool(np.array_equal(got, w.reshape(-1).cpu().numpy()))
        sol.close()
        ms = float(t.item())
        print(json.dumps({"scheme": a.scheme, "dtype": a.dtype, "n": n, "nsteps": a.nsteps, "ranks": world,
                          "backend": "gloo, host-staged, one GPU" if a.slab_host else "nccl, one GPU a rank",
                          "ms": ms, "cell_updates_per_s": n * a.nsteps / (ms * 1e-3),
                          "launches_per_rank": slab.launch_count(a.nsteps), "equal_to_whole_grid": same}))
    slab.close()
    dist.destroy_process_group()
    return 0 if (rank != 0 or same) else 1


def run_heat2d(a, S, inputs, torch, npd, dt_code):
    """2D heat on an n x n grid (--n is the side): swept2d_step_n or classic2d_step_n."""
    p = inputs.heat2d_problem(nx=a.n, ny=a.n, dtype=npd)
    sol = S.Solver2D(dt_code, a.n, a.n, p["dx"], p["dt"], p["alpha"], tile_w=a.tile, threads=a.threads,
                     persistent=1 if a.persistent else 0)
    u_init = torch.from_numpy(p["u0"]).cuda()
    u = u_init.clone()
    run = sol.step if a.path == "swept" else sol.classic
    run(u, a.nsteps)
    torch.cuda.synchronize()
    times = []
    for _ in range(a.repeat):
        u.copy_(u_init)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run(u, a.nsteps)
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    sol.sync_status()
    ms = float(np.median(times))
    print(json.dumps({"scheme": "heat2d", "dtype": a.dtype, "n": a.n, "nsteps": a.nsteps, "path": a.path,
                      "plan": sol.plan, "ms": ms, "cell_updates_per_s": a.n * a.n * a.nsteps / (ms * 1e-3)}))
    sol.close()
    return 0




def _event_ms(torch, fn, repeat):
    times = []
    for _ in range(repeat):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    return float(np.median(times))


def run_batch(a, S, inputs, torch, npd, dt_code):
    """The batched workload with a.count problems, one persistent launch per run."""
    spec = inputs.batch_problems(count=a.count)
    probs = inputs.batch_instances(spec, dtype=npd)
    for q in probs:
        q["tile_w"] = a.tile if a.tile and q["n"] % a.tile == 0 and q["n"] // a.tile >= 2 else 0
    b = S.Batch(probs, dt_code, threads=a.threads)
    u0 = b.pack([q["u0"] for q in probs])
    u = u0.clone()
    b.run(u)
    torch.cuda.synchronize()

    def once():
        u.copy_(u0)
        b.run(u)

    ms = _event_ms(torch, once, a.repeat)
    b.sync_status()
    work = int((spec["n"] * spec["steps"]).sum())
    print(json.dumps({"scheme": "batch", "dtype": a.dtype, "count": a.count, "items": b.items, "ms": ms,
                      "cell_updates_per_s": work / (ms * 1e-3)}))
    b.close()
    return 0


def run_adjoint(a, S, inputs, torch):
    """FP64 heat or KS: the checkpointing forward solve and the reverse sweep."""
    if a.scheme == "ks":
        p = inputs.ks_problem(n=a.n)
        sc, p0 = S.KS, p["nu"]
    elif a.scheme == "heat":
        p = inputs.heat_problem(n=a.n)
        sc, p0 = S.HEAT, p["alpha"]
    else:
        raise SystemExit("the adjoint covers heat and KS")
    sol = S.Solver(sc, S.F64, a.n, p["dx"], p["dt"], p0, tile_w=a.tile, threads=a.threads)
    ckpt = torch.empty(sol.ckpt_size(a.nsteps), dtype=torch.uint8, device="cuda")
    u0 = torch.from_numpy(p["u0"]).cuda()
    gT = torch.from_numpy(inputs.rng(62).standard_normal(a.n)).cuda()
    u = u0.clone()
    sol.forward_ckpt(u, a.nsteps, ckpt)
    sol.adjoint(gT, a.nsteps, ckpt)
    torch.cuda.synchronize()

    def fwd():
        u.copy_(u0)
        sol.forward_ckpt(u, a.nsteps, ckpt)

    f_ms = _event_ms(torch, fwd, a.repeat)
    b_ms = _event_ms(torch, lambda: sol.adjoint(gT, a.nsteps, ckpt), a.repeat)
    sol.sync_status()
    print(json.dumps({"scheme": a.scheme, "adjoint": 1, "n": a.n, "nsteps": a.nsteps, "plan": sol.plan,
                      "forward_ckpt_ms": f_ms, "adjoint_ms": b_ms}))
    sol.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
