"""Solves run under the debug build (libswept_debug.so, SWEPT_DEBUG=1), called by
test_debug_build.py in a child process, because a process loads one build.

Every execution mode of every kernel family runs on small seeded cases:
  - heat, KS and Euler, per pass, persistent and cluster, in shared memory and
    in warp tiles, periodic and insulated, with remainders, and on grids that
    are not a multiple of the tile width;
  - classic;
  - the batched solver, the adjoint, the no-allocation entry point;
  - a grid split over ranks (all ranks in this process), every scheme;
  - 2D per pass and persistent, both boundary conditions.
After each group the debug records must be clean (swept_debug_status), and
every result must equal the oracle bit for bit.  Prints one line per group and
exits non-zero on the first failure.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1612_02495_gb300 import inputs  # noqa: E402


def main():
    import torch

    from paper_1612_02495_gb300 import swept as S

    assert S.DEBUG_BUILD and os.path.basename(S.LIB_PATH) == "libswept_debug.so"
    enabled, rec = S.debug_status()
    assert enabled and rec is None, rec

    def clean(group):
        torch.cuda.synchronize()
        en, r = S.debug_status()
        if r is not None:
            raise SystemExit("%s: debug check failed: %s" % (group, r))
        print("clean:", group, flush=True)

    def run1d(sc, code, u0, args, nsteps, ref, **kw):
        sol = S.Solver(sc, code, u0.shape[-1], *args, **kw)
        u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        v = u.clone()
        sol.step(u, nsteps)
        sol.classic(v, nsteps)
        torch.cuda.synchronize()
        sol.sync_status()
        got = u.cpu().numpy()
        assert np.array_equal(got, v.cpu().numpy()), ("swept != classic", sc, kw)
        assert np.array_equal(got, ref), ("swept != oracle", sc, kw)
        sol.close()

    # heat: shared memory and warp tiles, every mode, both boundary conditions
    for dtype in (np.float64, np.float32):
        code = S.F64 if dtype == np.float64 else S.F32
        for n, W, nsteps, bc, extra in [(5 * 64, 64, 333, 1, {}), (8 * 32, 32, 101, 0, {"persistent": 1}),
                                        (6 * 64, 64, 77, 1, {"cluster": 1}),
                                        (4 * 64, 64, 131, 0, {"warp_tiles": 1}),
                                        (5 * 128, 128, 201, 1, {"warp_tiles": 1, "persistent": 1}),
                                        (3 * 256, 256, 99, 0, {"warp_tiles": 1, "cluster": 1})]:
            p = inputs.heat_problem(n=n, dtype=dtype)
            ref = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, bc=bc)
            run1d(S.HEAT, code, p["u0"], (p["dx"], p["dt"], p["alpha"]), nsteps, ref, bc=bc, tile_w=W, **extra)
    clean("heat")

    for dtype in (np.float64, np.float32):
        code = S.F64 if dtype == np.float64 else S.F32
        for n, W, nsteps, extra in [(3 * 128, 128, 257, {}), (2048, 64, 203, {"persistent": 1}),
                                    (8 * 128, 128, 99, {"cluster": 1}), (2048, 64, 101, {"warp_tiles": 1}),
                                    (4096, 256, 150, {"warp_tiles": 1, "persistent": 1}),
                                    (2048, 128, 77, {"chunk": 2})]:
            p = inputs.ks_problem(n=n, dtype=dtype)
            ref = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], nsteps, threads=8)
            run1d(S.KS, code, p["u0"], (p["dx"], p["dt"], p["nu"]), nsteps, ref, tile_w=W, **extra)
    clean("ks")

    for dtype in (np.float64, np.float32):
        code = S.F64 if dtype == np.float64 else S.F32
        for n, W, nsteps, bc, extra in [(1024, 64, 101, 1, {}), (1024, 64, 77, 1, {"chunk": 2, "threads": 64}),
                                        (2048, 128, 99, 1, {"persistent": 1}), (8 * 64, 64, 55, 1, {"cluster": 1}),
                                        (1024, 128, 33, 0, {})]:
            pr = inputs.euler_problem(n=n, dtype=dtype)
            U0 = pr["U0"]
            if bc == 0:
                x = (np.arange(n) + 0.5) / n
                rho = 1 + 0.2 * np.sin(2 * np.pi * x)
                u = 0.3 + 0.1 * np.cos(2 * np.pi * x)
                pp = 1 + 0.1 * np.sin(4 * np.pi * x)
                U0 = np.stack([rho, rho * u, pp / 0.4 + 0.5 * rho * u * u]).astype(dtype)
            ref = oracle.euler(U0, pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=bc, threads=8)
            run1d(S.EULER, code, U0, (pr["dx"], pr["dt"], pr["gamma"]), nsteps, ref, bc=bc, tile_w=W, **extra)
    clean("euler")

    # grids that are not a multiple of the tile (wide last tile), per pass and persistent
    for dtype in (np.float64, np.float32):
        code = S.F64 if dtype == np.float64 else S.F32
        for n, W, nsteps, bc, extra in [(1009, 64, 301, 0, {}), (1009, 32, 203, 1, {"persistent": 1}),
                                        (2 * 64 + 63, 64, 77, 1, {})]:
            p = inputs.heat_problem(n=n, dtype=dtype)
            ref = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, bc=bc)
            run1d(S.HEAT, code, p["u0"], (p["dx"], p["dt"], p["alpha"]), nsteps, ref, bc=bc, tile_w=W, **extra)
        for n, W, nsteps, extra in [(4099, 256, 155, {}), (1009, 64, 101, {"persistent": 1})]:
            p = inputs.ks_problem(n=n, dtype=dtype)
            ref = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], nsteps, threads=8)
            run1d(S.KS, code, p["u0"], (p["dx"], p["dt"], p["nu"]), nsteps, ref, tile_w=W, **extra)
        for n, W, nsteps, extra in [(1009, 64, 99, {}), (2 * 128 + 1, 128, 71, {"persistent": 1})]:
            pr = inputs.euler_problem(n=n, dtype=dtype)
            ref = oracle.euler(pr["U0"], pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=1, threads=8)
            run1d(S.EULER, code, pr["U0"], (pr["dx"], pr["dt"], pr["gamma"]), nsteps, ref, bc=1, tile_w=W, **extra)
    clean("ragged grids")

    # batched solver
    spec = inputs.batch_problems(count=24, seed=7, log2_lo=10, log2_hi=13, steps_lo=1, steps_hi=300)
    for dtype in (np.float64, np.float32):
        probs = inputs.batch_instances(spec, dtype=dtype)
        b = S.Batch(probs, S.F64 if dtype == np.float64 else S.F32)
        u = b.pack([q["u0"] for q in probs])
        b.run(u)
        torch.cuda.synchronize()
        b.sync_status()
        for q, x in zip(probs, b.unpack(u)):
            if q["scheme"] == 0:
                ref = oracle.heat(q["u0"], q["dx"], q["dt"], q["param"], q["nsteps"])
            else:
                ref = oracle.ks(q["u0"], q["dx"], q["dt"], q["param"], q["nsteps"], threads=8)
            assert np.array_equal(x, ref), ("batch", q["scheme"], q["n"], q["nsteps"])
        b.close()
    clean("batch")

    # adjoint (FP64 KS and heat)
    for sc, n, W, nsteps in [(S.KS, 384, 64, 77), (S.HEAT, 256, 32, 55)]:
        if sc == S.KS:
            p = inputs.ks_problem(n=n, seed=61)
            p0 = 1.0
        else:
            p = inputs.heat_problem(n=n, seed=63)
            p0 = p["alpha"]
        gT = inputs.rng(62).standard_normal(n)
        sol = S.Solver(sc, S.F64, n, p["dx"], p["dt"], p0, tile_w=W)
        ckpt = torch.empty(sol.ckpt_size(nsteps), dtype=torch.uint8, device="cuda")
        u = torch.from_numpy(p["u0"]).cuda()
        sol.forward_ckpt(u, nsteps, ckpt)
        g, _ = sol.adjoint(torch.from_numpy(gT).cuda(), nsteps, ckpt)
        torch.cuda.synchronize()
        sol.sync_status()
        if sc == S.KS:
            ref = oracle.ks_adjoint(p["u0"], p["dx"], p["dt"], p0, nsteps, gT)[0]
        else:
            ref = oracle.heat_adjoint(p["u0"], p["dx"], p["dt"], p0, nsteps, gT)[0]
        assert np.array_equal(g.cpu().numpy(), ref), ("adjoint", sc)
        sol.close()
    clean("adjoint")

    # a grid split over ranks: every rank's state and edge indices checked on the device
    for sc, n, W, nsteps, bc, nranks, extra in [(S.HEAT, 1009, 32, 203, 1, 3, {}), (S.HEAT, 1024, 64, 99, 0, 2,
                                                                                      {"warp_tiles": 1}),
                                                (S.KS, 4099, 128, 97, 0, 4, {}), (S.EULER, 1024, 64, 55, 1, 3, {})]:
        if sc == S.HEAT:
            p = inputs.heat_problem(n=n)
            u0, args = p["u0"], (p["dx"], p["dt"], p["alpha"])
            ref = oracle.heat(u0, *args, nsteps, bc=bc)
        elif sc == S.KS:
            p = inputs.ks_problem(n=n)
            u0, args = p["u0"], (p["dx"], p["dt"], p["nu"])
            ref = oracle.ks(u0, *args, nsteps, threads=8)
        else:
            pr = inputs.euler_problem(n=n)
            u0, args = pr["U0"], (pr["dx"], pr["dt"], pr["gamma"])
            ref = oracle.euler(u0, *args, nsteps, bc=bc, threads=8)
        slabs = [S.Slab(sc, S.F64, n, *args, r, nranks, bc=bc, tile_w=W, **extra) for r in range(nranks)]
        states = [s.local_state(torch.from_numpy(np.ascontiguousarray(u0))) for s in slabs]
        S.run_slabs_local(slabs, states, nsteps)
        torch.cuda.synchronize()
        got = np.concatenate([s.owned(u).cpu().numpy() for s, u in zip(slabs, states)], axis=1)
        assert np.array_equal(got.reshape(-1), np.asarray(ref).reshape(-1)), ("slab", sc, n, nranks)
        for s in slabs:
            s.close()
    clean("slabs")

    # 2D, per pass and persistent, both boundary conditions
    for dtype in (np.float64, np.float32):
        code = S.F64 if dtype == np.float64 else S.F32
        for nx, ny, W, nsteps, bc, pers in [(64, 48, 16, 37, 0, 0), (64, 48, 16, 37, 1, 1), (96, 64, 32, 100, 1, 0),
                                            (128, 128, 32, 70, 0, 1), (32, 32, 16, 7, 1, 1)]:
            q = inputs.heat2d_problem(nx=nx, ny=ny, dtype=dtype)
            sol = S.Solver2D(code, nx, ny, q["dx"], q["dt"], q["alpha"], tile_w=W, bc=bc, persistent=pers)
            u = torch.from_numpy(q["u0"]).cuda()
            v = u.clone()
            sol.step(u, nsteps)
            sol.classic(v, nsteps)
            torch.cuda.synchronize()
            sol.sync_status()
            ref = oracle.heat2d(q["u0"], q["dx"], q["dt"], q["alpha"], nsteps, bc=bc, threads=8)
            assert np.array_equal(u.cpu().numpy(), ref), ("2d", nx, ny, W, bc, pers)
            assert np.array_equal(v.cpu().numpy(), ref), ("2d classic", nx, ny, W, bc)
            sol.close()
    clean("2d")
    print("all clean")


if __name__ == "__main__":
    main()
