"""Autotuner for the swept plans: tile width W (which fixes the sub-timesteps
per pass, h = W / 2r) and threads per block.

The paper runs every power-of-two block size from 32 to 1024 and keeps the
best per problem size (Section "Results").  This tuner does the same on the
GPU at hand, by timing short probes of the real kernels with CUDA events,
and caches the winners in a JSON file keyed by device, scheme, dtype and size.

  tune_single(scheme, dtype, n, ...)  -> {"tile_w", "threads", "warp_tiles", "persistent", "cluster", "ms"}
  tune_batch(problems, dtype, ...)    -> {"tile_w", "threads", "rule", "ms"} for one batch plan

Both only launch the library's kernels through the C ABI.
"""
import json
import os

import numpy as np

from . import inputs
from . import swept as S

DEFAULT_CACHE = os.path.join(os.path.expanduser("~"), ".cache", "paper_1612_02495_gb300", "tune.json")
THREADS = (32, 64, 128, 256, 512)
MAX_CLUSTER_TILES = 16  # the largest (non-portable) thread-block cluster


def _radius(scheme):
    return 1 if scheme == S.HEAT else 2


def tile_candidates(scheme, n, max_w=1024, min_w=None):
    """Legal tile widths: multiples of 4r with at least 2 tiles.  Widths that
    divide n come first (powers of two, or n's other divisors when n is not a
    power of two); when no multiple of 4r divides n, the powers of two among
    the legal widths (the last tile then carries the n mod W extra points).
    Widths below min_w (default: 32, or 64 from 2^16 points on) are skipped."""
    q = 4 * _radius(scheme)
    if min_w is None:
        min_w = 64 if n >= (1 << 16) else 32
    legal = [w for w in range(q, max_w + 1, q) if n // w >= 2 and w >= min(min_w, max(q, n // 2))]
    out = [w for w in legal if n % w == 0] or legal
    pw = [w for w in out if w & (w - 1) == 0]
    return pw if pw else out


def _device_key():
    import torch

    p = torch.cuda.get_device_properties(torch.cuda.current_device())
    return "%s/%d" % (p.name, p.multi_processor_count)


def _load(path):
    try:
        with open(path) as f:
            return json.load(f)
    except Exception:
        return {}


def _store(path, table):
    try:
        os.makedirs(os.path.dirname(path), exist_ok=True)
        tmp = path + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1, sort_keys=True)
        os.replace(tmp, path)
    except OSError:
        pass


def problem(scheme, dtype, n):
    """Seeded initial state, (dx, dt, param) and boundary condition of the
    workload the tuner probes (the same recipe the tests and the bench use)."""
    npd = np.float64 if dtype == S.F64 else np.float32
    if scheme == S.KS:
        p = inputs.ks_problem(n=n, dtype=npd)
        return p["u0"], (p["dx"], p["dt"], p["nu"]), S.BC_PERIODIC
    if scheme == S.HEAT:
        p = inputs.heat_problem(n=n, dtype=npd)
        return p["u0"], (p["dx"], p["dt"], p["alpha"]), S.BC_PERIODIC
    p = inputs.euler_problem(n=n, dtype=npd)
    return p["U0"], (p["dx"], p["dt"], p["gamma"]), S.BC_REFLECTIVE


def _time(fn, reps):
    import torch

    fn()
    torch.cuda.synchronize()
    best = None
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        fn()
        b.record()
        torch.cuda.synchronize()
        t = a.elapsed_time(b)
        best = t if best is None else min(best, t)
    return best


def warp_tile_ok(scheme, W, n=None):
    """Tile widths the register (warp-tile) mapping supports: W = 32 P with
    P in {1, 2, 4, 8}, dividing n; heat and KS only."""
    P = W // 32
    return scheme != S.EULER and W % 32 == 0 and P in (1, 2, 4, 8) and (n is None or n % W == 0)


def tune_single(scheme, dtype, n, probe_steps=None, cache=DEFAULT_CACHE, refresh=False, reps=2, threads=THREADS,
                modes=(0, 1, 2), warp_tiles=True):
    """Best (tile_w, threads, warp_tiles, persistent, cluster) for swept_step_n
    on an n-point problem.  Tier mappings: shared-memory tiers with each of
    `threads`, and (warp_tiles) one warp per tile with the tier rows in
    registers.  Modes: 0 one launch per pass; 1 one persistent kernel; 2 one
    thread-block cluster holding every tile (tried only with at most
    MAX_CLUSTER_TILES tiles)."""
    import torch

    table = _load(cache) if cache else {}
    key = "single4/%s/%d/%d/%d/%s/%d" % (_device_key(), scheme, dtype, n, probe_steps, int(warp_tiles))
    if not refresh and key in table:
        return table[key]
    u0, args, bc = problem(scheme, dtype, n)
    h_steps = max(tile_candidates(scheme, n)) // (2 * _radius(scheme))
    steps = probe_steps or max(64, 4 * h_steps)
    best = None
    d0 = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    for W in tile_candidates(scheme, n):
        mappings = [(t, 0) for t in threads if t <= max(32, 2 * W)]
        if warp_tiles and warp_tile_ok(scheme, W, n):
            mappings.append((32, 1))
        for t, wt in mappings:
            for mode in modes:
                if mode == 2 and (n // W > MAX_CLUSTER_TILES or n % W):
                    continue
                try:
                    sol = S.Solver(scheme, dtype, n, *args, bc=bc, tile_w=W, threads=t, persistent=int(mode == 1),
                                   cluster=int(mode == 2), warp_tiles=wt)
                except S.SweptError:
                    continue  # e.g. a cluster window that does not fit in shared memory
                u = d0.clone()
                ms = _time(lambda: sol.step(u, steps), reps)
                sol.close()
                if best is None or ms < best["ms"]:
                    best = {"tile_w": W, "threads": t, "warp_tiles": wt, "persistent": int(mode == 1),
                            "cluster": int(mode == 2), "ms": ms, "probe_steps": steps}
    if cache:
        table = _load(cache)
        table[key] = best
        _store(cache, table)
    return best


def solver_from_plan(scheme, dtype, n, dx, dt, param0, plan, bc=S.BC_PERIODIC):
    """A Solver configured with a tune_single result."""
    return S.Solver(scheme, dtype, n, dx, dt, param0, bc=bc, tile_w=plan["tile_w"], threads=plan["threads"],
                    persistent=plan.get("persistent", 0), cluster=plan.get("cluster", 0),
                    warp_tiles=plan.get("warp_tiles", 0))


def tune_2d(dtype, nx, ny, probe_steps=200, tiles=(16, 32, 64, 128), threads=(256, 512, 1024), modes=(0, 1),
            cache=DEFAULT_CACHE, refresh=False, reps=2):
    """Best (tile_w, threads, persistent) for swept2d_step_n on an nx x ny 2D heat
    problem; modes: 0 one launch per pass, 1 the persistent queue kernel."""
    import torch

    table = _load(cache) if cache else {}
    key = "2d2/%s/%d/%d/%d/%d/%s" % (_device_key(), dtype, nx, ny, probe_steps, "".join(str(m) for m in modes))
    if not refresh and key in table:
        return table[key]
    npd = np.float64 if dtype == S.F64 else np.float32
    p = inputs.heat2d_problem(nx=nx, ny=ny, dtype=npd)
    d0 = torch.from_numpy(p["u0"]).cuda()
    best = None
    for W in tiles:
        for t in threads:
            for m in modes:
                try:
                    sol = S.Solver2D(dtype, nx, ny, p["dx"], p["dt"], p["alpha"], tile_w=W, threads=t, persistent=m)
                except S.SweptError:
                    continue  # tile not legal for this grid or dtype
                u = d0.clone()
                ms = _time(lambda: sol.step(u, probe_steps), reps)
                sol.sync_status()
                sol.close()
                if best is None or ms < best["ms"]:
                    best = {"tile_w": W, "threads": t, "persistent": m, "ms": ms, "probe_steps": probe_steps}
    if cache:
        table = _load(cache)
        table[key] = best
        _store(cache, table)
    return best


def _batch_tile(n, plan):
    """Tile width of an n-point batch problem under a batch plan: a uniform W
    where it divides n with two tiles, else the library default (0); or, for a
    size rule (cap, div), the largest power of two <= min(cap, n // div) that
    divides n."""
    rule = plan.get("rule")
    if rule:
        cap, div = rule
        w = 1
        while w * 2 <= min(cap, n // div):
            w *= 2
        while w >= 8 and n % w:
            w //= 2
        return w if w >= 8 and n // w >= 2 else 0
    W = plan["tile_w"]
    return W if (n % W == 0 and n // W >= 2) else 0


def tune_batch(problems, dtype, tiles=(128, 256, 512, 1024), threads=(64, 128, 256),
               rules=((1024, 4), (1024, 8), (512, 4), (1024, 16)), probe_fraction=0.05, cache=DEFAULT_CACHE,
               refresh=False, reps=1):
    """Best plan for a batch: every candidate is timed on the whole batch with
    each problem's step count scaled by probe_fraction (at least one step).
    First one tile width for every problem ({"tile_w", "threads"}); then, with
    the best thread count, tile widths by size class ({"rule": (cap, div)}: the
    largest power of two up to min(cap, n / div) for each problem)."""
    import torch

    sig = (len(problems), int(sum(q["n"] for q in problems)), int(sum(q["nsteps"] for q in problems)))
    table = _load(cache) if cache else {}
    key = "batch2/%s/%d/%d/%d/%d" % ((_device_key(), dtype) + sig)
    if not refresh and key in table:
        return table[key]
    probe = []
    for q in problems:
        r = dict(q)
        r["nsteps"] = max(1, int(q["nsteps"] * probe_fraction))
        probe.append(r)

    def trial(plan):
        tried = [dict(q, tile_w=_batch_tile(q["n"], plan)) for q in probe]
        b = S.Batch(tried, dtype, threads=plan["threads"])
        u0 = b.pack([q["u0"] for q in problems])
        u = u0.clone()
        ms = _time(lambda: (u.copy_(u0), b.run(u)), reps)
        b.close()
        del u, u0
        torch.cuda.empty_cache()
        return ms

    best = None
    for W in tiles:
        for t in threads:
            plan = {"tile_w": W, "threads": t, "rule": None}
            ms = trial(plan)
            if best is None or ms < best["ms"]:
                best = dict(plan, ms=ms, probe_fraction=probe_fraction)
    for rule in rules:
        plan = {"tile_w": 0, "threads": best["threads"], "rule": list(rule)}
        ms = trial(plan)
        if ms < best["ms"]:
            best = dict(plan, ms=ms, probe_fraction=probe_fraction)
    if cache:
        table = _load(cache)
        table[key] = best
        _store(cache, table)
    return best


def apply_batch_plan(problems, plan):
    """Problems with the tuned tile width set (a uniform width where it divides n,
    else the library default; or the plan's size rule)."""
    return [dict(q, tile_w=_batch_tile(q["n"], plan)) for q in problems]
