"""Benchmark: swept vs classic decomposition, Kuramoto-Sivashinsky, 1 GB300.

Workload (one bench step = one whole solve): KS u_t = -u u_x - u_xx - u_xxxx,
periodic, N = 2^20 FP64 points, L = 32 pi N / 128, dt = 0.005, IC
cos(x/16)(1 + sin(x/16)) + 1e-3 U(-1, 1) (seeded), 50,000 midpoint-RK2 steps,
swept rule with the library's default plan.  Metric: cell-updates/s
(N * timesteps / wall time), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (plain C, OpenMP over the host cores) on
a bounded window of the same workload; it is the reference arm of this repo.
Under torchrun (N > 1) every rank solves its own replica (weak scaling, no
collective on the data path); rank 0 prints one JSON line.
"""
import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N = 1 << 20
NSTEPS = 50000
METRIC = "cell-updates/s swept vs classic per-step GPU at 1 GB300; adjoint/forward time"
UNIT = "cell-updates/s"
WORKLOAD = "Kuramoto-Sivashinsky N=2^20 FP64 periodic, 50,000 midpoint-RK2 steps (dt=0.005, dx=pi/4)"
FP64_FLOPS_PER_SUBSTEP = 18  # 7 fma (2 flops) + 2 add + 2 mul per point per sub-timestep
FP64_INSTR_PER_SUBSTEP = 11
CLASSIC_BYTES_PER_UPDATE = 40
# FP64 roof of GB300: 152 SMs x 2 DFMA per clock x 2 flops x 2.07 GHz (nominal 1.25 TFLOP/s);
# the issue-rate probe measured 0.60e12 DFMA/s.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP64_INSTR_PEAK = 152 * 2 * 2.07e9
# Measured ceiling for FP64 instructions with two or more register operands, which every
# instruction of a stencil update has: the KS update's exact mix issues at 0.535e12/s
# (python -m paper_1612_02495_gb300.peaks; the nominal rate needs constant-bank operands).
FP64_KS_MIX_CEILING = 0.535e12
# dram__bytes_read.sum + dram__bytes_write.sum of one k_swept_diamond<double, KsOp> launch at
# N = 2^20, tile 1024, from an ncu capture; None: no capture of the current kernel
DIAMOND_TRAFFIC_BYTES = None
# the same for one k_swept_persist<double, KsOp> launch (a whole 50,000-step solve), per plan
# (tile, threads): dram__bytes_read.sum + dram__bytes_write.sum from an ncu capture of just those
# two counters and the duration, on the current kernel (tile 1024 / 512 threads: 11.56 MB read +
# 36.78 MB written; tile 1024 / 256 threads: 9.23 MB + 5.75 MB); a plan without a capture
# reports None
PERSIST_TRAFFIC = {(1024, 512): 48339456, (1024, 256): 9232128 + 5747968}


# Measured unit ceilings of GB300 (python -m paper_1612_02495_gb300.peaks, register-only probe loops):
# FP32 FMA 3.917e13/s (2 flops each), conflict-free 32-bit shared-memory loads 3.908e13 B/s.
FP32_PEAK_TFLOPS = 2 * 3.917e13 / 1e12
SMEM_PEAK_GBS = 3.908e13 / 1e9
# Algorithmic work per point-substep, counted from the per-point operators (ops.cuh; the 2D
# heat operator in swept2d.cuh): FP instructions (add, mul, fma; div and sqrt one each), flops
# (fma = 2) and shared-memory accesses per point of a tier in shared memory (stencil loads, the
# second stage's read of the point's own earlier tier, the store).  Euler per cell-substep:
# primitives (2 mul, 1 fma, 1 div), a face flux (2 sides x (12 reconstruction ops, 4 for
# momentum and energy, 1 mul, 1 div, 1 sqrt, 1 add) + 18 for the Rusanov flux), the update of
# 3 components (avg. 9 ops over the two stages).
# FP32 KS tiers advance aligned pairs of points (three paired loads and one paired store per
# pair, plus the second stage's paired read of the points' own earlier tier): 4.5 values a point.
WORK = {
    "heat": {"instr": 3, "flops": 4, "smem_acc": 4.0},
    "ks": {"instr": 11, "flops": 18, "smem_acc": 6.5, "smem_acc_paired_f32": 4.5},
    "euler": {"instr": 71, "flops": 82, "smem_acc": 34.5},
    "heat2d": {"instr": 5, "flops": 6, "smem_acc": 6.0},
}


def alu_roofline(scheme, f64, units, ms, kernel, registers=False, note=None):
    """Roofline of a swept kernel that did `units` point-substeps in `ms`: FP pipe
    (flops against the FP64 or FP32 roof) and shared memory (algorithmic accesses
    of the shared-memory tiers against the probed bandwidth; tiers in registers
    touch shared memory only at pass boundaries)."""
    w = WORK[scheme]
    rate = units / (ms * 1e-3)
    peak = FP64_PEAK_TFLOPS if f64 else FP32_PEAK_TFLOPS
    achieved = w["flops"] * rate / 1e12
    vb = 8 if f64 else 4
    acc = w["smem_acc"] if f64 else w.get("smem_acc_paired_f32", w["smem_acc"])
    smem_gbs = 0.0 if registers else acc * vb * rate / 1e9
    out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
           "traffic": None, "kernel": kernel, "kernel_ms": ms, "units": units,
           "peak_source": ("derived FP64 roof: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz" if f64 else
                           "measured FP32 FMA rate x 2 flop (probe)"),
           "algorithmic_per_unit": {"flops": w["flops"], "fp_instr": w["instr"],
                                    "smem_bytes": 0 if registers else acc * vb},
           "smem": {"achieved": smem_gbs, "peak": SMEM_PEAK_GBS, "unit": "GB/s", "frac": smem_gbs / SMEM_PEAK_GBS,
                    "peak_source": "measured conflict-free shared-memory loads (probe)"}}
    if registers:
        out["smem"]["note"] = "tiers in registers (warp tiles): shared memory only at pass boundaries"
    if note:
        out["note"] = note
    return out


def dominant_swept_kernel(sol, u, u0, nsteps, solve_ms):
    """(kernel name, point-substeps per launch, average launch ms, share) of the
    dominant kernel of a tuned 1D plan: the persistent or cluster kernel is one
    launch per solve (timed by the solve's CUDA events); per-pass plans time the
    diamond launches with CUDA events around each (swept_profile_passes)."""
    plan = sol.plan
    units = sol.n * plan["stages"] * nsteps
    P = plan["tile_w"] // 32 if plan.get("warp_tiles") else 0
    tmpl = "<%s, %s%s>" % ("double" if sol.dtype == 1 else "float",
                          {0: "HeatOp", 1: "KsOp", 2: "EulerOp"}[sol.scheme], ", %d" % P if P else "")
    if plan.get("persistent"):
        return "k_swept_persist" + tmpl, units, solve_ms, 1.0
    if plan.get("cluster"):
        return "k_swept_cluster" + tmpl, units, solve_ms, 1.0
    u.copy_(u0)
    prof = sol.profile_passes(u, nsteps)
    d_ms, d_n = prof["diamond"]
    total = max(sum(v[0] for v in prof.values()), 1e-9)
    if d_n == 0:
        return "all swept passes" + tmpl, units, total, 1.0
    return "k_swept_diamond" + tmpl, sol.n * plan["half_cycle"], d_ms / d_n, d_ms / total


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def max_over_ranks(value, dist, ws, device="cuda"):
    """Largest `value` over all ranks (the whole job takes as long as its slowest rank)."""
    if ws <= 1:
        return float(value)
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(work_per_rank, ms_max, ws):
    """Units processed by all ranks (each rank runs its own replica) per second."""
    return ws * work_per_rank / (ms_max * 1e-3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class Clocks:
    """nvidia-smi sampler running during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: SWEPT_CLOCKS_DIR if set, else the system temporary folder
        out_dir = os.environ.get("SWEPT_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, "swept_bench_clocks_rank%d.csv" % index)

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def cpu_oracle_rate(n, seconds, threads, probe_only=False):
    """Oracle cell-updates/s on a bounded window of the workload (grid N, few steps);
    probe_only: return (None, steps, None) for the window a 2-step probe sizes to `seconds`."""
    import oracle
    from paper_1612_02495_gb300 import inputs

    p = inputs.ks_problem(n=n)
    t0 = time.perf_counter()
    oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], 2, threads=threads)
    per_step = max(time.perf_counter() - t0, 1e-6) / 2
    steps = int(max(2, min(100000, seconds / per_step)))
    if probe_only:
        return None, steps, None
    t0 = time.perf_counter()
    oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], steps, threads=threads)
    dt = time.perf_counter() - t0
    return n * steps / dt, steps, dt


def measure_adjoint(S, inputs, torch, stream, k, barrier):
    """Adjoint workload: KS N=2^18 FP64, 5,000 steps.  Times (CUDA events, median of k)
    the forward solve, the checkpointing forward, and the reverse sweep that continues
    from it (dL/du0 and dL/dnu), with the default (sqrt) checkpoint memory."""
    n, nsteps = 1 << 18, 5000
    p = inputs.ks_problem(n=n, seed=71)
    sol = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], p["nu"])
    u0 = torch.from_numpy(p["u0"]).cuda()
    u = u0.clone()
    nb = sol.ckpt_size(nsteps)
    ck = torch.empty(nb, dtype=torch.uint8, device="cuda")
    gT = torch.from_numpy(inputs.rng(72).standard_normal(n)).cuda()
    g = torch.empty_like(gT)
    gp = torch.zeros(1, dtype=torch.float64, device="cuda")

    def ev(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        return a, b

    res = {"fwd": [], "fwd_ckpt": [], "adj": []}
    for i in range(k + 1):
        u.copy_(u0)
        e1 = ev(lambda: sol.step(u, nsteps))
        u.copy_(u0)
        e2 = ev(lambda: sol.forward_ckpt(u, nsteps, ck))
        e3 = ev(lambda: sol.adjoint(gT, nsteps, ck, g_u0=g, g_param=gp))
        barrier()
        if i > 0:  # first round warms the graphs
            for key, (a, b) in zip(("fwd", "fwd_ckpt", "adj"), (e1, e2, e3)):
                res[key].append(a.elapsed_time(b))
    sol.sync_status()
    seg = sol.plan["half_cycle"] // sol.plan["stages"]
    med = {key: float(np.median(v)) for key, v in res.items()}
    g_small = g.clone()
    # the same gradient with one segment: the forward records every tier (about 21 GB here), so the
    # reverse sweep recomputes nothing
    del ck
    slot = (n * 8 + 255) // 256 * 256
    nb_full = (2 * nsteps + 5) * slot + (1 << 20)
    ck = torch.empty(nb_full, dtype=torch.uint8, device="cuda")
    full = {"fwd_ckpt": [], "adj": []}
    for i in range(k + 1):
        u.copy_(u0)
        e2 = ev(lambda: sol.forward_ckpt(u, nsteps, ck))
        e3 = ev(lambda: sol.adjoint(gT, nsteps, ck, g_u0=g, g_param=gp))
        barrier()
        if i > 0:
            for key, (a, b) in zip(("fwd_ckpt", "adj"), (e2, e3)):
                full[key].append(a.elapsed_time(b))
    sol.sync_status()
    same = bool(torch.equal(g, g_small))
    fmed = {key: float(np.median(v)) for key, v in full.items()}
    del ck
    sol.close()
    return {"workload": "KS N=2^18 FP64, 5,000 steps, L = sum (u(T) - u_target)^2, grad wrt u0 and nu",
            "forward_ms": med["fwd"], "forward_ckpt_ms": med["fwd_ckpt"], "adjoint_ms": med["adj"],
            "adjoint_over_forward": med["adj"] / med["fwd"],
            "forward_plus_adjoint_over_forward": (med["fwd_ckpt"] + med["adj"]) / med["fwd"],
            "ckpt_bytes": nb, "steps_per_pass": seg,
            "one_segment": {"ckpt_bytes": nb_full, "forward_ckpt_ms": fmed["fwd_ckpt"], "adjoint_ms": fmed["adj"],
                            "adjoint_over_forward": fmed["adj"] / med["fwd"],
                            "forward_plus_adjoint_over_forward": (fmed["fwd_ckpt"] + fmed["adj"]) / med["fwd"],
                            "grad_u0_equal_to_checkpointed": same,
                            "note": "every tier taped by the forward; no recompute"}}


def _event_time(torch, stream, fn):
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    fn()
    b.record(stream)
    return a, b


def measure_fp32(S, inputs, autotune, torch, stream, barrier, ws):
    """The same KS workload (N=2^20, 50,000 steps) in FP32: swept vs classic."""
    p = inputs.ks_problem(n=N, dtype=np.float32)
    t = autotune.tune_single(S.KS, S.F32, N, probe_steps=8000)
    sol = autotune.solver_from_plan(S.KS, S.F32, N, p["dx"], p["dt"], p["nu"], t)
    u0 = torch.from_numpy(p["u0"]).cuda()
    u = u0.clone()
    res = {}
    for name, fn in (("swept", sol.step), ("classic", sol.classic)):
        fn(u, NSTEPS)
        barrier()
        ms = []
        for _ in range(2):
            u.copy_(u0)
            ev = _event_time(torch, stream, lambda: fn(u, NSTEPS))
            barrier()
            ms.append(ev[0].elapsed_time(ev[1]))
        res[name] = min(ms)
    sol.sync_status()
    kname, kunits, kms, share = dominant_swept_kernel(sol, u, u0, NSTEPS, res["swept"])
    sol.close()
    rf = alu_roofline("ks", False, kunits, kms, kname, registers=bool(t.get("warp_tiles")))
    rf["kernel_share"] = share
    return {"workload": "KS N=2^20 FP32, 50,000 steps", "tile_w": t["tile_w"], "threads": t["threads"],
            "plan": {k: t.get(k, 0) for k in ("tile_w", "threads", "warp_tiles", "persistent", "cluster")},
            "swept_ms": res["swept"], "classic_ms": res["classic"],
            "swept_value": ws * N * NSTEPS / (res["swept"] * 1e-3),
            "classic_value": ws * N * NSTEPS / (res["classic"] * 1e-3),
            "speedup_vs_classic": res["classic"] / res["swept"], "roofline": rf}


def measure_slab(S, inputs, torch, stream, barrier, ranks=(2, 8), nsteps=2000, W=1024, threads=256):
    """The KS 2^20 FP64 grid split over several ranks, all of them in this process on this GPU
    (launch i of every rank, then the transfers after it as device copies), against the
    whole-grid solve with one launch per pass; each split result must equal the whole grid."""
    p = inputs.ks_problem(n=N)
    ug = torch.from_numpy(p["u0"])
    sol = S.Solver(S.KS, S.F64, N, p["dx"], p["dt"], p["nu"], tile_w=W, threads=threads)
    u = ug.cuda()
    sol.step(u, nsteps)
    barrier()
    u.copy_(ug)
    ev = _event_time(torch, stream, lambda: sol.step(u, nsteps))
    barrier()
    whole_ms = ev[0].elapsed_time(ev[1])
    sol.sync_status()
    sol.close()
    rows = []
    for R in ranks:
        slabs = [S.Slab(S.KS, S.F64, N, p["dx"], p["dt"], p["nu"], r, R, tile_w=W, threads=threads)
                 for r in range(R)]
        states = [s.local_state(ug) for s in slabs]
        init = [x.clone() for x in states]
        S.run_slabs_local(slabs, states, nsteps)
        barrier()
        for x, y in zip(states, init):
            x.copy_(y)
        ev = _event_time(torch, stream, lambda: S.run_slabs_local(slabs, states, nsteps))
        barrier()
        got = torch.cat([s.owned(x) for s, x in zip(slabs, states)], dim=1).reshape(-1)
        rows.append({"ranks": R, "ms": ev[0].elapsed_time(ev[1]), "equal_to_whole_grid": bool(torch.equal(got, u)),
                     "launches_per_rank": slabs[0].launch_count(nsteps),
                     "transfer_values_per_pass": slabs[0].layout["half_cycle"] * 2 * 2})
        for s in slabs:
            s.close()
    return {"workload": "KS N=2^20 FP64, %d steps, split over ranks that all run on this one GPU "
                        "(tile %d, %d threads)" % (nsteps, W, threads),
            "whole_grid_ms": whole_ms, "splits": rows,
            "note": "one GPU runs every rank in turn, so this checks the partition and its launch cost, "
                    "not multi-GPU throughput"}


def measure_batch(S, inputs, autotune, torch, stream, barrier, ws, with_f64):
    """Batched workload: 4096 heat/KS problems, N = 2^U(10,18) rounded to 1024,
    1,000-20,000 steps, one persistent launch per run; FP32 (and FP64 on request)."""
    spec = inputs.batch_problems()
    work = int((spec["n"] * spec["steps"]).sum())
    out = {"workload": "4096 problems, N=2^U(10,18) (multiples of 1024), heat/KS 50/50, steps U{1000..20000}",
           "cell_updates": work}
    # point-substeps and flops of the whole batch (heat: 1 sub-step per step, KS: 2)
    heat = spec["kind"] == 0
    units = int((spec["n"] * spec["steps"] * np.where(heat, 1, 2)).sum())
    flops = float((spec["n"] * spec["steps"] * np.where(heat, WORK["heat"]["flops"], 2 * WORK["ks"]["flops"])).sum())
    smem_ks = {True: WORK["ks"]["smem_acc"], False: WORK["ks"]["smem_acc_paired_f32"]}
    # Runs of more than about 15 s are timed once, their graph capture inside the timed region
    # (a few ms); the FP32 swept batch (about 2 s) gets a warm-up and the best of two.
    # The FP64 tuner probes a narrower candidate set (each FP64 probe takes about 2.4 s).
    for dt, code, name in ((np.float32, S.F32, "f32"), (np.float64, S.F64, "f64")):
        if code == S.F64 and not with_f64:
            continue
        probs = inputs.batch_instances(spec, dtype=dt)
        if code == S.F64:
            plan = autotune.tune_batch(probs, code, tiles=(512, 1024), threads=(128, 256), rules=((1024, 8),))
        else:
            plan = autotune.tune_batch(probs, code)
        b = S.Batch(autotune.apply_batch_plan(probs, plan), code, threads=plan["threads"])
        u0 = b.pack([q["u0"] for q in probs])
        u = u0.clone()
        res = {}
        for kind, fn in (("swept", b.run), ("classic", b.run_classic)):
            runs = 2 if (code == S.F32 and kind == "swept") else 1
            if runs > 1:
                fn(u)  # warm-up: captures the graphs
                barrier()
            ms = []
            for _ in range(runs):
                u.copy_(u0)
                ev = _event_time(torch, stream, lambda: fn(u))
                barrier()
                ms.append(ev[0].elapsed_time(ev[1]))
            res[kind] = min(ms)
        b.sync_status()
        f64 = code == S.F64
        rf = alu_roofline("ks", f64, units, res["swept"], "k_batch<%s>" % ("double" if f64 else "float"))
        rf["achieved"] = flops / (res["swept"] * 1e-3) / 1e12
        rf["frac"] = rf["achieved"] / rf["peak"]
        smem_acc = float((spec["n"] * spec["steps"] * np.where(heat, WORK["heat"]["smem_acc"],
                                                                2 * smem_ks[f64])).sum())
        sg = smem_acc * (8 if f64 else 4) / (res["swept"] * 1e-3) / 1e9
        rf["smem"].update({"achieved": sg, "frac": sg / SMEM_PEAK_GBS})
        rf["algorithmic_per_unit"] = {"flops": flops / units, "note": "heat and KS point-substeps of the batch"}
        out[name] = {"ms": res["swept"], "value": ws * work / (res["swept"] * 1e-3), "unit": UNIT,
                     "classic_ms": res["classic"], "classic_value": ws * work / (res["classic"] * 1e-3),
                     "speedup_vs_classic": res["classic"] / res["swept"], "tile_w": plan["tile_w"],
                     "tile_rule": plan.get("rule"), "threads": plan["threads"], "items": b.items,
                     "timed_runs": {"swept": 2 if code == S.F32 else 1, "classic": 1}, "roofline": rf}
        b.close()
        del u, u0
        torch.cuda.empty_cache()
    return out


# swept (tuned plan) vs classic across the paper's sizes:
# (label, scheme, dtype, n, steps, tuner probe steps, timed repeats)
SIZE_CASES = [
    ("heat N=2^10 FP64 periodic, 10,000 steps", "heat", "f64", 1 << 10, 10000, 2000, 3),
    ("heat N=2^10 FP32 periodic, 10,000 steps", "heat", "f32", 1 << 10, 10000, 2000, 3),
    ("KS N=2^14 FP64, 5,000 steps", "ks", "f64", 1 << 14, 5000, 1000, 3),
    ("KS N=2^14 FP32, 5,000 steps", "ks", "f32", 1 << 14, 5000, 1000, 3),
    ("KS N=2^16 FP64, 5,000 steps", "ks", "f64", 1 << 16, 5000, 1000, 3),
    ("KS N=2^16 FP32, 5,000 steps", "ks", "f32", 1 << 16, 5000, 1000, 3),
    ("KS N=2^18 FP64, 2,000 steps", "ks", "f64", 1 << 18, 2000, 1000, 3),
    ("KS N=2^18 FP32, 2,000 steps", "ks", "f32", 1 << 18, 2000, 1000, 3),
    # a 200-step probe picked tile 256 (0.91x); over 2,000 steps the queue's load balance decides,
    # and tile 128 with 256 threads is 4.5 % faster at 20,480 steps
    ("Euler Sod N=2^16 FP64 reflective, to t=0.2 (81,920 steps)", "euler", "f64", 1 << 16, 81920, 2000, 1),
    ("Euler Sod N=2^20 FP64 reflective, 100 steps", "euler", "f64", 1 << 20, 100, 100, 3),
]


def measure_sizes(S, autotune, torch, stream, barrier, ws, flush):
    """Each SIZE_CASES workload with its autotuned swept plan and with the
    classic path (CUDA events on the launching stream, L2 flushed before each
    timed solve, best of three)."""
    codes = {"heat": S.HEAT, "ks": S.KS, "euler": S.EULER}
    out = []
    for label, scheme, dt, n, nsteps, probe, reps in SIZE_CASES:
        sc, code = codes[scheme], (S.F64 if dt == "f64" else S.F32)
        u0, args, bc = autotune.problem(sc, code, n)
        plan = autotune.tune_single(sc, code, n, probe_steps=probe)
        sol = autotune.solver_from_plan(sc, code, n, *args, plan, bc=bc)
        d0 = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
        u = d0.clone()
        res = {}
        for name, fn in (("swept", sol.step), ("classic", sol.classic)):
            fn(u, nsteps)
            best = None
            for _ in range(reps):
                u.copy_(d0)
                flush.zero_()
                ev = _event_time(torch, stream, lambda: fn(u, nsteps))
                barrier()
                t = ev[0].elapsed_time(ev[1])
                best = t if best is None else min(best, t)
            res[name] = best
        sol.sync_status()
        kname, kunits, kms, share = dominant_swept_kernel(sol, u, d0, nsteps, res["swept"])
        sol.close()
        rf = alu_roofline(scheme, dt == "f64", kunits, kms, kname, registers=bool(plan.get("warp_tiles")))
        rf["kernel_share"] = share
        row = {"workload": label, "swept_ms": res["swept"], "classic_ms": res["classic"],
               "speedup_vs_classic": res["classic"] / res["swept"],
               "swept_value": ws * n * nsteps / (res["swept"] * 1e-3),
               "classic_value": ws * n * nsteps / (res["classic"] * 1e-3),
               "plan": {k: plan.get(k, 0) for k in ("tile_w", "threads", "warp_tiles", "persistent", "cluster")},
               "roofline": rf}
        if scheme == "heat" and n == 1024:
            # the heat configuration names its plan: tiles of 64 points with 64 threads (tpb = 64)
            cs = S.Solver(sc, code, n, *args, bc=bc, tile_w=64, threads=64)
            cs.step(u, nsteps)
            best = None
            for _ in range(reps):
                u.copy_(d0)
                flush.zero_()
                ev = _event_time(torch, stream, lambda: cs.step(u, nsteps))
                barrier()
                t = ev[0].elapsed_time(ev[1])
                best = t if best is None else min(best, t)
            cs.sync_status()
            cs.close()
            row["tpb64"] = {"tile_w": 64, "threads": 64, "swept_ms": best,
                            "speedup_vs_classic": res["classic"] / best}
        out.append(row)
    return out


# the 2D swept decomposition (the paper's future work): 2D FTCS heat, periodic
HEAT2D_CASES = [
    ("heat2d 1024x1024 FP64, 1,000 steps", "f64", 1024, 1000),
    ("heat2d 1024x1024 FP32, 1,000 steps", "f32", 1024, 1000),
    ("heat2d 4096x4096 FP32, 100 steps", "f32", 4096, 100),
]


def measure_heat2d(S, autotune, torch, stream, barrier, ws, flush):
    """Each HEAT2D_CASES workload with its autotuned 2D swept plan and with the
    classic 2D path (CUDA events on the launching stream, L2 flushed before each
    timed solve, best of three)."""
    from paper_1612_02495_gb300 import inputs

    out = []
    for label, dt, n, nsteps in HEAT2D_CASES:
        code = S.F64 if dt == "f64" else S.F32
        plan = autotune.tune_2d(code, n, n, probe_steps=min(nsteps, 200))
        p = inputs.heat2d_problem(nx=n, ny=n, dtype=np.float64 if dt == "f64" else np.float32)
        sol = S.Solver2D(code, n, n, p["dx"], p["dt"], p["alpha"], tile_w=plan["tile_w"], threads=plan["threads"],
                         persistent=plan.get("persistent", 0))
        d0 = torch.from_numpy(p["u0"]).cuda()
        u = d0.clone()
        res = {}
        for name, fn in (("swept", sol.step), ("classic", sol.classic)):
            fn(u, nsteps)
            best = None
            for _ in range(3):
                u.copy_(d0)
                flush.zero_()
                ev = _event_time(torch, stream, lambda: fn(u, nsteps))
                barrier()
                t = ev[0].elapsed_time(ev[1])
                best = t if best is None else min(best, t)
            res[name] = best
        sol.sync_status()
        sol.close()
        pers = plan.get("persistent", 0)
        kname = ("k_persist2d<%s>" if pers else "k_pyr2d + k_bridge2d + k_octa2d <%s> (the solve's graph)") % (
            "double" if dt == "f64" else "float")
        rf = alu_roofline("heat2d", dt == "f64", n * n * nsteps, res["swept"], kname,
                          note=None if pers else "per-pass plan: the solve's time, launch gaps included")
        out.append({"workload": label, "swept_ms": res["swept"], "classic_ms": res["classic"],
                    "speedup_vs_classic": res["classic"] / res["swept"],
                    "swept_value": ws * n * n * nsteps / (res["swept"] * 1e-3), "unit": UNIT,
                    "plan": {"tile_w": plan["tile_w"], "threads": plan["threads"],
                             "persistent": plan.get("persistent", 0)}, "roofline": rf})
    return out


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    import oracle

    threads = os.cpu_count() or 1
    oracle.build.build()
    import oracle as orc
    from paper_1612_02495_gb300 import inputs

    # one bench step = the oracle on the full N=2^20 grid for a fixed window of
    # timesteps, sized once (from a 2-step probe) to about 8 s on these cores
    _, window, _ = cpu_oracle_rate(N, 8.0, threads, probe_only=True)
    p = inputs.ks_problem(n=N)
    times = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        orc.ks(p["u0"], p["dx"], p["dt"], p["nu"], window, threads=threads)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            times.append(dt)
    ms = float(np.mean(times)) * 1e3
    v = N * window / (ms * 1e-3)
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N, "nsteps": NSTEPS, "oracle_window_steps": window},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": "oracle (plain C, OpenMP over %d threads) on the full N=2^20 grid for a %d-step "
                                      "window per bench step (ms_per_step is that window's time)" % (threads, window)},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-classic", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-sizes", action="store_true")
    ap.add_argument("--no-2d", action="store_true")
    ap.add_argument("--no-slab", action="store_true", help="skip the split-grid line")
    ap.add_argument("--no-batch-f64", action="store_true", help="skip the FP64 batch (about 2 x 50 s)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    import __graft_entry__

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        dist.init_process_group("nccl")
    __graft_entry__.build() if rank == 0 else None
    if ws > 1:
        dist.barrier()
    from paper_1612_02495_gb300 import inputs
    from paper_1612_02495_gb300 import swept as S

    from paper_1612_02495_gb300 import autotune

    p = inputs.ks_problem(n=N, seed=1 + rank)
    tuned = autotune.tune_single(S.KS, S.F64, N, probe_steps=4000)
    sol = autotune.solver_from_plan(S.KS, S.F64, N, p["dx"], p["dt"], p["nu"], tuned)
    plan = sol.plan
    stream = torch.cuda.current_stream()
    u0 = torch.from_numpy(p["u0"]).cuda()
    u = u0.clone()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    launches_per_step = (2 * NSTEPS) // plan["half_cycle"] + 1 + (2 if (2 * NSTEPS) % plan["half_cycle"] else 0)

    def barrier():
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def timed(fn, k, w):
        for _ in range(w):
            u.copy_(u0)
            fn(u)
        barrier()
        total = 0.0
        evs = []
        for _ in range(k):
            u.copy_(u0)
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn(u)
            b.record(stream)
            evs.append((a, b))
        barrier()
        for a, b in evs:
            total += a.elapsed_time(b)
        return max_over_ranks(total / k, dist, ws)

    clocks = Clocks(local)
    clocks.start()
    ms = timed(lambda x: sol.step(x, NSTEPS), args.steps, args.warmup)
    clk = clocks.stop()
    sol.sync_status()
    value = whole_job_rate(N * NSTEPS, ms, ws)

    ms_classic = None
    if not args.no_classic:
        ms_classic = timed(lambda x: sol.classic(x, NSTEPS), max(1, args.steps // 2), 1)

    # end to end through the C ABI with host buffers (pinned): H2D + solve + D2H per step
    h_in = torch.from_numpy(p["u0"]).pin_memory()
    h_out = torch.empty_like(h_in).pin_memory()
    sol.run_host(h_in, h_out, u, NSTEPS)
    barrier()
    e2e_ms = []
    for _ in range(max(1, args.steps // 2)):
        t0 = time.perf_counter()
        sol.run_host(h_in, h_out, u, NSTEPS)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e = max_over_ranks(float(np.mean(e2e_ms)), dist, ws)

    peak_src = ("derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz (measured DFMA issue rate "
                "0.60e12/s = 1.20 TFLOP/s)")
    if plan.get("persistent"):
        # dominant kernel: the persistent swept kernel, one launch per solve; its
        # duration is the solve's event time (the launch also carries two 4-byte
        # memsets and a one-thread status kernel)
        units = N * 2 * NSTEPS
        roofline = {"bound": "alu", "achieved": FP64_FLOPS_PER_SUBSTEP * units / (ms * 1e-3) / 1e12,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "traffic": None if plan.get("warp_tiles") else PERSIST_TRAFFIC.get((plan["tile_w"], plan["threads"])),
                    "kernel": "k_swept_persist<double, KsOp<double>%s>" % (
                        ", %d" % (plan["tile_w"] // 32) if plan.get("warp_tiles") else ""), "peak_source": peak_src,
                    "pipe_frac": FP64_INSTR_PER_SUBSTEP * units / (ms * 1e-3) / FP64_INSTR_PEAK,
                    "frac_of_measured_mix_ceiling": FP64_INSTR_PER_SUBSTEP * units / (ms * 1e-3) / FP64_KS_MIX_CEILING,
                    "kernel_ms_avg": ms, "kernel_share": 1.0}
        if roofline["traffic"] is not None:
            roofline["traffic_note"] = "ncu capture of this plan's persistent launch (tile %d, %d threads), " \
                                       "50,000 steps" % (plan["tile_w"], plan["threads"])
        roofline["frac"] = roofline["achieved"] / FP64_PEAK_TFLOPS
        launches_per_step = 2
    else:
        # dominant kernel: the diamond pass, timed with CUDA events on the launching stream
        u.copy_(u0)
        prof = sol.profile_passes(u, NSTEPS)
        d_ms, d_n = prof["diamond"]
        d_avg = d_ms / max(d_n, 1)
        flops_per_diamond = FP64_FLOPS_PER_SUBSTEP * N * plan["half_cycle"]
        achieved = flops_per_diamond / (d_avg * 1e-3) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP64_PEAK_TFLOPS, "traffic": DIAMOND_TRAFFIC_BYTES,
                    "kernel": "k_swept_diamond<double, KsOp<double>%s>" % (
                        ", %d" % (plan["tile_w"] // 32) if plan.get("warp_tiles") else ""), "peak_source": peak_src,
                    "pipe_frac": (FP64_INSTR_PER_SUBSTEP * N * plan["half_cycle"] / (d_avg * 1e-3)) / FP64_INSTR_PEAK,
                    "frac_of_measured_mix_ceiling": (FP64_INSTR_PER_SUBSTEP * N * plan["half_cycle"] / (d_avg * 1e-3))
                    / FP64_KS_MIX_CEILING,
                    "diamond_ms_avg": d_avg, "diamond_share": d_ms / max(sum(v[0] for v in prof.values()), 1e-9)}
        if plan["tile_w"] != 1024:
            roofline["traffic"] = None  # the ncu figure is for tile 1024

    adjoint = None
    if not args.no_adjoint:
        adjoint = measure_adjoint(S, inputs, torch, stream, max(2, args.steps), barrier)
    fp32 = None
    if not args.no_fp32:
        fp32 = measure_fp32(S, inputs, autotune, torch, stream, barrier, ws)
    sizes = None
    if not args.no_sizes:
        sizes = measure_sizes(S, autotune, torch, stream, barrier, ws, flush)
    heat2d = None
    if not args.no_2d:
        heat2d = measure_heat2d(S, autotune, torch, stream, barrier, ws, flush)
    slab = None
    if not args.no_slab:
        slab = measure_slab(S, inputs, torch, stream, barrier)
    batched = None
    if not args.no_batch:
        batched = measure_batch(S, inputs, autotune, torch, stream, barrier, ws, not args.no_batch_f64)

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": N, "nsteps": NSTEPS, "tile_w": plan["tile_w"],
                      "threads": plan["threads"], "half_cycle": plan["half_cycle"],
                      "l2": "flushed (256 MB write) before every timed step", "parallelism": "replicas"},
           "gpu_launches": launches_per_step * args.steps,
           "e2e": {"value": ws * N * NSTEPS / (e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": N * 8,
                   "d2h_bytes_per_step": N * 8},
           "roofline": roofline, "clocks": clk}
    if adjoint:
        out["adjoint"] = adjoint
    if fp32:
        out["fp32"] = fp32
    if batched:
        out["batched"] = batched
    if sizes:
        out["sizes"] = sizes
    if heat2d:
        out["heat2d"] = heat2d
    if slab:
        out["slab"] = slab
    out["config"]["autotuned"] = {k: tuned.get(k, 0) for k in ("tile_w", "threads", "warp_tiles", "persistent",
                                                                "cluster")}
    if ms_classic:
        # classic moves the state through HBM/L2 every sub-timestep: stage 0 reads u and writes P,
        # stage 1 reads P and u and writes u: 5 values = 40 B per cell-update in FP64
        gbs = CLASSIC_BYTES_PER_UPDATE * N * NSTEPS / (ms_classic * 1e-3) / 1e9
        hbm = peaks().get("hbm_gbs")
        out["classic"] = {"value": ws * N * NSTEPS / (ms_classic * 1e-3), "ms_per_step": ms_classic,
                          "roofline": {"bound": "hbm", "achieved": gbs, "peak": hbm, "unit": "GB/s",
                                       "frac": (gbs / hbm) if hbm else None,
                                       "algorithmic_bytes_per_cell_update": CLASSIC_BYTES_PER_UPDATE,
                                       "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                                       "note": "FP64 classic is bound by the FP64 pipe, not HBM"}}
        out["speedup_vs_classic"] = ms_classic / ms
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r, st, secs = cpu_oracle_rate(N, 10.0, threads)
        r1, st1, secs1 = cpu_oracle_rate(N, 4.0, 1)
        out["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "oracle on the full N=2^20 grid for %d steps (%.1f s, OpenMP %d threads)"
                                         % (st, secs, threads),
                               "one_thread": {"value": r1, "unit": UNIT, "cores": 1,
                                              "sample": "same grid, %d steps (%.1f s, 1 thread)" % (st1, secs1)}}
    if rank == 0:
        print(json.dumps(out))
    sol.close()
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
