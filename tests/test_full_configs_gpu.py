"""GPU parity at the stated configurations: every workload compared with the
oracle at its own size and step count, in the launch configuration bench.py
times (the autotuner's plan from the same call).

  - KS N=2^20, 50,000 steps, FP32 and FP64: the whole final field equals the
    oracle bit for bit (OpenMP over the host cores), swept == classic, and
    the mean is conserved;
  - Euler Sod N=2^16 to t = 0.2 (81,920 steps): swept == classic == oracle
    bit for bit; N=2^22 over a 100-step window the same;
  - the adjoint workload, KS N=2^18 FP64, 5,000 steps, L = sum (u(T) -
    u_target)^2 with u_target the run from a seeded perturbation: dL/du0
    equals the oracle's reverse mode (same segment length) bit for bit, dL/dnu
    is within the derived bound, and 8 seeded directions plus dL/dnu agree
    with central differences of GPU forward solves;
  - the batched workload (4096 problems) in FP64 and FP32, sampled.

These take minutes of host time (the oracle is plain C); they are marked slow.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_1612_02495_gb300 import inputs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

HOST_THREADS = max(1, os.cpu_count() or 1)
EPS = 2.0 ** -52


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


def solve_both(S, sol, u0, nsteps):
    import torch

    u = torch.from_numpy(np.ascontiguousarray(u0)).cuda()
    v = u.clone()
    sol.step(u, nsteps)
    sol.classic(v, nsteps)
    torch.cuda.synchronize()
    sol.sync_status()
    return u.cpu().numpy(), v.cpu().numpy()


# --------------------------------------------------------------------------- KS 2^20 x 50,000
@pytest.mark.parametrize("dtype,probe", [(np.float64, 4000), (np.float32, 8000)])
def test_ks_2_20_full_run_whole_field(S, dtype, probe):
    """KS N=2^20, 50,000 steps in the plan bench.py times for this precision
    (tune_single with the same probe length): whole field == oracle bitwise."""
    from paper_1612_02495_gb300 import autotune

    n, nsteps = 1 << 20, 50000
    code = S.F64 if dtype == np.float64 else S.F32
    plan = autotune.tune_single(S.KS, code, n, probe_steps=probe)
    p = inputs.ks_problem(n=n, dtype=dtype)
    sol = autotune.solver_from_plan(S.KS, code, n, p["dx"], p["dt"], p["nu"], plan)
    sw, cl = solve_both(S, sol, p["u0"], nsteps)
    sol.close()
    assert sw.dtype == dtype
    assert np.array_equal(sw, cl), ("swept != classic", plan)
    # mean conservation (the advective and diffusive terms telescope under
    # periodic BCs); FP32 rounding of the per-step updates random-walks the sum
    bound = 1e-11 if dtype == np.float64 else 1e-5
    s0 = float(np.sum(p["u0"].astype(np.float64)))
    assert abs(float(np.sum(sw.astype(np.float64))) - s0) <= bound * float(np.sum(np.abs(p["u0"])))
    ref = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], nsteps, threads=HOST_THREADS)
    assert np.array_equal(sw, ref), ("swept != oracle bitwise", relerr(sw, ref), plan)


# --------------------------------------------------------------------------- Euler Sod
def _euler_case(S, n, nsteps, probe):
    from paper_1612_02495_gb300 import autotune

    pr = inputs.euler_problem(n=n)
    plan = autotune.tune_single(S.EULER, S.F64, n, probe_steps=probe)
    sol = autotune.solver_from_plan(S.EULER, S.F64, n, pr["dx"], pr["dt"], pr["gamma"], plan, bc=S.BC_REFLECTIVE)
    sw, cl = solve_both(S, sol, pr["U0"], nsteps)
    sol.close()
    assert np.array_equal(sw, cl), ("swept != classic", plan)
    ref = oracle.euler(pr["U0"], pr["dx"], pr["dt"], pr["gamma"], nsteps, bc=oracle.BC_MIRROR, threads=HOST_THREADS)
    assert np.array_equal(sw, ref), ("swept != oracle bitwise", relerr(sw, ref), plan)
    return pr, sw


def test_euler_sod_2_16_to_t_0_2(S):
    """Euler Sod N=2^16 to t = 0.2 (81,920 SSP-RK2 steps), bench plan (2,000-step
    tuner probes): swept == classic == oracle bit for bit; mass and energy are
    conserved by the reflective walls."""
    pr, sw = _euler_case(S, 1 << 16, 81920, 2000)
    assert pr["nsteps"] == 81920
    for c in (0, 2):
        s0 = math.fsum(pr["U0"][c].astype(np.float64))
        assert abs(math.fsum(sw[c]) - s0) <= 1e-10 * abs(s0), c


def test_euler_sod_2_22_window(S):
    """Euler Sod N=2^22, a 100-step window (the full run to t = 0.2 is 5.2e6
    steps), tuned plan: swept == classic == oracle bit for bit."""
    _euler_case(S, 1 << 22, 100, 100)


# --------------------------------------------------------------------------- adjoint 2^18 x 5,000
ADJ_N, ADJ_STEPS = 1 << 18, 5000


def _adjoint_setup(S):
    """Inputs of the adjoint workload from the oracle alone: u0, u_target =
    forward(u0 + 1e-3 eta) and dL/du(T) = 2 (u(T) - u_target)."""
    p = inputs.ks_problem(n=ADJ_N, seed=71)
    pert = 1e-3 * inputs.rng(72).standard_normal(ADJ_N)
    target = oracle.ks(p["u0"] + pert, p["dx"], p["dt"], 1.0, ADJ_STEPS, threads=HOST_THREADS)
    uT = oracle.ks(p["u0"], p["dx"], p["dt"], 1.0, ADJ_STEPS, threads=HOST_THREADS)
    return p, target, 2.0 * (uT - target)


def test_adjoint_configured_size_matches_oracle_reverse_mode(S):
    """GPU swept_adjoint (default checkpoint memory) against the oracle's reverse
    mode with the same segment length: dL/du0 bitwise, dL/dnu within
    1e-12 |ref| + 8 eps * condition (the bound of the smaller adjoint tests)."""
    import torch

    p, target, gT = _adjoint_setup(S)
    sol = S.Solver(S.KS, S.F64, ADJ_N, p["dx"], p["dt"], 1.0)
    ck = torch.empty(sol.ckpt_size(ADJ_STEPS), dtype=torch.uint8, device="cuda")
    g, gnu = sol.adjoint(torch.from_numpy(gT).cuda(), ADJ_STEPS, ck, u0=torch.from_numpy(p["u0"]).cuda())
    torch.cuda.synchronize()
    sol.sync_status()
    # the library's default segment: the whole number of passes (h/S steps each)
    # with the fewest stored states, ceil(nsteps / K) checkpoints + an S K + 1 tier tape
    k0 = sol.plan["half_cycle"] // sol.plan["stages"]
    S_ = sol.plan["stages"]
    seg = min(range(k0, ADJ_STEPS + 1, k0), key=lambda K: (-(-ADJ_STEPS // K) + S_ * K + 1, K))
    sol.close()
    ref, ref_nu, cond = oracle.ks_adjoint(p["u0"], p["dx"], p["dt"], 1.0, ADJ_STEPS, gT, seg=seg,
                                          with_condition=True, threads=HOST_THREADS)
    got = g.cpu().numpy()
    assert np.array_equal(got, ref), relerr(got, ref)
    gnu = float(gnu.cpu().numpy()[0])
    assert abs(gnu - ref_nu) <= 1e-12 * abs(ref_nu) + 8 * EPS * cond, (gnu, ref_nu, cond)


def test_adjoint_configured_size_central_differences(S):
    """8 seeded directions of dL/du0 and dL/dnu against central differences
    (h = 1e-6) of GPU forward solves, relative agreement 1e-6.  The loss is
    summed exactly (math.fsum) so that its own rounding stays below the
    difference quotient's."""
    import torch

    p, target, gT = _adjoint_setup(S)
    u0 = torch.from_numpy(p["u0"]).cuda()
    sol = S.Solver(S.KS, S.F64, ADJ_N, p["dx"], p["dt"], 1.0)
    ck = torch.empty(sol.ckpt_size(ADJ_STEPS), dtype=torch.uint8, device="cuda")
    g, gnu = sol.adjoint(torch.from_numpy(gT).cuda(), ADJ_STEPS, ck, u0=u0)
    torch.cuda.synchronize()
    sol.close()
    g = g.cpu().numpy()
    gnu = float(gnu.cpu().numpy()[0])
    sols = {}

    def loss(u_init, nu):
        if nu not in sols:
            sols[nu] = S.Solver(S.KS, S.F64, ADJ_N, p["dx"], p["dt"], nu)
        u = u_init.clone()
        sols[nu].step(u, ADJ_STEPS)
        d = u.cpu().numpy() - target
        return math.fsum(d * d)

    h = 1e-6
    pairs = []
    for s in range(8):
        v = inputs.rng(80 + s).standard_normal(ADJ_N)
        vd = torch.from_numpy(v).cuda()
        fd = (loss(u0 + h * vd, 1.0) - loss(u0 - h * vd, 1.0)) / (2 * h)
        pairs.append((fd, math.fsum(g * v)))
    worst = max(abs(fd - ad) / abs(ad) for fd, ad in pairs)
    fdnu = (loss(u0, 1.0 + h) - loss(u0, 1.0 - h)) / (2 * h)
    for x in sols.values():
        x.close()
    print("adjoint vs central differences: worst direction %.3g, nu %.3g (relative)"
          % (worst, abs(fdnu - gnu) / abs(gnu)))
    for fd, ad in pairs:
        assert abs(fd - ad) <= 1e-6 * abs(ad), (fd, ad, pairs)
    assert abs(fdnu - gnu) <= 1e-6 * abs(gnu), (fdnu, gnu, worst)


# --------------------------------------------------------------------------- batched FP64
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_full_batch_workload_bench_plan(S, dtype):
    """The batched workload (4096 problems) with the tuned batch plan bench.py
    uses: sampled problems equal their standalone swept solves bit for bit, and
    the four smallest plus two sampled ones equal the oracle."""
    import torch

    from paper_1612_02495_gb300 import autotune

    code = S.F64 if dtype == np.float64 else S.F32
    probs = inputs.batch_instances(inputs.batch_problems(), dtype=dtype)
    if code == S.F64:
        plan = autotune.tune_batch(probs, code, tiles=(512, 1024), threads=(128, 256), rules=((1024, 8),))
    else:
        plan = autotune.tune_batch(probs, code)
    tuned = autotune.apply_batch_plan(probs, plan)
    b = S.Batch(tuned, code, threads=plan["threads"])
    u = b.pack([q["u0"] for q in probs])
    b.run(u)
    torch.cuda.synchronize()
    b.sync_status()
    got = b.unpack(u)
    b.close()
    del u
    torch.cuda.empty_cache()
    rng = inputs.rng(506)
    sample = [int(i) for i in rng.choice(len(probs), size=12, replace=False)]
    for i in sample:
        q = tuned[i]
        sol = S.Solver(q["scheme"], code, q["n"], q["dx"], q["dt"], q["param"], tile_w=q["tile_w"])
        x = torch.from_numpy(q["u0"]).cuda()
        sol.step(x, q["nsteps"])
        torch.cuda.synchronize()
        sol.close()
        assert np.array_equal(got[i], x.cpu().numpy()), i
    small = sorted(range(len(probs)), key=lambda i: probs[i]["n"] * probs[i]["nsteps"])[:4]
    cheap = sorted(sample, key=lambda i: probs[i]["n"] * probs[i]["nsteps"])[:2]
    for i in small + cheap:
        q = probs[i]
        if q["scheme"] == 0:
            ref = oracle.heat(q["u0"], q["dx"], q["dt"], q["param"], q["nsteps"], threads=HOST_THREADS)
        else:
            ref = oracle.ks(q["u0"], q["dx"], q["dt"], q["param"], q["nsteps"], threads=HOST_THREADS)
        assert np.array_equal(got[i], ref), i
