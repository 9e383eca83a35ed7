"""Batched persistent solver (swept_batch_*) on the GPU.

Each problem of a batch must equal the standalone swept_step_n of the same
problem bit for bit (the batch runs the same passes), and the CPU oracle.
Covers mixed heat / KS problems of different sizes and step counts, tile
widths, FP32 and FP64, the full 4096-problem workload (sampled), and the
bounded waits: a queue whose first items are skipped must end with
SWEPT_ETIMEOUT and leave the GPU usable.
"""
import numpy as np
import pytest

import oracle
from paper_1612_02495_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1612_02495_gb300 import build as libbuild

    libbuild.build()
    from paper_1612_02495_gb300 import swept

    return swept


def oracle_run(q):
    if q["scheme"] == 0:
        return oracle.heat(q["u0"], q["dx"], q["dt"], q["param"], q["nsteps"])
    return oracle.ks(q["u0"], q["dx"], q["dt"], q["param"], q["nsteps"], threads=8)


def standalone(S, q, dtype):
    import torch

    sol = S.Solver(q["scheme"], dtype, q["n"], q["dx"], q["dt"], q["param"], tile_w=q.get("tile_w", 0) or 0)
    u = torch.from_numpy(q["u0"]).cuda()
    sol.step(u, q["nsteps"])
    torch.cuda.synchronize()
    sol.close()
    return u.cpu().numpy()


def small_spec(count, seed, steps_hi=400):
    return inputs.batch_problems(count=count, seed=seed, log2_lo=10, log2_hi=14, steps_lo=1, steps_hi=steps_hi)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_small_batch_matches_oracle_and_standalone(S, dtype):
    import torch

    probs = inputs.batch_instances(small_spec(40, 101), dtype=dtype)
    probs[0]["nsteps"] = 0  # a no-op problem
    code = S.F64 if dtype == np.float64 else S.F32
    b = S.Batch(probs, code)
    u = b.pack([q["u0"] for q in probs])
    b.run(u)
    torch.cuda.synchronize()
    b.sync_status()
    got = b.unpack(u)
    for q, x in zip(probs, got):
        assert np.array_equal(x, oracle_run(q)), (q["scheme"], q["n"], q["nsteps"])
    # rerunning from the state continues the solve (graph replay)
    b.run(u)
    torch.cuda.synchronize()
    again = b.unpack(u)
    for q, x, y in zip(probs[:6], got, again):
        q2 = dict(q, u0=x)
        assert np.array_equal(y, oracle_run(q2))
    b.close()


@pytest.mark.parametrize("tile_w,threads", [(64, 64), (128, 128), (256, 256), (512, 128)])
def test_batch_tile_widths(S, tile_w, threads):
    import torch

    probs = inputs.batch_instances(small_spec(24, 202, steps_hi=700), dtype=np.float64)
    for q in probs:
        q["tile_w"] = tile_w
    b = S.Batch(probs, S.F64, threads=threads)
    u = b.pack([q["u0"] for q in probs])
    b.run(u)
    torch.cuda.synchronize()
    b.sync_status()
    for q, x in zip(probs, b.unpack(u)):
        assert np.array_equal(x, standalone(S, q, S.F64))
    b.close()


def test_batch_rejects_bad_problems(S):
    q = dict(scheme=1, n=1000, nsteps=10, dx=0.785, dt=0.005, param=1.0, tile_w=64)  # 1000 % 64 != 0
    with pytest.raises(S.SweptError):
        S.Batch([q], S.F64)
    q = dict(scheme=2, n=1024, nsteps=10, dx=0.785, dt=0.005, param=1.0)  # Euler is not batched
    with pytest.raises(S.SweptError):
        S.Batch([q], S.F64)


def test_batch_bounded_wait_times_out_and_recovers(S):
    """Skip the first pass layer: every block then waits for tiles that never
    finish; the waits give up (SWEPT_ETIMEOUT) and a normal run afterwards is
    correct."""
    import torch

    probs = inputs.batch_instances(small_spec(6, 303, steps_hi=300), dtype=np.float64)
    for q in probs:
        q["nsteps"] = max(q["nsteps"], 200)
    b = S.Batch(probs, S.F64)
    layer0 = sum(q["n"] // 512 for q in probs)  # default tile 512: pass 0 has n/512 items per problem
    b.set_option(S.SWEPT_BATCH_SPIN_LIMIT, 2000)
    b.set_option(S.SWEPT_BATCH_START_ITEM, layer0)
    u = b.pack([q["u0"] for q in probs])
    b.run(u)
    torch.cuda.synchronize()
    with pytest.raises(S.SweptError) as e:
        b.sync_status()
    assert e.value.status == S.SWEPT_ETIMEOUT
    b.set_option(S.SWEPT_BATCH_START_ITEM, 0)
    b.set_option(S.SWEPT_BATCH_SPIN_LIMIT, 1 << 24)
    u = b.pack([q["u0"] for q in probs])
    b.run(u)
    torch.cuda.synchronize()
    b.sync_status()
    for q, x in zip(probs, b.unpack(u)):
        assert np.array_equal(x, oracle_run(q))
    b.close()


@pytest.mark.parametrize("dtype", [np.float32])
def test_full_batch_workload_sampled(S, dtype):
    """The batched workload: 4096 problems, N = 2^U(10,18) (multiples of 1024), heat/KS
    50/50, 1,000-20,000 steps, one persistent launch.  Sampled problems equal their
    standalone swept solves bit for bit; the smallest ones equal the oracle."""
    import torch

    code = S.F64 if dtype == np.float64 else S.F32
    probs = inputs.batch_instances(inputs.batch_problems(), dtype=dtype)
    b = S.Batch(probs, code)
    u = b.pack([q["u0"] for q in probs])
    b.run(u)
    torch.cuda.synchronize()
    b.sync_status()
    got = b.unpack(u)
    rng = inputs.rng(505)
    for i in rng.choice(len(probs), size=12, replace=False):
        assert np.array_equal(got[i], standalone(S, probs[i], code)), i
    small = sorted(range(len(probs)), key=lambda i: probs[i]["n"] * probs[i]["nsteps"])[:4]
    for i in small:
        assert np.array_equal(got[i], oracle_run(probs[i])), i
    b.close()


def test_batch_classic_baseline_equals_swept_and_oracle(S):
    """swept_batch_run_classic (one launch per global sub-timestep over every
    problem still running) equals swept_batch_run and the oracle bit for bit,
    in both precisions, with odd and even heat step counts."""
    import torch

    for dtype, code in ((np.float64, S.F64), (np.float32, S.F32)):
        probs = inputs.batch_instances(small_spec(10, 404, steps_hi=500), dtype=dtype)
        probs[0]["nsteps"] = 0
        b = S.Batch(probs, code)
        u0 = b.pack([q["u0"] for q in probs])
        u, v = u0.clone(), u0.clone()
        b.run(u)
        b.run_classic(v)
        b.run_classic(v)  # graph replay: a second advance from the result
        u2 = u.clone()
        b.run(u2)
        torch.cuda.synchronize()
        b.sync_status()
        assert torch.equal(v, u2)
        w = u0.clone()
        b.run_classic(w)
        torch.cuda.synchronize()
        assert torch.equal(w, u)
        for q, x in zip(probs, b.unpack(w)):
            assert np.array_equal(x, oracle_run(q)), (q["scheme"], q["n"], q["nsteps"])
        b.close()
