"""Largest sizes: a 1D grid of more than 2^31 points, so that every global,
edge and tile index needs 64 bits.

Heat FP32, N = 2^31 + 2^20 (8.6 GB of state, 34 GB of edge buffers), tile
1024, 600 steps (one full pass pair and a 88-step remainder), per-pass and
persistent.  The case runs first under the debug build, whose index checks
skip any out-of-range access, and must come out clean; only then does it run
on the release build.  Checks: swept == classic on the device, bit for bit,
and 8 sampled points equal the oracle advanced on a window around each point
that covers its domain of dependence (one point per step and side).  The input
is built on the device (a sum of sine modes, seeded amplitudes); the oracle's
windows are copied from it.
"""
import os
import subprocess
import sys

import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N = (1 << 31) + (1 << 20)
W = 1024
NSTEPS = 600

CASE = r'''
import sys, numpy as np, torch
from paper_1612_02495_gb300 import swept as S
N, W, NSTEPS, persistent = %d, %d, %d, %d
amp = np.random.default_rng(20161208).uniform(-1, 1, 4)
x = torch.arange(N, dtype=torch.float64, device="cuda") * (2 * np.pi / N)
u0 = sum(float(a) * torch.sin((k + 1) * x) for k, a in enumerate(amp)).to(torch.float32)
del x
dx = 2 * np.pi / N
dt = 0.25 * dx * dx
sol = S.Solver(S.HEAT, S.F32, N, dx, dt, 1.0, tile_w=W, persistent=persistent)
u = u0.clone()
sol.step(u, NSTEPS)
torch.cuda.synchronize()
sol.sync_status()
if S.DEBUG_BUILD:
    en, rec = S.debug_status()
    assert en and rec is None, rec
    print("debug clean")
    sys.exit(0)
v = u0.clone()
sol.classic(v, NSTEPS)
torch.cuda.synchronize()
assert torch.equal(u, v), "swept != classic"
reach = NSTEPS + 4
picks = [0, N - 1, (1 << 31) - 1, 1 << 31, 12345678901 %% N, N // 3, 2 * N // 3 + 7, N - W // 2]
np.save(sys.argv[1], np.array(picks, dtype=np.int64))
wins, outs = [], []
for c in picks:
    idx = torch.arange(c - reach, c + reach + 1, device="cuda") %% N
    wins.append(u0[idx].cpu().numpy())
    outs.append(float(u[c].item()))
np.save(sys.argv[2], np.stack(wins))
np.save(sys.argv[3], np.array(outs, dtype=np.float32))
print("release done")
'''


def _run(persistent, debug, tmp_path):
    env = dict(os.environ, PYTHONPATH=ROOT + os.pathsep + os.environ.get("PYTHONPATH", ""))
    env["SWEPT_DEBUG"] = "1" if debug else "0"
    files = [str(tmp_path / ("%s_%d.npy" % (n, persistent))) for n in ("picks", "wins", "outs")]
    r = subprocess.run([sys.executable, "-c", CASE % (N, W, NSTEPS, persistent)] + files, cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-3000:]
    return files


@pytest.mark.parametrize("persistent", [0, 1])
def test_heat_grid_beyond_2_31_points(persistent, tmp_path):
    from paper_1612_02495_gb300 import build as libbuild

    libbuild.build()
    libbuild.build(debug=True)
    _run(persistent, True, tmp_path)  # index checks first: nothing out of range can be touched
    picks_f, wins_f, outs_f = _run(persistent, False, tmp_path)
    wins, outs = np.load(wins_f), np.load(outs_f)
    dx = 2 * np.pi / N
    dt = 0.25 * dx * dx
    reach = NSTEPS + 4
    for w, got in zip(wins, outs):
        # the window is periodic in the oracle; its wrapped ends lie outside the centre's domain of dependence
        ref = oracle.heat(w, dx, dt, 1.0, NSTEPS)
        assert ref[reach] == got, (ref[reach], got)
