"""Seeded synthetic inputs shared by the tests, the bench and the smoke check.

This module only draws initial conditions and problem sizes; it contains none of
the schemes' arithmetic, so the GPU path and the CPU oracle stay independent.
All randomness comes from numpy's Philox generator seeded from SEED_BASE plus a
per-use offset, generated in FP64 on the host and cast at the end.

Workloads (shapes follow the paper's test problems, Section "Test cases"):
  heat   u_t = alpha u_xx on [0, 2 pi), periodic, IC = sum of 8 sine modes
         k = 1..8 with U(-1, 1) amplitudes, r = alpha dt / dx^2 = 0.25.
  ks     u_t = -u u_x - u_xx - nu u_xxxx, periodic on L = 32 pi N / 128
         (the stable reading of the length, dx = pi / 4), dt = 0.005,
         IC = cos(x/16)(1 + sin(x/16)) + 1e-3 U(-1, 1).
  euler  Sod tube on [0, 1]: (rho, u, p) = (1, 0, 1) for x < 0.5 and
         (0.125, 0, 0.1) after, rho and p each times (1 + 0.01 U(-1, 1)),
         gamma = 1.4, fixed dt = 0.4 dx / 2.5 rounded so that t = 0.2 is hit.
  batch  problems with N = 2^U(10, 18) rounded to a multiple of 1024 (so every
         tile width up to 512 divides every problem), heat / KS 50/50,
         steps ~ U{1000..20000}; per-problem ICs as above, seeded per problem.
"""
import math

import numpy as np

SEED_BASE = 20161208


def rng(offset=0):
    """Philox generator for SEED_BASE + offset."""
    return np.random.Generator(np.random.Philox(SEED_BASE + int(offset)))


def heat_problem(n=1024, r=0.25, alpha=1.0, modes=8, seed=0, dtype=np.float64):
    """Periodic heat problem; returns dict with u0, dx, dt, alpha, amps, x."""
    dx = 2.0 * math.pi / n
    dt = r * (dx * dx) / alpha
    amps = rng(seed).uniform(-1.0, 1.0, size=modes)
    x = np.arange(n, dtype=np.float64) * dx
    u0 = np.zeros(n, dtype=np.float64)
    for k in range(1, modes + 1):
        u0 += amps[k - 1] * np.sin(k * x)
    return dict(u0=u0.astype(dtype), dx=dx, dt=dt, alpha=alpha, amps=amps, x=x, r=r)


def heat2d_problem(nx=1024, ny=None, r=0.2, alpha=1.0, modes=4, seed=5, dtype=np.float64, noise=1e-3):
    """Periodic 2D heat problem on square cells, dx = 2 pi / nx (so the grid covers
    [0, 2 pi) x [0, 2 pi ny / nx)); u0 of shape (ny, nx) (x fastest) is
    sum_{k,l=1..modes} a_kl sin(2 pi k x / Lx) sin(2 pi l y / Ly), a_kl ~ U(-1, 1),
    plus noise * U(-1, 1) per point.  Fo = r (stable for r <= 1/4).  Returns a
    dict with u0, dx, dt, alpha, amps (modes x modes), r."""
    ny = nx if ny is None else ny
    dx = 2.0 * math.pi / nx
    dt = r * (dx * dx) / alpha
    g = rng(seed)
    amps = g.uniform(-1.0, 1.0, size=(modes, modes))
    x = np.arange(nx, dtype=np.float64) * dx
    y = np.arange(ny, dtype=np.float64) * dx
    Lx, Ly = nx * dx, ny * dx
    u0 = np.zeros((ny, nx), dtype=np.float64)
    for k in range(1, modes + 1):
        sx = np.sin(2.0 * math.pi * k * x / Lx)
        for l in range(1, modes + 1):
            u0 += amps[k - 1, l - 1] * np.outer(np.sin(2.0 * math.pi * l * y / Ly), sx)
    if noise:
        u0 += noise * g.uniform(-1.0, 1.0, size=(ny, nx))
    return dict(u0=u0.astype(dtype), dx=dx, dt=dt, alpha=alpha, amps=amps, r=r)


def ks_length(n):
    """Domain length for N points: 32 pi N / 128 (dx = pi / 4)."""
    return 32.0 * math.pi * n / 128.0


def ks_problem(n=1 << 14, seed=1, dtype=np.float64, dt=0.005, nu=1.0, noise=1e-3):
    """Periodic KS problem; returns dict with u0, dx, dt, nu, x."""
    L = ks_length(n)
    dx = L / n
    x = np.arange(n, dtype=np.float64) * dx
    u0 = np.cos(x / 16.0) * (1.0 + np.sin(x / 16.0)) + noise * rng(seed).uniform(-1.0, 1.0, size=n)
    return dict(u0=u0.astype(dtype), dx=dx, dt=dt, nu=nu, x=x, L=L)


def euler_dt(n, cfl=0.4, s_bound=2.5, t_end=0.2):
    """Fixed step for the Sod workload: 0.4 dx / 2.5, reset so nsteps * dt = t_end."""
    dx = 1.0 / n
    dt0 = cfl * dx / s_bound
    nsteps = int(math.ceil(t_end / dt0))
    return t_end / nsteps, nsteps


def euler_problem(n=1 << 16, seed=2, dtype=np.float64, gamma=1.4, perturb=0.01):
    """Sod tube (SoA conserved state of shape (3, n)); returns dict with U0, dx, dt, nsteps, gamma."""
    dx = 1.0 / n
    xc = (np.arange(n, dtype=np.float64) + 0.5) * dx
    rho = np.where(xc < 0.5, 1.0, 0.125)
    p = np.where(xc < 0.5, 1.0, 0.1)
    g = rng(seed)
    if perturb:
        rho = rho * (1.0 + perturb * g.uniform(-1.0, 1.0, size=n))
        p = p * (1.0 + perturb * g.uniform(-1.0, 1.0, size=n))
    u = np.zeros(n)
    U0 = np.stack([rho, rho * u, p / (gamma - 1.0) + 0.5 * rho * u * u])
    dt, nsteps = euler_dt(n)
    return dict(U0=U0.astype(dtype), dx=dx, dt=dt, nsteps=nsteps, gamma=gamma, x=xc)


def batch_problems(count=4096, seed=3, log2_lo=10, log2_hi=18, steps_lo=1000, steps_hi=20000, quantum=1024):
    """Sizes, scheme kinds (0 heat, 1 KS) and step counts of the batched workload."""
    g = rng(seed)
    raw = 2.0 ** g.uniform(log2_lo, log2_hi, size=count)
    n = (np.maximum(1, np.rint(raw / quantum)) * quantum).astype(np.int64)
    kind = g.integers(0, 2, size=count)
    steps = g.integers(steps_lo, steps_hi + 1, size=count)
    return dict(n=n, kind=kind, steps=steps)


def batch_instances(spec, dtype=np.float64, seed=4):
    """Per-problem parameters and initial states for a batch_problems() spec:
    list of dicts (scheme 0 heat / 1 KS, n, nsteps, dx, dt, param, u0)."""
    out = []
    for i, (n, kind, steps) in enumerate(zip(spec["n"], spec["kind"], spec["steps"])):
        n = int(n)
        if kind == 0:
            p = heat_problem(n=n, seed=seed * 100003 + i, dtype=dtype)
            out.append(dict(scheme=0, n=n, nsteps=int(steps), dx=p["dx"], dt=p["dt"], param=p["alpha"], u0=p["u0"]))
        else:
            p = ks_problem(n=n, seed=seed * 100003 + i, dtype=dtype)
            out.append(dict(scheme=1, n=n, nsteps=int(steps), dx=p["dx"], dt=p["dt"], param=p["nu"], u0=p["u0"]))
    return out
