"""Pins of the CPU oracle against what the mathematics fixes (no GPU needed).

Each test ties the oracle to something other than itself: an exact discrete
solution, a conservation law, a consistency order, an exact Riemann solution,
a library routine on a case that reduces to it, or a finite-difference check.
They are chosen so that a dropped term, a wrong sign, a shifted index or a
wrong coefficient in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import BC_MIRROR, BC_PERIODIC
from paper_1612_02495_gb300 import inputs
from tests.sod_exact import sod_density, star_state


def relerr(a, ref):
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(a - ref)) / np.max(np.abs(ref)))


# ---------------------------------------------------------------------------
# Heat (Eq. HeatDisc)
# ---------------------------------------------------------------------------

def heat_exact(prob, nsteps):
    """Exact discrete FTCS solution on Fourier modes, in long double:
    u_i^n = sum_k a_k g_k^n sin(k x_i),  g_k = 1 - 4 Fo sin^2(k dx / 2)."""
    n = prob["u0"].size
    ld = np.longdouble
    fo = ld(prob["alpha"]) * ld(prob["dt"]) / (ld(prob["dx"]) * ld(prob["dx"]))
    dx = ld(2) * ld(np.pi) / ld(n)
    x = np.arange(n, dtype=ld) * dx
    out = np.zeros(n, dtype=ld)
    for k, a in enumerate(prob["amps"], start=1):
        g = ld(1) - ld(4) * fo * np.sin(ld(k) * dx / ld(2)) ** 2
        out += ld(a) * g ** nsteps * np.sin(ld(k) * x)
    return out


def test_heat_exact_discrete_solution_fp64():
    """Heat, N=1024 FP64, r=0.25, 10,000 steps against the closed form (<= 1e-12)."""
    p = inputs.heat_problem(n=1024)
    u = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], 10000)
    assert relerr(u, heat_exact(p, 10000)) <= 1e-12


def test_heat_exact_discrete_solution_fp32():
    """FP32 twin: within 1e-5 of the exact discrete solution at 2,000 steps; at
    10,000 steps FP32 rounding has accumulated to ~2e-5 (bounded here by 3e-5)."""
    p = inputs.heat_problem(n=1024, dtype=np.float32)
    u = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], 2000)
    assert u.dtype == np.float32
    assert relerr(u, heat_exact(p, 2000)) <= 1e-5
    u = oracle.heat(p["u0"], p["dx"], p["dt"], p["alpha"], 10000)
    assert relerr(u, heat_exact(p, 10000)) <= 3e-5


def test_heat_circulant_matrix_power():
    """Tiny grid: FTCS is multiplication by a circulant matrix (numpy matrix_power)."""
    n, fo = 12, 0.3
    u0 = inputs.rng(11).uniform(-1, 1, n)
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] = 1 - 2 * fo
        A[i, (i + 1) % n] += fo
        A[i, (i - 1) % n] += fo
    dx, alpha = 0.5, 1.0
    dt = fo * dx * dx / alpha
    u = oracle.heat(u0, dx, dt, alpha, 7)
    assert relerr(u, np.linalg.matrix_power(A, 7) @ u0) <= 1e-14


def test_heat_mean_conserved_periodic():
    p = inputs.heat_problem(n=1000, seed=5)
    u0 = p["u0"] + 0.3
    u = oracle.heat(u0, p["dx"], p["dt"], p["alpha"], 3000)
    assert abs(u.sum() - u0.sum()) <= 1e-12 * np.abs(u0).sum()


def test_heat_insulated_cosine_eigenmode():
    """Mirror (insulated) ends: cos(k pi (i + 1/2) / N) is an exact discrete eigenvector
    with factor 1 - 4 Fo sin^2(k pi / (2N))."""
    n, k, fo, steps = 200, 3, 0.25, 500
    th = k * math.pi / n
    v = np.cos(th * (np.arange(n) + 0.5))
    dx, alpha = 1.0 / n, 1.0
    dt = fo * dx * dx / alpha
    u = oracle.heat(v, dx, dt, alpha, steps, bc=BC_MIRROR)
    g = 1 - 4 * fo * math.sin(th / 2) ** 2
    assert relerr(u, v * g ** steps) <= 1e-12


# ---------------------------------------------------------------------------
# Kuramoto-Sivashinsky (Eq. KSDisc + midpoint RK2)
# ---------------------------------------------------------------------------

def ks_exact_rhs(x, A, kap, nu):
    """f = -u u_x - u_xx - nu u_xxxx for u = A sin(kap x)."""
    s, c = np.sin(kap * x), np.cos(kap * x)
    return -(A * s) * (A * kap * c) + A * kap ** 2 * s - nu * A * kap ** 4 * s


def test_ks_consistency_second_order():
    """One tiny step: (u1 - u0)/dt -> f(u0) of the PDE at second order in dx
    (catches any wrong coefficient, sign or neighbour index in Eq. KSDisc)."""
    nu, A, kap, dt = 0.7, 1.3, 2.0, 1e-9
    errs = []
    for n in (64, 128, 256):
        dx = 2 * math.pi / n
        x = np.arange(n) * dx
        u0 = A * np.sin(kap * x)
        u1 = oracle.ks(u0, dx, dt, nu, 1)
        errs.append(np.max(np.abs((u1 - u0) / dt - ks_exact_rhs(x, A, kap, nu))))
    r1, r2 = errs[0] / errs[1], errs[1] / errs[2]
    assert 3.6 < r1 < 4.4 and 3.6 < r2 < 4.4, errs
    assert errs[2] < 0.05


def test_ks_linear_growth_matches_rk2_polynomial():
    """Tiny single mode: per-step factor is 1 + z + z^2/2 with z = dt lambda_k,
    lambda_k = s/dx^2 - nu s^2/dx^4, s = 4 sin^2(k dx / 2) (midpoint RK2)."""
    n, nu = 128, 1.0
    p = inputs.ks_problem(n=n)
    dx, dt = p["dx"], p["dt"]
    for k in (1, 5, 17, 40):
        x = np.arange(n) * dx
        eps = 1e-12
        u0 = eps * np.sin(k * 2 * math.pi / (n * dx) * x)
        steps = 50
        u = oracle.ks(u0, dx, dt, nu, steps)
        th = 2 * math.pi * k / n
        s = 4 * math.sin(th / 2) ** 2
        z = dt * (s / dx ** 2 - nu * s ** 2 / dx ** 4)
        g = (1 + z + z * z / 2) ** steps
        assert relerr(u, u0 * g) <= 1e-9, k


def test_ks_mean_conserved():
    p = inputs.ks_problem(n=4096)
    u = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], 2000)
    assert abs(u.sum() - p["u0"].sum()) <= 1e-12 * np.abs(p["u0"]).sum()


def test_ks_fp32_twin_tracks_fp64():
    p64 = inputs.ks_problem(n=2048)
    p32 = inputs.ks_problem(n=2048, dtype=np.float32)
    a = oracle.ks(p64["u0"], p64["dx"], p64["dt"], p64["nu"], 200)
    b = oracle.ks(p32["u0"], p32["dx"], p32["dt"], p32["nu"], 200)
    assert b.dtype == np.float32
    assert relerr(b, a) <= 1e-5


def test_ks_threads_do_not_change_result():
    p = inputs.ks_problem(n=4096)
    a = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], 50, threads=1)
    b = oracle.ks(p["u0"], p["dx"], p["dt"], p["nu"], 50, threads=4)
    assert np.array_equal(a, b)


# ---------------------------------------------------------------------------
# Euler (MUSCL-minmod + Rusanov + SSP-RK2; a reading, not in the paper)
# ---------------------------------------------------------------------------

def prim_to_cons(rho, u, p, gamma=1.4):
    return np.stack([rho, rho * u, p / (gamma - 1) + 0.5 * rho * u * u])


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_MIRROR])
def test_euler_uniform_state_exact(bc):
    n = 64
    U0 = prim_to_cons(np.full(n, 0.8), np.full(n, 0.0 if bc == BC_MIRROR else 0.3), np.full(n, 0.6))
    U = oracle.euler(U0, 1.0 / n, 0.2 / n, 1.4, 40, bc=bc)
    assert np.array_equal(U, U0)


def test_euler_periodic_conserves_mass_momentum_energy():
    n = 256
    g = inputs.rng(21)
    x = (np.arange(n) + 0.5) / n
    rho = 1 + 0.3 * np.sin(2 * np.pi * x) + 0.05 * g.uniform(-1, 1, n)
    u = 0.4 * np.cos(2 * np.pi * x)
    p = 1 + 0.2 * np.sin(4 * np.pi * x)
    U0 = prim_to_cons(rho, u, p)
    U = oracle.euler(U0, 1.0 / n, 0.3 / n, 1.4, 300, bc=BC_PERIODIC)
    for c in range(3):
        assert abs(U[c].sum() - U0[c].sum()) <= 1e-13 * np.abs(U0[c]).sum() * 10, c


def test_euler_reflective_conserves_mass_and_energy():
    pr = inputs.euler_problem(n=512)
    U = oracle.euler(pr["U0"], pr["dx"], pr["dt"], pr["gamma"], 400, bc=BC_MIRROR)
    for c in (0, 2):
        assert abs(U[c].sum() - pr["U0"][c].sum()) <= 1e-12 * np.abs(pr["U0"][c]).sum(), c


def test_euler_mirror_symmetry_exact():
    """A mirror-symmetric state stays exactly mirror-symmetric (rho, E even; m odd)."""
    n = 256
    x = (np.arange(n) + 0.5) / n
    rho = np.where(np.abs(x - 0.5) > 0.25, 1.0, 0.125)
    p = np.where(np.abs(x - 0.5) > 0.25, 1.0, 0.1)
    U0 = prim_to_cons(rho, np.zeros(n), p)
    dt, _ = inputs.euler_dt(n)
    U = oracle.euler(U0, 1.0 / n, dt, 1.4, 150, bc=BC_MIRROR)
    assert np.array_equal(U[0], U[0][::-1])
    assert np.array_equal(U[2], U[2][::-1])
    assert np.array_equal(U[1], -U[1][::-1])
    assert np.abs(U[1]).max() > 1e-3  # the waves did move


def test_euler_heun_composition():
    """One SSP-RK2 step equals 0.5 (U + S(S(U))) with S the forward-Euler stage."""
    pr = inputs.euler_problem(n=128)
    U0 = pr["U0"]
    S = lambda V: oracle.euler_stage(V, pr["dx"], pr["dt"], pr["gamma"], bc=BC_MIRROR)
    U1 = oracle.euler(U0, pr["dx"], pr["dt"], pr["gamma"], 1, bc=BC_MIRROR)
    assert np.array_equal(U1, 0.5 * (U0 + S(S(U0))))


def test_sod_exact_helper_star_state():
    # published star state of Sod's problem: p* = 0.30313, u* = 0.92745
    p, u = star_state((1.0, 0.0, 1.0), (0.125, 0.0, 0.1))
    assert abs(p - 0.30313) < 1e-5 and abs(u - 0.92745) < 1e-5


def test_euler_sod_converges_to_exact_riemann_solution():
    errs = []
    for n in (128, 256, 512, 1024):
        pr = inputs.euler_problem(n=n, perturb=0.0)
        U = oracle.euler(pr["U0"], pr["dx"], pr["dt"], pr["gamma"], pr["nsteps"], bc=BC_MIRROR)
        ex = sod_density(pr["x"], 0.2)
        errs.append(np.mean(np.abs(U[0] - ex)))
    for a, b in zip(errs, errs[1:]):
        assert b < 0.8 * a, errs
    assert errs[-1] < 4e-3, errs


# ---------------------------------------------------------------------------
# Adjoints (reverse mode of the FP64 forward)
# ---------------------------------------------------------------------------

def test_ks_adjoint_matches_central_differences():
    n, steps = 64, 40
    p = inputs.ks_problem(n=n, seed=31)
    u0, dx, dt, nu = p["u0"], p["dx"], p["dt"], 1.0
    target = oracle.ks(u0 + 1e-3 * inputs.rng(32).standard_normal(n), dx, dt, nu, steps)

    def loss(u, nu_):
        return float(np.sum((oracle.ks(u, dx, dt, nu_, steps) - target) ** 2))

    uT = oracle.ks(u0, dx, dt, nu, steps)
    g, gnu = oracle.ks_adjoint(u0, dx, dt, nu, steps, 2 * (uT - target), seg=7)
    h = 1e-6
    for s in range(4):
        v = inputs.rng(40 + s).standard_normal(n)
        fd = (loss(u0 + h * v, nu) - loss(u0 - h * v, nu)) / (2 * h)
        assert abs(fd - g @ v) <= 1e-6 * max(abs(fd), 1e-12) + 1e-9, (fd, g @ v)
    fdnu = (loss(u0, nu + h) - loss(u0, nu - h)) / (2 * h)
    assert abs(fdnu - gnu) <= 1e-6 * abs(fdnu) + 1e-9, (fdnu, gnu)


def test_ks_adjoint_checkpoint_segments_agree():
    p = inputs.ks_problem(n=96, seed=33)
    gT = inputs.rng(34).standard_normal(96)
    a = oracle.ks_adjoint(p["u0"], p["dx"], p["dt"], 1.0, 30, gT, seg=0)
    b = oracle.ks_adjoint(p["u0"], p["dx"], p["dt"], 1.0, 30, gT, seg=4)
    assert np.array_equal(a[0], b[0])
    assert abs(a[1] - b[1]) <= 1e-15 * abs(a[1])


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_MIRROR])
def test_heat_adjoint_closed_form(bc):
    """Heat is linear: dL/du0 = (A^T)^n gT; dL/dalpha against central differences."""
    n, fo, steps = 16, 0.3, 9
    dx, alpha = 0.25, 1.0
    dt = fo * dx * dx / alpha
    A = np.zeros((n, n))
    for i in range(n):
        A[i, i] += 1 - 2 * fo
        for j in (i - 1, i + 1):
            if 0 <= j < n:
                A[i, j] += fo
            elif bc == BC_PERIODIC:
                A[i, j % n] += fo
            else:
                A[i, i] += fo  # mirror ghost reads the cell itself
    u0 = inputs.rng(51).uniform(-1, 1, n)
    gT = inputs.rng(52).uniform(-1, 1, n)
    g, ga = oracle.heat_adjoint(u0, dx, dt, alpha, steps, gT, bc=bc)
    assert relerr(g, np.linalg.matrix_power(A.T, steps) @ gT) <= 1e-13
    h = 1e-6
    Lp = gT @ oracle.heat(u0, dx, dt, alpha + h, steps, bc=bc)
    Lm = gT @ oracle.heat(u0, dx, dt, alpha - h, steps, bc=bc)
    assert abs((Lp - Lm) / (2 * h) - ga) <= 1e-7 * abs(ga) + 1e-10


# ---------------------------------------------------------------------------
# 2D heat (FTCS 5-point; the 2D extension of Eq. HeatDisc)
# ---------------------------------------------------------------------------

def heat2d_exact_periodic(prob, nsteps):
    """Exact discrete solution on product sine modes, in long double:
    sin(2 pi k i / nx) sin(2 pi l j / ny) is an eigenvector of one step with factor
    g_kl = 1 - 4 Fo sin^2(pi k / nx) - 4 Fo sin^2(pi l / ny)."""
    ny, nx = prob["u0"].shape
    ld = np.longdouble
    fo = ld(prob["alpha"]) * ld(prob["dt"]) / (ld(prob["dx"]) * ld(prob["dx"]))
    pi = ld(np.pi)
    i = np.arange(nx, dtype=ld)
    j = np.arange(ny, dtype=ld)
    out = np.zeros((ny, nx), dtype=ld)
    m = prob["amps"].shape[0]
    for k in range(1, m + 1):
        for l in range(1, m + 1):
            g = ld(1) - ld(4) * fo * np.sin(pi * k / nx) ** 2 - ld(4) * fo * np.sin(pi * l / ny) ** 2
            out += ld(prob["amps"][k - 1, l - 1]) * g ** nsteps * np.outer(np.sin(ld(2) * pi * l * j / ny),
                                                                         np.sin(ld(2) * pi * k * i / nx))
    return out


def test_heat2d_exact_discrete_solution_periodic():
    """2D heat on a 128 x 96 grid (non-square, so a transposed index fails), 2,000 steps,
    against the product-mode closed form (<= 1e-12).  The grid is large enough that the
    slowest mode keeps 1 % of its amplitude, so the bound is not inflated by decay."""
    p = inputs.heat2d_problem(nx=128, ny=96, noise=0.0)
    u = oracle.heat2d(p["u0"], p["dx"], p["dt"], p["alpha"], 2000)
    assert relerr(u, heat2d_exact_periodic(p, 2000)) <= 1e-12


def test_heat2d_insulated_eigenvector():
    """Insulated (mirror) walls: cos(pi k (i + 1/2) / nx) cos(pi l (j + 1/2) / ny) is an exact
    eigenvector with factor 1 - 4 Fo sin^2(pi k / 2 nx) - 4 Fo sin^2(pi l / 2 ny)."""
    nx, ny, fo, steps = 80, 48, 0.2, 300
    dx = 0.1
    dt = fo * dx * dx
    ld = np.longdouble
    for k, l in ((1, 1), (3, 2), (5, 4)):
        ci = np.cos(np.pi * k * (np.arange(nx) + 0.5) / nx)
        cj = np.cos(np.pi * l * (np.arange(ny) + 0.5) / ny)
        u0 = np.outer(cj, ci)
        g = ld(1) - ld(4) * ld(fo) * np.sin(ld(np.pi) * k / (2 * nx)) ** 2 \
            - ld(4) * ld(fo) * np.sin(ld(np.pi) * l / (2 * ny)) ** 2
        u = oracle.heat2d(u0, dx, dt, 1.0, steps, bc=BC_MIRROR)
        assert relerr(u, np.asarray(u0, dtype=ld) * g ** steps) <= 1e-12


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_MIRROR])
def test_heat2d_conserves_sum(bc):
    """Periodic and insulated 2D heat conserve the total heat (no flux through walls)."""
    p = inputs.heat2d_problem(nx=32, ny=20, noise=0.3)
    u0 = p["u0"] + 0.5
    u = oracle.heat2d(u0, p["dx"], p["dt"], p["alpha"], 500, bc=bc)
    assert abs(u.sum() - u0.sum()) <= 1e-12 * np.abs(u0).sum() * 10


@pytest.mark.parametrize("bc", [BC_PERIODIC, BC_MIRROR])
def test_heat2d_matrix_power(bc):
    """Brute force on a 5 x 3 grid: the one-step matrix built from the stencil definition,
    raised to the 37th power, applied to a random state."""
    nx, ny, fo, steps = 5, 3, 0.23, 37
    u0 = inputs.rng(77).standard_normal((ny, nx))

    def idx(q, n):
        if 0 <= q < n:
            return q
        if bc == BC_PERIODIC:
            return q % n
        return -1 - q if q < 0 else 2 * n - 1 - q

    A = np.zeros((nx * ny, nx * ny))
    for j in range(ny):
        for i in range(nx):
            r = j * nx + i
            A[r, r] += 1 - 4 * fo
            for (ii, jj) in ((i - 1, j), (i + 1, j), (i, j - 1), (i, j + 1)):
                A[r, idx(jj, ny) * nx + idx(ii, nx)] += fo
    ref = (np.linalg.matrix_power(A, steps) @ u0.ravel()).reshape(ny, nx)
    u = oracle.heat2d(u0, 1.0, fo, 1.0, steps, bc=bc)
    assert relerr(u, ref) <= 1e-13


def test_heat2d_reduces_to_1d():
    """A field constant in y evolves as the 1D FTCS heat equation with the same Fo."""
    p1 = inputs.heat_problem(n=96, r=0.2)
    u2 = np.tile(p1["u0"], (16, 1))
    u = oracle.heat2d(u2, p1["dx"], p1["dt"], p1["alpha"], 300)
    ref = oracle.heat(p1["u0"], p1["dx"], p1["dt"], p1["alpha"], 300)
    assert relerr(u, np.tile(ref, (16, 1))) <= 1e-13


def test_heat2d_fp32_twin_and_threads():
    """FP32 twin within 1e-5 of FP64 at 500 steps; results independent of the thread count."""
    p64 = inputs.heat2d_problem(nx=64, ny=64)
    p32 = inputs.heat2d_problem(nx=64, ny=64, dtype=np.float32)
    a = oracle.heat2d(p64["u0"], p64["dx"], p64["dt"], p64["alpha"], 500)
    b = oracle.heat2d(p32["u0"], p32["dx"], p32["dt"], p32["alpha"], 500)
    assert b.dtype == np.float32 and relerr(b, a) <= 1e-5
    c = oracle.heat2d(p64["u0"], p64["dx"], p64["dt"], p64["alpha"], 500, threads=4)
    assert np.array_equal(a, c)
