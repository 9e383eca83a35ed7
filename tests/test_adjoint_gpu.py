"""GPU adjoint (swept_adjoint): the reverse swept sweep against the CPU oracle's
reverse mode on the same inputs, against central differences of GPU forward
solves, through torch.autograd, with and without recomputed segments.

dL/du0 is evaluated with the oracle's operation order, so it matches the
oracle bit for bit.  dL/dparam is a sum of N * S * nsteps products with a
second or fourth difference, of both signs and with heavy cancellation; the
GPU forms each term with the symmetric rewrite sum d4(lam) w = sum lam d4(w)
and adds them with compensated summation, the oracle in long double.  The
bound is 1e-12 relative plus 8 eps times the sum's condition
sum |lam| k |D|(|w|) (|D| the stencil with absolute weights), which covers the
few roundings of each term and the compensated sum's 2 eps.
"""

EPS = 2.0 ** -52


def param_tol(ref, cond):
    return 1e-12 * abs(ref) + 8 * EPS * cond
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


def gpu_adjoint(S, scheme, u0, dx, dt, p0, nsteps, gT, bc=0, tile_w=0, ckpt_bytes=0, via_forward=True):
    import torch

    sol = S.Solver(scheme, S.F64, u0.size, dx, dt, p0, bc=bc, tile_w=tile_w)
    nb = ckpt_bytes or sol.ckpt_size(nsteps)
    ckpt = torch.empty(nb, dtype=torch.uint8, device="cuda")
    u0d = torch.from_numpy(u0).cuda()
    gTd = torch.from_numpy(gT).cuda()
    if via_forward:
        u = u0d.clone()
        sol.forward_ckpt(u, nsteps, ckpt)
        g, gp = sol.adjoint(gTd, nsteps, ckpt)
    else:
        g, gp = sol.adjoint(gTd, nsteps, ckpt, u0=u0d)
    torch.cuda.synchronize()
    sol.sync_status()
    out = g.cpu().numpy(), float(gp.cpu().numpy()[0]), sol.plan
    sol.close()
    return out


KS_CASES = [
    # n, W, nsteps, ckpt mode
    (256, 32, 50, "default"),
    (256, 32, 50, "whole"),
    (384, 64, 77, "default"),
    (1024, 0, 203, "default"),
    (2048, 256, 64, "whole"),
]


@pytest.mark.parametrize("n,W,nsteps,mode", KS_CASES)
@pytest.mark.parametrize("via_forward", [True, False])
def test_ks_adjoint_matches_oracle(S, n, W, nsteps, mode, via_forward):
    p = inputs.ks_problem(n=n, seed=61)
    gT = inputs.rng(62).standard_normal(n)
    nb = 0
    if mode == "whole":
        nb = 8 * n * (2 * nsteps + 8) + (1 << 16)
    g, gnu, _ = gpu_adjoint(S, S.KS, p["u0"], p["dx"], p["dt"], 1.0, nsteps, gT, tile_w=W, ckpt_bytes=nb,
                            via_forward=via_forward)
    ref, ref_nu, cond = oracle.ks_adjoint(p["u0"], p["dx"], p["dt"], 1.0, nsteps, gT, with_condition=True)
    assert np.array_equal(g, ref), np.max(np.abs(g - ref)) / np.max(np.abs(ref))
    assert abs(gnu - ref_nu) <= param_tol(ref_nu, cond), (gnu, ref_nu, cond)


@pytest.mark.parametrize("bc", [0, 1])
@pytest.mark.parametrize("n,W,nsteps", [(64, 16, 37), (1024, 64, 500)])
def test_heat_adjoint_matches_oracle(S, bc, n, W, nsteps):
    p = inputs.heat_problem(n=n, seed=63)
    gT = inputs.rng(64).standard_normal(n)
    g, ga, _ = gpu_adjoint(S, S.HEAT, p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, gT, bc=bc, tile_w=W)
    ref, ref_a, cond = oracle.heat_adjoint(p["u0"], p["dx"], p["dt"], p["alpha"], nsteps, gT, bc=bc,
                                           with_condition=True)
    assert np.array_equal(g, ref)
    assert abs(ga - ref_a) <= param_tol(ref_a, cond), (ga, ref_a, cond)


def test_adjoint_rejects_fp32_and_euler(S):
    import torch

    sol = S.Solver(S.KS, S.F32, 256, 0.785, 0.005, 1.0, tile_w=32)
    with pytest.raises(S.SweptError):
        sol.ckpt_size(10)
    sol.close()
    sol = S.Solver(S.EULER, S.F64, 256, 1 / 256, 1e-4, 1.4, bc=1, tile_w=32)
    ck = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    g = torch.zeros(3 * 256, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SweptError):
        sol.adjoint(g, 10, ck, u0=g)
    sol.close()


def test_adjoint_requires_matching_forward(S):
    import torch

    sol = S.Solver(S.KS, S.F64, 256, 0.785, 0.005, 1.0, tile_w=32)
    ck = torch.empty(sol.ckpt_size(40), dtype=torch.uint8, device="cuda")
    g = torch.zeros(256, dtype=torch.float64, device="cuda")
    with pytest.raises(S.SweptError):
        sol.adjoint(g, 40, ck)  # no swept_forward_ckpt before
    sol.close()


def test_ks_adjoint_full_size_central_differences(S):
    """The adjoint workload: KS N=2^18 FP64, 5,000 steps, L = sum (u(T) - u_target)^2 with
    u_target from a seeded perturbed run; directional derivatives of dL/du0 and dL/dnu
    against central differences (h = 1e-6) of GPU forward solves."""
    import torch

    n, nsteps = 1 << 18, 5000
    p = inputs.ks_problem(n=n, seed=71)
    u0 = torch.from_numpy(p["u0"]).cuda()
    pert = torch.from_numpy(1e-3 * inputs.rng(72).standard_normal(n)).cuda()

    def forward(u_init, nu):
        sol = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], nu)
        u = u_init.clone()
        sol.step(u, nsteps)
        torch.cuda.synchronize()
        sol.close()
        return u

    target = forward(u0 + pert, 1.0)
    loss = lambda u: float(((u - target) ** 2).sum())
    uT = forward(u0, 1.0)
    sol = S.Solver(S.KS, S.F64, n, p["dx"], p["dt"], 1.0)
    ck = torch.empty(sol.ckpt_size(nsteps), dtype=torch.uint8, device="cuda")
    g, gnu = sol.adjoint(2 * (uT - target), nsteps, ck, u0=u0)
    torch.cuda.synchronize()
    sol.close()
    h = 1e-6
    for s in range(2):
        v = torch.from_numpy(inputs.rng(80 + s).standard_normal(n)).cuda()
        fd = (loss(forward(u0 + h * v, 1.0)) - loss(forward(u0 - h * v, 1.0))) / (2 * h)
        ad = float((g * v).sum())
        assert abs(fd - ad) <= 1e-5 * abs(ad), (fd, ad)
    fdnu = (loss(forward(u0, 1.0 + h)) - loss(forward(u0, 1.0 - h))) / (2 * h)
    assert abs(fdnu - float(gnu[0])) <= 1e-5 * abs(fdnu), (fdnu, float(gnu[0]))


def test_autograd_function(S):
    import torch

    n, nsteps = 512, 60
    p = inputs.ks_problem(n=n, seed=91)
    u0 = torch.from_numpy(p["u0"]).cuda().requires_grad_(True)
    nu = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    target = torch.from_numpy(inputs.rng(92).standard_normal(n)).cuda()
    uT = S.SweptSolve.apply(u0, nu, nsteps, dx=p["dx"], dt=p["dt"], tile_w=64)
    loss = ((uT - target) ** 2).sum()
    loss.backward()
    ref_uT = oracle.ks(p["u0"], p["dx"], p["dt"], 1.0, nsteps)
    assert np.array_equal(uT.detach().cpu().numpy(), ref_uT)
    gT = 2 * (ref_uT - target.cpu().numpy())
    ref, ref_nu, cond = oracle.ks_adjoint(p["u0"], p["dx"], p["dt"], 1.0, nsteps, gT, with_condition=True)
    assert np.array_equal(u0.grad.cpu().numpy(), ref)
    assert abs(float(nu.grad) - ref_nu) <= param_tol(ref_nu, cond)


def test_autograd_second_backward_with_retained_graph(S):
    """backward twice through a retained graph: the handle and its checkpoints
    stay alive with the autograd context, and both gradients equal the oracle's."""
    import torch

    n, nsteps = 512, 150
    p = inputs.ks_problem(n=n, seed=93)
    u0 = torch.from_numpy(p["u0"]).cuda().requires_grad_(True)
    nu = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    target = torch.from_numpy(inputs.rng(94).standard_normal(n)).cuda()
    uT = S.SweptSolve.apply(u0, nu, nsteps, dx=p["dx"], dt=p["dt"], tile_w=64)
    loss = ((uT - target) ** 2).sum()
    loss.backward(retain_graph=True)
    g1 = u0.grad.clone()
    u0.grad = None
    loss.backward()
    ref_uT = oracle.ks(p["u0"], p["dx"], p["dt"], 1.0, nsteps)
    ref = oracle.ks_adjoint(p["u0"], p["dx"], p["dt"], 1.0, nsteps, 2 * (ref_uT - target.cpu().numpy()))[0]
    assert np.array_equal(g1.cpu().numpy(), ref)
    assert np.array_equal(u0.grad.cpu().numpy(), ref)


def test_default_checkpoint_memory_is_the_smallest_layout(S):
    """swept_adjoint_ckpt_size gives the segment length with the least memory:
    at the adjoint workload's size (KS 2^18, 5,000 steps, tile 512: 64 steps per
    pass) that is one pass per segment, 79 checkpoints plus a 129-tier tape."""
    n = 1 << 18
    sol = S.Solver(S.KS, S.F64, n, 0.785, 0.005, 1.0, tile_w=512)
    nb = sol.ckpt_size(5000)
    sol.close()
    state = n * 8
    assert nb < (79 + 129 + 3) * state + (1 << 16), nb
    assert nb > (79 + 129) * state
