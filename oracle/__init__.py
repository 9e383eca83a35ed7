"""CPU oracle for the swept 1D stencil solvers (ctypes front end of liboracle.so).

TEST INFRASTRUCTURE ONLY.  This is the plain, slow, obviously correct definition
of what the GPU path computes: each scheme applied step by step over the whole
grid in FP64 (and an FP32 twin with the same evaluation order).  Only tests/,
__graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import
it.  The product package never imports it, and it imports nothing from the
product package.

Schemes (Magee & Niemeyer, arXiv:1612.02495):
  heat   FTCS, Eq. HeatDisc                                   (periodic or insulated)
  ks     Eq. KSDisc (u_i term read as -2 u_i) + midpoint RK2, Appendix (periodic)
  euler  MUSCL-minmod + Rusanov + SSP-RK2 (not in the paper)  (periodic or reflective)
  heat2d FTCS 5-point, the 2D extension of Eq. HeatDisc       (periodic or insulated)
Adjoints (not in the paper): exact discrete reverse mode of the FP64 forward.

Boundary codes used here: BC_PERIODIC = 0, BC_MIRROR = 1.
"""
import ctypes
import os

import numpy as np

from . import build as _build

BC_PERIODIC = 0
BC_MIRROR = 1

_lib = None
_D = ctypes.c_double
_I64 = ctypes.c_int64
_INT = ctypes.c_int
_P = ctypes.c_void_p


def lib():
    """Load (building first if needed) liboracle.so."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        for sfx in ("f64", "f32"):
            getattr(L, "oracle_heat_run_" + sfx).argtypes = [_P, _I64, _D, _D, _D, _INT, _I64, _INT]
            getattr(L, "oracle_ks_run_" + sfx).argtypes = [_P, _I64, _D, _D, _D, _I64, _INT]
            getattr(L, "oracle_euler_run_" + sfx).argtypes = [_P, _I64, _D, _D, _D, _INT, _I64, _INT]
            getattr(L, "oracle_euler_stage_" + sfx).argtypes = [_P, _P, _I64, _D, _D, _D, _INT]
            getattr(L, "oracle_heat2d_run_" + sfx).argtypes = [_P, _I64, _I64, _D, _D, _D, _INT, _I64, _INT]
        L.oracle_ks_adjoint_f64.argtypes = [_P, _I64, _D, _D, _D, _I64, _P, _P, _P, _I64, _P, _INT]
        L.oracle_heat_adjoint_f64.argtypes = [_P, _I64, _D, _D, _D, _INT, _I64, _P, _P, _P, _P]
        L.oracle_max_threads.restype = _INT
        _lib = L
    return _lib


def _sfx(dtype):
    dtype = np.dtype(dtype)
    if dtype == np.float64:
        return "f64"
    if dtype == np.float32:
        return "f32"
    raise TypeError("oracle supports float32 and float64, got %s" % dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc, what):
    if rc != 0:
        raise ValueError("%s: oracle returned %d (invalid arguments)" % (what, rc))


def max_threads():
    """Thread count OpenMP uses in this process (1 without OpenMP)."""
    return int(lib().oracle_max_threads())


def heat(u0, dx, dt, alpha, nsteps, bc=BC_PERIODIC, threads=1):
    """FTCS heat equation: u0 advanced `nsteps` steps (returns a new array, dtype kept)."""
    u = np.array(u0, copy=True, order="C")
    _check(getattr(lib(), "oracle_heat_run_" + _sfx(u.dtype))(_ptr(u), u.size, dx, dt, alpha, bc, nsteps, threads),
           "heat")
    return u


def heat2d(u0, dx, dt, alpha, nsteps, bc=BC_PERIODIC, threads=1):
    """2D FTCS heat equation on a square-celled grid; u0 has shape (ny, nx) (row-major,
    x fastest).  Returns u0 advanced `nsteps` steps (new array, dtype kept)."""
    u = np.array(u0, copy=True, order="C")
    if u.ndim != 2:
        raise ValueError("heat2d state must have shape (ny, nx)")
    ny, nx = u.shape
    _check(getattr(lib(), "oracle_heat2d_run_" + _sfx(u.dtype))(_ptr(u), nx, ny, dx, dt, alpha, bc, nsteps, threads),
           "heat2d")
    return u


def ks(u0, dx, dt, nu, nsteps, threads=1):
    """Kuramoto-Sivashinsky (periodic), midpoint RK2: `nsteps` full steps."""
    u = np.array(u0, copy=True, order="C")
    _check(getattr(lib(), "oracle_ks_run_" + _sfx(u.dtype))(_ptr(u), u.size, dx, dt, nu, nsteps, threads), "ks")
    return u


def euler(U0, dx, dt, gamma, nsteps, bc=BC_MIRROR, threads=1):
    """1D Euler, SoA state of shape (3, n) = (rho, m, E); `nsteps` SSP-RK2 steps."""
    U = np.array(U0, copy=True, order="C")
    if U.ndim != 2 or U.shape[0] != 3:
        raise ValueError("euler state must have shape (3, n)")
    _check(getattr(lib(), "oracle_euler_run_" + _sfx(U.dtype))(_ptr(U), U.shape[1], dx, dt, gamma, bc, nsteps,
                                                               threads), "euler")
    return U


def euler_stage(U0, dx, dt, gamma, bc=BC_MIRROR):
    """One explicit Euler stage U + dt L(U) of the finite-volume operator."""
    U = np.ascontiguousarray(U0)
    out = np.empty_like(U)
    _check(getattr(lib(), "oracle_euler_stage_" + _sfx(U.dtype))(_ptr(U), _ptr(out), U.shape[1], dx, dt, gamma, bc),
           "euler_stage")
    return out


def ks_adjoint(u0, dx, dt, nu, nsteps, gT, seg=0, with_condition=False, threads=1):
    """Discrete adjoint of `ks` (FP64): returns (dL/du0, dL/dnu) for dL/du(T) = gT; with
    with_condition, also the sum of the absolute values of dL/dnu's terms (its condition).
    seg = checkpoint segment length in steps (0: one segment); threads = OpenMP threads
    (dL/du0 does not depend on it; dL/dnu only through its double-double rounding)."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    gT = np.ascontiguousarray(gT, dtype=np.float64)
    g = np.empty_like(u0)
    gnu = np.zeros(2)
    _check(lib().oracle_ks_adjoint_f64(_ptr(u0), u0.size, dx, dt, nu, nsteps, _ptr(gT), _ptr(g), _ptr(gnu[0:]), seg,
                                       _ptr(gnu[1:]), int(threads)), "ks_adjoint")
    return (g, float(gnu[0]), float(gnu[1])) if with_condition else (g, float(gnu[0]))


def heat_adjoint(u0, dx, dt, alpha, nsteps, gT, bc=BC_PERIODIC, with_condition=False):
    """Discrete adjoint of `heat` (FP64): returns (dL/du0, dL/dalpha) for dL/du(T) = gT; with
    with_condition, also the sum of the absolute values of dL/dalpha's terms."""
    u0 = np.ascontiguousarray(u0, dtype=np.float64)
    gT = np.ascontiguousarray(gT, dtype=np.float64)
    g = np.empty_like(u0)
    ga = np.zeros(2)
    _check(lib().oracle_heat_adjoint_f64(_ptr(u0), u0.size, dx, dt, alpha, bc, nsteps, _ptr(gT), _ptr(g),
                                         _ptr(ga[0:]), _ptr(ga[1:])), "heat_adjoint")
    return (g, float(ga[0]), float(ga[1])) if with_condition else (g, float(ga[0]))
