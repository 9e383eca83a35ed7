/*
 * CPU oracle for the swept 1D stencil solvers.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the plain, slow definition that the
 * GPU path is checked against.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline leg of bench.py load it.  The product path (the CUDA library and
 * its Python binding) never loads, links or calls anything here, and this file
 * shares no code, header or constant table with it.
 *
 * What it follows (Magee & Niemeyer, "An initial investigation of the performance
 * of GPU-based swept time-space decomposition"):
 *   - heat:  FTCS, Eq. HeatDisc (Section "Test cases", Appendix);
 *   - KS:    5-point central differences, Eq. KSDisc, with midpoint RK2 (Appendix);
 *   - the swept rule reorders where and when each (point, sub-timestep) is
 *     evaluated but does not change the scheme (Section "Related work"), so the
 *     oracle is the scheme applied step by step over the whole grid;
 *   - constants (Fo, 1/(4 dx), 1/dx^2, 1/dx^4) are stored and multiplied rather
 *     than divided by (Section "Results", Fig. divisionComparison).
 * Not in the paper, and therefore readings: the Euler finite-volume scheme, the
 * viscosity factor nu on u_xxxx, the mirror ghost cells, and the adjoints.
 *
 * Compile in ISO C with -ffp-contract=off: every fused multiply-add is an
 * explicit fma()/fmaf() call, and no other product is fused.
 *
 * Boundary codes (this file's own): 0 = periodic, 1 = mirror (cell-centred walls:
 * insulated for heat, reflective with momentum negated for Euler).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

enum { OR_BC_PERIODIC = 0, OR_BC_MIRROR = 1 };

/* Index of grid neighbour j (may lie outside [0, n)) after the boundary rule.
 * Mirror walls sit at x = -1/2 and x = n - 1/2: cell -1-k reads cell k and cell
 * n+k reads cell n-1-k.  *flip (if given) is set to 1 when the value comes
 * through a wall (Euler negates the momentum there). */
static inline int64_t nb_index(int64_t j, int64_t n, int bc, int* flip) {
  if (flip) *flip = 0;
  if (j >= 0 && j < n) return j;
  if (bc == OR_BC_PERIODIC) {
    int64_t r = j % n;
    return r < 0 ? r + n : r;
  }
  if (flip) *flip = 1;
  if (j < 0) return -1 - j;
  return 2 * n - 1 - j;
}

#define REAL double
#define SFX(name) name##_f64
#define FMA fma
#define SQRT sqrt
#define FABS fabs
#include "scheme_body.inc"
#undef REAL
#undef SFX
#undef FMA
#undef SQRT
#undef FABS

#define REAL float
#define SFX(name) name##_f32
#define FMA fmaf
#define SQRT sqrtf
#define FABS fabsf
#include "scheme_body.inc"
#undef REAL
#undef SFX
#undef FMA
#undef SQRT
#undef FABS

/* ========================================================================= */
/* Discrete adjoints (reverse mode) of the FP64 forward schemes above.        */
/* Not in the paper.  They are the exact transposes of the forward sequence,  */
/* so they differentiate what the forward code computes, step by step.        */
/* ========================================================================= */

/*
 * KS.  Forward step m:  P = u + (dt/2) f(u);  u' = u + dt f(P),  f = -g.
 * With J(w) the Jacobian of g at w (periodic):
 *   (J(w)^T lam)_j = 2 c_a w_j (lam_{j-1} - lam_{j+1})
 *                  + c_2 (lam_{j+1} + lam_{j-1} - 2 lam_j)
 *                  + c_4 (lam_{j+2} - 4 lam_{j+1} + 6 lam_j - 4 lam_{j-1} + lam_{j-2})
 * (the linear stencils are symmetric, so they are their own transposes).
 * Reverse of step m, given lam' = dL/du^{m+1}:
 *   mu  = dL/dP  = -dt J(P)^T lam'
 *   lam = dL/du^m = lam' + mu - (dt/2) J(u^m)^T mu
 * Evaluation order of gT = J(w)^T lam at j:
 *   sp1 = lam_{j+1} + lam_{j-1};  sp2 = lam_{j+2} + lam_{j-2};  dl = lam_{j-1} - lam_{j+1}
 *   nl  = (ca2 * w_j) * dl            (ca2 = 2 c_a, exact)
 *   d2  = fma(-2, lam_j, sp1);  d4 = fma(6, lam_j, fma(-4, sp1, sp2))
 *   gT  = fma(c_4, d4, fma(c_2, d2, nl))
 *   mu  = mdt * gT(lam'; P)                       (mdt = -dt)
 *   lam = fma(mdth, gT(mu; u), lam' + mu)         (mdth = -dt/2)
 * Parameter derivative (c_4 = nu k4, k4 = 1/dx^4, dg/dnu = k4 d4(w)):
 *   dL/dnu = sum_m sum_j [ -dt lam'_j k4 d4(P)_j - (dt/2) mu_j k4 d4(u^m)_j ]
 * Each term is formed and added in double-double arithmetic (about 106
 * significand bits: Knuth's TwoSum for sums, Dekker's exact product through
 * fma), in the order m descending, j ascending, then rounded once to double.
 * With threads > 1 each thread sums its own contiguous range of j over all m
 * and the per-thread sums are added in thread order; the result then differs
 * from the one-thread order only by the double-double rounding (~1e-32 of the
 * condition below), far inside any tolerance built on that condition.
 * Also returned: the same sum with every factor replaced by its absolute
 * value and d4 by the absolute stencil |w_{j+2}| + 4|w_{j+1}| + 6|w_j| +
 * 4|w_{j-1}| + |w_{j-2}| -- the condition of the sum, which bounds the
 * rounding error of any evaluation of it that rounds each term a few times.
 */
static inline double ks_gT(const double* lam, const double* w, int64_t j, int64_t n, double ca2, double c2,
                           double c4) {
  const double lm2 = lam[nb_index(j - 2, n, OR_BC_PERIODIC, NULL)];
  const double lm1 = lam[nb_index(j - 1, n, OR_BC_PERIODIC, NULL)];
  const double l0 = lam[j];
  const double lp1 = lam[nb_index(j + 1, n, OR_BC_PERIODIC, NULL)];
  const double lp2 = lam[nb_index(j + 2, n, OR_BC_PERIODIC, NULL)];
  const double sp1 = lp1 + lm1;
  const double sp2 = lp2 + lm2;
  const double dl = lm1 - lp1;
  const double nl = (ca2 * w[j]) * dl;
  const double d2 = fma(-2.0, l0, sp1);
  const double d4 = fma(6.0, l0, fma(-4.0, sp1, sp2));
  return fma(c4, d4, fma(c2, d2, nl));
}

static inline double ks_d4_abs(const double* w, int64_t j, int64_t n) {
  return fabs(w[nb_index(j + 2, n, OR_BC_PERIODIC, NULL)]) + 4.0 * fabs(w[nb_index(j + 1, n, OR_BC_PERIODIC, NULL)]) +
         6.0 * fabs(w[j]) + 4.0 * fabs(w[nb_index(j - 1, n, OR_BC_PERIODIC, NULL)]) +
         fabs(w[nb_index(j - 2, n, OR_BC_PERIODIC, NULL)]);
}

/* Double-double accumulation (value hi + lo, |lo| <= ulp(hi)/2). */
typedef struct {
  double hi, lo;
} oracle_dd;

/* Knuth's TwoSum: s + e == a + b exactly. */
static inline oracle_dd dd_two_sum(double a, double b) {
  const double s = a + b;
  const double bp = s - a;
  const double e = (a - (s - bp)) + (b - bp);
  oracle_dd r = {s, e};
  return r;
}
/* |a| >= |b| (or a == 0): s + e == a + b exactly. */
static inline oracle_dd dd_fast_two_sum(double a, double b) {
  const double s = a + b;
  oracle_dd r = {s, b - (s - a)};
  return r;
}
/* Dekker's exact product via fma: p + e == a * b exactly. */
static inline oracle_dd dd_two_prod(double a, double b) {
  const double p = a * b;
  oracle_dd r = {p, fma(a, b, -p)};
  return r;
}
static inline oracle_dd dd_mul_d(oracle_dd a, double b) {
  oracle_dd p = dd_two_prod(a.hi, b);
  return dd_fast_two_sum(p.hi, fma(a.lo, b, p.lo));
}
static inline oracle_dd dd_add(oracle_dd a, oracle_dd b) {
  oracle_dd s = dd_two_sum(a.hi, b.hi);
  const oracle_dd t = dd_two_sum(a.lo, b.lo);
  s = dd_fast_two_sum(s.hi, s.lo + t.hi);
  return dd_fast_two_sum(s.hi, s.lo + t.lo);
}
/* a * b * c * d as a double-double (relative error ~1e-32) */
static inline oracle_dd dd_prod4(double a, double b, double c, double d) {
  return dd_mul_d(dd_mul_d(dd_two_prod(a, b), c), d);
}

static inline double ks_d4(const double* w, int64_t j, int64_t n) {
  const double sp1 = w[nb_index(j + 1, n, OR_BC_PERIODIC, NULL)] + w[nb_index(j - 1, n, OR_BC_PERIODIC, NULL)];
  const double sp2 = w[nb_index(j + 2, n, OR_BC_PERIODIC, NULL)] + w[nb_index(j - 2, n, OR_BC_PERIODIC, NULL)];
  return fma(6.0, w[j], fma(-4.0, sp1, sp2));
}

/*
 * u0: initial state (n); gT: dL/du(T) (n).  Outputs g_u0 = dL/du0 (n) and
 * *g_nu = dL/dnu.  The forward states are recomputed from checkpoints taken
 * every `seg` steps (seg <= 0: one segment holding every state).  The spatial
 * loops use `threads` OpenMP threads; g_u0 does not depend on the thread
 * count, *g_nu only through the double-double rounding (see above).
 */
int oracle_ks_adjoint_f64(const double* u0, int64_t n, double dx, double dt, double nu, int64_t nsteps,
                          const double* gT, double* g_u0, double* g_nu, int64_t seg, double* g_nu_abs, int threads) {
  if (!u0 || !gT || !g_u0 || !g_nu || n < 5 || nsteps < 0) return -1;
  if (seg <= 0 || seg > nsteps) seg = nsteps > 0 ? nsteps : 1;
  if (threads < 1) threads = 1;
  const ks_consts_f64 k = ks_make_consts_f64(dx, dt, nu);
  const double idx2 = 1.0 / (dx * dx);
  const double k4 = idx2 * idx2;
  const double ca2 = 2.0 * k.ca;
  const double mdt = -dt, mdth = -0.5 * dt;
  const int64_t nck = (nsteps + seg - 1) / seg + 1;
  double* ck = (double*)malloc((size_t)(nck * n) * sizeof(double));      /* checkpoints u^{c*seg} */
  double* tape_u = (double*)malloc((size_t)(seg * n) * sizeof(double));  /* u^m in a segment */
  double* tape_p = (double*)malloc((size_t)(seg * n) * sizeof(double));  /* P^m in a segment */
  double* lam = (double*)malloc((size_t)n * sizeof(double));
  double* mu = (double*)malloc((size_t)n * sizeof(double));
  double* cur = (double*)malloc((size_t)n * sizeof(double));
  oracle_dd* part = (oracle_dd*)calloc((size_t)threads, sizeof(oracle_dd));   /* per-thread dL/dnu */
  double* part_abs = (double*)calloc((size_t)threads, sizeof(double));         /* per-thread condition */
  if (!ck || !tape_u || !tape_p || !lam || !mu || !cur || !part || !part_abs) {
    free(ck); free(tape_u); free(tape_p); free(lam); free(mu); free(cur); free(part); free(part_abs);
    return -2;
  }
  /* forward sweep keeping checkpoints */
  memcpy(cur, u0, (size_t)n * sizeof(double));
  for (int64_t m = 0; m < nsteps; ++m) {
    if (m % seg == 0) memcpy(ck + (m / seg) * n, cur, (size_t)n * sizeof(double));
    ks_step_f64(cur, mu, n, &k, threads);
  }
  memcpy(lam, gT, (size_t)n * sizeof(double));
  const int64_t nseg = (nsteps + seg - 1) / seg;
  for (int64_t s = nseg - 1; s >= 0; --s) {
    const int64_t m0 = s * seg;
    const int64_t m1 = (m0 + seg < nsteps) ? m0 + seg : nsteps;
    /* recompute the segment's forward states */
    memcpy(cur, ck + s * n, (size_t)n * sizeof(double));
    for (int64_t m = m0; m < m1; ++m) {
      double* tu = tape_u + (m - m0) * n;
      double* tp = tape_p + (m - m0) * n;
      memcpy(tu, cur, (size_t)n * sizeof(double));
      int64_t i;
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
      for (i = 0; i < n; ++i) tp[i] = fma(k.mdth, ks_g_f64(cur, i, n, k.ca, k.c2, k.c4), cur[i]);
#pragma omp parallel for num_threads(threads) schedule(static) if (threads > 1)
      for (i = 0; i < n; ++i) cur[i] = fma(k.mdt, ks_g_f64(tp, i, n, k.ca, k.c2, k.c4), cur[i]);
    }
    /* reverse through the segment */
    for (int64_t m = m1 - 1; m >= m0; --m) {
      const double* tu = tape_u + (m - m0) * n;
      const double* tp = tape_p + (m - m0) * n;
#pragma omp parallel num_threads(threads) if (threads > 1)
      {
#ifdef _OPENMP
        const int t = omp_get_thread_num();
#else
        const int t = 0;
#endif
        int64_t j;
        oracle_dd acc_t = part[t];  /* thread-local copies: no false sharing in the loop */
        double abs_t = part_abs[t];
#pragma omp for schedule(static)
        for (j = 0; j < n; ++j) mu[j] = k.mdt * ks_gT(lam, tp, j, n, ca2, k.c2, k.c4);
        /* (implicit barrier: mu is complete before it is read by the stencil) */
#pragma omp for schedule(static)
        for (j = 0; j < n; ++j) {
          acc_t = dd_add(acc_t, dd_prod4(mdt, lam[j], k4, ks_d4(tp, j, n)));
          acc_t = dd_add(acc_t, dd_prod4(mdth, mu[j], k4, ks_d4(tu, j, n)));
          abs_t += dt * fabs(lam[j]) * k4 * ks_d4_abs(tp, j, n);
          abs_t += (0.5 * dt) * fabs(mu[j]) * k4 * ks_d4_abs(tu, j, n);
          /* lam is read by the stencil, so compute into cur and copy back */
          cur[j] = fma(k.mdth, ks_gT(mu, tu, j, n, ca2, k.c2, k.c4), lam[j] + mu[j]);
        }
        part[t] = acc_t;
        part_abs[t] = abs_t;
      }
      memcpy(lam, cur, (size_t)n * sizeof(double));
    }
  }
  memcpy(g_u0, lam, (size_t)n * sizeof(double));
  oracle_dd acc = {0.0, 0.0};
  double acc_abs = 0.0;
  for (int t = 0; t < threads; ++t) {
    acc = dd_add(acc, part[t]);
    acc_abs += part_abs[t];
  }
  *g_nu = acc.hi + acc.lo;
  if (g_nu_abs) *g_nu_abs = acc_abs;
  free(ck); free(tape_u); free(tape_p); free(lam); free(mu); free(cur); free(part); free(part_abs);
  return 0;
}

/*
 * Heat (FTCS), FP64.  Forward T' = fma(Fo, T_{i+1} + T_{i-1}, c1 T_i) is linear
 * with a symmetric stencil, so the reverse step applies the same update to lam:
 *   lam_j = fma(Fo, lam'_{j+1} + lam'_{j-1}, c1 lam'_j)
 * (mirror boundaries: the transpose of "ghost -1 reads cell 0" adds the ghost's
 * weight back onto cell 0, which is again the mirror update).
 * dL/dalpha = sum_m sum_i lam'_i (dt/dx^2) (T_{i+1} + T_{i-1} - 2 T_i)^m, and its
 * condition sum_m sum_i |lam'_i| (dt/dx^2) (|T_{i+1}| + |T_{i-1}| + 2 |T_i|)^m.
 */
int oracle_heat_adjoint_f64(const double* u0, int64_t n, double dx, double dt, double alpha, int bc,
                            int64_t nsteps, const double* gT, double* g_u0, double* g_alpha, double* g_alpha_abs) {
  if (!u0 || !gT || !g_u0 || !g_alpha || n < 3 || nsteps < 0 || (bc != OR_BC_PERIODIC && bc != OR_BC_MIRROR))
    return -1;
  const double fo_d = (alpha * dt) / (dx * dx);
  const double fo = fo_d, c1 = 1.0 - 2.0 * fo_d;
  const double kk = dt / (dx * dx);
  double* tape = (double*)malloc((size_t)((nsteps + 1) * n) * sizeof(double));
  double* lam = (double*)malloc((size_t)n * sizeof(double));
  double* nxt = (double*)malloc((size_t)n * sizeof(double));
  if (!tape || !lam || !nxt) { free(tape); free(lam); free(nxt); return -2; }
  memcpy(tape, u0, (size_t)n * sizeof(double));
  for (int64_t m = 0; m < nsteps; ++m) heat_step_f64(tape + m * n, tape + (m + 1) * n, n, fo, c1, bc, 1);
  memcpy(lam, gT, (size_t)n * sizeof(double));
  long double acc = 0.0L, acc_abs = 0.0L;
  for (int64_t m = nsteps - 1; m >= 0; --m) {
    const double* T = tape + m * n;
    for (int64_t i = 0; i < n; ++i) {
      const long double tp = (long double)T[nb_index(i + 1, n, bc, NULL)];
      const long double tm = (long double)T[nb_index(i - 1, n, bc, NULL)];
      acc += (long double)lam[i] * (long double)kk * ((tp + tm) - 2.0L * (long double)T[i]);
      acc_abs += fabsl((long double)lam[i]) * (long double)kk * (fabsl(tp) + fabsl(tm) + 2.0L * fabsl((long double)T[i]));
    }
    heat_step_f64(lam, nxt, n, fo, c1, bc, 1);
    memcpy(lam, nxt, (size_t)n * sizeof(double));
  }
  memcpy(g_u0, lam, (size_t)n * sizeof(double));
  *g_alpha = (double)acc;
  if (g_alpha_abs) *g_alpha_abs = (double)acc_abs;
  free(tape); free(lam); free(nxt);
  return 0;
}

/* Threads OpenMP will use for `threads` requests (1 when built without OpenMP). */
int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
