// Per-point stencil operators of the three schemes, in a fixed operation order.
//
// Every floating-point operation is an explicit round-to-nearest intrinsic
// (__fma_rn, __dadd_rn, __dmul_rn, __ddiv_rn, __dsqrt_rn and the float forms),
// so the compiler cannot contract or reorder them; the swept kernels and the
// classic kernels call the same operator, which is what makes the two paths
// agree bit for bit.  Constants are stored and multiplied instead of divided by
// (Section "Results", Fig. divisionComparison).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "swept_geom.cuh"

namespace swept {

__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float div_rn(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
__device__ __forceinline__ float sqrt_rn(float a) { return __fsqrt_rn(a); }
__device__ __forceinline__ double sqrt_rn(double a) { return __dsqrt_rn(a); }

// ---------------------------------------------------------------------------
// Heat, FTCS (Eq. HeatDisc): T' = Fo (T_{i+1} + T_{i-1}) + (1 - 2 Fo) T_i
// order: s = T_{i+1} + T_{i-1};  T' = fma(Fo, s, c1 * T_i)
// ---------------------------------------------------------------------------
template <typename T>
struct HeatOp {
  static constexpr int R = 1, S = 1, C = 1;
  struct K {
    T fo, c1;
  };
  // v[0..2] = T_{i-1}, T_i, T_{i+1} at the previous tier
  template <int STAGE>
  __device__ __forceinline__ static T point(const T* v, T /*prev2*/, const K& k) {
    const T s = add_rn(v[2], v[0]);
    return fma_rn(k.fo, s, mul_rn(k.c1, v[1]));
  }
};

// ---------------------------------------------------------------------------
// Kuramoto-Sivashinsky, Eq. KSDisc (u_i term read as -2 u_i, factor nu on the
// fourth difference), midpoint RK2 (Appendix).  f = -g with
//   sp1 = u_{i+1} + u_{i-1};  sp2 = u_{i+2} + u_{i-2}
//   nl  = fma(u_{i+1}, u_{i+1}, -(u_{i-1} u_{i-1}))
//   d2  = fma(-2, u_i, sp1);  d4 = fma(6, u_i, fma(-4, sp1, sp2))
//   g   = fma(c_4, d4, fma(c_2, d2, c_a nl))
// stage 0 (predictor, odd tiers):  P  = fma(-dt/2, g(u), u_i)
// stage 1 (final, even tiers):     u' = fma(-dt,   g(P), u_i)   u_i from two tiers back
// ---------------------------------------------------------------------------
template <typename T>
struct KsOp {
  static constexpr int R = 2, S = 2, C = 1;
  struct K {
    T ca, c2, c4, mdth, mdt;
  };
  __device__ __forceinline__ static T g(const T* v, const K& k) {
    const T sp1 = add_rn(v[3], v[1]);
    const T sp2 = add_rn(v[4], v[0]);
    const T nl = fma_rn(v[3], v[3], -mul_rn(v[1], v[1]));
    const T d2 = fma_rn(T(-2), v[2], sp1);
    const T d4 = fma_rn(T(6), v[2], fma_rn(T(-4), sp1, sp2));
    return fma_rn(k.c4, d4, fma_rn(k.c2, d2, mul_rn(k.ca, nl)));
  }
  // v[0..4] = u_{i-2} .. u_{i+2} at the previous tier; prev2 = u_i two tiers back
  template <int STAGE>
  __device__ __forceinline__ static T point(const T* v, T prev2, const K& k) {
    if (STAGE == 0) return fma_rn(k.mdth, g(v, k), v[2]);
    return fma_rn(k.mdt, g(v, k), prev2);
  }
};

// ---------------------------------------------------------------------------
// 1D Euler, finite volume (not in the paper): MUSCL-minmod on primitives,
// Rusanov flux, SSP-RK2.  Order (per face i+1/2 from cells i-1..i+2):
//   cell:   u = m / rho;  p = gm1 fma(-(0.5 m), u, E)
//   qL = q_i + 0.5 minmod(q_i - q_{i-1}, q_{i+1} - q_i)
//   qR = q_{i+1} - 0.5 minmod(q_{i+1} - q_i, q_{i+2} - q_{i+1})
//   mX = rhoX uX;  EX = fma(0.5 mX, uX, pX igm1);  cX = sqrt((gamma pX) / rhoX)
//   s  = max(|uL| + cL, |uR| + cR)
//   F  = 0.5 fma(-s, UR - UL, FL + FR),  F = (m, fma(m, u, p), u (E + p))
//   stage 0:  U1 = fma(-dt/dx, F+ - F-, U)
//   stage 1:  t = fma(-dt/dx, F+ - F-, U1);  U' = 0.5 (U + t)
// Across a reflective wall a cell is read as its mirror with u negated.
// ---------------------------------------------------------------------------
// minmod(a, b): the argument of smaller magnitude when a and b are both
// positive or both negative, else 0.  Evaluated on the integer pipe from the
// IEEE bit patterns: for values of one sign, magnitude order is the order of
// the patterns' magnitude fields, and with equal sign bits a <= b (both
// positive) and a >= b (both negative) are both "bits(a) <= bits(b)" as signed
// integers.  The selection equals the comparison form for every non-NaN input
// (signed zeros, subnormals, infinities included), without spending FP64 issue
// slots on sign tests and compares.
__device__ __forceinline__ double minmod(double a, double b) {
  const long long ia = __double_as_longlong(a), ib = __double_as_longlong(b);
  const long long mag = 0x7fffffffffffffffLL;
  const bool same_sign_nonzero = ((ia ^ ib) >= 0) && (ia & mag) != 0 && (ib & mag) != 0;
  return same_sign_nonzero ? (ia <= ib ? a : b) : 0.0;
}
__device__ __forceinline__ float minmod(float a, float b) {
  const int ia = __float_as_int(a), ib = __float_as_int(b);
  const int mag = 0x7fffffff;
  const bool same_sign_nonzero = ((ia ^ ib) >= 0) && (ia & mag) != 0 && (ib & mag) != 0;
  return same_sign_nonzero ? (ia <= ib ? a : b) : 0.0f;
}
// the larger of two non-negative values, by their bit patterns (same rule)
__device__ __forceinline__ double max_nonneg(double a, double b) {
  return __double_as_longlong(a) >= __double_as_longlong(b) ? a : b;
}
__device__ __forceinline__ float max_nonneg(float a, float b) { return __float_as_int(a) >= __float_as_int(b) ? a : b; }

template <typename T>
struct EulerOp {
  static constexpr int R = 2, S = 2, C = 3;
  struct K {
    T gamma, gm1, igm1, mdtdx;
  };
  struct Prim {
    T r, u, p;
  };
  __device__ __forceinline__ static Prim prim(T r, T m, T e, const K& k) {
    Prim w;
    w.r = r;
    w.u = div_rn(m, r);
    w.p = mul_rn(k.gm1, fma_rn(-mul_rn(T(0.5), m), w.u, e));
    return w;
  }
  // One side of a face: the MUSCL-minmod reconstructed state with its
  // momentum, energy and wave-speed bound.  Left side from cells a, b, c
  // (value at the right end of b), right side from b, c, d (left end of c).
  struct Side {
    T r, u, p, m, E, sp;
  };
  __device__ __forceinline__ static void finish_side(Side& X, const K& k) {
    X.m = mul_rn(X.r, X.u);
    X.E = fma_rn(mul_rn(T(0.5), X.m), X.u, mul_rn(X.p, k.igm1));
    const T c = sqrt_rn(div_rn(mul_rn(k.gamma, X.p), X.r));
    X.sp = add_rn(fabs(X.u), c);
  }
  __device__ __forceinline__ static Side left_side(const Prim& a, const Prim& b, const Prim& c, const K& k) {
    Side L;
    L.r = add_rn(b.r, mul_rn(T(0.5), minmod(sub_rn(b.r, a.r), sub_rn(c.r, b.r))));
    L.u = add_rn(b.u, mul_rn(T(0.5), minmod(sub_rn(b.u, a.u), sub_rn(c.u, b.u))));
    L.p = add_rn(b.p, mul_rn(T(0.5), minmod(sub_rn(b.p, a.p), sub_rn(c.p, b.p))));
    finish_side(L, k);
    return L;
  }
  __device__ __forceinline__ static Side right_side(const Prim& b, const Prim& c, const Prim& d, const K& k) {
    Side R;
    R.r = sub_rn(c.r, mul_rn(T(0.5), minmod(sub_rn(c.r, b.r), sub_rn(d.r, c.r))));
    R.u = sub_rn(c.u, mul_rn(T(0.5), minmod(sub_rn(c.u, b.u), sub_rn(d.u, c.u))));
    R.p = sub_rn(c.p, mul_rn(T(0.5), minmod(sub_rn(c.p, b.p), sub_rn(d.p, c.p))));
    finish_side(R, k);
    return R;
  }
  // Rusanov flux from the two sides: 1/2 (F(L) + F(R)) - 1/2 s (U_R - U_L),
  // s = the larger of |u| + c over the two sides
  // sp = |u| + c >= 0 on both sides
  __device__ __forceinline__ static T smax(const Side& L, const Side& R) { return max_nonneg(L.sp, R.sp); }
  __device__ __forceinline__ static T flux0(const Side& L, const Side& R, T s) {
    return mul_rn(T(0.5), fma_rn(-s, sub_rn(R.r, L.r), add_rn(L.m, R.m)));
  }
  __device__ __forceinline__ static T flux1(const Side& L, const Side& R, T s) {
    return mul_rn(T(0.5), fma_rn(-s, sub_rn(R.m, L.m), add_rn(fma_rn(L.m, L.u, L.p), fma_rn(R.m, R.u, R.p))));
  }
  __device__ __forceinline__ static T flux2(const Side& L, const Side& R, T s) {
    return mul_rn(T(0.5),
                  fma_rn(-s, sub_rn(R.E, L.E), add_rn(mul_rn(L.u, add_rn(L.E, L.p)), mul_rn(R.u, add_rn(R.E, R.p)))));
  }
  // Rusanov flux through the face between cells b and c, from cells a, b, c, d
  __device__ __forceinline__ static void flux(const Prim& a, const Prim& b, const Prim& c, const Prim& d, const K& k,
                                              T& F0, T& F1, T& F2) {
    const Side L = left_side(a, b, c, k);
    const Side R = right_side(b, c, d, k);
    const T s = smax(L, R);
    F0 = flux0(L, R, s);
    F1 = flux1(L, R, s);
    F2 = flux2(L, R, s);
  }
  template <int STAGE>
  __device__ __forceinline__ static T update(T fp, T fm, T in_self, T prev2, const K& k) {
    if (STAGE == 0) return fma_rn(k.mdtdx, sub_rn(fp, fm), in_self);
    const T t = fma_rn(k.mdtdx, sub_rn(fp, fm), in_self);
    return mul_rn(T(0.5), add_rn(prev2, t));
  }
};

// ---------------------------------------------------------------------------
// Discrete adjoints (not in the paper): the exact transposes of the forward
// operation sequence, run backwards in time as the same two-stage, radius-r
// stencil, with the forward state of each tier read from a tape.
//
// KS, reverse of one step m (lam' = dL/du^{m+1}):
//   gT(lam; w)_j = fma(c_4, d4, fma(c_2, d2, (2 c_a w_j)(lam_{j-1} - lam_{j+1})))
//     with sp1, sp2, d2, d4 of lam as in the forward operator
//   stage 0:  mu  = -dt gT(lam'; P^m)                       (odd reverse tiers)
//   stage 1:  lam = fma(-dt/2, gT(mu; u^m), lam' + mu)      (even reverse tiers)
// dL/dnu = sum -dt k4 lam'_j d4(P^m)_j - (dt/2) k4 mu_j d4(u^m)_j, accumulated as
// the equal sums -dt k4 d4(lam')_j P^m_j and -(dt/2) k4 d4(mu)_j u^m_j (the
// periodic fourth difference is symmetric), so the d4 already computed in gT
// is reused.
// ---------------------------------------------------------------------------
// Compensated (Kahan) accumulation of the parameter derivative: the error is
// about 2 eps sum|terms|, independent of the number of terms; the value is
// the double-double (s, -c).
struct KahanAcc {
  double s = 0.0, c = 0.0;
  __device__ __forceinline__ void add(double x) {
    const double y = __dsub_rn(x, c);
    const double t = __dadd_rn(s, y);
    c = __dsub_rn(__dsub_rn(t, s), y);
    s = t;
  }
};

template <typename T>
struct KsAdjOp {
  static constexpr int R = 2, S = 2, C = 1;
  struct K {
    T ca2, c2, c4, mdt, mdth, mdtk4, mdthk4;
  };
  // v[0..4] = lam_{j-2} .. lam_{j+2}; w = forward state at j; d4 returned for dnu
  __device__ __forceinline__ static T gT(const T* v, T w, const K& k, T& d4) {
    const T sp1 = add_rn(v[3], v[1]);
    const T sp2 = add_rn(v[4], v[0]);
    const T dl = sub_rn(v[1], v[3]);
    const T nl = mul_rn(mul_rn(k.ca2, w), dl);
    const T d2 = fma_rn(T(-2), v[2], sp1);
    d4 = fma_rn(T(6), v[2], fma_rn(T(-4), sp1, sp2));
    return fma_rn(k.c4, d4, fma_rn(k.c2, d2, nl));
  }
  template <int STAGE>
  __device__ __forceinline__ static T point(const T* v, T prev2, T w, const K& k, KahanAcc& acc) {
    T d4;
    const T g = gT(v, w, k, d4);
    if (STAGE == 0) {
      acc.add((double)mul_rn(mul_rn(k.mdtk4, d4), w));
      return mul_rn(k.mdt, g);
    }
    acc.add((double)mul_rn(mul_rn(k.mdthk4, d4), w));
    return fma_rn(k.mdth, g, add_rn(prev2, v[2]));
  }
};

// Heat: FTCS is linear with a symmetric stencil, so the reverse step is the
// forward update applied to lam:  lam_j = fma(Fo, lam'_{j+1} + lam'_{j-1}, c1 lam'_j).
// dL/dalpha = sum (dt/dx^2) lam'_j (T_{j+1} + T_{j-1} - 2 T_j)^m, accumulated as
// the equal sum (dt/dx^2) (lam'_{j+1} + lam'_{j-1} - 2 lam'_j) T^m_j.
template <typename T>
struct HeatAdjOp {
  static constexpr int R = 1, S = 1, C = 1;
  struct K {
    T fo, c1, kk;
  };
  template <int STAGE>
  __device__ __forceinline__ static T point(const T* v, T /*prev2*/, T w, const K& k, KahanAcc& acc) {
    const T s = add_rn(v[2], v[0]);
    acc.add((double)mul_rn(mul_rn(k.kk, fma_rn(T(-2), v[1], s)), w));
    return fma_rn(k.fo, s, mul_rn(k.c1, v[1]));
  }
};

}  // namespace swept
