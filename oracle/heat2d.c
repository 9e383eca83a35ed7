/*
 * CPU oracle for the 2D heat equation solved with the 2D swept decomposition.
 *
 * TEST INFRASTRUCTURE ONLY.  Like swept_oracle.c, this file is the plain
 * definition the GPU path is checked against.  Only tests/ and bench.py's
 * CPU-baseline leg load it.  It shares no code, header or constant with the
 * product library.
 *
 * The paper solves 1D problems and names two dimensions as future work
 * (Section "Conclusion").  The 2D problem here is the direct extension of its
 * heat test case, Eq. HeatDisc, to a square-celled nx x ny grid (a reading):
 *
 *   T'_{i,j} = Fo (T_{i-1,j} + T_{i+1,j} + T_{i,j-1} + T_{i,j+1}) + (1 - 4 Fo) T_{i,j},
 *   Fo = alpha dt / dx^2 (stable for Fo <= 1/4),
 *
 * stored row-major, u[j * nx + i] with i along x.  Evaluation order (fixed, the
 * GPU path evaluates the same one):
 *   sx = T_{i-1,j} + T_{i+1,j};  sy = T_{i,j-1} + T_{i,j+1};  s = sx + sy;
 *   T' = fma(Fo, s, c1 * T_{i,j}),  c1 = 1 - 4 Fo computed in double, then rounded.
 *
 * Boundaries per axis, as in the 1D oracle: 0 = periodic, 1 = mirror walls at
 * -1/2 and n - 1/2 (insulated).
 *
 * Compile in ISO C with -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* index of neighbour j (may lie outside [0, n)) after the boundary rule */
static inline int64_t h2_index(int64_t j, int64_t n, int bc) {
  if (j >= 0 && j < n) return j;
  if (bc == 0) {
    int64_t r = j % n;
    return r < 0 ? r + n : r;
  }
  return j < 0 ? -1 - j : 2 * n - 1 - j;
}

#define H2_BODY(REAL, SFX, FMA)                                                                           \
  int oracle_heat2d_run_##SFX(REAL* u, int64_t nx, int64_t ny, double dx, double dt, double alpha, int bc,  \
                              int64_t nsteps, int threads) {                                                \
    if (!u || nx < 1 || ny < 1 || !(dx > 0) || !(dt > 0) || nsteps < 0 || (bc != 0 && bc != 1)) return 1; \
    const double fo_d = alpha * dt / (dx * dx);                                                             \
    const REAL fo = (REAL)fo_d;                                                                             \
    const REAL c1 = (REAL)(1.0 - 4.0 * fo_d);                                                               \
    const int64_t n = nx * ny;                                                                              \
    REAL* v = (REAL*)malloc((size_t)n * sizeof(REAL));                                                      \
    if (!v) return 2;                                                                                       \
    (void)threads;                                                                                          \
    for (int64_t m = 0; m < nsteps; ++m) {                                                                  \
      int64_t j;                                                                                            \
      _Pragma("omp parallel for num_threads(threads > 0 ? threads : 1) schedule(static)")                   \
      for (j = 0; j < ny; ++j) {                                                                            \
        const int64_t js = h2_index(j - 1, ny, bc), jn = h2_index(j + 1, ny, bc);                           \
        for (int64_t i = 0; i < nx; ++i) {                                                                  \
          const int64_t iw = h2_index(i - 1, nx, bc), ie = h2_index(i + 1, nx, bc);                         \
          const REAL t = u[j * nx + i];                                                                     \
          const REAL sx = u[j * nx + iw] + u[j * nx + ie];                                                  \
          const REAL sy = u[js * nx + i] + u[jn * nx + i];                                                  \
          const REAL s = sx + sy;                                                                           \
          v[j * nx + i] = FMA(fo, s, c1 * t);                                                               \
        }                                                                                                   \
      }                                                                                                     \
      memcpy(u, v, (size_t)n * sizeof(REAL));                                                               \
    }                                                                                                       \
    free(v);                                                                                                \
    return 0;                                                                                               \
  }

H2_BODY(double, f64, fma)
H2_BODY(float, f32, fmaf)
