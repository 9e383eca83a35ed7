// Host-side plan of a slab solve: a grid split over ranks (one GPU each), each
// rank running blocks [b0, b0 + nb) of every swept pass (Slab, swept_geom.cuh).
// Shared by the runtime (slab.cu) and the host schedule replay (check.cpp), so
// that the replay checks exactly the launches and transfers the runtime uses.
//
// Between two launches a rank trades with its two neighbours only (a ring of
// ranks, for both boundary conditions: with mirror walls the wrapped tile
// holds the two walls' sides, as on one GPU):
//   - before a diamond, down or gap pass: half an edge block, 2R h C values.
//     An odd pass (tiles shifted right by W/2) reads the left edges of the tile
//     right of the slab, so each rank sends the left edges of its first tile
//     to its left neighbour; an even pass reads the right edges of the tile
//     left of the slab, so each rank sends the right edges of its last tile to
//     its right neighbour.  This is the one exchange per half cycle of the
//     swept rule (Section "First-order", Fig. collection), now between GPUs.
//   - after an odd down pass: the new tiles straddle the slab ends, so the
//     W/2 points each rank computed past its end go to the right neighbour;
//     after the remainder's gap pass, the R rem points past its end.
// A rank therefore owns the same points [x0, x1) before and after a solve.
#pragma once
#include <stdint.h>

#include "swept_geom.cuh"
#include "swept_phases.cuh"

namespace swept {

struct LaunchDesc {
  int kind = 0;  // 0 up (run_up), 1 diamond / down / gap (run_diamond)
  int odd = 0;
  int mode = MODE_DIAMOND;
  int hh = 0;
  int64_t pass = 0;  // as for_each_launch: 0..q main passes, -1 up-trapezoid, -2 gap pass
  int ein = 0, eout = 0;
};

inline int64_t launch_total(const Geom& g, int64_t n_sub) {
  const int64_t q = n_sub / g.h, rem = n_sub % g.h;
  return (q > 0 ? q + 1 : 0) + (rem > 0 ? 2 : 0);
}

// launch i of for_each_launch (0 <= i < launch_total)
inline LaunchDesc launch_at(const Geom& g, int64_t n_sub, int64_t i) {
  const int64_t q = n_sub / g.h;
  const int rem = (int)(n_sub % g.h);
  const int64_t main = q > 0 ? q + 1 : 0;
  LaunchDesc d;
  if (i < main) {
    d.pass = i;
    d.hh = g.h;
    if (i == 0) {
      d.kind = 0;
    } else {
      d.kind = 1;
      d.odd = (int)(i & 1);
      d.mode = i == q ? MODE_DOWN : MODE_DIAMOND;
    }
  } else {
    d.hh = rem;
    d.mode = MODE_GAP;
    d.kind = i == main ? 0 : 1;
    d.odd = d.kind;
    d.pass = i == main ? -1 : -2;
  }
  if (d.kind == 0) {
    d.eout = d.pass >= 0 ? (int)(d.pass & 1) : 0;
  } else {
    d.ein = d.pass >= 1 ? (int)((d.pass - 1) & 1) : 0;
    d.eout = d.pass >= 1 ? (int)(d.pass & 1) : 1;
  }
  return d;
}

// at most this many transfers follow one launch: a state message per component (C <= 3) each
// way, then one edge message each way
constexpr int kMaxXfers = 2 * 3 + 2;

// one transfer between neighbouring ranks (the C ABI's swept_slab_xfer)
struct Xfer {
  int peer;    // -1 left neighbour, +1 right neighbour
  int recv;    // 0 send, 1 receive
  int region;  // 0 edge buffer 0, 1 edge buffer 1, 2 state array
  int64_t offset, count;
};

// first point past the slab (N for the last slab)
inline int64_t slab_end(const Geom& g, const Slab& sl) { return tile_start(g, sl.b0 + sl.nb); }

// The slab of rank `rank` of `nranks`: tiles split as evenly as possible.
inline Slab make_slab(const Geom& g, int rank, int nranks) {
  Slab sl;
  sl.b0 = g.nt * rank / nranks;
  sl.nb = g.nt * (rank + 1) / nranks - sl.b0;
  sl.x0 = tile_start(g, sl.b0);
  sl.ul = slab_end(g, sl) - sl.x0 + g.W / 2;
  sl.ns = sl.nb + 2 < g.nt ? sl.nb + 2 : g.nt;
  return sl;
}

// The transfers due after launch i of an n_sub-sub-timestep solve (before
// launch i + 1), in the order a rank posts them; returns how many (<= 2 C + 2 <= kMaxXfers).
// A rank's k-th send to a neighbour matches that neighbour's k-th receive from
// the opposite side.
inline int slab_xfers(const Geom& g, const Slab& sl, int64_t n_sub, int64_t i, Xfer* out) {
  int n = 0;
  const int64_t total = launch_total(g, n_sub);
  if (i < 0 || i >= total) return 0;
  const LaunchDesc cur = launch_at(g, n_sub, i);
  // state past the slab's end, written by an odd down pass or the gap pass
  int64_t m = 0;
  if (cur.kind == 1 && cur.mode == MODE_DOWN && cur.odd) m = g.W / 2;
  if (cur.kind == 1 && cur.mode == MODE_GAP) m = (int64_t)g.R * cur.hh;
  if (m > 0) {
    const int64_t past = slab_end(g, sl) - sl.x0;
    for (int c = 0; c < g.C; ++c) {
      out[n++] = Xfer{+1, 0, 2, c * sl.ul + past, m};
      out[n++] = Xfer{-1, 1, 2, c * sl.ul, m};
    }
  }
  if (i + 1 < total) {
    const LaunchDesc nx = launch_at(g, n_sub, i + 1);
    if (nx.kind == 1) {
      const int64_t half = g.E / 2;
      if (nx.odd) {
        out[n++] = Xfer{-1, 0, nx.ein, slab_slot(g, sl, sl.b0) * g.E, half};
        out[n++] = Xfer{+1, 1, nx.ein, slab_slot(g, sl, (sl.b0 + sl.nb) % g.nt) * g.E, half};
      } else {
        out[n++] = Xfer{+1, 0, nx.ein, slab_slot(g, sl, sl.b0 + sl.nb - 1) * g.E + half, half};
        out[n++] = Xfer{-1, 1, nx.ein, slab_slot(g, sl, (sl.b0 + g.nt - 1) % g.nt) * g.E + half, half};
      }
    }
  }
  return n;
}

}  // namespace swept
