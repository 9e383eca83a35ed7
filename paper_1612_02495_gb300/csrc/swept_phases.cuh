// The work of one block in one swept pass, written once over an execution
// context `Cx`.  The CUDA kernels instantiate it with a device context (real
// arithmetic in shared memory, __syncthreads between tiers); the host-side
// schedule checker instantiates it with a symbolic context that tracks which
// (point, sub-timestep) every buffer cell holds.
//
// Context interface (all indices local to the block's window unless noted):
//   for_range(lo, hi, f)           f(i) for i in [lo, hi), spread over the block
//   sync()                         block-wide barrier
//   load_u(row, c, j, x)           window[row][c][j] = u[c][x mod N]
//   store_u(row, c, j, x)          u[c][x mod N] = window[row][c][j]
//   load_edge(row, c, j, e)        window[row][c][j] = edges_in[e]
//   store_edge(row, c, j, e)       edges_out[e] = window[row][c][j]
//   level(s, base, lo, hi, origin, wall)
//                                  compute sub-timestep (base + s) on [lo, hi)
//                                  into row s&1 from row (s-1)&1 (and row s&1
//                                  for the second stage), then sync
//   kSlab (optional, with member `sl`)
//                                  the context runs one slab of a grid split
//                                  over ranks: edge indices go to the slab's
//                                  own slots (slab_slot)
#pragma once
#include <type_traits>

#include "swept_geom.cuh"

namespace swept {

template <class Cx, class = void>
struct is_slab_ctx : std::false_type {};
template <class Cx>
struct is_slab_ctx<Cx, std::enable_if_t<Cx::kSlab>> : std::true_type {};

// offset of an edge value of `tile` (edge_index), in the context's edge buffers
template <class Cx>
SW_HD int64_t edge_at(const Cx& cx, const Geom& g, int64_t tile, int side, int s, int c, int k) {
  if constexpr (is_slab_ctx<Cx>::value)
    return edge_index(g, slab_slot(g, cx.sl, tile), side, s, c, k);
  else
    return edge_index(g, tile, side, s, c, k);
}
// offset of flat-top value k of component c (top_index), in the context's edge buffers
template <class Cx>
SW_HD int64_t top_at(const Cx& cx, const Geom& g, int c, int k) {
  if constexpr (is_slab_ctx<Cx>::value)
    return cx.sl.ns * (int64_t)g.E + (int64_t)c * g.X + k;
  else
    return top_index(g, c, k);
}

// f(s) for the tiers s = 1..n in order, two per trip: with a stage count that
// is a compile-time constant (two-stage schemes alternate stages), each call's
// stage is then a constant the compiler can fold.
template <class F>
SW_HD void for_tiers(int n, F&& f) {
  int s = 1;
  for (; s + 1 <= n; s += 2) {
    f(s);
    f(s + 1);
  }
  if (s <= n) f(s);
}

// Up-triangle (pass 0, Fig. SweptPseudo) or, with hh < h, the trapezoid that
// starts the remainder: load tile b from u, compute tiers 1..hh, export the
// 2R edge values of tiers 0..hh-1 on both sides; with write_top, also write
// tier hh (the trapezoid's top, non-empty when hh < h) back to u.  The wide
// last tile (X > 0) is a trapezoid even at hh = h; without write_top it
// exports its flat top (tier h) to the flat-top slot of edges_out.
template <class Cx>
SW_HD void run_up(Cx& cx, const Geom& g_in, int64_t b, int hh, bool write_top) {
  const Geom g = fixed_geom<Cx>(g_in);
  const int w = tile_width(g, b);
  const int64_t x0 = b * (int64_t)g.W;
  const int64_t origin = x0 - g.R;
  cx.for_range(0, w * g.C, [&](int i) {
    const int c = g.C == 1 ? 0 : i / w, k = i - c * w;
    cx.load_u(0, c, g.R + k, x0 + k);
  });
  cx.sync();
  for_tiers(hh, [&](int s) { cx.level(s, 0, g.R + g.R * s, g.R + w - g.R * s, origin, NO_WALL); });
  const int per_level = g.C * 2 * g.R;
  const int per_side = hh * per_level;
  cx.for_range(0, 2 * per_side, [&](int i) {
    const int side = i >= per_side ? 1 : 0;
    const int rem = i - side * per_side;
    const int s = rem / per_level;
    const int c = (rem - s * per_level) / (2 * g.R);
    const int k = rem % (2 * g.R);
    cx.store_edge(s & 1, c, edge_pos(g, side, s, k, w), edge_at(cx, g, b, side, s, c, k));
  });
  if (write_top) {
    const int lo = g.R + g.R * hh, tw = w - 2 * g.R * hh;
    if (tw > 0)
      cx.for_range(0, tw * g.C, [&](int i) {
        const int c = g.C == 1 ? 0 : i / tw, k = i - c * tw;
        cx.store_u(hh & 1, c, lo + k, origin + lo + k);
      });
  } else if (w > g.W && hh == g.h) {
    const int lo = g.R + g.W / 2;
    cx.for_range(0, g.X * g.C, [&](int i) {
      const int c = g.C == 1 ? 0 : i / g.X, k = i - c * g.X;
      cx.store_edge(g.h & 1, c, lo + k, top_at(cx, g, c, k));
    });
  }
}

// Diamond pass p >= 1 for block b (odd = p & 1): insert the neighbouring
// tiles' edges (Fig. extraction), grow the complementary triangle for hh tiers.
//   MODE_DIAMOND: then shrink the new tile (tiers 1..h-1 relative to it) and
//                 export its edges to tile slot b of edges_out;
//   MODE_DOWN:    write the completed tier h of the new tile to u (the only
//                 point where a full tier exists, Section "First-order");
//   MODE_GAP:     hh < h, write the grown gap [c - R hh, c + R hh) of tier hh
//                 (completes the remainder trapezoids).
// Block nt - 1 of a diamond or down pass on a grid with X > 0 owns the wide
// tile: it also inserts the previous pass's flat top (tier h) beside its
// diamond, and in MODE_DIAMOND shrinks through tier h and exports the new
// flat top.
template <class Cx>
SW_HD void run_diamond(Cx& cx, const Geom& g_in, int64_t b, int odd, int mode, int hh) {
  const Geom g = fixed_geom<Cx>(g_in);
  const bool wide = g.X > 0 && b == g.nt - 1 && mode != MODE_GAP;
  const int w = wide ? g.W + g.X : g.W;  // width of this block's tile
  const int dofs = wide && odd ? g.X : 0;  // the diamond's offset inside the tile (flat top on its left)
  // first point of the block's tile: odd passes shift the tiling right by W/2;
  // a gap window is the plain window around boundary (b + 1) W (N for b = nt - 1)
  const int64_t t0 = b * (int64_t)g.W + (odd ? g.W / 2 : 0) + (odd && !wide && b == g.nt - 1 ? g.X : 0);
  const int64_t origin = t0 - g.R;
  const int64_t tl = left_tile(g, odd, b);
  const int64_t tr = right_tile(g, odd, b);
  const int per_level = g.C * 2 * g.R;
  const int per_side = hh * per_level;
  cx.for_range(0, 2 * per_side, [&](int i) {
    const int which = i >= per_side ? 1 : 0;  // 0: right edges of the left tile, 1: left edges of the right tile
    const int rem = i - which * per_side;
    const int s = rem / per_level;
    const int cc = (rem - s * per_level) / (2 * g.R);
    const int k = rem % (2 * g.R);
    const int side = which == 0 ? 1 : 0;
    const int64_t tile = which == 0 ? tl : tr;
    cx.load_edge(s & 1, cc, dofs + insert_pos(g, side, s, k), edge_at(cx, g, tile, side, s, cc, k));
  });
  if (wide) {
    const int lo = odd ? g.R : g.R + g.W;
    cx.for_range(0, g.X * g.C, [&](int i) {
      const int cc = g.C == 1 ? 0 : i / g.X, k = i - cc * g.X;
      cx.load_edge(g.h & 1, cc, lo + k, top_at(cx, g, cc, k));
    });
  }
  cx.sync();
  const int wall = window_wall(g, origin, w + 2 * g.R);
  for_tiers(hh, [&](int s) { cx.level(s, 0, dofs + grow_lo(g, s), dofs + grow_hi(g, s), origin, wall); });
  if (mode == MODE_DIAMOND) {
    const int top = wide ? g.h : g.h - 1;  // a triangle's tier h is empty; a wide tile's is its flat top
    for_tiers(top, [&](int s) { cx.level(s, g.h, g.R + g.R * s, g.R + w - g.R * s, origin, wall); });
    const int per_side_h = g.h * per_level;
    cx.for_range(0, 2 * per_side_h, [&](int i) {
      const int side = i >= per_side_h ? 1 : 0;
      const int rem = i - side * per_side_h;
      const int s = rem / per_level;
      const int cc = (rem - s * per_level) / (2 * g.R);
      const int k = rem % (2 * g.R);
      cx.store_edge(s & 1, cc, edge_pos(g, side, s, k, w), edge_at(cx, g, b, side, s, cc, k));
    });
    if (wide) {
      const int lo = g.R + g.W / 2;
      cx.for_range(0, g.X * g.C, [&](int i) {
        const int cc = g.C == 1 ? 0 : i / g.X, k = i - cc * g.X;
        cx.store_edge(g.h & 1, cc, lo + k, top_at(cx, g, cc, k));
      });
    }
  } else if (mode == MODE_DOWN) {
    cx.for_range(0, w * g.C, [&](int i) {
      const int cc = g.C == 1 ? 0 : i / w, k = i - cc * w;
      cx.store_u(g.h & 1, cc, g.R + k, origin + g.R + k);
    });
  } else {
    const int lo = grow_lo(g, hh), gw = grow_hi(g, hh) - lo;
    cx.for_range(0, gw * g.C, [&](int i) {
      const int cc = g.C == 1 ? 0 : i / gw, k = i - cc * gw;
      cx.store_u(hh & 1, cc, lo + k, origin + lo + k);
    });
  }
}

// The persistent form of the launch sequence below: item (layer kp, tile b),
// item = kp * nt + b, runs launch kp's work for block b.  Before it runs it
// waits until each tile tile[i] has completed layer need[i] (a tile's layers
// complete in order, each one waiting for the tile's previous layer); this
// returns how many such inputs the item has (0..3).  The zig-zag makes a
// diamond depend on the two tiles it reads; the remainder trapezoid reads the
// state the down-triangle wrote over its tile (tiles b-1, b, b+1 cover every
// case); the gap pass reads the edges of the two trapezoids beside it.
SW_HD int persist_deps(const Geom& g, int64_t n_sub, int kp, int64_t b, int64_t* tile, int* need) {
  const int64_t q = n_sub / g.h;
  const int rem = (int)(n_sub % g.h);
  const int main_passes = q > 0 ? (int)q + 1 : 0;
  if (kp > 0 && kp < main_passes) {
    tile[0] = left_tile(g, kp & 1, b);
    tile[1] = right_tile(g, kp & 1, b);
    need[0] = need[1] = kp - 1;
    return 2;
  }
  if (kp == main_passes && q > 0 && rem > 0) {
    tile[0] = (b + g.nt - 1) % g.nt;
    tile[1] = b;
    tile[2] = (b + 1) % g.nt;
    need[0] = need[1] = need[2] = (int)q;
    return 3;
  }
  if (kp == main_passes + 1 && rem > 0) {
    tile[0] = b;
    tile[1] = (b + 1) % g.nt;
    need[0] = need[1] = main_passes;
    return 2;
  }
  return 0;
}

// The launch sequence for n_sub sub-timesteps: q = n_sub / h full passes
// (up, q-1 diamonds, down) and, for rem = n_sub % h, an up-trapezoid and a
// gap pass.  `emit(kind, odd, mode, hh, pass)` is called once per launch:
//   kind 0 = up (run_up), kind 1 = diamond (run_diamond).
// The edge buffer written by pass k is k & 1 (ping-pong); the remainder pair
// uses buffer 0 -> read by its gap pass.
template <class F>
inline void for_each_launch(const Geom& g, int64_t n_sub, F emit) {
  const int64_t q = n_sub / g.h;
  const int rem = (int)(n_sub % g.h);
  if (q > 0) {
    emit(0, 0, MODE_DIAMOND, g.h, (int64_t)0);
    for (int64_t p = 1; p < q; ++p) emit(1, (int)(p & 1), MODE_DIAMOND, g.h, p);
    emit(1, (int)(q & 1), MODE_DOWN, g.h, q);
  }
  if (rem > 0) {
    emit(0, 0, MODE_GAP, rem, (int64_t)-1);
    emit(1, 1, MODE_GAP, rem, (int64_t)-2);
  }
}

}  // namespace swept
