// Index arithmetic of the swept rule (shared by the CUDA kernels and the
// host-side schedule checker, so the checker replays exactly what the kernels do).
//
// Swept rule (Magee & Niemeyer, Section "First-order", Figs. firstorder and
// collection; Section "Second-order extended stencil", Fig. secondordersolution):
//   - a tile ("node") of W points is advanced as a triangle: sub-timestep s is
//     computed on the points whose radius-R stencil at s-1 is still inside the
//     tile, i.e. the tile shrinks by R on each side per sub-timestep;
//   - the 2R values at each end of every tier are the "edges" written to the
//     global left/right arrays; a tier's values survive in a two-row buffer
//     (even tiers in row 0, odd tiers in row 1) because the interior of row
//     s&1 is overwritten only by tier s+2, which is narrower by 2R per side;
//   - the next pass centres a block on each tile boundary c, re-inserts the
//     left tile's right edges and the right tile's left edges, grows the
//     complementary triangle on [c - R s, c + R s) up to s = h = W/(2R), where
//     it spans a whole tile shifted by W/2, and then shrinks that tile again;
//   - passes alternate between boundaries at (b+1) W (odd pass: tiles move
//     right by W/2) and b W + W/2 (even pass: tiles move back), the zig-zag.
// Local coordinates: a block's window is W + 2R points; a tile sits at
// local [R, W + R); a diamond window centred on c sits at global
// [c - W/2 - R, c + W/2 + R).
//
// Grids that are not a multiple of W (the problem statement fixes only a grid
// of n points): the last tile, nt - 1, is wider by X = n - nt W points
// (0 < X < W).  Its triangle cannot close, so it is a trapezoid whose top
// (X points at tier h, the "flat top") is complete at the end of the pass.
// Every pass hands that flat top to block nt - 1 of the next pass (one more
// slot, index nt, in the edge buffers), whose tile is then the W-wide diamond
// plus the flat top: on the left of the diamond in odd passes (the tiling
// shifted right by W/2), on its right in even passes.  The shrink of a wide
// tile stops at tier h with a new flat top in the middle of the tile.  All
// diamonds keep height h, so the zig-zag is unchanged; only block nt - 1 of
// every up, diamond and down pass does the extra X points per tier.  The
// remainder's gap passes are plain W windows around the tile boundaries.
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define SW_HD __host__ __device__ __forceinline__
#else
#define SW_HD inline
#endif

namespace swept {

constexpr int NO_WALL = -(1 << 30);

enum PassMode : int { MODE_DIAMOND = 0, MODE_DOWN = 1, MODE_GAP = 2 };

struct Geom {
  int64_t N;   // grid points
  int64_t nt;  // tiles, N / W
  int W;       // tile width
  int R;       // stencil radius of one sub-timestep
  int S;       // sub-timesteps (stages) per timestep
  int C;       // values per point
  int h;       // W / (2R): sub-timesteps per pass
  int M;       // W + X + 2R: window width (the row stride; W + 2R when X = 0)
  int E;       // values per tile in an edge buffer: 2 sides * h * C * 2R
  int bc;      // 0 periodic, 1 mirror walls at -1/2 and N-1/2
  int chunk;   // consecutive points one thread advances per tier (1 = strided mapping)
  int P = 0;   // tiers in registers: points per lane of the one warp that owns a tile (0 = in shared memory)
  int X = 0;   // extra width of the last tile (N - nt W, 0 <= X < W)
};

// edge-buffer slots per buffer: one per tile, plus the flat-top slot when X > 0
SW_HD int64_t edge_slots(const Geom& g) { return g.nt + (g.X > 0 ? 1 : 0); }
// first point of tile b of the unshifted tiling (b = nt gives N)
SW_HD int64_t tile_start(const Geom& g, int64_t b) { return b < g.nt ? b * (int64_t)g.W : g.N; }
// width of tile b (the same for the tile of block b in the shifted tiling)
SW_HD int tile_width(const Geom& g, int64_t b) { return g.W + (b == g.nt - 1 ? g.X : 0); }
// offset of flat-top value k (0..X-1) of component c in an edge buffer
SW_HD int64_t top_index(const Geom& g, int c, int k) { return g.nt * (int64_t)g.E + (int64_t)c * g.X + k; }

SW_HD int64_t floor_div(int64_t a, int64_t b) {
  int64_t q = a / b;
  return (a % b != 0 && ((a < 0) != (b < 0))) ? q - 1 : q;
}

SW_HD int64_t wrap_n(int64_t x, int64_t n) {
  int64_t r = x % n;
  return r < 0 ? r + n : r;
}

// stage (0-based) of the update that produces sub-timestep level s >= 1
SW_HD int stage_of(const Geom& g, int s) { return (s - 1) % g.S; }

// the same with the scheme's stage count Op::S as a compile-time constant
template <class Op>
SW_HD int stage_c(int s) {
  return Op::S == 1 ? 0 : (s - 1) % Op::S;
}

// The geometry as a pass sees it in context Cx: the stencil radius and the
// values per point replaced by the constants the context fixes at compile
// time (Cx::kR, Cx::kC; 0 keeps the runtime field, as in the host checker),
// so that on the device the index arithmetic of the phases folds to constants.
template <class Cx>
SW_HD Geom fixed_geom(const Geom& g) {
  Geom f = g;
  if (Cx::kR > 0) f.R = Cx::kR;
  if (Cx::kC > 0) f.C = Cx::kC;
  return f;
}

// tile tiers: level s on local [R + R s, W + R - R s)
SW_HD int up_lo(const Geom& g, int s) { return g.R + g.R * s; }
SW_HD int up_hi(const Geom& g, int s) { return g.W + g.R - g.R * s; }
// complementary (growing) triangle: level s on local [W/2 + R - R s, W/2 + R + R s)
SW_HD int grow_lo(const Geom& g, int s) { return g.W / 2 + g.R - g.R * s; }
SW_HD int grow_hi(const Geom& g, int s) { return g.W / 2 + g.R + g.R * s; }

// edge k (0..2R-1) of level s of a tile of width w, side 0 = left end, 1 = right end
SW_HD int edge_pos(const Geom& g, int side, int s, int k, int w) {
  return side == 0 ? g.R + g.R * s + k : w - g.R - g.R * s + k;
}
SW_HD int edge_pos(const Geom& g, int side, int s, int k) { return edge_pos(g, side, s, k, g.W); }
// where an edge lands in the diamond window: the right edges (side 1) of the
// tile left of c, and the left edges (side 0) of the tile right of c
SW_HD int insert_pos(const Geom& g, int side, int s, int k) {
  return side == 1 ? g.W / 2 - g.R - g.R * s + k : g.W / 2 + g.R + g.R * s + k;
}
// offset of an edge value in an edge buffer (per tile block of E values)
SW_HD int64_t edge_index(const Geom& g, int64_t tile, int side, int s, int c, int k) {
  return tile * (int64_t)g.E + ((int64_t)(side * g.h + s) * g.C + c) * (2 * g.R) + k;
}

// A slab of a grid split over several ranks (the multi-GPU swept solver that
// the paper names as future work, Section "Conclusion"): the nt tiles are
// divided into contiguous runs, and a rank runs blocks [b0, b0 + nb) of every
// pass.  Its state array holds global points [x0, x0 + ul) of each component
// at index c ul + (x - x0), with no wrap-around: the blocks of an odd pass
// reach W/2 points past the slab's end, which the right neighbour owns.  Its
// edge buffers hold ns = min(nb + 2, nt) tile slots: the neighbours' tiles
// b0 - 1 and b0 + nb (mod nt, "ghost" slots filled by the exchange) around
// its own tiles, then the flat-top slot when X > 0.
struct Slab {
  int64_t b0 = 0, nb = 0;  // first block and number of blocks of this slab
  int64_t x0 = 0, ul = 0;  // global point of state index 0; values per component
  int64_t ns = 0;          // tile slots of each edge buffer (before the flat-top slot)
};
// slot of tile t (0 <= t < nt) in a slab's edge buffers: (t - b0 + 1) mod nt
SW_HD int64_t slab_slot(const Geom& g, const Slab& sl, int64_t t) {
  int64_t d = t - sl.b0 + 1;
  if (d < 0) d += g.nt;
  else if (d >= g.nt) d -= g.nt;
  return d;
}
// values of one edge buffer of a slab
SW_HD int64_t slab_edge_values(const Geom& g, const Slab& sl) {
  return sl.ns * (int64_t)g.E + (g.X > 0 ? (int64_t)g.C * g.X : 0);
}

// pass p >= 1: boundary (diamond centre) handled by block b, and its two tiles
SW_HD int64_t pass_center(const Geom& g, int odd, int64_t b) {
  return odd ? (b + 1) * (int64_t)g.W : b * (int64_t)g.W + g.W / 2;
}
SW_HD int64_t left_tile(const Geom& g, int odd, int64_t b) { return odd ? b : (b + g.nt - 1) % g.nt; }
SW_HD int64_t right_tile(const Geom& g, int odd, int64_t b) { return odd ? (b + 1) % g.nt : b; }

// Local index of the first point after a mirror wall (x = k N) inside the
// window [origin, origin + m), or NO_WALL (periodic, or no wall inside).
SW_HD int window_wall(const Geom& g, int64_t origin, int m) {
  if (g.bc == 0) return NO_WALL;
  const int64_t xw = (floor_div(origin, g.N) + 1) * g.N;
  return (xw < origin + m) ? (int)(xw - origin) : NO_WALL;
}
// position read for neighbour offset d of point j: across a wall, the mirror
// image (the boundary rule applied at the split node, Section "First-order")
SW_HD int nbr(int j, int d, int wall) {
  const int q = j + d;
  return (wall != NO_WALL && ((j < wall) != (q < wall))) ? 2 * wall - 1 - q : q;
}
SW_HD bool through_wall(int j, int d, int wall) { return wall != NO_WALL && ((j < wall) != (j + d < wall)); }

}  // namespace swept
