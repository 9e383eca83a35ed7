// Two-dimensional swept decomposition: geometry, pass phases and launch
// sequence, shared by the CUDA kernels and the host-side schedule checker.
//
// The paper decomposes 1D problems and names two dimensions as future work
// (Section "Conclusion").  This is that extension for a 2D stencil of radius R
// on a periodic nx x ny grid of W x W tiles, h = W / (2R) levels per half
// cycle.  At level s every point falls in exactly one of four regions, by
// its distances dx, dy to the nearest tile boundary line of the current tiling:
//   pyramid   dx >= R s and dy >= R s   (the tile's shrinking square)
//   x-bridge  dx <  R s and dy >= R s   (grows across a vertical boundary,
//                                        shrinks along it)
//   y-bridge  dx >= R s and dy <  R s
//   corner    dx <  R s and dy <  R s   (the square growing around a corner)
// A pyramid needs only itself, a bridge its two pyramids and itself, a corner
// everything around it.  So a half cycle runs in two launches:
//   BRIDGE: every x- and y-bridge from the pyramids' side strips;
//   OCTA:   every corner square grown from the pyramids' corner patches and
//           the bridges' end bands up to a full tile of the half-shifted
//           tiling, then (like the 1D diamond) shrunk as that tile's pyramid,
//           exporting its side strips for the next BRIDGE.
// The first launch is a plain pyramid (PYR) of each tile.  The last OCTA
// writes its completed tile (level h) back to the state.  A remainder of
// rem < h levels runs PYR, BRIDGE and OCTA truncated at rem, each writing its
// level-rem region (the four regions of level rem partition the grid).
//
// Each block holds an (W + 2R)^2 window of two level rows (even levels in
// row 0, odd levels in row 1), as in the 1D two-row buffer.  Exchange data:
//   strips  per tile and level s < h, its four 2R-wide side strips of length
//           W - 2Rs (sides: 0 left, 1 right, 2 bottom, 3 top), two buffers
//           used in turn (an OCTA reads one and writes the other);
//   bands   per bridge and level s < h, its two 2R-wide end bands of length
//           2Rs (end 0 at the low end of its shrinking axis, 1 at the high end).
#pragma once
#include <stdint.h>

#include "swept_geom.cuh"

namespace swept2d {

using swept::wrap_n;

enum Kind2 : int { K_PYR = 0, K_BRIDGE = 1, K_OCTA = 2 };
// FULL: a complete pass that exports; DOWN: the last OCTA, writes its tile;
// GAP: a remainder pass, writes its level-hh region
enum Mode2 : int { M2_FULL = 0, M2_DOWN = 1, M2_GAP = 2 };

struct Geom2 {
  int64_t nx, ny;    // grid points along x (fastest) and y
  int64_t ntx, nty;  // tiles along x and y
  int W;             // tile width
  int R;             // stencil radius
  int h;             // W / (2R)
  int M;             // W + 2R: window width
  int64_t Ph;        // sum over s < h of the strip length W - 2Rs
  int64_t Bh;        // sum over s < h of the band length 2Rs
  int64_t Es;        // values per tile in a strip buffer: 4 sides * 2R * Ph
  int64_t Eb;        // values per bridge in the band buffer: 2 ends * 2R * Bh
  int bc;            // 0 periodic, 1 mirror walls at -1/2 and n - 1/2 on both axes (insulated)
};

// Along one axis of n points, the local index of the first point after a
// mirror wall (a multiple of n) inside the window [origin, origin + M), or
// NO_WALL (periodic, or no wall inside).  A window is shorter than n, so it
// holds at most one wall per axis; the points on its two sides are the two
// ends of the domain, and a stencil read across the wall takes the mirror
// image on the reader's own side (swept::nbr).
SW_HD int axis_wall(int bc, int64_t n, int64_t origin, int M) {
  if (bc == 0) return swept::NO_WALL;
  const int64_t xw = (swept::floor_div(origin, n) + 1) * n;
  return xw < origin + M ? (int)(xw - origin) : swept::NO_WALL;
}

SW_HD int strip_len(const Geom2& g, int s) { return g.W - 2 * g.R * s; }
SW_HD int64_t strip_off(const Geom2& g, int s) { return (int64_t)s * g.W - (int64_t)g.R * s * (s - 1); }
// offset of (side, s, k, p) inside one tile's strip block (< Es, fits 32 bits);
// the tile's block starts at tile * Es
SW_HD int strip_in_tile(const Geom2& g, int side, int s, int k, int p) {
  return side * (2 * g.R) * (int)g.Ph + 2 * g.R * (s * g.W - g.R * s * (s - 1)) + k * strip_len(g, s) + p;
}
SW_HD int64_t band_off(const Geom2& g, int s) { return (int64_t)g.R * s * (s - 1); }
// offset of (end, s, k, p) inside one bridge's band block (< Eb); the
// bridge's block starts at bridge * Eb
SW_HD int band_in_bridge(const Geom2& g, int end, int s, int k, int p) {
  return end * (2 * g.R) * (int)g.Bh + 2 * g.R * (g.R * s * (s - 1)) + k * (2 * g.R * s) + p;
}
SW_HD int64_t tile_id(const Geom2& g, int64_t tx, int64_t ty) { return wrap_n(ty, g.nty) * g.ntx + wrap_n(tx, g.ntx); }
// x-bridge between tiles (tx, ty) and (tx+1, ty); y-bridge between (tx, ty) and (tx, ty+1)
SW_HD int64_t xbridge_id(const Geom2& g, int64_t tx, int64_t ty) { return tile_id(g, tx, ty); }
SW_HD int64_t ybridge_id(const Geom2& g, int64_t tx, int64_t ty) { return g.ntx * g.nty + tile_id(g, tx, ty); }

// The geometry with the radius the context fixes at compile time (Cx::kR; 0
// keeps the runtime field, as the host checker does), so that on the device
// the index arithmetic of the phases folds to constants.
template <class Cx>
SW_HD Geom2 fixed_geom2(const Geom2& g) {
  Geom2 f = g;
  if (Cx::kR > 0) f.R = Cx::kR;
  return f;
}

// Export the four side strips of levels 0..hh-1 of the pyramid whose tile sits
// at local [R, W + R)^2 (level s in row s & 1 on [R + Rs, W + R - Rs)^2).
template <class Cx>
SW_HD void export_strips(Cx& cx, const Geom2& g_in, int64_t tile, int hh) {
  const Geom2 g = fixed_geom2<Cx>(g_in);
  const int R = g.R, W = g.W;
  const int64_t base = tile * g.Es;
  cx.for_grid(4 * 2 * R * hh, W, [&](int o, int p) {
    int rest, s;
    cx.divmod(o, hh, rest, s);
    const int k = rest % (2 * R);
    const int side = rest / (2 * R);
    if (p >= strip_len(g, s)) return;
    const int across = side == 0 || side == 2 ? R + R * s + k : W - R - R * s + k;
    const int along = R + R * s + p;
    const int lx = side < 2 ? across : along;
    const int ly = side < 2 ? along : across;
    cx.store_strip(s & 1, lx, ly, base + strip_in_tile(g, side, s, k, p));
  });
}

// Pyramid of tile (tx, ty) of the tiling with offset par * W/2: levels 1..hh,
// strips of levels 0..hh-1; with write_top, level hh written back (remainder).
template <class Cx>
SW_HD void run_pyr(Cx& cx, const Geom2& g_in, int64_t tx, int64_t ty, int par, int hh, bool write_top) {
  const Geom2 g = fixed_geom2<Cx>(g_in);
  const int R = g.R, W = g.W;
  const int64_t X0 = par * (W / 2) + tx * W, Y0 = par * (W / 2) + ty * W;
  const int64_t ox = X0 - R, oy = Y0 - R;
  cx.for_grid(W, W, [&](int b, int a) { cx.load_u(0, R + a, R + b, X0 + a, Y0 + b); });
  cx.sync();
  for (int s = 1; s <= hh; ++s) cx.level(s, 0, R + R * s, W + R - R * s, R + R * s, W + R - R * s, ox, oy);
  export_strips(cx, g, tile_id(g, tx, ty), hh);
  if (write_top) {
    const int lo = R + R * hh, w = W - 2 * R * hh;
    if (w > 0) cx.for_grid(w, w, [&](int b, int a) { cx.store_u(hh & 1, lo + a, lo + b, ox + lo + a, oy + lo + b); });
  }
}

// Bridge `bid` (x-bridges first, then y-bridges) of the tiling with offset
// par * W/2: the two pyramids' facing strips inserted, levels 1..hh grown
// across the boundary and shrunk along it, end bands of levels 0..hh-1
// exported; with write_top, level hh written back (remainder).
template <class Cx>
SW_HD void run_bridge(Cx& cx, const Geom2& g_in, int64_t bid, int par, int hh, bool write_top) {
  const Geom2 g = fixed_geom2<Cx>(g_in);
  const int R = g.R, W = g.W, half = W / 2;
  const bool ydir = bid >= g.ntx * g.nty;
  const int64_t t = ydir ? bid - g.ntx * g.nty : bid;
  const int64_t tx = t % g.ntx, ty = t / g.ntx;
  const int64_t o = par * half;
  // window origin; local (u, v) = (grow-axis, shrink-axis) coordinates
  const int64_t ox = ydir ? o + tx * W - R : o + (tx + 1) * W - half - R;
  const int64_t oy = ydir ? o + (ty + 1) * W - half - R : o + ty * W - R;
  const int64_t lo_base = tile_id(g, tx, ty) * g.Es;
  const int64_t hi_base = (ydir ? tile_id(g, tx, ty + 1) : tile_id(g, tx + 1, ty)) * g.Es;
  // strips: the low tile's high side (1 right / 3 top), the high tile's low side (0 / 2)
  cx.for_grid(2 * 2 * R * hh, W, [&](int oo, int p) {
    int rest, s;
    cx.divmod(oo, hh, rest, s);
    const int k = rest % (2 * R);
    const int which = rest / (2 * R);
    if (p >= strip_len(g, s)) return;
    const int gpos = which == 0 ? half - R - R * s + k : half + R + R * s + k;  // grow axis
    const int spos = R + R * s + p;                                             // shrink axis
    const int side = which == 0 ? (ydir ? 3 : 1) : (ydir ? 2 : 0);
    const int64_t e = (which == 0 ? lo_base : hi_base) + strip_in_tile(g, side, s, k, p);
    if (ydir)
      cx.load_strip(s & 1, spos, gpos, e);
    else
      cx.load_strip(s & 1, gpos, spos, e);
  });
  cx.sync();
  for (int s = 1; s <= hh; ++s) {
    const int g0 = half + R - R * s, g1 = half + R + R * s, s0 = R + R * s, s1 = W + R - R * s;
    if (ydir)
      cx.level(s, 0, s0, s1, g0, g1, ox, oy);
    else
      cx.level(s, 0, g0, g1, s0, s1, ox, oy);
  }
  const int64_t bbase = (ydir ? ybridge_id(g, tx, ty) : xbridge_id(g, tx, ty)) * g.Eb;
  cx.for_grid(2 * 2 * R * hh, 2 * R * hh, [&](int oo, int p) {
    int rest, s;
    cx.divmod(oo, hh, rest, s);
    const int k = rest % (2 * R);
    const int end = rest / (2 * R);
    if (p >= 2 * R * s) return;
    const int gpos = half + R - R * s + p;
    const int spos = end == 0 ? R + R * s + k : W - R - R * s + k;
    const int64_t e = bbase + band_in_bridge(g, end, s, k, p);
    if (ydir)
      cx.store_band(s & 1, spos, gpos, e);
    else
      cx.store_band(s & 1, gpos, spos, e);
  });
  if (write_top) {
    const int g0 = half + R - R * hh, gw = 2 * R * hh, s0 = R + R * hh, sw = W - 2 * R * hh;
    if (sw > 0)
      cx.for_grid(ydir ? gw : sw, ydir ? sw : gw, [&](int b2, int a) {
        const int lx = ydir ? s0 + a : g0 + a;
        const int ly = ydir ? g0 + b2 : s0 + b2;
        cx.store_u(hh & 1, lx, ly, ox + lx, oy + ly);
      });
  }
}

// Octahedron producing tile (tx, ty) of the tiling with offset odd * W/2: its
// centre is a corner of the previous tiling.  The corner patches of the four
// pyramids around it and the end bands of the four bridges meeting there are
// inserted, the square around the corner grown for levels 1..hh, then
//   M2_FULL: shrunk as the new tile's pyramid (levels 1..h-1 past h) and its
//            strips exported;
//   M2_DOWN: the completed tile (level h) written back;
//   M2_GAP:  the grown square of level hh written back (remainder).
template <class Cx>
SW_HD void run_octa(Cx& cx, const Geom2& g_in, int64_t tx, int64_t ty, int odd, int mode, int hh) {
  const Geom2 g = fixed_geom2<Cx>(g_in);
  const int R = g.R, W = g.W, half = W / 2, lc = half + R;
  const int64_t X0 = odd * half + tx * W, Y0 = odd * half + ty * W;
  const int64_t ox = X0 - R, oy = Y0 - R;
  // previous tiling: tiles left/right of the corner (x) and below/above it (y)
  const int64_t lx_t = odd ? tx : tx - 1, rx_t = odd ? tx + 1 : tx;
  const int64_t ly_t = odd ? ty : ty - 1, uy_t = odd ? ty + 1 : ty;
  // the four bridges meeting at the corner and the four tiles around it
  const int64_t xb_up = xbridge_id(g, lx_t, uy_t) * g.Eb, xb_dn = xbridge_id(g, lx_t, ly_t) * g.Eb;
  const int64_t yb_r = ybridge_id(g, rx_t, ly_t) * g.Eb, yb_l = ybridge_id(g, lx_t, ly_t) * g.Eb;
  const int64_t t_ur = tile_id(g, rx_t, uy_t) * g.Es, t_ul = tile_id(g, lx_t, uy_t) * g.Es;
  const int64_t t_lr = tile_id(g, rx_t, ly_t) * g.Es, t_ll = tile_id(g, lx_t, ly_t) * g.Es;
  // bands: x-bridges above (low end) and below (high end), y-bridges right
  // (low end) and left (high end)
  cx.for_grid(4 * 2 * R * hh, 2 * R * hh, [&](int oo, int p) {
    int rest, s;
    cx.divmod(oo, hh, rest, s);
    const int k = rest % (2 * R);
    const int piece = rest / (2 * R);
    if (p >= 2 * R * s) return;
    const int along = lc - R * s + p;
    const int near_hi = lc + R * s + k, near_lo = lc - R * s - 2 * R + k;
    if (piece == 0)
      cx.load_band(s & 1, along, near_hi, xb_up + band_in_bridge(g, 0, s, k, p));
    else if (piece == 1)
      cx.load_band(s & 1, along, near_lo, xb_dn + band_in_bridge(g, 1, s, k, p));
    else if (piece == 2)
      cx.load_band(s & 1, near_hi, along, yb_r + band_in_bridge(g, 0, s, k, p));
    else
      cx.load_band(s & 1, near_lo, along, yb_l + band_in_bridge(g, 1, s, k, p));
  });
  // pyramid corner patches from the left (side 0) / right (side 1) strips
  cx.for_grid(4 * 2 * R * hh, 2 * R, [&](int oo, int p) {
    int rest, s;
    cx.divmod(oo, hh, rest, s);
    const int k = rest % (2 * R);
    const int piece = rest / (2 * R);  // 0 upper-right, 1 upper-left, 2 lower-right, 3 lower-left
    const bool right = piece == 0 || piece == 2, upper = piece < 2;
    const int lx = right ? lc + R * s + k : lc - R * s - 2 * R + k;
    const int ly = upper ? lc + R * s + p : lc - R * s - 2 * R + p;
    const int pos = upper ? p : strip_len(g, s) - 2 * R + p;
    const int64_t base = piece == 0 ? t_ur : (piece == 1 ? t_ul : (piece == 2 ? t_lr : t_ll));
    cx.load_strip(s & 1, lx, ly, base + strip_in_tile(g, right ? 0 : 1, s, k, pos));
  });
  cx.sync();
  for (int s = 1; s <= hh; ++s) cx.level(s, 0, lc - R * s, lc + R * s, lc - R * s, lc + R * s, ox, oy);
  if (mode == M2_FULL) {
    for (int s = 1; s < g.h; ++s) cx.level(s, g.h, R + R * s, W + R - R * s, R + R * s, W + R - R * s, ox, oy);
    export_strips(cx, g, tile_id(g, tx, ty), g.h);
  } else if (mode == M2_DOWN) {
    cx.for_grid(W, W, [&](int b, int a) { cx.store_u(g.h & 1, R + a, R + b, X0 + a, Y0 + b); });
  } else {
    const int lo = lc - R * hh, w = 2 * R * hh;
    cx.for_grid(w, w, [&](int b, int a) { cx.store_u(hh & 1, lo + a, lo + b, ox + lo + a, oy + lo + b); });
  }
}

// The launch sequence for n levels: q = n / h full half cycles (PYR, then q
// times BRIDGE + OCTA, the last OCTA writing the state) and, for rem = n % h,
// a PYR / BRIDGE / OCTA triple truncated at rem.
//   emit(kind, par, mode, hh, cycle):  cycle c >= 0 of a full pass (PYR: 0;
//   BRIDGE and OCTA of half cycle c >= 1), -1 for the remainder.  par is the
//   tiling parity of PYR / BRIDGE (offset par * W/2) and of the tiling an
//   OCTA produces.  Strips: PYR and OCTA of cycle c write buffer c & 1;
//   BRIDGE and OCTA of cycle c read buffer (c - 1) & 1; the remainder uses
//   buffer 0.
template <class F>
inline void for_each_launch2d(const Geom2& g, int64_t n, F emit) {
  const int64_t q = n / g.h;
  const int rem = (int)(n % g.h);
  if (q > 0) {
    emit(K_PYR, 0, M2_FULL, g.h, (int64_t)0);
    for (int64_t c = 1; c <= q; ++c) {
      emit(K_BRIDGE, (int)((c - 1) & 1), M2_FULL, g.h, c);
      emit(K_OCTA, (int)(c & 1), c == q ? M2_DOWN : M2_FULL, g.h, c);
    }
  }
  if (rem > 0) {
    emit(K_PYR, 0, M2_GAP, rem, (int64_t)-1);
    emit(K_BRIDGE, 0, M2_GAP, rem, (int64_t)-1);
    emit(K_OCTA, 1, M2_GAP, rem, (int64_t)-1);
  }
}

// ---------------------------------------------------------------------------
// Persistent form of the launch sequence: one queue of items run by a
// persistent kernel whose blocks order themselves only through waits on
// per-tile and per-bridge counters.  Queue order (T = tiles):
//   PYR of cycle 0 (T items) | per half cycle c = 1..q: BRIDGE_c (2T), OCTA_c (T)
//   | remainder: PYR (T), BRIDGE (2T), OCTA (T)
// Counters: tile_done[t] = stage of the last finished PYR / OCTA of tile slot t
// (PYR 0, OCTA_c c, remainder PYR q + 1); bridge_done[b] likewise for the
// bridges (BRIDGE_c c, remainder q + 1).  Buffers: strips of cycle c in
// S[c & 1]; bands of cycle c in B[c & 1]; the remainder uses S[q & 1] and
// B[(q + 1) & 1].
// ---------------------------------------------------------------------------
struct PItem {
  int kind;     // K_PYR, K_BRIDGE, K_OCTA
  int64_t c;    // half cycle (PYR of cycle 0: 0); -1 for the remainder
  int64_t idx;  // tile slot (PYR, OCTA) or bridge id (BRIDGE)
};

SW_HD int64_t persist2d_items(const Geom2& g, int64_t n) {
  const int64_t T = g.ntx * g.nty, q = n / g.h;
  return (q > 0 ? T + q * 3 * T : 0) + (n % g.h ? 4 * T : 0);
}

SW_HD PItem persist2d_item(const Geom2& g, int64_t n, int64_t item) {
  const int64_t T = g.ntx * g.nty, q = n / g.h;
  const int64_t main_items = q > 0 ? T + q * 3 * T : 0;
  PItem it;
  if (item < main_items) {
    if (item < T) {
      it.kind = K_PYR;
      it.c = 0;
      it.idx = item;
      return it;
    }
    const int64_t rel = item - T;
    it.c = rel / (3 * T) + 1;
    const int64_t r = rel - (it.c - 1) * 3 * T;
    if (r < 2 * T) {
      it.kind = K_BRIDGE;
      it.idx = r;
    } else {
      it.kind = K_OCTA;
      it.idx = r - 2 * T;
    }
    return it;
  }
  const int64_t rel = item - main_items;
  it.c = -1;
  if (rel < T) {
    it.kind = K_PYR;
    it.idx = rel;
  } else if (rel < 3 * T) {
    it.kind = K_BRIDGE;
    it.idx = rel - T;
  } else {
    it.kind = K_OCTA;
    it.idx = rel - 3 * T;
  }
  return it;
}

// The waits of an item: up to four (counter, index, stage) triples; counter 0
// is tile_done, 1 is bridge_done.  Returns their number.
SW_HD int persist2d_deps(const Geom2& g, int64_t n, const PItem& it, int* counter, int64_t* index, int64_t* need) {
  const int64_t q = n / g.h;
  const int64_t tx = it.idx % g.ntx, ty = (it.idx / g.ntx) % g.nty;
  if (it.c == 0) return 0;  // the first pyramid
  if (it.c > 0 || it.kind != K_PYR) {
    const int64_t c = it.c > 0 ? it.c : q + 1;  // remainder bridges and corners are stage q + 1
    if (it.kind == K_BRIDGE) {
      // its two pyramids of the previous tiling: the last OCTA (or PYR) of those slots
      const bool ydir = it.idx >= g.ntx * g.nty;
      const int64_t t = ydir ? it.idx - g.ntx * g.nty : it.idx;
      const int64_t bx = t % g.ntx, by = t / g.ntx;
      counter[0] = counter[1] = 0;
      index[0] = tile_id(g, bx, by);
      index[1] = ydir ? tile_id(g, bx, by + 1) : tile_id(g, bx + 1, by);
      need[0] = need[1] = it.c > 0 ? c - 1 : q + 1;  // the remainder waits for the remainder pyramid
      return 2;
    }
    // K_OCTA: the four bridges meeting at its corner (through them, the four tiles)
    const int odd = it.c > 0 ? (int)(it.c & 1) : 1;
    const int64_t lx_t = odd ? tx : tx - 1, rx_t = odd ? tx + 1 : tx;
    const int64_t ly_t = odd ? ty : ty - 1, uy_t = odd ? ty + 1 : ty;
    counter[0] = counter[1] = counter[2] = counter[3] = 1;
    index[0] = xbridge_id(g, lx_t, uy_t);
    index[1] = xbridge_id(g, lx_t, ly_t);
    index[2] = ybridge_id(g, rx_t, ly_t);
    index[3] = ybridge_id(g, lx_t, ly_t);
    need[0] = need[1] = need[2] = need[3] = c;
    return 4;
  }
  // remainder PYR of tile (tx, ty) of the unshifted tiling: the last full OCTA
  // wrote the state over it from the (tx-1 .. tx) x (ty-1 .. ty) slots of its
  // tiling (one slot when that tiling is unshifted); none when q = 0
  if (q == 0) return 0;
  for (int i = 0; i < 4; ++i) {
    counter[i] = 0;
    index[i] = tile_id(g, tx - (i & 1), ty - (i >> 1));
    need[i] = q;
  }
  return 4;
}

// The counter an item sets when it finishes: (counter, index, stage) as in
// persist2d_deps.  Every item sets one; nothing waits on the remainder OCTA's.
SW_HD void persist2d_signal(const Geom2& g, int64_t n, const PItem& it, int* counter, int64_t* index,
                            int64_t* stage) {
  *counter = it.kind == K_BRIDGE ? 1 : 0;
  *index = it.idx;
  *stage = it.c >= 0 ? it.c : n / g.h + 1;
}

// What an item runs: buffers (strip in/out, band in/out), tiling parity
// (PYR / BRIDGE) or produced tiling (OCTA), mode, levels and the absolute level
// of its local level 0.  Shared by the persistent kernel and the replay.
struct PWork {
  int s_in, s_out, b_in, b_out, par, mode, hh;
  int64_t base;
};
SW_HD PWork persist2d_work(const Geom2& g, int64_t n, const PItem& it) {
  const int64_t q = n / g.h;
  const int rem = (int)(n % g.h);
  PWork w;
  w.s_in = w.s_out = w.b_in = w.b_out = 0;
  if (it.c >= 0) {
    const int cp = (int)((it.c + 1) & 1), cc = (int)(it.c & 1);  // parities of c - 1 and c
    w.hh = g.h;
    w.base = it.c > 0 ? (it.c - 1) * (int64_t)g.h : 0;
    w.mode = (it.kind == K_OCTA && it.c == q) ? M2_DOWN : M2_FULL;
    if (it.kind == K_PYR) {
      w.s_out = 0;
      w.par = 0;
    } else if (it.kind == K_BRIDGE) {
      w.s_in = cp;
      w.b_out = cc;
      w.par = cp;
    } else {
      w.s_in = cp;
      w.s_out = cc;
      w.b_in = cc;
      w.par = cc;
    }
  } else {
    w.hh = rem;
    w.base = q * (int64_t)g.h;
    w.mode = M2_GAP;
    w.s_in = w.s_out = (int)(q & 1);
    w.b_in = w.b_out = (int)((q + 1) & 1);
    w.par = it.kind == K_OCTA ? 1 : 0;
  }
  return w;
}

inline int64_t launch_count2d(const Geom2& g, int64_t n) {
  const int64_t q = n / g.h;
  return (q > 0 ? 1 + 2 * q : 0) + (n % g.h ? 3 : 0);
}

}  // namespace swept2d
