// Host-side symbolic replay of the 2D swept launch sequence, or of the
// persistent kernel's queue (swept2d_check_schedule).
//
// Runs the same phase code as the kernels (swept2d.cuh) over every block, with
// buffers that hold (point, level) tags instead of values, and checks:
//   - a point of level L is computed only when its five stencil inputs hold
//     level L - 1 of the right grid points, found from the periodic grid
//     itself (independently of the window arithmetic);
//   - every point of every level 1..n is computed exactly once;
//   - blocks of one launch never touch a global location another block of
//     the same launch writes;
//   - persistent queue: every item waits only for earlier items, each counter
//     only grows, and every access to a global location happens after the
//     item that last wrote it (and a write after every item that read the old
//     value), through the waits' transitive closure;
//   - every window index stays inside the window and every strip and band
//     index inside its buffer;
//   - at the end the state holds level n at every point.
#include <stdio.h>

#include <string>
#include <vector>

#include "swept2d.cuh"

namespace swept2d {
namespace {

struct Tag {
  int64_t p = -1;    // grid point y * nx + x
  int64_t lvl = -1;  // level
};

struct Access {
  int64_t stamp = -1;
  int64_t writer = -1;
  int64_t reader = -1;  // -2: read by several blocks
};

struct HbLoc {  // persistent mode: per global location
  int64_t writer = -1;
  std::vector<int64_t> readers;
};

// buffers: the state, the two strip buffers, the two band buffers
enum Buf2 { B2_U = 0, B2_S0 = 1, B2_S1 = 2, B2_B0 = 3, B2_B1 = 4 };

struct Sim2 {
  Geom2 g;
  int64_t n = 0;
  std::vector<Tag> u, s[2], b[2];
  std::vector<Access> au, as[2], ab[2];
  bool hb_mode = false;
  std::vector<std::vector<uint64_t>> anc;  // ancestors of each item (bitsets)
  std::vector<HbLoc> hb[5];
  std::vector<uint8_t> count;  // (n + 1) * nx * ny
  int64_t stamp = 0;
  int64_t computed = 0;
  std::string err;

  void fail(const std::string& m) {
    if (err.empty()) err = m;
  }
  bool before(int64_t a, int64_t b) const { return a == b || ((anc[(size_t)b][(size_t)(a >> 6)] >> (a & 63)) & 1); }
  std::vector<Access>& acc(Buf2 k) {
    return k == B2_U ? au : (k == B2_S0 || k == B2_S1) ? as[k - B2_S0] : ab[k - B2_B0];
  }
  void note(Buf2 k, size_t i, int64_t block, bool write, const char* what) {
    if (hb_mode) return note_hb(k, i, block, write, what);
    Access& x = acc(k)[i];
    if (x.stamp != stamp) x = Access{stamp, -1, -1};
    char m[160];
    if (write) {
      if ((x.writer != -1 && x.writer != block) || (x.reader != -1 && x.reader != block)) {
        snprintf(m, sizeof m, "race on %s[%zu] between blocks in launch %lld", what, i, (long long)stamp);
        fail(m);
      }
      x.writer = block;
    } else {
      if (x.writer != -1 && x.writer != block) {
        snprintf(m, sizeof m, "block %lld reads %s[%zu] written by block %lld in the same launch", (long long)block,
                 what, i, (long long)x.writer);
        fail(m);
      }
      x.reader = (x.reader == -1 || x.reader == block) ? block : -2;
    }
  }
  void note_hb(Buf2 k, size_t i, int64_t item, bool write, const char* what) {
    HbLoc& x = hb[k][i];
    char m[200];
    if (x.writer >= 0 && !before(x.writer, item)) {
      snprintf(m, sizeof m, "item %lld %s %s[%zu] written by item %lld, which it does not wait for", (long long)item,
               write ? "overwrites" : "reads", what, i, (long long)x.writer);
      return fail(m);
    }
    if (!write) {
      if (x.readers.empty() || x.readers.back() != item) x.readers.push_back(item);
      return;
    }
    for (int64_t r : x.readers)
      if (!before(r, item)) {
        snprintf(m, sizeof m, "item %lld overwrites %s[%zu] that item %lld reads, without waiting for it",
                 (long long)item, what, i, (long long)r);
        return fail(m);
      }
    x.writer = item;
    x.readers.clear();
  }
};

struct Host2Ctx {
  static constexpr int kR = 0;  // radius from the geometry
  Sim2& sim;
  const Geom2& g;
  int64_t block;
  int64_t base_level;  // absolute level of the launch's local level 0
  int sin, sout, bin, bout;
  std::vector<Tag> w;  // two rows of M x M tags

  Host2Ctx(Sim2& s, int64_t b, int64_t base, int si, int so, int bi = 0, int bo = 0)
      : sim(s), g(s.g), block(b), base_level(base), sin(si), sout(so), bin(bi), bout(bo),
        w((size_t)2 * s.g.M * s.g.M) {}

  template <class F>
  void for_grid(int nout, int nin, F&& f) {
    for (int o = 0; o < nout; ++o)
      for (int i = 0; i < nin; ++i) f(o, i);
  }
  void sync() {}
  void divmod(int a, int b, int& q, int& r) const {
    if (a < 0 || a > 1024 || b < 1 || b > 256) sim.fail("divmod operands outside the device's exact range");
    q = a / b;
    r = a % b;
  }
  int64_t wrap_once(int64_t x, int64_t n) const {
    if (x < -n || x >= 2 * n) sim.fail("window more than one period outside the grid");
    return wrap_n(x, n);
  }
  Tag& cell(int r, int lx, int ly) {
    if (lx < 0 || lx >= g.M || ly < 0 || ly >= g.M) {
      sim.fail("window index out of range");
      static Tag dummy;
      return dummy;
    }
    return w[((size_t)r * g.M + ly) * g.M + lx];
  }
  int64_t gp(int64_t gx, int64_t gy) const { return wrap_once(gy, g.ny) * g.nx + wrap_once(gx, g.nx); }
  void load_u(int r, int lx, int ly, int64_t gx, int64_t gy) {
    const size_t i = (size_t)gp(gx, gy);
    sim.note(B2_U, i, block, false, "u");
    cell(r, lx, ly) = sim.u[i];
  }
  void store_u(int r, int lx, int ly, int64_t gx, int64_t gy) {
    const size_t i = (size_t)gp(gx, gy);
    sim.note(B2_U, i, block, true, "u");
    const Tag t = cell(r, lx, ly);
    if (t.p != (int64_t)i) sim.fail("store_u writes the value of another point");
    sim.u[i] = t;
  }
  void load_strip(int r, int lx, int ly, int64_t e) {
    if (e < 0 || (size_t)e >= sim.s[sin].size()) return sim.fail("strip index out of range");
    sim.note(sin ? B2_S1 : B2_S0, (size_t)e, block, false, "strips");
    cell(r, lx, ly) = sim.s[sin][(size_t)e];
  }
  void store_strip(int r, int lx, int ly, int64_t e) {
    if (e < 0 || (size_t)e >= sim.s[sout].size()) return sim.fail("strip index out of range");
    sim.note(sout ? B2_S1 : B2_S0, (size_t)e, block, true, "strips");
    sim.s[sout][(size_t)e] = cell(r, lx, ly);
  }
  void load_band(int r, int lx, int ly, int64_t e) {
    if (e < 0 || (size_t)e >= sim.b[bin].size()) return sim.fail("band index out of range");
    sim.note(bin ? B2_B1 : B2_B0, (size_t)e, block, false, "bands");
    cell(r, lx, ly) = sim.b[bin][(size_t)e];
  }
  void store_band(int r, int lx, int ly, int64_t e) {
    if (e < 0 || (size_t)e >= sim.b[bout].size()) return sim.fail("band index out of range");
    sim.note(bout ? B2_B1 : B2_B0, (size_t)e, block, true, "bands");
    sim.b[bout][(size_t)e] = cell(r, lx, ly);
  }
  // The grid point the stencil of (x, y) (in [0, n)) reads at offset (dx, dy),
  // from the boundary rule itself (independent of the window arithmetic):
  // periodic wraps; mirror walls at -1/2 and n - 1/2 reflect -1 to 0 and n to n - 1.
  int64_t physical_neighbour(int64_t x, int64_t y, int dx, int dy) const {
    auto axis = [&](int64_t v, int64_t n) {
      if (g.bc == 0) return wrap_n(v, n);
      if (v < 0) return -1 - v;
      if (v >= n) return 2 * n - 1 - v;
      return v;
    };
    return axis(y + dy, g.ny) * g.nx + axis(x + dx, g.nx);
  }
  void level(int s, int base, int x0, int x1, int y0, int y1, int64_t ox, int64_t oy) {
    const int64_t L = base_level + base + s;
    const int row = s & 1;
    static const int dxs[5] = {0, -1, 1, 0, 0}, dys[5] = {0, 0, 0, -1, 1};
    const int wx = axis_wall(g.bc, g.nx, ox, g.M), wy = axis_wall(g.bc, g.ny, oy, g.M);
    char m[220];
    for (int ly = y0; ly < y1; ++ly)
      for (int lx = x0; lx < x1; ++lx) {
        const int64_t gx = ox + lx, gy = oy + ly;
        for (int d = 0; d < 5; ++d) {
          // the window cell the kernels read: across a wall, the mirror image
          const Tag t = cell(row ^ 1, swept::nbr(lx, dxs[d], wx), swept::nbr(ly, dys[d], wy));
          const int64_t want = physical_neighbour(wrap_once(gx, g.nx), wrap_once(gy, g.ny), dxs[d], dys[d]);
          if (t.p != want || t.lvl != L - 1) {
            snprintf(m, sizeof m,
                     "block %lld level %lld point (%lld, %lld): input (%d, %d) holds (point %lld, level %lld), "
                     "expected (%lld, %lld)",
                     (long long)block, (long long)L, (long long)wrap_n(gx, g.nx), (long long)wrap_n(gy, g.ny),
                     dxs[d], dys[d], (long long)t.p, (long long)t.lvl, (long long)want, (long long)(L - 1));
            return sim.fail(m);
          }
        }
      }
    for (int ly = y0; ly < y1; ++ly)
      for (int lx = x0; lx < x1; ++lx) {
        const int64_t p = gp(ox + lx, oy + ly);
        cell(row, lx, ly) = Tag{p, L};
        if (L >= 1 && L <= sim.n) {
          uint8_t& c = sim.count[(size_t)L * g.nx * g.ny + (size_t)p];
          if (c < 255) ++c;
        }
        ++sim.computed;
      }
  }
};

}  // namespace

namespace {

void init_sim2(Sim2& sim, const Geom2& g, int64_t n) {
  sim.g = g;
  sim.n = n;
  const int64_t np = g.nx * g.ny;
  sim.u.resize((size_t)np);
  for (int64_t p = 0; p < np; ++p) sim.u[(size_t)p] = Tag{p, 0};
  for (int i = 0; i < 2; ++i) {
    sim.s[i].assign((size_t)(g.ntx * g.nty * g.Es), Tag{});
    sim.as[i].assign(sim.s[i].size(), Access{});
    sim.b[i].assign((size_t)(2 * g.ntx * g.nty * g.Eb), Tag{});
    sim.ab[i].assign(sim.b[i].size(), Access{});
  }
  sim.au.assign((size_t)np, Access{});
  sim.count.assign((size_t)(n + 1) * (size_t)np, 0);
}

void final_checks2(Sim2& sim) {
  const Geom2& g = sim.g;
  const int64_t np = g.nx * g.ny, n = sim.n;
  if (sim.err.empty())
    for (int64_t p = 0; p < np; ++p) {
      const Tag t = sim.u[(size_t)p];
      if (t.p != p || t.lvl != n) {
        char m[160];
        snprintf(m, sizeof m, "final state at point %lld holds (point %lld, level %lld), expected level %lld",
                 (long long)p, (long long)t.p, (long long)t.lvl, (long long)n);
        sim.fail(m);
        break;
      }
    }
  if (sim.err.empty())
    for (int64_t L = 1; L <= n && sim.err.empty(); ++L)
      for (int64_t p = 0; p < np; ++p) {
        const uint8_t c = sim.count[(size_t)L * np + (size_t)p];
        if (c != 1) {
          char m[160];
          snprintf(m, sizeof m, "point %lld of level %lld computed %d times", (long long)p, (long long)L, (int)c);
          sim.fail(m);
          break;
        }
      }
}

// The queue item that sets counter `counter` (0 tile_done, 1 bridge_done) of
// slot `index` to `stage`, from the queue layout of the persistent kernel:
//   PYR_0 (T) | per half cycle c: BRIDGE_c (2T), OCTA_c (T) | remainder PYR (T), BRIDGE (2T), OCTA (T)
int64_t setter_item(const Geom2& g, int64_t n, int counter, int64_t index, int64_t stage) {
  const int64_t T = g.ntx * g.nty, q = n / g.h;
  const int64_t main_items = q > 0 ? T + q * 3 * T : 0;
  if (counter == 0) {
    if (index < 0 || index >= T) return -1;
    if (stage == 0) return q > 0 ? index : -1;
    if (stage >= 1 && stage <= q) return T + (stage - 1) * 3 * T + 2 * T + index;
    if (stage == q + 1 && n % g.h) return main_items + index;
    return -1;
  }
  if (index < 0 || index >= 2 * T) return -1;
  if (stage >= 1 && stage <= q) return T + (stage - 1) * 3 * T + index;
  if (stage == q + 1 && n % g.h) return main_items + T + index;
  return -1;
}

void replay_launches(Sim2& sim) {
  const Geom2& g = sim.g;
  const int64_t n = sim.n, q = n / g.h, tiles = g.ntx * g.nty;
  for_each_launch2d(g, n, [&](int kind, int par, int mode, int hh, int64_t c) {
    ++sim.stamp;
    const int64_t base = c >= 1 ? (c - 1) * (int64_t)g.h : (c == 0 ? 0 : q * (int64_t)g.h);
    const int in = c >= 1 ? (int)((c - 1) & 1) : 0;
    const int out = c >= 0 ? (int)(c & 1) : 1;
    if (kind == K_PYR) {
      for (int64_t b = 0; b < tiles && sim.err.empty(); ++b) {
        Host2Ctx cx(sim, b, base, 0, c >= 0 ? out : 0);
        run_pyr(cx, g, b % g.ntx, b / g.ntx, par, hh, mode == M2_GAP);
      }
    } else if (kind == K_BRIDGE) {
      for (int64_t b = 0; b < 2 * tiles && sim.err.empty(); ++b) {
        Host2Ctx cx(sim, b, base, in, out);
        run_bridge(cx, g, b, par, hh, mode == M2_GAP);
      }
    } else {
      for (int64_t b = 0; b < tiles && sim.err.empty(); ++b) {
        Host2Ctx cx(sim, b, base, in, out);
        run_octa(cx, g, b % g.ntx, b / g.ntx, par, mode, hh);
      }
    }
  });
}

// Persistent queue: items in queue order, each after the items its waits name
// (and, transitively, theirs); accesses checked for happens-before.
void replay_persistent(Sim2& sim, int64_t drop_item) {
  const Geom2& g = sim.g;
  const int64_t n = sim.n, items = persist2d_items(g, n);
  sim.hb_mode = true;
  const size_t words = (size_t)((items + 63) / 64);
  sim.anc.assign((size_t)items, std::vector<uint64_t>(words, 0));
  sim.hb[B2_U].assign(sim.u.size(), HbLoc{});
  for (int i = 0; i < 2; ++i) {
    sim.hb[B2_S0 + i].assign(sim.s[i].size(), HbLoc{});
    sim.hb[B2_B0 + i].assign(sim.b[i].size(), HbLoc{});
  }
  const size_t T = (size_t)(g.ntx * g.nty);
  std::vector<int64_t> last_set[2] = {std::vector<int64_t>(T, -1), std::vector<int64_t>(2 * T, -1)};
  std::vector<int64_t> prev_stage[2] = {std::vector<int64_t>(T, -1), std::vector<int64_t>(2 * T, -1)};
  for (int64_t it = 0; it < items && sim.err.empty(); ++it) {
    const PItem pi = persist2d_item(g, n, it);
    int counter[4];
    int64_t index[4], need[4];
    const int nd = persist2d_deps(g, n, pi, counter, index, need);
    for (int i = 0; i < nd; ++i) {
      if (it == drop_item && i == nd - 1) break;  // planted mistake (tests only)
      const int64_t d = setter_item(g, n, counter[i], index[i], need[i]);
      if (d < 0 || d >= it) {
        char m[200];
        snprintf(m, sizeof m, "item %lld waits for counter %d slot %lld stage %lld, set by no earlier item",
                 (long long)it, counter[i], (long long)index[i], (long long)need[i]);
        sim.fail(m);
        break;
      }
      auto& a = sim.anc[(size_t)it];
      const auto& ad = sim.anc[(size_t)d];
      for (size_t w = 0; w < words; ++w) a[w] |= ad[w];
      a[(size_t)(d >> 6)] |= 1ull << (d & 63);
    }
    if (!sim.err.empty()) break;
    // counters only grow: the previous setter of this item's counter is an ancestor
    int sc;
    int64_t si, ss;
    persist2d_signal(g, n, pi, &sc, &si, &ss);
    int64_t& prev = last_set[sc][(size_t)si];
    if (prev >= 0 && (!sim.before(prev, it) || prev_stage[sc][(size_t)si] > ss)) {
      char m[200];
      snprintf(m, sizeof m, "item %lld sets counter %d slot %lld to %lld without waiting for item %lld that set %lld",
               (long long)it, sc, (long long)si, (long long)ss, (long long)prev,
               (long long)prev_stage[sc][(size_t)si]);
      sim.fail(m);
      break;
    }
    prev = it;
    prev_stage[sc][(size_t)si] = ss;
    const PWork w = persist2d_work(g, n, pi);
    Host2Ctx cx(sim, it, w.base, w.s_in, w.s_out, w.b_in, w.b_out);
    const int64_t tx = pi.idx % g.ntx, ty = pi.idx / g.ntx;
    if (pi.kind == K_PYR)
      run_pyr(cx, g, tx, ty, w.par, w.hh, w.mode == M2_GAP);
    else if (pi.kind == K_BRIDGE)
      run_bridge(cx, g, pi.idx, w.par, w.hh, w.mode == M2_GAP);
    else
      run_octa(cx, g, tx, ty, w.par, w.mode, w.hh);
  }
}

}  // namespace

bool check_schedule2d(const Geom2& g, int64_t n, bool persistent, int64_t drop_item, int64_t* computed,
                      std::string* err) {
  Sim2 sim;
  init_sim2(sim, g, n);
  if (persistent)
    replay_persistent(sim, drop_item);
  else
    replay_launches(sim);
  final_checks2(sim);
  if (computed) *computed = sim.computed;
  if (!sim.err.empty()) {
    if (err) *err = sim.err;
    return false;
  }
  return true;
}

}  // namespace swept2d
