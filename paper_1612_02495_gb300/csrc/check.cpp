// Host-side symbolic replay of the swept launch sequence (swept_check_schedule).
//
// Runs the same pass phases as the kernels (swept_phases.cuh) over every block,
// with buffers that hold (point, sub-timestep) tags instead of values, and
// checks the swept rule's invariants:
//   - a point of tier L is computed only when every stencil input (through the
//     boundary rule) holds tier L-1 of the right point, and, for the second
//     stage of a two-stage scheme, the point itself holds tier L-2;
//   - every point of every tier 1..n_sub is computed exactly once;
//   - blocks of one launch never touch a global location another block of the
//     same launch writes (no race between blocks);
//   - at the end the state holds tier n_sub at every point.
#include <stdio.h>

#include <string>
#include <vector>

#include "runtime.h"
#include "swept_phases.cuh"

namespace swept {
namespace {

struct Tag {
  int64_t x = -1;
  int64_t lvl = -1;
};

struct Access {  // per global location, within the current launch
  int64_t stamp = -1;
  int64_t writer = -1;
  int64_t reader = -1;  // -2: read by several blocks
};

struct Sim {
  Geom g;
  int64_t n_sub = 0;
  std::vector<Tag> u;
  std::vector<Tag> e[2];
  std::vector<Access> au, ae[2];
  std::vector<uint8_t> count;  // (n_sub + 1) * N
  int64_t stamp = 0;
  int64_t computed = 0;
  std::string err;

  void fail(const std::string& m) {
    if (err.empty()) err = m;
  }
  void note(std::vector<Access>& a, size_t i, int64_t block, bool write, const char* what) {
    Access& x = a[i];
    if (x.stamp != stamp) x = Access{stamp, -1, -1};
    if (write) {
      if ((x.writer != -1 && x.writer != block) || (x.reader != -1 && x.reader != block)) {
        char b[160];
        snprintf(b, sizeof b, "race on %s[%zu] between blocks in launch %lld", what, i, (long long)stamp);
        fail(b);
      }
      x.writer = block;
    } else {
      if (x.writer != -1 && x.writer != block) {
        char b[160];
        snprintf(b, sizeof b, "block %lld reads %s[%zu] written by block %lld in the same launch", (long long)block,
                 what, i, (long long)x.writer);
        fail(b);
      }
      x.reader = (x.reader == -1 || x.reader == block) ? block : -2;
    }
  }
};

struct HostCtx {
  static constexpr int kR = 0, kC = 0;  // stencil constants from the geometry
  Sim& sim;
  const Geom& g;
  int64_t block;
  int64_t base_level;  // absolute tier of the pass's local tier 0
  int ein, eout;
  std::vector<Tag> sm;

  HostCtx(Sim& s, int64_t b, int64_t base, int ei, int eo)
      : sim(s), g(s.g), block(b), base_level(base), ein(ei), eout(eo), sm((size_t)2 * s.g.C * s.g.M) {}

  template <class F>
  void for_range(int lo, int hi, F&& f) {
    for (int i = lo; i < hi; ++i) f(i);
  }
  void sync() {}
  Tag& cell(int r, int c, int j) {
    if (j < 0 || j >= g.M) {
      sim.fail("window index out of range");
      static Tag dummy;
      return dummy;
    }
    return sm[(size_t)(r * g.C + c) * g.M + j];
  }
  void load_u(int r, int c, int j, int64_t x) {
    const size_t i = (size_t)(c * g.N + wrap_n(x, g.N));
    sim.note(sim.au, i, block, false, "u");
    cell(r, c, j) = sim.u[i];
  }
  void store_u(int r, int c, int j, int64_t x) {
    const size_t i = (size_t)(c * g.N + wrap_n(x, g.N));
    sim.note(sim.au, i, block, true, "u");
    const Tag t = cell(r, c, j);
    if (t.x != wrap_n(x, g.N)) sim.fail("store_u writes a value of another point");
    sim.u[i] = t;
  }
  void load_edge(int r, int c, int j, int64_t e) {
    if (e < 0 || (size_t)e >= sim.e[ein].size()) return sim.fail("edge index out of range");
    sim.note(sim.ae[ein], (size_t)e, block, false, "edges");
    cell(r, c, j) = sim.e[ein][(size_t)e];
  }
  void store_edge(int r, int c, int j, int64_t e) {
    if (e < 0 || (size_t)e >= sim.e[eout].size()) return sim.fail("edge index out of range");
    sim.note(sim.ae[eout], (size_t)e, block, true, "edges");
    sim.e[eout][(size_t)e] = cell(r, c, j);
  }
  // The grid point whose value the stencil of point x reads at offset d, from
  // the boundary rule itself (independent of the window arithmetic):
  // periodic wraps; a mirror wall at -1/2 (N-1/2) reflects -1-k to k (N+k to N-1-k).
  int64_t physical_neighbour(int64_t x, int d) const {
    const int64_t y = x + d;
    if (g.bc == 0) return wrap_n(y, g.N);
    if (y < 0) return -1 - y;
    if (y >= g.N) return 2 * g.N - 1 - y;
    return y;
  }
  void level(int s, int base, int lo, int hi, int64_t origin, int wall) {
    const int64_t L = base_level + base + s;
    const int row = s & 1;
    const int stage = stage_of(g, s);
    char b[200];
    for (int j = lo; j < hi; ++j) {
      const int64_t x = wrap_n(origin + j, g.N);
      for (int c = 0; c < g.C; ++c) {
        for (int d = -g.R; d <= g.R; ++d) {
          const int q = nbr(j, d, wall);
          const Tag t = cell(row ^ 1, c, q);
          const int64_t want = physical_neighbour(x, d);
          if (t.x != want || t.lvl != L - 1) {
            snprintf(b, sizeof b,
                     "block %lld tier %lld point %lld: input at offset %d holds (point %lld, tier %lld), "
                     "expected (%lld, %lld)",
                     (long long)block, (long long)L, (long long)x, d, (long long)t.x, (long long)t.lvl,
                     (long long)want, (long long)(L - 1));
            return sim.fail(b);
          }
        }
        if (g.S == 2 && stage == 1) {
          const Tag t = cell(row, c, j);
          if (t.x != x || t.lvl != L - 2) {
            snprintf(b, sizeof b, "block %lld tier %lld point %lld: second stage misses tier %lld of the point",
                     (long long)block, (long long)L, (long long)x, (long long)(L - 2));
            return sim.fail(b);
          }
        }
      }
    }
    for (int j = lo; j < hi; ++j) {
      const int64_t x = wrap_n(origin + j, g.N);
      for (int c = 0; c < g.C; ++c) cell(row, c, j) = Tag{x, L};
      if (L >= 1 && L <= sim.n_sub) {
        uint8_t& n = sim.count[(size_t)L * g.N + x];
        if (n < 255) ++n;
      }
      ++sim.computed;
    }
  }
};

}  // namespace

swept_status check_schedule(swept_handle* h, int64_t nsteps, int64_t* computed) {
  Sim sim;
  sim.g = h->g;
  const Geom& g = sim.g;
  sim.n_sub = nsteps * g.S;
  if ((double)(sim.n_sub + 1) * (double)g.N > 4e8) {
    h->err = "schedule check too large (n_sub * N > 4e8)";
    return SWEPT_EINVAL;
  }
  sim.u.resize((size_t)g.C * g.N);
  for (int c = 0; c < g.C; ++c)
    for (int64_t x = 0; x < g.N; ++x) sim.u[(size_t)(c * g.N + x)] = Tag{x, 0};
  for (int b = 0; b < 2; ++b) {
    sim.e[b].assign((size_t)g.nt * g.E, Tag{});
    sim.ae[b].assign((size_t)g.nt * g.E, Access{});
  }
  sim.au.assign((size_t)g.C * g.N, Access{});
  sim.count.assign((size_t)(sim.n_sub + 1) * g.N, 0);
  const int64_t q = sim.n_sub / g.h;
  for_each_launch(g, sim.n_sub, [&](int kind, int odd, int mode, int hh, int64_t pass) {
    ++sim.stamp;
    // absolute tier of local tier 0 of this launch
    const int64_t base = pass >= 0 ? (kind == 0 ? 0 : (pass - 1) * (int64_t)g.h) : q * (int64_t)g.h;
    for (int64_t b = 0; b < g.nt && sim.err.empty(); ++b) {
      if (kind == 0) {
        const int out = pass >= 0 ? (int)(pass & 1) : 0;
        HostCtx cx(sim, b, base, 0, out);
        run_up(cx, g, b, hh, mode == MODE_GAP);
      } else {
        const int in = pass >= 1 ? (int)((pass - 1) & 1) : 0;
        const int out = pass >= 1 ? (int)(pass & 1) : 1;
        HostCtx cx(sim, b, base, in, out);
        run_diamond(cx, g, b, odd, mode, hh);
      }
    }
  });
  if (sim.err.empty()) {
    for (int c = 0; c < g.C && sim.err.empty(); ++c)
      for (int64_t x = 0; x < g.N; ++x) {
        const Tag t = sim.u[(size_t)(c * g.N + x)];
        if (t.x != x || t.lvl != sim.n_sub) {
          char b[160];
          snprintf(b, sizeof b, "final state at point %lld holds (point %lld, tier %lld), expected tier %lld",
                   (long long)x, (long long)t.x, (long long)t.lvl, (long long)sim.n_sub);
          sim.fail(b);
          break;
        }
      }
  }
  if (sim.err.empty()) {
    for (int64_t L = 1; L <= sim.n_sub && sim.err.empty(); ++L)
      for (int64_t x = 0; x < g.N; ++x) {
        const uint8_t n = sim.count[(size_t)L * g.N + x];
        if (n != 1) {
          char b[160];
          snprintf(b, sizeof b, "point %lld of tier %lld computed %d times", (long long)x, (long long)L, (int)n);
          sim.fail(b);
          break;
        }
      }
  }
  if (computed) *computed = sim.computed;
  if (!sim.err.empty()) {
    h->err = sim.err;
    return SWEPT_EDEVICE;
  }
  return SWEPT_OK;
}

}  // namespace swept
