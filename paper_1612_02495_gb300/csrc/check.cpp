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
// For a slab of a grid split over ranks (swept_slab_check and the per-rank
// swept_slab_sym_* replay) each rank's blocks run over that rank's own state
// array and edge buffers, and the transfers of slab_xfers move tags between
// the ranks' buffers; the same invariants are checked over all ranks.
// For a persistent handle the replay runs the persistent kernel's item queue
// instead of launches.  Its blocks order themselves only through the waits of
// persist_deps, so the check there is on the happens-before relation those
// waits create: every read of a global location must happen after the item
// that wrote it, and every write after the location's previous writer and
// every item that read that earlier value.
#include <stdio.h>

#include <algorithm>
#include <string>
#include <vector>

#include "runtime.h"
#include "slab_plan.h"
#include "swept_phases.cuh"
#include "swept_slab.h"

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

struct HbLoc {  // per global location, persistent mode
  int64_t writer = -1;           // item that wrote the current value (-1: the initial state)
  std::vector<int64_t> readers;  // items that read the current value
};

enum Buf { BUF_U = 0, BUF_E0 = 1, BUF_E1 = 2 };

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
  // persistent mode: item ancestors (bitsets over item ids) and per-location history
  bool hb_mode = false;
  std::vector<std::vector<uint64_t>> anc;
  std::vector<HbLoc> hb[3];

  void fail(const std::string& m) {
    if (err.empty()) err = m;
  }
  bool before(int64_t a, int64_t b) const { return a == b || ((anc[(size_t)b][(size_t)(a >> 6)] >> (a & 63)) & 1); }
  void note(Buf buf, size_t i, int64_t block, bool write, const char* what) {
    if (hb_mode) return note_hb(buf, i, block, write, what);
    std::vector<Access>& a = buf == BUF_U ? au : ae[buf - BUF_E0];
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
  // `block` is the item id in persistent mode
  void note_hb(Buf buf, size_t i, int64_t item, bool write, const char* what) {
    HbLoc& x = hb[buf][i];
    char b[200];
    if (x.writer >= 0 && !before(x.writer, item)) {
      snprintf(b, sizeof b, "item %lld %s %s[%zu] written by item %lld, which it does not wait for", (long long)item,
               write ? "overwrites" : "reads", what, i, (long long)x.writer);
      return fail(b);
    }
    if (!write) {
      if (x.readers.empty() || x.readers.back() != item) x.readers.push_back(item);
      return;
    }
    for (int64_t r : x.readers)
      if (!before(r, item)) {
        snprintf(b, sizeof b, "item %lld overwrites %s[%zu] that item %lld reads, without waiting for it",
                 (long long)item, what, i, (long long)r);
        return fail(b);
      }
    x.writer = item;
    x.readers.clear();
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
    sim.note(BUF_U, i, block, false, "u");
    cell(r, c, j) = sim.u[i];
  }
  void store_u(int r, int c, int j, int64_t x) {
    const size_t i = (size_t)(c * g.N + wrap_n(x, g.N));
    sim.note(BUF_U, i, block, true, "u");
    const Tag t = cell(r, c, j);
    if (t.x != wrap_n(x, g.N)) sim.fail("store_u writes a value of another point");
    sim.u[i] = t;
  }
  void load_edge(int r, int c, int j, int64_t e) {
    if (e < 0 || (size_t)e >= sim.e[ein].size()) return sim.fail("edge index out of range");
    sim.note(ein == 0 ? BUF_E0 : BUF_E1, (size_t)e, block, false, "edges");
    cell(r, c, j) = sim.e[ein][(size_t)e];
  }
  void store_edge(int r, int c, int j, int64_t e) {
    if (e < 0 || (size_t)e >= sim.e[eout].size()) return sim.fail("edge index out of range");
    sim.note(eout == 0 ? BUF_E0 : BUF_E1, (size_t)e, block, true, "edges");
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

// final state and exactly-once checks shared by both replays
void final_checks(Sim& sim) {
  const Geom& g = sim.g;
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
}

void init_sim(Sim& sim, const Geom& g, int64_t n_sub) {
  sim.g = g;
  sim.n_sub = n_sub;
  sim.u.resize((size_t)g.C * g.N);
  for (int c = 0; c < g.C; ++c)
    for (int64_t x = 0; x < g.N; ++x) sim.u[(size_t)(c * g.N + x)] = Tag{x, 0};
  for (int b = 0; b < 2; ++b) {
    sim.e[b].assign((size_t)edge_slots(g) * g.E, Tag{});
    sim.ae[b].assign((size_t)edge_slots(g) * g.E, Access{});
  }
  sim.au.assign((size_t)g.C * g.N, Access{});
  sim.count.assign((size_t)(n_sub + 1) * g.N, 0);
}

// The persistent kernel's item queue (k_swept_persist), in queue order, which
// is one order its waits allow; races are judged on the waits alone.
swept_status check_persistent(swept_handle* h, int64_t nsteps, int64_t* computed) {
  Sim sim;
  const Geom& g0 = h->g;
  init_sim(sim, g0, nsteps * g0.S);
  const Geom& g = sim.g;
  const int64_t q = sim.n_sub / g.h;
  const int rem = (int)(sim.n_sub % g.h);
  const int main_passes = q > 0 ? (int)q + 1 : 0;
  const int64_t layers = main_passes + (rem > 0 ? 2 : 0);
  const int64_t items = layers * g.nt;
  if (items > 8192) {
    h->err = "persistent schedule check too large (more than 8192 items)";
    return SWEPT_EINVAL;
  }
  sim.hb_mode = true;
  const size_t words = (size_t)((items + 63) / 64);
  sim.anc.assign((size_t)items, std::vector<uint64_t>(words, 0));
  sim.hb[BUF_U].assign((size_t)g.C * g.N, HbLoc{});
  sim.hb[BUF_E0].assign((size_t)edge_slots(g) * g.E, HbLoc{});
  sim.hb[BUF_E1].assign((size_t)edge_slots(g) * g.E, HbLoc{});
  for (int64_t it = 0; it < items && sim.err.empty(); ++it) {
    const int kp = (int)(it / g.nt);
    const int64_t b = it - (int64_t)kp * g.nt;
    int64_t dep_tile[3];
    int dep_need[3];
    const int ndep = persist_deps(g, sim.n_sub, kp, b, dep_tile, dep_need);
    for (int i = 0; i < ndep; ++i) {
      const int64_t d = (int64_t)dep_need[i] * g.nt + dep_tile[i];
      if (d < 0 || d >= it) {
        sim.fail("persistent item waits for an item that is not earlier in the queue");
        break;
      }
      auto& a = sim.anc[(size_t)it];
      const auto& ad = sim.anc[(size_t)d];
      for (size_t w = 0; w < words; ++w) a[w] |= ad[w];
      a[(size_t)(d >> 6)] |= 1ull << (d & 63);
    }
    if (!sim.err.empty()) break;
    if (kp < main_passes) {
      if (kp == 0) {
        HostCtx cx(sim, it, 0, 0, 0);
        run_up(cx, g, b, g.h, false);
      } else {
        HostCtx cx(sim, it, (int64_t)(kp - 1) * g.h, (kp - 1) & 1, kp & 1);
        run_diamond(cx, g, b, kp & 1, kp == q ? MODE_DOWN : MODE_DIAMOND, g.h);
      }
    } else if (kp == main_passes) {
      HostCtx cx(sim, it, q * g.h, 0, 0);
      run_up(cx, g, b, rem, true);
    } else {
      HostCtx cx(sim, it, q * g.h, 0, 1);
      run_diamond(cx, g, b, 1, MODE_GAP, rem);
    }
  }
  final_checks(sim);
  if (computed) *computed = sim.computed;
  if (!sim.err.empty()) {
    h->err = sim.err;
    return SWEPT_EDEVICE;
  }
  return SWEPT_OK;
}

swept_status check_schedule(swept_handle* h, int64_t nsteps, int64_t* computed) {
  if ((double)(nsteps * h->g.S + 1) * (double)h->g.N > 4e8) {
    h->err = "schedule check too large (n_sub * N > 4e8)";
    return SWEPT_EINVAL;
  }
  if (h->persistent) return check_persistent(h, nsteps, computed);
  Sim sim;
  init_sim(sim, h->g, nsteps * h->g.S);
  const Geom& g = sim.g;
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
  final_checks(sim);
  if (computed) *computed = sim.computed;
  if (!sim.err.empty()) {
    h->err = sim.err;
    return SWEPT_EDEVICE;
  }
  return SWEPT_OK;
}

}  // namespace swept

// ---------------------------------------------------------------------------
// slab replay: one rank of a grid split over ranks (slab_plan.h)
// ---------------------------------------------------------------------------
namespace swept {
namespace {

// HostCtx over a slab: the state at c ul + (x - x0), edge slots by slab_slot
struct SlabHostCtx : HostCtx {
  static constexpr bool kSlab = true;
  Slab sl;
  SlabHostCtx(Sim& s, const Slab& slab, int64_t b, int64_t base, int ei, int eo)
      : HostCtx(s, b, base, ei, eo), sl(slab) {}
  bool state_index(int c, int64_t x, size_t* out) {
    const int64_t i = x - sl.x0;
    if (i < 0 || i >= sl.ul) {
      char b[160];
      snprintf(b, sizeof b, "block %lld touches point %lld outside the slab's state array [%lld, %lld)",
               (long long)block, (long long)x, (long long)sl.x0, (long long)(sl.x0 + sl.ul));
      sim.fail(b);
      return false;
    }
    *out = (size_t)(c * sl.ul + i);
    return true;
  }
  void load_u(int r, int c, int j, int64_t x) {
    size_t i;
    if (!state_index(c, x, &i)) return;
    sim.note(BUF_U, i, block, false, "u");
    cell(r, c, j) = sim.u[i];
  }
  void store_u(int r, int c, int j, int64_t x) {
    size_t i;
    if (!state_index(c, x, &i)) return;
    sim.note(BUF_U, i, block, true, "u");
    const Tag t = cell(r, c, j);
    if (t.x != wrap_n(x, g.N)) sim.fail("store_u writes a value of another point");
    sim.u[i] = t;
  }
};

}  // namespace

// the plan and slab of swept_slab_init (slab.cu)
swept_status slab_plan(const swept_config* cfg, int rank, int nranks, Geom* g, Slab* sl, swept_handle** plan_out);

}  // namespace swept

struct swept_slab_sym {
  swept::Geom g;
  swept::Slab sl;
  int64_t n_sub = 0;
  swept::Sim sim;
};

namespace {

void set_msg(char* msg, size_t len, const std::string& m) {
  if (msg && len > 0) snprintf(msg, len, "%s", m.c_str());
}

swept_status sym_fail(swept_slab_sym* s, char* msg, size_t len) {
  set_msg(msg, len, s->sim.err);
  return SWEPT_EDEVICE;
}

}  // namespace

extern "C" {

swept_status swept_slab_sym_init(const swept_config* cfg, int32_t rank, int32_t nranks, int64_t nsteps,
                                 swept_slab_sym** out) {
  using namespace swept;
  if (!out || nsteps < 0) return SWEPT_EINVAL;
  *out = nullptr;
  Geom g;
  Slab sl;
  const swept_status st = slab_plan(cfg, rank, nranks, &g, &sl, nullptr);
  if (st != SWEPT_OK) return st;
  const int64_t n_sub = nsteps * g.S;
  if ((double)(n_sub + 1) * (double)g.N > 4e8) return SWEPT_EINVAL;
  swept_slab_sym* s = new swept_slab_sym();
  s->g = g;
  s->sl = sl;
  s->n_sub = n_sub;
  Sim& sim = s->sim;
  sim.g = g;
  sim.n_sub = n_sub;
  const int64_t x1 = slab_end(g, sl);
  sim.u.assign((size_t)(g.C * sl.ul), Tag{});
  for (int c = 0; c < g.C; ++c)
    for (int64_t x = sl.x0; x < x1; ++x) sim.u[(size_t)(c * sl.ul + (x - sl.x0))] = Tag{x, 0};
  sim.au.assign(sim.u.size(), Access{});
  for (int b = 0; b < 2; ++b) {
    sim.e[b].assign((size_t)slab_edge_values(g, sl), Tag{});
    sim.ae[b].assign(sim.e[b].size(), Access{});
  }
  sim.count.assign((size_t)(n_sub + 1) * g.N, 0);
  *out = s;
  return SWEPT_OK;
}

swept_status swept_slab_sym_buffer(swept_slab_sym* s, int32_t region, int64_t** tags, int64_t* values) {
  if (!s || !tags || !values || region < 0 || region > 2) return SWEPT_EINVAL;
  std::vector<swept::Tag>& v = region == 2 ? s->sim.u : s->sim.e[region];
  static_assert(sizeof(swept::Tag) == 2 * sizeof(int64_t), "a tag is two int64 (point, sub-timestep)");
  *tags = reinterpret_cast<int64_t*>(v.data());
  *values = (int64_t)v.size();
  return SWEPT_OK;
}

swept_status swept_slab_sym_launch(swept_slab_sym* s, int64_t i, char* msg, size_t len) {
  using namespace swept;
  if (!s) return SWEPT_EINVAL;
  const Geom& g = s->g;
  if (i < 0 || i >= launch_total(g, s->n_sub)) return SWEPT_EINVAL;
  Sim& sim = s->sim;
  ++sim.stamp;
  const LaunchDesc d = launch_at(g, s->n_sub, i);
  const int64_t q = s->n_sub / g.h;
  const int64_t base = d.pass >= 0 ? (d.kind == 0 ? 0 : (d.pass - 1) * (int64_t)g.h) : q * (int64_t)g.h;
  for (int64_t b = s->sl.b0; b < s->sl.b0 + s->sl.nb && sim.err.empty(); ++b) {
    SlabHostCtx cx(sim, s->sl, b, base, d.ein, d.eout);
    if (d.kind == 0)
      run_up(cx, g, b, d.hh, d.mode == MODE_GAP);
    else
      run_diamond(cx, g, b, d.odd, d.mode, d.hh);
  }
  if (!sim.err.empty()) return sym_fail(s, msg, len);
  return SWEPT_OK;
}

swept_status swept_slab_sym_finish(swept_slab_sym* s, int32_t* counts, char* msg, size_t len) {
  using namespace swept;
  if (!s || !counts) return SWEPT_EINVAL;
  Sim& sim = s->sim;
  const Geom& g = s->g;
  const int64_t x1 = slab_end(g, s->sl);
  for (int c = 0; c < g.C && sim.err.empty(); ++c)
    for (int64_t x = s->sl.x0; x < x1; ++x) {
      const Tag t = sim.u[(size_t)(c * s->sl.ul + (x - s->sl.x0))];
      if (t.x != x || t.lvl != s->n_sub) {
        char b[200];
        snprintf(b, sizeof b, "final state at point %lld holds (point %lld, tier %lld), expected tier %lld",
                 (long long)x, (long long)t.x, (long long)t.lvl, (long long)s->n_sub);
        sim.fail(b);
        break;
      }
    }
  if (!sim.err.empty()) return sym_fail(s, msg, len);
  for (size_t i = 0; i < sim.count.size(); ++i) counts[i] += sim.count[i];
  return SWEPT_OK;
}

void swept_slab_sym_free(swept_slab_sym* s) { delete s; }

swept_status swept_slab_check(const swept_config* cfg, int32_t nranks, int64_t nsteps, int64_t* computed, char* msg,
                              size_t len) {
  using namespace swept;
  if (!cfg || nranks < 1 || nsteps < 0) return SWEPT_EINVAL;
  {
    // every rank's replay keeps a count per (sub-timestep, point) of the whole grid
    const int stages = cfg->scheme == SWEPT_HEAT ? 1 : 2;
    if ((double)(nsteps * stages + 1) * (double)cfg->n * (double)nranks > 2e9) {
      set_msg(msg, len, "slab check too large ((nsteps S + 1) n nranks > 2e9)");
      return SWEPT_EINVAL;
    }
  }
  std::vector<swept_slab_sym*> r((size_t)nranks, nullptr);
  auto cleanup = [&]() {
    for (auto* p : r) swept_slab_sym_free(p);
  };
  for (int k = 0; k < nranks; ++k) {
    const swept_status st = swept_slab_sym_init(cfg, k, nranks, nsteps, &r[(size_t)k]);
    if (st != SWEPT_OK) {
      cleanup();
      set_msg(msg, len, "swept_slab_sym_init failed");
      return st;
    }
  }
  const Geom& g = r[0]->g;
  const int64_t n_sub = r[0]->n_sub;
  const int64_t total = launch_total(g, n_sub);
  std::vector<std::vector<Xfer>> xs((size_t)nranks);
  for (int64_t i = 0; i < total; ++i) {
    for (int k = 0; k < nranks; ++k) {
      const swept_status st = swept_slab_sym_launch(r[(size_t)k], i, msg, len);
      if (st != SWEPT_OK) {
        cleanup();
        return st;
      }
    }
    for (int k = 0; k < nranks; ++k) {
      Xfer x[kMaxXfers];
      const int m = slab_xfers(g, r[(size_t)k]->sl, n_sub, i, x);
      xs[(size_t)k].assign(x, x + m);
    }
    // the j-th send of rank k to side p lands in the j-th receive of rank k + p from side -p
    for (int k = 0; k < nranks; ++k) {
      for (int p : {-1, +1}) {
        const int q = ((k + p) % nranks + nranks) % nranks;
        std::vector<const Xfer*> sends, recvs;
        for (const Xfer& x : xs[(size_t)k])
          if (!x.recv && x.peer == p) sends.push_back(&x);
        for (const Xfer& x : xs[(size_t)q])
          if (x.recv && x.peer == -p) recvs.push_back(&x);
        if (sends.size() != recvs.size()) {
          cleanup();
          set_msg(msg, len, "sends and receives between neighbours do not pair up");
          return SWEPT_EDEVICE;
        }
        for (size_t j = 0; j < sends.size(); ++j) {
          const Xfer& a = *sends[j];
          const Xfer& b = *recvs[j];
          std::vector<Tag>& src = a.region == 2 ? r[(size_t)k]->sim.u : r[(size_t)k]->sim.e[a.region];
          std::vector<Tag>& dst = b.region == 2 ? r[(size_t)q]->sim.u : r[(size_t)q]->sim.e[b.region];
          if (a.count != b.count || a.offset < 0 || b.offset < 0 || a.offset + a.count > (int64_t)src.size() ||
              b.offset + b.count > (int64_t)dst.size()) {
            cleanup();
            set_msg(msg, len, "a transfer's count or range does not fit its buffers");
            return SWEPT_EDEVICE;
          }
          const std::vector<Tag> tmp(src.begin() + a.offset, src.begin() + a.offset + a.count);
          std::copy(tmp.begin(), tmp.end(), dst.begin() + b.offset);
        }
      }
    }
  }
  std::vector<int32_t> counts((size_t)(n_sub + 1) * g.N, 0);
  int64_t sum = 0;
  for (int k = 0; k < nranks; ++k) {
    const swept_status st = swept_slab_sym_finish(r[(size_t)k], counts.data(), msg, len);
    if (st != SWEPT_OK) {
      cleanup();
      return st;
    }
    sum += r[(size_t)k]->sim.computed;
  }
  for (int64_t L = 1; L <= n_sub; ++L)
    for (int64_t x = 0; x < g.N; ++x)
      if (counts[(size_t)(L * g.N + x)] != 1) {
        char b[160];
        snprintf(b, sizeof b, "point %lld of tier %lld computed %d times over all ranks", (long long)x, (long long)L,
                 (int)counts[(size_t)(L * g.N + x)]);
        set_msg(msg, len, b);
        cleanup();
        return SWEPT_EDEVICE;
      }
  if (computed) *computed = sum;
  cleanup();
  set_msg(msg, len, "");
  return SWEPT_OK;
}

}  // extern "C"
