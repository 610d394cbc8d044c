// cts_host.cpp -- pure host logic of the scheduler: the unit planner, the
// first-fit carrier arena and the drift-time estimate.  No CUDA here, so
// these are testable without a device (see include/cts_host.h).
#include "cts_host_impl.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <climits>
#include <cstring>
#include <map>
#include <vector>

#include "cts_host.h"

namespace cts {

// ---------------------------------------------------------------------------
// Unit planner (a stream-K style partition).  The pair work of one step is
// the sequence of i-tiles (tile_i carriers of one species of one slot, each
// against all n sources of its slot); its total cost W = sum ni * n is cut
// into G equal contiguous shares, one per persistent CTA, at j granularity
// (rounded to multiples of 4 sources).  A tile cut by a share boundary is
// computed in several segments whose partial sums are combined by the CTA
// that finishes last, so every CTA gets the same number of pairs (to within
// 4 * tile_i) and no dynamic queue is needed.
// ---------------------------------------------------------------------------
namespace {
struct Tile {
  int32_t slot, spec, i0, ni, n;
  double c0;  // cumulative cost before the tile
};
}  // namespace

int plan_units(const int32_t* n_h, const int32_t* n_e, int n_slots, int tile_i, int grid,
               bool allow_split, int max_units, int64_t partial_cap, std::vector<UnitPlan>* out,
               std::vector<int32_t>* cta_begin, int64_t* partial_floats, bool dynamic,
               bool slot_major) {
  out->clear();
  cta_begin->assign((size_t)std::max(grid, 0) + 1, 0);
  *partial_floats = 0;
  if (tile_i <= 0 || grid <= 0 || n_slots < 0 || max_units <= 0) return -1;
  std::vector<Tile> tiles;
  std::vector<double> slot_c0((size_t)std::max(n_slots, 0), 0.0), slot_w(slot_c0);
  double W = 0.0;
  for (int s = 0; s < n_slots; ++s) {
    const int nh = std::max(n_h[s], 0), ne = std::max(n_e[s], 0);
    slot_c0[s] = W;
    slot_w[s] = (double)(nh + ne) * (double)(nh + ne);
    if (nh <= 0) continue;  // an event with no hole is finished
    const int n = nh + ne;
    for (int spec = 0; spec < 2; ++spec) {
      const int ni_tot = spec ? ne : nh;
      for (int i0 = 0; i0 < ni_tot; i0 += tile_i) {
        const int ni = std::min(tile_i, ni_tot - i0);
        tiles.push_back(Tile{s, spec, i0, ni, n, W});
        W += (double)ni * (double)n;
      }
    }
  }
  if ((int64_t)tiles.size() > max_units) return -2;
  if (tiles.empty()) return 0;
  auto emit = [&](const Tile& t, int j0, int j1, int split, int nsplit, int iblock, int pbase) {
    UnitPlan u;
    u.slot = t.slot;
    u.spec = t.spec;
    u.i0 = t.i0;
    u.ni = t.ni;
    u.j0 = j0;
    u.j1 = j1;
    u.split = split;
    u.nsplit = nsplit;
    u.iblock = iblock;
    u.pbase = pbase;
    out->push_back(u);
  };
  // CTAs that get work: enough that each share holds >= kPlanMinPairs pairs.
  const int g_eff = allow_split ? (int)std::max(1.0, std::min((double)grid,
                                                             std::floor(W / (kPlanMinJ * (double)tile_i))))
                                : grid;
  if (dynamic && !allow_split) dynamic = false;
  if (!dynamic && (!allow_split || g_eff == 1)) {
    // whole tiles, longest-processing-time first onto the least loaded CTA
    std::vector<int> order(tiles.size());
    for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
      return (double)tiles[a].ni * tiles[a].n > (double)tiles[b].ni * tiles[b].n;
    });
    std::vector<double> load((size_t)grid, 0.0);
    std::vector<std::vector<int>> per((size_t)grid);
    for (int t : order) {
      const int g = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      load[g] += (double)tiles[t].ni * tiles[t].n;
      per[g].push_back(t);
    }
    for (int g = 0; g < grid; ++g) {
      (*cta_begin)[g] = (int32_t)out->size();
      for (int t : per[g]) emit(tiles[t], 0, tiles[t].n, 0, 1, -1, 0);
    }
    (*cta_begin)[grid] = (int32_t)out->size();
    return 0;
  }
  if (dynamic) {
    // Guided pieces for a dynamic queue (factoring): piece sizes halve batch
    // by batch toward the end of the step's work (w/2 ... w/64), all sorted
    // largest first;
    // CTAs that run faster simply take more of them.
    const double w = W / grid;
    int iblock = 0;
    int64_t pfl = 0;
    int64_t reserved = 0;  // partial-sum floats of the tiles split so far
    struct Piece { int t, j0, j1, k, ns; };
    std::vector<Piece> pieces;
    for (size_t ti = 0; ti < tiles.size(); ++ti) {
      const Tile& t = tiles[ti];
      // position of the tile in the work the schedule drains: the whole step,
      // or (slot_major) its own slot's step
      const double f = slot_major ? (t.c0 - slot_c0[t.slot]) / slot_w[t.slot] : t.c0 / W;
      // factoring: the first half of the work in pieces of w/2, the next
      // quarter in w/4, ... down to w/64
      const double target = f < 0.5 ? 0.5 * w : f < 0.75 ? 0.25 * w : f < 0.875 ? 0.125 * w
                          : f < 0.9375 ? w / 16.0 : f < 0.96875 ? w / 32.0 : w / 64.0;
      int ns = (int)std::max(1.0, std::ceil((double)t.ni * t.n / target));
      ns = std::min({ns, std::max(1, t.n / kPlanDynMinJ), kPlanDynMaxPieces});
      // each piece of a split tile needs its own 3 * tile_i partial sums (the
      // tile's pieces are added in piece order): run the tile whole once the
      // buffer is spoken for
      if (ns > 1) {
        if (reserved + (int64_t)3 * tile_i * ns > partial_cap) ns = 1;
        else reserved += (int64_t)3 * tile_i * ns;
      }
      for (int k = 0; k < ns; ++k) {
        int j0 = (int)((int64_t)t.n * k / ns) & ~3, j1 = k + 1 == ns ? t.n : (int)((int64_t)t.n * (k + 1) / ns) & ~3;
        if (k > 0) j0 = pieces.back().j1;
        pieces.push_back(Piece{(int)ti, j0, j1, k, ns});
      }
      if (ns > 1) {
        for (int k = 0; k < ns; ++k) pieces[pieces.size() - ns + k].ns = ns;
      }
    }
    // partial-sum regions per split tile
    std::vector<int> pb(tiles.size(), 0), ib(tiles.size(), -1);
    for (const Piece& pc : pieces)
      if (pc.ns > 1 && pc.k == 0) {
        pb[pc.t] = (int)pfl;
        ib[pc.t] = iblock++;
        pfl += (int64_t)3 * tile_i * pc.ns;
      }
    std::stable_sort(pieces.begin(), pieces.end(), [&](const Piece& a, const Piece& b) {
      if (slot_major && tiles[a.t].slot != tiles[b.t].slot)
        return tiles[a.t].slot < tiles[b.t].slot;
      return (double)tiles[a.t].ni * (a.j1 - a.j0) > (double)tiles[b.t].ni * (b.j1 - b.j0);
    });
    if ((int64_t)pieces.size() > max_units) return -2;
    for (const Piece& pc : pieces)
      emit(tiles[pc.t], pc.j0, pc.j1, pc.k, pc.ns, ib[pc.t], pb[pc.t]);
    for (int g = 0; g <= grid; ++g) (*cta_begin)[g] = g == grid ? (int32_t)out->size() : 0;
    *partial_floats = pfl;
    return 0;
  }
  const double share = W / g_eff;
  // j boundary inside tile t for cumulative cost x (multiple of 4, clamped)
  auto bnd = [&](const Tile& t, double x) -> int {
    const double j = std::ceil((x - t.c0) / t.ni - 1e-9);
    int jj = (int)std::max(0.0, std::min((double)t.n, j));
    jj = (jj + 3) & ~3;
    return std::min(jj, t.n);
  };
  int iblock = 0;
  int64_t pfl = 0;
  int next_cta = 0;
  for (const Tile& t : tiles) {
    const double c1 = t.c0 + (double)t.ni * t.n;
    int g_first = (int)std::floor(t.c0 / share);
    int g_last = (int)std::floor((c1 - 1e-6) / share);
    g_first = std::min(std::max(g_first, 0), g_eff - 1);
    g_last = std::min(std::max(g_last, g_first), g_eff - 1);
    // segments [bnd(g*share), bnd((g+1)*share)) for g in [g_first, g_last]
    std::vector<std::pair<int, std::pair<int, int>>> segs;
    for (int g = g_first; g <= g_last; ++g) {
      const int j0 = g == g_first ? 0 : bnd(t, g * share);
      const int j1 = g == g_last ? t.n : bnd(t, (g + 1) * share);
      if (j1 > j0) segs.push_back({g, {j0, j1}});
    }
    const int ns = (int)segs.size();
    int pbase = 0, ib = -1;
    if (ns > 1) {
      if (pfl + (int64_t)3 * tile_i * ns > partial_cap) {
        // no room for partial sums: run the tile whole on its first CTA
        segs.assign(1, {segs.front().first, {0, t.n}});
      } else {
        pbase = (int)pfl;
        ib = iblock++;
        pfl += (int64_t)3 * tile_i * ns;
      }
    }
    const int nsf = (int)segs.size();
    for (int k = 0; k < nsf; ++k) {
      const int g = segs[k].first;
      while (next_cta <= g) (*cta_begin)[next_cta++] = (int32_t)out->size();
      emit(t, segs[k].second.first, segs[k].second.second, k, nsf, ib, pbase);
    }
  }
  while (next_cta <= grid) (*cta_begin)[next_cta++] = (int32_t)out->size();
  if ((int64_t)out->size() > max_units) return -2;
  *partial_floats = pfl;
  return 0;
}

// ---------------------------------------------------------------------------
// Symmetric planner.  Each unordered pair of carriers of an event is one
// term of Eq. 4 for both carriers (Newton's third law), so a step needs
// N(N-1)/2 pair evaluations.  With tiles of 64 carriers per species range and
// I blocks of 4 tiles, the pairs are covered exactly once by the (block b,
// tile g) combinations with
//   same species:  g >= first tile of b (tiles of b itself: the pairs of
//                  tile u < g of the block, and tile g = u with itself),
//   b holes, g electrons: every g,
// and a unit is a rectangle blocks [ib0, ib1) x tiles [jt0, jt1) of them (the
// kernel skips combinations of a rectangle below the diagonal).  Every unit
// writes one partial field per tile of its blocks and per tile of its J
// range; a tile's field is the sum of its partials in unit order.
// ---------------------------------------------------------------------------
void sym_shape(int ntiles, int* rb, int* rj) {
  // small events: short units, so that each step of an event is spread over
  // many warps; large events: fewer, larger units (fewer partial fields)
  if (ntiles <= 160) {
    *rb = 1;
    *rj = 8;
  } else if (ntiles <= 640) {
    *rb = 2;
    *rj = 16;
  } else {
    *rb = 8;
    *rj = 16;
  }
}

namespace {

// The plan of one slot with th hole tiles and te electron tiles: its pair
// units longest first (partials numbered from 0), its update units, and the
// partial lists of its tiles in unit order.
SymSlotTemplate sym_slot_template(int th, int te) {
  constexpr int B = kSymPlanTpb;
  SymSlotTemplate T;
  int rb, rj;
  sym_shape(th + te, &rb, &rj);
  std::vector<SymUnitPlan> su;
  std::vector<int64_t> work;
  auto rows = [&](int spec_i, int nti, int spec_j, int ntj, bool same) {
    const int nb = (nti + B - 1) / B;
    for (int b0 = 0; b0 < nb; b0 += rb) {
      const int b1 = std::min(b0 + rb, nb);
      for (int g = same ? b0 * B : 0; g < ntj; g += rj) {
        const int g1 = std::min(g + rj, ntj);
        int64_t w = 0;  // tile pairs evaluated
        for (int b = b0; b < b1; ++b) {
          const int lo = same ? std::max(g, b * B) : g;
          w += (int64_t)std::max(g1 - lo, 0) * std::min(B, nti - b * B);
        }
        su.push_back(SymUnitPlan{0, spec_i, spec_j, b0, b1, g, g1, 0, 0, 0, 0, 0});
        work.push_back(w);
      }
    }
  };
  rows(0, th, 0, th, true);
  if (te > 0) {
    rows(0, th, 1, te, false);
    rows(1, te, 1, te, true);
  }
  // the slot's pair units longest first; its first unit does the
  // bookkeeping of a launch's first step
  std::vector<int> order(su.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return work[a] > work[b]; });
  for (size_t k = 0; k < order.size(); ++k) {
    SymUnitPlan u = su[order[k]];
    u.duty = k == 0;
    u.p_i = (int32_t)T.n_partials;
    T.n_partials += (int64_t)(u.ib1 - u.ib0) * B;
    u.p_j = (int32_t)T.n_partials;
    T.n_partials += u.jt1 - u.jt0;
    T.pair.push_back(u);
  }
  // update units: a few tiles each (at most 64 units a slot)
  const int nt = th + te;
  const int tu = std::max(kSymPlanUpdateTiles, (nt + 63) / 64);
  for (int t = 0; t < nt; t += tu)
    T.upd.push_back(SymUnitPlan{0, 0, 0, 0, 0, t, std::min(t + tu, nt), 0, 0, 0, 1,
                                (int32_t)T.pair.size()});
  // per-tile partial lists, in unit order
  auto each = [&](const SymUnitPlan& u, auto&& f) {
    const int nti = u.spec_i ? te : th;
    const int ti0 = u.spec_i ? th : 0, tj0 = u.spec_j ? th : 0;
    for (int b = u.ib0; b < u.ib1; ++b)
      for (int q = 0; q < B && b * B + q < nti; ++q) f(ti0 + b * B + q, u.p_i + (b - u.ib0) * B + q);
    for (int g = u.jt0; g < u.jt1; ++g) f(tj0 + g, u.p_j + (g - u.jt0));
  };
  T.lcnt.assign((size_t)nt, 0);
  for (const SymUnitPlan& u : T.pair) each(u, [&](int t, int) { T.lcnt[(size_t)t]++; });
  std::vector<int32_t> start((size_t)nt, 0), fill((size_t)nt, 0);
  int64_t acc = 0;
  for (int t = 0; t < nt; ++t) {
    start[(size_t)t] = (int32_t)acc;
    acc += T.lcnt[(size_t)t];
  }
  T.lists.assign((size_t)acc, -1);
  for (const SymUnitPlan& u : T.pair)
    each(u, [&](int t, int pp) { T.lists[(size_t)(start[(size_t)t] + fill[(size_t)t]++)] = pp; });
  return T;
}

}  // namespace

int plan_sym(const int32_t* n_h, const int32_t* n_e, int n_slots, int max_units, SymPlan* out) {
  out->units.clear();
  out->tiles.clear();
  out->lists.clear();
  out->slot_tile0.assign((size_t)std::max(n_slots, 0), -1);
  out->slot_ntiles.assign((size_t)std::max(n_slots, 0), 0);
  out->n_partials = 0;
  if (n_slots < 0 || max_units <= 0) return -1;
  constexpr int T = kSymPlanTile;
  std::vector<std::pair<int, const SymSlotTemplate*>> upd;  // update units still to place
  size_t upd_head = 0;
  auto place_updates = [&](const std::pair<int, const SymSlotTemplate*>& e) {
    for (SymUnitPlan u : e.second->upd) {
      u.slot = e.first;
      out->units.push_back(u);
    }
  };
  for (int s = 0; s < n_slots; ++s) {
    const int nh = std::max(n_h[s], 0), ne = std::max(n_e[s], 0);
    if (nh <= 0) continue;  // an event with no hole is finished
    const int th = (nh + T - 1) / T, te = (ne + T - 1) / T;
    auto it = out->memo.find({th, te});
    if (it == out->memo.end()) it = out->memo.emplace(std::make_pair(th, te), sym_slot_template(th, te)).first;
    const SymSlotTemplate& st = it->second;
    const int64_t pbase = out->n_partials;
    if (pbase + st.n_partials > INT32_MAX) return -2;
    const int64_t lbase = (int64_t)out->lists.size();
    out->slot_tile0[s] = (int32_t)out->tiles.size();
    out->slot_ntiles[s] = th + te;
    int64_t lp = lbase;
    for (int spec = 0, q = 0; spec < 2; ++spec) {
      const int n = spec ? ne : nh, nt = spec ? te : th;
      for (int t = 0; t < nt; ++t, ++q) {
        const int32_t lc = st.lcnt[(size_t)q];
        out->tiles.push_back(SymTilePlan{s, spec, t, std::min(T, n - T * t), (int32_t)lp, lc});
        lp += lc;
      }
    }
    const size_t l0 = out->lists.size(), nl = st.lists.size();
    out->lists.resize(l0 + nl);
    int32_t* ld = out->lists.data() + l0;
    const int32_t pb = (int32_t)pbase;
    for (size_t q = 0; q < nl; ++q) ld[q] = st.lists[q] + pb;
    const size_t u0 = out->units.size(), nu = st.pair.size();
    out->units.resize(u0 + nu);
    SymUnitPlan* ud = out->units.data() + u0;
    for (size_t q = 0; q < nu; ++q) {
      ud[q] = st.pair[q];
      ud[q].slot = s;
      ud[q].p_i += pb;
      ud[q].p_j += pb;
    }
    out->n_partials += st.n_partials;
    // a slot's update units follow the pair units of kSymPlanUpdateLag more
    // slots, so that its pair work is usually done when they are taken
    upd.emplace_back(s, &st);
    if (upd.size() - upd_head > (size_t)kSymPlanUpdateLag) place_updates(upd[upd_head++]);
    if ((int64_t)out->units.size() > max_units) return -2;
  }
  for (; upd_head < upd.size(); ++upd_head) place_updates(upd[upd_head]);
  if ((int64_t)out->units.size() > max_units) return -2;
  return 0;
}

// ---------------------------------------------------------------------------
// First-fit arena with coalescing free list.
// ---------------------------------------------------------------------------
ArenaAllocator::ArenaAllocator(int64_t capacity) : capacity_(capacity) {
  if (capacity > 0) free_[0] = capacity;
}

int64_t ArenaAllocator::alloc(int64_t n) {
  if (n <= 0) n = 1;
  n = (n + kArenaAlign - 1) / kArenaAlign * kArenaAlign;
  for (auto it = free_.begin(); it != free_.end(); ++it) {
    if (it->second >= n) {
      const int64_t off = it->first, len = it->second;
      free_.erase(it);
      if (len > n) free_[off + n] = len - n;
      used_[off] = n;
      in_use_ += n;
      return off;
    }
  }
  return -1;
}

void ArenaAllocator::release(int64_t off) {
  auto u = used_.find(off);
  if (u == used_.end()) return;
  int64_t start = off, len = u->second;
  used_.erase(u);
  in_use_ -= len;
  auto next = free_.lower_bound(start);
  if (next != free_.end() && next->first == start + len) {
    len += next->second;
    next = free_.erase(next);
  }
  if (next != free_.begin()) {
    auto prev = std::prev(next);
    if (prev->first + prev->second == start) {
      start = prev->first;
      len += prev->second;
      free_.erase(prev);
    }
  }
  free_[start] = len;
}

int64_t ArenaAllocator::largest_free() const {
  int64_t best = 0;
  for (const auto& kv : free_) best = std::max(best, kv.second);
  return best;
}

// Drift-only transit time of a hole, integrated with the midpoint rule over
// 256 cells: t = integral dz / (mu(E(z)) E(z)), the quantity of Eq. 9.
double estimate_steps(double H, double Vb, double Vd, double mu0_cm2, double vsat_cms,
                      double beta, double dt_ps, double depth) {
  if (!(H > 0) || !(dt_ps > 0)) return 0.0;
  const double mu0 = mu0_cm2 * 0.1, vsat = vsat_cms * 1e-5;
  const double z0 = std::min(std::max(H - depth, 0.0), H);
  const int cells = 256;
  double t = 0.0;
  for (int c = 0; c < cells; ++c) {
    const double z = (c + 0.5) * z0 / cells;
    const double E = (Vb - Vd) / H + 2.0 * Vd * (H - z) / (H * H);
    if (!(E > 0)) return 1e9;
    const double mu = mu0 / std::pow(1.0 + std::pow(mu0 * E / vsat, beta), 1.0 / beta);
    t += (z0 / cells) / (mu * E);
  }
  return t / (dt_ps * 1e-3);
}

// ---------------------------------------------------------------------------
// Fano-distributed carrier count (Sec. 4.2): mean E / 3.62 eV, variance F
// times the mean, drawn as round(mean + sqrt(F mean) g) from the event's
// counter-based stream.  Philox4x32-10 (Salmon et al., SC'11) and the
// Box-Muller cosine branch, written for the host.
// ---------------------------------------------------------------------------
namespace {
struct Philox {
  uint32_t c[4];
  uint32_t k[2];
  void rounds() {
    for (int r = 0; r < 10; ++r) {
      const uint64_t a = (uint64_t)0xD2511F53u * c[0];
      const uint64_t b = (uint64_t)0xCD9E8D57u * c[2];
      const uint32_t x0 = (uint32_t)(b >> 32) ^ c[1] ^ k[0];
      const uint32_t x2 = (uint32_t)(a >> 32) ^ c[3] ^ k[1];
      c[1] = (uint32_t)b;
      c[3] = (uint32_t)a;
      c[0] = x0;
      c[2] = x2;
      k[0] += 0x9E3779B9u;
      k[1] += 0xBB67AE85u;
    }
  }
};
constexpr uint32_t kPurposeFano = 2;
constexpr double kEvPerPair = 3.62;
}  // namespace

int fano_pairs(uint64_t seed, uint64_t event_id, double energy_keV, double fano) {
  const double mean = energy_keV * 1000.0 / kEvPerPair;
  if (!(fano > 0.0)) return (int)std::llround(mean);
  Philox g{{0u, 0u, (uint32_t)event_id, (uint32_t)(event_id >> 32) ^ (kPurposeFano << 28)},
           {(uint32_t)seed, (uint32_t)(seed >> 32)}};
  g.rounds();
  const double u0 = ((double)(g.c[0] >> 9) + 0.5) / 8388608.0;
  const double u1 = ((double)(g.c[1] >> 9) + 0.5) / 8388608.0;
  const double z = std::sqrt(-2.0 * std::log(u0)) * std::cos(2.0 * 3.14159265358979323846 * u1);
  const double n = std::floor(mean + std::sqrt(fano * mean) * z + 0.5);
  return n < 1.0 ? 1 : (int)n;
}

// ---------------------------------------------------------------------------
// Generalised Gaussian model of the collected cloud (Sec. 3, Eqs. 8, 10, 11).
// ---------------------------------------------------------------------------
namespace {
// profile log-likelihood of Eq. 8 at shape b, given the logs of |x| (zeros
// contribute nothing to the sum of |x|^b and are passed as -inf)
double ggd_profile(const std::vector<double>& lx, double b, double* alpha) {
  double sum = 0.0;
  for (double l : lx) sum += std::exp(b * l);
  const double n = (double)lx.size();
  const double a = std::pow(b * sum / n, 1.0 / b);
  *alpha = a;
  return n * (std::log(b / (2.0 * a)) - std::lgamma(1.0 / b) - 1.0 / b);
}

// solve the k x k system m x = r by Gaussian elimination with partial pivoting
bool solve_small(std::vector<double> m, std::vector<double> r, int k, double* x) {
  for (int c = 0; c < k; ++c) {
    int piv = c;
    for (int i = c + 1; i < k; ++i)
      if (std::fabs(m[i * k + c]) > std::fabs(m[piv * k + c])) piv = i;
    if (!(std::fabs(m[piv * k + c]) > 0.0)) return false;
    if (piv != c) {
      for (int j = 0; j < k; ++j) std::swap(m[c * k + j], m[piv * k + j]);
      std::swap(r[c], r[piv]);
    }
    for (int i = c + 1; i < k; ++i) {
      const double f = m[i * k + c] / m[c * k + c];
      for (int j = c; j < k; ++j) m[i * k + j] -= f * m[c * k + j];
      r[i] -= f * r[c];
    }
  }
  for (int c = k - 1; c >= 0; --c) {
    double v = r[c];
    for (int j = c + 1; j < k; ++j) v -= m[c * k + j] * x[j];
    x[c] = v / m[c * k + c];
  }
  return true;
}
}  // namespace

double beta_of_t(const double* p, double t) {
  const double u = t - p[1];
  return 2.0 + (u > 0.0 ? p[0] * std::pow(u, p[2]) : 0.0) + p[3] * std::exp(p[4] * t);
}

double alpha_of_t(const double* p, double t) {
  return p[0] + p[1] * std::sqrt(t) + p[2] * t + p[3] * t * t;
}

int fit_ggd(const double* x, int64_t n, double* alpha, double* beta) {
  if (!x || n < 2) return -1;
  std::vector<double> lx((size_t)n);
  bool any = false;
  for (int64_t i = 0; i < n; ++i) {
    const double v = std::fabs(x[i]);
    if (!std::isfinite(v)) return -1;
    any |= v > 0.0;
    lx[(size_t)i] = v > 0.0 ? std::log(v) : -INFINITY;
  }
  if (!any) return -1;
  // golden-section search of the profile likelihood over log(beta)
  const double r = 0.6180339887498949;
  double lo = std::log(0.3), hi = std::log(20.0), a = 0.0;
  double x1 = hi - r * (hi - lo), x2 = lo + r * (hi - lo);
  double f1 = ggd_profile(lx, std::exp(x1), &a), f2 = ggd_profile(lx, std::exp(x2), &a);
  while (hi - lo > 1e-12) {
    if (f1 > f2) {
      hi = x2;
      x2 = x1;
      f2 = f1;
      x1 = hi - r * (hi - lo);
      f1 = ggd_profile(lx, std::exp(x1), &a);
    } else {
      lo = x1;
      x1 = x2;
      f1 = f2;
      x2 = lo + r * (hi - lo);
      f2 = ggd_profile(lx, std::exp(x2), &a);
    }
  }
  *beta = std::exp(0.5 * (lo + hi));
  ggd_profile(lx, *beta, alpha);
  return 0;
}

int fit_alpha_t(const double* t, const double* y, const double* w, int n, double* p) {
  if (n < 4) return -1;
  std::vector<double> m(16, 0.0), r(4, 0.0);
  for (int i = 0; i < n; ++i) {
    if (!(t[i] >= 0.0)) return -1;
    const double wi = w ? w[i] * w[i] : 1.0;
    const double f[4] = {1.0, std::sqrt(t[i]), t[i], t[i] * t[i]};
    for (int a = 0; a < 4; ++a) {
      r[a] += wi * f[a] * y[i];
      for (int b = 0; b < 4; ++b) m[a * 4 + b] += wi * f[a] * f[b];
    }
  }
  return solve_small(m, r, 4, p) ? 0 : -1;
}

// Levenberg-Marquardt (Marquardt 1963) for Eq. 11 from the starting point p,
// with forward-difference derivatives; sigma weights the residuals.
int fit_beta_t(const double* t, const double* y, const double* sigma, int n, double* p) {
  if (n < 5) return -1;
  auto cost = [&](const double* q) {
    double c = 0.0;
    for (int i = 0; i < n; ++i) {
      const double e = (y[i] - beta_of_t(q, t[i])) / (sigma ? sigma[i] : 1.0);
      c += e * e;
    }
    return c;
  };
  double c0 = cost(p), lambda = 1e-3;
  if (!std::isfinite(c0)) return -1;
  std::vector<double> J((size_t)n * 5), e((size_t)n);
  for (int it = 0; it < 500; ++it) {
    for (int i = 0; i < n; ++i) {
      const double s = sigma ? sigma[i] : 1.0;
      const double f0 = beta_of_t(p, t[i]);
      e[(size_t)i] = (y[i] - f0) / s;
      for (int k = 0; k < 5; ++k) {
        double q[5] = {p[0], p[1], p[2], p[3], p[4]};
        const double h = 1e-7 * std::max(1.0, std::fabs(p[k]));
        q[k] += h;
        J[(size_t)i * 5 + k] = (beta_of_t(q, t[i]) - f0) / (h * s);
      }
    }
    std::vector<double> A(25, 0.0), g(5, 0.0);
    for (int i = 0; i < n; ++i)
      for (int a = 0; a < 5; ++a) {
        g[a] += J[(size_t)i * 5 + a] * e[(size_t)i];
        for (int b = 0; b < 5; ++b) A[a * 5 + b] += J[(size_t)i * 5 + a] * J[(size_t)i * 5 + b];
      }
    bool improved = false;
    for (int tries = 0; tries < 30 && !improved; ++tries) {
      std::vector<double> M = A;
      for (int a = 0; a < 5; ++a) M[a * 5 + a] *= 1.0 + lambda;
      double d[5];
      if (solve_small(M, g, 5, d)) {
        double q[5];
        for (int k = 0; k < 5; ++k) q[k] = p[k] + d[k];
        const double c1 = cost(q);
        if (std::isfinite(c1) && c1 < c0) {
          const double rel = (c0 - c1) / std::max(c0, 1e-300);
          for (int k = 0; k < 5; ++k) p[k] = q[k];
          c0 = c1;
          lambda = std::max(lambda * 0.3, 1e-12);
          improved = true;
          if (rel < 1e-15) return 0;
          break;
        }
      }
      lambda *= 10.0;
    }
    if (!improved) return 0;  // no step lowers the cost: a minimum
  }
  return 0;
}

// ---------------------------------------------------------------------------
// Variant-table cache file: "cts-variant-table 1", the device name, the
// number of kernel variants the table was measured against, then one
// "min_pairs variant" line per entry.
// ---------------------------------------------------------------------------
int table_save(const char* path, const char* device, int32_t n_variants, const int64_t* mins,
               const int32_t* vars, int32_t n) {
  if (!path || !device || n < 0 || (n > 0 && (!mins || !vars))) return -1;
  FILE* f = std::fopen(path, "w");
  if (!f) return -3;
  bool ok = std::fprintf(f, "cts-variant-table 1\n%s\n%d %d\n", device, n_variants, n) > 0;
  for (int32_t q = 0; q < n && ok; ++q)
    ok = std::fprintf(f, "%lld %d\n", (long long)mins[q], vars[q]) > 0;
  ok = (std::fclose(f) == 0) && ok;
  return ok ? 0 : -3;
}

int table_load(const char* path, const char* device, int32_t n_variants, int64_t* mins,
               int32_t* vars, int32_t cap, int32_t* n) {
  if (!path || !device || !n || cap < 0) return -1;
  FILE* f = std::fopen(path, "r");
  if (!f) return -3;
  char line[512];
  int rc = 0;
  int nv = 0, cnt = 0;
  if (!std::fgets(line, sizeof line, f) || std::strcmp(line, "cts-variant-table 1\n") != 0) rc = -2;
  if (!rc && !std::fgets(line, sizeof line, f)) rc = -2;
  if (!rc) {
    line[std::strcspn(line, "\n")] = 0;
    if (std::strcmp(line, device) != 0) rc = -4;  // measured on another device
  }
  if (!rc && std::fscanf(f, "%d %d", &nv, &cnt) != 2) rc = -2;
  if (!rc && (nv != n_variants || cnt < 0 || cnt > cap)) rc = nv != n_variants ? -4 : -2;
  long long prev = -1;
  for (int q = 0; !rc && q < cnt; ++q) {
    long long m = 0;
    int v = 0;
    if (std::fscanf(f, "%lld %d", &m, &v) != 2 || m < 0 || m < prev || v < 1 || v > n_variants)
      rc = -2;
    else {
      mins[q] = m;
      vars[q] = v;
      prev = m;
    }
  }
  std::fclose(f);
  *n = rc ? 0 : cnt;
  return rc;
}

}  // namespace cts

extern "C" {

int cts_plan_units(const int32_t* n_h, const int32_t* n_e, int32_t n_slots, int32_t tile_i,
                   int32_t grid, int32_t allow_split, int32_t max_units, int64_t partial_cap,
                   cts_unit_t* out, int32_t* n_out, int32_t* cta_begin,
                   int64_t* partial_floats) {
  if (!n_h || !n_e || !out || !n_out || !partial_floats || !cta_begin) return -1;
  std::vector<cts::UnitPlan> units;
  std::vector<int32_t> begin;
  const int rc = cts::plan_units(n_h, n_e, n_slots, tile_i, grid, allow_split != 0, max_units,
                                 partial_cap, &units, &begin, partial_floats, allow_split >= 2,
                                 allow_split == 3);
  if (rc != 0) return rc;
  for (size_t k = 0; k < units.size(); ++k) {
    const cts::UnitPlan& u = units[k];
    out[k] = cts_unit_t{u.slot, u.spec, u.i0, u.ni, u.j0, u.j1, u.split, u.nsplit, u.iblock,
                        u.pbase};
  }
  for (size_t g = 0; g < begin.size(); ++g) cta_begin[g] = begin[g];
  *n_out = (int32_t)units.size();
  return 0;
}

int cts_plan_sym(const int32_t* n_h, const int32_t* n_e, int32_t n_slots, int32_t max_units,
                 cts_sym_unit_t* units, int32_t* n_units, cts_sym_tile_t* tiles,
                 int32_t tiles_cap, int32_t* n_tiles, int32_t* lists, int64_t lists_cap,
                 int64_t* n_partials) {
  if (!n_h || !n_e || !units || !n_units || !tiles || !n_tiles || !lists || !n_partials ||
      n_slots < 0 || max_units <= 0 || tiles_cap < 0 || lists_cap < 0)
    return -1;
  cts::SymPlan plan;
  const int rc = cts::plan_sym(n_h, n_e, n_slots, max_units, &plan);
  if (rc != 0) return rc;
  if ((int64_t)plan.tiles.size() > tiles_cap || (int64_t)plan.lists.size() > lists_cap) return -2;
  for (size_t k = 0; k < plan.units.size(); ++k) {
    const cts::SymUnitPlan& u = plan.units[k];
    units[k] = cts_sym_unit_t{u.slot, u.spec_i, u.spec_j, u.ib0, u.ib1, u.jt0, u.jt1,
                              u.p_i, u.p_j, u.duty, u.kind, u.npair};
  }
  for (size_t k = 0; k < plan.tiles.size(); ++k) {
    const cts::SymTilePlan& t = plan.tiles[k];
    tiles[k] = cts_sym_tile_t{t.slot, t.spec, t.tile, t.n, t.lptr, t.lcnt};
  }
  for (size_t k = 0; k < plan.lists.size(); ++k) lists[k] = plan.lists[k];
  *n_units = (int32_t)plan.units.size();
  *n_tiles = (int32_t)plan.tiles.size();
  *n_partials = plan.n_partials;
  return 0;
}

int cts_arena_replay(int64_t capacity, const int64_t* ops, int32_t n_ops, int64_t* result) {
  if (!ops || !result || capacity < 0) return -1;
  cts::ArenaAllocator a(capacity);
  for (int k = 0; k < n_ops; ++k) {
    if (ops[k] > 0) {
      result[k] = a.alloc(ops[k]);
    } else {
      const int64_t which = -ops[k] - 1;
      if (which < 0 || which >= k) return -1;
      if (result[which] >= 0) a.release(result[which]);
      result[k] = 0;
    }
  }
  return 0;
}

int cts_fano_pairs(uint64_t seed, uint64_t event_id, double energy_keV, double fano,
                   int32_t* n_pairs) {
  if (!n_pairs || !(energy_keV > 0.0) || !(fano >= 0.0)) return -1;
  *n_pairs = cts::fano_pairs(seed, event_id, energy_keV, fano);
  return 0;
}

int cts_fit_ggd(const double* x, int64_t n, double* alpha, double* beta) {
  if (!alpha || !beta) return -1;
  return cts::fit_ggd(x, n, alpha, beta);
}

int cts_fit_alpha_t(const double* t, const double* alpha, const double* w, int32_t n,
                    double* p_alpha) {
  if (!t || !alpha || !p_alpha) return -1;
  return cts::fit_alpha_t(t, alpha, w, n, p_alpha);
}

int cts_fit_beta_t(const double* t, const double* beta, const double* sigma, int32_t n,
                   double* p_beta) {
  if (!t || !beta || !p_beta) return -1;
  return cts::fit_beta_t(t, beta, sigma, n, p_beta);
}

int cts_ggd_params_at(const double* p_alpha, const double* p_beta, double t, double* alpha,
                      double* beta) {
  if (!p_alpha || !p_beta || !alpha || !beta || !(t >= 0.0)) return -1;
  *alpha = cts::alpha_of_t(p_alpha, t);
  *beta = cts::beta_of_t(p_beta, t);
  return (*alpha > 0.0 && *beta > 0.0) ? 0 : -2;
}

int cts_variant_table_save(const char* path, const char* device, int32_t n_variants,
                           const int64_t* min_pairs, const int32_t* variants, int32_t n) {
  return cts::table_save(path, device, n_variants, min_pairs, variants, n);
}

int cts_variant_table_load(const char* path, const char* device, int32_t n_variants,
                           int64_t* min_pairs, int32_t* variants, int32_t cap, int32_t* n) {
  return cts::table_load(path, device, n_variants, min_pairs, variants, cap, n);
}

double cts_estimate_steps(double thickness_um, double bias_V, double depletion_V, double mu0_cm2,
                          double vsat_cms, double beta, double dt_ps, double depth_um) {
  return cts::estimate_steps(thickness_um, bias_V, depletion_V, mu0_cm2, vsat_cms, beta, dt_ps,
                             depth_um);
}

}  // extern "C"
