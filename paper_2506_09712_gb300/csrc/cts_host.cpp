// cts_host.cpp -- pure host logic of the scheduler: the unit planner, the
// first-fit carrier arena and the drift-time estimate.  No CUDA here, so
// these are testable without a device (see include/cts_host.h).
#include "cts_host_impl.h"

#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "cts_host.h"

namespace cts {

// ---------------------------------------------------------------------------
// Unit planner.  Each slot's i's are cut into tiles of tile_i; a tile is cut
// into nsplit j ranges when the step has too little work to fill the GPU with
// whole tiles (few or small events), so every CTA still gets a unit of about
// `target` pairs.  Units are sorted by cost, largest first (LPT order for the
// dynamic per-step work counter).
// ---------------------------------------------------------------------------
int plan_units(const int32_t* n_h, const int32_t* n_e, int n_slots, int tile_i, int grid,
               bool allow_split, int max_units, int64_t partial_cap, std::vector<UnitPlan>* out,
               int64_t* partial_floats) {
  out->clear();
  *partial_floats = 0;
  if (tile_i <= 0 || grid <= 0 || n_slots < 0 || max_units <= 0) return -1;
  double total = 0.0;
  int64_t tiles = 0;
  for (int s = 0; s < n_slots; ++s) {
    const int64_t nh = std::max(n_h[s], 0), ne = std::max(n_e[s], 0);
    if (nh <= 0) continue;  // an event with no hole is finished
    const double n = (double)(nh + ne);
    total += n * n;
    tiles += (nh + tile_i - 1) / tile_i + (ne + tile_i - 1) / tile_i;
  }
  if (tiles > max_units) return -2;
  // Aim for >= 4 units per CTA, each at least one shared-memory stage deep.
  const double target = std::max(total / (4.0 * grid), (double)tile_i * (double)kPlanMinJ);
  int64_t units_left = max_units - tiles;  // budget for extra split units
  int iblock = 0;
  int64_t pfl = 0;
  for (int s = 0; s < n_slots; ++s) {
    const int nh = std::max(n_h[s], 0), ne = std::max(n_e[s], 0);
    if (nh <= 0) continue;
    const int n = nh + ne;
    for (int spec = 0; spec < 2; ++spec) {
      const int ni_tot = spec ? ne : nh;
      for (int i0 = 0; i0 < ni_tot; i0 += tile_i) {
        const int ni = std::min(tile_i, ni_tot - i0);
        int ns = 1;
        if (allow_split) {
          const double want = std::floor((double)ni * (double)n / target + 0.5);
          ns = (int)std::max(1.0, std::min(want, (double)kPlanMaxSplit));
          ns = std::min(ns, std::max(1, n / kPlanMinJ));
          if (ns > 1 && (int64_t)(ns - 1) > units_left) ns = (int)std::max<int64_t>(1, units_left + 1);
          if (ns > 1 && pfl + (int64_t)ns * 3 * tile_i > partial_cap) ns = 1;
        }
        const int pbase = ns > 1 ? (int)pfl : 0;
        for (int sp = 0; sp < ns; ++sp) {
          UnitPlan u;
          u.slot = s;
          u.spec = spec;
          u.i0 = i0;
          u.ni = ni;
          u.j0 = (int)((int64_t)n * sp / ns);
          u.j1 = (int)((int64_t)n * (sp + 1) / ns);
          u.split = sp;
          u.nsplit = ns;
          u.iblock = ns > 1 ? iblock : -1;
          u.pbase = pbase;
          out->push_back(u);
        }
        if (ns > 1) {
          units_left -= ns - 1;
          pfl += (int64_t)ns * 3 * tile_i;
          ++iblock;
        }
      }
    }
  }
  std::stable_sort(out->begin(), out->end(), [](const UnitPlan& a, const UnitPlan& b) {
    return (int64_t)a.ni * (a.j1 - a.j0) > (int64_t)b.ni * (b.j1 - b.j0);
  });
  *partial_floats = pfl;
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

}  // namespace cts

extern "C" {

int cts_plan_units(const int32_t* n_h, const int32_t* n_e, int32_t n_slots, int32_t tile_i,
                   int32_t grid, int32_t allow_split, int32_t max_units, int64_t partial_cap,
                   cts_unit_t* out, int32_t* n_out, int64_t* partial_floats) {
  if (!n_h || !n_e || !out || !n_out || !partial_floats) return -1;
  std::vector<cts::UnitPlan> units;
  const int rc = cts::plan_units(n_h, n_e, n_slots, tile_i, grid, allow_split != 0, max_units,
                                 partial_cap, &units, partial_floats);
  if (rc != 0) return rc;
  for (size_t k = 0; k < units.size(); ++k) {
    const cts::UnitPlan& u = units[k];
    out[k] = cts_unit_t{u.slot, u.spec, u.i0, u.ni, u.j0, u.j1, u.split, u.nsplit, u.iblock,
                        u.pbase};
  }
  *n_out = (int32_t)units.size();
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

double cts_estimate_steps(double thickness_um, double bias_V, double depletion_V, double mu0_cm2,
                          double vsat_cms, double beta, double dt_ps, double depth_um) {
  return cts::estimate_steps(thickness_um, bias_V, depletion_V, mu0_cm2, vsat_cms, beta, dt_ps,
                             depth_um);
}

}  // extern "C"
