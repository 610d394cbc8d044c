// cts_host_impl.h -- C++ interface of the pure host logic (cts_host.cpp).
#pragma once
#include <cstdint>
#include <map>
#include <utility>
#include <vector>

namespace cts {

constexpr int kPlanMinJ = 256;        // shortest j range of a static share's segment
constexpr int kPlanDynMinJ = 64;      // shortest j range of a dynamic-queue piece
constexpr int kPlanDynMaxPieces = 128;  // most dynamic-queue pieces per tile
constexpr int64_t kArenaAlign = 32; // arena entries are handed out in multiples of this

struct UnitPlan {
  int32_t slot, spec, i0, ni, j0, j1, split, nsplit, iblock, pbase;
};

// Static mode: cta_begin receives grid + 1 offsets, CTA g runs units
// [begin[g], begin[g+1]).  Dynamic mode: units form one queue (largest first)
// that CTAs pull from with an atomic counter; cta_begin is all zeros except
// begin[grid] = number of units.  slot_major (dynamic only): the queue holds
// each slot's pieces together, slot after slot, the piece sizes shrinking
// within each slot, so that a queue replayed for several steps finishes every
// slot's step long before the slot's next step is reached.
int plan_units(const int32_t* n_h, const int32_t* n_e, int n_slots, int tile_i, int grid,
               bool allow_split, int max_units, int64_t partial_cap, std::vector<UnitPlan>* out,
               std::vector<int32_t>* cta_begin, int64_t* partial_floats, bool dynamic,
               bool slot_major = false);

// Plan of the symmetric pair kernel (see cts_plan_sym in cts_host.h): units,
// tiles and the per-tile partial lists of one step of the resident slots.
constexpr int kSymPlanTile = 64;   // carriers per tile
constexpr int kSymPlanTpb = 4;     // tiles per I block
constexpr int kSymPlanUpdateTiles = 1;  // tiles per update unit (at least)
constexpr int kSymPlanUpdateLag = 32;   // slots of pair units before a slot's update units
struct SymUnitPlan {
  // kind 0: pair unit; kind 1: update unit of the slot's tiles [jt0, jt1)
  // (slot-local numbering, holes then electrons), after its npair pair units
  int32_t slot, spec_i, spec_j, ib0, ib1, jt0, jt1, p_i, p_j, duty, kind, npair;
};
struct SymTilePlan {
  int32_t slot, spec, tile, n, lptr, lcnt;
};
// The plan of one slot with th hole tiles and te electron tiles, numbered
// from the slot's first partial and its first tile (slot field 0).
struct SymSlotTemplate {
  std::vector<SymUnitPlan> pair;   // pair units, longest first
  std::vector<SymUnitPlan> upd;    // update units
  std::vector<int32_t> lcnt;       // partials listed per tile (holes, then electrons)
  std::vector<int32_t> lists;      // the slot's tile lists, tile after tile
  int64_t n_partials = 0;
};
struct SymPlan {
  std::vector<SymUnitPlan> units;
  std::vector<SymTilePlan> tiles;
  std::vector<int32_t> lists;         // partial indices, tile by tile
  std::vector<int32_t> slot_tile0;    // global index of a slot's first tile (-1: none)
  std::vector<int32_t> slot_ntiles;   // tiles of the slot
  int64_t n_partials = 0;             // partial tiles the units write
  // slot plans by (th, te), kept across calls on the same SymPlan
  std::map<std::pair<int, int>, SymSlotTemplate> memo;
};
// Unit shape (I blocks x J tiles) of a slot with `ntiles` tiles.
void sym_shape(int ntiles, int* rb, int* rj);
int plan_sym(const int32_t* n_h, const int32_t* n_e, int n_slots, int max_units, SymPlan* out);

// Fano-distributed carrier-pair count of one photon (see cts_fano_pairs).
int fano_pairs(uint64_t seed, uint64_t event_id, double energy_keV, double fano);

// Generalised Gaussian model (see the cts_fit_* entry points).
double alpha_of_t(const double* p, double t);
double beta_of_t(const double* p, double t);
int fit_ggd(const double* x, int64_t n, double* alpha, double* beta);
int fit_alpha_t(const double* t, const double* y, const double* w, int n, double* p);
int fit_beta_t(const double* t, const double* y, const double* sigma, int n, double* p);

// Variant-table cache file (see cts_variant_table_save / _load).
int table_save(const char* path, const char* device, int32_t n_variants, const int64_t* mins,
               const int32_t* vars, int32_t n);
int table_load(const char* path, const char* device, int32_t n_variants, int64_t* mins,
               int32_t* vars, int32_t cap, int32_t* n);

class ArenaAllocator {
 public:
  explicit ArenaAllocator(int64_t capacity = 0);
  int64_t alloc(int64_t n);  // offset, or -1 if no block fits
  void release(int64_t off);
  int64_t capacity() const { return capacity_; }
  int64_t in_use() const { return in_use_; }
  int64_t largest_free() const;

 private:
  int64_t capacity_;
  int64_t in_use_ = 0;
  std::map<int64_t, int64_t> free_;  // offset -> length
  std::map<int64_t, int64_t> used_;  // offset -> length
};

double estimate_steps(double H, double Vb, double Vd, double mu0_cm2, double vsat_cms,
                      double beta, double dt_ps, double depth);

}  // namespace cts
