// cts_internal.h -- data layout shared by the kernels (cts_kernels.cu) and the
// host runtime (cts_runtime.cu).  Not part of the public ABI (include/cts.h).
//
// Device memory layout (one arena of carriers shared by all resident events):
//   px, py, pz   FP64 absolute positions (um), by arena index
//   sh[2]        FP32 float4 shadow (x - ax, y - ay, z - az[species], 0),
//                double-buffered by step parity; the pair kernel reads only it
//   cid          carrier id inside its event (Philox counter, result index)
//   fx, fy       FP64 collection position, by (slot base + carrier id)
//   rstep        retire step by (slot base + carrier id)
//   cstate       state by (slot base + carrier id): bits 0-1 = 0 active,
//                1 collected, 2 exited; bit 2 = electron
// Each event (slot) owns [base, base + cap_h + cap_e): holes first (compacted
// to n_h entries at every chunk boundary), electrons from base + cap_h.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace cts {

constexpr int kStateActive = 0;
constexpr int kStateCollected = 1;
constexpr int kStateExited = 2;
constexpr int kStateMask = 3;
constexpr int kElectronBit = 4;

constexpr int kErrNumeric = 1;    // non-finite displacement
constexpr int kErrTimeout = 2;    // bounded wait on a copy gave up
constexpr int kErrBounds = 4;     // index outside its slot (checked build)
constexpr int kErrPlan = 8;       // a unit descriptor disagrees with its slot

constexpr float kParked = 1.0e18f;  // shadow coordinate of retired carriers
constexpr int kChunkJ = 1024;       // j entries per shared-memory stage
constexpr int kFoldJ = 256;         // sources summed in plain FP32 before a Kahan fold
constexpr int kMaxK = 256;          // largest chunk (steps per host check)
constexpr int kMaxGrid = 8192;      // largest persistent grid

// Derived physical constants (all in um, ns, V).
struct Phys {
  double H;          // thickness
  double ea, eb;     // drift field magnitude E(z) = ea - eb z
  double kc;         // e / (4 pi eps0 eps_r), V um
  double kT;         // kT / e, V
  double dt;         // ns
  double mu0[2], vsat[2], beta[2];  // [0] holes, [1] electrons; um^2/(V ns), um/ns
  double pitch;
  float f_ea, f_eb, f_kc, f_kT, f_dt, f_eps2, f_H;
  float f_mu0[2], f_vsat[2], f_beta[2], f_ibeta[2];
  int32_t mob_model, repulsion, drift, diffusion;
  int32_t species, grid_n;
  int64_t max_steps;
  // optional non-uniform drift field: drift_n samples (device memory) at
  // z = k H / (drift_n - 1), linearly interpolated; drift_n = 0 keeps Eq. 6
  const float* drift_tab;
  int32_t drift_n;
  float f_drift_inv_dz;
  // pixel weighting potentials of the 3 x 3 window around the centre pixel:
  // the window's lower-left corner, the image pairs summed term by term and
  // the coefficients of the remaining pairs' expansion in 1/n
  double wp_x0, wp_y0;
  float wp_c3, wp_c5;
  int32_t wp_pairs;
};

// Per-slot state, resident in device memory.
struct SlotDev {
  uint64_t seed, event_id;
  int64_t base;             // arena offset
  int32_t cap_h, cap_e;     // allocated entries per species
  int32_t n_h, n_e;         // range lengths (compacted at chunk boundaries)
  int32_t act_h, act_e;     // active carriers at the chunk start
  int32_t n_total;          // carrier ids 0 .. n_total-1
  int32_t step0;            // event-local step at the chunk start
  int32_t running;          // 1 while stepping
  int32_t flags;            // kErr* bits
  int32_t n_steps;          // steps executed so far
  int32_t status;           // final status (set at the close)
  double ax, ay;            // lateral anchor (um)
  double az[2][2];          // [step parity][species] z anchor (um)
  unsigned long long interactions;
  // initial condition
  int32_t kind, n_pairs;
  double energy_keV, depth_um, x0, y0, sigma_um, track_len_um, theta_deg, phi_deg;
  int64_t explicit_off;     // offset (records) into the explicit staging buffer
};

// One explicit carrier, already in arena order (holes then electrons).
struct ExplicitRec {
  double x, y, z;
  int32_t cid;
  int32_t sign;
};

// A unit of pair work as the step kernel reads it: TI i's of one species of
// one slot against a j range of the concatenated [holes | electrons] list,
// with the arena offsets resolved on the host so that the first source copy
// and the i loads can start as soon as the descriptor arrives.
struct alignas(16) Unit {
  int64_t ioff;      // arena index of the first i
  int64_t hoff;      // arena index of the first hole source
  int64_t eoff;      // arena index of the first electron source
  int32_t slot;
  int32_t flags;     // kUnit* bits
  int32_t ni;        // i's in the unit
  int32_t len_h;     // hole sources
  int32_t len_e;     // electron sources
  int32_t nsplit;    // pieces of the tile (> 1: FP64 partial sums + combine)
  int32_t iblock;    // combine counter (nsplit > 1)
  int32_t pbase;     // FP64 offset of the tile's partial sums: piece k at
                     // pbase + 3 * tile_i * k
  int32_t ntiles;    // tiles of the slot (its step is done when all are updated)
  int32_t split;     // this piece's index k
};
static_assert(sizeof(Unit) == 64, "unit descriptor is four 16-byte words");
constexpr int kUnitElectrons = 1;  // the i's are electrons
constexpr int kUnitDuty = 2;       // the slot's per-step bookkeeping runs in this unit
constexpr int kUnitOddStep = 4;    // the slot's chunk starts on an odd step

// Summary of one slot after a chunk (copied to the host).
struct SlotSummary {
  int32_t running;
  int32_t done;
  int32_t status;
  int32_t n_steps;
  int32_t n_h, n_e;        // range lengths after compaction
  int32_t act_h, act_e;
  int32_t flags;
  int32_t pad;
  unsigned long long interactions;
};

// Per-slot readout results (device), filled by the binning kernel.
struct SlotReadout {
  long long n_collected;
  long long n_outside;
  long long n_lost;
  long long pad;
};

struct Arena {
  double *px, *py, *pz;
  float4* sh[2];
  int32_t* cid;
  double *fx, *fy;
  int32_t* rstep;
  int8_t* cstate;
  int64_t capacity;
};

// ---- the symmetric pair kernel (Newton's third law) ----------------------
// Every unordered pair of an event is evaluated once and its term added to
// both carriers.  Carriers of each species range are cut into tiles of
// kSymTile; an I block is kSymTpb consecutive tiles of one species (one warp
// holds its 32 * 2 * kSymTpb carriers in registers).  The pair matrix of a
// step is covered by the (block b, tile g) combinations with g at or after
// block b's first tile (same species) or g an electron tile (b a hole
// block); a pair unit is a rectangle of them: blocks [ib0, ib1) x tiles
// [jt0, jt1) of one (I species, J species) pair, run by one warp.  It writes
// one FP32 partial field per tile it touches (kSymTile x 3 floats, at fixed
// indices) and counts them per tile.  Update units follow the pair units of
// their slot in the queue: once all of a tile's partials are in, a warp sums
// them in a fixed order (compensated FP32) and updates the tile's carriers.
constexpr int kSymTile = 64;        // carriers per tile (32 lanes x 2)
constexpr int kSymRI = 8;           // i's per lane
constexpr int kSymTpb = kSymRI / 2; // tiles per I block
constexpr int kSymBlock = 32 * kSymRI;
constexpr int kSymMaxRJ = 16;       // J tiles per unit at most (shared-memory sums)
constexpr int kSymFold = 4;         // J tiles summed in registers before a fold
constexpr int kSymPartFloats = 3 * kSymTile;  // one tile's partial field

constexpr int kSymIElectrons = 1;   // the unit's I blocks are electrons
constexpr int kSymJElectrons = 2;   // the unit's J tiles are electrons
constexpr int kSymDuty = 4;         // the slot's per-step bookkeeping of the launch's first step
constexpr int kSymOddStep = 8;      // the slot's chunk starts on an odd step
constexpr int kSymUpdate = 16;      // an update unit (tiles [jt0, jt1) of the slot)

struct alignas(16) SymUnit {
  int64_t ibase;     // arena index of carrier 0 of the I species range
  int64_t jbase;     // arena index of carrier 0 of the J species range
  int32_t slot;
  int32_t flags;     // kSym* bits
  int32_t ib0, ib1;  // I blocks (species-local)
  int32_t jt0, jt1;  // J tiles (species-local); update units: the slot's tiles
  int32_t ni, nj;    // carriers in the I and J species ranges
  int32_t pI;        // first I partial: block ib0 + q, tile u -> pI + q * kSymTpb + u
  int32_t pJ;        // first J partial: tile jt0 + t -> pJ + t
  int32_t tI, tJ;    // global tile index of species-local tile 0 of I and of J;
                     // update units: of the slot's tile 0
  int32_t ntiles;    // tiles of the slot (its step is done when all are updated)
  int32_t npair;     // pair units of the slot
  int32_t pad[2];
};
static_assert(sizeof(SymUnit) == 80, "symmetric unit descriptor layout");

// A tile of one slot: its carriers and the list of partials that make its field.
struct alignas(16) SymTile {
  int64_t off;       // arena index of the tile's first carrier
  int32_t slot;
  int32_t spec;      // 0 holes, 1 electrons
  int32_t n;         // carriers in the tile (<= kSymTile)
  int32_t lptr;      // first entry of its partial list
  int32_t lcnt;      // partials in the list
  int32_t ntiles;    // tiles of its slot
};
static_assert(sizeof(SymTile) == 32, "symmetric tile descriptor layout");

// Per-slot values of one step, written once (by the warp that finishes the
// slot's previous step, or identically by the units of a launch's first
// step) and read by every unit of the step.
struct alignas(16) SymStep {
  double azn[2];     // frame anchors of the next step
  int32_t nah, nae;  // active carriers of each species
  int32_t step;      // event-local step
  int32_t skip;      // 1: the slot runs no pairs at this step
  float s_off;       // electron frame z anchor minus the hole frame's (FP32)
  int32_t pad[3];
};
static_assert(sizeof(SymStep) == 48, "symmetric step record layout");

struct SymArgs {
  const SymUnit* units;     // one step's units (replayed for every step of a launch)
  const int32_t* n_units;   // [1] units per step
  const SymTile* tiles;     // every tile of every planned slot
  const int32_t* lists;     // partial indices, per tile (CSR by SymTile.lptr)
  float* part;              // partials [n][3][kSymTile]
  int32_t* tile_ctr;        // partials written per tile (returned to 0 by its update)
  SymStep* rec;             // [K][S]
  int32_t* ready;           // [K][S]: rec valid
  int64_t n_part;           // partial fields in the buffer (bounds checks)
  int32_t n_tiles;          // tiles planned (bounds checks)
};

struct StepArgs {
  Arena A;
  SlotDev* slots;
  const Unit* units;
  const int32_t* cta_begin;  // [grid + 1]: CTA g runs units [cta_begin[g], cta_begin[g+1])
  int32_t* unit_counter;     // [K]: dynamic queue position per step (dynamic plans)
  int32_t dynamic;           // 1: pull units from unit_counter instead of cta_begin
  int32_t* ret;              // [K][S][2]
  double* partial;           // partial sums of split tiles: per piece 3 x tile_i entries of
                             // 8 bytes, each the compensated FP32 pair (S, c) of a sum S - c
  int32_t* combine_count;    // per i-block
  int32_t* tiles_done;       // [K][S]: tiles of each slot updated at each chunk step
  float* field_out;          // FIELD_ONLY output, SoA [3][capacity]
  int32_t* err;              // global error bits
  unsigned long long* trace; // optional: per CTA {smid, t_start, t_end, pairs, units,
                             //   ns in prologues, in pair loops, in epilogues}
  Phys ph;
  int32_t S;                 // slot count
  int32_t fused;             // 1: update positions; 0: write field_out
  double* induced;           // [K][S]: charge induced at each chunk step (e); NULL = off
  double* induced_px;        // [K][S][9]: the same per pixel of the 3 x 3 window; NULL = off
  SymArgs sym;               // the symmetric kernel's plan and buffers
};

// ---- kernel launchers (cts_kernels.cu) ----------------------------------
struct Variant {
  int nt;       // threads per CTA
  int r;        // i's per thread
  const char* name;
  int ctas_per_sm;  // 0: as many as fit; else a fixed count
  int dynamic;      // 1: guided dynamic queue; 0: static equal shares
  int sym;          // 1: the symmetric kernel (SymUnit plans, warp-level queue)
};
int variant_count();
Variant variant_info(int v);
cudaError_t variant_occupancy(int v, int* blocks_per_sm);
size_t variant_smem(int v);

// Steps k0 .. k0 + nk - 1 of the chunk in one launch (nk > 1 needs a dynamic
// variant and a slot-major plan).
cudaError_t launch_step(int v, const StepArgs& a, int k0, int nk, int grid, cudaStream_t s);
cudaError_t launch_update(const StepArgs& a, int k, int n_slots_list, const int32_t* slot_list,
                          int grid, cudaStream_t s);
cudaError_t launch_init(const Phys& ph, Arena A, SlotDev* slots, const int32_t* slot_list,
                        int n, const ExplicitRec* explicit_buf, cudaStream_t s);
cudaError_t launch_close(const Phys& ph, Arena A, SlotDev* slots, const int32_t* slot_list,
                         int n, const int32_t* ret, int S, int K, SlotSummary* summary,
                         cudaStream_t s);
cudaError_t launch_bin(const Phys& ph, Arena A, const SlotDev* slots, const int32_t* slot_list,
                       int n, int32_t* pixels, SlotReadout* readout, cudaStream_t s);
cudaError_t launch_bin_points(const Phys& ph, const double* x, const double* y, int64_t n,
                              int32_t* pixels, long long* outside, cudaStream_t s);
// Simplified spherical model: one cluster of `cluster` CTAs (1, 2 or 4) per
// slot for steps k0 .. k0 + nk - 1; events of at most kSphMax holes (keys in
// shared memory).
constexpr int kSphMax = 16384;
// spherical_prepare raises the kernel's shared-memory limit on the current
// device and finds how many clusters of each width are resident at once
// (once per handle, at sim_init, outside any stream capture).
cudaError_t spherical_prepare();
// The cluster width for `slots` resident events: `request` when it is 1, 2
// or 4, else the widest with which all slots' clusters are resident at once.
int spherical_cluster(int slots, int request);
cudaError_t launch_spherical(const StepArgs& a, int k0, int nk, int cluster, cudaStream_t s);

// Fast generation from the generalised Gaussian model: one CTA per event.
struct GenEvent {
  unsigned long long seed, id;
  int32_t n_pairs, pad;
  double x0, y0, alpha, beta;
};
static_assert(sizeof(GenEvent) == 56, "generation record layout");
cudaError_t launch_generate(const GenEvent* ev, int n_events, double pitch_um, int grid_n,
                            int32_t* pixels, unsigned long long* outside, cudaStream_t s);

// Readout of pixel-count maps: one CTA per event (grid_n <= 32).  ClusterRec
// has the layout of the public sim_cluster_t.
struct ClusterRec {
  int32_t accepted, vetoed, cx, cy;
  double e_cluster;
  double e[9];
};
static_assert(sizeof(ClusterRec) == 96, "cluster record layout");
constexpr int kReadoutMaxGrid = 32;
struct ReadoutArgs {
  const int32_t* counts;
  const unsigned long long* seeds;
  const unsigned long long* ids;
  double* pixel_keV;    // optional
  ClusterRec* clusters;
  unsigned long long* spectrum;
  int32_t grid_n, n_bins;
  double ev_per_pair, noise_keV, beam_keV, window_keV, veto_factor, spec_lo_keV, spec_bin_keV;
};
cudaError_t launch_readout(const ReadoutArgs& r, int n_events, cudaStream_t s);

// 16 FMA lane-ops per thread and iteration; 256 threads per CTA.
cudaError_t launch_fma_chain(bool packed, float* out, int grid, int iters, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                          uint32_t* curand_out, cudaStream_t s);
cudaError_t launch_normals(const unsigned long long* in, int64_t n, double* out, cudaStream_t s);

}  // namespace cts
