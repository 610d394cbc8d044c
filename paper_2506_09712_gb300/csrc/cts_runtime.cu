// cts_runtime.cu -- host runtime behind include/cts.h: handle, device arena,
// admission queue, slot scheduler, graph-captured K-step chunks, readout and
// the serving thread.  All arithmetic of the method runs in cts_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "cts.h"
#include "cts_host_impl.h"
#include "cts_internal.h"

using namespace cts;

namespace {

double now_ns() {
  return (double)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr int kDefaultSlots = 256;
constexpr int kDefaultK = 32;
constexpr size_t kLaunchLogCap = size_t(1) << 20;
constexpr int64_t kDefaultBudget = 1ll << 30;
// Default kernel choice per chunk: the symmetric kernel from this many
// resident carrier pairs per step (sum of N^2), the per-pair kernel below.
// Whole 64-event 20 keV batches with the 12-warp symmetric kernel, 32-step
// chunks: 462 / 458 / 452 / 448 ms with the switch at 1.2e8 / 1.8e8 / 2.8e8
// / 4.0e8 pairs (about 17 partly collected events)
constexpr double kSymMinWork = 4.0e8;
// SERVE keeps the 8-warp symmetric kernel and the switch at 2.8e8 pairs: at
// the moderate occupancy of a served stream (about 27 mixed events at 0.7x
// saturation) its steps are shorter; the serving mix's p50 / p99 latency at
// 0.7x saturation: 129 / 257 ms, against 141 / 298 ms with the 12-warp
// kernel and the 4.0e8 switch (the same saturation rate, 259 events/s)
constexpr double kSymMinWorkServe = 2.8e8;
// The symmetric kernel's warps per SM: 12 (two rotation steps per loop
// iteration) while every running event has at most kSymLargeTiles tiles,
// 1.8 % faster than 8 on the 20 keV batch; 8 once an event is larger (its
// units are 8 blocks x 16 tiles; measured 6 % faster on the 200 keV tracks)
constexpr int kSymVariant = 0;        // sym_nt384_r8_warp
constexpr int kSymVariantLarge = 12;  // sym_nt256_r8_warp
constexpr int kSymLargeTiles = 640;
constexpr int kPairVariant = 1;  // nt256_r2_jpair_dyn
constexpr int kSymVariantPlain = 0;  // sym_nt384_r8_warp
constexpr int kMaxUnits = 1 << 16;
constexpr int kMaxSymUnits = 1 << 18;  // units of one step of the symmetric kernel
// upload_sym_plan: the plan needs more units or tiles than the buffers hold
constexpr int kSymPlanTooLarge = 1;
constexpr int kDefaultQueue = 1 << 16;
// arena (positions, two shadows, id, collection point, step, state), explicit
// staging, split-tile accumulators (3 doubles) and the PLAIN field buffer
constexpr int64_t kBytesPerCarrier = 24 + 32 + 4 + 16 + 4 + 1 + 32 + 24 + 12;

struct EventRec {
  sim_event_t ev{};
  std::vector<double> xyz;
  std::vector<int8_t> sign;
  int32_t n_pairs = 0;
  int32_t cap_h = 0, cap_e = 0;
  double t_submit = 0.0;
  int64_t order = 0;
};

struct Done {
  uint64_t event_id = 0;
  int32_t status = 0, n_carriers = 0;
  int64_t n_steps = 0, n_collected = 0, n_outside = 0, n_lost = 0, interactions = 0;
  double t_submit = 0, t_start = 0, t_done = 0;
  std::vector<int32_t> pixels;
  std::vector<double> final_xy;
  std::vector<int32_t> rstep;
  std::vector<double> induced;  // charge on the collecting surface after each step (e)
  std::vector<double> induced_px;  // [step][9]: the same on the 3 x 3 centre pixels
  int64_t order = 0;
};

struct HostSlot {
  bool used = false;
  bool running = false;
  bool needs_init = false;
  bool finished_on_device = false;  // readout done, results still on the device
  EventRec rec;
  int64_t base = 0;
  double t_start = 0;
  int32_t n_h = 0, n_e = 0;
  int32_t status = 0;
  int64_t n_steps = 0, interactions = 0;
  std::vector<double> induced;  // per executed step (options.keep_induced)
  double induced_q = 0.0;
  std::vector<double> induced_px;  // [step][9] per executed step
  double induced_pxq[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
};

}  // namespace

struct sim_t {
  sim_sensor_t sensor{};
  sim_field_t field{};
  sim_mobility_t mob{};
  sim_options_t opt{};
  Phys ph{};
  int device = 0, sm_count = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int S = 0, K = 0, variant = 0, grid = 0, tile_i = 0, dynamic = 0;
  bool sym = false;  // the current variant is the symmetric kernel
  int64_t capacity = 0, partial_cap = 0;
  std::atomic<bool> broken{false};  // read by polling threads while the engine runs
  std::string err;

  // device buffers
  Arena A{};
  SlotDev* d_slots = nullptr;
  SlotSummary* d_summary = nullptr;
  SlotReadout* d_readout = nullptr;
  int32_t* d_pixels = nullptr;
  Unit* d_units = nullptr;
  int32_t* d_cta_begin = nullptr;
  int32_t* d_unit_counter = nullptr;
  int32_t* d_ret = nullptr;
  double* d_partial = nullptr;
  int32_t* d_combine = nullptr;
  int32_t* d_tiles_done = nullptr;
  float* d_drift = nullptr;           // sampled drift field (optional)
  double* d_induced = nullptr;        // [K][S] induced charge per chunk step (keep_induced)
  double* h_induced = nullptr;
  double* d_induced_px = nullptr;     // [K][S][9] the same per pixel of the 3 x 3 window
  double* h_induced_px = nullptr;
  std::vector<double> drift_host;     // the caller's samples, copied at init
  int32_t* d_err = nullptr;
  float* d_field = nullptr;
  ExplicitRec* d_explicit = nullptr;
  int32_t* d_list = nullptr;
  // pinned host staging
  SlotSummary* h_summary = nullptr;
  Unit* h_units = nullptr;
  int32_t* h_cta_begin = nullptr;
  int32_t* h_list = nullptr;
  SlotDev* h_slotdev = nullptr;
  SlotReadout* h_readout = nullptr;
  int32_t* h_pixels = nullptr;
  int32_t* h_err = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  std::vector<cudaEvent_t> lev;  // per-launch events (time_launches): K + 1

  // the symmetric kernel's plan of the current chunk and its buffers (the
  // partial fields and lists grow with the plan; growing them drops the
  // captured graphs, which hold their addresses)
  SymPlan splan;
  SymUnit* d_sym_units = nullptr;
  SymUnit* h_sym_units = nullptr;
  int32_t* d_sym_nu = nullptr;
  int32_t* h_sym_nu = nullptr;
  SymTile* d_sym_tiles = nullptr;
  SymTile* h_sym_tiles = nullptr;
  int64_t sym_tiles_cap = 0;
  int32_t* d_sym_lists = nullptr;
  int32_t* h_sym_lists = nullptr;
  int64_t sym_lists_cap = 0;
  float* d_sym_part = nullptr;
  int64_t sym_part_cap = 0;  // partial fields (3 x 64 floats each)
  int32_t* d_sym_ctr = nullptr;     // partials written per tile
  SymStep* d_sym_rec = nullptr;
  int32_t* d_sym_ready = nullptr;

  // host state
  std::vector<HostSlot> slots;
  ArenaAllocator alloc;
  std::deque<std::array<double, 4>> launch_log;  // (ms, pairs, running, symmetric) per launch
  std::vector<UnitPlan> plan;
  std::vector<int32_t> plan_begin;
  std::mutex qmu;
  std::condition_variable qcv;
  std::deque<EventRec> queue;
  std::mutex dmu;
  std::condition_variable dcv;
  std::deque<Done> done;
  std::mutex drive_mu;
  std::thread engine;
  std::atomic<bool> stop{false};
  int64_t order_counter = 0;
  std::atomic<int> inject{0};  // set by sim_debug_inject from any thread
  std::vector<int> staged;  // slots admitted by sim_stage, in staging order

  // one captured K-step chunk per kernel variant and launch shape
  // (index 2 * variant + 1 for one launch per chunk)
  std::vector<cudaGraphExec_t> graphs;
  std::vector<int> graph_K;
  // per-variant occupancy (CTAs per SM), queried once
  std::vector<int> occ_cache;
  // variant table: a chunk whose resident pair work W satisfies
  // W >= table_min[k] (largest such k) runs table_var[k]; empty = fixed variant
  std::vector<int64_t> table_min;
  std::vector<int> table_var;
  int base_variant = 0;
  int sph_cluster = 1;  // CTAs per event of the spherical model
  std::string autotune_cache;  // copied from the options
  std::string device_name;

  // stats
  int64_t st_events = 0, st_inter = 0, st_steps = 0, st_launch = 0, st_chunks = 0,
          st_rejected = 0;
  double st_ms = 0.0, st_kernel_ms = 0.0;
  int64_t st_kernel_launches = 0, st_h2d = 0, st_d2h = 0;
};

namespace {

// An NVTX range for the scope (named phases in nsys / ncu timelines; inert
// without a profiler attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      s->broken = true;                                                            \
      s->err = std::string(#call) + ": " + cudaGetErrorString(e_);                 \
      return SIM_ECUDA;                                                            \
    }                                                                              \
  } while (0)

// Host<->device copies of the library, counted for the statistics.
cudaError_t h2d(sim_t* s, void* dst, const void* src, size_t bytes) {
  s->st_h2d += (int64_t)bytes;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream);
}
cudaError_t d2h(sim_t* s, void* dst, const void* src, size_t bytes) {
  s->st_d2h += (int64_t)bytes;
  return cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->stream);
}

bool finite_all(std::initializer_list<double> v) {
  for (double x : v)
    if (!std::isfinite(x)) return false;
  return true;
}

int validate_params(const sim_sensor_t* se, const sim_field_t* f, const sim_mobility_t* m) {
  if (!se || !f || !m) return SIM_EINVAL;
  if (!finite_all({se->thickness_um, se->bias_V, se->depletion_V, se->temperature_K, se->eps_r,
                   se->pitch_um, se->dt_ps, se->softening_um}))
    return SIM_EINVAL;
  if (!(se->thickness_um > 0) || !(se->temperature_K > 0) || !(se->eps_r > 0) ||
      !(se->pitch_um > 0) || !(se->dt_ps > 0) || se->softening_um < 0)
    return SIM_EINVAL;
  if (!(se->depletion_V >= 0) || !(se->bias_V >= se->depletion_V)) return SIM_EINVAL;
  if (se->grid_n < 1 || se->grid_n > 4096 || se->max_steps < 1) return SIM_EINVAL;
  if (se->species != CTS_HOLES && se->species != CTS_BOTH) return SIM_EINVAL;
  // the simplified spherical model moves holes only (Sec. 2.2)
  if (f->spherical != 0 && f->spherical != 1) return SIM_EINVAL;
  if (f->spherical && se->species != CTS_HOLES) return SIM_EINVAL;
  if (se->drift_table_n != 0) {
    if (se->drift_table_n < 2 || se->drift_table_n > 4096 || !se->drift_table_Vum)
      return SIM_EINVAL;
    for (int32_t k = 0; k < se->drift_table_n; ++k)
      if (!std::isfinite(se->drift_table_Vum[k]) || !(se->drift_table_Vum[k] > 0.0))
        return SIM_EINVAL;
  }
  if (m->model != CTS_MOB_CT && m->model != CTS_MOB_CONST) return SIM_EINVAL;
  if (!(m->mu0_h > 0) || !(m->vsat_h > 0) || !(m->beta_h > 0)) return SIM_EINVAL;
  if (se->species == CTS_BOTH && (!(m->mu0_e > 0) || !(m->vsat_e > 0) || !(m->beta_e > 0)))
    return SIM_EINVAL;
  return SIM_OK;
}

Phys make_phys(const sim_sensor_t& se, const sim_field_t& f, const sim_mobility_t& m) {
  const double e = 1.602176634e-19, eps0 = 8.8541878128e-12, kb = 1.380649e-23;
  Phys p{};
  p.H = se.thickness_um;
  p.ea = (se.bias_V + se.depletion_V) / se.thickness_um;  // E at z = 0
  p.eb = 2.0 * se.depletion_V / (se.thickness_um * se.thickness_um);
  p.kc = e / (4.0 * M_PI * eps0 * se.eps_r) * 1e6;
  p.kT = kb * se.temperature_K / e;
  p.dt = se.dt_ps * 1e-3;
  p.mu0[0] = m.mu0_h * 0.1;
  p.vsat[0] = m.vsat_h * 1e-5;
  p.beta[0] = m.beta_h;
  p.mu0[1] = m.mu0_e * 0.1;
  p.vsat[1] = m.vsat_e * 1e-5;
  p.beta[1] = m.beta_e > 0 ? m.beta_e : 1.0;
  p.pitch = se.pitch_um;
  p.f_ea = (float)p.ea;
  p.f_eb = (float)p.eb;
  p.f_kc = (float)p.kc;
  p.f_kT = (float)p.kT;
  p.f_dt = (float)p.dt;
  const double eps = se.softening_um > 0 ? se.softening_um : 1e-6;
  p.f_eps2 = (float)(eps * eps);
  p.f_H = (float)p.H;
  for (int s = 0; s < 2; ++s) {
    p.f_mu0[s] = (float)p.mu0[s];
    p.f_vsat[s] = (float)(p.vsat[s] > 0 ? p.vsat[s] : 1.0);
    p.f_beta[s] = (float)p.beta[s];
    p.f_ibeta[s] = (float)(1.0 / p.beta[s]);
    if (!(p.vsat[s] > 0)) p.vsat[s] = 1.0;
  }
  p.mob_model = m.model;
  p.repulsion = f.repulsion;
  p.drift = f.drift;
  p.diffusion = f.diffusion;
  p.species = se.species;
  p.grid_n = se.grid_n;
  p.max_steps = se.max_steps;
  // Pixel weighting potentials of the 3 x 3 window around the centre pixel
  // c = grid_n / 2: its lower-left corner, then the image pairs.  A pair n of
  // images of a pixel of area A behaves for large n like
  //   -A z / (4 pi H^3 n^3) + A z (3 <r^2> - 2 z^2) / (16 pi H^5 n^5),
  // which holds while the lateral distance r stays well below 2 n H: M pairs
  // are summed term by term, M from the grid's half-diagonal (2.5 r / H,
  // at least 2; the truncation then stays below 2e-7 within the grid, under
  // the FP32 evaluation's own error), and the rest by these two terms with
  // zeta(3) and zeta(5) less their partial sums.
  {
    const int c = se.grid_n / 2;
    p.wp_x0 = p.wp_y0 = ((double)(c - 1) - 0.5 * (double)se.grid_n) * se.pitch_um;
    const double rho = 0.5 * std::sqrt(2.0) * (double)se.grid_n * se.pitch_um;
    const int M = (int)std::min(64.0, std::max(2.0, std::ceil(2.5 * rho / se.thickness_um)));
    double s3 = 1.2020569031595942854, s5 = 1.0369277551433699263;
    for (int n = 1; n <= M; ++n) {
      s3 -= 1.0 / ((double)n * n * n);
      s5 -= 1.0 / ((double)n * n * n * n * n);
    }
    const double A = se.pitch_um * se.pitch_um, H = se.thickness_um;
    p.wp_pairs = M;
    p.wp_c3 = (float)(-A * s3 / (4.0 * M_PI * H * H * H));
    p.wp_c5 = (float)(A * s5 / (16.0 * M_PI * H * H * H * H * H));
  }
  return p;
}

// Resolve and validate one event; fills counts of holes and electrons.
int prepare_event(sim_t* s, const sim_event_t* ev, EventRec* r) {
  if (!ev) return SIM_EINVAL;
  r->ev = *ev;
  r->ev.explicit_xyz = nullptr;
  r->ev.explicit_sign = nullptr;
  if (ev->kind != CTS_PHOTON && ev->kind != CTS_TRACK && ev->kind != CTS_EXPLICIT)
    return SIM_EINVAL;
  if (ev->n_pairs < 0) return SIM_EINVAL;
  if (ev->kind == CTS_EXPLICIT) {
    if (ev->n_pairs > 0 && !ev->explicit_xyz) return SIM_EINVAL;
    const int n = ev->n_pairs;
    r->xyz.assign(ev->explicit_xyz, ev->explicit_xyz + 3 * (size_t)n);
    r->sign.assign((size_t)n, 1);
    if (ev->explicit_sign) r->sign.assign(ev->explicit_sign, ev->explicit_sign + n);
    for (double v : r->xyz)
      if (!std::isfinite(v)) return SIM_EINVAL;
    int nh = 0;
    for (int8_t g : r->sign) {
      if (g != 1 && g != -1) return SIM_EINVAL;
      nh += g > 0;
    }
    if (nh < n && s->sensor.species != CTS_BOTH) return SIM_EINVAL;
    r->n_pairs = n;
    r->cap_h = nh;
    r->cap_e = n - nh;
  } else {
    if (!finite_all({ev->energy_keV, ev->depth_um, ev->x_um, ev->y_um, ev->sigma_um,
                     ev->track_len_um, ev->theta_deg, ev->phi_deg}))
      return SIM_EINVAL;
    if (ev->energy_keV < 0) return SIM_EINVAL;
    if (ev->kind == CTS_PHOTON && (ev->depth_um < 0 || ev->depth_um > s->sensor.thickness_um))
      return SIM_EINVAL;
    if (ev->kind == CTS_TRACK && (ev->track_len_um < 0 || ev->theta_deg < 0 ||
                                  ev->theta_deg >= 90.0))
      return SIM_EINVAL;
    const double np = ev->n_pairs > 0 ? (double)ev->n_pairs
                                      : std::llround(ev->energy_keV * 1000.0 / 3.62);
    if (np > 5.0e8) return SIM_ENOMEM_BUDGET;
    r->n_pairs = (int32_t)np;
    r->cap_h = r->n_pairs;
    r->cap_e = s->sensor.species == CTS_BOTH ? r->n_pairs : 0;
  }
  if ((int64_t)r->cap_h + r->cap_e > s->capacity) return SIM_ENOMEM_BUDGET;
  if (s->field.spherical && r->cap_h > kSphMax) return SIM_EINVAL;
  return SIM_OK;
}

int free_slot_index(sim_t* s) {
  for (int k = 0; k < s->S; ++k)
    if (!s->slots[k].used) return k;
  return -1;
}

int running_limit(sim_t* s) { return s->opt.mode == CTS_MODE_PLAIN ? 1 : s->S; }

int count_used(sim_t* s) {
  int c = 0;
  for (auto& h : s->slots) c += h.used;
  return c;
}

// Place an event into a free slot: arena block, host mirror, descriptor upload.
int place_event(sim_t* s, int slot, EventRec&& r, int64_t base) {
  HostSlot& h = s->slots[slot];
  h = HostSlot{};
  h.used = true;
  h.running = true;
  h.needs_init = true;
  h.base = base;
  h.t_start = now_ns();
  h.n_h = r.cap_h;
  h.n_e = r.cap_e;
  SlotDev& d = s->h_slotdev[slot];
  d = SlotDev{};
  d.seed = r.ev.seed;
  d.event_id = r.ev.event_id;
  d.base = base;
  d.cap_h = r.cap_h;
  d.cap_e = r.cap_e;
  d.n_total = r.cap_h + r.cap_e;
  d.kind = r.ev.kind;
  d.n_pairs = r.n_pairs;
  d.energy_keV = r.ev.energy_keV;
  d.depth_um = r.ev.depth_um;
  d.x0 = r.ev.x_um;
  d.y0 = r.ev.y_um;
  d.sigma_um = r.ev.sigma_um;
  d.track_len_um = r.ev.track_len_um;
  d.theta_deg = r.ev.theta_deg;
  d.phi_deg = r.ev.phi_deg;
  d.explicit_off = base;
  if (r.ev.kind == CTS_EXPLICIT) {
    // records in arena order: holes first, then electrons; the anchor is the
    // centroid of the given positions
    std::vector<ExplicitRec> rec((size_t)d.n_total);
    double cx = 0, cy = 0, cz = 0;
    int kh = 0, ke = r.cap_h;
    for (int c = 0; c < r.n_pairs; ++c) {
      ExplicitRec e{r.xyz[3 * c], r.xyz[3 * c + 1], r.xyz[3 * c + 2], c, r.sign[c]};
      rec[r.sign[c] > 0 ? kh++ : ke++] = e;
      cx += e.x;
      cy += e.y;
      cz += e.z;
    }
    if (r.n_pairs > 0) {
      d.x0 = cx / r.n_pairs;
      d.y0 = cy / r.n_pairs;
      d.depth_um = s->sensor.thickness_um - cz / r.n_pairs;
    }
    if (!rec.empty())
      CK(h2d(s, s->d_explicit + base, rec.data(), rec.size() * sizeof(ExplicitRec)));
    // keep the staging alive until the copy is done
    CK(cudaStreamSynchronize(s->stream));
  }
  h.rec = std::move(r);
  CK(h2d(s, s->d_slots + slot, &d, sizeof(SlotDev)));
  return SIM_OK;
}

// Admit queued events while slots and arena space allow (FIFO).  The queue
// lock is held only to take an event off the queue: placing it (descriptor
// upload, and for explicit events a stream synchronisation) runs outside it,
// so sim_submit from other threads never waits behind the device.  Slots and
// the arena belong to the driving thread (drive_mu).
int admit(sim_t* s) {
  NvtxRange range("cts admit");
  for (;;) {
    EventRec rec;
    int slot = -1;
    int64_t base = -1;
    {
      std::lock_guard<std::mutex> lk(s->qmu);
      if (s->queue.empty()) break;
      if (count_used(s) >= running_limit(s)) break;
      slot = free_slot_index(s);
      if (slot < 0) break;
      EventRec& r = s->queue.front();
      const int64_t n = std::max<int64_t>((int64_t)r.cap_h + r.cap_e, 1);
      base = s->alloc.alloc(n);
      if (base < 0) break;
      rec = std::move(r);
      s->queue.pop_front();
    }
    const int rc = place_event(s, slot, std::move(rec), base);
    if (rc) return rc;
  }
  return SIM_OK;
}

int launch_inits(sim_t* s) {
  int n = 0;
  for (int k = 0; k < s->S; ++k)
    if (s->slots[k].used && s->slots[k].needs_init) {
      s->h_list[n++] = k;
      s->slots[k].needs_init = false;
    }
  if (!n) return SIM_OK;
  CK(h2d(s, s->d_list, s->h_list, n * sizeof(int32_t)));
  CK(launch_init(s->ph, s->A, s->d_slots, s->d_list, n, s->d_explicit, s->stream));
  // keep h_list stable until the copy has been consumed
  CK(cudaStreamSynchronize(s->stream));
  s->st_launch += 1;
  return SIM_OK;
}

bool capturing(sim_t* s) {
  cudaStreamCaptureStatus st = cudaStreamCaptureStatusNone;
  cudaStreamIsCapturing(s->stream, &st);
  return st == cudaStreamCaptureStatusActive;
}

StepArgs step_args(sim_t* s, bool fused) {
  StepArgs a{};
  a.A = s->A;
  a.slots = s->d_slots;
  a.units = s->d_units;
  a.cta_begin = s->d_cta_begin;
  a.unit_counter = s->d_unit_counter;
  a.dynamic = s->dynamic;
  a.ret = s->d_ret;
  a.partial = s->d_partial;
  a.combine_count = s->d_combine;
  a.tiles_done = s->d_tiles_done;
  a.induced = s->d_induced;
  a.induced_px = s->d_induced_px;
  a.field_out = s->d_field;
  a.err = s->d_err;
  a.ph = s->ph;
  a.S = s->S;
  a.fused = fused ? 1 : 0;
  a.sym.units = s->d_sym_units;
  a.sym.n_units = s->d_sym_nu;
  a.sym.tiles = s->d_sym_tiles;
  a.sym.lists = s->d_sym_lists;
  a.sym.part = s->d_sym_part;
  a.sym.tile_ctr = s->d_sym_ctr;
  a.sym.rec = s->d_sym_rec;
  a.sym.ready = s->d_sym_ready;
  a.sym.n_part = s->sym_part_cap;
  a.sym.n_tiles = (int32_t)s->sym_tiles_cap;
  return a;
}

// Where a slot's carriers sit in the arena, as the unit descriptors need it.
struct SlotGeom {
  int64_t base = 0;
  int32_t cap_h = 0, n_h = 0;
  int64_t step0 = 0;  // event-local step at the chunk start
};

// Device descriptors of planned units: arena offsets of each unit's i's and
// of its hole and electron sources, and the parity of the slot's first step.
void device_units(const std::vector<UnitPlan>& plan, const std::vector<SlotGeom>& g, Unit* out) {
  // every tile has exactly one piece with split 0
  std::vector<int32_t> ntiles(g.size(), 0);
  for (const UnitPlan& u : plan)
    if (u.split == 0) ++ntiles[u.slot];
  for (size_t q = 0; q < plan.size(); ++q) {
    const UnitPlan& u = plan[q];
    const SlotGeom& sg = g[u.slot];
    const int h1 = std::min(u.j1, sg.n_h);
    const int e0 = std::max(u.j0, sg.n_h);
    Unit d{};
    d.ioff = sg.base + (u.spec ? sg.cap_h : 0) + u.i0;
    d.hoff = sg.base + u.j0;
    d.eoff = sg.base + sg.cap_h + (e0 - sg.n_h);
    d.slot = u.slot;
    d.flags = (u.spec ? kUnitElectrons : 0) |
              (u.spec == 0 && u.i0 == 0 && u.split == 0 ? kUnitDuty : 0) |
              ((sg.step0 & 1) ? kUnitOddStep : 0);
    d.ni = u.ni;
    d.len_h = std::max(h1 - u.j0, 0);
    d.len_e = std::max(u.j1 - e0, 0);
    d.nsplit = u.nsplit;
    d.iblock = u.iblock;
    d.pbase = u.pbase;
    d.split = u.split;
    d.ntiles = ntiles[u.slot];
    out[q] = d;
  }
}

// The captured chunk graphs hold buffer addresses: drop them when a buffer
// moves (they are captured again at the next chunk).
void drop_graphs(sim_t* s) {
  for (size_t g = 0; g < s->graphs.size(); ++g) {
    if (s->graphs[g]) cudaGraphExecDestroy(s->graphs[g]);
    s->graphs[g] = nullptr;
    s->graph_K[g] = -1;
  }
}

// Grows the symmetric kernel's list and partial buffers to hold `lists`
// entries and `parts` partial fields (by half again, to spare later growth).
int sym_reserve(sim_t* s, int64_t lists, int64_t parts) {
  if (lists > s->sym_lists_cap) {
    const int64_t cap = std::max<int64_t>(lists + lists / 2, 1 << 16);
    drop_graphs(s);
    if (s->d_sym_lists) cudaFree(s->d_sym_lists);
    if (s->h_sym_lists) cudaFreeHost(s->h_sym_lists);
    s->d_sym_lists = nullptr;
    s->h_sym_lists = nullptr;
    s->sym_lists_cap = 0;
    CK(cudaMalloc((void**)&s->d_sym_lists, (size_t)cap * sizeof(int32_t)));
    CK(cudaMallocHost((void**)&s->h_sym_lists, (size_t)cap * sizeof(int32_t)));
    s->sym_lists_cap = cap;
  }
  if (parts > s->sym_part_cap) {
    const int64_t cap = std::max<int64_t>(parts + parts / 2, 1 << 12);
    drop_graphs(s);
    if (s->d_sym_part) cudaFree(s->d_sym_part);
    s->d_sym_part = nullptr;
    s->sym_part_cap = 0;
    CK(cudaMalloc((void**)&s->d_sym_part, (size_t)cap * kSymPartFloats * sizeof(float)));
    s->sym_part_cap = cap;
  }
  return SIM_OK;
}

// Where a slot sits for the symmetric plan: its arena range, species range
// lengths and first step of the chunk.
struct SymGeom {
  int64_t base = 0;
  int32_t cap_h = 0, n_h = 0, n_e = 0;
  int64_t step0 = 0;
};

// Plan the symmetric kernel's step for the given slots and upload units,
// tiles and partial lists.
int upload_sym_plan(sim_t* s, const std::vector<SymGeom>& g) {
  const int n_slots = (int)g.size();
  std::vector<int32_t> nh(n_slots), ne(n_slots);
  for (int k = 0; k < n_slots; ++k) {
    nh[k] = g[k].n_h;
    ne[k] = g[k].n_e;
  }
  SymPlan& P = s->splan;
  const int prc = plan_sym(nh.data(), ne.data(), n_slots, kMaxSymUnits, &P);
  if (prc == -2 || (prc == 0 && (int64_t)P.tiles.size() > s->sym_tiles_cap)) return kSymPlanTooLarge;
  if (prc != 0) {
    s->err = "symmetric unit plan failed";
    return SIM_EINVAL;
  }
  int rc = sym_reserve(s, (int64_t)P.lists.size(), P.n_partials);
  if (rc) return rc;
  const int nu = (int)P.units.size();
  for (int q = 0; q < nu; ++q) {
    const SymUnitPlan& u = P.units[q];
    const SymGeom& sg = g[u.slot];
    const int th = (sg.n_h + kSymTile - 1) / kSymTile;
    SymUnit d{};
    d.slot = u.slot;
    d.ntiles = P.slot_ntiles[u.slot];
    d.npair = u.npair;
    d.jt0 = u.jt0;
    d.jt1 = u.jt1;
    if (u.kind == 1) {
      d.flags = kSymUpdate | ((sg.step0 & 1) ? kSymOddStep : 0);
      d.tI = d.tJ = P.slot_tile0[u.slot];
    } else {
      d.ibase = sg.base + (u.spec_i ? sg.cap_h : 0);
      d.jbase = sg.base + (u.spec_j ? sg.cap_h : 0);
      d.flags = (u.spec_i ? kSymIElectrons : 0) | (u.spec_j ? kSymJElectrons : 0) |
                (u.duty ? kSymDuty : 0) | ((sg.step0 & 1) ? kSymOddStep : 0);
      d.ib0 = u.ib0;
      d.ib1 = u.ib1;
      d.ni = u.spec_i ? sg.n_e : sg.n_h;
      d.nj = u.spec_j ? sg.n_e : sg.n_h;
      d.pI = u.p_i;
      d.pJ = u.p_j;
      d.tI = P.slot_tile0[u.slot] + (u.spec_i ? th : 0);
      d.tJ = P.slot_tile0[u.slot] + (u.spec_j ? th : 0);
    }
    s->h_sym_units[q] = d;
  }
  for (size_t t = 0; t < P.tiles.size(); ++t) {
    const SymTilePlan& tp = P.tiles[t];
    const SymGeom& sg = g[tp.slot];
    SymTile d{};
    d.off = sg.base + (tp.spec ? sg.cap_h : 0) + (int64_t)kSymTile * tp.tile;
    d.slot = tp.slot;
    d.spec = tp.spec;
    d.n = tp.n;
    d.lptr = tp.lptr;
    d.lcnt = tp.lcnt;
    d.ntiles = P.slot_ntiles[tp.slot];
    s->h_sym_tiles[t] = d;
  }
  std::memcpy(s->h_sym_lists, P.lists.data(), P.lists.size() * sizeof(int32_t));
  *s->h_sym_nu = nu;
  CK(h2d(s, s->d_sym_units, s->h_sym_units, std::max(nu, 1) * sizeof(SymUnit)));
  CK(h2d(s, s->d_sym_tiles, s->h_sym_tiles, std::max<size_t>(P.tiles.size(), 1) * sizeof(SymTile)));
  CK(h2d(s, s->d_sym_lists, s->h_sym_lists, std::max<size_t>(P.lists.size(), 1) * sizeof(int32_t)));
  CK(h2d(s, s->d_sym_nu, s->h_sym_nu, sizeof(int32_t)));
  return SIM_OK;
}

// Build and upload the unit list of the running slots.
int upload_units(sim_t* s, bool allow_split, bool slot_major = false) {
  if (s->sym) {
    std::vector<SymGeom> geom(s->S);
    for (int k = 0; k < s->S; ++k) {
      const HostSlot& h = s->slots[k];
      geom[k].base = h.base;
      geom[k].cap_h = h.rec.cap_h;
      geom[k].step0 = h.n_steps;
      if (h.used && h.running) {
        geom[k].n_h = h.n_h;
        geom[k].n_e = h.n_e;
      }
    }
    return upload_sym_plan(s, geom);
  }
  std::vector<int32_t> nh(s->S, 0), ne(s->S, 0);
  for (int k = 0; k < s->S; ++k)
    if (s->slots[k].used && s->slots[k].running) {
      nh[k] = s->slots[k].n_h;
      ne[k] = s->slots[k].n_e;
    }
  int64_t pfl = 0;
  const bool split = allow_split && s->ph.repulsion;
  const int rc = plan_units(nh.data(), ne.data(), s->S, s->tile_i, s->grid, split, kMaxUnits,
                            s->partial_cap, &s->plan, &s->plan_begin, &pfl,
                            split && s->dynamic, split && s->dynamic && slot_major);
  if (rc != 0) {
    s->err = "unit plan does not fit the unit buffer";
    return SIM_EINVAL;
  }
  if (pfl > s->partial_cap) {
    // the kernels would write partial sums past their buffer
    s->err = "unit plan exceeds the partial-sum buffer";
    return SIM_ECUDA;
  }
  const int n = (int)s->plan.size();
  std::vector<SlotGeom> geom(s->S);
  for (int k = 0; k < s->S; ++k) {
    const HostSlot& h = s->slots[k];
    geom[k].base = h.base;
    geom[k].cap_h = h.rec.cap_h;
    geom[k].n_h = h.n_h;
    geom[k].step0 = h.n_steps;
  }
  device_units(s->plan, geom, s->h_units);
  std::memcpy(s->h_cta_begin, s->plan_begin.data(), (s->grid + 1) * sizeof(int32_t));
  CK(h2d(s, s->d_units, s->h_units, std::max(n, 1) * sizeof(Unit)));
  CK(h2d(s, s->d_cta_begin, s->h_cta_begin, (s->grid + 1) * sizeof(int32_t)));
  return SIM_OK;
}

// Issue one chunk: K fused steps (one launch per chunk, or one per step), or
// in PLAIN mode field + update launches for one step; then the close kernel
// and the summary copy.
int issue_chunk(sim_t* s, int K, bool multi) {
  const bool plain = s->opt.mode == CTS_MODE_PLAIN;
  CK(cudaMemsetAsync(s->d_unit_counter, 0, K * sizeof(int32_t), s->stream));
  CK(cudaMemsetAsync(s->d_ret, 0, (size_t)K * s->S * 2 * sizeof(int32_t), s->stream));
  CK(cudaMemsetAsync(s->d_tiles_done, 0, (size_t)K * s->S * sizeof(int32_t), s->stream));
  if (s->sym)
    CK(cudaMemsetAsync(s->d_sym_ready, 0, (size_t)K * s->S * sizeof(int32_t), s->stream));
  if (s->d_induced)
    CK(cudaMemsetAsync(s->d_induced, 0, (size_t)K * s->S * sizeof(double), s->stream));
  if (s->d_induced_px)
    CK(cudaMemsetAsync(s->d_induced_px, 0, (size_t)K * s->S * 9 * sizeof(double), s->stream));
  if (s->field.spherical) {
    // the spherical model: one cluster of CTAs per slot runs all K steps of
    // its event
    const StepArgs a = step_args(s, true);
    const bool timed = s->opt.time_launches != 0 && !plain;
    const unsigned evflag = capturing(s) ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (timed) CK(cudaEventRecordWithFlags(s->lev[0], s->stream, evflag));
    CK(launch_spherical(a, 0, K, s->sph_cluster, s->stream));
    if (timed) CK(cudaEventRecordWithFlags(s->lev[1], s->stream, evflag));
    s->st_launch += 1;
  } else if (plain) {
    const StepArgs a = step_args(s, false);
    CK(launch_step(s->variant, a, 0, 1, s->grid, s->stream));
    // one thread per carrier of the running event (the grid is captured
    // nowhere: PLAIN chunks are launched directly)
    int n = 0;
    for (const HostSlot& h : s->slots)
      if (h.used && h.running) n = std::max(n, h.n_h + h.n_e);
    const int grid = std::min(std::max(1, (n + 255) / 256), s->sm_count * 4);
    CK(launch_update(a, 0, 1, s->d_list, grid, s->stream));
    s->st_launch += 2;
  } else {
    const StepArgs a = step_args(s, true);
    const bool timed = s->opt.time_launches != 0;
    // inside a stream capture the events become external event-record nodes
    const unsigned evflag = capturing(s) ? cudaEventRecordExternal : cudaEventRecordDefault;
    if (timed) CK(cudaEventRecordWithFlags(s->lev[0], s->stream, evflag));
    if (multi) {
      CK(launch_step(s->variant, a, 0, K, s->grid, s->stream));
      if (timed) CK(cudaEventRecordWithFlags(s->lev[1], s->stream, evflag));
      s->st_launch += 1;
    } else {
      for (int k = 0; k < K; ++k) {
        CK(launch_step(s->variant, a, k, 1, s->grid, s->stream));
        if (timed) CK(cudaEventRecordWithFlags(s->lev[k + 1], s->stream, evflag));
      }
      s->st_launch += K;
    }
  }
  CK(launch_close(s->ph, s->A, s->d_slots, nullptr, s->S, s->d_ret, s->S, K, s->d_summary,
                  s->stream));
  s->st_launch += 1;
  CK(d2h(s, s->h_summary, s->d_summary, s->S * sizeof(SlotSummary)));
  if (s->d_induced) CK(d2h(s, s->h_induced, s->d_induced, (size_t)K * s->S * sizeof(double)));
  if (s->d_induced_px)
    CK(d2h(s, s->h_induced_px, s->d_induced_px, (size_t)K * s->S * 9 * sizeof(double)));
  CK(d2h(s, s->h_err, s->d_err, sizeof(int32_t)));
  return SIM_OK;
}

int set_variant(sim_t* s, int v);

int run_chunk(sim_t* s) {
  NvtxRange range("cts chunk");
  const bool plain = s->opt.mode == CTS_MODE_PLAIN;
  const int K = plain ? 1 : s->K;
  if (plain) {
    // the update launch walks the running slot listed in d_list
    int n = 0;
    for (int k = 0; k < s->S; ++k)
      if (s->slots[k].used && s->slots[k].running) s->h_list[n++] = k;
    CK(h2d(s, s->d_list, s->h_list, std::max(n, 1) * sizeof(int32_t)));
  }
  if (!plain && !s->table_min.empty()) {
    double W = 0.0;
    for (auto& h : s->slots)
      if (h.used && h.running) W += (double)(h.n_h + h.n_e) * (double)(h.n_h + h.n_e);
    int v = s->table_var[0];
    for (size_t q = 0; q < s->table_min.size(); ++q)
      if (W >= (double)s->table_min[q]) v = s->table_var[q];
    int rcv = set_variant(s, v);
    if (rcv) return rcv;
  } else if (!plain && s->opt.variant == 0) {
    // the default choice per chunk: the symmetric kernel while the resident
    // pair work fills the GPU, the per-pair kernel (finer work units, shorter
    // steps) below it; the events' state is the same for both
    double W = 0.0;
    int max_tiles = 0;
    for (auto& h : s->slots)
      if (h.used && h.running) {
        W += (double)(h.n_h + h.n_e) * (double)(h.n_h + h.n_e);
        max_tiles = std::max(max_tiles, (h.n_h + kSymTile - 1) / kSymTile +
                                            (h.n_e + kSymTile - 1) / kSymTile);
      }
    const bool serve = s->opt.mode == CTS_MODE_SERVE;
    const int sym_v = (serve || max_tiles > kSymLargeTiles) ? kSymVariantLarge : kSymVariant;
    int rcv = set_variant(s, W >= (serve ? kSymMinWorkServe : kSymMinWork) ? sym_v : kPairVariant);
    if (rcv) return rcv;
  }
  // one launch for the whole chunk: the queue replays the step's pieces K
  // times, slot by slot
  const bool sph = s->field.spherical != 0;
  int rc = SIM_OK;
  if (!sph && s->sym) {
    // a symmetric plan larger than its buffers: this chunk runs the per-pair kernel
    rc = upload_units(s, true, true);
    if (rc == kSymPlanTooLarge) {
      rc = set_variant(s, kPairVariant);
      if (rc) return rc;
    } else if (rc) {
      return rc;
    }
  }
  const bool multi = !plain && !sph && s->dynamic && (s->sym || s->ph.repulsion) &&
                     !s->opt.step_launches;
  // PLAIN splits tiles too: one event alone must still spread over the SMs
  if (!sph && !s->sym) rc = upload_units(s, true, multi);
  if (rc) return rc;
  const int gi = sph ? 2 * variant_count() : 2 * s->variant + (multi ? 1 : 0);
  const int nl = (multi || sph) ? 1 : K;  // step-kernel launches in the chunk
  CK(cudaEventRecord(s->ev0, s->stream));
  if (!plain && !s->opt.disable_graphs) {
    cudaGraphExec_t& graph = s->graphs[gi];
    if (!graph || s->graph_K[gi] != K) {
      if (graph) {
        cudaGraphExecDestroy(graph);
        graph = nullptr;
      }
      cudaGraph_t g = nullptr;
      CK(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
      const int64_t launches = s->st_launch, hb = s->st_h2d, db = s->st_d2h;
      rc = issue_chunk(s, K, multi);
      s->st_launch = launches;
      s->st_h2d = hb;
      s->st_d2h = db;
      cudaError_t ce = cudaStreamEndCapture(s->stream, &g);
      if (rc) return rc;
      CK(ce);
      CK(cudaGraphInstantiate(&graph, g, 0));
      cudaGraphDestroy(g);
      s->graph_K[gi] = K;
    }
    CK(cudaGraphLaunch(graph, s->stream));
    s->st_launch += nl + 1;
    s->st_d2h += (int64_t)s->S * sizeof(SlotSummary) + sizeof(int32_t);
  } else {
    rc = issue_chunk(s, K, multi);
    if (rc) return rc;
  }
  CK(cudaEventRecord(s->ev1, s->stream));
  CK(cudaStreamSynchronize(s->stream));
  float ms = 0.f;
  CK(cudaEventElapsedTime(&ms, s->ev0, s->ev1));
  s->st_ms += ms;
  if (s->opt.time_launches && !plain) {
    double pairs = 0.0;
    if (s->sym) {
      for (const HostSlot& h : s->slots)
        if (h.used && h.running && h.n_h > 0) pairs += (double)(h.n_h + h.n_e) * (h.n_h + h.n_e);
    } else {
      for (const UnitPlan& u : s->plan) pairs += (double)u.ni * (double)(u.j1 - u.j0);
    }
    double running = 0.0;
    for (const HostSlot& h : s->slots) running += h.used && h.running;
    for (int k = 0; k < nl; ++k) {
      float lm = 0.f;
      CK(cudaEventElapsedTime(&lm, s->lev[k], s->lev[k + 1]));
      s->st_kernel_ms += lm;
      if (s->launch_log.size() >= kLaunchLogCap) s->launch_log.pop_front();
      s->launch_log.push_back({(double)lm, pairs * (K / nl), running, s->sym ? 1.0 : 0.0});
    }
    s->st_kernel_launches += nl;
  }
  s->st_steps += K;
  s->st_chunks += 1;
  if (*s->h_err & kErrTimeout) {
    s->broken = true;
    s->err = "a bounded device wait gave up";
    return SIM_ETIMEOUT;
  }
  if (*s->h_err & kErrPlan) {
    s->broken = true;
    s->err = "a unit descriptor disagrees with its slot on the device";
    return SIM_ECUDA;
  }
  if (*s->h_err & kErrBounds) {
    s->broken = true;
    s->err = "an index left its slot's range on the device (checked build)";
    return SIM_ECUDA;
  }
  return SIM_OK;
}

// Collect results of slots finished on the device (readout already binned).
int fetch_results(sim_t* s, const std::vector<int>& fin) {
  if (fin.empty()) return SIM_OK;
  NvtxRange range("cts readout");
  const int npix = s->sensor.grid_n * s->sensor.grid_n;
  const bool keep = s->opt.keep_final_xy != 0;
  std::vector<std::vector<double>> fx(fin.size()), fy(fin.size());
  std::vector<std::vector<int32_t>> rs(fin.size());
  for (size_t q = 0; q < fin.size(); ++q) {
    const int slot = fin[q];
    CK(d2h(s, s->h_pixels + (int64_t)slot * npix, s->d_pixels + (int64_t)slot * npix,
           npix * sizeof(int32_t)));
    CK(d2h(s, s->h_readout + slot, s->d_readout + slot, sizeof(SlotReadout)));
    if (keep) {
      const HostSlot& h = s->slots[slot];
      const int n = h.rec.cap_h + h.rec.cap_e;
      fx[q].resize(n);
      fy[q].resize(n);
      rs[q].resize(n);
      if (n) {
        CK(d2h(s, fx[q].data(), s->A.fx + h.base, n * sizeof(double)));
        CK(d2h(s, fy[q].data(), s->A.fy + h.base, n * sizeof(double)));
        CK(d2h(s, rs[q].data(), s->A.rstep + h.base, n * sizeof(int32_t)));
      }
    }
  }
  CK(cudaStreamSynchronize(s->stream));
  const double t = now_ns();
  std::vector<Done> out;
  for (size_t q = 0; q < fin.size(); ++q) {
    const int slot = fin[q];
    HostSlot& h = s->slots[slot];
    Done d;
    d.event_id = h.rec.ev.event_id;
    d.status = h.status;
    d.n_carriers = h.rec.cap_h + h.rec.cap_e;
    d.n_steps = h.n_steps;
    d.n_collected = s->h_readout[slot].n_collected;
    d.n_outside = s->h_readout[slot].n_outside;
    d.n_lost = s->h_readout[slot].n_lost;
    d.interactions = h.interactions;
    d.t_submit = h.rec.t_submit;
    d.t_start = h.t_start;
    d.t_done = t;
    d.order = h.rec.order;
    d.pixels.assign(s->h_pixels + (int64_t)slot * npix, s->h_pixels + (int64_t)(slot + 1) * npix);
    if (keep) {
      const int n = d.n_carriers;
      d.final_xy.resize(2 * (size_t)n);
      for (int c = 0; c < n; ++c) {
        d.final_xy[2 * c] = fx[q][c];
        d.final_xy[2 * c + 1] = fy[q][c];
      }
      d.rstep = std::move(rs[q]);
    }
    d.induced = std::move(h.induced);
    d.induced_px = std::move(h.induced_px);
    s->st_events += 1;
    s->st_inter += d.interactions;
    out.push_back(std::move(d));
    s->alloc.release(h.base);
    h = HostSlot{};
  }
  {
    std::lock_guard<std::mutex> lk(s->dmu);
    for (auto& d : out) s->done.push_back(std::move(d));
  }
  s->dcv.notify_all();
  return SIM_OK;
}

// One scheduling round: admit, initialise, step one chunk, retire.
// defer = true keeps finished results on the device (sim_execute).
int pump(sim_t* s, bool defer, bool* progressed) {
  *progressed = false;
  if (s->broken) return SIM_ECUDA;
  if (s->inject == SIM_ECUDA) {
    s->broken = true;
    s->err = "injected CUDA failure";
    return SIM_ECUDA;
  }
  int rc = admit(s);
  if (rc) return rc;
  rc = launch_inits(s);
  if (rc) return rc;
  bool any = false;
  for (auto& h : s->slots) any |= h.used && h.running;
  if (!any) return SIM_OK;
  rc = run_chunk(s);
  if (rc) return rc;
  *progressed = true;
  const bool inject_numeric = s->inject == SIM_ENUMERIC;
  if (inject_numeric) s->inject = 0;
  std::vector<int> fin;
  for (int k = 0; k < s->S; ++k) {
    HostSlot& h = s->slots[k];
    if (!h.used || !h.running) continue;
    const SlotSummary& m = s->h_summary[k];
    if (m.flags & kErrBounds) {
      s->broken = true;
      s->err = "an index left its slot's range on the device (checked build)";
      return SIM_ECUDA;
    }
    if (s->h_induced || s->h_induced_px) {
      // the steps this chunk executed for the slot, in order
      const int K = s->opt.mode == CTS_MODE_PLAIN ? 1 : s->K;
      const int64_t ran = std::min<int64_t>(std::max<int64_t>(m.n_steps - h.n_steps, 0), K);
      for (int64_t kk = 0; kk < ran; ++kk) {
        if (s->h_induced) {
          h.induced_q += s->h_induced[kk * s->S + k];
          h.induced.push_back(h.induced_q);
        }
        if (s->h_induced_px)
          for (int j = 0; j < 9; ++j) {
            h.induced_pxq[j] += s->h_induced_px[(kk * s->S + k) * 9 + j];
            h.induced_px.push_back(h.induced_pxq[j]);
          }
      }
    }
    h.n_h = m.n_h;
    h.n_e = m.n_e;
    h.n_steps = m.n_steps;
    h.interactions = (int64_t)m.interactions;
    if (m.done || inject_numeric) {
      h.running = false;
      h.status = inject_numeric ? SIM_ENUMERIC : m.status;
      fin.push_back(k);
    }
  }
  if (inject_numeric) {
    // the device still thinks these slots run: stop them there too
    for (int k : fin) {
      const int zero = 0;
      CK(cudaMemcpyAsync(&s->d_slots[k].running, &zero, sizeof(int), cudaMemcpyHostToDevice,
                         s->stream));
      CK(cudaStreamSynchronize(s->stream));
    }
  }
  if (fin.empty()) return SIM_OK;
  for (size_t q = 0; q < fin.size(); ++q) s->h_list[q] = fin[q];
  CK(h2d(s, s->d_list, s->h_list, fin.size() * sizeof(int32_t)));
  CK(launch_bin(s->ph, s->A, s->d_slots, s->d_list, (int)fin.size(), s->d_pixels, s->d_readout,
                s->stream));
  s->st_launch += 1;
  if (defer) {
    CK(cudaStreamSynchronize(s->stream));
    for (int k : fin) s->slots[k].finished_on_device = true;
    return SIM_OK;
  }
  return fetch_results(s, fin);
}

void copy_out(const Done& d, sim_result_t* r, int grid_n) {
  r->event_id = d.event_id;
  r->status = d.status;
  r->n_carriers = d.n_carriers;
  r->n_steps = d.n_steps;
  r->n_collected = d.n_collected;
  r->n_outside = d.n_outside;
  r->n_lost = d.n_lost;
  r->interactions = d.interactions;
  r->t_submit_ns = d.t_submit;
  r->t_start_ns = d.t_start;
  r->t_done_ns = d.t_done;
  if (r->pixels) std::memcpy(r->pixels, d.pixels.data(), (size_t)grid_n * grid_n * sizeof(int32_t));
  const int64_t n = std::min<int64_t>(r->capacity, d.n_carriers);
  if (r->final_xy) {
    for (int64_t c = 0; c < n; ++c) {
      r->final_xy[2 * c] = d.final_xy.empty() ? NAN : d.final_xy[2 * c];
      r->final_xy[2 * c + 1] = d.final_xy.empty() ? NAN : d.final_xy[2 * c + 1];
    }
  }
  if (r->retire_step)
    for (int64_t c = 0; c < n; ++c) r->retire_step[c] = d.rstep.empty() ? -2 : d.rstep[c];
  if (r->induced_e) {
    const int64_t m = std::min<int64_t>(r->induced_capacity, (int64_t)d.induced.size());
    for (int64_t k = 0; k < m; ++k) r->induced_e[k] = d.induced[(size_t)k];
    for (int64_t k = m; k < r->induced_capacity; ++k) r->induced_e[k] = NAN;
  }
  if (r->induced_px) {
    const int64_t m = std::min<int64_t>(r->induced_capacity, (int64_t)d.induced_px.size() / 9);
    for (int64_t k = 0; k < 9 * m; ++k) r->induced_px[k] = d.induced_px[(size_t)k];
    for (int64_t k = 9 * m; k < 9 * r->induced_capacity; ++k) r->induced_px[k] = NAN;
  }
}

void engine_main(sim_t* s) {
  cudaSetDevice(s->device);
  while (!s->stop.load()) {
    bool progressed = false;
    int rc;
    {
      std::lock_guard<std::mutex> lk(s->drive_mu);
      rc = pump(s, false, &progressed);
    }
    if (rc) {
      s->dcv.notify_all();
      std::unique_lock<std::mutex> lk(s->qmu);
      s->qcv.wait_for(lk, std::chrono::milliseconds(5));
      continue;
    }
    if (!progressed) {
      std::unique_lock<std::mutex> lk(s->qmu);
      if (s->queue.empty() && !s->stop.load())
        s->qcv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
}

template <typename T>
int dalloc(sim_t* s, T** p, size_t count) {
  CK(cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T)));
  return SIM_OK;
}
template <typename T>
int halloc(sim_t* s, T** p, size_t count) {
  CK(cudaMallocHost((void**)p, std::max<size_t>(count, 1) * sizeof(T)));
  std::memset((void*)*p, 0, std::max<size_t>(count, 1) * sizeof(T));
  return SIM_OK;
}

// Makes `device` current for a stateless entry point and restores the
// caller's current device when the call returns.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int device) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(device);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

int check_device(int device, int* sms) {
  int n = 0;
  if (cudaGetDeviceCount(&n) != cudaSuccess || n <= device || device < 0) return SIM_ENODEV;
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, device) != cudaSuccess) return SIM_ENODEV;
  if (p.major != 10 || p.minor != 3) return SIM_ENODEV;  // built for sm_103a only
  *sms = p.multiProcessorCount;
  return SIM_OK;
}

int alloc_all(sim_t* s) {
  const int64_t C = s->capacity;
  int rc = 0;
#define AL(p, n) \
  if ((rc = dalloc(s, &(p), (size_t)(n))) != 0) return rc
#define HL(p, n) \
  if ((rc = halloc(s, &(p), (size_t)(n))) != 0) return rc
  AL(s->A.px, C);
  AL(s->A.py, C);
  AL(s->A.pz, C);
  AL(s->A.sh[0], C);
  AL(s->A.sh[1], C);
  AL(s->A.cid, C);
  AL(s->A.fx, C);
  AL(s->A.fy, C);
  AL(s->A.rstep, C);
  AL(s->A.cstate, C);
  s->A.capacity = C;
  AL(s->d_slots, s->S);
  AL(s->d_summary, s->S);
  AL(s->d_readout, s->S);
  AL(s->d_pixels, (int64_t)s->S * s->sensor.grid_n * s->sensor.grid_n);
  AL(s->d_units, kMaxUnits);
  AL(s->d_cta_begin, kMaxGrid + 1);
  AL(s->d_unit_counter, kMaxK);
  AL(s->d_ret, (int64_t)kMaxK * s->S * 2);
  AL(s->d_partial, s->partial_cap);
  AL(s->d_combine, kMaxUnits);
  AL(s->d_tiles_done, (int64_t)kMaxK * s->S);
  if (s->opt.keep_induced & SIM_INDUCED_TOTAL) AL(s->d_induced, (int64_t)kMaxK * s->S);
  if (s->opt.keep_induced & SIM_INDUCED_PIXELS) AL(s->d_induced_px, (int64_t)kMaxK * s->S * 9);
  AL(s->d_err, 1);
  AL(s->d_explicit, C);
  AL(s->d_list, s->S);
  if (s->opt.mode == CTS_MODE_PLAIN) AL(s->d_field, 3 * C);
  // symmetric kernel: a slot of n carriers has at most n / 64 + 2 tiles
  s->sym_tiles_cap = C / kSymTile + 2 * (int64_t)s->S + 1;
  AL(s->d_sym_units, kMaxSymUnits);
  AL(s->d_sym_nu, 1);
  AL(s->d_sym_tiles, s->sym_tiles_cap);
  AL(s->d_sym_ctr, s->sym_tiles_cap);
  AL(s->d_sym_rec, (int64_t)kMaxK * s->S);
  AL(s->d_sym_ready, (int64_t)kMaxK * s->S);

  HL(s->h_sym_units, kMaxSymUnits);
  HL(s->h_sym_nu, 1);
  HL(s->h_sym_tiles, s->sym_tiles_cap);
  HL(s->h_summary, s->S);
  HL(s->h_units, kMaxUnits);
  HL(s->h_cta_begin, kMaxGrid + 1);
  HL(s->h_list, s->S);
  HL(s->h_slotdev, s->S);
  HL(s->h_readout, s->S);
  HL(s->h_pixels, (int64_t)s->S * s->sensor.grid_n * s->sensor.grid_n);
  HL(s->h_err, 1);
  if (s->opt.keep_induced & SIM_INDUCED_TOTAL) HL(s->h_induced, (int64_t)kMaxK * s->S);
  if (s->opt.keep_induced & SIM_INDUCED_PIXELS) HL(s->h_induced_px, (int64_t)kMaxK * s->S * 9);
#undef AL
#undef HL
  CK(cudaMemset(s->d_slots, 0, s->S * sizeof(SlotDev)));
  CK(cudaMemset(s->d_combine, 0, kMaxUnits * sizeof(int32_t)));
  CK(cudaMemset(s->d_partial, 0, std::max<int64_t>(s->partial_cap, 1) * sizeof(double)));
  CK(cudaMemset(s->d_err, 0, sizeof(int32_t)));
  CK(cudaMemset(s->d_sym_nu, 0, sizeof(int32_t)));
  CK(cudaMemset(s->d_sym_ctr, 0, (size_t)s->sym_tiles_cap * sizeof(int32_t)));

  CK(cudaEventCreate(&s->ev0));
  CK(cudaEventCreate(&s->ev1));
  s->lev.assign(kMaxK + 1, nullptr);
  for (auto& e : s->lev) CK(cudaEventCreate(&e));
  return SIM_OK;
}

void free_all(sim_t* s) {
  for (auto g : s->graphs)
    if (g) cudaGraphExecDestroy(g);
  void* dev[] = {s->A.px, s->A.py, s->A.pz, s->A.sh[0], s->A.sh[1], s->A.cid, s->A.fx, s->A.fy,
                 s->A.rstep, s->A.cstate, s->d_slots, s->d_summary, s->d_readout, s->d_pixels,
                 s->d_units, s->d_cta_begin, s->d_unit_counter, s->d_ret, s->d_partial,
                 s->d_combine, s->d_tiles_done, s->d_induced, s->d_err, s->d_field, s->d_explicit,
                 s->d_list, s->d_drift, s->d_induced_px, s->d_sym_units, s->d_sym_nu,
                 s->d_sym_tiles, s->d_sym_lists, s->d_sym_part, s->d_sym_ctr, s->d_sym_rec,
                 s->d_sym_ready};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {s->h_summary, s->h_units, s->h_cta_begin, s->h_list, s->h_slotdev, s->h_readout,
                  s->h_pixels, s->h_err, s->h_induced, s->h_induced_px, s->h_sym_units,
                  s->h_sym_nu, s->h_sym_tiles, s->h_sym_lists};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  if (s->ev0) cudaEventDestroy(s->ev0);
  if (s->ev1) cudaEventDestroy(s->ev1);
  for (auto e : s->lev)
    if (e) cudaEventDestroy(e);
  if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
}

// Pick the pair-kernel variant: explicit option, else the symmetric kernel
// (BATCHED and SERVE then choose per chunk by the resident work).  PLAIN, one
// event at a time, keeps the 12-warp symmetric kernel: measured on the 20 keV
// batch 9.5 events/s, against 7.8 with 8 warps and 8.3 for the per-pair kernel.
int choose_variant(sim_t* s) {
  if (s->opt.variant >= 1 && s->opt.variant <= variant_count()) return s->opt.variant - 1;
  return s->opt.mode == CTS_MODE_PLAIN ? kSymVariantPlain : kSymVariant;
}

int set_variant(sim_t* s, int v) {
  if (v == s->variant && s->grid > 0) return SIM_OK;
  int occ = s->occ_cache[v];
  if (occ <= 0) {
    CK(variant_occupancy(v, &occ));
    if (occ < 1) occ = 1;
    s->occ_cache[v] = occ;
  }
  const Variant vi = variant_info(v);
  if (vi.ctas_per_sm > 0) occ = std::min(occ, vi.ctas_per_sm);
  s->variant = v;
  s->grid = std::min(s->sm_count * occ, kMaxGrid);
  s->tile_i = vi.nt * vi.r;
  s->dynamic = vi.dynamic;
  s->sym = vi.sym != 0;
  return SIM_OK;
}

}  // namespace

// ============================================================================
// C ABI
// ============================================================================
extern "C" {

const char* sim_strerror(int code) {
  switch (code) {
    case SIM_OK: return "ok";
    case SIM_EINVAL: return "invalid argument";
    case SIM_ENOMEM_BUDGET: return "event larger than the device budget";
    case SIM_EAGAIN: return "admission queue full";
    case SIM_ETIMEOUT: return "timed out";
    case SIM_ECUDA: return "CUDA error";
    case SIM_EMAXSTEPS: return "step cap reached with holes still moving";
    case SIM_ENUMERIC: return "non-finite field or position";
    case SIM_ESTATE: return "call not valid in this mode or state";
    case SIM_ENODEV: return "no sm_103 CUDA device";
    default: return "unknown status";
  }
}

int sim_init(const sim_sensor_t* sensor, const sim_field_t* field, const sim_mobility_t* mobility,
             const sim_options_t* options, sim_t** out) {
  if (!out) return SIM_EINVAL;
  *out = nullptr;
  int rc = validate_params(sensor, field, mobility);
  if (rc) return rc;
  sim_options_t opt{};
  if (options) opt = *options;
  else opt.mode = CTS_MODE_BATCHED;
  if (opt.mode < CTS_MODE_PLAIN || opt.mode > CTS_MODE_SERVE) return SIM_EINVAL;
  if (opt.max_slots < 0 || opt.chunk_steps < 0 || opt.chunk_steps > kMaxK ||
      opt.max_carriers < 0 || opt.hbm_budget_bytes < 0 || opt.queue_capacity < 0 ||
      opt.variant < 0 || opt.variant > variant_count())
    return SIM_EINVAL;
  if (opt.sph_cluster != 0 && opt.sph_cluster != 1 && opt.sph_cluster != 2 &&
      opt.sph_cluster != 4)
    return SIM_EINVAL;
  if (opt.keep_induced < 0 || opt.keep_induced > (SIM_INDUCED_TOTAL | SIM_INDUCED_PIXELS))
    return SIM_EINVAL;
  // the 3 x 3 window around the centre pixel must lie inside the grid
  if ((opt.keep_induced & SIM_INDUCED_PIXELS) && sensor->grid_n < 3) return SIM_EINVAL;
  int sms = 0;
  rc = check_device(opt.device, &sms);
  if (rc) return rc;
  if (cudaSetDevice(opt.device) != cudaSuccess) return SIM_ENODEV;

  sim_t* s = new sim_t();
  s->sensor = *sensor;
  if (!(s->sensor.softening_um > 0)) s->sensor.softening_um = 1e-6;
  if (sensor->drift_table_n >= 2)
    s->drift_host.assign(sensor->drift_table_Vum, sensor->drift_table_Vum + sensor->drift_table_n);
  s->sensor.drift_table_Vum = s->drift_host.empty() ? nullptr : s->drift_host.data();
  s->sensor.drift_table_n = (int32_t)s->drift_host.size();
  s->field = *field;
  s->mob = *mobility;
  s->opt = opt;
  s->device = opt.device;
  s->sm_count = sms;
  s->ph = make_phys(s->sensor, s->field, s->mob);
  s->S = opt.mode == CTS_MODE_PLAIN ? 1 : (opt.max_slots > 0 ? opt.max_slots : kDefaultSlots);
  s->K = opt.chunk_steps > 0 ? opt.chunk_steps : kDefaultK;
  if (s->opt.queue_capacity == 0) s->opt.queue_capacity = kDefaultQueue;
  const int64_t budget = opt.hbm_budget_bytes > 0 ? opt.hbm_budget_bytes : kDefaultBudget;
  s->capacity = opt.max_carriers > 0 ? opt.max_carriers : std::max<int64_t>(budget / kBytesPerCarrier, 1024);
  if (s->capacity > (1ll << 28)) s->capacity = 1ll << 28;
  s->partial_cap = std::min<int64_t>(3 * (s->capacity + 64 * 4096), 64ll << 20);
  s->slots.resize(s->S);
  s->alloc = ArenaAllocator(s->capacity);
  if (opt.stream) {
    s->stream = (cudaStream_t)opt.stream;
  } else {
    if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return SIM_ECUDA;
    }
    s->own_stream = true;
  }
  s->graphs.assign(2 * variant_count() + 1, nullptr);
  s->graph_K.assign(2 * variant_count() + 1, -1);
  s->occ_cache.assign(variant_count(), 0);
  s->variant = -1;
  rc = alloc_all(s);
  if (!rc && !s->drift_host.empty()) {
    const size_t n = s->drift_host.size();
    std::vector<float> f(s->drift_host.begin(), s->drift_host.end());
    if (cudaMalloc(&s->d_drift, n * sizeof(float)) != cudaSuccess ||
        cudaMemcpy(s->d_drift, f.data(), n * sizeof(float), cudaMemcpyHostToDevice) != cudaSuccess) {
      rc = SIM_ECUDA;
    } else {
      s->ph.drift_tab = s->d_drift;
      s->ph.drift_n = (int32_t)n;
      s->ph.f_drift_inv_dz = (float)((double)(n - 1) / s->ph.H);
    }
  }
  if (!rc) rc = set_variant(s, choose_variant(s));
  if (!rc && s->field.spherical) {
    if (spherical_prepare() != cudaSuccess) rc = SIM_ECUDA;
    else s->sph_cluster = spherical_cluster(s->S, s->opt.sph_cluster);
  }
  s->base_variant = s->variant;
  {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, opt.device) == cudaSuccess) s->device_name = prop.name;
  }
  if (opt.autotune_cache) s->autotune_cache = opt.autotune_cache;
  s->opt.autotune_cache = nullptr;  // the caller's string is not kept
  if (!rc && !s->autotune_cache.empty()) {
    // a cached table measured on this device and build, if there is one
    std::vector<int64_t> mins(64);
    std::vector<int32_t> vars(64);
    int32_t n = 0;
    if (table_load(s->autotune_cache.c_str(), s->device_name.c_str(), variant_count(),
                   mins.data(), vars.data(), 64, &n) == 0 && n > 0) {
      s->table_min.assign(mins.begin(), mins.begin() + n);
      s->table_var.assign((size_t)n, 0);
      for (int q = 0; q < n; ++q) s->table_var[q] = vars[q] - 1;
    }
  }
  if (rc) {
    free_all(s);
    delete s;
    return rc;
  }
  if (opt.mode == CTS_MODE_SERVE) s->engine = std::thread(engine_main, s);
  *out = s;
  return SIM_OK;
}

int sim_destroy(sim_t* s) {
  if (!s) return SIM_EINVAL;
  if (s->engine.joinable()) {
    s->stop.store(true);
    s->qcv.notify_all();
    s->engine.join();
  }
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  free_all(s);
  delete s;
  return SIM_OK;
}

int sim_submit(sim_t* s, const sim_event_t* ev, int n_ev, int* n_accepted) {
  if (n_accepted) *n_accepted = 0;
  if (!s || (!ev && n_ev > 0) || n_ev < 0) return SIM_EINVAL;
  if (s->broken) return SIM_ECUDA;
  int acc = 0;
  int rc = SIM_OK;
  {
    std::lock_guard<std::mutex> lk(s->qmu);
    for (int k = 0; k < n_ev; ++k) {
      if ((int)s->queue.size() >= s->opt.queue_capacity) {
        rc = SIM_EAGAIN;
        break;
      }
      EventRec r;
      rc = prepare_event(s, &ev[k], &r);
      if (rc) break;
      r.t_submit = now_ns();
      r.order = s->order_counter++;
      s->queue.push_back(std::move(r));
      ++acc;
    }
    if (rc) s->st_rejected += n_ev - acc;
  }
  s->qcv.notify_all();
  if (n_accepted) *n_accepted = acc;
  return rc;
}

int sim_poll(sim_t* s, sim_result_t* out, int max_out, int* n_out, int timeout_ms) {
  if (n_out) *n_out = 0;
  if (!s || max_out < 0 || (max_out > 0 && !out)) return SIM_EINVAL;
  if (s->inject == SIM_ETIMEOUT) {
    s->inject = 0;
    return SIM_ETIMEOUT;
  }
  const double deadline = now_ns() + (timeout_ms < 0 ? 1e30 : timeout_ms * 1e6);
  cudaSetDevice(s->device);
  for (;;) {
    {
      std::lock_guard<std::mutex> lk(s->dmu);
      if (!s->done.empty() && max_out > 0) {
        int n = 0;
        while (n < max_out && !s->done.empty()) {
          copy_out(s->done.front(), &out[n], s->sensor.grid_n);
          s->done.pop_front();
          ++n;
        }
        if (n_out) *n_out = n;
        return SIM_OK;
      }
    }
    if (s->broken) return SIM_ECUDA;
    if (s->opt.mode == CTS_MODE_SERVE) {
      std::unique_lock<std::mutex> lk(s->dmu);
      if (s->done.empty()) {
        const double left_ms = (deadline - now_ns()) * 1e-6;
        if (left_ms <= 0) return SIM_ETIMEOUT;
        s->dcv.wait_for(lk, std::chrono::microseconds((int64_t)std::min(left_ms, 50.0) * 1000 + 1));
      }
      continue;
    }
    bool progressed = false;
    int rc;
    {
      std::lock_guard<std::mutex> lk(s->drive_mu);
      rc = pump(s, false, &progressed);
    }
    if (rc) return rc;
    if (!progressed) {
      // both queues at once, in the order sim_run takes them
      std::scoped_lock lk(s->qmu, s->dmu);
      if (s->done.empty() && (s->queue.empty() || now_ns() > deadline)) return SIM_ETIMEOUT;
    }
    if (now_ns() > deadline) {
      std::lock_guard<std::mutex> lk(s->dmu);
      if (s->done.empty()) return SIM_ETIMEOUT;
    }
  }
}

int sim_run(sim_t* s, const sim_event_t* ev, int n, sim_result_t* out) {
  if (!s || n < 0 || (n > 0 && (!ev || !out))) return SIM_EINVAL;
  int64_t first_order;
  {
    std::lock_guard<std::mutex> dl(s->drive_mu);
    for (auto& h : s->slots)
      if (h.used) return SIM_ESTATE;
    std::scoped_lock lk(s->qmu, s->dmu);
    if (!s->queue.empty() || !s->done.empty()) return SIM_ESTATE;
    first_order = s->order_counter;
  }
  int submitted = 0;
  int got = 0;
  std::vector<char> have((size_t)n, 0);
  while (got < n) {
    if (submitted < n) {
      int acc = 0;
      const int rc = sim_submit(s, ev + submitted, n - submitted, &acc);
      submitted += acc;
      if (rc && rc != SIM_EAGAIN) return rc;
    }
    Done d;
    bool have_done = false;
    {
      std::lock_guard<std::mutex> lk(s->dmu);
      if (!s->done.empty()) {
        d = std::move(s->done.front());
        s->done.pop_front();
        have_done = true;
      }
    }
    if (have_done) {
      const int64_t idx = d.order - first_order;
      if (idx >= 0 && idx < n && !have[idx]) {
        copy_out(d, &out[idx], s->sensor.grid_n);
        have[idx] = 1;
        ++got;
      }
      continue;
    }
    if (s->opt.mode == CTS_MODE_SERVE) {
      std::unique_lock<std::mutex> lk(s->dmu);
      if (s->done.empty()) s->dcv.wait_for(lk, std::chrono::milliseconds(5));
      if (s->broken) return SIM_ECUDA;
      continue;
    }
    bool progressed = false;
    int rc;
    {
      std::lock_guard<std::mutex> lk(s->drive_mu);
      rc = pump(s, false, &progressed);
    }
    if (rc) return rc;
    if (!progressed) {
      std::scoped_lock lk(s->qmu, s->dmu);
      if (s->done.empty() && s->queue.empty() && submitted >= n) return SIM_ESTATE;
    }
  }
  return SIM_OK;
}

int sim_stage(sim_t* s, const sim_event_t* ev, int n) {
  if (!s || n < 0 || (n > 0 && !ev)) return SIM_EINVAL;
  if (s->opt.mode != CTS_MODE_BATCHED) return SIM_ESTATE;
  if (s->broken) return SIM_ECUDA;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  for (auto& h : s->slots)
    if (h.used) return SIM_ESTATE;
  if (n > s->S) return SIM_ENOMEM_BUDGET;
  std::vector<EventRec> recs((size_t)n);
  int64_t need = 0;
  for (int k = 0; k < n; ++k) {
    const int rc = prepare_event(s, &ev[k], &recs[k]);
    if (rc) return rc;
    recs[k].t_submit = now_ns();
    recs[k].order = k;
    need += std::max<int64_t>((int64_t)recs[k].cap_h + recs[k].cap_e, 1);
  }
  if (need > s->capacity) return SIM_ENOMEM_BUDGET;
  s->staged.clear();
  for (int k = 0; k < n; ++k) {
    const int64_t base = s->alloc.alloc(std::max<int64_t>((int64_t)recs[k].cap_h + recs[k].cap_e, 1));
    if (base < 0) return SIM_ENOMEM_BUDGET;
    const int rc = place_event(s, k, std::move(recs[k]), base);
    if (rc) return rc;
    s->staged.push_back(k);
  }
  CK(cudaStreamSynchronize(s->stream));
  return SIM_OK;
}

int sim_execute(sim_t* s) {
  if (!s) return SIM_EINVAL;
  if (s->opt.mode != CTS_MODE_BATCHED) return SIM_ESTATE;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  for (;;) {
    bool any = false;
    for (auto& h : s->slots) any |= h.used && (h.running || h.needs_init);
    if (!any) break;
    bool progressed = false;
    // staged events only: nothing is admitted from the queue meanwhile
    std::deque<EventRec> parked;
    {
      std::lock_guard<std::mutex> lk(s->qmu);
      parked.swap(s->queue);
    }
    const int rc = pump(s, true, &progressed);
    {
      std::lock_guard<std::mutex> lk(s->qmu);
      for (auto it = parked.rbegin(); it != parked.rend(); ++it) s->queue.push_front(std::move(*it));
    }
    if (rc) return rc;
  }
  return SIM_OK;
}

int sim_collect(sim_t* s, sim_result_t* out, int max_out, int* n_out) {
  if (n_out) *n_out = 0;
  if (!s || max_out < 0 || (max_out > 0 && !out)) return SIM_EINVAL;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  std::vector<int> fin;
  for (int k : s->staged)
    if (s->slots[k].used && s->slots[k].finished_on_device) fin.push_back(k);
  const int rc = fetch_results(s, fin);
  if (rc) return rc;
  s->staged.clear();
  std::vector<Done> all;
  {
    std::lock_guard<std::mutex> lk(s->dmu);
    while (!s->done.empty()) {
      all.push_back(std::move(s->done.front()));
      s->done.pop_front();
    }
  }
  std::sort(all.begin(), all.end(), [](const Done& a, const Done& b) { return a.order < b.order; });
  int n = 0;
  for (auto& d : all) {
    if (n < max_out) copy_out(d, &out[n], s->sensor.grid_n);
    ++n;
  }
  if (n_out) *n_out = std::min(n, max_out);
  return SIM_OK;
}

int sim_get_stats(sim_t* s, sim_stats_t* o) {
  if (!s || !o) return SIM_EINVAL;
  *o = sim_stats_t{};
  o->events_done = s->st_events;
  o->interactions = s->st_inter;
  o->steps_launched = s->st_steps;
  o->kernel_launches = s->st_launch;
  o->chunks = s->st_chunks;
  {
    std::lock_guard<std::mutex> lk(s->qmu);
    o->queue_depth = (int64_t)s->queue.size();
  }
  o->rejected = s->st_rejected;
  o->sm_count = s->sm_count;
  o->variant = s->variant;
  o->device_ms = s->st_ms;
  o->step_kernel_ms = s->st_kernel_ms;
  o->step_kernel_launches = s->st_kernel_launches;
  o->h2d_bytes = s->st_h2d;
  o->d2h_bytes = s->st_d2h;
  o->symmetric = s->sym ? 1 : 0;
  o->sph_cluster = s->field.spherical ? s->sph_cluster : 0;
  return SIM_OK;
}

int sim_debug_inject(sim_t* s, int fault) {
  if (!s) return SIM_EINVAL;
  if (fault != 0 && fault != SIM_ENUMERIC && fault != SIM_ETIMEOUT && fault != SIM_ECUDA)
    return SIM_EINVAL;
  s->inject = fault;
  return SIM_OK;
}

// ---- kernel-level entry points --------------------------------------------

int sim_debug_field(sim_t* s, const float* x, const float* y, const float* z, int32_t n_h,
                    int32_t n_e, double* out_E) {
  if (!s || n_h < 0 || n_e < 0 || (n_h + n_e > 0 && (!x || !y || !z || !out_E)))
    return SIM_EINVAL;
  if (n_e > 0 && s->sensor.species != CTS_BOTH) return SIM_EINVAL;
  const int n = n_h + n_e;
  if (n == 0) return SIM_OK;
  if (n_h == 0) return SIM_EINVAL;  // the planner skips events without holes
  std::lock_guard<std::mutex> dl(s->drive_mu);
  cudaSetDevice(s->device);
  // a private arena and slot: the handle's resident events are untouched
  sim_t* t = s;
  Arena A{};
  SlotDev* d_slot = nullptr;
  float* d_field = nullptr;
  std::vector<float4> sh((size_t)n);
  for (int c = 0; c < n; ++c) sh[c] = make_float4(x[c], y[c], z[c], 0.0f);
  std::vector<UnitPlan> plan;
  std::vector<int32_t> begin;
  int64_t pfl = 0;
  const int32_t nh = n_h, ne = n_e;
  if (t->sym) {
    SymGeom g;
    g.cap_h = n_h;
    g.n_h = n_h;
    g.n_e = n_e;
    const int rcs = upload_sym_plan(t, std::vector<SymGeom>{g});
    if (rcs == kSymPlanTooLarge) return SIM_ENOMEM_BUDGET;
    if (rcs) return rcs;
  } else if (plan_units(&nh, &ne, 1, t->tile_i, t->grid, t->ph.repulsion != 0, kMaxUnits,
                        t->partial_cap, &plan, &begin, &pfl,
                        t->ph.repulsion != 0 && t->dynamic) != 0 ||
             pfl > t->partial_cap) {
    return SIM_EINVAL;
  }
  int rc = SIM_OK;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&A.sh[0], n * sizeof(float4))) != cudaSuccess) break;
    A.sh[1] = A.sh[0];
    A.capacity = n;
    if ((e = cudaMalloc(&d_slot, sizeof(SlotDev))) != cudaSuccess) break;
    if ((e = cudaMalloc(&d_field, 3 * (size_t)n * sizeof(float))) != cudaSuccess) break;
    SlotDev sd{};
    sd.base = 0;
    sd.cap_h = n_h;
    sd.cap_e = n_e;
    sd.n_h = n_h;
    sd.n_e = n_e;
    sd.act_h = n_h;
    sd.act_e = n_e;
    sd.n_total = n;
    sd.running = 1;
    if ((e = cudaMemcpyAsync(A.sh[0], sh.data(), n * sizeof(float4), cudaMemcpyHostToDevice,
                             s->stream)) != cudaSuccess)
      break;
    if ((e = cudaMemcpyAsync(d_slot, &sd, sizeof(SlotDev), cudaMemcpyHostToDevice, s->stream)) !=
        cudaSuccess)
      break;
    if (!t->sym) {
      SlotGeom sg;
      sg.cap_h = n_h;
      sg.n_h = n_h;
      device_units(plan, std::vector<SlotGeom>{sg}, s->h_units);
      std::memcpy(s->h_cta_begin, begin.data(), begin.size() * sizeof(int32_t));
      if ((e = cudaMemcpyAsync(s->d_units, s->h_units,
                               std::max<size_t>(plan.size(), 1) * sizeof(Unit),
                               cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
        break;
      if ((e = cudaMemcpyAsync(s->d_cta_begin, s->h_cta_begin, begin.size() * sizeof(int32_t),
                               cudaMemcpyHostToDevice, s->stream)) != cudaSuccess)
        break;
    }
    if ((e = cudaMemsetAsync(s->d_unit_counter, 0, sizeof(int32_t), s->stream)) != cudaSuccess)
      break;
    if ((e = cudaMemsetAsync(s->d_ret, 0, 2 * sizeof(int32_t), s->stream)) != cudaSuccess) break;
    StepArgs a = step_args(s, false);
    a.A = A;
    a.slots = d_slot;
    a.field_out = d_field;
    a.S = 1;
    if ((e = launch_step(s->variant, a, 0, 1, s->grid, s->stream)) != cudaSuccess) break;
    std::vector<float> f(3 * (size_t)n);
    if ((e = cudaMemcpyAsync(f.data(), d_field, 3 * (size_t)n * sizeof(float),
                             cudaMemcpyDeviceToHost, s->stream)) != cudaSuccess)
      break;
    if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess) break;
    for (int c = 0; c < n; ++c) {
      out_E[3 * c] = f[c];
      out_E[3 * c + 1] = f[(size_t)n + c];
      out_E[3 * c + 2] = f[2 * (size_t)n + c];
    }
  } while (0);
  if (e != cudaSuccess) {
    s->err = cudaGetErrorString(e);
    rc = SIM_ECUDA;
  }
  if (A.sh[0]) cudaFree(A.sh[0]);
  if (d_slot) cudaFree(d_slot);
  if (d_field) cudaFree(d_field);
  return rc;
}

int sim_debug_trace_step(sim_t* s, uint64_t* out, int32_t max_ctas, int32_t* n_ctas) {
  if (!s || !out || !n_ctas || max_ctas < 0) return SIM_EINVAL;
  if (s->opt.mode != CTS_MODE_BATCHED) return SIM_ESTATE;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  cudaSetDevice(s->device);
  int rc = launch_inits(s);
  if (rc) return rc;
  bool any = false;
  for (auto& h : s->slots) any |= h.used && h.running;
  if (!any) return SIM_ESTATE;
  rc = upload_units(s, true);
  if (rc == kSymPlanTooLarge) rc = SIM_ENOMEM_BUDGET;
  if (rc) return rc;
  float* d_field = nullptr;
  unsigned long long* d_trace = nullptr;
  cudaError_t e = cudaSuccess;
  // broadcast kernels: one record per CTA; the symmetric kernel: a counter,
  // the capacity and one record per unit, from word 8
  const size_t words = s->sym ? 8 * ((size_t)std::max(max_ctas, 0) + 1) : (size_t)8 * s->grid;
  std::vector<unsigned long long> h(words);
  do {
    if ((e = cudaMalloc(&d_field, 3 * (size_t)s->capacity * sizeof(float)))) break;
    if ((e = cudaMalloc(&d_trace, h.size() * sizeof(unsigned long long)))) break;
    if ((e = cudaMemsetAsync(d_trace, 0, h.size() * sizeof(unsigned long long), s->stream))) break;
    if (s->sym) {
      const unsigned long long cap = (unsigned long long)std::max(max_ctas, 0);
      if ((e = cudaMemcpyAsync(d_trace + 1, &cap, sizeof(cap), cudaMemcpyHostToDevice, s->stream)))
        break;
    }
    if ((e = cudaMemsetAsync(s->d_ret, 0, (size_t)s->S * 2 * sizeof(int32_t), s->stream))) break;
    if ((e = cudaMemsetAsync(s->d_unit_counter, 0, sizeof(int32_t), s->stream))) break;
    StepArgs a = step_args(s, false);
    a.field_out = d_field;
    a.trace = d_trace;
    if ((e = launch_step(s->variant, a, 0, 1, s->grid, s->stream))) break;
    if ((e = cudaMemcpyAsync(h.data(), d_trace, h.size() * sizeof(unsigned long long),
                             cudaMemcpyDeviceToHost, s->stream)))
      break;
    if ((e = cudaStreamSynchronize(s->stream))) break;
  } while (0);
  if (d_field) cudaFree(d_field);
  if (d_trace) cudaFree(d_trace);
  if (e != cudaSuccess) {
    s->err = cudaGetErrorString(e);
    return SIM_ECUDA;
  }
  if (s->sym) {
    const int n = (int)std::min<unsigned long long>(h[0], (unsigned long long)max_ctas);
    for (int r = 0; r < n; ++r)
      for (int q = 0; q < 8; ++q) out[8 * r + q] = h[8 + 8 * (size_t)r + q];
    *n_ctas = n;
    return SIM_OK;
  }
  const int n = std::min(max_ctas, s->grid);
  for (int g = 0; g < n; ++g)
    for (int q = 0; q < 8; ++q) out[8 * g + q] = h[8 * (size_t)g + q];
  *n_ctas = n;
  return SIM_OK;
}

int sim_debug_launch_log(sim_t* s, double* out, int32_t cap, int32_t* n_out) {
  if (!s || cap < 0 || !n_out || (cap > 0 && !out)) return SIM_EINVAL;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  const int n = (int)std::min<size_t>((size_t)cap, s->launch_log.size());
  for (int q = 0; q < n; ++q)
    for (int c = 0; c < 4; ++c) out[4 * q + c] = s->launch_log[q][c];
  s->launch_log.clear();
  *n_out = n;
  return SIM_OK;
}

int sim_set_variants(sim_t* s, const int64_t* min_pairs, const int32_t* variants, int32_t n) {
  if (!s || n < 0 || (n > 0 && (!min_pairs || !variants))) return SIM_EINVAL;
  for (int q = 0; q < n; ++q) {
    if (variants[q] < 1 || variants[q] > variant_count() || min_pairs[q] < 0) return SIM_EINVAL;
    if (q > 0 && min_pairs[q] < min_pairs[q - 1]) return SIM_EINVAL;
  }
  std::lock_guard<std::mutex> dl(s->drive_mu);
  s->table_min.assign(min_pairs, min_pairs + n);
  s->table_var.assign((size_t)n, 0);
  for (int q = 0; q < n; ++q) s->table_var[q] = variants[q] - 1;
  if (n == 0) return set_variant(s, s->base_variant);
  return SIM_OK;
}

int sim_reset(sim_t* s) {
  if (!s) return SIM_EINVAL;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  {
    std::lock_guard<std::mutex> lk(s->qmu);
    s->queue.clear();
  }
  {
    std::lock_guard<std::mutex> lk(s->dmu);
    s->done.clear();
  }
  cudaSetDevice(s->device);
  if (s->stream) cudaStreamSynchronize(s->stream);
  for (int k = 0; k < s->S; ++k) {
    HostSlot& h = s->slots[k];
    if (!h.used) continue;
    const int zero = 0;
    CK(cudaMemcpyAsync(&s->d_slots[k].running, &zero, sizeof(int), cudaMemcpyHostToDevice,
                       s->stream));
    s->alloc.release(h.base);
    h = HostSlot{};
  }
  s->staged.clear();
  CK(cudaStreamSynchronize(s->stream));
  return SIM_OK;
}

int sim_debug_time_step(sim_t* s, int32_t variant, int32_t reps, double* ms_per_launch) {
  if (!s || !ms_per_launch || reps < 1 || variant < 0 || variant > variant_count())
    return SIM_EINVAL;
  if (s->opt.mode != CTS_MODE_BATCHED) return SIM_ESTATE;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  cudaSetDevice(s->device);
  int rc = launch_inits(s);
  if (rc) return rc;
  bool any = false;
  for (auto& h : s->slots) any |= h.used && h.running;
  if (!any) return SIM_ESTATE;
  const int saved = s->variant;
  if (variant > 0) {
    rc = set_variant(s, variant - 1);
    if (rc) return rc;
  }
  rc = upload_units(s, true);
  if (rc == kSymPlanTooLarge) rc = SIM_ENOMEM_BUDGET;
  float* d_field = nullptr;
  cudaError_t e = cudaSuccess;
  float ms = 0.f;
  do {
    if (rc) break;
    if ((e = cudaMalloc(&d_field, 3 * (size_t)s->capacity * sizeof(float)))) break;
    if ((e = cudaMemsetAsync(s->d_ret, 0, (size_t)s->S * 2 * sizeof(int32_t), s->stream))) break;
    StepArgs a = step_args(s, false);
    a.field_out = d_field;
    for (int r = 0; r <= reps && e == cudaSuccess; ++r) {  // launch 0 warms up
      if (r == 1 && (e = cudaEventRecord(s->ev0, s->stream))) break;
      if ((e = cudaMemsetAsync(s->d_unit_counter, 0, sizeof(int32_t), s->stream))) break;
      if ((e = launch_step(s->variant, a, 0, 1, s->grid, s->stream))) break;
    }
    if (e) break;
    if ((e = cudaEventRecord(s->ev1, s->stream))) break;
    if ((e = cudaStreamSynchronize(s->stream))) break;
    if ((e = cudaEventElapsedTime(&ms, s->ev0, s->ev1))) break;
  } while (0);
  if (d_field) cudaFree(d_field);
  const int rc2 = set_variant(s, saved);
  if (rc) return rc;
  if (e != cudaSuccess) {
    s->err = cudaGetErrorString(e);
    return SIM_ECUDA;
  }
  *ms_per_launch = ms / reps;
  return rc2;
}

int sim_get_variants(sim_t* s, int64_t* min_pairs, int32_t* variants, int32_t cap,
                     int32_t* n_out) {
  if (!s || !n_out || cap < 0 || (cap > 0 && (!min_pairs || !variants))) return SIM_EINVAL;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  const int n = (int)s->table_min.size();
  for (int q = 0; q < n && q < cap; ++q) {
    min_pairs[q] = s->table_min[q];
    variants[q] = s->table_var[q] + 1;
  }
  *n_out = n;
  return SIM_OK;
}

int sim_autotune(sim_t* s, const sim_event_t* ev, int32_t n, int32_t reps, int32_t* n_buckets) {
  if (!s || !ev || n < 1 || reps < 1 || !n_buckets) return SIM_EINVAL;
  if (s->opt.mode != CTS_MODE_BATCHED) return SIM_ESTATE;
  int rc = sim_reset(s);
  if (rc) return rc;
  // batch sizes n, n/2, ..., 1; for each the pair work W and the fastest variant
  std::vector<std::pair<double, int>> best;
  for (int m = std::min(n, s->S); m >= 1; m /= 2) {
    rc = sim_stage(s, ev, m);
    if (rc) return rc;
    double W = 0.0;
    for (auto& h : s->slots)
      if (h.used) W += (double)(h.n_h + h.n_e) * (double)(h.n_h + h.n_e);
    int bv = -1;
    double bt = 1e30;
    for (int v = 1; v <= variant_count(); ++v) {
      double ms = 0.0;
      rc = sim_debug_time_step(s, v, reps, &ms);
      if (rc) return rc;
      if (ms < bt) {
        bt = ms;
        bv = v;
      }
    }
    best.push_back({W, bv});
    rc = sim_reset(s);
    if (rc) return rc;
    if (m == 1) break;
  }
  std::sort(best.begin(), best.end());
  std::vector<int64_t> mins;
  std::vector<int32_t> vars;
  for (size_t q = 0; q < best.size(); ++q) {
    const double lo = q == 0 ? 0.0 : std::sqrt(best[q - 1].first * best[q].first);
    if (!vars.empty() && vars.back() == best[q].second) continue;  // merge equal neighbours
    mins.push_back((int64_t)lo);
    vars.push_back(best[q].second);
  }
  rc = sim_set_variants(s, mins.data(), vars.data(), (int32_t)mins.size());
  *n_buckets = (int32_t)mins.size();
  if (!rc && !s->autotune_cache.empty())
    table_save(s->autotune_cache.c_str(), s->device_name.c_str(), variant_count(), mins.data(),
               vars.data(), (int32_t)mins.size());
  return rc;
}

int sim_debug_bin(sim_t* s, const double* x, const double* y, int64_t n, int32_t* pixels,
                  int64_t* outside) {
  if (!s || n < 0 || !pixels || !outside || (n > 0 && (!x || !y))) return SIM_EINVAL;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  cudaSetDevice(s->device);
  const int npix = s->sensor.grid_n * s->sensor.grid_n;
  double *dx = nullptr, *dy = nullptr;
  int32_t* dp = nullptr;
  long long* dout = nullptr;
  cudaError_t e = cudaSuccess;
  do {
    if ((e = cudaMalloc(&dx, std::max<int64_t>(n, 1) * sizeof(double))) != cudaSuccess) break;
    if ((e = cudaMalloc(&dy, std::max<int64_t>(n, 1) * sizeof(double))) != cudaSuccess) break;
    if ((e = cudaMalloc(&dp, npix * sizeof(int32_t))) != cudaSuccess) break;
    if ((e = cudaMalloc(&dout, sizeof(long long))) != cudaSuccess) break;
    if (n > 0) {
      if ((e = cudaMemcpyAsync(dx, x, n * sizeof(double), cudaMemcpyHostToDevice, s->stream))) break;
      if ((e = cudaMemcpyAsync(dy, y, n * sizeof(double), cudaMemcpyHostToDevice, s->stream))) break;
    }
    if ((e = cudaMemsetAsync(dp, 0, npix * sizeof(int32_t), s->stream))) break;
    if ((e = cudaMemsetAsync(dout, 0, sizeof(long long), s->stream))) break;
    if ((e = launch_bin_points(s->ph, dx, dy, n, dp, dout, s->stream))) break;
    long long o = 0;
    if ((e = cudaMemcpyAsync(pixels, dp, npix * sizeof(int32_t), cudaMemcpyDeviceToHost, s->stream))) break;
    if ((e = cudaMemcpyAsync(&o, dout, sizeof(long long), cudaMemcpyDeviceToHost, s->stream))) break;
    if ((e = cudaStreamSynchronize(s->stream))) break;
    *outside = o;
  } while (0);
  if (dx) cudaFree(dx);
  if (dy) cudaFree(dy);
  if (dp) cudaFree(dp);
  if (dout) cudaFree(dout);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

int sim_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                     uint32_t* curand_out) {
  if (n < 0 || (n > 0 && (!ctr || !key || !out))) return SIM_EINVAL;
  int sms = 0;
  if (check_device(0, &sms)) return SIM_ENODEV;
  cudaSetDevice(0);
  uint32_t *dc = nullptr, *dk = nullptr, *dout = nullptr, *dcur = nullptr;
  cudaError_t e = cudaSuccess;
  const size_t m = (size_t)std::max<int64_t>(n, 1);
  do {
    if ((e = cudaMalloc(&dc, 4 * m * sizeof(uint32_t)))) break;
    if ((e = cudaMalloc(&dk, 2 * m * sizeof(uint32_t)))) break;
    if ((e = cudaMalloc(&dout, 4 * m * sizeof(uint32_t)))) break;
    if (curand_out && (e = cudaMalloc(&dcur, 4 * m * sizeof(uint32_t)))) break;
    if (n > 0) {
      if ((e = cudaMemcpy(dc, ctr, 4 * n * sizeof(uint32_t), cudaMemcpyHostToDevice))) break;
      if ((e = cudaMemcpy(dk, key, 2 * n * sizeof(uint32_t), cudaMemcpyHostToDevice))) break;
    }
    if ((e = launch_philox(dc, dk, n, dout, dcur, 0))) break;
    if ((e = cudaDeviceSynchronize())) break;
    if (n > 0) {
      if ((e = cudaMemcpy(out, dout, 4 * n * sizeof(uint32_t), cudaMemcpyDeviceToHost))) break;
      if (curand_out &&
          (e = cudaMemcpy(curand_out, dcur, 4 * n * sizeof(uint32_t), cudaMemcpyDeviceToHost)))
        break;
    }
  } while (0);
  cudaFree(dc);
  cudaFree(dk);
  cudaFree(dout);
  if (dcur) cudaFree(dcur);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

int sim_generate(const sim_gen_event_t* events, int32_t n_events, double pitch_um, int32_t grid_n,
                 int32_t device, int32_t* pixels, int64_t* outside) {
  static_assert(sizeof(sim_gen_event_t) == sizeof(GenEvent), "generation record layout");
  if (n_events < 0 || device < 0 || grid_n < 1 || grid_n > kReadoutMaxGrid ||
      !(pitch_um > 0.0) || !std::isfinite(pitch_um))
    return SIM_EINVAL;
  if (n_events > 0 && (!events || !pixels)) return SIM_EINVAL;
  for (int32_t k = 0; k < n_events; ++k) {
    const sim_gen_event_t& e = events[k];
    if (e.n_pairs < 0 || !(e.alpha > 0.0) || !(e.beta >= 0.3 && e.beta <= 20.0) ||
        !std::isfinite(e.alpha) || !std::isfinite(e.x_um) || !std::isfinite(e.y_um))
      return SIM_EINVAL;
  }
  int sms = 0;
  if (check_device(device, &sms)) return SIM_ENODEV;
  DeviceGuard guard(device);
  if (n_events == 0) return SIM_OK;
  const size_t ne = (size_t)n_events, np = (size_t)grid_n * grid_n;
  GenEvent* dev = nullptr;
  int32_t* dp = nullptr;
  unsigned long long* dout = nullptr;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaSuccess;
  std::vector<unsigned long long> hout(outside ? ne : 0);
  do {
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) break;
    if ((e = cudaMalloc(&dev, ne * sizeof(GenEvent)))) break;
    if ((e = cudaMalloc(&dp, ne * np * sizeof(int32_t)))) break;
    if ((e = cudaMalloc(&dout, ne * sizeof(unsigned long long)))) break;
    if ((e = cudaMemcpyAsync(dev, events, ne * sizeof(GenEvent), cudaMemcpyHostToDevice, st)))
      break;
    if ((e = launch_generate(dev, n_events, pitch_um, grid_n, dp, dout, st))) break;
    if ((e = cudaMemcpyAsync(pixels, dp, ne * np * sizeof(int32_t), cudaMemcpyDeviceToHost, st)))
      break;
    if (outside && (e = cudaMemcpyAsync(hout.data(), dout, ne * sizeof(unsigned long long),
                                        cudaMemcpyDeviceToHost, st)))
      break;
    if ((e = cudaStreamSynchronize(st))) break;
    for (size_t k = 0; k < hout.size(); ++k) outside[k] = (int64_t)hout[k];
  } while (0);
  cudaFree(dev);
  cudaFree(dp);
  cudaFree(dout);
  if (st) cudaStreamDestroy(st);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

int sim_readout(const sim_readout_params_t* prm, const int32_t* counts, const uint64_t* seeds,
                const uint64_t* event_ids, int32_t n_events, int32_t device, double* pixel_keV,
                sim_cluster_t* clusters, int64_t* spectrum) {
  static_assert(sizeof(sim_cluster_t) == sizeof(ClusterRec), "cluster record layout");
  if (!prm || n_events < 0 || device < 0) return SIM_EINVAL;
  const int g = prm->grid_n;
  if (g < 1 || g > kReadoutMaxGrid || prm->n_bins < 0) return SIM_EINVAL;
  if (prm->n_bins > 0 && (!spectrum || !(prm->spec_bin_keV > 0.0))) return SIM_EINVAL;
  if (!(prm->noise_keV >= 0.0) || !(prm->window_keV >= 0.0) || !(prm->ev_per_pair > 0.0))
    return SIM_EINVAL;
  if (n_events > 0 && (!counts || !seeds || !event_ids || !clusters)) return SIM_EINVAL;
  int sms = 0;
  if (check_device(device, &sms)) return SIM_ENODEV;
  DeviceGuard guard(device);
  if (n_events == 0) return SIM_OK;
  const size_t np = (size_t)g * g, ne = (size_t)n_events;
  ReadoutArgs r{};
  r.grid_n = g;
  r.n_bins = prm->n_bins;
  r.ev_per_pair = prm->ev_per_pair;
  r.noise_keV = prm->noise_keV;
  r.beam_keV = prm->beam_keV;
  r.window_keV = prm->window_keV;
  r.veto_factor = prm->veto_factor;
  r.spec_lo_keV = prm->spec_lo_keV;
  r.spec_bin_keV = prm->spec_bin_keV;
  int32_t* dc = nullptr;
  unsigned long long *ds = nullptr, *di = nullptr, *dh = nullptr;
  double* de = nullptr;
  ClusterRec* dcl = nullptr;
  cudaStream_t st = nullptr;
  cudaError_t e = cudaSuccess;
  std::vector<unsigned long long> hist((size_t)std::max(prm->n_bins, 1), 0ull);
  do {
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking))) break;
    if ((e = cudaMalloc(&dc, ne * np * sizeof(int32_t)))) break;
    if ((e = cudaMalloc(&ds, ne * sizeof(unsigned long long)))) break;
    if ((e = cudaMalloc(&di, ne * sizeof(unsigned long long)))) break;
    if ((e = cudaMalloc(&dcl, ne * sizeof(ClusterRec)))) break;
    if (pixel_keV && (e = cudaMalloc(&de, ne * np * sizeof(double)))) break;
    if (prm->n_bins > 0) {
      if ((e = cudaMalloc(&dh, (size_t)prm->n_bins * sizeof(unsigned long long)))) break;
      if ((e = cudaMemsetAsync(dh, 0, (size_t)prm->n_bins * sizeof(unsigned long long), st)))
        break;
    }
    if ((e = cudaMemcpyAsync(dc, counts, ne * np * sizeof(int32_t), cudaMemcpyHostToDevice, st)))
      break;
    if ((e = cudaMemcpyAsync(ds, seeds, ne * sizeof(uint64_t), cudaMemcpyHostToDevice, st))) break;
    if ((e = cudaMemcpyAsync(di, event_ids, ne * sizeof(uint64_t), cudaMemcpyHostToDevice, st)))
      break;
    r.counts = dc;
    r.seeds = ds;
    r.ids = di;
    r.pixel_keV = de;
    r.clusters = dcl;
    r.spectrum = dh;
    if ((e = launch_readout(r, n_events, st))) break;
    if ((e = cudaMemcpyAsync(clusters, dcl, ne * sizeof(ClusterRec), cudaMemcpyDeviceToHost, st)))
      break;
    if (de && (e = cudaMemcpyAsync(pixel_keV, de, ne * np * sizeof(double),
                                   cudaMemcpyDeviceToHost, st)))
      break;
    if (dh && (e = cudaMemcpyAsync(hist.data(), dh, (size_t)prm->n_bins * sizeof(unsigned long long),
                                   cudaMemcpyDeviceToHost, st)))
      break;
    if ((e = cudaStreamSynchronize(st))) break;
    for (int b = 0; b < prm->n_bins; ++b) spectrum[b] += (int64_t)hist[b];
  } while (0);
  cudaFree(dc);
  cudaFree(ds);
  cudaFree(di);
  cudaFree(dcl);
  if (de) cudaFree(de);
  if (dh) cudaFree(dh);
  if (st) cudaStreamDestroy(st);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

int sim_build_flags(void) {
#ifdef CTS_BOUNDS_CHECK
  return SIM_BUILD_BOUNDS_CHECK;
#else
  return 0;
#endif
}

int sim_debug_fma_peak(int32_t device, int32_t packed, double* flops_per_s) {
  if (!flops_per_s || device < 0) return SIM_EINVAL;
  int sms = 0;
  if (check_device(device, &sms)) return SIM_ENODEV;
  DeviceGuard guard(device);
  const int grid = sms * 8;  // 2048 threads per SM
  const int iters = 1 << 11;
  float* d = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaSuccess;
  float best = 0.0f;
  do {
    if ((e = cudaMalloc(&d, (size_t)grid * 256 * sizeof(float)))) break;
    if ((e = cudaEventCreate(&e0)) || (e = cudaEventCreate(&e1))) break;
    if ((e = launch_fma_chain(packed != 0, d, grid, iters / 8, 0))) break;  // warm-up
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      if ((e = cudaEventRecord(e0, 0))) break;
      if ((e = launch_fma_chain(packed != 0, d, grid, iters, 0))) break;
      if ((e = cudaEventRecord(e1, 0))) break;
      if ((e = cudaEventSynchronize(e1))) break;
      float ms = 0.0f;
      if ((e = cudaEventElapsedTime(&ms, e0, e1))) break;
      if (best == 0.0f || ms < best) best = ms;
    }
  } while (0);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (d) cudaFree(d);
  if (e != cudaSuccess || !(best > 0.0f)) return SIM_ECUDA;
  // 16 FMA lane-ops = 32 flops per thread and iteration
  *flops_per_s = (double)grid * 256.0 * iters * 32.0 / (best * 1e-3);
  return SIM_OK;
}

int sim_debug_normals(const uint64_t* in, int64_t n, double* out) {
  if (n < 0 || (n > 0 && (!in || !out))) return SIM_EINVAL;
  int sms = 0;
  if (check_device(0, &sms)) return SIM_ENODEV;
  cudaSetDevice(0);
  unsigned long long* din = nullptr;
  double* dout = nullptr;
  cudaError_t e = cudaSuccess;
  const size_t m = (size_t)std::max<int64_t>(n, 1);
  do {
    if ((e = cudaMalloc(&din, 5 * m * sizeof(unsigned long long)))) break;
    if ((e = cudaMalloc(&dout, 3 * m * sizeof(double)))) break;
    if (n > 0 && (e = cudaMemcpy(din, in, 5 * n * sizeof(uint64_t), cudaMemcpyHostToDevice))) break;
    if ((e = launch_normals(din, n, dout, 0))) break;
    if ((e = cudaDeviceSynchronize())) break;
    if (n > 0 && (e = cudaMemcpy(out, dout, 3 * n * sizeof(double), cudaMemcpyDeviceToHost))) break;
  } while (0);
  cudaFree(din);
  cudaFree(dout);
  return e == cudaSuccess ? SIM_OK : SIM_ECUDA;
}

int sim_debug_trajectory(sim_t* s, const sim_event_t* ev, int64_t n_steps, double* pos_out,
                         int8_t* state_out, int64_t capacity, int64_t* steps_done) {
  if (!s || !ev || n_steps < 0 || !pos_out || !state_out || !steps_done) return SIM_EINVAL;
  if (s->opt.mode != CTS_MODE_BATCHED) return SIM_ESTATE;
  std::lock_guard<std::mutex> dl(s->drive_mu);
  for (auto& h : s->slots)
    if (h.used) return SIM_ESTATE;
  {
    std::lock_guard<std::mutex> lk(s->qmu);
    if (!s->queue.empty()) return SIM_ESTATE;
  }
  cudaSetDevice(s->device);
  EventRec r;
  int rc = prepare_event(s, ev, &r);
  if (rc) return rc;
  const int n = r.cap_h + r.cap_e;
  if (capacity < n) return SIM_EINVAL;
  const int64_t base = s->alloc.alloc(std::max(n, 1));
  if (base < 0) return SIM_ENOMEM_BUDGET;
  const Phys saved = s->ph;
  s->ph.max_steps = std::min<int64_t>(s->ph.max_steps, n_steps);
  const int savedK = s->K;
  const int saved_graphs = s->opt.disable_graphs;
  s->opt.disable_graphs = 1;
  s->K = (int)std::min<int64_t>(std::max<int64_t>(n_steps, 1), savedK);
  rc = place_event(s, 0, std::move(r), base);
  while (!rc) {
    bool any = s->slots[0].used && (s->slots[0].running || s->slots[0].needs_init);
    if (!any) break;
    rc = launch_inits(s);
    if (rc) break;
    if (!s->slots[0].running) break;
    rc = run_chunk(s);
    if (rc) break;
    const SlotSummary& m = s->h_summary[0];
    s->slots[0].n_h = m.n_h;
    s->slots[0].n_e = m.n_e;
    s->slots[0].n_steps = m.n_steps;
    if (m.done) s->slots[0].running = false;
  }
  if (!rc) {
    std::vector<double> px(n), py(n), pz(n), fx(n), fy(n);
    std::vector<int32_t> cid(n);
    std::vector<int8_t> cs(n);
    const int nh = s->slots[0].n_h, ne = s->slots[0].n_e;
    do {
      if (n == 0) break;
      cudaError_t e = cudaSuccess;
      if ((e = cudaMemcpy(px.data(), s->A.px + base, n * sizeof(double), cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(py.data(), s->A.py + base, n * sizeof(double), cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(pz.data(), s->A.pz + base, n * sizeof(double), cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(fx.data(), s->A.fx + base, n * sizeof(double), cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(fy.data(), s->A.fy + base, n * sizeof(double), cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(cid.data(), s->A.cid + base, n * sizeof(int32_t), cudaMemcpyDeviceToHost)) ||
          (e = cudaMemcpy(cs.data(), s->A.cstate + base, n, cudaMemcpyDeviceToHost))) {
        s->err = cudaGetErrorString(e);
        rc = SIM_ECUDA;
        break;
      }
      for (int c = 0; c < n; ++c) {
        pos_out[3 * c] = pos_out[3 * c + 1] = pos_out[3 * c + 2] = NAN;
        state_out[c] = (int8_t)(cs[c] & kStateMask);
        if ((cs[c] & kStateMask) == kStateCollected) {
          pos_out[3 * c] = fx[c];
          pos_out[3 * c + 1] = fy[c];
        }
      }
      // active carriers are the compacted prefixes of the two species ranges
      const int hole_len = s->slots[0].running ? nh : nh;
      for (int q = 0; q < hole_len + ne; ++q) {
        const int64_t idx = q < hole_len ? q : s->slots[0].rec.cap_h + (q - hole_len);
        const int id = cid[idx];
        if (id < 0 || id >= n) continue;
        if ((cs[id] & kStateMask) != kStateActive) continue;
        pos_out[3 * id] = px[idx];
        pos_out[3 * id + 1] = py[idx];
        pos_out[3 * id + 2] = pz[idx];
      }
    } while (0);
    *steps_done = s->slots[0].n_steps;
  }
  s->ph = saved;
  s->K = savedK;
  s->opt.disable_graphs = saved_graphs;
  s->alloc.release(base);
  s->slots[0] = HostSlot{};
  return rc;
}

int sim_debug_step(sim_t* s, uint64_t seed, uint64_t event_id, int32_t n, const double* xyz,
                   const int8_t* sign, double* xyz_out, int8_t* state_out) {
  if (!s || n < 1 || !xyz || !xyz_out || !state_out) return SIM_EINVAL;
  sim_event_t ev{};
  ev.kind = CTS_EXPLICIT;
  ev.seed = seed;
  ev.event_id = event_id;
  ev.n_pairs = n;
  ev.explicit_xyz = xyz;
  ev.explicit_sign = sign;
  int64_t done = 0;
  const int rc = sim_debug_trajectory(s, &ev, 1, xyz_out, state_out, n, &done);
  if (rc) return rc;
  return done == 1 ? SIM_OK : SIM_ESTATE;
}


}  // extern "C"
