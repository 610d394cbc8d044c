/*
 * cts.h -- C ABI of the GB300 (sm_103a) charge-transport library.
 *
 * The library simulates the brute-force drift-diffusion-repulsion Monte Carlo
 * of Xie et al., arXiv 2506.09712 (Sec. 2.1 and Algorithm 1): the cloud of
 * electron-hole pairs that one X-ray photon (or one electron track) leaves in
 * a planar silicon sensor is stepped in time; each step computes the O(N^2)
 * Coulomb field on every carrier (Eq. 4), adds the sensor's drift field
 * (Eq. 6), moves each carrier by mu(|E|) E dt plus a Gaussian diffusion step
 * of variance 2 D dt per axis with D = mu kT/e (Eqs. 1, 3, 5), collects holes
 * at the readout surface and finally bins the collected holes into pixels
 * (the readout of Sec. 4.2).
 *
 * Units: lengths um, times ps (dt) / ns (results), potentials V, mobility
 * cm^2/(V s), saturation velocity cm/s, temperature K.  Frame: z is measured
 * from the collecting (pixel) surface, z = 0 the readout electrode and
 * z = thickness the entrance surface; the drift field is -E(z) e_z with
 * E(z) = (V_bias - V_depletion)/H + 2 V_depletion (H - z)/H^2 (Eq. 6 with
 * z = H - z_paper).  The pixel grid is grid_n x grid_n pixels of pitch_um,
 * centred on x = y = 0: pixel index floor(x / pitch + grid_n / 2).
 *
 * Conventions of every entry point:
 *   - return 0 (SIM_OK) or a negative SIM_E* code; no exceptions or aborts
 *     cross the ABI; sim_strerror() names a code;
 *   - pointers are host pointers unless the name says dev_; the library copies
 *     what it needs before returning and never keeps a caller pointer;
 *   - the handle owns all device memory it allocates (cudaMalloc at sim_init,
 *     sized by sim_options_t) and frees it in sim_destroy;
 *   - one thread may call sim_submit while another calls sim_poll; any other
 *     concurrent use of one handle is not allowed.
 */
#ifndef CTS_H_
#define CTS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define SIM_OK 0
#define SIM_EINVAL (-1)        /* invalid argument or parameter */
#define SIM_ENOMEM_BUDGET (-2) /* event larger than the handle's device budget */
#define SIM_EAGAIN (-3)        /* admission queue full: retry later */
#define SIM_ETIMEOUT (-4)      /* sim_poll: nothing completed in time; or a
                                  bounded device wait gave up */
#define SIM_ECUDA (-5)         /* a CUDA call failed (the handle is unusable) */
#define SIM_EMAXSTEPS (-6)     /* per event: step cap reached, holes remain */
#define SIM_ENUMERIC (-7)      /* per event: non-finite field or position */
#define SIM_ESTATE (-8)        /* call not valid in this mode or state */
#define SIM_ENODEV (-9)        /* no CUDA device, or not an sm_103 device */

/* ---- enumerations ------------------------------------------------------- */
#define CTS_HOLES 1      /* only holes are tracked (the readout collects holes) */
#define CTS_BOTH 3       /* electrons and holes (Sec. 2.1: both species) */
#define CTS_MOB_CT 0     /* mu0 / (1 + (mu0 E / vsat)^beta)^(1/beta) */
#define CTS_MOB_CONST 1  /* mu = mu0 (closed-form tests) */
#define CTS_PHOTON 0     /* Gaussian cloud around the absorption point */
#define CTS_TRACK 1      /* pairs uniform along a straight segment */
#define CTS_EXPLICIT 2   /* initial positions given by the caller */
#define CTS_MODE_PLAIN 0   /* one event at a time, two launches per step */
#define CTS_MODE_BATCHED 1 /* resident events packed per launch, graph chunks */
#define CTS_MODE_SERVE 2   /* BATCHED driven by a background engine thread */

/* Sensor and stepping (Sec. 2; Algorithm 1 inputs H, T, V_bias, V_depletion).
 * species: CTS_HOLES or CTS_BOTH.  softening_um: Plummer length eps in the
 * pair field (r^2 + eps^2)^(-3/2); 0 selects the default 1e-6 um. */
typedef struct sim_sensor_t {
  double thickness_um;
  double bias_V;
  double depletion_V;
  double temperature_K;
  double eps_r;
  double pitch_um;
  double dt_ps;
  double softening_um;
  int64_t max_steps;
  int32_t grid_n;
  int32_t species;
  /* Optional non-uniform drift field replacing Eq. 6: drift_table_n (2 ..
   * 4096) samples of the field magnitude (V/um, > 0, pointing toward the
   * collecting surface like Eq. 6) at z = k H / (n - 1) from the collecting
   * surface, linearly interpolated; copied at sim_init.  n = 0 (and NULL)
   * keeps Eq. 6.  The drift-time estimate used to order work stays Eq. 6. */
  const double* drift_table_Vum;
  int32_t drift_table_n;
} sim_sensor_t;

/* Switches of the three transport terms (1 = on); all on reproduces Eqs. 3, 5.
 * spherical = 1 replaces the pairwise repulsion field (Eq. 4) by the
 * simplified spherical model of Sec. 2.2 (Eq. 7): field k_C Q(<r) (r - c) / r^3
 * about the mean position c of the event's active holes, Q(<r) the number of
 * holes strictly closer to c.  It needs species CTS_HOLES and events of at
 * most 16384 carriers (SIM_EINVAL otherwise); the result's interactions then
 * count one field evaluation per active hole and step.  The debug field and
 * timing hooks always use the pairwise field. */
typedef struct sim_field_t {
  int32_t repulsion;
  int32_t drift;
  int32_t diffusion;
  int32_t spherical;
} sim_field_t;

/* Field-dependent mobility (Sec. 2.1, Jacoboni-Canali form), per species. */
typedef struct sim_mobility_t {
  int32_t model;      /* CTS_MOB_CT or CTS_MOB_CONST */
  int32_t reserved;
  double mu0_h, vsat_h, beta_h; /* holes: cm^2/Vs, cm/s, exponent */
  double mu0_e, vsat_e, beta_e; /* electrons (CTS_BOTH only) */
} sim_mobility_t;

/* Execution options.  Zero fields select defaults. */
/* options.keep_induced flags (may be combined). */
#define SIM_INDUCED_TOTAL 1  /* the whole collecting surface (sim_result_t.induced_e) */
#define SIM_INDUCED_PIXELS 2 /* the 3 x 3 pixels around the grid's centre pixel
                                (sim_result_t.induced_px); needs grid_n >= 3 */

typedef struct sim_options_t {
  int32_t mode;            /* CTS_MODE_* */
  int32_t device;          /* CUDA device ordinal */
  int32_t max_slots;       /* events resident at once (default 256) */
  int32_t chunk_steps;     /* steps per chunk between host checks (default 32) */
  int64_t max_carriers;    /* carrier arena capacity (default: from budget) */
  int64_t hbm_budget_bytes;/* device bytes the handle may allocate (default 1 GiB) */
  int32_t queue_capacity;  /* bound of the admission queue (default 65536) */
  int32_t variant;         /* pair-kernel variant + 1; 0 = default choice: per
                              chunk, the symmetric kernel when the running
                              events hold at least 4.0e8 carrier pairs (sum
                              of N^2) -- variant 1 (12 warps per SM), or 13
                              (8 warps) once an event has more than 640
                              tiles of 64 carriers -- the per-pair kernel
                              (variant 2) below that; SERVE: variant 13 from
                              2.8e8 pairs, else variant 2; PLAIN: variant 1 */
  int32_t disable_graphs;  /* 1 = launch K-step chunks directly, not as CUDA graphs */
  int32_t keep_final_xy;   /* 1 = keep collected (x, y) and retire steps for poll */
  int32_t time_launches;   /* 1 = time every step-kernel launch with CUDA events */
  int32_t keep_induced;    /* SIM_INDUCED_* flags: record the induced charge per
                              step (sim_result_t); 0 = off */
  int32_t step_launches;   /* 1 = one step-kernel launch per step; 0 = one launch
                              per chunk with dynamic-queue variants: a slot's
                              next step starts as soon as all of its tiles are
                              updated, without a device-wide barrier */
  void* stream;            /* cudaStream_t to launch on; NULL = own stream */
  const char* autotune_cache; /* file of a variant table (cts_host.h): loaded by
                              sim_init when it matches this device and build,
                              written by sim_autotune; NULL = none */
  int32_t sph_cluster;     /* spherical model: CTAs per event (1, 2 or 4); 0 =
                              the widest with which all max_slots events are
                              resident at once.  Results do not depend on it. */
  int32_t reserved;
} sim_options_t;

/* One event (Algorithm 1 inputs: E, absorption depth h, plus the entry point).
 * n_pairs = 0 takes round(E / 3.62 eV) (Sec. 2); sigma_um < 0 takes Eq. 2,
 * sigma = 0.0044 E^1.75 um.  With CTS_BOTH each pair is one hole and one
 * electron at the same start point.  CTS_TRACK: segment of track_len_um from
 * the entry point on the back surface, polar angle theta from the inward
 * normal, azimuth phi, Gaussian sigma perpendicular to it.  CTS_EXPLICIT:
 * explicit_xyz holds n_pairs positions (x0 y0 z0 x1 ...), explicit_sign +1
 * (hole) / -1 (electron) or NULL for all holes; both are copied at submit. */
typedef struct sim_event_t {
  uint64_t event_id;
  uint64_t seed;
  int32_t kind;
  int32_t n_pairs;
  double energy_keV;
  double depth_um;
  double x_um, y_um;
  double sigma_um;
  double track_len_um, theta_deg, phi_deg;
  const double* explicit_xyz;
  const int8_t* explicit_sign;
} sim_event_t;

/* One completed event.  The caller owns the arrays and sets their pointers
 * (and capacity) before sim_poll / sim_collect; NULL arrays are skipped.
 * final_xy: (x, y) at collection per carrier id (NaN if not collected);
 * retire_step: step of collection/exit per carrier id, -1 = before the first
 * step, -2 = never.  Times are host steady-clock ns. */
typedef struct sim_result_t {
  uint64_t event_id;
  int32_t status;        /* SIM_OK, SIM_EMAXSTEPS, SIM_ENUMERIC */
  int32_t n_carriers;    /* carriers of the event (both species) */
  int64_t n_steps;       /* steps executed until every hole was collected */
  int64_t n_collected;   /* holes collected by the readout */
  int64_t n_outside;     /* collected holes outside the pixel grid */
  int64_t n_lost;        /* electrons still moving when the event stopped */
  int64_t interactions;  /* sum over steps of N_act (N_act - 1) */
  double t_submit_ns, t_start_ns, t_done_ns;
  int32_t* pixels;       /* grid_n * grid_n counts, row-major [iy][ix] */
  double* final_xy;      /* 2 * capacity */
  int32_t* retire_step;  /* capacity */
  int64_t capacity;      /* entries available in final_xy / retire_step */
  /* Transient signal (options.keep_induced & SIM_INDUCED_TOTAL): the charge
   * (units of e) induced on the whole collecting surface after each executed
   * step, by the Shockley-Ramo theorem with the planar weighting potential
   * 1 - z/H (a carrier of charge q moving from z_a to z_b adds
   * q (z_a - z_b) / H; carriers that leave stop at the surface).  The paper
   * names the weighting field as the extension towards transient signals
   * (Sec. 5.3).  Entries beyond n_steps are NaN; NULL skips. */
  double* induced_e;
  int64_t induced_capacity;  /* steps available in induced_e and induced_px */
  /* Per-pixel transient signals (options.keep_induced & SIM_INDUCED_PIXELS):
   * 9 * induced_capacity doubles, [step][b][a], the charge induced on grid
   * pixel (c - 1 + a, c - 1 + b), c = grid_n / 2, after each executed step:
   * q (phi(end) - phi(start)) summed over moves, phi the pixel's weighting
   * potential in the planar sensor (Laplace's equation, 1 on the pixel and 0
   * on the rest of the collecting surface and on the back surface, pixels
   * tiling the surface).  A collected carrier ends with phi = 1 on the pixel
   * that reads it out, an exited one with 0.  NaN beyond n_steps; NULL skips. */
  double* induced_px;
} sim_result_t;

typedef struct sim_stats_t {
  int64_t events_done;
  int64_t interactions;
  int64_t steps_launched;   /* step-kernel launches (one per step per chunk) */
  int64_t kernel_launches;  /* all kernel launches issued by the library */
  int64_t chunks;
  int64_t queue_depth;
  int64_t rejected;
  int32_t sm_count;
  int32_t variant;          /* pair-kernel variant in use */
  double device_ms;         /* device time of executed chunks (CUDA events) */
  double step_kernel_ms;    /* summed step-kernel launch times (time_launches) */
  int64_t step_kernel_launches; /* launches timed into step_kernel_ms */
  int64_t h2d_bytes;        /* bytes copied host -> device by the library */
  int64_t d2h_bytes;        /* bytes copied device -> host by the library */
  int32_t symmetric;        /* 1: the variant in use evaluates each unordered pair
                               once and adds it to both carriers (Newton's third
                               law); 0: every ordered pair */
  int32_t sph_cluster;      /* spherical model: CTAs per event; 0 otherwise */
} sim_stats_t;

typedef struct sim_t sim_t;

/* Create a handle: validates parameters (SIM_EINVAL), checks for an sm_103
 * device (SIM_ENODEV) and allocates the device arena (SIM_ECUDA on failure). */
int sim_init(const sim_sensor_t* sensor, const sim_field_t* field,
             const sim_mobility_t* mobility, const sim_options_t* options,
             sim_t** out);

/* Queue n_ev events (copied).  *n_accepted counts the accepted prefix; the
 * first event not accepted sets the return code: SIM_EINVAL (bad event),
 * SIM_ENOMEM_BUDGET (larger than the arena), SIM_EAGAIN (queue full). */
int sim_submit(sim_t* sim, const sim_event_t* ev, int n_ev, int* n_accepted);

/* Fill up to max_out completed results (arrays supplied by the caller).
 * Waits up to timeout_ms for the first one (0 = do not wait, < 0 = until
 * one completes).  In PLAIN and BATCHED modes the calling thread drives the
 * GPU; in SERVE mode the engine thread does.  SIM_ETIMEOUT if none. */
int sim_poll(sim_t* sim, sim_result_t* out, int max_out, int* n_out,
             int timeout_ms);

/* Convenience: submit n events, drive them to completion, return results in
 * submission order (out[k] receives event k). */
int sim_run(sim_t* sim, const sim_event_t* ev, int n, sim_result_t* out);

/* Device-resident batch (BATCHED mode): sim_stage admits the events and
 * uploads their descriptors; sim_execute runs all staged events to completion
 * with results kept in device memory (only per-chunk control words cross to
 * the host); sim_collect copies the results out, in staging order. */
int sim_stage(sim_t* sim, const sim_event_t* ev, int n);
int sim_execute(sim_t* sim);
int sim_collect(sim_t* sim, sim_result_t* out, int max_out, int* n_out);

/* Kernel variant per chunk (the autotuner's output): a chunk whose resident
 * pair work W = sum over events of (n_h + n_e)^2 is at least min_pairs[k]
 * (largest such k; min_pairs ascending) runs variants[k] (1-based, as in
 * sim_options_t.variant).  n = 0 restores the fixed variant. */
int sim_set_variants(sim_t* sim, const int64_t* min_pairs, const int32_t* variants, int32_t n);

/* Read the variant table back: up to cap entries; *n_out = table length. */
int sim_get_variants(sim_t* sim, int64_t* min_pairs, int32_t* variants, int32_t cap,
                     int32_t* n_out);

/* Autotuner (BATCHED mode, idle handle): stages the first n, n/2, n/4, ..., 1
 * of the given representative events, times every kernel variant on each
 * (sim_debug_time_step, `reps` launches), and installs the table that runs
 * the fastest variant for each range of resident pair work (boundaries at
 * the geometric means of the measured work).  *n_buckets = table length.
 * The handle is idle again afterwards. */
int sim_autotune(sim_t* sim, const sim_event_t* ev, int32_t n, int32_t reps, int32_t* n_buckets);

/* Drop every queued, resident or completed-but-unpolled event (their results
 * are discarded); the handle is then idle. */
int sim_reset(sim_t* sim);

int sim_get_stats(sim_t* sim, sim_stats_t* out);
int sim_destroy(sim_t* sim);
const char* sim_strerror(int code);

/* ---- kernel-level entry points (used by the parity tests) ---------------- */

/* Eq. 4 field of n_h holes followed by n_e electrons at FP32 positions
 * x, y, z (um), through the same pair kernel and tile schedule as the step
 * loop.  out_E receives 3*(n_h+n_e) doubles (Ex, Ey, Ez per carrier, V/um)
 * holding the FP32 results. */
int sim_debug_field(sim_t* sim, const float* x, const float* y, const float* z,
                    int32_t n_h, int32_t n_e, double* out_E);

/* Readout binning kernel on n collected positions; pixels gets grid_n^2
 * counts (overwritten), *outside the number outside the grid. */
int sim_debug_bin(sim_t* sim, const double* x, const double* y, int64_t n,
                  int32_t* pixels, int64_t* outside);

/* Philox4x32-10 on the device: ctr[4n], key[2n] -> out[4n]; and the same
 * blocks from the CUDA toolkit's curand Philox for ctr words (c0, c1, 0, 0)
 * when curand_out is not NULL (both on device 0 of the handle-less call). */
int sim_debug_philox(const uint32_t* ctr, const uint32_t* key, int64_t n,
                     uint32_t* out, uint32_t* curand_out);

/* The device's diffusion normals for (seed, event, purpose, carrier, step)
 * tuples: in[5n] as u64 (seed, event, purpose, carrier, step) -> out[3n]. */
int sim_debug_normals(const uint64_t* in, int64_t n, double* out);

/* Run one event for at most n_steps steps (or until every hole is
 * collected) and return FP64 positions (3 per carrier id) and states
 * (0 active, 1 collected, 2 exited) when it stopped; *steps_done receives the
 * steps executed.  Uses the BATCHED path with a single slot. */
int sim_debug_trajectory(sim_t* sim, const sim_event_t* ev, int64_t n_steps,
                         double* pos_out, int8_t* state_out, int64_t capacity,
                         int64_t* steps_done);

/* One time step of Algorithm 1 (Sec. 2.1; the field of Eq. 4, the moves of
 * Eqs. 3, 5, 6, then collection and exit) through the library's step kernel,
 * from given FP64 positions: n carriers, xyz[3n] (um, x y z per carrier) and
 * sign[n] (+1 hole, -1 electron; NULL = all holes), all active, taken as
 * carriers 0 .. n-1 of an event (seed, event_id) at its step 0, so carrier c
 * draws its diffusion normals from counter (c, 0).  Writes the positions
 * after the step to xyz_out[3n] (a collected hole: its collection point x, y
 * and NaN z; an electron that left: NaN) and the states (0 active, 1
 * collected, 2 exited) to state_out[n].  The handle must be BATCHED with no
 * event resident or queued (SIM_ESTATE).  For one-step parity tests: both
 * sides start from the same state, so trajectory divergence cannot hide the
 * difference of a single step. */
int sim_debug_step(sim_t* sim, uint64_t seed, uint64_t event_id, int32_t n, const double* xyz,
                   const int8_t* sign, double* xyz_out, int8_t* state_out);

/* One step of the pair kernel (field only: the staged events do not move)
 * on the events admitted by sim_stage, with a trace.  Kernels that evaluate
 * every ordered pair: out[8g..8g+7] = (SM id, start ns, end ns, pairs,
 * units, ns in unit prologues, ns in pair loops, ns in epilogues) of CTA g,
 * for up to max_ctas CTAs; *n_ctas receives the grid size.  The symmetric
 * kernel (sim_stats_t.symmetric): one record per unit, out[8r..8r+7] = (SM
 * id, ns when the warp took it, ns when it was done, queue position, kind: 0
 * pair unit / 1 update unit, ns waiting for its inputs, ns working, warp),
 * up to max_ctas records; *n_ctas receives the records written.  For
 * load-balance and latency studies. */
int sim_debug_trace_step(sim_t* sim, uint64_t* out, int32_t max_ctas, int32_t* n_ctas);

/* Allocation-free pair field, for callers that cannot allocate device
 * memory (they work inside another framework's memory pool or under a fixed
 * device budget, or must avoid the device-wide synchronisation of cudaMalloc
 * and cudaFree).  The paper has no counterpart.  Inputs dev_x, dev_y,
 * dev_z: n_h holes followed by n_e electrons, FP32 positions in um,
 * caller-owned device memory.  Output dev_E: 3 * (n_h + n_e) floats, Ex
 * of every carrier, then Ey, then Ez (V/um), caller-owned device memory.
 * eps_r: relative permittivity; softening_um: Plummer length (finite;
 * 0 selects 1e-6 um).  Work is queued on
 * `stream` (a cudaStream_t, NULL = legacy default) and the call returns
 * without waiting for it.
 * It allocates nothing: its working storage is one fixed array compiled into
 * the library (about 3 MB of device memory on every GPU that loads the
 * library, held until the process exits), so at most 131072 carriers are
 * accepted; larger inputs return SIM_ENOMEM_BUDGET before anything runs.
 * The first call on a device looks up that array's device address (set-up,
 * once per device, with the device current); make that first call before any
 * stream capture.  Every call uses the same array and leaves it for the next
 * call: calls that overlap on the GPU (other streams, other host threads)
 * race and must be serialised by the caller.  Returns SIM_OK, SIM_EINVAL,
 * SIM_ENOMEM_BUDGET, SIM_ENODEV (no sm_103 device current) or SIM_ECUDA. */
int cts_field_noalloc(const float* dev_x, const float* dev_y, const float* dev_z,
                      int32_t n_h, int32_t n_e, double eps_r, double softening_um,
                      float* dev_E, void* stream);

/* Time `reps` launches of the pair kernel (field only: positions do not move)
 * on the events admitted by sim_stage, with kernel variant `variant`
 * (1-based; 0 = the current one); *ms_per_launch receives the mean launch
 * time from CUDA events.  The autotuner's measurement. */
int sim_debug_time_step(sim_t* sim, int32_t variant, int32_t reps, double* ms_per_launch);

/* Detector readout of simulated events (Sec. 4.1 describes the selection of
 * the measured clusters; Sec. 4.2 applies it, with Fano statistics and about
 * 0.13 keV of noise, to simulated events).  Parameters: */
typedef struct sim_readout_params_t {
  int32_t grid_n;        /* pixels per side of each count map (1 .. 32) */
  int32_t n_bins;        /* bins of the single-pixel spectrum (0 = none) */
  double ev_per_pair;    /* eV per carrier pair (3.62) */
  double noise_keV;      /* Gaussian noise per pixel, standard deviation (0.13); 0 = none */
  double beam_keV;       /* photon energy: centre of the cluster-energy window */
  double window_keV;     /* half width of the window (1.0) */
  double veto_factor;    /* pile-up threshold in units of noise_keV (3.0) */
  double spec_lo_keV;    /* lower edge of the spectrum's first bin */
  double spec_bin_keV;   /* spectrum bin width (0.1) */
} sim_readout_params_t;

/* One event's cluster.  Pixel energy = count * ev_per_pair + noise * g, g the
 * first Box-Muller normal of the event's stream at (carrier = pixel index
 * iy * grid_n + ix, step 0, purpose 3).  The centre (cx, cy) is the pixel of
 * largest energy (first in row-major order on ties); e[9] holds the 3 x 3
 * pixels around it, row-major, NaN off the grid; e_cluster is their sum.
 * vetoed = some pixel of the 7 x 7 window outside the 3 x 3, on the grid,
 * exceeds veto_factor * noise_keV (pile-up cut); accepted = not vetoed and
 * |e_cluster - beam_keV| <= window_keV.  Off-grid pixels are not read out. */
typedef struct sim_cluster_t {
  int32_t accepted, vetoed, cx, cy;
  double e_cluster;
  double e[9];
} sim_cluster_t;

/* Readout of n_events pixel-count maps (host memory, n_events x grid_n x
 * grid_n int32, row-major per event, e.g. sim_result_t.pixels) with per-event
 * seeds and ids on GPU `device`: writes clusters[n_events], optionally the
 * noisy pixel energies pixel_keV[n_events x grid_n^2] (NULL to skip), and
 * adds to spectrum[n_bins] (NULL if n_bins = 0) one count per on-grid pixel
 * of every accepted cluster, in bin floor((e - spec_lo_keV) / spec_bin_keV).
 * All buffers are the caller's host memory; the call allocates device memory
 * for the copies and synchronises.  Returns SIM_OK, SIM_EINVAL, SIM_ENODEV
 * or SIM_ECUDA. */
int sim_readout(const sim_readout_params_t* prm, const int32_t* counts, const uint64_t* seeds,
                const uint64_t* event_ids, int32_t n_events, int32_t device, double* pixel_keV,
                sim_cluster_t* clusters, int64_t* spectrum);

/* Fast event generation (Sec. 4.2) from the generalised Gaussian model of
 * Sec. 3 (Eq. 8): one event's n_pairs carriers land at (x_um, y_um) plus
 * independent x and y offsets drawn from GGD(alpha, beta) (alpha, beta from
 * cts_ggd_params_at at the event's drift time; n_pairs e.g. from
 * cts_fano_pairs), binned like simulated events into grid_n x grid_n pixels
 * of pitch pitch_um centred on the origin.  Offsets are alpha G^(1/beta)
 * with a random sign, G ~ Gamma(1/beta) by Marsaglia-Tsang rejection for
 * Gamma(1/beta + 1) and a U^beta boost, drawn in FP32 from the event's
 * counter-based stream (purpose 4). */
typedef struct sim_gen_event_t {
  uint64_t seed, event_id;
  int32_t n_pairs;
  int32_t reserved;
  double x_um, y_um;
  double alpha, beta;
} sim_gen_event_t;

/* Generate n_events events (host array) on GPU `device`: pixel counts into
 * pixels[n_events x grid_n^2] (row-major per event) and carriers that land
 * off the grid into outside[n_events] (NULL to skip), both host memory.
 * grid_n 1 .. 32, alpha > 0, beta in [0.3, 20], n_pairs >= 0.  Allocates
 * device memory for the copies and synchronises.  Returns SIM_OK,
 * SIM_EINVAL, SIM_ENODEV or SIM_ECUDA. */
int sim_generate(const sim_gen_event_t* events, int32_t n_events, double pitch_um, int32_t grid_n,
                 int32_t device, int32_t* pixels, int64_t* outside);

/* FP32 FMA throughput of device `device` (CUDA ordinal) measured by chains of
 * independent fused multiply-adds, packed f32x2 (packed = 1) or scalar: the
 * attainable counterpart of the nominal FP32 peak that the pair kernel's
 * 16 flops per interaction are compared with (Sec. 2.1, Eq. 4 is FP32 FMA
 * work).  *flops_per_s receives the best of three timed launches (2 flops per
 * FMA lane).  Allocates a small output buffer.  Returns SIM_OK, SIM_EINVAL,
 * SIM_ENODEV or SIM_ECUDA. */
int sim_debug_fma_peak(int32_t device, int32_t packed, double* flops_per_s);

/* Compile-time options of this library build (no device needed):
 * SIM_BUILD_BOUNDS_CHECK when it was compiled with -DCTS_BOUNDS_CHECK.  That
 * build's kernels check the arena index ranges of every slot, unit and
 * carrier they touch; an index outside its range is recorded and the access
 * skipped (never made), and the calls that ran the kernel then fail with
 * SIM_ECUDA ("an index left its slot's range").  A debugging aid in place of
 * a sanitizer; the default build compiles none of these checks. */
#define SIM_BUILD_BOUNDS_CHECK 1
int sim_build_flags(void);

/* Per-launch log of the step kernel, kept while the handle was created with
 * options.time_launches != 0 (at most 1 << 20 entries, oldest dropped).
 * Copies up to `cap` entries, oldest first, as quadruples (kernel ms from
 * CUDA events around the launch, ordered carrier pairs the launch covers
 * including carriers retired since the last compaction, events running in
 * the chunk, 1 if the symmetric kernel ran and 0 otherwise) into
 * out[4 * cap], writes the count to *n_out and clears the log.  Returns
 * SIM_OK or SIM_EINVAL. */
int sim_debug_launch_log(sim_t* sim, double* out, int32_t cap, int32_t* n_out);

/* Host-side fault injection for the failure-path tests: the next chunk (or
 * poll) reports the given code as if the device or queue had raised it
 * (SIM_ENUMERIC, SIM_ETIMEOUT, SIM_ECUDA); 0 clears. */
int sim_debug_inject(sim_t* sim, int fault);

#ifdef __cplusplus
}
#endif
#endif /* CTS_H_ */
