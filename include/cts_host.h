/*
 * cts_host.h -- host-side planning entry points of the charge-transport
 * library (no GPU needed).  They expose the scheduler's pure host logic so it
 * can be checked on machines without a device; the GPU path calls the same
 * code.  Paper reference: the pair sum of Eq. 4 (Sec. 2.1) must cover every
 * ordered pair (i, j) of carriers of one event exactly once per step; these
 * functions decide how that O(N^2) work is cut into units for the GPU.
 */
#ifndef CTS_HOST_H_
#define CTS_HOST_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One unit of pair work: i's [i0, i0 + ni) of species spec (0 holes, 1
 * electrons) of slot `slot`, against sources [j0, j1) of the slot's
 * concatenated [holes | electrons] list.  Units of one i-block share iblock
 * and are split into nsplit j ranges (split = 0 .. nsplit - 1); piece split
 * of a tile writes its partial sums to the FP64 entries [pbase + 3 * tile_i *
 * split, + 3 * tile_i) (nsplit > 1), and the pieces are added in split order. */
typedef struct cts_unit_t {
  int32_t slot, spec, i0, ni, j0, j1, split, nsplit, iblock, pbase;
} cts_unit_t;

/* Plan the units of one step for n_slots resident events with n_h[s] holes
 * and n_e[s] electrons (slots with n_h <= 0 are finished and get no work).
 * tile_i = i's per tile (threads x i's per thread of the pair kernel); grid =
 * persistent CTAs.  allow_split = 1: the total pair work is cut into `grid`
 * equal contiguous shares (tiles cut at j multiples of 4, segments of a tile
 * share iblock/pbase for their partial sums), grouped by CTA: CTA g runs
 * units [cta_begin[g], cta_begin[g+1]).  allow_split = 2: guided pieces for a
 * dynamic queue (largest first; piece sizes halve from w/2 to w/64 of a CTA's
 * share w over the last half of the work) that CTAs pull from;
 * cta_begin[grid] = number of units, the rest 0.  allow_split = 3: the same
 * pieces ordered slot by slot, the halving applied within each slot's work
 * (the queue a multi-step launch replays once per step).
 * allow_split = 0: whole tiles dealt out longest first.  Units are written to
 * out (capacity max_units); cta_begin has grid + 1 entries.  *n_out = units,
 * *partial_floats = FP64 partial-sum entries needed (limit partial_cap).
 * Returns 0, -1 for bad arguments, -2 if max_units is too small. */
int cts_plan_units(const int32_t* n_h, const int32_t* n_e, int32_t n_slots, int32_t tile_i,
                   int32_t grid, int32_t allow_split, int32_t max_units, int64_t partial_cap,
                   cts_unit_t* out, int32_t* n_out, int32_t* cta_begin,
                   int64_t* partial_floats);

/* The symmetric pair kernel's plan of one step (Eq. 4, Sec. 2.1, evaluated
 * once per unordered pair and added to both carriers: Newton's third law).
 * Each species range of a slot (n_h[s] holes, n_e[s] electrons; slots with
 * n_h <= 0 get no work) is cut into tiles of 64 carriers (the last one
 * shorter); an I block is 4 consecutive tiles of one species.  The pairs are
 * covered exactly once by the (block b, tile g) combinations with g at or
 * after b's first tile (same species; within b's own tiles, tile u pairs with
 * the tiles v > u of the block and with itself) and with every electron tile
 * g of a hole block b.  A pair unit (kind 0) is a rectangle of them, blocks
 * [ib0, ib1) of species spec_i x tiles [jt0, jt1) of species spec_j, of one
 * slot, run by one warp (the kernel skips the combinations below the
 * diagonal).  It writes one partial field (3 x 64 floats) for every existing
 * tile of its blocks, at index p_i + (b - ib0) * 4 + u, and for every tile of
 * its J range, at p_j + (g - jt0).  Pair units are listed slot by slot,
 * longest first within a slot; duty marks the first of each slot.  An update
 * unit (kind 1) covers the slot's tiles [jt0, jt1) (slot-local, holes then
 * electrons; at most 64 update units a slot); it waits until each tile's
 * lcnt partials are written, then sums them and moves the tile's carriers;
 * npair counts the slot's pair units.  A slot's update units follow the pair
 * units of the next 32 slots (or the end of the list).  Tiles are listed slot by slot, holes then
 * electrons; a tile's field is the sum of the partials lists[lptr .. lptr +
 * lcnt), in unit order.  units has room for max_units entries, tiles for
 * tiles_cap, lists for lists_cap; *n_partials receives the number of partial
 * fields.  Returns 0, -1 for bad arguments, -2 if a capacity is too small. */
typedef struct cts_sym_unit_t {
  int32_t slot, spec_i, spec_j, ib0, ib1, jt0, jt1, p_i, p_j, duty, kind, npair;
} cts_sym_unit_t;
typedef struct cts_sym_tile_t {
  int32_t slot, spec, tile, n, lptr, lcnt;
} cts_sym_tile_t;
int cts_plan_sym(const int32_t* n_h, const int32_t* n_e, int32_t n_slots, int32_t max_units,
                 cts_sym_unit_t* units, int32_t* n_units, cts_sym_tile_t* tiles,
                 int32_t tiles_cap, int32_t* n_tiles, int32_t* lists, int64_t lists_cap,
                 int64_t* n_partials);

/* First-fit carrier arena of the scheduler, for tests: replays n_ops
 * operations (size > 0: allocate size entries and write the offset, or -1 if
 * it does not fit, to result[k]; size < 0: free the block allocated by
 * operation -size-1) on an arena of `capacity` entries. Returns 0 or -1. */
int cts_arena_replay(int64_t capacity, const int64_t* ops, int32_t n_ops, int64_t* result);

/* Estimated transit steps of a hole from depth_um below the entrance surface
 * to the readout, by the drift-only integral dt = dz / (mu(E) E) over the
 * Eq. 6 field (the integral of Eq. 9); used to order work longest first. */
double cts_estimate_steps(double thickness_um, double bias_V, double depletion_V,
                          double mu0_cm2, double vsat_cms, double beta, double dt_ps,
                          double depth_um);

/* Autotune cache (sim_options_t.autotune_cache): a text file holding a
 * variant table (sim_set_variants) with the name of the device and the
 * number of kernel variants it was measured against.  save returns 0, -1 for
 * bad arguments, -3 if the file cannot be written.  load fills up to cap
 * entries and *n; returns 0, -1 for bad arguments, -2 for a malformed file,
 * -3 if it cannot be opened, -4 if it was measured on another device or
 * library build (then *n = 0). */
int cts_variant_table_save(const char* path, const char* device, int32_t n_variants,
                           const int64_t* min_pairs, const int32_t* variants, int32_t n);
int cts_variant_table_load(const char* path, const char* device, int32_t n_variants,
                           int64_t* min_pairs, int32_t* variants, int32_t cap, int32_t* n);

/* Carrier-pair count of one photon with Fano statistics (Sec. 4.2 applies a
 * Fano factor of 0.13 to the number of carriers): mean E / 3.62 eV, variance
 * fano times the mean, drawn as round(mean + sqrt(fano * mean) * g) with g the
 * first Box-Muller normal of the event's counter-based stream (Philox4x32-10,
 * key = seed, counter = (0, 0, event low word, event high word ^ 2 << 28)),
 * at least 1.  fano = 0 gives round(E / 3.62 eV).  The result goes into
 * sim_event_t.n_pairs.  Returns 0, or -1 for a null pointer, energy <= 0 or
 * fano < 0. */
int cts_fano_pairs(uint64_t seed, uint64_t event_id, double energy_keV, double fano,
                   int32_t* n_pairs);

/* Generalised Gaussian model of the collected cloud (Sec. 3).  Eq. 8, read
 * as the two-sided density beta / (2 alpha Gamma(1/beta)) exp(-(|x|/alpha)^beta)
 * of positions x relative to the photon's entry point.
 *
 * cts_fit_ggd: maximum-likelihood (alpha, beta) of n samples (for a given
 * beta the optimum has alpha^beta = beta / n sum |x|^beta; beta is found by
 * golden section on the profile likelihood over [0.3, 20]).  Returns 0, or -1
 * for n < 2, all-zero or non-finite samples. */
int cts_fit_ggd(const double* x, int64_t n, double* alpha, double* beta);

/* Eq. 10, alpha(t) = p0 + p1 sqrt(t) + p2 t + p3 t^2 of the drift time t
 * (ns): weighted linear least squares of n >= 4 points (w = NULL: equal
 * weights; else residuals are multiplied by w).  Writes p_alpha[4]; returns
 * 0, or -1 for bad input or a singular system. */
int cts_fit_alpha_t(const double* t, const double* alpha, const double* w, int32_t n,
                    double* p_alpha);

/* Eq. 11, read as beta(t) = 2 + p0 max(t - p1, 0)^p2 + p3 exp(p4 t) (the
 * printed power of t - p1 is undefined below p1): Levenberg-Marquardt least
 * squares of n >= 5 points from the starting point in p_beta[5], which
 * receives the fit; sigma (NULL = 1) divides the residuals.  Returns 0, or
 * -1 for bad input or a non-finite cost at the start. */
int cts_fit_beta_t(const double* t, const double* beta, const double* sigma, int32_t n,
                   double* p_beta);

/* alpha(t) and beta(t) of Eqs. 10 and 11 at drift time t >= 0.  Returns 0,
 * -1 for bad input, -2 if either comes out non-positive. */
int cts_ggd_params_at(const double* p_alpha, const double* p_beta, double t, double* alpha,
                      double* beta);

#ifdef __cplusplus
}
#endif
#endif /* CTS_HOST_H_ */
