/*
 * cts_oracle.c -- plain FP64 CPU oracle of the brute-force drift-diffusion-
 * repulsion charge-transport Monte Carlo (Xie et al., "Optimization and
 * validation of charge transport simulation for hybrid pixel detectors
 * incorporating the repulsion effect", arXiv 2506.09712).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * execute this file; only the test suite, the smoke check and the benchmark's
 * CPU-baseline leg use it.  It shares no source with the CUDA path.
 *
 * Everything here is written for clarity, not speed: double loops, FP64,
 * one OpenMP pragma over carriers (or over events).  Each function names the
 * passage of the paper (or the published definition) it follows.
 *
 * Frame and units (readings of the paper, all listed in the design notes):
 *   lengths in um, times in ns, potentials in V, fields in V/um,
 *   mobilities in um^2/(V ns), velocities in um/ns.
 *   z is measured from the collecting (pixel) surface: z = 0 is the readout
 *   electrode, z = H the entrance (back) surface.  The paper's Eq. 6 puts the
 *   entrance at z_paper = 0, so z = H - z_paper and the drift-field vector is
 *   -E(z) e_z with E(z) = (Vb - Vd)/H + 2 Vd (H - z)/H^2.
 *
 * Parity status: pinned (closed forms, invariants, a library Philox, exact
 * small configurations, hand-built readout maps, the statistics of the Fano
 * and noise draws, and for the pixel weighting potential the Fourier-integral
 * solution, quadrature of the Poisson kernel and the sum over all pixels) --
 * see tests/test_oracle_*.py.  The paper's own
 * printed physics numbers (Table 1, GGD betas) depend on unprinted mobility
 * parameters and are checked only qualitatively.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Physical constants: SI 2019 exact values (e, k_B) and CODATA 2018 eps0.   */
/* ------------------------------------------------------------------------ */
static const double OR_E_CHARGE = 1.602176634e-19;  /* C   */
static const double OR_EPS0 = 8.8541878128e-12;     /* F/m */
static const double OR_KB = 1.380649e-23;           /* J/K */
static const double OR_PI = 3.14159265358979323846;
/* Section 2: 3.62 eV per electron-hole pair. */
static const double OR_EV_PER_PAIR = 3.62;

enum { OR_OK = 0, OR_EMAXSTEPS = -6, OR_EINVAL = -1 };
enum { OR_HOLES = 1, OR_BOTH = 3 };
enum { OR_MOB_CT = 0, OR_MOB_CONST = 1 };
enum { OR_PHOTON = 0, OR_TRACK = 1, OR_EXPLICIT = 2 };
enum { OR_ACTIVE = 0, OR_COLLECTED = 1, OR_RETIRED = 2 };
enum { OR_PURPOSE_DIFFUSION = 0, OR_PURPOSE_INIT = 1, OR_PURPOSE_FANO = 2,
       OR_PURPOSE_NOISE = 3, OR_PURPOSE_GGD = 4 };

typedef struct {
  double thickness_um;   /* H */
  double bias_V;         /* V_bias */
  double depletion_V;    /* V_depletion */
  double temperature_K;  /* T */
  double eps_r;          /* relative permittivity, 11.7 for Si (Sec. 2.1) */
  double pitch_um;       /* pixel pitch */
  int32_t grid_n;        /* pixels per side of the readout grid */
  double dt_ps;          /* time step */
  int64_t max_steps;     /* step cap */
  int32_t species;       /* OR_HOLES or OR_BOTH */
  double softening_um;   /* Plummer softening; 0 = exact Eq. 4 */
  int32_t repulsion, drift, diffusion; /* switches of the three terms */
  int32_t mob_model;     /* OR_MOB_CT or OR_MOB_CONST */
  double mu0_h, vsat_h, beta_h; /* holes: cm^2/Vs, cm/s, - */
  double mu0_e, vsat_e, beta_e; /* electrons */
  int32_t spherical;     /* 1: repulsion by the simplified spherical model (Eq. 7) */
  const double* drift_table; /* optional E(z) samples (V/um) at z = k H / (n - 1) */
  int32_t drift_table_n;     /* 0: Eq. 6 */
} or_params_t;

typedef struct {
  uint64_t seed, event_id;
  int32_t kind;
  double energy_keV;
  int32_t n_pairs;        /* 0: round(E / 3.62 eV) */
  double depth_um;        /* absorption depth below the entrance surface */
  double x_um, y_um;      /* entry point */
  double sigma_um;        /* < 0: Eq. 2 */
  double track_len_um, theta_deg, phi_deg; /* OR_TRACK */
  const double* explicit_xyz; /* OR_EXPLICIT: 3*n_pairs, x0 y0 z0 x1 ... */
  const int8_t* explicit_sign; /* +1 hole, -1 electron; NULL = all holes */
} or_event_t;

typedef struct {
  int32_t status;
  int64_t n_steps, n_collected, n_outside, n_lost, interactions;
  int32_t* pixels;      /* grid_n^2, may be NULL */
  double* final_x;      /* per carrier; holes that were collected */
  double* final_y;
  int32_t* retire_step; /* per carrier; -2 = never retired */
  double* pos_out;      /* 3 * n_carriers, positions when the run stopped */
  int8_t* state_out;    /* per carrier */
  int8_t* sign_out;     /* per carrier */
  double* induced;      /* optional: charge induced on the collecting surface
                           after each step, in units of e */
  int64_t induced_capacity;
  double* induced_px;   /* optional: 9 * induced_capacity, the charge induced on
                           the 3 x 3 pixels around the grid's centre pixel after
                           each step, [step][row-major 3 x 3] */
} or_result_t;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as   */
/* easy as 1, 2, 3", SC'11): four 32-bit counter words, two key words, ten   */
/* rounds of two 32x32->64 multiplies; the key is bumped by the Weyl        */
/* constants between rounds.                                                 */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                      uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
  const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint64_t p0 = (uint64_t)M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += W0; k1 += W1;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The stream layout of this project: key = seed, counter = (carrier, step,
 * event low word, event high word XOR purpose << 28). */
static void or_stream_words(uint64_t seed, uint64_t event_id, uint32_t purpose,
                            uint32_t carrier, uint32_t step, uint32_t out[4]) {
  uint32_t ctr[4] = {carrier, step, (uint32_t)event_id,
                     (uint32_t)(event_id >> 32) ^ (purpose << 28)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, out);
}

/* Uniform in (0,1) from the top 23 bits: ((w >> 9) + 1/2) / 2^23.  Every such
 * value is exactly representable in FP32 as well as FP64. */
double or_uniform(uint32_t w) {
  return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* Three standard normals by the Box-Muller transform (Box & Muller 1958):
 * (n0, n1) from the pair (u0, u1), n2 from the cosine branch of (u2, u3). */
void or_normals3(uint64_t seed, uint64_t event_id, uint32_t purpose,
                 uint32_t carrier, uint32_t step, double n[3]) {
  uint32_t w[4];
  or_stream_words(seed, event_id, purpose, carrier, step, w);
  double u0 = or_uniform(w[0]), u1 = or_uniform(w[1]);
  double u2 = or_uniform(w[2]), u3 = or_uniform(w[3]);
  double r01 = sqrt(-2.0 * log(u0));
  double r23 = sqrt(-2.0 * log(u2));
  n[0] = r01 * cos(2.0 * OR_PI * u1);
  n[1] = r01 * sin(2.0 * OR_PI * u1);
  n[2] = r23 * cos(2.0 * OR_PI * u3);
}

/* ------------------------------------------------------------------------ */
/* Material model                                                            */
/* ------------------------------------------------------------------------ */

/* k_C = e / (4 pi eps0 eps_r), in V um (Eq. 4 prefactor per unit charge). */
double or_coulomb_k(double eps_r) {
  return OR_E_CHARGE / (4.0 * OR_PI * OR_EPS0 * eps_r) * 1.0e6;
}

/* kT/e in V (Einstein relation, Eq. 1: D = mu kT/e). */
double or_thermal_voltage(double temperature_K) {
  return OR_KB * temperature_K / OR_E_CHARGE;
}

/* Carrier count, Section 2 and Algorithm 1: N = round(E / 3.62 eV). */
int32_t or_n_pairs(double energy_keV) {
  return (int32_t)lround(energy_keV * 1000.0 / OR_EV_PER_PAIR);
}

/* Initial cloud width, Eq. 2: sigma = 0.0044 * E^1.75 um (E in keV). */
double or_sigma_um(double energy_keV) {
  return 0.0044 * pow(energy_keV, 1.75);
}

/* Drift-field magnitude, Eq. 6, with z measured from the pixel side. */
double or_drift_field(const or_params_t* P, double z) {
  double H = P->thickness_um;
  if (P->drift_table_n >= 2) {
    /* a non-uniform profile given as samples, linearly interpolated, the
     * ends held beyond [0, H] */
    const int32_t n = P->drift_table_n;
    double u = z / H * (double)(n - 1);
    if (u < 0.0) u = 0.0;
    if (u > (double)(n - 1)) u = (double)(n - 1);
    int32_t k = (int32_t)floor(u);
    if (k > n - 2) k = n - 2;
    const double w = u - (double)k;
    return P->drift_table[k] + w * (P->drift_table[k + 1] - P->drift_table[k]);
  }
  return (P->bias_V - P->depletion_V) / H +
         2.0 * P->depletion_V * (H - z) / (H * H);
}

/* Field-dependent mobility (Sec. 2.1, Jacoboni-Canali form):
 * mu(E) = mu0 / (1 + (mu0 E / vsat)^beta)^(1/beta); returns um^2/(V ns). */
double or_mobility(const or_params_t* P, int sign, double E) {
  double mu0 = (sign > 0 ? P->mu0_h : P->mu0_e) * 0.1;   /* cm^2/Vs -> um^2/(V ns) */
  double vsat = (sign > 0 ? P->vsat_h : P->vsat_e) * 1e-5; /* cm/s -> um/ns */
  double beta = sign > 0 ? P->beta_h : P->beta_e;
  if (P->mob_model == OR_MOB_CONST) return mu0;
  return mu0 / pow(1.0 + pow(mu0 * E / vsat, beta), 1.0 / beta);
}

/* ------------------------------------------------------------------------ */
/* Repulsion field, Eq. 4, read as a field: E_i = sum_{j != i} q_j r_ij /    */
/* (4 pi eps0 eps_r |r_ij|^3), r_ij from carrier j to carrier i.  The       */
/* printed q_i q_j is a force; the velocity below carries the sign of q_i.  */
/* With softening eps > 0 the denominator is (r^2 + eps^2)^(3/2).  A pair   */
/* at zero distance (with eps = 0) contributes nothing.                     */
/* Rows in [row0, row1) are computed; only active carriers are sources.     */
/* ------------------------------------------------------------------------ */
void or_field_rows(int64_t n, const double* x, const double* y, const double* z,
                   const int8_t* sign, const int8_t* active,
                   const int64_t* rows, int64_t n_rows, double kc, double eps,
                   int parallel, double* ex, double* ey, double* ez) {
  double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 16) if (parallel)
  for (int64_t r = 0; r < n_rows; ++r) {
    int64_t i = rows[r];
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int64_t j = 0; j < n; ++j) {
      if (j == i) continue;
      if (active && active[j] != OR_ACTIVE) continue;
      double dx = x[i] - x[j], dy = y[i] - y[j], dz = z[i] - z[j];
      double r2 = dx * dx + dy * dy + dz * dz + eps2;
      if (r2 == 0.0) continue;
      double inv_r3 = 1.0 / (r2 * sqrt(r2));
      double q = sign ? (double)sign[j] : 1.0;
      sx += q * dx * inv_r3;
      sy += q * dy * inv_r3;
      sz += q * dz * inv_r3;
    }
    ex[r] = kc * sx;
    ey[r] = kc * sy;
    ez[r] = kc * sz;
  }
}

void or_field(int64_t n, const double* x, const double* y, const double* z,
              const int8_t* sign, const int8_t* active, double kc, double eps,
              int parallel, double* ex, double* ey, double* ez) {
  int64_t* rows = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int64_t i = 0; i < n; ++i) rows[i] = i;
  or_field_rows(n, x, y, z, sign, active, rows, n, kc, eps, parallel, ex, ey, ez);
  free(rows);
}

/* ------------------------------------------------------------------------ */
/* Readout: pixel index floor(x / pitch + n/2) on a grid centred on x = 0.   */
/* ------------------------------------------------------------------------ */
int or_pixel_of(const or_params_t* P, double x, double y, int32_t* ix, int32_t* iy) {
  double fx = floor(x / P->pitch_um + 0.5 * (double)P->grid_n);
  double fy = floor(y / P->pitch_um + 0.5 * (double)P->grid_n);
  if (fx < 0.0 || fy < 0.0 || fx >= (double)P->grid_n || fy >= (double)P->grid_n)
    return 0;
  *ix = (int32_t)fx;
  *iy = (int32_t)fy;
  return 1;
}

void or_bin(const or_params_t* P, int64_t n, const double* x, const double* y,
            int32_t* pixels, int64_t* outside) {
  int64_t out = 0;
  for (int64_t c = 0; c < n; ++c) {
    int32_t ix, iy;
    if (or_pixel_of(P, x[c], y[c], &ix, &iy))
      pixels[(int64_t)iy * P->grid_n + ix] += 1;
    else
      ++out;
  }
  *outside += out;
}

/* ------------------------------------------------------------------------ */
/* Simplified spherical model (Sec. 2.2, Eq. 7): the repulsion field of a    */
/* hole at distance r from the cloud centre is k_C Q(<r) / r^3 times its     */
/* offset from the centre, Q(<r) the number of holes strictly closer.  The    */
/* centre is the mean position of the active holes.  Written as the plain     */
/* double loop over pairs (no sorting), holes only.                          */
/* ------------------------------------------------------------------------ */
void or_field_spherical(int64_t n_act, const int64_t* rows, const double* x, const double* y,
                        const double* z, double kc, double* ex, double* ey, double* ez) {
  double cx = 0.0, cy = 0.0, cz = 0.0;
  for (int64_t r = 0; r < n_act; ++r) {
    cx += x[rows[r]];
    cy += y[rows[r]];
    cz += z[rows[r]];
  }
  if (n_act > 0) {
    cx /= (double)n_act;
    cy /= (double)n_act;
    cz /= (double)n_act;
  }
  double* d2 = (double*)calloc((size_t)(n_act > 0 ? n_act : 1), sizeof(double));
  for (int64_t r = 0; r < n_act; ++r) {
    const int64_t c = rows[r];
    const double dx = x[c] - cx, dy = y[c] - cy, dz = z[c] - cz;
    d2[r] = dx * dx + dy * dy + dz * dz;
  }
  for (int64_t r = 0; r < n_act; ++r) {
    int64_t q = 0;
    for (int64_t s = 0; s < n_act; ++s)
      if (d2[s] < d2[r]) ++q;
    const int64_t c = rows[r];
    ex[r] = ey[r] = ez[r] = 0.0;
    if (q == 0) continue;
    const double rr = sqrt(d2[r]);
    const double f = kc * (double)q / (d2[r] * rr);
    ex[r] = f * (x[c] - cx);
    ey[r] = f * (y[c] - cy);
    ez[r] = f * (z[c] - cz);
  }
  free(d2);
}

/* ------------------------------------------------------------------------ */
/* Event initialisation (Algorithm 1, first step; Sec. 2.1 and Eq. 2).       */
/* ------------------------------------------------------------------------ */
int64_t or_event_carriers(const or_params_t* P, const or_event_t* ev) {
  int64_t n = ev->kind == OR_EXPLICIT ? ev->n_pairs
              : (ev->n_pairs > 0 ? ev->n_pairs : or_n_pairs(ev->energy_keV));
  if (ev->kind == OR_EXPLICIT) return n;
  return P->species == OR_BOTH ? 2 * n : n;
}

void or_init_event(const or_params_t* P, const or_event_t* ev, double* x,
                   double* y, double* z, int8_t* sign) {
  if (ev->kind == OR_EXPLICIT) {
    for (int64_t c = 0; c < ev->n_pairs; ++c) {
      x[c] = ev->explicit_xyz[3 * c + 0];
      y[c] = ev->explicit_xyz[3 * c + 1];
      z[c] = ev->explicit_xyz[3 * c + 2];
      sign[c] = ev->explicit_sign ? ev->explicit_sign[c] : (int8_t)1;
    }
    return;
  }
  int64_t np = ev->n_pairs > 0 ? ev->n_pairs : or_n_pairs(ev->energy_keV);
  double sigma = ev->sigma_um >= 0.0 ? ev->sigma_um : or_sigma_um(ev->energy_keV);
  double z_entry = P->thickness_um - ev->depth_um;
  /* Track direction: polar angle theta from the inward normal (-e_z), azimuth
   * phi; the segment starts at the entry point on the back surface. */
  double th = ev->theta_deg * OR_PI / 180.0, ph = ev->phi_deg * OR_PI / 180.0;
  double ux = sin(th) * cos(ph), uy = sin(th) * sin(ph), uz = -cos(th);
  /* two unit vectors perpendicular to the track */
  double ax = cos(th) * cos(ph), ay = cos(th) * sin(ph), az = sin(th);
  double bx = -sin(ph), by = cos(ph), bz = 0.0;
  for (int64_t p = 0; p < np; ++p) {
    double n[3];
    or_normals3(ev->seed, ev->event_id, OR_PURPOSE_INIT, (uint32_t)p, 0u, n);
    double cx, cy, cz;
    if (ev->kind == OR_TRACK) {
      uint32_t w[4];
      or_stream_words(ev->seed, ev->event_id, OR_PURPOSE_INIT, (uint32_t)p, 1u, w);
      double s = or_uniform(w[0]) * ev->track_len_um;
      cx = ev->x_um + s * ux + sigma * (n[0] * ax + n[1] * bx);
      cy = ev->y_um + s * uy + sigma * (n[0] * ay + n[1] * by);
      cz = P->thickness_um + s * uz + sigma * (n[0] * az + n[1] * bz);
    } else {
      cx = ev->x_um + sigma * n[0];
      cy = ev->y_um + sigma * n[1];
      cz = z_entry + sigma * n[2];
    }
    x[p] = cx; y[p] = cy; z[p] = cz; sign[p] = 1;
    if (P->species == OR_BOTH) {
      x[np + p] = cx; y[np + p] = cy; z[np + p] = cz; sign[np + p] = -1;
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Boundaries.  Holes reaching z <= 0 are collected by the readout (stop    */
/* rule of Sec. 2.1); holes beyond the back surface are reflected.          */
/* Electrons reaching z >= H leave through the back contact; electrons      */
/* below z = 0 are reflected.                                               */
/* ------------------------------------------------------------------------ */
static void or_boundaries(const or_params_t* P, int64_t n, double* x, double* y,
                          double* z, const int8_t* sign, int8_t* state,
                          int64_t step, or_result_t* R) {
  double H = P->thickness_um;
  for (int64_t c = 0; c < n; ++c) {
    if (state[c] != OR_ACTIVE) continue;
    if (sign[c] > 0) {
      if (z[c] <= 0.0) {
        state[c] = OR_COLLECTED;
        if (R->final_x) R->final_x[c] = x[c];
        if (R->final_y) R->final_y[c] = y[c];
        if (R->retire_step) R->retire_step[c] = (int32_t)step;
      } else if (z[c] > H) {
        z[c] = 2.0 * H - z[c];
      }
    } else {
      if (z[c] >= H) {
        state[c] = OR_RETIRED;
        if (R->retire_step) R->retire_step[c] = (int32_t)step;
      } else if (z[c] < 0.0) {
        z[c] = -z[c];
      }
    }
  }
}

/* ------------------------------------------------------------------------ */
/* Pixel weighting potential (Shockley-Ramo; the weighting field that the    */
/* paper names as the extension towards transient signals, Sec. 5.3).       */
/* The weighting potential phi of a pixel solves Laplace's equation in the   */
/* sensor slab 0 < z < H with phi = 1 on the pixel's rectangle of the        */
/* collecting surface z = 0, phi = 0 on the rest of that surface and on the  */
/* back surface z = H (pixels tile the surface; no gaps).                    */
/*                                                                           */
/* Half space: the Dirichlet Poisson kernel zeta / (2 pi r^3) integrated     */
/* over a rectangle is the solid angle / 2 pi; for the corner offsets        */
/* u = X - x, v = Y - y it is the signed sum over the four corners of        */
/*   F(u, v, zeta) = atan(u v / (zeta sqrt(u^2 + v^2 + zeta^2))) / (2 pi),   */
/* an odd function of zeta (zeta -> 0+: 1 inside, 0 outside).                */
/* Slab: images at z + 2 n H (n over all integers) make phi vanish on z = H; */
/* the series converges when the terms n and -n are taken together, and a    */
/* pair n behaves for large n like                                           */
/*   -A z / (4 pi H^3 n^3) + A z (3 <r^2> - 2 z^2) / (16 pi H^5 n^5),        */
/* A the pixel's area and <r^2> the mean square lateral distance from the    */
/* point to the pixel's area.  The oracle sums the pairs up to n = 32 and   */
/* the rest by these two terms (zeta(3) and zeta(5) less the partial sums);  */
/* the next term is of order A z r^4 / (H^7 n^7): below 1e-10 for points     */
/* over the pixel grids used here.                                           */
/* ------------------------------------------------------------------------ */
#define OR_WEIGHT_PAIRS 32
static const double OR_ZETA3 = 1.2020569031595942854;
static const double OR_ZETA5 = 1.0369277551433699263;

static double or_corner(double u, double v, double zeta) {
  double r = sqrt(u * u + v * v + zeta * zeta);
  if (zeta == 0.0) {  /* the limit zeta -> 0+ */
    double uv = u * v;
    return uv > 0.0 ? 0.25 : (uv < 0.0 ? -0.25 : 0.0);
  }
  return atan(u * v / (zeta * r)) / (2.0 * OR_PI);
}

/* Half-space potential of the rectangle [x1, x2] x [y1, y2] at height zeta. */
double or_rect_solid_angle(double x, double y, double zeta, double x1, double x2,
                           double y1, double y2) {
  return or_corner(x2 - x, y2 - y, zeta) - or_corner(x1 - x, y2 - y, zeta) -
         or_corner(x2 - x, y1 - y, zeta) + or_corner(x1 - x, y1 - y, zeta);
}

/* Weighting potential of the pixel [x1, x2) x [y1, y2) at (x, y, z) of a
 * sensor of thickness H (n_pairs image pairs, then the two-term tail). */
double or_weighting_potential(double x, double y, double z, double x1, double x2,
                              double y1, double y2, double H, int32_t n_pairs) {
  if (z >= H) return 0.0;
  if (z <= 0.0) return (x >= x1 && x < x2 && y >= y1 && y < y2) ? 1.0 : 0.0;
  double phi = or_rect_solid_angle(x, y, z, x1, x2, y1, y2);
  double s3 = OR_ZETA3, s5 = OR_ZETA5;
  for (int32_t n = 1; n <= n_pairs; ++n) {
    phi += or_rect_solid_angle(x, y, z + 2.0 * n * H, x1, x2, y1, y2);
    phi += or_rect_solid_angle(x, y, z - 2.0 * n * H, x1, x2, y1, y2);
    s3 -= 1.0 / ((double)n * n * n);
    s5 -= 1.0 / ((double)n * n * n * n * n);
  }
  double a = x2 - x1, b = y2 - y1, A = a * b;
  double cx = 0.5 * (x1 + x2) - x, cy = 0.5 * (y1 + y2) - y;
  double r2 = cx * cx + cy * cy + (a * a + b * b) / 12.0;
  phi += -A * z / (4.0 * OR_PI * H * H * H) * s3 +
         A * z * (3.0 * r2 - 2.0 * z * z) / (16.0 * OR_PI * pow(H, 5.0)) * s5;
  return phi;
}

/* The 3 x 3 pixels around the grid's centre pixel (grid_n / 2, grid_n / 2),
 * row-major [b][a] for the grid pixel (c - 1 + a, c - 1 + b).  On the
 * collecting surface (z <= 0) a pixel's potential is 1 exactly when the point
 * is read out in it (the readout's own pixel rule), on the back surface 0. */
void or_window_potentials(const or_params_t* P, double x, double y, double z,
                          double phi[9]) {
  int32_t c = P->grid_n / 2;
  double p = P->pitch_um, half = 0.5 * (double)P->grid_n;
  for (int k = 0; k < 9; ++k) phi[k] = 0.0;
  if (z >= P->thickness_um) return;
  if (z <= 0.0) {
    int32_t ix, iy;
    if (or_pixel_of(P, x, y, &ix, &iy) && abs(ix - c) <= 1 && abs(iy - c) <= 1)
      phi[(iy - c + 1) * 3 + (ix - c + 1)] = 1.0;
    return;
  }
  for (int b = 0; b < 3; ++b)
    for (int a = 0; a < 3; ++a) {
      double x1 = ((double)(c - 1 + a) - half) * p, y1 = ((double)(c - 1 + b) - half) * p;
      phi[b * 3 + a] = or_weighting_potential(x, y, z, x1, x1 + p, y1, y1 + p,
                                              P->thickness_um, OR_WEIGHT_PAIRS);
    }
}

/* ------------------------------------------------------------------------ */
/* The moves of one step (Eqs. 3, 5): for active carrier c = rows[r] with    */
/* repulsion field (ex, ey, ez)[r] at the step start, total field E = E_rep  */
/* + drift field (Eq. 6), mobility mu(|E|), drift sign(q) mu E dt and the     */
/* Gaussian diffusion step sqrt(2 D dt) g, D = mu kT/e, g from the event's   */
/* stream at counter (c, step).  New positions go to (nx, ny, nz)[r].        */
/* ------------------------------------------------------------------------ */
static void or_moves(const or_params_t* P, uint64_t seed, uint64_t event_id, int64_t step,
                     int64_t n_act, const int64_t* rows, const double* x, const double* y,
                     const double* z, const int8_t* sign, const double* ex, const double* ey,
                     const double* ez, int parallel, double* nx, double* ny, double* nz) {
  double kT = or_thermal_voltage(P->temperature_K);
  double dt = P->dt_ps * 1e-3; /* ps -> ns */
#pragma omp parallel for schedule(static) if (parallel)
  for (int64_t r = 0; r < n_act; ++r) {
    int64_t c = rows[r];
    double Ex = ex[r], Ey = ey[r], Ez = ez[r];
    if (P->drift) Ez += -or_drift_field(P, z[c]);
    double Emag = sqrt(Ex * Ex + Ey * Ey + Ez * Ez);
    double mu = or_mobility(P, sign[c], Emag);
    double s = (double)sign[c];
    double dx = s * mu * Ex * dt, dy = s * mu * Ey * dt, dz = s * mu * Ez * dt;
    if (P->diffusion) {
      double D = mu * kT;
      double g[3];
      or_normals3(seed, event_id, OR_PURPOSE_DIFFUSION, (uint32_t)c, (uint32_t)step, g);
      double a = sqrt(2.0 * D * dt);
      dx += a * g[0]; dy += a * g[1]; dz += a * g[2];
    }
    nx[r] = x[c] + dx; ny[r] = y[c] + dy; nz[r] = z[c] + dz;
  }
}

/* ------------------------------------------------------------------------ */
/* One event, Algorithm 1: repeat {repulsion field of every carrier from the */
/* positions at the start of the step; drift field Eq. 6; mobility from     */
/* |E_drift + E_repulsion|; D = mu kT/e; x, y by Eq. 3 and z by Eq. 5 with  */
/* Gaussian steps of variance 2 D dt} until every hole is collected.         */
/* ------------------------------------------------------------------------ */
int or_run_event(const or_params_t* P, const or_event_t* ev, or_result_t* R,
                 int parallel) {
  int64_t n = or_event_carriers(P, ev);
  double* x = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* y = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* z = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* ex = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* ey = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* ez = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  int64_t* rows = (int64_t*)calloc((size_t)(n > 0 ? n : 1), sizeof(int64_t));
  int8_t* sign = (int8_t*)calloc((size_t)(n > 0 ? n : 1), 1);
  int8_t* state = (int8_t*)calloc((size_t)(n > 0 ? n : 1), 1);

  double kc = or_coulomb_k(P->eps_r);

  double* nx = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* ny = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  double* nz = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));

  R->status = OR_OK;
  R->n_steps = R->n_collected = R->n_outside = R->n_lost = R->interactions = 0;
  if (R->pixels)
    memset(R->pixels, 0, sizeof(int32_t) * (size_t)P->grid_n * (size_t)P->grid_n);
  if (R->retire_step)
    for (int64_t c = 0; c < n; ++c) R->retire_step[c] = -2;
  if (R->final_x)
    for (int64_t c = 0; c < n; ++c) R->final_x[c] = NAN;
  if (R->final_y)
    for (int64_t c = 0; c < n; ++c) R->final_y[c] = NAN;

  or_init_event(P, ev, x, y, z, sign);
  for (int64_t c = 0; c < n; ++c) state[c] = OR_ACTIVE;
  or_boundaries(P, n, x, y, z, sign, state, -1, R);

  double* ox = NULL;  /* step-start positions, for the pixel signals */
  double* oy = NULL;
  double induced_px[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  if (R->induced_px) {
    ox = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    oy = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
    for (int64_t k = 0; k < 9 * R->induced_capacity; ++k) R->induced_px[k] = NAN;
  }

  int64_t step = 0;
  double induced_q = 0.0;
  for (;; ++step) {
    int64_t holes_active = 0, n_act = 0;
    for (int64_t c = 0; c < n; ++c) {
      if (state[c] != OR_ACTIVE) continue;
      rows[n_act++] = c;
      if (sign[c] > 0) ++holes_active;
    }
    if (holes_active == 0) break;
    if (step >= P->max_steps) { R->status = OR_EMAXSTEPS; break; }
    /* pair terms of Eq. 4, or (spherical model) field evaluations */
    R->interactions += P->spherical ? n_act : n_act * (n_act - 1);

    /* Field of every active carrier from the positions at the step start. */
    if (P->repulsion && P->spherical) {
      or_field_spherical(n_act, rows, x, y, z, kc, ex, ey, ez);
    } else if (P->repulsion) {
      or_field_rows(n, x, y, z, sign, state, rows, n_act, kc, P->softening_um,
                    parallel, ex, ey, ez);
    } else {
      for (int64_t r = 0; r < n_act; ++r) ex[r] = ey[r] = ez[r] = 0.0;
    }
    /* Moves (all from step-start positions, then committed together). */
    or_moves(P, ev->seed, ev->event_id, step, n_act, rows, x, y, z, sign, ex, ey, ez, parallel,
             nx, ny, nz);
    for (int64_t r = 0; r < n_act; ++r) {
      int64_t c = rows[r];
      ez[r] = z[c];  /* the depth before the move, for the induced charge */
      if (ox) { ox[r] = x[c]; oy[r] = y[c]; }
      x[c] = nx[r]; y[c] = ny[r]; z[c] = nz[r];
    }
    or_boundaries(P, n, x, y, z, sign, state, step, R);
    /* Shockley-Ramo with the weighting potential 1 - z / H of the whole
     * collecting surface (a planar sensor): a charge q moving from z_a to z_b
     * induces q (z_a - z_b) / H; carriers that left stop at the surface. */
    for (int64_t r = 0; r < n_act; ++r) {
      int64_t c = rows[r];
      double zb = z[c] < 0.0 ? 0.0 : (z[c] > P->thickness_um ? P->thickness_um : z[c]);
      induced_q += (double)sign[c] * (ez[r] - zb) / P->thickness_um;
    }
    if (R->induced && step < R->induced_capacity) R->induced[step] = induced_q;
    /* The same theorem per pixel: q (phi_p(end) - phi_p(start)) with each
     * pixel's weighting potential (end point held on [0, H]). */
    if (R->induced_px) {
      double* d = (double*)malloc(sizeof(double) * 9 * (size_t)(n_act > 0 ? n_act : 1));
#pragma omp parallel for schedule(static) if (parallel)
      for (int64_t r = 0; r < n_act; ++r) {
        int64_t c = rows[r];
        double zb = z[c] < 0.0 ? 0.0 : (z[c] > P->thickness_um ? P->thickness_um : z[c]);
        double pa[9], pb[9];
        or_window_potentials(P, ox[r], oy[r], ez[r], pa);
        or_window_potentials(P, x[c], y[c], zb, pb);
        for (int k = 0; k < 9; ++k) d[9 * r + k] = (double)sign[c] * (pb[k] - pa[k]);
      }
      for (int64_t r = 0; r < n_act; ++r)
        for (int k = 0; k < 9; ++k) induced_px[k] += d[9 * r + k];
      free(d);
      if (step < R->induced_capacity)
        for (int k = 0; k < 9; ++k) R->induced_px[9 * step + k] = induced_px[k];
    }
  }
  R->n_steps = step;

  /* Readout of the collected holes; electrons still moving are dropped. */
  int64_t outside = 0;
  for (int64_t c = 0; c < n; ++c) {
    if (state[c] == OR_COLLECTED) {
      R->n_collected += 1;
      int32_t ix, iy;
      if (or_pixel_of(P, x[c], y[c], &ix, &iy)) {
        if (R->pixels) R->pixels[(int64_t)iy * P->grid_n + ix] += 1;
      } else {
        ++outside;
      }
    } else if (state[c] == OR_ACTIVE && sign[c] < 0) {
      R->n_lost += 1;
    }
  }
  R->n_outside = outside;
  if (R->pos_out)
    for (int64_t c = 0; c < n; ++c) {
      R->pos_out[3 * c + 0] = x[c];
      R->pos_out[3 * c + 1] = y[c];
      R->pos_out[3 * c + 2] = z[c];
    }
  if (R->state_out) memcpy(R->state_out, state, (size_t)n);
  if (R->sign_out) memcpy(R->sign_out, sign, (size_t)n);

  free(x); free(y); free(z); free(ex); free(ey); free(ez);
  free(nx); free(ny); free(nz);
  free(rows); free(sign); free(state);
  free(ox); free(oy);
  return R->status;
}

/* Independent events in parallel (one OpenMP thread per event). */
void or_run_events(const or_params_t* P, const or_event_t* evs, int64_t n_ev,
                   or_result_t* R) {
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t e = 0; e < n_ev; ++e) or_run_event(P, &evs[e], &R[e], 0);
}

/* ------------------------------------------------------------------------ */
/* One time step of Algorithm 1 from a given state (one-step parity tests):  */
/* the repulsion field of every active carrier from the positions given,     */
/* the moves at step index `step`, committed together, then the boundaries.  */
/* x, y, z, state: n carriers laid out as or_init_event does (holes, then    */
/* the pairs' electrons), updated in place.  Returns the active carriers     */
/* before the step.                                                          */
/* ------------------------------------------------------------------------ */
int64_t or_step(const or_params_t* P, uint64_t seed, uint64_t event_id, int64_t step,
                int64_t n, double* x, double* y, double* z, const int8_t* sign,
                int8_t* state, int parallel) {
  size_t m = (size_t)(n > 0 ? n : 1);
  int64_t* rows = (int64_t*)calloc(m, sizeof(int64_t));
  double* ex = (double*)calloc(m, sizeof(double));
  double* ey = (double*)calloc(m, sizeof(double));
  double* ez = (double*)calloc(m, sizeof(double));
  double* nx = (double*)calloc(m, sizeof(double));
  double* ny = (double*)calloc(m, sizeof(double));
  double* nz = (double*)calloc(m, sizeof(double));
  int64_t n_act = 0;
  for (int64_t c = 0; c < n; ++c)
    if (state[c] == OR_ACTIVE) rows[n_act++] = c;
  if (P->repulsion)
    or_field_rows(n, x, y, z, sign, state, rows, n_act, or_coulomb_k(P->eps_r),
                  P->softening_um, parallel, ex, ey, ez);
  or_moves(P, seed, event_id, step, n_act, rows, x, y, z, sign, ex, ey, ez, parallel, nx, ny, nz);
  for (int64_t r = 0; r < n_act; ++r) {
    int64_t c = rows[r];
    x[c] = nx[r]; y[c] = ny[r]; z[c] = nz[r];
  }
  or_result_t R;
  memset(&R, 0, sizeof R);
  or_boundaries(P, n, x, y, z, sign, state, step, &R);
  free(rows); free(ex); free(ey); free(ez); free(nx); free(ny); free(nz);
  return n_act;
}

int or_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}


/* ------------------------------------------------------------------------ */
/* Detector readout (Sec. 4.1 selection; Sec. 4.2 event generation).         */
/* ------------------------------------------------------------------------ */

/* Carrier-pair count with Fano statistics (Sec. 4.2 applies a Fano factor of
 * 0.13): the mean is E / 3.62 eV and the variance F times the mean; a normal
 * approximation, N = round(mean + sqrt(F * mean) * g), g the first normal of
 * the event's FANO stream (carrier 0, step 0), at least 1 pair.  F = 0 gives
 * or_n_pairs exactly. */
int32_t or_fano_pairs(uint64_t seed, uint64_t event_id, double energy_keV, double fano) {
  const double mean = energy_keV * 1000.0 / OR_EV_PER_PAIR;
  if (!(fano > 0.0)) return or_n_pairs(energy_keV);
  double g[3];
  or_normals3(seed, event_id, OR_PURPOSE_FANO, 0u, 0u, g);
  const double n = floor(mean + sqrt(fano * mean) * g[0] + 0.5);
  return n < 1.0 ? 1 : (int32_t)n;
}

/* Readout of one event's pixel counts (grid_n x grid_n, row-major, index
 * iy * grid_n + ix), following the selection described in Sec. 4.1 and the
 * generation in Sec. 4.2:
 *   energy of pixel p: e_p = counts_p * ev_per_pair / 1000 + noise * g_p keV,
 *     g_p the first normal of the event's NOISE stream at carrier p;
 *   centre: the pixel of largest e (the first in row-major order on ties);
 *   cluster: the 3 x 3 pixels around the centre that lie on the grid, its
 *     energy the sum of their e;
 *   pile-up veto: a pixel of the 7 x 7 window around the centre, outside the
 *     3 x 3, on the grid, with e > veto_factor * noise rejects the event;
 *   window: the event is accepted only if |cluster energy - beam| <= window.
 * Pixels off the grid are not read out: they neither add nor veto.  Writes
 * e[grid_n^2], cluster[9] (row-major 3 x 3 around the centre, NaN off the
 * grid), *cx, *cy, *e_cluster and returns 1 if the event is accepted. */
int or_readout_event(const int32_t* counts, int32_t grid_n, uint64_t seed, uint64_t event_id,
                     double ev_per_pair, double noise_keV, double beam_keV, double window_keV,
                     double veto_factor, double* e, double* cluster, int32_t* cx, int32_t* cy,
                     double* e_cluster, int32_t* vetoed) {
  const int32_t n = grid_n;
  int32_t best = 0;
  for (int32_t p = 0; p < n * n; ++p) {
    double g[3] = {0.0, 0.0, 0.0};
    if (noise_keV > 0.0) or_normals3(seed, event_id, OR_PURPOSE_NOISE, (uint32_t)p, 0u, g);
    e[p] = (double)counts[p] * ev_per_pair * 1e-3 + noise_keV * g[0];
    if (e[p] > e[best]) best = p;
  }
  const int32_t bx = best % n, by = best / n;
  double sum = 0.0;
  for (int32_t dy = -1; dy <= 1; ++dy)
    for (int32_t dx = -1; dx <= 1; ++dx) {
      const int32_t x = bx + dx, y = by + dy;
      const int on = x >= 0 && y >= 0 && x < n && y < n;
      const double v = on ? e[y * n + x] : NAN;
      cluster[(dy + 1) * 3 + (dx + 1)] = v;
      if (on) sum += v;
    }
  int32_t veto = 0;
  for (int32_t dy = -3; dy <= 3; ++dy)
    for (int32_t dx = -3; dx <= 3; ++dx) {
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
      const int32_t x = bx + dx, y = by + dy;
      if (x < 0 || y < 0 || x >= n || y >= n) continue;
      if (e[y * n + x] > veto_factor * noise_keV) veto = 1;
    }
  *cx = bx;
  *cy = by;
  *e_cluster = sum;
  *vetoed = veto;
  return !veto && fabs(sum - beam_keV) <= window_keV;
}

/* Single-pixel spectrum (Sec. 4.1: single-pixel energies of the accepted
 * 3 x 3 clusters): each on-grid cluster pixel of an accepted event adds one
 * count to bin floor((e - lo) / width) of n_bins, values outside ignored. */
void or_spectrum_add(const double* cluster, int32_t accepted, double lo_keV, double width_keV,
                     int32_t n_bins, int64_t* hist) {
  if (!accepted) return;
  for (int k = 0; k < 9; ++k) {
    const double v = cluster[k];
    if (isnan(v)) continue;
    const double b = floor((v - lo_keV) / width_keV);
    if (b >= 0.0 && b < (double)n_bins) hist[(int64_t)b] += 1;
  }
}


/* ------------------------------------------------------------------------ */
/* Generalised Gaussian model of the collected cloud (Sec. 3.1, Eq. 8) and   */
/* fast event generation from it (Sec. 4.2).                                 */
/* ------------------------------------------------------------------------ */

/* Eq. 8: f(x) = beta / (2 alpha Gamma(1/beta)) exp(-(|x|/alpha)^beta), the
 * density on the whole line (the printed form omits the factor 1/2 of the
 * two-sided density and the absolute value). */
double or_ggd_pdf(double x, double alpha, double beta) {
  return beta / (2.0 * alpha * tgamma(1.0 / beta)) * exp(-pow(fabs(x) / alpha, beta));
}

/* Maximum-likelihood fit of Eq. 8 to samples centred at 0: for a given beta
 * the likelihood is largest at alpha^beta = (beta / n) sum |x|^beta; the
 * profile log-likelihood is maximised over beta in [0.3, 20] by golden
 * section on log beta (it is unimodal there for real data).  Returns 0, -1 if
 * n < 2 or all samples are 0. */
static double or_ggd_profile(const double* x, int64_t n, double beta, double* alpha) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += pow(fabs(x[i]), beta);
  const double a = pow(beta * s / (double)n, 1.0 / beta);
  *alpha = a;
  return (double)n * (log(beta / (2.0 * a)) - lgamma(1.0 / beta) - 1.0 / beta);
}

int or_fit_ggd(const double* x, int64_t n, double* alpha, double* beta) {
  if (n < 2) return -1;
  int any = 0;
  for (int64_t i = 0; i < n; ++i) any |= x[i] != 0.0;
  if (!any) return -1;
  const double g = 0.5 * (sqrt(5.0) - 1.0);
  double lo = log(0.3), hi = log(20.0), a;
  double c = hi - g * (hi - lo), d = lo + g * (hi - lo);
  double fc = or_ggd_profile(x, n, exp(c), &a), fd = or_ggd_profile(x, n, exp(d), &a);
  for (int it = 0; it < 200 && hi - lo > 1e-12; ++it) {
    if (fc > fd) {
      hi = d; d = c; fd = fc;
      c = hi - g * (hi - lo);
      fc = or_ggd_profile(x, n, exp(c), &a);
    } else {
      lo = c; c = d; fc = fd;
      d = lo + g * (hi - lo);
      fd = or_ggd_profile(x, n, exp(d), &a);
    }
  }
  *beta = exp(0.5 * (lo + hi));
  or_ggd_profile(x, n, *beta, alpha);
  return 0;
}

/* One standard Gamma(shape) variate, shape > 0, from the event's GGD stream:
 * Gamma(shape + 1) by Marsaglia and Tsang's squeeze-free rejection (ACM TOMS
 * 26, 2000) with attempt k drawing (z, u) from counter (carrier, 4 k + axis'),
 * then the boost Gamma(shape) = Gamma(shape + 1) U^(1 / shape) with U from a
 * counter of its own.  axis' = 2 * axis for the rejection loop. */
static double or_gamma(uint64_t seed, uint64_t ev, uint32_t carrier, uint32_t axis, double shape,
                       uint32_t* sign_word) {
  const double d = shape + 1.0 - 1.0 / 3.0, c = 1.0 / sqrt(9.0 * d);
  double g = d;
  for (uint32_t k = 0; k < 64; ++k) {
    uint32_t w[4];
    or_stream_words(seed, ev, OR_PURPOSE_GGD, carrier, 4u * k + 2u * axis, w);
    const double z = sqrt(-2.0 * log(or_uniform(w[0]))) * cos(2.0 * OR_PI * or_uniform(w[1]));
    const double v1 = 1.0 + c * z;
    if (v1 <= 0.0) continue;
    const double v = v1 * v1 * v1;
    if (log(or_uniform(w[2])) < 0.5 * z * z + d - d * v + d * log(v)) {
      g = d * v;
      break;
    }
  }
  uint32_t b[4];
  or_stream_words(seed, ev, OR_PURPOSE_GGD, carrier, 4u * 64u + axis, b);
  *sign_word = b[1];
  return g * pow(or_uniform(b[0]), 1.0 / shape);
}

/* One GGD(alpha, beta) variate: alpha G^(1/beta), G ~ Gamma(1/beta), with a
 * random sign (the generalised Gaussian is |X|/alpha = G^(1/beta)). */
double or_ggd_sample(uint64_t seed, uint64_t ev, uint32_t carrier, uint32_t axis, double alpha,
                     double beta) {
  uint32_t sw;
  const double g = or_gamma(seed, ev, carrier, axis, 1.0 / beta, &sw);
  const double m = alpha * pow(g, 1.0 / beta);
  return (sw >> 31) ? -m : m;
}

/* Fast generation of one event (Sec. 4.2): n carriers with x and y drawn
 * independently from GGD(alpha, beta) about the entry point (x0, y0), binned
 * into the grid_n x grid_n pixels of pitch p centred on the origin (the same
 * pixel rule as the readout of simulated events).  Adds to pixels and
 * *outside. */
void or_generate_event(uint64_t seed, uint64_t ev, int32_t n, double x0, double y0, double alpha,
                       double beta, double pitch_um, int32_t grid_n, int32_t* pixels,
                       int64_t* outside) {
  for (int32_t c = 0; c < n; ++c) {
    const double x = x0 + or_ggd_sample(seed, ev, (uint32_t)c, 0u, alpha, beta);
    const double y = y0 + or_ggd_sample(seed, ev, (uint32_t)c, 1u, alpha, beta);
    const double fx = floor(x / pitch_um + 0.5 * (double)grid_n);
    const double fy = floor(y / pitch_um + 0.5 * (double)grid_n);
    if (fx < 0.0 || fy < 0.0 || fx >= (double)grid_n || fy >= (double)grid_n) {
      *outside += 1;
      continue;
    }
    pixels[(int64_t)fy * grid_n + (int64_t)fx] += 1;
  }
}
