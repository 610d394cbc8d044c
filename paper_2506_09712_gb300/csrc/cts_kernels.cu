// cts_kernels.cu -- sm_103a kernels of the brute-force charge-transport step
// (Xie et al., arXiv 2506.09712, Sec. 2.1 and Algorithm 1).
//
//   step_kernel   one time step for every resident event: the Eq. 4 pair
//                 field of a tile of carriers (FP32, rsqrt, Kahan-compensated
//                 across j chunks staged in shared memory by TMA bulk copies),
//                 then drift (Eq. 6), mobility, diffusion and the FP64
//                 position update of Eqs. 3 and 5, collection and exit.
//                 Persistent CTAs pull (event, i-tile, j-split) units from a
//                 per-step counter; j-splits are combined in FP64 by the CTA
//                 that finishes last.
//   update_kernel the update alone (two-launch PLAIN path).
//   init_kernel   the initial cloud of each new event (Algorithm 1, Eq. 2).
//   close_kernel  end-of-chunk bookkeeping and order-preserving compaction.
//   bin_kernel    warp-aggregated pixel readout of collected holes.
#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <curand_kernel.h>

#include <cstdint>

#include "cts_internal.h"

namespace cts {
namespace {

// ---------------------------------------------------------------------------
// Counter-based random numbers: Philox4x32-10 (Salmon et al., SC'11).
// Counter = (carrier, step, event lo, event hi ^ purpose << 28), key = seed.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint2 k) {
#pragma unroll
  for (int round = 0; round < 10; ++round) {
    const uint32_t hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo0 = 0xD2511F53u * c.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z);
    const uint32_t lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    k.x += 0x9E3779B9u;
    k.y += 0xBB67AE85u;
  }
  return c;
}

__device__ __forceinline__ uint4 stream_words(uint64_t seed, uint64_t ev, uint32_t purpose,
                                              uint32_t carrier, uint32_t step) {
  const uint4 c = make_uint4(carrier, step, (uint32_t)ev, (uint32_t)(ev >> 32) ^ (purpose << 28));
  return philox10(c, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// ((w >> 9) + 1/2) * 2^-23: exact in FP32 and FP64.
__device__ __forceinline__ float uniform_f(uint32_t w) {
  return ((float)(w >> 9) + 0.5f) * 1.1920928955078125e-07f;
}
__device__ __forceinline__ double uniform_d(uint32_t w) {
  return ((double)(w >> 9) + 0.5) * 1.1920928955078125e-07;
}

// Box-Muller: (n0, n1) from (u0, u1), n2 from the cosine branch of (u2, u3).
__device__ __forceinline__ float3 normals_f(uint4 w) {
  const float r01 = sqrtf(-2.0f * logf(uniform_f(w.x)));
  const float r23 = sqrtf(-2.0f * logf(uniform_f(w.z)));
  float s1, c1;
  sincospif(2.0f * uniform_f(w.y), &s1, &c1);
  const float c3 = cospif(2.0f * uniform_f(w.w));
  return make_float3(r01 * c1, r01 * s1, r23 * c3);
}
__device__ __forceinline__ double3 normals_d(uint4 w) {
  const double r01 = sqrt(-2.0 * log(uniform_d(w.x)));
  const double r23 = sqrt(-2.0 * log(uniform_d(w.z)));
  double s1, c1;
  sincospi(2.0 * uniform_d(w.y), &s1, &c1);
  const double c3 = cospi(2.0 * uniform_d(w.w));
  return make_double3(r01 * c1, r01 * s1, r23 * c3);
}

// ---------------------------------------------------------------------------
// Material model (Sec. 2.1): mu(E) = mu0 / (1 + (mu0 E / vsat)^beta)^(1/beta).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float mobility_f(const Phys& ph, int spec, float E) {
  const float mu0 = ph.f_mu0[spec];
  if (ph.mob_model == 1) return mu0;
  const float x = mu0 * E / ph.f_vsat[spec];
  return mu0 / powf(1.0f + powf(x, ph.f_beta[spec]), ph.f_ibeta[spec]);
}

// Drift-field magnitude at depth z (Eq. 6, or the handle's sampled profile).
__device__ __forceinline__ float drift_E(const Phys& ph, float z) {
  if (ph.drift_n < 2) return ph.f_ea - ph.f_eb * z;
  const float u = fminf(fmaxf(z * ph.f_drift_inv_dz, 0.0f), (float)(ph.drift_n - 1));
  const int k = min((int)u, ph.drift_n - 2);
  const float e0 = __ldg(ph.drift_tab + k), e1 = __ldg(ph.drift_tab + k + 1);
  return fmaf(u - (float)k, e1 - e0, e0);
}

// Frame anchor of a species for the next step: the drift-only motion of the
// cloud centre (its displacement in FP32, accumulated in FP64).  One body
// (noinline) so every CTA that evaluates it for a slot gets the same bits.
__device__ __noinline__ double anchor_next(const Phys& ph, int spec, double z) {
  if (!ph.drift) return z;
  const float E = drift_E(ph, (float)z);
  const float dz = mobility_f(ph, spec, E) * E * ph.f_dt;
  const double zn = spec == 0 ? __dsub_rn(z, (double)dz) : __dadd_rn(z, (double)dz);
  return fmin(fmax(zn, 0.0), ph.H);
}

// ---------------------------------------------------------------------------
// TMA bulk copies into shared memory, completed on an mbarrier.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes,
                                            uint64_t* bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after kWaitLimit polls (far beyond any copy time).
constexpr uint32_t kWaitLimit = 1u << 24;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kWaitLimit; ++it)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// Bounded wait for a counter written by other CTAs of the launch to reach
// target (acquire); about two seconds at most, then false.
constexpr unsigned long long kCountWaitNs = 2000000000ull;
__device__ __forceinline__ bool wait_count_bounded(const int32_t* ctr, int target) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (uint32_t it = 0;; ++it) {
    int v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(ctr) : "memory");
    if (v >= target) {
      asm volatile("fence.proxy.async.global;" ::: "memory");
      return true;
    }
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > kCountWaitNs) return false;
    __nanosleep(it < 32 ? 64 : 512);
  }
}

__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly,
// s = fl(a + b).
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}


// The pair loop over n staged sources: acc_i += (r_i - r_j) / (|r_i - r_j|^2 +
// eps^2)^(3/2), or the reversed difference for sources of the opposite sign.
template <int R, bool NEG, int JU>
__device__ __forceinline__ void pair_chunk(const float4* __restrict__ sj, int n,
                                           const float (&xi)[R], const float (&yi)[R],
                                           const float (&zi)[R], float (&ax)[R], float (&ay)[R],
                                           float (&az)[R], float eps2) {
  int j = 0;
  for (; j + JU <= n; j += JU) {
#pragma unroll
    for (int h = 0; h < JU; ++h) {
      const float4 q = sj[j + h];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float dx = NEG ? q.x - xi[r] : xi[r] - q.x;
        const float dy = NEG ? q.y - yi[r] : yi[r] - q.y;
        const float dz = NEG ? q.z - zi[r] : zi[r] - q.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        const float rs = rsqrt_approx(r2);
        const float w = (rs * rs) * rs;
        ax[r] = fmaf(dx, w, ax[r]);
        ay[r] = fmaf(dy, w, ay[r]);
        az[r] = fmaf(dz, w, az[r]);
      }
    }
  }
  for (; j < n; ++j) {
    const float4 q = sj[j];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const float dx = NEG ? q.x - xi[r] : xi[r] - q.x;
      const float dy = NEG ? q.y - yi[r] : yi[r] - q.y;
      const float dz = NEG ? q.z - zi[r] : zi[r] - q.z;
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
      const float rs = rsqrt_approx(r2);
      const float w = (rs * rs) * rs;
      ax[r] = fmaf(dx, w, ax[r]);
      ay[r] = fmaf(dy, w, ay[r]);
      az[r] = fmaf(dz, w, az[r]);
    }
  }
}

// The same pair loop on packed FP32 pairs (two i's per 64-bit register pair,
// Blackwell's two-wide FMA/ADD/MUL): half the FP32 instruction issues.
// Differences come from one rounding of x_j * (-1) + x_i, i.e. exactly the
// rounded x_i - x_j of the scalar loop.
template <int P, bool NEG, int JU>
__device__ __forceinline__ void pair_chunk_packed(const float4* __restrict__ sj, int n,
                                                  const float2 (&xi)[P], const float2 (&yi)[P],
                                                  const float2 (&zi)[P], float2 (&ax)[P],
                                                  float2 (&ay)[P], float2 (&az)[P],
                                                  float eps2s) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 eps2 = make_float2(eps2s, eps2s);
#pragma unroll JU
  for (int j = 0; j < n; ++j) {
    const float4 q = sj[j];
    const float2 qx = make_float2(q.x, q.x);
    const float2 qy = make_float2(q.y, q.y);
    const float2 qz = make_float2(q.z, q.z);
#pragma unroll
    for (int r = 0; r < P; ++r) {
      const float2 dx = NEG ? __ffma2_rn(xi[r], m1, qx) : __ffma2_rn(qx, m1, xi[r]);
      const float2 dy = NEG ? __ffma2_rn(yi[r], m1, qy) : __ffma2_rn(qy, m1, yi[r]);
      const float2 dz = NEG ? __ffma2_rn(zi[r], m1, qz) : __ffma2_rn(qz, m1, zi[r]);
      float2 r2 = __ffma2_rn(dz, dz, eps2);
      r2 = __ffma2_rn(dy, dy, r2);
      r2 = __ffma2_rn(dx, dx, r2);
      const float2 rs = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
      const float2 w = __fmul2_rn(__fmul2_rn(rs, rs), rs);
      ax[r] = __ffma2_rn(dx, w, ax[r]);
      ay[r] = __ffma2_rn(dy, w, ay[r]);
      az[r] = __ffma2_rn(dz, w, az[r]);
    }
  }
}

// The pair loop with two sources per packed FP32 lane pair: sources come from
// a struct-of-arrays copy of the chunk (x[], y[], z[]), so one 128-bit load
// yields the (x_j, x_j+1) and (x_j+2, x_j+3) register pairs directly; the i
// position is held duplicated, (x_i, x_i).  m is a multiple of 4 (the copy is
// padded with parked sources, which contribute exactly zero).  Accumulators
// hold (sum over even j, sum over odd j).  Only the first RA of the R i slots
// are computed (the rest of a ragged tile holds no carriers).
template <int R, int RA, bool NEG>
__device__ __forceinline__ void pair_chunk_jpacked(const float* __restrict__ xs,
                                                   const float* __restrict__ ys,
                                                   const float* __restrict__ zs, int m,
                                                   const float2 (&xi)[R], const float2 (&yi)[R],
                                                   const float2 (&zi)[R], float2 (&ax)[R],
                                                   float2 (&ay)[R], float2 (&az)[R],
                                                   float eps2s) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 eps2 = make_float2(eps2s, eps2s);
#pragma unroll 2
  for (int j = 0; j < m; j += 4) {
    const float4 X = *reinterpret_cast<const float4*>(xs + j);
    const float4 Y = *reinterpret_cast<const float4*>(ys + j);
    const float4 Z = *reinterpret_cast<const float4*>(zs + j);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const float2 qx = h ? make_float2(X.z, X.w) : make_float2(X.x, X.y);
      const float2 qy = h ? make_float2(Y.z, Y.w) : make_float2(Y.x, Y.y);
      const float2 qz = h ? make_float2(Z.z, Z.w) : make_float2(Z.x, Z.y);
#pragma unroll
      for (int r = 0; r < RA; ++r) {
        const float2 dx = NEG ? __ffma2_rn(xi[r], m1, qx) : __ffma2_rn(qx, m1, xi[r]);
        const float2 dy = NEG ? __ffma2_rn(yi[r], m1, qy) : __ffma2_rn(qy, m1, yi[r]);
        const float2 dz = NEG ? __ffma2_rn(zi[r], m1, qz) : __ffma2_rn(qz, m1, zi[r]);
        float2 r2 = __ffma2_rn(dz, dz, eps2);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dx, dx, r2);
        const float2 rs = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
        const float2 w = __fmul2_rn(__fmul2_rn(rs, rs), rs);
        ax[r] = __ffma2_rn(dx, w, ax[r]);
        ay[r] = __ffma2_rn(dy, w, ay[r]);
        az[r] = __ffma2_rn(dz, w, az[r]);
      }
    }
  }
}

// Kahan step (Higham, Accuracy and Stability, Alg. 4.2): s += t with the
// running compensation c.
__device__ __forceinline__ void kahan_add(float& s, float& c, float t) {
  const float y = t - c;
  const float u = s + y;
  c = (u - s) - y;
  s = u;
}

// The readout's pixel of a collected carrier: floor(x / pitch + n/2) per axis
// in FP64 (row-major key), -1 outside the grid.
__device__ __forceinline__ int pixel_at(double pitch, int grid_n, double x, double y) {
  const double half = 0.5 * (double)grid_n;
  const double fx = floor(__dadd_rn(__ddiv_rn(x, pitch), half));
  const double fy = floor(__dadd_rn(__ddiv_rn(y, pitch), half));
  if (!(fx >= 0.0 && fy >= 0.0 && fx < (double)grid_n && fy < (double)grid_n)) return -1;
  return (int)fy * grid_n + (int)fx;
}

__device__ __forceinline__ int pixel_key(const Phys& ph, double x, double y) {
  return pixel_at(ph.pitch, ph.grid_n, x, y);
}

#ifdef CTS_BOUNDS_CHECK
// Checked build (-DCTS_BOUNDS_CHECK): index checks that record kErrBounds and
// skip the access instead of making it.  A slot owns the arena entries
// [base, base + cap_h + cap_e), and its carrier ids are below n_total, which
// does not exceed that count.
__device__ __forceinline__ bool slot_in_arena(const Arena& A, const SlotDev* S) {
  const int64_t n = (int64_t)S->cap_h + S->cap_e;
  return S->base >= 0 && S->cap_h >= 0 && S->cap_e >= 0 && S->base + n <= A.capacity &&
         S->n_total >= 0 && S->n_total <= n;
}

// A unit's i range and source ranges lie in the arena, its slot in the table.
__device__ __forceinline__ bool unit_in_arena(const StepArgs& a, const Unit& U) {
  const int64_t cap = a.A.capacity;
  return U.slot >= 0 && U.slot < a.S && U.ni >= 0 && U.len_h >= 0 && U.len_e >= 0 &&
         U.ioff >= 0 && U.ioff + U.ni <= cap && U.hoff >= 0 && U.hoff + U.len_h <= cap &&
         U.eoff >= 0 && U.eoff + U.len_e <= cap;
}
#endif

// Weighting potentials (Shockley-Ramo) of the 3 x 3 pixels around the grid's
// centre pixel c = grid_n / 2 at (x, y, z), z on [0, H]; w[b * 3 + a] is grid
// pixel (c - 1 + a, c - 1 + b).  A pixel's potential solves Laplace's
// equation in the slab with 1 on the pixel and 0 on the rest of both
// surfaces.  Half space: the solid angle of the pixel / 2 pi, the signed sum
// over its corners (offsets u, v) of F = sign(zeta) atan2(u v, |zeta| r) / 2 pi,
// r = |(u, v, zeta)|; slab: images at z + 2 n H, n = -M..M (a corner shared by
// neighbouring pixels is evaluated once), the pairs beyond M by their
// expansion z (c3 + c5 (3 <r^2> - 2 z^2)), <r^2> the mean square lateral
// distance to the pixel's area.  On the collecting surface a pixel's
// potential is 1 where the readout puts the point, on the back surface 0.
// FP32 (the offsets from FP64 positions).  Not inlined: every position goes
// through the same code, so a carrier's potential at the end of a step equals
// the one at the start of the next bit for bit and the signals telescope.
__device__ __noinline__ void window_potentials(double x, double y, double z, double wx0,
                                               double wy0, double pitch, int grid_n, double H,
                                               int M, float c3, float c5, float* w) {
#pragma unroll
  for (int k = 0; k < 9; ++k) w[k] = 0.0f;
  if (z >= H) return;
  if (z <= 0.0) {
    const int key = pixel_at(pitch, grid_n, x, y);
    if (key < 0) return;
    const int c = grid_n / 2;
    const int a = key % grid_n - c + 1, b = key / grid_n - c + 1;
    if (a >= 0 && a < 3 && b >= 0 && b < 3) w[b * 3 + a] = 1.0f;
    return;
  }
  float u[4], v[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    u[i] = (float)(wx0 + (double)i * pitch - x);
    v[i] = (float)(wy0 + (double)i * pitch - y);
  }
  float acc[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = 0.0f;
  const float zf = (float)z, h2 = (float)(2.0 * H);
  for (int n = -M; n <= M; ++n) {
    const float zeta = fmaf((float)n, h2, zf);
    const float az = fabsf(zeta), sg = zeta < 0.0f ? -1.0f : 1.0f, z2 = zeta * zeta;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float r = sqrtf(fmaf(u[i], u[i], fmaf(v[j], v[j], z2)));
        const float f = sg * atan2f(u[i] * v[j], az * r);
        // corner (i, j) is the upper-right corner of pixel (i-1, j-1), the
        // upper-left of (i, j-1), the lower-right of (i-1, j), the lower-left of (i, j)
        if (i >= 1 && j >= 1) acc[(j - 1) * 3 + (i - 1)] += f;
        if (i <= 2 && j >= 1) acc[(j - 1) * 3 + i] -= f;
        if (i >= 1 && j <= 2) acc[j * 3 + (i - 1)] -= f;
        if (i <= 2 && j <= 2) acc[j * 3 + i] += f;
      }
    }
  }
  const float inv2pi = 0.159154943091895336f, q2 = (float)(pitch * pitch / 6.0);
#pragma unroll
  for (int b = 0; b < 3; ++b) {
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      const float cx = (float)(wx0 + ((double)a + 0.5) * pitch - x);
      const float cy = (float)(wy0 + ((double)b + 0.5) * pitch - y);
      const float r2 = fmaf(cx, cx, fmaf(cy, cy, q2));
      w[b * 3 + a] = fmaf(acc[b * 3 + a], inv2pi, zf * fmaf(c5, fmaf(3.0f, r2, -2.0f * zf * zf), c3));
    }
  }
}

// Position update of one active carrier (Eqs. 3, 5, 6; Sec. 2.1) at arena
// index idx, carrier id and state st, position (x, y, z) at the start of the
// step, with the field E (V/um) of its step: collection/exit and (SHADOW) the
// next shadow entry.  When the induced charge is recorded, returns H times
// the charge (units of e) the move induces on the collecting surface
// (Shockley-Ramo, weighting potential 1 - z/H, the end point held on [0, H]);
// else 0.  IND: 0 records nothing, 1 the whole surface, 2 also adds
// q (phi(end) - phi(start)) of the 3 x 3 window's pixels to qpx.  *retired
// (when given) is set when the carrier left.
template <int IND, bool SHADOW = true>
__device__ __forceinline__ double update_carrier_at(const StepArgs& a, SlotDev* S, int slot,
                                                  int spec, int64_t idx, int id, int8_t st,
                                                  double x, double y, double z, int step, int p,
                                                  int k, float Ex, float Ey, float Ez, double azn,
                                                  double* qpx = nullptr,
                                                  bool* retired = nullptr) {
  const Phys& ph = a.ph;
  [[maybe_unused]] float4* __restrict__ shout = a.A.sh[p ^ 1];
  const int64_t rid = S->base + id;
#ifdef CTS_BOUNDS_CHECK
  if (idx < 0 || idx >= a.A.capacity || slot < 0 || slot >= a.S || k < 0 || k >= kMaxK ||
      id < 0 || id >= S->n_total || rid < 0 || rid >= a.A.capacity) {
    atomicOr(a.err, kErrBounds);
    return 0.0;
  }
#endif
  [[maybe_unused]] const double x_start = x, y_start = y, z_start = z;
  if (ph.drift) Ez -= drift_E(ph, (float)z);
  const float Em = sqrtf(Ex * Ex + Ey * Ey + Ez * Ez);
  const float mu = mobility_f(ph, spec, Em);
  const float c = (spec ? -mu : mu) * ph.f_dt;
  float dx = c * Ex, dy = c * Ey, dz = c * Ez;
  if (ph.diffusion) {
    const float3 n = normals_f(stream_words(S->seed, S->event_id, 0u, (uint32_t)id, (uint32_t)step));
    const float amp = sqrtf(2.0f * mu * ph.f_kT * ph.f_dt);
    dx = fmaf(amp, n.x, dx);
    dy = fmaf(amp, n.y, dy);
    dz = fmaf(amp, n.z, dz);
  }
  if (!(isfinite(dx) && isfinite(dy) && isfinite(dz))) atomicOr(&S->flags, kErrNumeric);
  x += (double)dx;
  y += (double)dy;
  z += (double)dz;
  int retire = 0;
  if (spec == 0) {
    if (z <= 0.0) retire = kStateCollected;
    else if (z > ph.H) z = 2.0 * ph.H - z;
  } else {
    if (z >= ph.H) retire = kStateExited;
    else if (z < 0.0) z = -z;
  }
  a.A.px[idx] = x;
  a.A.py[idx] = y;
  a.A.pz[idx] = z;
  if (retired) *retired = retire != 0;
  if (retire) {
    a.A.cstate[rid] = (int8_t)((st & kElectronBit) | retire);
    a.A.rstep[rid] = step;
    if (retire == kStateCollected) {
      a.A.fx[rid] = x;
      a.A.fy[rid] = y;
    }
    atomicAdd(&a.ret[((int64_t)k * a.S + slot) * 2 + spec], 1);
    if constexpr (SHADOW) shout[idx] = make_float4(kParked, kParked, kParked, 0.0f);
  } else if constexpr (SHADOW) {
    shout[idx] = make_float4((float)(x - S->ax), (float)(y - S->ay), (float)(z - azn), 0.0f);
  }
  if constexpr (IND == 0) {
    return 0.0;
  } else {
    if (IND == 1 && !a.induced) return 0.0;
    const double zb = fmin(fmax(z, 0.0), ph.H);
    if constexpr (IND == 2) {
      float w0[9], w1[9];
      window_potentials(x_start, y_start, z_start, ph.wp_x0, ph.wp_y0, ph.pitch, ph.grid_n, ph.H,
                        ph.wp_pairs, ph.wp_c3, ph.wp_c5, w0);
      window_potentials(x, y, zb, ph.wp_x0, ph.wp_y0, ph.pitch, ph.grid_n, ph.H, ph.wp_pairs,
                        ph.wp_c3, ph.wp_c5, w1);
#pragma unroll
      for (int j = 0; j < 9; ++j)
        qpx[j] += spec ? (double)w0[j] - (double)w1[j] : (double)w1[j] - (double)w0[j];
    }
    if (!a.induced) return 0.0;
    return spec ? zb - z_start : z_start - zb;
  }
}

// update_carrier_at for the carrier at arena index idx, its id, state and
// position read here; a carrier that is not active gets a parked shadow.
template <int IND, bool SHADOW = true>
__device__ __forceinline__ double update_carrier(const StepArgs& a, SlotDev* S, int slot, int spec,
                                               int64_t idx, int step, int p, int k, float Ex,
                                               float Ey, float Ez, double azn,
                                               double* qpx = nullptr) {
#ifdef CTS_BOUNDS_CHECK
  if (idx < 0 || idx >= a.A.capacity) {
    atomicOr(a.err, kErrBounds);
    return 0.0;
  }
#endif
  const int id = a.A.cid[idx];
  const int64_t rid = S->base + id;
#ifdef CTS_BOUNDS_CHECK
  if (id < 0 || id >= S->n_total || rid < 0 || rid >= a.A.capacity) {
    atomicOr(a.err, kErrBounds);
    return 0.0;
  }
#endif
  const int8_t st = __ldcg(a.A.cstate + rid);
  if ((st & kStateMask) != kStateActive) {
    if constexpr (SHADOW) a.A.sh[p ^ 1][idx] = make_float4(kParked, kParked, kParked, 0.0f);
    return 0.0;
  }
  const double x = __ldcg(a.A.px + idx), y = __ldcg(a.A.py + idx), z = __ldcg(a.A.pz + idx);
  return update_carrier_at<IND, SHADOW>(a, S, slot, spec, idx, id, st, x, y, z, step, p, k, Ex,
                                        Ey, Ez, azn, qpx);
}

// Adds a warp's induced charges (H times, from update_carrier) to the slot's
// per-step total (all 32 lanes of the warp call this).
__device__ __forceinline__ void add_induced(const StepArgs& a, int k, int slot, double q) {
  if (!a.induced) return;
  for (int o = 16; o > 0; o >>= 1) q += __shfl_down_sync(0xffffffffu, q, o);
  if ((threadIdx.x & 31) == 0 && q != 0.0)
    atomicAdd(a.induced + (int64_t)k * a.S + slot, q / a.ph.H);
}

// Adds a warp's per-pixel induced charges (from update_carrier) to the slot's
// per-step record of the 3 x 3 window (all 32 lanes of the warp call this).
__device__ __forceinline__ void add_induced_px(const StepArgs& a, int k, int slot,
                                               const double (&q)[9]) {
  if (!a.induced_px) return;
  double* out = a.induced_px + ((int64_t)k * a.S + slot) * 9;
#pragma unroll
  for (int j = 0; j < 9; ++j) {
    double v = q[j];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(out + j, v);
  }
}

// Per-slot duties of a step, done once per slot: interaction count, step
// count and the next frame anchors.
__device__ __forceinline__ void slot_duties(const StepArgs& a, SlotDev* S, int step, int p,
                                            int nah, int nae, double azn0, double azn1) {
  const long long n = (long long)nah + (long long)nae;
  atomicAdd(&S->interactions, (unsigned long long)(n * (n - 1)));
  S->n_steps = step + 1;
  S->az[p ^ 1][0] = azn0;
  S->az[p ^ 1][1] = azn1;
}

// Active carriers of a slot at chunk step k.
__device__ __forceinline__ void active_counts(const StepArgs& a, const SlotDev* S, int slot, int k,
                                              int& nah, int& nae) {
  nah = S->act_h;
  nae = S->act_e;
  for (int kk = 0; kk < k; ++kk) {
    nah -= a.ret[((int64_t)kk * a.S + slot) * 2 + 0];
    nae -= a.ret[((int64_t)kk * a.S + slot) * 2 + 1];
  }
}

// ---------------------------------------------------------------------------
// The step kernel.
// ---------------------------------------------------------------------------
// MODE 0: scalar FP32 pair loop; 1: packed over pairs of i's; 2: packed over
// pairs of sources (struct-of-arrays copy of each chunk in shared memory).
// IND: 0 records no induced charge (none of that code is compiled in), 1 the
// whole collecting surface, 2 also the pixels of the 3 x 3 window.
template <int NT, int R, int MODE, int JU, int MINB, int IND>
__global__ void __launch_bounds__(NT, MINB) step_kernel(StepArgs a, int k0, int nk) {
  constexpr int TI = NT * R;
  static_assert(MODE != 1 || R % 2 == 0, "packed-i variants pair i's two by two");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  float4* stage = reinterpret_cast<float4*>(smem_raw);  // [2][kChunkJ]
  // MODE 2: struct-of-arrays copy of the current chunk, padded to a multiple of 4
  float* soa_x = reinterpret_cast<float*>(smem_raw + 2 * kChunkJ * sizeof(float4));
  float* soa_y = soa_x + kChunkJ;
  float* soa_z = soa_y + kChunkJ;
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int s_skip, s_last, s_nah, s_nae, s_step;
  __shared__ double s_azn[2];
  __shared__ float s_off;

  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_fence_init();
  }
  __syncthreads();
  uint32_t uses[2] = {0u, 0u};
  bool failed = false;
  const float eps2 = a.ph.f_eps2;
  unsigned long long t_start = 0, pairs_done = 0, n_units_done = 0;
  unsigned long long ns_pro = 0, ns_loop = 0, ns_epi = 0, t_mark = 0;
  auto now_ns = [&]() {
    unsigned long long t = 0;
    if (a.trace) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
  };
  if (a.trace && tid == 0) t_start = now_ns();
  // This CTA's share of the launch's pair work: a static equal-cost range of
  // one step, or pieces pulled from the queue, which lists the step's units
  // once for each of the nk steps k0 .. k0 + nk - 1 of the launch.
  __shared__ int s_u;
  const int n_u = a.cta_begin[gridDim.x];
  const int q_begin = a.dynamic ? 0 : a.cta_begin[blockIdx.x];
  const int q_end = a.dynamic ? n_u * nk : a.cta_begin[blockIdx.x + 1];
  int q = q_begin;
  for (;;) {
    if (a.dynamic) {
      if (tid == 0) s_u = atomicAdd(&a.unit_counter[k0], 1);
      __syncthreads();
      q = s_u;
    }
    if (q >= q_end) break;
    if (tid == 0) t_mark = now_ns();
    const int kq = a.dynamic ? q / n_u : 0;
    const int k = k0 + kq;
    const Unit U = a.units[a.dynamic ? q - kq * n_u : q];
    if (!a.dynamic) ++q;
#ifdef CTS_BOUNDS_CHECK
    if (!unit_in_arena(a, U) || k >= kMaxK || !slot_in_arena(a.A, a.slots + U.slot)) {
      if (tid == 0) atomicOr(a.err, kErrBounds);
      failed = true;
      break;
    }
#endif
    SlotDev* S = a.slots + U.slot;
    if (kq > 0) {
      // A later step of the launch starts once every tile of the slot has
      // been updated at the step before.  The pieces of that step sit earlier
      // in the queue and were taken by running CTAs, so the wait ends.
      bool ok = true;
      if (tid == 0)
        ok = wait_count_bounded(a.tiles_done + (int64_t)(k - 1) * a.S + U.slot, U.ntiles);
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(a.err, kErrTimeout);
        failed = true;
        break;
      }
    }
    const int spec = U.flags & kUnitElectrons;
    const int p = ((U.flags & kUnitOddStep ? 1 : 0) + k) & 1;
    const float4* __restrict__ shin = a.A.sh[p];
    const int nch_h = a.ph.repulsion ? (U.len_h + kChunkJ - 1) / kChunkJ : 0;
    const int nch = a.ph.repulsion ? nch_h + (U.len_e + kChunkJ - 1) / kChunkJ : 0;
    auto chunk_src = [&](int c, int& cnt) -> const float4* {
      if (c < nch_h) {
        cnt = min(kChunkJ, U.len_h - c * kChunkJ);
        return shin + U.hoff + (int64_t)c * kChunkJ;
      }
      const int ce = c - nch_h;
      cnt = min(kChunkJ, U.len_e - ce * kChunkJ);
      return shin + U.eoff + (int64_t)ce * kChunkJ;
    };
    // The descriptor carries every offset, so the first source copy and the
    // i loads go out before the slot's per-step scalars are known; a unit of
    // a finished slot only waits for its copy and is dropped.
    if (tid == 0 && nch > 0) {
      int cnt;
      const float4* src = chunk_src(0, cnt);
      tma_load_1d(stage, src, (uint32_t)cnt * 16u, &bar[0]);
    }
    float4 qi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int li = r * NT + tid;
      qi[r] = li < U.ni ? __ldcg(shin + U.ioff + li) : make_float4(kParked, kParked, kParked, 0.0f);
    }
    // Prologue, spread over warps so its latencies overlap: warp 0 sums the
    // slot's retire counters of the earlier steps of this chunk (one load per
    // lane), warps 1 and 2 predict the next frame anchor of each species.
    {
      const int warp = tid >> 5, lane = tid & 31;
      if (warp == 0) {
        int dh = 0, de = 0;
        for (int kk = lane; kk < k; kk += 32) {
          dh += __ldcg(a.ret + ((int64_t)kk * a.S + U.slot) * 2 + 0);
          de += __ldcg(a.ret + ((int64_t)kk * a.S + U.slot) * 2 + 1);
        }
        dh = __reduce_add_sync(0xffffffffu, dh);
        de = __reduce_add_sync(0xffffffffu, de);
        if (lane == 0) {
          const int nah = S->act_h - dh, nae = S->act_e - de;
          const int step = S->step0 + k;
          const bool plan_ok = (step & 1) == p;
          if (!plan_ok) atomicOr(a.err, kErrPlan);
          s_nah = nah;
          s_nae = nae;
          s_step = step;
          s_skip = !plan_ok || (!S->running) || nah <= 0 || (int64_t)step >= a.ph.max_steps;
        }
      } else if (warp <= 2 && lane == 0) {
        const int sp = warp - 1;
        s_azn[sp] = anchor_next(a.ph, sp, __ldcg(&S->az[p][sp]));
        if (sp == 1) s_off = (float)(__ldcg(&S->az[p][1]) - __ldcg(&S->az[p][0]));
      }
    }
    __syncthreads();
    // A finished slot runs no pairs: its pieces only let the copy issued above
    // land and take part in the tile's completion below.
    const bool skip = s_skip;
    if (skip && nch > 0) {
      const bool ok = mbar_wait_bounded(&bar[0], uses[0] & 1u);
      uses[0]++;
      if (__syncthreads_or(!ok)) {
        if (tid == 0) atomicOr(a.err, kErrTimeout);
        failed = true;
        break;
      }
    }
    const int nch_run = skip ? 0 : nch;
    if (!skip && tid == 0 && a.fused && (U.flags & kUnitDuty))
      slot_duties(a, S, s_step, s_step & 1, s_nah, s_nae, s_azn[0], s_azn[1]);
    const int step = s_step;
    if (!skip) {
      pairs_done += (unsigned long long)U.ni * (unsigned long long)(U.len_h + U.len_e);
      n_units_done += 1;
    }
    if (tid == 0 && a.trace) {
      const unsigned long long t = now_ns();
      ns_pro += t - t_mark;
      t_mark = t;
    }

    float xi[R], yi[R], zi[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      xi[r] = qi[r].x;
      yi[r] = qi[r].y;
      zi[r] = qi[r].z + (spec ? s_off : 0.0f);  // hole frame
    }
    float sx[R], sy[R], sz[R], cx[R], cy[R], cz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) sx[r] = sy[r] = sz[r] = cx[r] = cy[r] = cz[r] = 0.0f;

    if (a.ph.repulsion) {
      for (int c = 0; c < nch_run; ++c) {
        const int st = c & 1;
        int cnt;
        chunk_src(c, cnt);
        if (tid == 0 && c + 1 < nch_run) {
          int cn;
          const float4* src = chunk_src(c + 1, cn);
          tma_load_1d(stage + (st ^ 1) * kChunkJ, src, (uint32_t)cn * 16u, &bar[st ^ 1]);
        }
        const bool ok = mbar_wait_bounded(&bar[st], uses[st] & 1u);
        uses[st]++;
        if (__syncthreads_or(!ok)) {
          // A copy never completed: record it, give the copy still in flight
          // a bounded wait, and stop this CTA.
          if (tid == 0) {
            atomicOr(a.err, kErrTimeout);
            if (c + 1 < nch_run) mbar_wait_bounded(&bar[st ^ 1], uses[st ^ 1] & 1u);
          }
          failed = true;
          break;
        }
        if (c == nch_h) {
          // electron sources: positions of the i's in the electron frame
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int li = r * NT + tid;
            const float zq = li < U.ni ? __ldcg(shin + U.ioff + li).z : kParked;
            zi[r] = spec ? zq : zq - s_off;
          }
        }
        const float4* sj = stage + st * kChunkJ;
        int cnt_eff = cnt;
        if constexpr (MODE == 2) {
          cnt_eff = (cnt + 3) & ~3;
          for (int e = tid; e < cnt_eff; e += NT) {
            const float4 q = e < cnt ? sj[e] : make_float4(kParked, kParked, kParked, 0.0f);
            soa_x[e] = q.x;
            soa_y[e] = q.y;
            soa_z[e] = q.z;
          }
          __syncthreads();
        }
        // plain FP32 sums over at most kFoldJ sources, then a Kahan fold
        for (int sub = 0; sub < cnt_eff; sub += kFoldJ) {
          const int m = min(kFoldJ, cnt_eff - sub);
          float tx[R], ty[R], tz[R];
          if constexpr (MODE == 2) {
            float2 qx2[R], qy2[R], qz2[R], ax2[R], ay2[R], az2[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
              qx2[r] = make_float2(xi[r], xi[r]);
              qy2[r] = make_float2(yi[r], yi[r]);
              qz2[r] = make_float2(zi[r], zi[r]);
              ax2[r] = ay2[r] = az2[r] = make_float2(0.0f, 0.0f);
            }
            // a tile whose carriers fill at most half of the i slots computes
            // only that half
            constexpr int RH = R > 1 ? R / 2 : 1;
            const bool half = R > 1 && U.ni <= RH * NT;
            if (c < nch_h) {
              if (half)
                pair_chunk_jpacked<R, RH, false>(soa_x + sub, soa_y + sub, soa_z + sub, m, qx2,
                                                 qy2, qz2, ax2, ay2, az2, eps2);
              else
                pair_chunk_jpacked<R, R, false>(soa_x + sub, soa_y + sub, soa_z + sub, m, qx2,
                                                qy2, qz2, ax2, ay2, az2, eps2);
            } else {
              if (half)
                pair_chunk_jpacked<R, RH, true>(soa_x + sub, soa_y + sub, soa_z + sub, m, qx2,
                                                qy2, qz2, ax2, ay2, az2, eps2);
              else
                pair_chunk_jpacked<R, R, true>(soa_x + sub, soa_y + sub, soa_z + sub, m, qx2,
                                               qy2, qz2, ax2, ay2, az2, eps2);
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
              tx[r] = ax2[r].x + ax2[r].y;
              ty[r] = ay2[r].x + ay2[r].y;
              tz[r] = az2[r].x + az2[r].y;
            }
          } else if constexpr (MODE == 1) {
            constexpr int P = R / 2;
            float2 px2[P], py2[P], pz2[P], ax2[P], ay2[P], az2[P];
#pragma unroll
            for (int q = 0; q < P; ++q) {
              px2[q] = make_float2(xi[2 * q], xi[2 * q + 1]);
              py2[q] = make_float2(yi[2 * q], yi[2 * q + 1]);
              pz2[q] = make_float2(zi[2 * q], zi[2 * q + 1]);
              ax2[q] = ay2[q] = az2[q] = make_float2(0.0f, 0.0f);
            }
            if (c < nch_h)
              pair_chunk_packed<P, false, JU>(sj + sub, m, px2, py2, pz2, ax2, ay2, az2,
                                                   eps2);
            else
              pair_chunk_packed<P, true, JU>(sj + sub, m, px2, py2, pz2, ax2, ay2, az2,
                                                  eps2);
#pragma unroll
            for (int q = 0; q < P; ++q) {
              tx[2 * q] = ax2[q].x; tx[2 * q + 1] = ax2[q].y;
              ty[2 * q] = ay2[q].x; ty[2 * q + 1] = ay2[q].y;
              tz[2 * q] = az2[q].x; tz[2 * q + 1] = az2[q].y;
            }
          } else {
#pragma unroll
            for (int r = 0; r < R; ++r) tx[r] = ty[r] = tz[r] = 0.0f;
            if (c < nch_h)
              pair_chunk<R, false, JU>(sj + sub, m, xi, yi, zi, tx, ty, tz, eps2);
            else
              pair_chunk<R, true, JU>(sj + sub, m, xi, yi, zi, tx, ty, tz, eps2);
          }
#pragma unroll
          for (int r = 0; r < R; ++r) {
            kahan_add(sx[r], cx[r], tx[r]);
            kahan_add(sy[r], cy[r], ty[r]);
            kahan_add(sz[r], cz[r], tz[r]);
          }
        }
        __syncthreads();
      }
      if (failed) break;
    }
    if (tid == 0 && a.trace) {
      const unsigned long long t = now_ns();
      ns_loop += t - t_mark;
      t_mark = t;
    }
    float vx[R], vy[R], vz[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
      vx[r] = sx[r] - cx[r];
      vy[r] = sy[r] - cy[r];
      vz[r] = sz[r] - cz[r];
    }

    // Completion of the tile: each piece writes its compensated sum, the
    // pair (S, c) of FP32 values whose difference S - c it stands for, to
    // its own slot; the CTA finishing the tile's last piece adds the pieces
    // in piece order (the same bits every run) by error-free FP32 sums, the
    // rounding errors and compensations gathered apart (Neumaier's form of
    // compensated summation), updates the tile's carriers and counts the
    // tile as done.  No FP64 arithmetic: it is slow on this GPU, and the
    // last piece's CTA is on the step's critical path.
    bool last = true;
    if (U.nsplit > 1) {
      float2* acc = reinterpret_cast<float2*>(a.partial + U.pbase);
      if (!skip) {
        float2* mine = acc + (int64_t)U.split * 3 * TI;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int li = r * NT + tid;
          if (li < U.ni) {
            mine[li] = make_float2(sx[r], cx[r]);
            mine[TI + li] = make_float2(sy[r], cy[r]);
            mine[2 * TI + li] = make_float2(sz[r], cz[r]);
          }
        }
      }
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        const int old = atomicAdd(&a.combine_count[U.iblock], 1);
        s_last = (old == U.nsplit - 1);
        if (s_last) a.combine_count[U.iblock] = 0;
      }
      __syncthreads();
      last = s_last;
      if (last && !skip) {
        __threadfence();
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int li = r * NT + tid;
          if (li < U.ni) {
            float hx = 0.0f, hy = 0.0f, hz = 0.0f, lx = 0.0f, ly = 0.0f, lz = 0.0f;
            for (int k = 0; k < U.nsplit; ++k) {
              const float2* pk = acc + (int64_t)k * 3 * TI;
              const float2 px = __ldcg(pk + li), py = __ldcg(pk + TI + li),
                           pz = __ldcg(pk + 2 * TI + li);
              float e;
              two_sum(hx, px.x, hx, e);
              lx = __fadd_rn(lx, __fsub_rn(e, px.y));
              two_sum(hy, py.x, hy, e);
              ly = __fadd_rn(ly, __fsub_rn(e, py.y));
              two_sum(hz, pz.x, hz, e);
              lz = __fadd_rn(lz, __fsub_rn(e, pz.y));
            }
            vx[r] = __fadd_rn(hx, lx);
            vy[r] = __fadd_rn(hy, ly);
            vz[r] = __fadd_rn(hz, lz);
          }
        }
      }
    }

    if (last) {
      const float kc = a.ph.f_kc;
      if (skip) {
      } else if (a.fused) {
        if constexpr (IND > 0) {
          double q = 0.0;
          double qpx[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int li = r * NT + tid;
            if (li < U.ni)
              q += update_carrier<IND>(a, S, U.slot, spec, U.ioff + li, step, p, k, kc * vx[r],
                                       kc * vy[r], kc * vz[r], s_azn[spec], qpx);
          }
          add_induced(a, k, U.slot, q);
          if constexpr (IND == 2) add_induced_px(a, k, U.slot, qpx);
        } else {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            const int li = r * NT + tid;
            if (li < U.ni)
              update_carrier<0>(a, S, U.slot, spec, U.ioff + li, step, p, k, kc * vx[r],
                                kc * vy[r], kc * vz[r], s_azn[spec]);
          }
        }
      } else {
        const int64_t cap = a.A.capacity;
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const int li = r * NT + tid;
          if (li < U.ni) {
            const int64_t idx = U.ioff + li;
            a.field_out[idx] = kc * vx[r];
            a.field_out[cap + idx] = kc * vy[r];
            a.field_out[2 * cap + idx] = kc * vz[r];
          }
        }
      }
      // publish the tile's positions, states and counters before counting it
      __threadfence();
      __syncthreads();
      if (tid == 0) {
        asm volatile("fence.proxy.async.global;" ::: "memory");
        atomicAdd(a.tiles_done + (int64_t)k * a.S + U.slot, 1);
      }
    }
    if (tid == 0 && a.trace) ns_epi += now_ns() - t_mark;
    __syncthreads();
  }
  if (a.trace && tid == 0) {
    unsigned long long t_end = now_ns();
    unsigned smid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
    unsigned long long* t = a.trace + 8 * (size_t)blockIdx.x;
    t[0] = smid;
    t[1] = t_start;
    t[2] = t_end;
    t[3] = pairs_done;
    t[4] = n_units_done;
    t[5] = ns_pro;
    t[6] = ns_loop;
    t[7] = ns_epi;
  }
}

// ---------------------------------------------------------------------------
// The symmetric step kernel: every unordered pair of an event once per step,
// its term added to both carriers (Newton's third law), one warp per unit.
// ---------------------------------------------------------------------------
// A warp holds an I block (32 * RI carriers, i-slot r of lane l = carrier
// r * 32 + l, so tile u of the block is i-slots 2u and 2u + 1) as duplicated
// FP32 pairs, and walks the unit's J tiles.  A J tile sits in shared memory
// as 32 pairs (carrier m, carrier m + 32); in rotation step s lane l takes
// pair (l + s) mod 32, so its i's meet all 64 carriers of the tile in 32
// steps, and the J sums move with their pair from lane to lane by shuffle
// (home again after the 32nd).  Both the i's and the j's accumulate
// d w, d = r_i - r_j, w = (|d|^2 + eps^2)^(-3/2): the i's field is s_j times
// their sum, the j's field -s_i times theirs.
//
// Shared memory per warp (floats): the staged tile (3 x 32 float2), the J
// sums of the unit's tiles [kSymMaxRJ][3][64] and the I sums of the current
// block [3][kSymBlock].
constexpr int kSymStageFloats = 3 * 64;
constexpr int kSymWarpFloats = kSymStageFloats + kSymMaxRJ * kSymPartFloats + 3 * kSymBlock;

// The pairs of one (block, tile) combination.  QD = kSymTpb: every i-slot
// pairs with the tile both ways.  Otherwise tile t = r / 2 of the block pairs
// both ways if t < qd, with itself (i sums only: every ordered pair of the
// tile once) if t == qd, not at all if t > qd or t >= vt (tiles past the
// species' end); QD in [0, kSymTpb) fixes qd at compile time (a full block's
// own tiles), QD = -1 takes qd and vt at run time.  UNR rotation steps per
// loop iteration.
template <int RI, int QD, int UNR>
__device__ __forceinline__ void sym_tile_pairs(const float2* __restrict__ sx,
                                               const float2* __restrict__ sy,
                                               const float2* __restrict__ sz, int lane,
                                               const float2 (&xi)[RI], const float2 (&yi)[RI],
                                               const float2 (&zi)[RI], float2 (&aix)[RI],
                                               float2 (&aiy)[RI], float2 (&aiz)[RI], float2& ajx,
                                               float2& ajy, float2& ajz, float eps2s, int qd_rt,
                                               int vt_rt) {
  const float2 m1 = make_float2(-1.0f, -1.0f);
  const float2 eps2 = make_float2(eps2s, eps2s);
  const int src = (lane + 1) & 31;
  const int qd = QD >= 0 ? QD : qd_rt;
  const int vt = QD >= 0 ? kSymTpb : vt_rt;
#pragma unroll UNR
  for (int s = 0; s < 32; ++s) {
    const int jj = (lane + s) & 31;
    const float2 xj = sx[jj], yj = sy[jj], zj = sz[jj];
#pragma unroll
    for (int r = 0; r < RI; ++r) {
      const int t = r >> 1;
      if (t >= vt || t > qd) continue;
      const float2 dx = __ffma2_rn(xj, m1, xi[r]);
      const float2 dy = __ffma2_rn(yj, m1, yi[r]);
      const float2 dz = __ffma2_rn(zj, m1, zi[r]);
      float2 r2 = __ffma2_rn(dz, dz, eps2);
      r2 = __ffma2_rn(dy, dy, r2);
      r2 = __ffma2_rn(dx, dx, r2);
      const float2 rs = make_float2(rsqrt_approx(r2.x), rsqrt_approx(r2.y));
      const float2 w = __fmul2_rn(__fmul2_rn(rs, rs), rs);
      aix[r] = __ffma2_rn(dx, w, aix[r]);
      aiy[r] = __ffma2_rn(dy, w, aiy[r]);
      aiz[r] = __ffma2_rn(dz, w, aiz[r]);
      if (t < qd) {
        ajx = __ffma2_rn(dx, w, ajx);
        ajy = __ffma2_rn(dy, w, ajy);
        ajz = __ffma2_rn(dz, w, ajz);
      }
    }
    ajx.x = __shfl_sync(0xffffffffu, ajx.x, src);
    ajx.y = __shfl_sync(0xffffffffu, ajx.y, src);
    ajy.x = __shfl_sync(0xffffffffu, ajy.x, src);
    ajy.y = __shfl_sync(0xffffffffu, ajy.y, src);
    ajz.x = __shfl_sync(0xffffffffu, ajz.x, src);
    ajz.y = __shfl_sync(0xffffffffu, ajz.y, src);
  }
}

// Adds the i sums held in registers to the block's sums in shared memory and
// clears them (every kSymFold tiles: at most 128 terms per register half).
template <int RI>
__device__ __forceinline__ void sym_fold_i(float* iacc, int lane, float2 (&aix)[RI],
                                           float2 (&aiy)[RI], float2 (&aiz)[RI]) {
#pragma unroll
  for (int r = 0; r < RI; ++r) {
    const int c = r * 32 + lane;
    iacc[c] += aix[r].x + aix[r].y;
    iacc[kSymBlock + c] += aiy[r].x + aiy[r].y;
    iacc[2 * kSymBlock + c] += aiz[r].x + aiz[r].y;
    aix[r] = aiy[r] = aiz[r] = make_float2(0.0f, 0.0f);
  }
}

// The values of step k for a slot, computed by the unit itself at the first
// step of a launch (the same inputs give every unit the same bits).
__device__ SymStep sym_first_record(const StepArgs& a, const SymUnit& U, SlotDev* S, int k,
                                    int lane) {
  int dh = 0, de = 0;
  for (int kk = lane; kk < k; kk += 32) {
    dh += __ldcg(a.ret + ((int64_t)kk * a.S + U.slot) * 2 + 0);
    de += __ldcg(a.ret + ((int64_t)kk * a.S + U.slot) * 2 + 1);
  }
  dh = __reduce_add_sync(0xffffffffu, dh);
  de = __reduce_add_sync(0xffffffffu, de);
  SymStep R{};
  R.nah = __ldcg(&S->act_h) - dh;
  R.nae = __ldcg(&S->act_e) - de;
  R.step = __ldcg(&S->step0) + k;
  const int p = R.step & 1;
  const bool plan_ok = ((((U.flags & kSymOddStep) ? 1 : 0) + k) & 1) == p;
  if (!plan_ok && lane == 0) atomicOr(a.err, kErrPlan);
  R.skip = !plan_ok || !__ldcg(&S->running) || R.nah <= 0 || (int64_t)R.step >= a.ph.max_steps;
  if (!R.skip) {
    double z0 = 0.0, z1 = 0.0;
    if (lane == 0) {
      const double az0 = __ldcg(&S->az[p][0]), az1 = __ldcg(&S->az[p][1]);
      R.s_off = (float)(az1 - az0);
      z0 = anchor_next(a.ph, 0, az0);
      z1 = anchor_next(a.ph, 1, az1);
    }
    R.s_off = __shfl_sync(0xffffffffu, R.s_off, 0);
    R.azn[0] = __shfl_sync(0xffffffffu, z0, 0);
    R.azn[1] = __shfl_sync(0xffffffffu, z1, 0);
  }
  return R;
}

// Marks steps k .. k_end - 1 of a finished slot as skipped (idempotent).
__device__ void sym_skip_from(const StepArgs& a, int slot, int k, int k_end, const SymStep& R) {
  for (int kk = k; kk < k_end; ++kk) {
    SymStep N = R;
    N.skip = 1;
    a.sym.rec[(int64_t)kk * a.S + slot] = N;
    __threadfence();
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a.sym.ready + (int64_t)kk * a.S + slot),
                 "r"(1)
                 : "memory");
  }
}

// Written by the warp that finished the last tile of step k (lane 0): the
// slot's values for step k + 1, its per-step bookkeeping, and the flag the
// units of step k + 1 wait for.
__device__ void sym_next_record(const StepArgs& a, SlotDev* S, int slot, const SymStep& R, int k,
                                int k_end) {
  __threadfence();
  SymStep N{};
  N.nah = R.nah - __ldcg(a.ret + ((int64_t)k * a.S + slot) * 2 + 0);
  N.nae = R.nae - __ldcg(a.ret + ((int64_t)k * a.S + slot) * 2 + 1);
  N.step = R.step + 1;
  const int pn = N.step & 1;
  N.skip = !__ldcg(&S->running) || N.nah <= 0 || (int64_t)N.step >= a.ph.max_steps;
  if (!N.skip) {
    const double az0 = __ldcg(&S->az[pn][0]), az1 = __ldcg(&S->az[pn][1]);
    N.s_off = (float)(az1 - az0);
    N.azn[0] = anchor_next(a.ph, 0, az0);
    N.azn[1] = anchor_next(a.ph, 1, az1);
    if (a.fused) slot_duties(a, S, N.step, pn, N.nah, N.nae, N.azn[0], N.azn[1]);
    a.sym.rec[(int64_t)(k + 1) * a.S + slot] = N;
    __threadfence();
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(a.sym.ready +
                                                              (int64_t)(k + 1) * a.S + slot),
                 "r"(1)
                 : "memory");
  } else {
    sym_skip_from(a, slot, k + 1, k_end, N);
  }
}

// The field of one tile (the sum of its partials in list order, FP64) and its
// carriers' update, by one warp.  The slot's values of step k come from its
// step record; the warp that counts the slot's last tile of the step writes
// the record of the next step.
template <int IND>
__device__ void sym_tile_update(const StepArgs& a, int gt, int k, int k_end, int lane) {
  __threadfence();
  const SymTile T = a.sym.tiles[gt];
  const int slot = T.slot;
  SlotDev* S = a.slots + slot;
  SymStep R;
  {
    const SymStep* rp = a.sym.rec + (int64_t)k * a.S + slot;
    const double2 az = __ldcg(reinterpret_cast<const double2*>(rp));
    const int4 w0 = __ldcg(reinterpret_cast<const int4*>(rp) + 1);
    R.azn[0] = az.x;
    R.azn[1] = az.y;
    R.nah = w0.x;
    R.nae = w0.y;
    R.step = w0.z;
    R.skip = w0.w;
  }
  const float kc = a.ph.f_kc;
  const int p = R.step & 1;
  // The list, 32 entries at a time (one per lane); entry l goes to group
  // l mod 4, each group a compensated FP32 sum in list order, then the
  // groups in order: a fixed order (the same bits every run), four loads in
  // flight, and no FP64 (a slow pipe on this part).
  float sx[2][4], cx[2][4], sy[2][4], cy[2][4], sz[2][4], cz[2][4];
#pragma unroll
  for (int h = 0; h < 2; ++h)
#pragma unroll
    for (int g = 0; g < 4; ++g) sx[h][g] = cx[h][g] = sy[h][g] = cy[h][g] = sz[h][g] = cz[h][g] = 0.0f;
  for (int l0 = 0; l0 < T.lcnt; l0 += 32) {
    const int nl = min(32, T.lcnt - l0);
    const int mine = lane < nl ? __ldg(a.sym.lists + T.lptr + l0 + lane) : -1;
    for (int l = 0; l < nl; l += 4) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        const int idx = __shfl_sync(0xffffffffu, mine, (l + g) & 31);
        if (l + g < nl) {
          const float* src = a.sym.part + (int64_t)idx * kSymPartFloats;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            kahan_add(sx[h][g], cx[h][g], __ldcg(src + c));
            kahan_add(sy[h][g], cy[h][g], __ldcg(src + kSymTile + c));
            kahan_add(sz[h][g], cz[h][g], __ldcg(src + 2 * kSymTile + c));
          }
        }
      }
    }
  }
  float fx[2], fy[2], fz[2];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    float tx = 0.0f, ux = 0.0f, ty = 0.0f, uy = 0.0f, tz = 0.0f, uz = 0.0f;
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      kahan_add(tx, ux, sx[h][g] - cx[h][g]);
      kahan_add(ty, uy, sy[h][g] - cy[h][g]);
      kahan_add(tz, uz, sz[h][g] - cz[h][g]);
    }
    fx[h] = tx - ux;
    fy[h] = ty - uy;
    fz[h] = tz - uz;
  }
  [[maybe_unused]] double q = 0.0;
  [[maybe_unused]] double qpx[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int c = lane + 32 * h;
    if (c < T.n) {
      const float Ex = kc * fx[h], Ey = kc * fy[h], Ez = kc * fz[h];
      const int64_t idx = T.off + c;
      if (a.fused) {
        if constexpr (IND > 0)
          q += update_carrier<IND>(a, S, slot, T.spec, idx, R.step, p, k, Ex, Ey, Ez,
                                   R.azn[T.spec], qpx);
        else
          update_carrier<0>(a, S, slot, T.spec, idx, R.step, p, k, Ex, Ey, Ez, R.azn[T.spec]);
      } else {
        const int64_t cap = a.A.capacity;
        a.field_out[idx] = Ex;
        a.field_out[cap + idx] = Ey;
        a.field_out[2 * cap + idx] = Ez;
      }
    }
  }
  if constexpr (IND > 0) {
    if (a.fused) {
      add_induced(a, k, slot, q);
      if constexpr (IND == 2) add_induced_px(a, k, slot, qpx);
    }
  }
  if (lane == 0) a.sym.tile_ctr[gt] = 0;
  // publish the tile's positions, states and counters before counting it
  __threadfence();
  __syncwarp();
  if (lane == 0) {
    const int old = atomicAdd(a.tiles_done + (int64_t)k * a.S + slot, 1);
    if (old + 1 == T.ntiles && k + 1 < k_end) sym_next_record(a, S, slot, R, k, k_end);
  }
  __syncwarp();
}

// Debug trace of the symmetric kernel (a.trace: [0] records written, [1]
// capacity, records of 8 words from [8]): SM, time pulled, time done, queue
// position, kind (0 pair, 1 update), ns waiting, ns working, warp.
__device__ __forceinline__ unsigned long long sym_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ void sym_trace(const StepArgs& a, int qi, int kind, unsigned long long t0,
                          unsigned long long t1, unsigned long long t2) {
  const unsigned long long r = atomicAdd(a.trace, 1ull);
  if (r >= a.trace[1]) return;
  unsigned smid;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(smid));
  unsigned long long* o = a.trace + 8 + 8 * r;
  o[0] = smid;
  o[1] = t0;
  o[2] = t2;
  o[3] = (unsigned long long)qi;
  o[4] = (unsigned long long)kind;
  o[5] = t1 - t0;
  o[6] = t2 - t1;
  o[7] = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
}

template <int RI, int NT, int IND>
__global__ void __launch_bounds__(NT, 1) sym_kernel(StepArgs a, int k0, int nk) {
  static_assert(RI == kSymRI, "the planner's block is 32 * kSymRI carriers");
  static_assert(kSymTpb == 4, "the block's own tiles are specialised for four tiles");
  // rotation steps per loop iteration: two for 12 warps per SM (measured on
  // the 20 keV batch: 1.2 % faster than one), one for 8 (5 % slower with two)
  constexpr int kUnr = NT > 256 ? 2 : 1;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* wsm = reinterpret_cast<float*>(smem_raw) + (size_t)warp * kSymWarpFloats;
  float2* sx = reinterpret_cast<float2*>(wsm);
  float2* sy = sx + 32;
  float2* sz = sy + 32;
  float* jacc = wsm + kSymStageFloats;
  float* iacc = jacc + kSymMaxRJ * kSymPartFloats;
  const float eps2 = a.ph.f_eps2;
  const int n_u = __ldcg(a.sym.n_units);
  const int k_end = k0 + nk;
  // warps start pulling units in order of their index within the CTA, so
  // that the first units of a launch spread over every SM
  if (lane == 0 && warp > 0) {
    const unsigned long long t0 = sym_now();
    while (sym_now() - t0 < 400ull * (unsigned long long)warp) {
    }
  }
  __syncwarp();
  for (;;) {
    int qi = 0;
    if (lane == 0) qi = atomicAdd(&a.unit_counter[k0], 1);
    qi = __shfl_sync(0xffffffffu, qi, 0);
    if (qi >= n_u * nk) break;
    const unsigned long long tr0 = (a.trace && lane == 0) ? sym_now() : 0ull;
    const int kq = qi / n_u, k = k0 + kq;
    const SymUnit U = a.sym.units[qi - kq * n_u];
#ifdef CTS_BOUNDS_CHECK
    {
      const int64_t cap = a.A.capacity;
      const bool upd = (U.flags & kSymUpdate) != 0;
      const bool bad =
          U.slot < 0 || U.slot >= a.S || k >= kMaxK || U.jt0 < 0 || U.jt1 < U.jt0 ||
          U.tJ < 0 || U.tJ + U.jt1 > a.sym.n_tiles ||
          (!upd && (U.ib0 < 0 || U.ib1 < U.ib0 || U.jt1 - U.jt0 > kSymMaxRJ || U.ni < 0 ||
                    U.nj < 0 || U.ibase < 0 || U.ibase + U.ni > cap || U.jbase < 0 ||
                    U.jbase + U.nj > cap || U.pI < 0 || U.pJ < 0 ||
                    (int64_t)U.pJ + (U.jt1 - U.jt0) > a.sym.n_part ||
                    (int64_t)U.pI + (int64_t)(U.ib1 - U.ib0) * kSymTpb > a.sym.n_part ||
                    U.tI < 0 || U.tI + U.ib1 * kSymTpb > a.sym.n_tiles + kSymTpb));
      if (bad) {
        if (lane == 0) atomicOr(a.err, kErrBounds);
        break;
      }
    }
#endif
    SlotDev* S = a.slots + U.slot;
    SymStep R;
    if (kq == 0) {
      R = sym_first_record(a, U, S, k, lane);
      if (R.skip) {
        if (lane == 0) sym_skip_from(a, U.slot, k + 1, k_end, R);
        continue;
      }
      // every unit of the slot writes the same record (its tile updates read it)
      if (lane == 0) a.sym.rec[(int64_t)k * a.S + U.slot] = R;
      if ((U.flags & kSymDuty) && a.fused && lane == 0)
        slot_duties(a, S, R.step, R.step & 1, R.nah, R.nae, R.azn[0], R.azn[1]);
    } else {
      // the slot's previous step is complete once its record is published;
      // the units it waits for sit earlier in the queue, so the wait ends
      bool ok = false;
      {
        unsigned long long t0 = 0, tn;
        if (lane == 0) asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
        for (;;) {
          int v = 0;
          if (lane == 0)
            asm volatile("ld.acquire.gpu.global.b32 %0, [%1];"
                         : "=r"(v)
                         : "l"(a.sym.ready + (int64_t)k * a.S + U.slot)
                         : "memory");
          if (__shfl_sync(0xffffffffu, v, 0)) {
            ok = true;
            break;
          }
          int late = 0;
          if (lane == 0) {
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(tn));
            late = tn - t0 > kCountWaitNs;
            __nanosleep(128);
          }
          if (__shfl_sync(0xffffffffu, late, 0)) break;
        }
      }
      if (!ok) {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        break;
      }
      const SymStep* rp = a.sym.rec + (int64_t)k * a.S + U.slot;
      const double2 az = __ldcg(reinterpret_cast<const double2*>(rp));
      const int4 w0 = __ldcg(reinterpret_cast<const int4*>(rp) + 1);
      const int4 w1 = __ldcg(reinterpret_cast<const int4*>(rp) + 2);
      R.azn[0] = az.x;
      R.azn[1] = az.y;
      R.nah = w0.x;
      R.nae = w0.y;
      R.step = w0.z;
      R.skip = w0.w;
      R.s_off = __int_as_float(w1.x);
      if (R.skip) continue;
    }
    if (U.flags & kSymUpdate) {
      // an update unit: each of its tiles once all of the tile's partials are
      // in (the pair units writing them sit earlier in the queue, so the
      // waits end)
      const unsigned long long tr1 = (a.trace && lane == 0) ? sym_now() : 0ull;
      bool ok = true;
      for (int t = U.jt0; t < U.jt1 && ok; ++t) {
        const int gt = U.tJ + t;
        if (lane == 0) ok = wait_count_bounded(a.sym.tile_ctr + gt, __ldg(&a.sym.tiles[gt].lcnt));
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) sym_tile_update<IND>(a, gt, k, k_end, lane);
      }
      if (!ok) {
        if (lane == 0) atomicOr(a.err, kErrTimeout);
        break;
      }
      if (a.trace && lane == 0) sym_trace(a, qi, 1, tr0, tr1, sym_now());
      continue;
    }
    const unsigned long long tr1 = (a.trace && lane == 0) ? sym_now() : 0ull;
    const int p = R.step & 1;
    const float4* __restrict__ sh = a.A.sh[p];
    const int sI = U.flags & kSymIElectrons ? 1 : 0;
    const int sJ = U.flags & kSymJElectrons ? 1 : 0;
    const bool same = sI == sJ;
    const float offI = sI ? R.s_off : 0.0f, offJ = sJ ? R.s_off : 0.0f;
    const int nti = (U.ni + kSymTile - 1) / kSymTile;
    const int nj_t = U.jt1 - U.jt0;
    if (a.ph.repulsion) {
      for (int e = lane; e < nj_t * kSymPartFloats; e += 32) jacc[e] = 0.0f;
      for (int b = U.ib0; b < U.ib1; ++b) {
        const int bt0 = b * kSymTpb;
        const int vt = min(kSymTpb, nti - bt0);
        float2 xi[RI], yi[RI], zi[RI], aix[RI], aiy[RI], aiz[RI];
#pragma unroll
        for (int r = 0; r < RI; ++r) {
          const int ii = b * kSymBlock + r * 32 + lane;
          const float4 q =
              ii < U.ni ? __ldcg(sh + U.ibase + ii) : make_float4(kParked, kParked, kParked, 0.0f);
          xi[r] = make_float2(q.x, q.x);
          yi[r] = make_float2(q.y, q.y);
          const float z = q.z + offI;
          zi[r] = make_float2(z, z);
          aix[r] = aiy[r] = aiz[r] = make_float2(0.0f, 0.0f);
        }
        for (int e = lane; e < 3 * kSymBlock; e += 32) iacc[e] = 0.0f;
        const int g_first = same ? max(U.jt0, bt0) : U.jt0;
        // the first tile's positions; later ones are fetched one tile ahead
        float4 p0 = make_float4(kParked, kParked, kParked, 0.0f), p1 = p0;
        if (g_first < U.jt1) {
          const int j0 = g_first * kSymTile + lane;
          if (j0 < U.nj) p0 = __ldcg(sh + U.jbase + j0);
          if (j0 + 32 < U.nj) p1 = __ldcg(sh + U.jbase + j0 + 32);
        }
        int nf = 0;
        for (int g = g_first; g < U.jt1; ++g) {
          __syncwarp();
          sx[lane] = make_float2(p0.x, p1.x);
          sy[lane] = make_float2(p0.y, p1.y);
          sz[lane] = make_float2(p0.z + offJ, p1.z + offJ);
          __syncwarp();
          if (g + 1 < U.jt1) {
            const int j0 = (g + 1) * kSymTile + lane;
            p0 = j0 < U.nj ? __ldcg(sh + U.jbase + j0) : make_float4(kParked, kParked, kParked, 0.0f);
            p1 = j0 + 32 < U.nj ? __ldcg(sh + U.jbase + j0 + 32)
                                : make_float4(kParked, kParked, kParked, 0.0f);
          }
          float2 ajx = make_float2(0.0f, 0.0f), ajy = ajx, ajz = ajx;
          const int qd = same ? g - bt0 : kSymTpb;
#define CTS_SYM_PAIRS(QD)                                                                  \
  sym_tile_pairs<RI, QD, kUnr>(sx, sy, sz, lane, xi, yi, zi, aix, aiy, aiz, ajx, ajy, ajz, \
                               eps2, min(qd, kSymTpb), vt)
          if (vt < kSymTpb) CTS_SYM_PAIRS(-1);
          else if (qd >= kSymTpb) CTS_SYM_PAIRS(kSymTpb);
          else if (qd == 0) CTS_SYM_PAIRS(0);
          else if (qd == 1) CTS_SYM_PAIRS(1);
          else if (qd == 2) CTS_SYM_PAIRS(2);
          else CTS_SYM_PAIRS(3);
#undef CTS_SYM_PAIRS
          float* jt = jacc + (g - U.jt0) * kSymPartFloats;
          jt[lane] += ajx.x;
          jt[32 + lane] += ajx.y;
          jt[kSymTile + lane] += ajy.x;
          jt[kSymTile + 32 + lane] += ajy.y;
          jt[2 * kSymTile + lane] += ajz.x;
          jt[2 * kSymTile + 32 + lane] += ajz.y;
          if (++nf == kSymFold) {
            sym_fold_i<RI>(iacc, lane, aix, aiy, aiz);
            nf = 0;
          }
        }
        if (nf) sym_fold_i<RI>(iacc, lane, aix, aiy, aiz);
        __syncwarp();
        // the block's i fields: s_j times the sums
        const float sgn = sJ ? -1.0f : 1.0f;
        for (int u = 0; u < vt; ++u) {
          float* dst = a.sym.part + (int64_t)(U.pI + (b - U.ib0) * kSymTpb + u) * kSymPartFloats;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            dst[c * kSymTile + lane] = sgn * iacc[c * kSymBlock + u * kSymTile + lane];
            dst[c * kSymTile + 32 + lane] = sgn * iacc[c * kSymBlock + u * kSymTile + 32 + lane];
          }
        }
      }
      __syncwarp();
      // the tiles' j fields: -s_i times the sums
      const float sgn = sI ? 1.0f : -1.0f;
      for (int t = 0; t < nj_t; ++t) {
        float* dst = a.sym.part + (int64_t)(U.pJ + t) * kSymPartFloats;
        for (int e = lane; e < kSymPartFloats; e += 32) dst[e] = sgn * jacc[t * kSymPartFloats + e];
      }
    } else {
      // no repulsion: zero fields (the partials still complete their tiles)
      for (int b = U.ib0; b < U.ib1; ++b) {
        const int vt = min(kSymTpb, nti - b * kSymTpb);
        for (int u = 0; u < vt; ++u) {
          float* dst = a.sym.part + (int64_t)(U.pI + (b - U.ib0) * kSymTpb + u) * kSymPartFloats;
          for (int e = lane; e < kSymPartFloats; e += 32) dst[e] = 0.0f;
        }
      }
      for (int t = 0; t < nj_t; ++t) {
        float* dst = a.sym.part + (int64_t)(U.pJ + t) * kSymPartFloats;
        for (int e = lane; e < kSymPartFloats; e += 32) dst[e] = 0.0f;
      }
    }
    // the unit's partials are in: count them for their tiles' update units
    __threadfence();
    __syncwarp();
    {
      const int nI = min(U.ib1 * kSymTpb, nti) - U.ib0 * kSymTpb;
      const int ntot = nI + nj_t;
      for (int e = lane; e < ntot; e += 32) {
        const int gt = e < nI ? U.tI + U.ib0 * kSymTpb + e : U.tJ + U.jt0 + (e - nI);
        atomicAdd(a.sym.tile_ctr + gt, 1);
      }
    }
    if (a.trace && lane == 0) sym_trace(a, qi, 0, tr0, tr1, sym_now());
  }
}

// Update alone: reads the field written by a FIELD_ONLY step launch.
// PX: the instantiation that records the 3 x 3 window's pixels too.
template <bool PX>
__global__ void update_kernel(StepArgs a, int k, const int32_t* slot_list, int n_slots) {
  for (int q = 0; q < n_slots; ++q) {
    const int slot = slot_list[q];
    SlotDev* S = a.slots + slot;
    int nah, nae;
    active_counts(a, S, slot, k, nah, nae);
    const int step = S->step0 + k;
    if (!S->running || nah <= 0 || (int64_t)step >= a.ph.max_steps) continue;
    const int p = step & 1;
    const double azn0 = anchor_next(a.ph, 0, S->az[p][0]);
    const double azn1 = anchor_next(a.ph, 1, S->az[p][1]);
    if (blockIdx.x == 0 && threadIdx.x == 0) slot_duties(a, S, step, p, nah, nae, azn0, azn1);
    const int n = S->n_h + S->n_e;
    const int64_t cap = a.A.capacity;
    double qi = 0.0;
    double qpx[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
      const int spec = t < S->n_h ? 0 : 1;
      const int64_t idx = S->base + (spec ? S->cap_h + (t - S->n_h) : t);
      qi += update_carrier<PX ? 2 : 1>(a, S, slot, spec, idx, step, p, k, a.field_out[idx],
                                       a.field_out[cap + idx], a.field_out[2 * cap + idx],
                                       spec ? azn1 : azn0, qpx);
    }
    add_induced(a, k, slot, qi);
    if constexpr (PX) add_induced_px(a, k, slot, qpx);
  }
}

// ---------------------------------------------------------------------------
// Block-wide order-preserving compaction of one species range (in place).
// ---------------------------------------------------------------------------
constexpr int kAuxThreads = 256;

__device__ int block_exclusive_scan(int v, int* warp_sums, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned m = __ballot_sync(0xffffffffu, v != 0);
  const int within = __popc(m & ((1u << lane) - 1u));
  if (lane == 0) warp_sums[warp] = __popc(m);
  __syncthreads();
  if (threadIdx.x == 0) {
    int acc = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      const int t = warp_sums[w];
      warp_sums[w] = acc;
      acc += t;
    }
    *total = acc;
  }
  __syncthreads();
  return warp_sums[warp] + within;
}

__device__ int compact_range(const Arena& A, int64_t start, int n, int64_t rbase, int p,
                             int* warp_sums, int* total) {
  int out = 0;
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int i = c0 + threadIdx.x;
    int keep = 0, id = 0;
    double x = 0, y = 0, z = 0;
    float4 s = make_float4(0, 0, 0, 0);
    if (i < n) {
      id = A.cid[start + i];
      keep = (A.cstate[rbase + id] & kStateMask) == kStateActive;
      if (keep) {
        x = A.px[start + i];
        y = A.py[start + i];
        z = A.pz[start + i];
        s = A.sh[p][start + i];
      }
    }
    const int pos = block_exclusive_scan(keep, warp_sums, total);
    const int tot = *total;
    __syncthreads();
    if (keep) {
      const int64_t d = start + out + pos;
      A.px[d] = x;
      A.py[d] = y;
      A.pz[d] = z;
      A.cid[d] = id;
      A.sh[p][d] = s;
    }
    out += tot;
    __syncthreads();
  }
  return out;
}

__global__ void __launch_bounds__(kAuxThreads) close_kernel(Phys ph, Arena A, SlotDev* slots,
                                                            const int32_t* ret, int S_count, int K,
                                                            SlotSummary* summary) {
  __shared__ int warp_sums[kAuxThreads / 32];
  __shared__ int total;
  const int slot = blockIdx.x;
  SlotDev* S = slots + slot;
  SlotSummary sm{};
  if (!S->running) {
    if (threadIdx.x == 0) summary[slot] = sm;
    return;
  }
#ifdef CTS_BOUNDS_CHECK
  if (!slot_in_arena(A, S) || S->n_h < 0 || S->n_h > S->cap_h || S->n_e < 0 ||
      S->n_e > S->cap_e) {
    // stop the slot without touching its arena range; the host sees the flag
    if (threadIdx.x == 0) {
      S->flags |= kErrBounds;
      S->running = 0;
      sm.done = 1;
      sm.status = -5;
      sm.flags = S->flags;
      summary[slot] = sm;
    }
    return;
  }
#endif
  int nah = S->act_h, nae = S->act_e;
  for (int kk = 0; kk < K; ++kk) {
    nah -= ret[((int64_t)kk * S_count + slot) * 2 + 0];
    nae -= ret[((int64_t)kk * S_count + slot) * 2 + 1];
  }
  int done = 0, status = 0;
  if (S->flags & kErrNumeric) {
    done = 1;
    status = -7;
  } else if (nah <= 0) {
    done = 1;
  } else if ((int64_t)S->step0 + K >= ph.max_steps) {
    done = 1;
    status = -6;
  }
  int n_h = S->n_h, n_e = S->n_e;
  if (!done) {
    const int p = (S->step0 + K) & 1;
    if (nah != n_h) n_h = compact_range(A, S->base, n_h, S->base, p, warp_sums, &total);
    if (nae != n_e) n_e = compact_range(A, S->base + S->cap_h, n_e, S->base, p, warp_sums, &total);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    if (!done) {
      S->n_h = n_h;
      S->n_e = n_e;
      S->act_h = nah;
      S->act_e = nae;
      S->step0 += K;
    } else {
      S->running = 0;
      S->status = status;
      S->act_h = nah;
      S->act_e = nae;
    }
    sm.running = !done;
    sm.done = done;
    sm.status = status;
    sm.n_steps = S->n_steps;
    sm.n_h = n_h;
    sm.n_e = n_e;
    sm.act_h = nah;
    sm.act_e = nae;
    sm.flags = S->flags;
    sm.interactions = S->interactions;
    summary[slot] = sm;
  }
}

// ---------------------------------------------------------------------------
// Initial cloud (Algorithm 1, first step; Eq. 2), one CTA per new slot.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kAuxThreads) init_kernel(Phys ph, Arena A, SlotDev* slots,
                                                           const int32_t* slot_list,
                                                           const ExplicitRec* ex) {
  __shared__ int ret_h, ret_e;
  SlotDev* S = slots + slot_list[blockIdx.x];
  if (threadIdx.x == 0) {
    ret_h = 0;
    ret_e = 0;
  }
  __syncthreads();
  const int np = S->n_pairs;
  const double H = ph.H;
  const double sigma = S->sigma_um >= 0.0 ? S->sigma_um : 0.0044 * pow(S->energy_keV, 1.75);
  const double z_entry = H - S->depth_um;
  const double th = S->theta_deg * (M_PI / 180.0), phi = S->phi_deg * (M_PI / 180.0);
  const double ux = sin(th) * cos(phi), uy = sin(th) * sin(phi), uz = -cos(th);
  const double axv = cos(th) * cos(phi), ayv = cos(th) * sin(phi), azv = sin(th);
  const double bxv = -sin(phi), byv = cos(phi);
  // frame anchor: the absorption point, or the midpoint of a track
  const double half = S->kind == 1 ? 0.5 * S->track_len_um : 0.0;
  const double ax0 = S->x0 + half * ux, ay0 = S->y0 + half * uy;
  const double az0 = fmin(fmax(S->kind == 1 ? H + half * uz : z_entry, 0.0), H);
  const int total_entries = S->cap_h + S->cap_e;
#ifdef CTS_BOUNDS_CHECK
  // the slot's range, the explicit records it reads, and every carrier id
  __shared__ int bad;
  if (threadIdx.x == 0)
    bad = !slot_in_arena(A, S) || S->n_pairs < 0 || S->n_pairs > S->cap_h ||
          (S->kind == 2 && (S->explicit_off < 0 || S->explicit_off + total_entries > A.capacity));
  __syncthreads();
  const int loop_end = bad ? 0 : total_entries;
#else
  const int loop_end = total_entries;
#endif

  for (int e = threadIdx.x; e < loop_end; e += blockDim.x) {
    const int spec = e < S->cap_h ? 0 : 1;
    const int64_t idx = S->base + e;
    double x, y, z;
    int id;
    if (S->kind == 2) {
      const ExplicitRec r = ex[S->explicit_off + e];
      x = r.x; y = r.y; z = r.z; id = r.cid;
    } else {
      const int pidx = spec ? e - S->cap_h : e;
      id = spec ? np + pidx : pidx;
      const double3 n = normals_d(stream_words(S->seed, S->event_id, 1u, (uint32_t)pidx, 0u));
      if (S->kind == 1) {
        const uint4 w = stream_words(S->seed, S->event_id, 1u, (uint32_t)pidx, 1u);
        const double s = uniform_d(w.x) * S->track_len_um;
        x = S->x0 + s * ux + sigma * (n.x * axv + n.y * bxv);
        y = S->y0 + s * uy + sigma * (n.x * ayv + n.y * byv);
        z = H + s * uz + sigma * (n.x * azv);
      } else {
        x = S->x0 + sigma * n.x;
        y = S->y0 + sigma * n.y;
        z = z_entry + sigma * n.z;
      }
    }
    const int64_t rid = S->base + id;
#ifdef CTS_BOUNDS_CHECK
    if (id < 0 || id >= total_entries) {
      atomicOr(&S->flags, kErrBounds);
      continue;
    }
#endif
    int state = kStateActive;
    if (spec == 0) {
      if (z <= 0.0) state = kStateCollected;
      else if (z > H) z = 2.0 * H - z;
    } else {
      if (z >= H) state = kStateExited;
      else if (z < 0.0) z = -z;
    }
    A.px[idx] = x;
    A.py[idx] = y;
    A.pz[idx] = z;
    A.cid[idx] = id;
    A.cstate[rid] = (int8_t)((spec ? kElectronBit : 0) | state);
    A.rstep[rid] = state == kStateActive ? -2 : -1;
    A.fx[rid] = state == kStateCollected ? x : __longlong_as_double(0x7ff8000000000000LL);
    A.fy[rid] = state == kStateCollected ? y : __longlong_as_double(0x7ff8000000000000LL);
    if (state != kStateActive) {
      atomicAdd(spec ? &ret_e : &ret_h, 1);
      A.sh[0][idx] = make_float4(kParked, kParked, kParked, 0.0f);
    } else {
      A.sh[0][idx] = make_float4((float)(x - ax0), (float)(y - ay0), (float)(z - az0), 0.0f);
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    S->ax = ax0;
    S->ay = ay0;
    S->az[0][0] = S->az[0][1] = az0;
    S->az[1][0] = S->az[1][1] = az0;
    S->n_h = S->cap_h;
    S->n_e = S->cap_e;
    S->act_h = S->cap_h - ret_h;
    S->act_e = S->cap_e - ret_e;
    S->step0 = 0;
    S->n_steps = 0;
#ifdef CTS_BOUNDS_CHECK
    S->flags = (bad || (S->flags & kErrBounds)) ? kErrBounds : 0;
#else
    S->flags = 0;
#endif
    S->status = 0;
    S->interactions = 0ull;
    S->running = 1;
  }
}

// ---------------------------------------------------------------------------
// Readout: pixel = floor(x / pitch + n/2) per axis (pixel_key), warp-aggregated
// counts.
// ---------------------------------------------------------------------------

// key >= 0: pixel; -1: outside; -2: nothing.  Lanes with equal keys add once.
__device__ __forceinline__ void warp_count(int key, int32_t* pix, int* outside) {
  const unsigned grp = __match_any_sync(0xffffffffu, key);
  const int leader = __ffs(grp) - 1;
  if ((int)(threadIdx.x & 31) == leader) {
    if (key >= 0) atomicAdd(pix + key, __popc(grp));
    else if (key == -1) atomicAdd(outside, __popc(grp));
  }
}

__global__ void __launch_bounds__(kAuxThreads) bin_kernel(Phys ph, Arena A, const SlotDev* slots,
                                                          const int32_t* slot_list,
                                                          int32_t* pixels, SlotReadout* readout) {
  __shared__ int outside, collected, lost;
  const int slot = slot_list[blockIdx.x];
  const SlotDev* S = slots + slot;
  const int npix = ph.grid_n * ph.grid_n;
  int32_t* pix = pixels + (int64_t)slot * npix;
  for (int t = threadIdx.x; t < npix; t += blockDim.x) pix[t] = 0;
  if (threadIdx.x == 0) outside = collected = lost = 0;
  __syncthreads();
#ifdef CTS_BOUNDS_CHECK
  const int n = slot_in_arena(A, S) ? S->n_total : 0;
#else
  const int n = S->n_total;
#endif
  const int n_round = (n + blockDim.x - 1) / blockDim.x * blockDim.x;
  for (int id = threadIdx.x; id < n_round; id += blockDim.x) {
    int key = -2;
    if (id < n) {
      const int8_t st = A.cstate[S->base + id];
      if ((st & kStateMask) == kStateCollected) {
        key = pixel_key(ph, A.fx[S->base + id], A.fy[S->base + id]);
        atomicAdd(&collected, 1);
      } else if ((st & kStateMask) == kStateActive && (st & kElectronBit)) {
        atomicAdd(&lost, 1);
      }
    }
    warp_count(key, pix, &outside);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    SlotReadout r{};
    r.n_collected = collected;
    r.n_outside = outside;
    r.n_lost = lost;
    readout[slot] = r;
  }
}

__global__ void bin_points_kernel(Phys ph, const double* x, const double* y, int64_t n,
                                  int32_t* pix, long long* outside_total) {
  __shared__ int outside;
  if (threadIdx.x == 0) outside = 0;
  __syncthreads();
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t n_round = (n + stride - 1) / stride * stride;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n_round; i += stride) {
    const int key = i < n ? pixel_key(ph, x[i], y[i]) : -2;
    warp_count(key, pix, &outside);
  }
  __syncthreads();
  if (threadIdx.x == 0)
    atomicAdd(reinterpret_cast<unsigned long long*>(outside_total), (unsigned long long)outside);
}

// ---------------------------------------------------------------------------
// Simplified spherical model (Sec. 2.2, Eq. 7), holes only.  One cluster of
// C CTAs (C = 1, 2 or 4, chosen by the host so that the resident events fill
// the SMs) runs all K steps of a chunk for one event: an event's step needs
// only its own carriers.  CTA r of the cluster owns a contiguous range of the
// event's holes, whole groups of kSphGroup.  Per step:
//  1. the centre of the active holes in FP64: every group is summed in a
//     fixed order (lane l adds holes l, l + 32, ... of the group, then a lane
//     tree), the group sums likewise (group g by lane g mod 32, then a lane
//     tree; the other CTAs' group sums read through distributed shared
//     memory), so the centre does not depend on C;
//  2. the keys of the own holes: the squared distance's FP64 bit pattern
//     (non-negative doubles order like their bits), written to the arena's
//     second FP32 shadow (8 bytes of each 16-byte entry); the FP32 offset
//     from the centre and the carrier id go to the first shadow.  The
//     spherical model uses neither shadow for anything else;
//  3. after a cluster barrier every CTA bins all keys of the event in shared
//     memory (bins of equal width in key space over the keys' range at the
//     previous step of the chunk, about logarithmic in r^2; keys outside go
//     to the end bins) and lists each bin's keys;
//  4. the enclosed count Q(<r) = the number of keys strictly below a hole's
//     key: the keys of lower bins (the bin's list start) plus the smaller
//     keys of its own bin; the field k_C Q (r - c) / r^3 and the fused
//     update of the own holes.
// A step whose fullest bin holds more than kSphBinMax keys (radii piled up
// at one value) ranks by a bitonic sort of all keys in every CTA instead: the
// first position of a key's run in sorted order.  Q is an exact count either
// way, so the results depend neither on the bins nor on C.  FP64 arithmetic
// is slow on this GPU, so a hole costs few FP64 operations per step: three
// adds for the centre, six for its key, three conversions for its offset,
// and the update's own.  The holes' states live in shared memory during a
// launch (read from the arena at its first step), so each pass issues all of
// a hole's global loads at once.
// ---------------------------------------------------------------------------
constexpr int kSphBins = 4096;
constexpr int kSphBinMax = 256;
constexpr int kSphGroup = 256;
constexpr int kSphGroups = kSphMax / kSphGroup;

__device__ __forceinline__ unsigned long long shfl_down_u64(unsigned long long v, int o) {
  return (unsigned long long)__shfl_down_sync(0xffffffffu, (long long)v, o);
}

// Bin of a key in the range [lo, lo + (kSphBins << shift)).
__device__ __forceinline__ int sph_bin(unsigned long long kv, unsigned long long lo, int shift) {
  if (kv <= lo) return 0;
  const unsigned long long b = (kv - lo) >> shift;
  return b >= (unsigned long long)kSphBins ? kSphBins - 1 : (int)b;
}

// The smallest shift with fewer than kSphBins bins over [lo, hi].
__device__ __forceinline__ int sph_shift(unsigned long long lo, unsigned long long hi) {
  if (hi <= lo) return 0;
  const int bits = 64 - __clzll((long long)(hi - lo));  // bit length of the span
  return bits > 12 ? bits - 12 : 0;
}

template <bool PX>
__global__ void __launch_bounds__(1024, 1) spherical_kernel(StepArgs a, int k0, int nk) {
  namespace cg = cooperative_groups;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks(), rank = (int)cl.block_rank();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  unsigned long long* kb = reinterpret_cast<unsigned long long*>(smem_raw);  // [kSphMax]
  uint16_t* idx = reinterpret_cast<uint16_t*>(kb + kSphMax);                  // [kSphMax]
  int32_t* bstart = reinterpret_cast<int32_t*>(idx + kSphMax);                // [kSphBins]
  int32_t* bcount = bstart + kSphBins;                                         // [kSphBins]
  double* gsum = reinterpret_cast<double*>(bcount + kSphBins);                 // [kSphGroups][4]
  int8_t* act = reinterpret_cast<int8_t*>(gsum + 4 * kSphGroups);             // [kSphMax]
  __shared__ int32_t wsum[32];
  __shared__ int s_most;
  __shared__ int s_nah;
  __shared__ double s_c[3];
  __shared__ double s_azn;
  __shared__ unsigned long long s_rng[2];  // the keys' range: this step's, being found
  __shared__ unsigned long long s_lo;      // the bins' range
  __shared__ int s_shift;
  const int slot = blockIdx.x / C;
  if (slot >= a.S) return;
  SlotDev* S = a.slots + slot;
  if (!S->running) return;
  const int nh = S->n_h;
  if (nh <= 0 || nh > kSphMax) {
    if (nh > kSphMax && threadIdx.x == 0 && rank == 0) atomicOr(a.err, kErrPlan);
    return;
  }
#ifdef CTS_BOUNDS_CHECK
  if (!slot_in_arena(a.A, S) || nh > S->cap_h || k0 < 0 || k0 + nk > kMaxK) {
    if (threadIdx.x == 0 && rank == 0) atomicOr(a.err, kErrBounds);
    return;
  }
#endif
  // every CTA of the cluster passes this point (the tests above read the
  // same slot), so the cluster barriers below are uniform
  int p2 = 2;
  while (p2 < nh) p2 <<= 1;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int ng = (nh + kSphGroup - 1) / kSphGroup;  // groups of kSphGroup holes
  const int gpc = (ng + C - 1) / C;                   // groups per CTA
  const int g0 = min(ng, rank * gpc), g1 = min(ng, g0 + gpc);
  const int lo = g0 * kSphGroup, hi = min(nh, g1 * kSphGroup), m = hi - lo;  // own holes
  const unsigned long long kNone = ~0ull;
  const int64_t base = S->base;
  // per hole: FP32 offset and id (first shadow), key (second shadow)
  float4* __restrict__ off = a.A.sh[0];
  unsigned long long* __restrict__ kscr = reinterpret_cast<unsigned long long*>(a.A.sh[1]);
  const Phys& ph = a.ph;
  for (int t = lo + tid; t < hi; t += nt) act[t - lo] = __ldcg(a.A.cstate + base + a.A.cid[base + t]);
  if (tid == 0) {
    s_rng[0] = kNone;
    s_rng[1] = 0ull;
  }
  __syncthreads();
  for (int kq = 0; kq < nk; ++kq) {
    const int k = k0 + kq;
    const int step = S->step0 + k;
    const int p = step & 1;
    // 1. group sums of the own groups
    for (int g = g0 + warp; g < g1; g += nt >> 5) {
      double x = 0.0, y = 0.0, z = 0.0;
      int c = 0;
#pragma unroll
      for (int r = 0; r < kSphGroup / 32; ++r) {
        const int t = g * kSphGroup + r * 32 + lane;
        if (t < nh && (act[t - lo] & kStateMask) == kStateActive) {
          x += __ldcg(a.A.px + base + t);
          y += __ldcg(a.A.py + base + t);
          z += __ldcg(a.A.pz + base + t);
          ++c;
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
        z += __shfl_down_sync(0xffffffffu, z, o);
      }
      c = __reduce_add_sync(0xffffffffu, c);
      if (lane == 0) {
        gsum[4 * g + 0] = x;
        gsum[4 * g + 1] = y;
        gsum[4 * g + 2] = z;
        gsum[4 * g + 3] = (double)c;
      }
    }
    cl.sync();
    // 2. the centre from all groups of the cluster (the three divisions on
    // lanes 0, 1, 2 at once); the bins' range: the previous step's keys
    if (warp == 0) {
      double x = 0.0, y = 0.0, z = 0.0, c = 0.0;
      for (int g = lane; g < ng; g += 32) {
        const int r = g / gpc;
        const double* src = r == rank ? gsum : cl.map_shared_rank(gsum, r);
        x += src[4 * g + 0];
        y += src[4 * g + 1];
        z += src[4 * g + 2];
        c += src[4 * g + 3];
      }
      for (int o = 16; o > 0; o >>= 1) {
        x += __shfl_down_sync(0xffffffffu, x, o);
        y += __shfl_down_sync(0xffffffffu, y, o);
        z += __shfl_down_sync(0xffffffffu, z, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
      }
      x = __shfl_sync(0xffffffffu, x, 0);
      y = __shfl_sync(0xffffffffu, y, 0);
      z = __shfl_sync(0xffffffffu, z, 0);
      c = __shfl_sync(0xffffffffu, c, 0);
      if (lane < 3) s_c[lane] = (lane == 0 ? x : lane == 1 ? y : z) / c;
      if (lane == 0) {
        s_nah = (int)c;
        s_lo = s_rng[0];
        s_shift = sph_shift(s_rng[0], s_rng[1]);
        s_rng[0] = kNone;
        s_rng[1] = 0ull;
        s_most = 0;
      }
    }
    for (int b = tid; b < kSphBins; b += nt) bcount[b] = 0;
    __syncthreads();
    const int nah = s_nah;
    if (nah <= 0 || (int64_t)step >= ph.max_steps) break;
    const double sx = s_c[0], sy = s_c[1], sz = s_c[2];
    if (tid == 0) {
      const double azn = anchor_next(ph, 0, __ldcg(&S->az[p][0]));
      s_azn = azn;
      if (rank == 0) {
        atomicAdd(&S->interactions, (unsigned long long)nah);
        S->n_steps = step + 1;
        S->az[p ^ 1][0] = azn;
        S->az[p ^ 1][1] = azn;
      }
    }
    // keys of the own holes (retired holes: kNone) and their FP32 offsets
    for (int t = lo + tid; t < hi; t += nt) {
      unsigned long long kv = kNone;
      if ((act[t - lo] & kStateMask) == kStateActive) {
        const int64_t ai = base + t;
        const int id = a.A.cid[ai];
        const double dx = __ldcg(a.A.px + ai) - sx, dy = __ldcg(a.A.py + ai) - sy,
                     dz = __ldcg(a.A.pz + ai) - sz;
        kv = (unsigned long long)__double_as_longlong(dx * dx + dy * dy + dz * dz);
        off[ai] = make_float4((float)dx, (float)dy, (float)dz, __int_as_float(id));
      }
      kscr[2 * (base + t)] = kv;
    }
    cl.sync();
    // 3. all keys of the event: the bin counts and the keys' range (which
    // sets the next step's bins; at a chunk's first step, in a pass of its
    // own, this step's)
    {
      unsigned long long blo = s_lo;
      int shift = s_shift;
      if (kq == 0) {
        unsigned long long klo = kNone, khi = 0ull;
        for (int t = tid; t < nh; t += nt) {
          const unsigned long long kv = __ldcg(kscr + 2 * (base + t));
          if (kv != kNone) {
            klo = min(klo, kv);
            khi = max(khi, kv);
          }
        }
        for (int o = 16; o > 0; o >>= 1) {
          klo = min(klo, shfl_down_u64(klo, o));
          khi = max(khi, shfl_down_u64(khi, o));
        }
        if (lane == 0 && klo != kNone) {
          atomicMin(&s_rng[0], klo);
          atomicMax(&s_rng[1], khi);
        }
        __syncthreads();
        blo = s_rng[0];
        shift = sph_shift(s_rng[0], s_rng[1]);
        if (tid == 0) {
          s_lo = blo;
          s_shift = shift;
        }
      }
      unsigned long long klo = kNone, khi = 0ull;
      for (int t = tid; t < nh; t += nt) {
        const unsigned long long kv = __ldcg(kscr + 2 * (base + t));
        if (kv != kNone) {
          atomicAdd(&bcount[sph_bin(kv, blo, shift)], 1);
          klo = min(klo, kv);
          khi = max(khi, kv);
        }
      }
      if (kq > 0) {
        for (int o = 16; o > 0; o >>= 1) {
          klo = min(klo, shfl_down_u64(klo, o));
          khi = max(khi, shfl_down_u64(khi, o));
        }
        if (lane == 0 && klo != kNone) {
          atomicMin(&s_rng[0], klo);
          atomicMax(&s_rng[1], khi);
        }
      }
    }
    __syncthreads();
    const unsigned long long blo = s_lo;
    const int shift = s_shift;
    // exclusive scan of the bin counts (kSphBins / nt per thread) and the
    // fullest bin
    {
      constexpr int kPer = kSphBins / 1024;
      int local[kPer], acc = 0, most = 0;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        local[q] = bcount[tid * kPer + q];
        most = max(most, local[q]);
        acc += local[q];
      }
      int incl = acc;
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      most = __reduce_max_sync(0xffffffffu, most);
      if (lane == 31) wsum[warp] = incl;
      if (lane == 0) atomicMax(&s_most, most);
      __syncthreads();
      if (tid == 0) {
        int run = 0;
        for (int w = 0; w < (nt >> 5); ++w) {
          const int v = wsum[w];
          wsum[w] = run;
          run += v;
        }
      }
      __syncthreads();
      int bs = wsum[warp] + incl - acc;
#pragma unroll
      for (int q = 0; q < kPer; ++q) {
        bstart[tid * kPer + q] = bs;
        bs += local[q];
        bcount[tid * kPer + q] = 0;
      }
    }
    __syncthreads();
    const bool fallback = s_most > kSphBinMax;
    const float kcf = ph.f_kc;
    const double azn = s_azn;
    double qi = 0.0;
    double qpx[9] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0};
    if (!fallback) {
      // each bin's keys (the order within a bin does not matter: a hole
      // counts the smaller keys of its bin)
      for (int t = tid; t < nh; t += nt) {
        const unsigned long long kv = __ldcg(kscr + 2 * (base + t));
        if (kv != kNone) {
          const int b = sph_bin(kv, blo, shift);
          kb[bstart[b] + atomicAdd(&bcount[b], 1)] = kv;
        }
      }
      __syncthreads();
      // 4. field and update of the own active holes (key, offset, id and
      // position loads issued together)
      for (int t = tid; t < m; t += nt) {
        if ((act[t] & kStateMask) != kStateActive) continue;
        const int64_t ai = base + lo + t;
        const unsigned long long kt = __ldcg(kscr + 2 * ai);
        const float4 o = off[ai];
        const double x = __ldcg(a.A.px + ai), y = __ldcg(a.A.py + ai), z = __ldcg(a.A.pz + ai);
        float ex = 0.0f, ey = 0.0f, ez = 0.0f;
        int q = 0;
        if (ph.repulsion) {
          const int b = sph_bin(kt, blo, shift);
          const int s0 = bstart[b], s1 = s0 + bcount[b];
          q = s0;
          for (int u = s0; u < s1; ++u) q += kb[u] < kt;
        }
        if (q > 0) {
          // offsets and the enclosed count from FP64 positions, the field
          // itself in FP32 like the pairwise path
          const float rs = rsqrtf((float)__longlong_as_double((long long)kt));
          const float f = kcf * (float)q * rs * rs * rs;
          ex = f * o.x;
          ey = f * o.y;
          ez = f * o.z;
        }
        bool gone = false;
        qi += update_carrier_at<PX ? 2 : 1, false>(a, S, slot, 0, ai, __float_as_int(o.w), act[t],
                                                    x, y, z, step, p, k, ex, ey, ez, azn, qpx,
                                                    &gone);
        if (gone) act[t] = (int8_t)kStateCollected;
      }
    } else {
      // every CTA ranks all keys by a bitonic sort (padding and retired
      // holes sort last) and updates its own holes
      for (int t = tid; t < p2; t += nt) {
        kb[t] = t < nh ? __ldcg(kscr + 2 * (base + t)) : kNone;
        idx[t] = (uint16_t)t;
      }
      __syncthreads();
      for (int size = 2; size <= p2; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
          for (int t = tid; t < (p2 >> 1); t += nt) {
            const int l0 = 2 * t - (t & (stride - 1)), h0 = l0 + stride;
            const bool up = (l0 & size) == 0;
            const unsigned long long kl = kb[l0], kh = kb[h0];
            if ((kl > kh) == up) {
              kb[l0] = kh;
              kb[h0] = kl;
              const uint16_t il = idx[l0];
              idx[l0] = idx[h0];
              idx[h0] = il;
            }
          }
          __syncthreads();
        }
      for (int j = tid; j < p2; j += nt) {
        const int t = idx[j];
        const unsigned long long kt = kb[j];
        if (t < lo || t >= hi || kt == kNone) continue;
        const int64_t ai = base + t;
        const float4 o = off[ai];
        const double x = __ldcg(a.A.px + ai), y = __ldcg(a.A.py + ai), z = __ldcg(a.A.pz + ai);
        float ex = 0.0f, ey = 0.0f, ez = 0.0f;
        int q = 0;
        if (ph.repulsion) {
          q = j;
          while (q > 0 && kb[q - 1] == kt) --q;
        }
        if (q > 0) {
          const float rs = rsqrtf((float)__longlong_as_double((long long)kt));
          const float f = kcf * (float)q * rs * rs * rs;
          ex = f * o.x;
          ey = f * o.y;
          ez = f * o.z;
        }
        bool gone = false;
        qi += update_carrier_at<PX ? 2 : 1, false>(a, S, slot, 0, ai, __float_as_int(o.w),
                                                    act[t - lo], x, y, z, step, p, k, ex, ey, ez,
                                                    azn, qpx, &gone);
        if (gone) act[t - lo] = (int8_t)kStateCollected;
      }
    }
    add_induced(a, k, slot, qi);
    if constexpr (PX) add_induced_px(a, k, slot, qpx);
    __syncthreads();
  }
  // the other CTAs may still read this CTA's group sums
  cl.sync();
}

// ---------------------------------------------------------------------------
// Fast event generation (Sec. 4.2) from the generalised Gaussian model
// (Eq. 8): x and y of every carrier drawn independently as alpha G^(1/beta)
// with a random sign, G ~ Gamma(1/beta) = Gamma(1/beta + 1) U^beta, the
// Gamma(shape >= 1) variate by Marsaglia and Tsang's rejection method (ACM
// TOMS 26, 2000).  Attempt k of axis a draws from counter (carrier, 4k + 2a),
// the boost and the sign from (carrier, 256 + a), purpose 4.  FP32 arithmetic;
// one CTA per event bins its carriers in shared memory.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ggd_variate(uint64_t seed, uint64_t ev, uint32_t carrier,
                                             uint32_t axis, float alpha, float beta) {
  const float shape = 1.0f / beta;
  const float d = shape + 1.0f - 1.0f / 3.0f, c = rsqrtf(9.0f * d);
  float g = d;
  for (uint32_t k = 0; k < 64; ++k) {
    const uint4 w = stream_words(seed, ev, 4u, carrier, 4u * k + 2u * axis);
    const float z = sqrtf(-2.0f * logf(uniform_f(w.x))) * cospif(2.0f * uniform_f(w.y));
    const float v1 = fmaf(c, z, 1.0f);
    if (v1 <= 0.0f) continue;
    const float v = v1 * v1 * v1;
    if (logf(uniform_f(w.z)) < 0.5f * z * z + d - d * v + d * logf(v)) {
      g = d * v;
      break;
    }
  }
  const uint4 b = stream_words(seed, ev, 4u, carrier, 256u + axis);
  g *= powf(uniform_f(b.x), beta);
  const float m = alpha * powf(g, beta == 0.0f ? 1.0f : 1.0f / beta);
  return (b.y >> 31) ? -m : m;
}

__global__ void __launch_bounds__(256) generate_kernel(const GenEvent* __restrict__ evs,
                                                       double pitch_um, int grid_n,
                                                       int32_t* pixels,
                                                       unsigned long long* outside) {
  __shared__ int hist[kReadoutMaxGrid * kReadoutMaxGrid];
  __shared__ int out_count;
  const GenEvent e = evs[blockIdx.x];
  const int np = grid_n * grid_n;
  for (int p = threadIdx.x; p < np; p += blockDim.x) hist[p] = 0;
  if (threadIdx.x == 0) out_count = 0;
  __syncthreads();
  const float a = (float)e.alpha, be = (float)e.beta;
  const float inv_pitch = (float)(1.0 / pitch_um), half = 0.5f * (float)grid_n;
  int lost = 0;
  for (int c = threadIdx.x; c < e.n_pairs; c += blockDim.x) {
    const float x = (float)e.x0 + ggd_variate(e.seed, e.id, (uint32_t)c, 0u, a, be);
    const float y = (float)e.y0 + ggd_variate(e.seed, e.id, (uint32_t)c, 1u, a, be);
    const float fx = floorf(x * inv_pitch + half), fy = floorf(y * inv_pitch + half);
    if (fx < 0.0f || fy < 0.0f || fx >= (float)grid_n || fy >= (float)grid_n) {
      ++lost;
      continue;
    }
    atomicAdd(&hist[(int)fy * grid_n + (int)fx], 1);
  }
  if (lost) atomicAdd(&out_count, lost);
  __syncthreads();
  for (int p = threadIdx.x; p < np; p += blockDim.x)
    pixels[(int64_t)blockIdx.x * np + p] = hist[p];
  if (threadIdx.x == 0) outside[blockIdx.x] = (unsigned long long)out_count;
}

// ---------------------------------------------------------------------------
// Detector readout of pixel-count maps (Sec. 4.1 selection, Sec. 4.2 noise):
// one CTA per event.  Pixel energies with Gaussian noise from the event's
// stream (purpose 3, carrier = pixel), the centre at the largest pixel (first
// in row-major order on ties), the 3 x 3 cluster, the 7 x 7 pile-up veto and
// the cluster-energy window; accepted clusters add their on-grid pixels to
// the single-pixel spectrum.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) readout_kernel(ReadoutArgs r) {
  __shared__ double e[kReadoutMaxGrid * kReadoutMaxGrid];
  __shared__ double wv[8];
  __shared__ int wi[8];
  const int ev = blockIdx.x, n = r.grid_n, np = n * n;
  const int32_t* cnt = r.counts + (int64_t)ev * np;
  const uint64_t seed = r.seeds[ev], id = r.ids[ev];
  double best = -INFINITY;
  int bi = np;
  for (int p = threadIdx.x; p < np; p += blockDim.x) {
    double g = 0.0;
    if (r.noise_keV > 0.0) g = normals_d(stream_words(seed, id, 3u, (uint32_t)p, 0u)).x;
    const double v = (double)cnt[p] * r.ev_per_pair * 1e-3 + r.noise_keV * g;
    e[p] = v;
    if (r.pixel_keV) r.pixel_keV[(int64_t)ev * np + p] = v;
    if (v > best || (v == best && p < bi)) {
      best = v;
      bi = p;
    }
  }
  // (largest energy, smallest index) over the block
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, o);
    const int oi = __shfl_down_sync(0xffffffffu, bi, o);
    if (ov > best || (ov == best && oi < bi)) {
      best = ov;
      bi = oi;
    }
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) {
    wv[warp] = best;
    wi[warp] = bi;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
    if (wv[w] > best || (wv[w] == best && wi[w] < bi)) {
      best = wv[w];
      bi = wi[w];
    }
  const int bx = bi % n, by = bi / n;
  ClusterRec c;
  c.e_cluster = 0.0;
  for (int dy = -1; dy <= 1; ++dy)
    for (int dx = -1; dx <= 1; ++dx) {
      const int x = bx + dx, y = by + dy;
      const bool on = x >= 0 && y >= 0 && x < n && y < n;
      const double v = on ? e[y * n + x] : __longlong_as_double(0x7ff8000000000000ll);
      c.e[(dy + 1) * 3 + (dx + 1)] = v;
      if (on) c.e_cluster += v;
    }
  int veto = 0;
  for (int dy = -3; dy <= 3; ++dy)
    for (int dx = -3; dx <= 3; ++dx) {
      if (dx >= -1 && dx <= 1 && dy >= -1 && dy <= 1) continue;
      const int x = bx + dx, y = by + dy;
      if (x < 0 || y < 0 || x >= n || y >= n) continue;
      if (e[y * n + x] > r.veto_factor * r.noise_keV) veto = 1;
    }
  c.cx = bx;
  c.cy = by;
  c.vetoed = veto;
  c.accepted = !veto && fabs(c.e_cluster - r.beam_keV) <= r.window_keV;
  r.clusters[ev] = c;
  if (c.accepted && r.spectrum)
    for (int k = 0; k < 9; ++k) {
      const double v = c.e[k];
      if (isnan(v)) continue;
      const double b = floor((v - r.spec_lo_keV) / r.spec_bin_keV);
      if (b >= 0.0 && b < (double)r.n_bins) atomicAdd(r.spectrum + (int64_t)b, 1ull);
    }
}

// FP32 FMA throughput probe: independent FMA chains per thread (packed f32x2
// or scalar), the denominator the pair kernel's FP32 work is compared with.
template <bool PACKED>
__global__ void __launch_bounds__(256) fma_chain_kernel(float* out, int iters) {
  constexpr int C = 8;
  float2 a[C];
#pragma unroll
  for (int q = 0; q < C; ++q) a[q] = make_float2(threadIdx.x * 1e-3f + q, 0.5f * q);
  const float2 m = make_float2(0.999f, 0.999f), c = make_float2(1e-3f, 1e-3f);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int q = 0; q < C; ++q) {
      if (PACKED) {
        a[q] = __ffma2_rn(a[q], m, c);
      } else {
        a[q].x = fmaf(a[q].x, m.x, c.x);
        a[q].y = fmaf(a[q].y, m.y, c.y);
      }
    }
  }
  float s = 0.0f;
#pragma unroll
  for (int q = 0; q < C; ++q) s += a[q].x + a[q].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void philox_kernel(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                              uint32_t* curand_out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 o = philox10(c, make_uint2(key[2 * i], key[2 * i + 1]));
  out[4 * i] = o.x;
  out[4 * i + 1] = o.y;
  out[4 * i + 2] = o.z;
  out[4 * i + 3] = o.w;
  if (curand_out) {
    // curand's Philox4_32_10 stream: counter words (c0, c1) advance with the
    // offset (4 outputs per counter value), (c2, c3) hold the subsequence.
    curandStatePhilox4_32_10_t st;
    const unsigned long long seed = ((unsigned long long)key[2 * i + 1] << 32) | key[2 * i];
    const unsigned long long sub = ((unsigned long long)c.w << 32) | c.z;
    const unsigned long long off = (((unsigned long long)c.y << 32) | c.x) * 4ull;
    curand_init(seed, sub, off, &st);
    const uint4 r = curand4(&st);
    curand_out[4 * i] = r.x;
    curand_out[4 * i + 1] = r.y;
    curand_out[4 * i + 2] = r.z;
    curand_out[4 * i + 3] = r.w;
  }
}

__global__ void normals_kernel(const unsigned long long* in, int64_t n, double* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const unsigned long long* t = in + 5 * i;
  const float3 v = normals_f(stream_words(t[0], t[1], (uint32_t)t[2], (uint32_t)t[3], (uint32_t)t[4]));
  out[3 * i] = v.x;
  out[3 * i + 1] = v.y;
  out[3 * i + 2] = v.z;
}

// ---------------------------------------------------------------------------
// Variant table.
// ---------------------------------------------------------------------------
struct VariantEntry {
  int nt, r;
  const char* name;
  void (*fn)(StepArgs, int, int);
  int ctas_per_sm, dynamic, mode;
  void (*fn_ind)(StepArgs, int, int);  // the same kernel recording the induced charge
  void (*fn_px)(StepArgs, int, int);   // ... and the 3 x 3 window's pixel signals
};

// (threads, i's per thread, packed f32x2, j unroll, min CTAs per SM [register
// cap], CTAs per SM launched [0 = all that fit], dynamic queue).  Entry 0 is
// the default: the symmetric kernel (each unordered pair once, one warp per
// unit, 12 warps per SM).  The others evaluate every ordered pair: sources
// paired in packed FP32 lanes, 512-carrier tiles, guided dynamic queue first.
#define CTS_V(NT, R, MODE, JU, MB, CPS, DYN, NAME) \
  {NT, R, NAME, step_kernel<NT, R, MODE, JU, MB, 0>, CPS, DYN, MODE, \
   step_kernel<NT, R, MODE, JU, MB, 1>, step_kernel<NT, R, MODE, JU, MB, 2>}
#define CTS_SYM(NT, NAME) \
  {NT, kSymRI, NAME, sym_kernel<kSymRI, NT, 0>, 1, 1, 3, sym_kernel<kSymRI, NT, 1>, \
   sym_kernel<kSymRI, NT, 2>}
const VariantEntry kVariants[] = {
    CTS_SYM(384, "sym_nt384_r8_warp"),
    CTS_V(256, 2, 2, 4, 3, 0, 1, "nt256_r2_jpair_dyn"),
    CTS_V(256, 4, 2, 4, 2, 0, 1, "nt256_r4_jpair_dyn"),
    CTS_V(128, 2, 2, 4, 6, 0, 1, "nt128_r2_jpair_dyn"),
    CTS_V(128, 4, 2, 4, 4, 0, 1, "nt128_r4_jpair_dyn"),
    CTS_V(512, 1, 2, 4, 2, 0, 1, "nt512_r1_jpair_dyn"),
    CTS_V(128, 4, 1, 4, 4, 0, 1, "nt128_r4_ipair_dyn"),
    CTS_V(256, 2, 1, 4, 3, 0, 1, "nt256_r2_ipair_dyn"),
    CTS_V(128, 4, 1, 4, 4, 0, 0, "nt128_r4_ipair_static"),
    CTS_V(512, 2, 1, 4, 1, 1, 0, "nt512_r2_ipair_1sm_static"),
    CTS_V(256, 2, 0, 4, 3, 0, 1, "nt256_r2_scalar_dyn"),
    CTS_V(256, 2, 0, 2, 4, 0, 0, "nt256_r2_scalar_static"),
    CTS_SYM(256, "sym_nt256_r8_warp"),
};
#undef CTS_V
#undef CTS_SYM
constexpr int kNumVariants = sizeof(kVariants) / sizeof(kVariants[0]);
constexpr size_t kStageBytes = 2 * kChunkJ * sizeof(float4);
constexpr size_t kSoaBytes = 3 * kChunkJ * sizeof(float);
size_t smem_of(const VariantEntry& e) {
  if (e.mode == 3) return (size_t)(e.nt / 32) * kSymWarpFloats * sizeof(float);
  return kStageBytes + (e.mode == 2 ? kSoaBytes : 0);
}

}  // namespace

int variant_count() { return kNumVariants; }

Variant variant_info(int v) {
  const VariantEntry& e = kVariants[v];
  return Variant{e.nt, e.r, e.name, e.ctas_per_sm, e.dynamic, e.mode == 3 ? 1 : 0};
}

size_t variant_smem(int v) { return smem_of(kVariants[v]); }

cudaError_t variant_occupancy(int v, int* blocks_per_sm) {
  const VariantEntry& e = kVariants[v];
  cudaError_t err = cudaFuncSetAttribute(e.fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem_of(e));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(e.fn_ind, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_of(e));
  if (err != cudaSuccess) return err;
  err = cudaFuncSetAttribute(e.fn_px, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem_of(e));
  if (err != cudaSuccess) return err;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, e.fn, e.nt, smem_of(e));
}

cudaError_t launch_step(int v, const StepArgs& a, int k0, int nk, int grid, cudaStream_t s) {
  const VariantEntry& e = kVariants[v];
  (a.induced_px ? e.fn_px : (a.induced ? e.fn_ind : e.fn))<<<grid, e.nt, smem_of(e), s>>>(
      a, k0, nk);
  return cudaGetLastError();
}

cudaError_t launch_update(const StepArgs& a, int k, int n_slots_list, const int32_t* slot_list,
                          int grid, cudaStream_t s) {
  if (a.induced_px)
    update_kernel<true><<<grid, 256, 0, s>>>(a, k, slot_list, n_slots_list);
  else
    update_kernel<false><<<grid, 256, 0, s>>>(a, k, slot_list, n_slots_list);
  return cudaGetLastError();
}

cudaError_t launch_init(const Phys& ph, Arena A, SlotDev* slots, const int32_t* slot_list, int n,
                        const ExplicitRec* explicit_buf, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  init_kernel<<<n, kAuxThreads, 0, s>>>(ph, A, slots, slot_list, explicit_buf);
  return cudaGetLastError();
}

cudaError_t launch_close(const Phys& ph, Arena A, SlotDev* slots, const int32_t* /*slot_list*/,
                         int n, const int32_t* ret, int S, int K, SlotSummary* summary,
                         cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  close_kernel<<<n, kAuxThreads, 0, s>>>(ph, A, slots, ret, S, K, summary);
  return cudaGetLastError();
}

cudaError_t launch_bin(const Phys& ph, Arena A, const SlotDev* slots, const int32_t* slot_list,
                       int n, int32_t* pixels, SlotReadout* readout, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  bin_kernel<<<n, kAuxThreads, 0, s>>>(ph, A, slots, slot_list, pixels, readout);
  return cudaGetLastError();
}

cudaError_t launch_bin_points(const Phys& ph, const double* x, const double* y, int64_t n,
                              int32_t* pixels, long long* outside, cudaStream_t s) {
  const int threads = 256;
  int grid = (int)((n + threads - 1) / threads);
  grid = grid < 1 ? 1 : (grid > 4096 ? 4096 : grid);
  bin_points_kernel<<<grid, threads, 0, s>>>(ph, x, y, n, pixels, outside);
  return cudaGetLastError();
}

constexpr size_t kSphSmem =
    (size_t)kSphMax * (sizeof(unsigned long long) + sizeof(uint16_t) + sizeof(int8_t)) +
    2 * kSphBins * sizeof(int32_t) + (size_t)kSphGroups * 4 * sizeof(double);
static_assert(kSphSmem <= 227 * 1024, "spherical kernel shared memory");

// Largest number of resident clusters of C spherical CTAs (0 = unknown).
int g_sph_clusters[5] = {0, 0, 0, 0, 0};

cudaError_t spherical_prepare() {
  cudaError_t e = cudaFuncSetAttribute(spherical_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSphSmem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(spherical_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)kSphSmem);
  if (e != cudaSuccess) return e;
  for (int c = 1; c <= 4; c <<= 1) {
    cudaLaunchConfig_t cfg{};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)c;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.gridDim = dim3((unsigned)c, 1, 1);
    cfg.blockDim = dim3(1024, 1, 1);
    cfg.dynamicSmemBytes = kSphSmem;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, spherical_kernel<false>, &cfg);
    if (e != cudaSuccess) return e;
    g_sph_clusters[c] = n;
  }
  return cudaSuccess;
}

int spherical_cluster(int slots, int request) {
  if (request == 1 || request == 2 || request == 4) return request;
  // the widest cluster with which every slot's cluster is resident at once
  for (int c = 4; c >= 2; c >>= 1)
    if (slots <= g_sph_clusters[c]) return c;
  return 1;
}

cudaError_t launch_spherical(const StepArgs& a, int k0, int nk, int cluster, cudaStream_t s) {
  if (a.S <= 0) return cudaSuccess;
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)cluster;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)(a.S * cluster), 1, 1);
  cfg.blockDim = dim3(1024, 1, 1);
  cfg.dynamicSmemBytes = kSphSmem;
  cfg.stream = s;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (a.induced_px) return cudaLaunchKernelEx(&cfg, spherical_kernel<true>, a, k0, nk);
  return cudaLaunchKernelEx(&cfg, spherical_kernel<false>, a, k0, nk);
}

cudaError_t launch_generate(const GenEvent* ev, int n_events, double pitch_um, int grid_n,
                            int32_t* pixels, unsigned long long* outside, cudaStream_t s) {
  if (n_events > 0) generate_kernel<<<n_events, 256, 0, s>>>(ev, pitch_um, grid_n, pixels, outside);
  return cudaGetLastError();
}

cudaError_t launch_readout(const ReadoutArgs& r, int n_events, cudaStream_t s) {
  if (n_events > 0) readout_kernel<<<n_events, 256, 0, s>>>(r);
  return cudaGetLastError();
}

cudaError_t launch_fma_chain(bool packed, float* out, int grid, int iters, cudaStream_t s) {
  if (packed)
    fma_chain_kernel<true><<<grid, 256, 0, s>>>(out, iters);
  else
    fma_chain_kernel<false><<<grid, 256, 0, s>>>(out, iters);
  return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, const uint32_t* key, int64_t n, uint32_t* out,
                          uint32_t* curand_out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  philox_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(ctr, key, n, out, curand_out);
  return cudaGetLastError();
}

cudaError_t launch_normals(const unsigned long long* in, int64_t n, double* out, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  normals_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(in, n, out);
  return cudaGetLastError();
}

}  // namespace cts
