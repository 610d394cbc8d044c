// cts_noalloc.cu -- a repulsion-field entry point that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host that hands this library only
// the device buffers it owns (a plugin inside another framework's memory
// pool, a process with a fixed device-memory budget, code that must not
// synchronise the device the way cudaMalloc/cudaFree can).  For them,
// cts_field_noalloc computes the same pair field as the library's field
// kernel, with the caller's device buffers for inputs and output, and keeps
// its working storage (per-carrier FP64 accumulators and per-tile counters)
// in one file-scope __device__ array of fixed size instead of allocating it.
// That array is part of the library image: every GPU that loads the library
// holds it (about 3 MB) until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "cts.h"

namespace {

constexpr int kNaMaxCarriers = 131072;  // largest n_h + n_e accepted
constexpr int kNaThreads = 128;
constexpr int kNaR = 4;                 // carriers per thread
constexpr int kNaTile = kNaThreads * kNaR;
constexpr int kNaMaxTiles = kNaMaxCarriers / kNaTile;
constexpr int kNaStage = 256;           // sources staged in shared memory per pass
constexpr int kNaMaxSplit = 32;
constexpr int kNaMaxDevices = 64;
// layout: acc[3][kNaMaxCarriers] FP64, then one 64-bit counter per tile
constexpr size_t kNaWords = 3 * (size_t)kNaMaxCarriers + kNaMaxTiles;

static __device__ __align__(256) unsigned long long cts_noalloc_scratch[kNaWords];

__device__ __forceinline__ float na_rsqrt(float v) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// Eq. 4 read as a field: E_i = k sum_j s_j (r_i - r_j) / (|r_i - r_j|^2 + eps^2)^(3/2)
// with s_j = +1 for the first n_h carriers (holes) and -1 for the rest.
// Block b handles tile b / n_split of the i's against source range split
// b % n_split; the block that completes a tile's last split writes the tile's
// output and returns its accumulators and counter to zero.
__global__ void __launch_bounds__(kNaThreads) field_noalloc_kernel(
    const float* __restrict__ x, const float* __restrict__ y, const float* __restrict__ z,
    int n_h, int n_e, int n_split, float kc, float eps2, float* __restrict__ out,
    unsigned long long* scratch) {
  __shared__ float4 sj[kNaStage];
  __shared__ int s_last;
  const int n = n_h + n_e;
  const int tile = blockIdx.x / n_split, split = blockIdx.x % n_split;
  const int i0 = tile * kNaTile;
  const int j0 = (int)((long long)n * split / n_split);
  const int j1 = (int)((long long)n * (split + 1) / n_split);
  double* acc = reinterpret_cast<double*>(scratch);
  unsigned long long* count = scratch + 3 * (size_t)kNaMaxCarriers;

  float xi[kNaR], yi[kNaR], zi[kNaR], sx[kNaR], sy[kNaR], sz[kNaR], cx[kNaR], cy[kNaR],
      cz[kNaR];
#pragma unroll
  for (int r = 0; r < kNaR; ++r) {
    const int i = i0 + r * kNaThreads + threadIdx.x;
    xi[r] = i < n ? x[i] : 0.0f;
    yi[r] = i < n ? y[i] : 0.0f;
    zi[r] = i < n ? z[i] : 0.0f;
    sx[r] = sy[r] = sz[r] = cx[r] = cy[r] = cz[r] = 0.0f;
  }
  for (int jb = j0; jb < j1; jb += kNaStage) {
    const int m = min(kNaStage, j1 - jb);
    for (int t = threadIdx.x; t < m; t += kNaThreads) {
      const int j = jb + t;
      sj[t] = make_float4(x[j], y[j], z[j], j < n_h ? 1.0f : -1.0f);
    }
    __syncthreads();
    float tx[kNaR], ty[kNaR], tz[kNaR];
#pragma unroll
    for (int r = 0; r < kNaR; ++r) tx[r] = ty[r] = tz[r] = 0.0f;
    for (int t = 0; t < m; ++t) {
      const float4 q = sj[t];
#pragma unroll
      for (int r = 0; r < kNaR; ++r) {
        const float dx = xi[r] - q.x, dy = yi[r] - q.y, dz = zi[r] - q.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
        const float rs = na_rsqrt(r2);
        const float w = q.w * ((rs * rs) * rs);
        tx[r] = fmaf(dx, w, tx[r]);
        ty[r] = fmaf(dy, w, ty[r]);
        tz[r] = fmaf(dz, w, tz[r]);
      }
    }
#pragma unroll
    for (int r = 0; r < kNaR; ++r) {  // Kahan fold of this pass
      float u = tx[r] - cx[r], v = sx[r] + u;
      cx[r] = (v - sx[r]) - u;
      sx[r] = v;
      u = ty[r] - cy[r];
      v = sy[r] + u;
      cy[r] = (v - sy[r]) - u;
      sy[r] = v;
      u = tz[r] - cz[r];
      v = sz[r] + u;
      cz[r] = (v - sz[r]) - u;
      sz[r] = v;
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < kNaR; ++r) {
    const int i = i0 + r * kNaThreads + threadIdx.x;
    if (i < n) {
      atomicAdd(acc + i, (double)sx[r] - (double)cx[r]);
      atomicAdd(acc + kNaMaxCarriers + i, (double)sy[r] - (double)cy[r]);
      atomicAdd(acc + 2 * kNaMaxCarriers + i, (double)sz[r] - (double)cz[r]);
    }
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long old = atomicAdd(count + tile, 1ull);
    s_last = old == (unsigned long long)(n_split - 1);
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();
#pragma unroll
  for (int r = 0; r < kNaR; ++r) {
    const int i = i0 + r * kNaThreads + threadIdx.x;
    if (i < n) {
      out[i] = kc * (float)__ldcg(acc + i);
      out[n + i] = kc * (float)__ldcg(acc + kNaMaxCarriers + i);
      out[2 * n + i] = kc * (float)__ldcg(acc + 2 * kNaMaxCarriers + i);
      acc[i] = 0.0;
      acc[kNaMaxCarriers + i] = 0.0;
      acc[2 * kNaMaxCarriers + i] = 0.0;
    }
  }
  if (threadIdx.x == 0) count[tile] = 0ull;
}

// Device address of the scratch array, looked up once per device (with that
// device current) and cached.
std::mutex g_na_mu;
void* g_na_addr[kNaMaxDevices] = {};
int g_na_sms[kNaMaxDevices] = {};

int na_setup(int dev, void** addr, int* sms) {
  std::lock_guard<std::mutex> lk(g_na_mu);
  if (dev < 0 || dev >= kNaMaxDevices) return SIM_ENODEV;
  if (!g_na_addr[dev]) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) return SIM_ENODEV;
    if (prop.major != 10 || prop.minor != 3) return SIM_ENODEV;
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, cts_noalloc_scratch) != cudaSuccess || !p) return SIM_ECUDA;
    g_na_addr[dev] = p;
    g_na_sms[dev] = prop.multiProcessorCount;
  }
  *addr = g_na_addr[dev];
  *sms = g_na_sms[dev];
  return SIM_OK;
}

}  // namespace

extern "C" int cts_field_noalloc(const float* dev_x, const float* dev_y, const float* dev_z,
                                 int32_t n_h, int32_t n_e, double eps_r, double softening_um,
                                 float* dev_E, void* stream) {
  if (n_h < 0 || n_e < 0 || !(eps_r > 0) || !(softening_um >= 0) || !std::isfinite(eps_r) ||
      !std::isfinite(softening_um))
    return SIM_EINVAL;
  const int64_t n = (int64_t)n_h + n_e;
  if (n > kNaMaxCarriers) return SIM_ENOMEM_BUDGET;  // beyond the fixed scratch
  if (n == 0) return SIM_OK;
  if (!dev_x || !dev_y || !dev_z || !dev_E) return SIM_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return SIM_ENODEV;
  void* scratch = nullptr;
  int sms = 0;
  const int rc = na_setup(dev, &scratch, &sms);
  if (rc != SIM_OK) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  const int tiles = (int)((n + kNaTile - 1) / kNaTile);
  // the accumulators and counters this call uses start at zero
  double* acc = (double*)scratch;
  for (int c = 0; c < 3; ++c)
    if (cudaMemsetAsync(acc + (size_t)c * kNaMaxCarriers, 0, (size_t)n * sizeof(double), s) !=
        cudaSuccess)
      return SIM_ECUDA;
  if (cudaMemsetAsync((unsigned long long*)scratch + 3 * (size_t)kNaMaxCarriers, 0,
                      (size_t)tiles * sizeof(unsigned long long), s) != cudaSuccess)
    return SIM_ECUDA;
  int n_split = (4 * sms + tiles - 1) / tiles;
  n_split = n_split < 1 ? 1 : (n_split > kNaMaxSplit ? kNaMaxSplit : n_split);
  if (n_split > n / 64) n_split = (int)(n / 64 > 1 ? n / 64 : 1);
  const double e = 1.602176634e-19, eps0 = 8.8541878128e-12;
  const float kc = (float)(e / (4.0 * M_PI * eps0 * eps_r) * 1e6);
  const double eps = softening_um > 0 ? softening_um : 1e-6;
  field_noalloc_kernel<<<tiles * n_split, kNaThreads, 0, s>>>(
      dev_x, dev_y, dev_z, n_h, n_e, n_split, kc, (float)(eps * eps), dev_E,
      (unsigned long long*)scratch);
  return cudaGetLastError() == cudaSuccess ? SIM_OK : SIM_ECUDA;
}
