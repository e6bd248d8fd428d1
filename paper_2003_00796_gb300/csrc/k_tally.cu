// k_tally.cu -- batch flush and finalisation of the dose tally (Sec. 4.2.3,
// Eq. 1-2), phantom validation, and the device Philox fill used by tests.
//
// Flush: the FP32 batch tile B (one float per voxel, filled by the transport
// kernels' atomics) is folded into FP64 accumulators S1 += B, S2 += B^2 / n_k
// and zeroed. Finalise: mean = S1 / N, var(mean) = (S2 - N mean^2) / (N (K-1)),
// divided by the voxel mass for dose. Both are streaming, HBM-bound kernels.
#include <algorithm>

#include "gbmc_internal.h"

namespace gb {

constexpr int kStreamBlock = 256;

// fold the K batch tiles into the FP64 accumulators: per voxel
// S1 += sum_k B_k and S2 += sum_k B_k^2 / n_k; zero the tiles. Tiles and
// accumulators are padded to a multiple of 4 voxels (float4 / double2 access);
// all-zero quads are skipped, which keeps sparse (pencil-beam) doses cheap.
__global__ void __launch_bounds__(kStreamBlock) k_flush_tiles(float* __restrict__ tiles,
                                                              int64_t stride4, int K,
                                                              const double* __restrict__ inv_n,
                                                              double* __restrict__ s1,
                                                              double* __restrict__ s2,
                                                              double* __restrict__ dep) {
  // K <= GBMC_MAX_BATCHES (gbmc_create and gbmc_run_noalloc reject more)
  __shared__ double sinv[GBMC_MAX_BATCHES];
  for (int k = threadIdx.x; k < K && k < GBMC_MAX_BATCHES; k += blockDim.x) sinv[k] = inv_n[k];
  __syncthreads();
  double acc = 0.0;
  float4* t4 = reinterpret_cast<float4*>(tiles);
  double2* a2 = reinterpret_cast<double2*>(s1);
  double2* b2 = reinterpret_cast<double2*>(s2);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < stride4; i += stride) {
    double a0 = 0, a1 = 0, a2s = 0, a3 = 0, q0 = 0, q1 = 0, q2 = 0, q3 = 0;
    bool any = false;
    for (int k = 0; k < K; ++k) {
      const int64_t j = (int64_t)k * stride4 + i;
      const float4 b = t4[j];
      if (b.x != 0.0f || b.y != 0.0f || b.z != 0.0f || b.w != 0.0f) {
        const double w = sinv[k < GBMC_MAX_BATCHES ? k : GBMC_MAX_BATCHES - 1];
        any = true;
        a0 += b.x; a1 += b.y; a2s += b.z; a3 += b.w;
        q0 += (double)b.x * b.x * w; q1 += (double)b.y * b.y * w;
        q2 += (double)b.z * b.z * w; q3 += (double)b.w * b.w * w;
        t4[j] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    if (any) {
      double2 x0 = a2[2 * i], x1 = a2[2 * i + 1], y0 = b2[2 * i], y1 = b2[2 * i + 1];
      x0.x += a0; x0.y += a1; x1.x += a2s; x1.y += a3;
      y0.x += q0; y0.y += q1; y1.x += q2; y1.y += q3;
      a2[2 * i] = x0; a2[2 * i + 1] = x1; b2[2 * i] = y0; b2[2 * i + 1] = y1;
      acc += (a0 + a1) + (a2s + a3);
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(dep, acc);
}

cudaError_t launch_flush_tiles(float* tiles, int64_t stride, int K, const double* inv_n,
                               double* s1, double* s2, double* dep, int sms, cudaStream_t s) {
  const int64_t stride4 = stride >> 2;
  const int64_t need = (stride4 + kStreamBlock - 1) / kStreamBlock;
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(need, 1), (int64_t)sms * 8);
  k_flush_tiles<<<grid, kStreamBlock, 0, s>>>(tiles, stride4, K, inv_n, s1, s2, dep);
  return cudaGetLastError();
}

// the same fold into caller-owned accumulators of exactly nvox doubles with
// no alignment guarantee: scalar, bounds-checked accesses
__global__ void __launch_bounds__(kStreamBlock) k_flush_tiles_scalar(float* __restrict__ tiles,
                                                                     int64_t stride, int64_t nvox,
                                                                     int K,
                                                                     const double* __restrict__ inv_n,
                                                                     double* __restrict__ s1,
                                                                     double* __restrict__ s2,
                                                                     double* __restrict__ dep) {
  double acc = 0.0;
  const int64_t gs = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += gs) {
    double a = 0.0, q = 0.0;
    bool any = false;
    for (int k = 0; k < K; ++k) {
      const int64_t j = (int64_t)k * stride + i;
      const float b = tiles[j];
      if (b != 0.0f) {
        any = true;
        a += b;
        q += (double)b * b * inv_n[k];
        tiles[j] = 0.0f;
      }
    }
    if (any) {
      s1[i] += a;
      s2[i] += q;
      acc += a;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0 && acc != 0.0) atomicAdd(dep, acc);
}

cudaError_t launch_flush_tiles_scalar(float* tiles, int64_t stride, int64_t nvox, int K,
                                      const double* inv_n, double* s1, double* s2, double* dep,
                                      int sms, cudaStream_t s) {
  const int64_t need = (nvox + kStreamBlock - 1) / kStreamBlock;
  const int grid = (int)std::min<int64_t>(std::max<int64_t>(need, 1), (int64_t)sms * 8);
  k_flush_tiles_scalar<<<grid, kStreamBlock, 0, s>>>(tiles, stride, nvox, K, inv_n, s1, s2, dep);
  return cudaGetLastError();
}

__global__ void k_finalize(const double* __restrict__ s1, const double* __restrict__ s2,
                           const float* __restrict__ rho, int64_t nvox, double n_hist,
                           double k_batches, double vol, int dose, double* __restrict__ mean,
                           double* __restrict__ var) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
    const double m = s1[i] / n_hist;
    double v = (k_batches > 1.0) ? (s2[i] - n_hist * m * m) / (n_hist * (k_batches - 1.0)) : 0.0;
    if (v < 0.0) v = 0.0;
    double scale = 1.0;
    if (dose) scale = 1.0 / ((double)rho[i] * vol);
    mean[i] = m * scale;
    if (var) var[i] = v * scale * scale;
  }
}

cudaError_t launch_finalize(const double* s1, const double* s2, const float* rho, int64_t nvox,
                            double n_hist, double k_batches, double vol, int dose, double* mean,
                            double* var, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((nvox + 255) / 256, 152 * 8);
  k_finalize<<<std::max(grid, 1), 256, 0, s>>>(s1, s2, rho, nvox, n_hist, k_batches, vol, dose,
                                                 mean, var);
  return cudaGetLastError();
}

// add another tally's moments: s1 += x1, s2 += x2 (nvox doubles each)
__global__ void k_add_moments(double* __restrict__ s1, double* __restrict__ s2,
                              const double* __restrict__ x1, const double* __restrict__ x2,
                              int64_t nvox) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
    s1[i] += x1[i];
    s2[i] += x2[i];
  }
}

cudaError_t launch_add_moments(double* s1, double* s2, const double* x1, const double* x2,
                               int64_t nvox, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((nvox + 255) / 256, 152 * 8);
  k_add_moments<<<std::max(grid, 1), 256, 0, s>>>(s1, s2, x1, x2, nvox);
  return cudaGetLastError();
}

// 1 / n_k for the K batches of a run of n histories (batch k holds
// floor((k+1)n/K) - floor(kn/K) histories)
__global__ void k_batch_weights(double* inv_n, uint64_t n, int K) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const uint64_t a = (uint64_t)(((unsigned __int128)n * (uint64_t)k) / (uint64_t)K);
    const uint64_t b = (uint64_t)(((unsigned __int128)n * (uint64_t)(k + 1)) / (uint64_t)K);
    inv_n[k] = 1.0 / (double)(b - a);
  }
}

cudaError_t launch_batch_weights(double* inv_n, uint64_t n_hist, int K, cudaStream_t s) {
  k_batch_weights<<<(K + 255) / 256, 256, 0, s>>>(inv_n, n_hist, K);
  return cudaGetLastError();
}

__global__ void k_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                              const PhiloxKeys K, uint32_t* out, int n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    U4 c;
    c.x = c0 + (uint32_t)i; c.y = c1; c.z = c2; c.w = c3;
    const U4 o = philox4x32_10(c, K);   // the round-key form the transport kernels use
    out[4 * i + 0] = o.x; out[4 * i + 1] = o.y; out[4 * i + 2] = o.z; out[4 * i + 3] = o.w;
  }
}

cudaError_t launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                               uint32_t k1, uint32_t* out, int n, cudaStream_t s) {
  const int grid = std::max(1, std::min((n + 255) / 256, 4096));
  k_philox_fill<<<grid, 256, 0, s>>>(c0, c1, c2, c3, philox_keys(k0, k1), out, n);
  return cudaGetLastError();
}

// material ids < n_mat and finite positive densities; per-material max density
// Each thread keeps its own count of invalid voxels and its own maximum
// density per material over its grid-stride share; the warp then combines
// them and one lane issues one atomic per material (an atomic per voxel on
// the few rho_max words serialised in L2: about 1 ms per 2 M voxels)
__global__ void k_validate(const uint8_t* __restrict__ mat, const float* __restrict__ rho,
                           int64_t nvox, int n_mat, unsigned int* bad, float* rho_max) {
  static_assert(GBMC_MAX_MAT == 4, "one register per material below");
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  unsigned int nbad = 0, m0 = 0, m1 = 0, m2 = 0, m3 = 0;   // positive floats order like their bits
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride) {
    const int m = mat[i];
    const float r = rho[i];
    if (m >= n_mat || !(r > 0.0f) || !isfinite(r)) {
      ++nbad;
    } else {
      const unsigned int b = __float_as_uint(r);
      if (m == 0) m0 = max(m0, b);
      else if (m == 1) m1 = max(m1, b);
      else if (m == 2) m2 = max(m2, b);
      else m3 = max(m3, b);
    }
  }
  const unsigned full = 0xffffffffu;
  nbad = __reduce_add_sync(full, nbad);
  m0 = __reduce_max_sync(full, m0);
  m1 = __reduce_max_sync(full, m1);
  m2 = __reduce_max_sync(full, m2);
  m3 = __reduce_max_sync(full, m3);
  if ((threadIdx.x & 31) == 0) {
    unsigned int* rm = reinterpret_cast<unsigned int*>(rho_max);
    if (nbad) atomicAdd(bad, nbad);
    if (m0) atomicMax(rm + 0, m0);
    if (m1 && n_mat > 1) atomicMax(rm + 1, m1);
    if (m2 && n_mat > 2) atomicMax(rm + 2, m2);
    if (m3 && n_mat > 3) atomicMax(rm + 3, m3);
  }
}

cudaError_t launch_validate_phantom(const uint8_t* mat, const float* rho, int64_t nvox, int n_mat,
                                    unsigned int* bad, float* rho_max, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((nvox + 255) / 256, 152 * 8);
  k_validate<<<std::max(grid, 1), 256, 0, s>>>(mat, rho, nvox, n_mat, bad, rho_max);
  return cudaGetLastError();
}

}  // namespace gb
