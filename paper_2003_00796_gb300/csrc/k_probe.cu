// k_probe.cu -- measured peaks of the pipes that bound the transport kernels:
// FP32 fused multiply-add, 32-bit integer multiply-add, the special-function
// unit (base-2 logarithm and exponential, sine), and float atomic adds that
// resolve in L2. Nothing on the transport path is a dense contraction and its
// working set stays on chip, so these -- not HBM bandwidth or tensor-core
// throughput -- are the roofline denominators of the transport kernels. The
// paper has no counterpart (it reports CPU run times only); these are
// measurement helpers of this library.
//
// Each probe keeps every SM busy with many independent dependency chains per
// thread (enough warps and instruction-level parallelism to hide the pipe's
// latency), so its rate is the pipe's issue-limited throughput at the clock
// the GPU runs at. The special-function probes use the PTX approximate
// instructions directly, one per operation.
#include <algorithm>

#include "gbmc_internal.h"

namespace gb {

constexpr int kProbeBlock = 256;
constexpr int kProbeChains = 8;

// FP32: kProbeChains chains of fmaf per thread, iters rounds
__global__ void __launch_bounds__(kProbeBlock) k_probe_ffma(float* out, int iters, float a, float b) {
  float x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c)   // PTX, so that no compiler pass can merge rounds
        asm("fma.rn.f32 %0, %0, %1, %2;" : "+f"(x[c]) : "f"(a), "f"(b));
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  if (s == 1.2345e-30f) out[blockIdx.x] = s;   // keeps the chains live; never true in practice
}

// INT32: chains of 32-bit multiply-add (the Philox round's multiplier work)
__global__ void __launch_bounds__(kProbeBlock) k_probe_imad(unsigned* out, int iters, unsigned a, unsigned b) {
  unsigned x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = threadIdx.x * 2654435761u + c;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c)   // PTX: integer rounds would otherwise fold
        asm("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[c]) : "r"(a), "r"(b));
  }
  unsigned s = 0;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s ^= x[c];
  if (s == 0x9e3779b9u && threadIdx.x == 7) out[blockIdx.x] = s;
}

__device__ __forceinline__ float mufu(int kind, float x) {
  float y;
  if (kind == 0) asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  else if (kind == 1) asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  else asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// special-function unit: chains of one approximate transcendental each
template <int KIND>
__global__ void __launch_bounds__(kProbeBlock) k_probe_mufu(float* out, int iters) {
  float x[kProbeChains];
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) x[c] = 1.5f + (float)(threadIdx.x + c) * 1e-3f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < kProbeChains; ++c) x[c] = mufu(KIND, x[c]);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < kProbeChains; ++c) s += x[c];
  if (s == 1.2345e-30f) out[blockIdx.x] = s;
}

// float atomic adds (no return value, as the tally issues them) to addresses
// spread over a buffer that stays in L2: every thread adds to a pseudo-random
// word each round
__global__ void __launch_bounds__(kProbeBlock) k_probe_red(float* buf, unsigned mask, int iters) {
  unsigned h = (blockIdx.x * blockDim.x + threadIdx.x) * 2654435761u + 12345u;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      h = h * 1664525u + 1013904223u;
      atomicAdd(buf + ((h >> 3) & mask), 1.0f);
    }
  }
}

}  // namespace gb

using namespace gb;

extern "C" gbmc_status gbmc_probe_peak(int device, int kind, int iters, double* ops, double* ms) {
  if (!ops || !ms || iters < 1 || kind < GBMC_PROBE_FFMA || kind > GBMC_PROBE_L2_ATOMIC)
    return GBMC_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GBMC_ERR_CUDA;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return GBMC_ERR_CUDA;
  const int blocks = sms * 8;     // 8 resident blocks of 256 threads per SM: 64 warps
  const size_t red_words = (size_t)1 << 23;   // 32 MB of float counters (L2 is 129 MB)
  float* buf = nullptr;
  if (cudaMalloc((void**)&buf, kind == GBMC_PROBE_L2_ATOMIC ? red_words * 4 : (size_t)blocks * 4) != cudaSuccess)
    return GBMC_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess && kind == GBMC_PROBE_L2_ATOMIC) e = cudaMemset(buf, 0, red_words * 4);
  float t = 0.f;
  for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep) {   // the first launch warms up
    e = cudaEventRecord(e0, 0);
    switch (kind) {
      case GBMC_PROBE_FFMA: k_probe_ffma<<<blocks, kProbeBlock>>>(buf, iters, 0.999f, 1e-4f); break;
      case GBMC_PROBE_IMAD:
        k_probe_imad<<<blocks, kProbeBlock>>>(reinterpret_cast<unsigned*>(buf), iters, 0xD2511F53u, 7u);
        break;
      case GBMC_PROBE_LG2: k_probe_mufu<0><<<blocks, kProbeBlock>>>(buf, iters); break;
      case GBMC_PROBE_EX2: k_probe_mufu<1><<<blocks, kProbeBlock>>>(buf, iters); break;
      case GBMC_PROBE_SIN: k_probe_mufu<2><<<blocks, kProbeBlock>>>(buf, iters); break;
      default: k_probe_red<<<blocks, kProbeBlock>>>(buf, (unsigned)(red_words - 1), iters); break;
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(buf);
  if (e != cudaSuccess) return GBMC_ERR_CUDA;
  const double per_thread = (double)iters * 4.0 * (kind == GBMC_PROBE_L2_ATOMIC ? 1.0 : kProbeChains);
  *ops = per_thread * (double)blocks * kProbeBlock;
  *ms = t;
  return GBMC_OK;
}
