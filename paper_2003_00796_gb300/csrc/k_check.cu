// k_check.cu -- the checked build's index test, exposed for tests: which
// library variant this is (gbmc_build_checked), and the test itself run on the
// device for given (index, bound) pairs (gbmc_check_index). The paper has no
// counterpart; see the checked-build section of gbmc.h.
#include <vector>

#include "gbmc_internal.h"

namespace gb {

// one pair per thread; reads and writes only [0, n) of its own buffers
__global__ void k_check_index(const int* __restrict__ idx, const long long* __restrict__ bound, int n,
                              int* __restrict__ out, unsigned int* __restrict__ flags) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  uint32_t err = 0;
  out[i] = chk(idx[i], (int64_t)bound[i], err);
  flags[i] = err;
}

}  // namespace gb

extern "C" int gbmc_build_checked(void) { return gb::kChecked ? 1 : 0; }

extern "C" gbmc_status gbmc_check_index(int device, const int* idx, const int64_t* bound, int n,
                                        int* out, uint32_t* flags) {
  if (n < 0 || (n > 0 && (!idx || !bound || !out || !flags))) return GBMC_ERR_ARG;
  if (n == 0) return GBMC_OK;
  if (cudaSetDevice(device) != cudaSuccess) return GBMC_ERR_CUDA;
  // one allocation: bounds (8 B), indices, results, flags (4 B each) per pair
  const size_t bytes = (size_t)n * (8 + 4 + 4 + 4);
  char* d = nullptr;
  if (cudaMalloc((void**)&d, bytes) != cudaSuccess) return GBMC_ERR_OOM;
  long long* d_bound = reinterpret_cast<long long*>(d);
  int* d_idx = reinterpret_cast<int*>(d + (size_t)n * 8);
  int* d_out = d_idx + n;
  unsigned int* d_flags = reinterpret_cast<unsigned int*>(d_out + n);
  std::vector<long long> hb(bound, bound + n);
  gbmc_status st = GBMC_OK;
  if (cudaMemcpy(d_bound, hb.data(), (size_t)n * 8, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d_idx, idx, (size_t)n * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
    st = GBMC_ERR_CUDA;
  } else {
    gb::k_check_index<<<(n + 255) / 256, 256>>>(d_idx, d_bound, n, d_out, d_flags);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(out, d_out, (size_t)n * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(flags, d_flags, (size_t)n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      st = GBMC_ERR_CUDA;
  }
  cudaFree(d);
  return st;
}
