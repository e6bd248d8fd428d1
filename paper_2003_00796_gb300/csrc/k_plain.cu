// k_plain.cu -- the plain one-history-per-thread kernel: each thread runs whole
// histories (grid-stride over the run's history ids), keeping secondaries on a
// per-thread LIFO stack in local memory. This is the GPU transcription of the
// paper's history loop (Sec. 4.1, Fig. "flowTally"; per-type stacks of Sec. 5.2
// become one per-thread stack), and the baseline the wavefront kernels are
// measured against. One launch covers a whole run; each history scores into the
// tile of its batch.
#include "gbmc_internal.h"
#include "transport.cuh"

namespace gb {

// stage the FP32 tables into shared memory (16-byte vector copies)
// stage both table regions (the whole blob) into shared memory
__device__ __forceinline__ void stage_tables(const DevProblem& P, float* stab) {
  const int n = P.tab_e_off + P.tab_e_floats;
  const int n4 = n >> 2;
  const float4* src = reinterpret_cast<const float4*>(P.tab);
  float4* dst = reinterpret_cast<float4*>(stab);
  for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
  for (int i = (n4 << 2) + threadIdx.x; i < n; i += blockDim.x) stab[i] = __ldg(P.tab + i);
  __syncthreads();
}

__device__ __forceinline__ void track_init(Track& t, const DevProblem& P, const float* stab) {
  t.P = &P; t.J = &P.job; t.tab_g = stab; t.tab_e = stab + P.tab_e_off;
  t.tile = P.job.tile; t.pa = nullptr; t.pe = 0.0f;
  t.c_tent = t.c_real = t.c_estep = t.c_cross = t.c_hard = t.c_part = 0;
  t.l_src = t.l_esc = t.l_pair = 0.0;
  t.err = 0;
  t.mode = M_TALLY; t.wv = nullptr; t.G = 0.0f;
  t.check = false; t.l_dep = 0.0;
  t.vr = false;
}

// warp-reduce the per-thread counters and ledger, one atomic per warp
__device__ __forceinline__ void track_commit(Track& t) {
  const DevProblem& P = *t.P;
  score_flush(t);
  __syncwarp();
  const unsigned full = 0xffffffffu;
  uint32_t c[NCOUNT] = {t.c_tent, t.c_real, t.c_estep, t.c_cross, t.c_hard, t.c_part};
  double l[3] = {t.l_src, t.l_esc, t.l_pair};
#pragma unroll
  for (int k = 0; k < NCOUNT; ++k) c[k] = __reduce_add_sync(full, c[k]);
#pragma unroll
  for (int k = 0; k < 3; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) l[k] += __shfl_xor_sync(full, l[k], o);
  const uint32_t e = __reduce_or_sync(full, t.err);
  if ((threadIdx.x & 31) == 0) {
#pragma unroll
    for (int k = 0; k < NCOUNT; ++k)
      if (c[k]) atomicAdd(P.counters + k, (unsigned long long)c[k]);
    atomicAdd(P.ledger + 0, l[0]);
    atomicAdd(P.ledger + 2, l[1]);
    atomicAdd(P.ledger + 3, l[2]);
    if (e) atomicOr(P.err, e);
  }
}

// CHECK: the per-history energy ledger (FP64): for every history, source
// energy = deposits + escapes + 2 mc^2 (pair productions - annihilations); the
// largest relative residual over the run goes to ledger[4] and the number of
// histories checked to ledger[5]
// VR: weighted particles (variance reduction); without it every weight is 1
template <int CAP, bool CHECK, bool VR>
__global__ void __launch_bounds__(256) k_plain(const DevProblem P) {
  extern __shared__ float4 smem4[];
  float* stab = reinterpret_cast<float*>(smem4);
  stage_tables(P, stab);
  Track t;
  track_init(t, P, stab);
  t.check = CHECK;
  t.vr = VR;
  StackSink<CAP> st;
  double worst = 0.0, n_checked = 0.0;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < P.job.run_n; h += stride) {
    const double s0 = t.l_src, d0 = t.l_dep, e0 = t.l_esc, p0 = t.l_pair;
    Live p;
    primary(t, P.job.run_first + (uint32_t)h, p);
    t.l_src += p.E;
    for (int guard = 0; guard < (1 << 20); ++guard) {
      track_to_death(t, st, p);
      if (st.sp == 0) break;
      live_from(p, st.s[--st.sp]);
      if (!VR) p.wt = 1.0f;
    }
    if (CHECK) {
      const double src = t.l_src - s0;
      const double res = src - ((t.l_dep - d0) + (t.l_esc - e0) + (t.l_pair - p0));
      worst = fmax(worst, fabs(res) / src);
      n_checked += 1.0;
    }
  }
  if (CHECK) {
    // a non-negative double orders like its bit pattern
    atomicMax(reinterpret_cast<unsigned long long*>(P.ledger + 4),
              (unsigned long long)__double_as_longlong(worst));
    atomicAdd(P.ledger + 5, n_checked);
  }
  track_commit(t);
}

// ---------------------------------------------------------------------------
// Path-replay adjoint: each thread takes whole histories and runs each one
// twice from its Philox key (the same random numbers, so the same path):
// first summing G = sum of deposits e w_v, then scattering G times the
// likelihood-ratio score of every tentative photon collision, and the explicit
// -e w_v / rho_v of every deposit, into the batch tile. Recomputation instead
// of storing paths; the job's tiles hold the gradient here.
// ---------------------------------------------------------------------------
template <int CAP>
__device__ __forceinline__ void plain_history(Track& t, StackSink<CAP>& st, uint32_t hist) {
  Live p;
  primary(t, hist, p);
  st.sp = 0;
  for (int guard = 0; guard < (1 << 20); ++guard) {
    track_to_death(t, st, p);
    if (st.sp == 0) break;
    live_from(p, st.s[--st.sp]);
    p.wt = 1.0f;   // the adjoint runs analog histories
  }
}

template <int CAP>
__global__ void __launch_bounds__(256) k_adjoint(const DevProblem P, const float* __restrict__ wv) {
  extern __shared__ float4 smem4[];
  float* stab = reinterpret_cast<float*>(smem4);
  stage_tables(P, stab);
  Track t;
  track_init(t, P, stab);
  t.wv = wv;
  StackSink<CAP> st;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  for (uint64_t h = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; h < P.job.run_n; h += stride) {
    const uint32_t hist = P.job.run_first + (uint32_t)h;
    t.mode = M_G_SUM;
    t.G = 0.0f;
    plain_history(t, st, hist);
    t.mode = M_SCATTER;
    plain_history(t, st, hist);
    score_flush(t);
  }
  track_commit(t);
}

cudaError_t launch_adjoint(const DevProblem& P, const float* wv, int grid, int block, cudaStream_t s) {
  const size_t smem = plain_smem_bytes(P);
  auto kern = k_adjoint<48>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(P, wv);
  return cudaGetLastError();
}

// w_v = g_v / (rho_v V) in FP32 from dL/dD (FP64)
__global__ void k_adjoint_weights(const double* __restrict__ g, const float* __restrict__ rho,
                                  int64_t nvox, double inv_vol, float* __restrict__ wv) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nvox; i += stride)
    wv[i] = (float)(g[i] * inv_vol / (double)rho[i]);
}

cudaError_t launch_adjoint_weights(const double* g, const float* rho, int64_t nvox, double vol,
                                   float* wv, cudaStream_t s) {
  const int grid = (int)std::min<int64_t>((nvox + 255) / 256, 152 * 8);
  k_adjoint_weights<<<std::max(grid, 1), 256, 0, s>>>(g, rho, nvox, 1.0 / vol, wv);
  return cudaGetLastError();
}

size_t plain_smem_bytes(const DevProblem& P) {
  return ((size_t)(P.tab_e_off + P.tab_e_floats) * 4 + 15) & ~(size_t)15;
}

cudaError_t launch_plain(const DevProblem& P, int grid, int block, cudaStream_t s, bool check) {
  const size_t smem = plain_smem_bytes(P);
  auto kern = P.vr_on ? (check ? k_plain<48, true, true> : k_plain<48, false, true>)
                      : (check ? k_plain<48, true, false> : k_plain<48, false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(P);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// First real interaction of each primary photon (cross-engine check)
// ---------------------------------------------------------------------------
__global__ void k_first_interaction(const DevProblem P, uint32_t hist0, int n, float* xyz,
                                    int* type) {
  extern __shared__ float4 smem4[];
  float* stab = reinterpret_cast<float*>(smem4);
  stage_tables(P, stab);
  Track t;
  track_init(t, P, stab);
  for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
    Live p;
    primary(t, hist0 + (uint32_t)h, p);
    int ty = 0;
    const GridPos gp = egrid(t, p.E);
    const float mbar = exp2_tab(t.tab_g + P.off_major, gp);
    for (int it = 0; it < kCapWoodcock; ++it) {
      const U4 wb = rng_block(p.rng, rng_take_blocks(p.rng, 1u), P.job.keys);
      const float s = neg_log(word_to_uniform(wb.x)) / mbar;
      p.x = fmaf(s, p.u, p.x); p.y = fmaf(s, p.v, p.y); p.z = fmaf(s, p.w, p.z);
      int ix, iy, iz;
      const int vox = locate(P.job, p.x, p.y, p.z, p.u, p.v, p.w, ix, iy, iz);
      if (vox < 0) break;
      const int m = P.job.mat[vox];
      const float mum = exp2_tab(tq(t, Q_MU_TOT, m), gp);
      if (word_to_uniform(wb.y) * mbar >= P.job.rho[vox] * mum) continue;
      const float co = exp2_tab(tq(t, Q_MU_CO, m), gp);
      const float pe = exp2_tab(tq(t, Q_MU_PE, m), gp);
      const float ray = exp2_tab(tq(t, Q_MU_RAY, m), gp);
      const float c = word_to_uniform(wb.z) * mum;
      ty = (c < co) ? 1 : (c < co + pe) ? 2 : (c < co + pe + ray || p.E <= 2.0f * kMec2f) ? 3 : 4;
      break;
    }
    type[h] = ty;
    xyz[3 * h + 0] = ty ? p.x : 0.0f;
    xyz[3 * h + 1] = ty ? p.y : 0.0f;
    xyz[3 * h + 2] = ty ? p.z : 0.0f;
  }
}

cudaError_t launch_first_interactions(const DevProblem& P, uint32_t hist0, int n, float* xyz,
                                      int* type, cudaStream_t s) {
  const size_t smem = plain_smem_bytes(P);
  cudaError_t e = cudaFuncSetAttribute(k_first_interaction,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int block = 256, grid = (n + block - 1) / block;
  k_first_interaction<<<grid, block, smem, s>>>(P, hist0, n, xyz, type);
  return cudaGetLastError();
}

}  // namespace gb
