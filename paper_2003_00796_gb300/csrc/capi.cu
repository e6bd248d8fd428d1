// capi.cu -- the C ABI of include/gbmc.h: context, inputs, the batch loop of a
// run, and the read-back of dose, variance and statistics.
//
// A run of N histories is split into K batches (batch k holds histories
// [first + floor(kN/K), first + floor((k+1)N/K))); each batch is one transport
// launch into the FP32 tile followed by one flush into the FP64 accumulators.
// This is the GPU form of the paper's tally treatment (Sec. 4.3: partial
// counters summed, then Eq. 1-2); the batch estimator gives the variance.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>
#include <vector>

#include "gbmc_internal.h"

using namespace gb;

// queue capacity: 16 Mi particles per queue, 5 queues of 64-byte records = 5.4 GB
static constexpr int kDefaultQueueCap = 1 << 24;

// one job of the last batched run (device memory owned by the context)
struct BatchJob {
  int64_t nvox = 0, stride = 0;
  double vol = 0.0;
  uint8_t* d_mat = nullptr;
  float* d_rho = nullptr;
  float* d_major = nullptr;
  float* d_bins = nullptr;
  int* d_alias = nullptr;
  float* d_tile = nullptr;
  double* d_s12 = nullptr;     // S1 | S2, stride doubles each
  double* d_inv_n = nullptr;
  uint64_t n_hist = 0;
  int K = 0;
  int n_bins = -1;             // source bins held in d_bins / d_alias
};

struct gbmc_ctx {
  int device = -1;
  bool host_only = false;
  gbmc_options opt{};
  std::string err;
  int sm_count = 0;
  // device memory of the problem-sized buffers (all allocated by dalloc):
  // bytes held, per buffer, and the context's limit (0: none)
  size_t mem_limit = 0, mem_used = 0;
  std::unordered_map<void*, size_t> mem_held;
  // materials and tables
  bool have_mat = false;
  std::vector<gbmc_material> mats;
  gbmc_transport tp{};
  Tables T;
  float* d_tab = nullptr;
  // phantom
  bool have_ph = false;
  int nx = 0, ny = 0, nz = 0;
  double dx = 0, dy = 0, dz = 0;
  int64_t nvox = 0;
  int64_t nvox_alloc = 0;      // voxels the phantom and tally buffers were allocated for
  unsigned int* d_valid = nullptr;   // phantom validation: bad count, per-material max density
  uint8_t* d_mat = nullptr;
  float* d_rho = nullptr;
  double rho_max[GBMC_MAX_MAT] = {};
  bool have_maj = false;       // photon majorant from fixed densities (gbmc_set_majorant)
  gbmc_vr vr{1.0, 1.0, 0.0, 0.0, 1};   // variance reduction (off)
  double rho_maj[GBMC_MAX_MAT] = {};
  // adjoint scratch: gradient S1, S2 (tile_stride doubles each), counters,
  // ledger and error flag of the replays; w_v (tile_stride floats)
  double* d_adj = nullptr;
  float* d_wv = nullptr;
  float* d_gbuf = nullptr;     // G_h per history of the wavefront adjoint's chunk
  uint64_t gbuf_len = 0;
  int64_t adj_stride = 0;
  // source
  bool have_src = false;
  gbmc_source src{};
  float* d_bins = nullptr;     // prob[n], edges[n+1] (floats), then alias ints
  int* d_alias = nullptr;
  // tally: K batch tiles of tile_stride floats (nvox rounded up to 4), FP64 sums
  float* d_tile = nullptr;
  int64_t tile_stride = 0;
  double* d_s1 = nullptr;
  double* d_s2 = nullptr;
  double* d_inv_n = nullptr;   // 1 / n_k of the current run's batches
  double* d_out = nullptr;     // 2 * nvox scratch for get_dose with host outputs
  uint64_t n_hist = 0, k_batches = 0;
  // wavefront queues: photon and charged, input and output
  float* d_qmem = nullptr;
  int q_cap = 0;
  unsigned int* d_qcnt = nullptr;
  unsigned int* h_qcnt = nullptr;  // pinned
  PassState* d_pass = nullptr;     // pass state written by the pass-control kernel
  PassState* h_pass = nullptr;     // pinned copy
  cudaStream_t cap_stream = nullptr;   // private streams for graph capture (the pass
  cudaStream_t cap_stream2 = nullptr;  // loop's photon branch is captured on the second)
  unsigned long long* d_loop = nullptr;  // graph loop iterations, passes with work (device)
  // instantiated pass loops of recent wavefront runs, with the launch
  // parameters each was built with (most recent first)
  std::vector<std::pair<std::vector<unsigned char>, cudaGraphExec_t>> wf_graphs;
  uint64_t graph_launches = 0;
  uint64_t n_kernels = 0;           // kernel launches for gbmc_run (incl. graph replays)
  uint64_t batch_prim[2] = {0, 0};  // batched run: primaries per particle class
  uint64_t batch_hist = 0, batch_k = 0;   // histories and batches of batched runs (statistics)
  std::vector<BatchJob> batch;      // jobs of the last batched run
  bool batch_ready = false;         // ... which completed (every job buffer in place)
  int batch_ncls[2] = {-1, -1};     // its jobs per particle class
  DevJob* d_jobs = nullptr;
  uint64_t* d_cls_first = nullptr;  // both classes' prefix arrays
  int* d_cls_job = nullptr;
  double* d_bout = nullptr;         // host-output scratch of gbmc_get_job_dose
  int64_t bout_len = 0;
  // bookkeeping (device)
  unsigned long long* d_counters = nullptr;
  double* d_ledger = nullptr;  // e_src, e_dep, e_esc, e_pair_net, checked: max residual, count
  unsigned int* d_err = nullptr;
  cudaStream_t last_stream = nullptr;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timed = false;
  // per-launch timing (opt.timing): event pairs, folded into the sums on read
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<int, int>> ev_transport, ev_flush, ev_photon, ev_drain;   // indices into ev_pool
  size_t ev_used = 0;
  double transport_ms = 0.0, flush_ms = 0.0, photon_ms = 0.0, drain_ms = 0.0;
  uint64_t n_transport = 0, n_flush = 0, n_photon = 0, n_drain = 0;
};

// next free event of the pool (grown on demand)
static cudaError_t pool_event(gbmc_ctx* ctx, int* idx) {
  if (ctx->ev_used == ctx->ev_pool.size()) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    ctx->ev_pool.push_back(e);
  }
  *idx = (int)ctx->ev_used++;
  return cudaSuccess;
}

// fold recorded launch timings into the sums (the stream must be complete)
static cudaError_t fold_timings(gbmc_ctx* ctx) {
  for (auto& pr : ctx->ev_transport) {
    float ms = 0.f;
    cudaError_t r = cudaEventElapsedTime(&ms, ctx->ev_pool[pr.first], ctx->ev_pool[pr.second]);
    if (r != cudaSuccess) return r;
    ctx->transport_ms += ms;
  }
  for (auto& pr : ctx->ev_flush) {
    float ms = 0.f;
    cudaError_t r = cudaEventElapsedTime(&ms, ctx->ev_pool[pr.first], ctx->ev_pool[pr.second]);
    if (r != cudaSuccess) return r;
    ctx->flush_ms += ms;
  }
  for (auto& pr : ctx->ev_photon) {
    float ms = 0.f;
    cudaError_t r = cudaEventElapsedTime(&ms, ctx->ev_pool[pr.first], ctx->ev_pool[pr.second]);
    if (r != cudaSuccess) return r;
    ctx->photon_ms += ms;
  }
  for (auto& pr : ctx->ev_drain) {
    float ms = 0.f;
    cudaError_t r = cudaEventElapsedTime(&ms, ctx->ev_pool[pr.first], ctx->ev_pool[pr.second]);
    if (r != cudaSuccess) return r;
    ctx->drain_ms += ms;
  }
  ctx->n_transport += ctx->ev_transport.size();
  ctx->n_flush += ctx->ev_flush.size();
  ctx->n_photon += ctx->ev_photon.size();
  ctx->n_drain += ctx->ev_drain.size();
  ctx->ev_transport.clear();
  ctx->ev_flush.clear();
  ctx->ev_photon.clear();
  ctx->ev_drain.clear();
  ctx->ev_used = 0;
  return cudaSuccess;
}

static gbmc_status fail(gbmc_ctx* c, gbmc_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

static gbmc_status cuda_fail(gbmc_ctx* c, cudaError_t e, const char* where) {
  return fail(c, GBMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
  do {                                                             \
    cudaError_t e_ = (call);                                       \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);       \
  } while (0)

// a problem-sized buffer leaves the context's memory account
static void mem_release(gbmc_ctx* ctx, void* p) {
  auto it = ctx->mem_held.find(p);
  if (it == ctx->mem_held.end()) return;
  ctx->mem_used -= it->second;
  ctx->mem_held.erase(it);
}

// (re)allocate a problem-sized buffer of n elements: the old one is freed,
// and a request beyond the context's memory limit fails like cudaMalloc
template <class T>
static gbmc_status dalloc(gbmc_ctx* ctx, T** p, size_t n) {
  if (*p) { mem_release(ctx, *p); cudaFree(*p); *p = nullptr; }
  if (n == 0) return GBMC_OK;
  const size_t bytes = n * sizeof(T);
  if (ctx->mem_limit && ctx->mem_used + bytes > ctx->mem_limit)
    return fail(ctx, GBMC_ERR_OOM, "device memory limit of the context: " + std::to_string(bytes) +
                                       " bytes asked with " + std::to_string(ctx->mem_used) + " of " +
                                       std::to_string(ctx->mem_limit) + " held");
  cudaError_t e = cudaMalloc((void**)p, bytes);
  if (e != cudaSuccess) { *p = nullptr; return fail(ctx, GBMC_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e)); }
  ctx->mem_used += bytes;
  ctx->mem_held[(void*)*p] = bytes;
  return GBMC_OK;
}

template <class T>
static gbmc_status upload(gbmc_ctx* ctx, T** d, const T* h, size_t n) {
  gbmc_status st = dalloc(ctx, d, n);
  if (st != GBMC_OK) return st;
  if (n) CK(cudaMemcpy(*d, h, n * sizeof(T), cudaMemcpyHostToDevice));
  return GBMC_OK;
}

// upload into an existing buffer of the same size (keep = the caller knows
// it has n elements), else into a new one
template <class T>
static gbmc_status upload_keep(gbmc_ctx* ctx, T** d, const T* h, size_t n, bool keep) {
  if (!(keep && *d && n)) return upload(ctx, d, h, n);
  CK(cudaMemcpy(*d, h, n * sizeof(T), cudaMemcpyHostToDevice));
  return GBMC_OK;
}

extern "C" {

gbmc_status gbmc_create(gbmc_ctx** out, int device, const gbmc_options* opt) {
  if (!out) return GBMC_ERR_ARG;
  *out = nullptr;
  gbmc_ctx* ctx = new (std::nothrow) gbmc_ctx();
  if (!ctx) return GBMC_ERR_OOM;
  if (opt) ctx->opt = *opt;
  if (ctx->opt.n_batches == 0) ctx->opt.n_batches = 40;
  if (ctx->opt.block == 0) ctx->opt.block = 256;
  if (ctx->opt.stack_cap == 0) ctx->opt.stack_cap = 48;
  if (ctx->opt.photon_budget == 0) ctx->opt.photon_budget = 16;
  if (ctx->opt.charged_budget == 0) ctx->opt.charged_budget = 32;
  if (ctx->opt.n_batches < 2 || ctx->opt.n_batches > GBMC_MAX_BATCHES || ctx->opt.block < 32 ||
      ctx->opt.block > 256 ||
      (ctx->opt.block & 31) || ctx->opt.kernel < 0 || ctx->opt.kernel > 1 ||
      ctx->opt.photon_budget < 1 || ctx->opt.charged_budget < 1 || ctx->opt.pass_target < 0 ||
      ctx->opt.queue_cap < 0 || ctx->opt.blocks_per_sm < 0 || ctx->opt.stack_cap != 48 ||
      (ctx->opt.ledger_check != 0 && ctx->opt.kernel != GBMC_KERNEL_PLAIN)) {
    delete ctx;
    return GBMC_ERR_ARG;
  }
  ctx->device = device;
  if (device < 0) {  // host-only context: tables and host helpers, no GPU
    ctx->host_only = true;
    *out = ctx;
    return GBMC_OK;
  }
  cudaError_t e = cudaSetDevice(device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_counters, sizeof(unsigned long long) * NCOUNT);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_ledger, sizeof(double) * 6);
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_err, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMalloc((void**)&ctx->d_loop, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(ctx->d_loop, 0, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev0);
  if (e == cudaSuccess) e = cudaEventCreate(&ctx->ev1);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * NCOUNT);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_ledger, 0, sizeof(double) * 6);
  if (e == cudaSuccess) e = cudaMemset(ctx->d_err, 0, sizeof(unsigned int));
  if (e != cudaSuccess) {
    gbmc_destroy(ctx);
    return GBMC_ERR_CUDA;
  }
  *out = ctx;
  return GBMC_OK;
}

static void free_batch(gbmc_ctx* ctx) {
  for (BatchJob& b : ctx->batch) {
    void* ptrs[] = {b.d_mat, b.d_rho, b.d_major, b.d_bins, b.d_alias, b.d_tile, b.d_s12, b.d_inv_n};
    for (void* q : ptrs) if (q) { mem_release(ctx, q); cudaFree(q); }
  }
  ctx->batch.clear();
  ctx->batch_ready = false;
  void* ptrs[] = {ctx->d_jobs, ctx->d_cls_first, ctx->d_cls_job, ctx->d_bout};
  for (void* q : ptrs) if (q) { mem_release(ctx, q); cudaFree(q); }
  ctx->d_jobs = nullptr; ctx->d_cls_first = nullptr; ctx->d_cls_job = nullptr; ctx->d_bout = nullptr;
  ctx->bout_len = 0;
  ctx->batch_ncls[0] = ctx->batch_ncls[1] = -1;
}

void gbmc_destroy(gbmc_ctx* ctx) {
  if (!ctx) return;
  if (!ctx->host_only) {
    cudaSetDevice(ctx->device);
    free_batch(ctx);
    void* ptrs[] = {ctx->d_tab, ctx->d_mat, ctx->d_rho, ctx->d_bins, ctx->d_alias, ctx->d_tile,
                    ctx->d_s1, ctx->d_s2, ctx->d_out, ctx->d_counters, ctx->d_ledger, ctx->d_err,
                    ctx->d_inv_n, ctx->d_qmem, ctx->d_qcnt, ctx->d_adj, ctx->d_wv, ctx->d_gbuf,
                    ctx->d_valid};
    for (void* p : ptrs) if (p) cudaFree(p);
    if (ctx->h_qcnt) cudaFreeHost(ctx->h_qcnt);
    if (ctx->h_pass) cudaFreeHost(ctx->h_pass);
    if (ctx->d_pass) cudaFree(ctx->d_pass);
    for (auto& g : ctx->wf_graphs) cudaGraphExecDestroy(g.second);
    if (ctx->d_loop) cudaFree(ctx->d_loop);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
    if (ctx->ev0) cudaEventDestroy(ctx->ev0);
    if (ctx->ev1) cudaEventDestroy(ctx->ev1);
    for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  }
  delete ctx;
}

const char* gbmc_last_error(const gbmc_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

gbmc_status gbmc_set_mem_limit(gbmc_ctx* ctx, uint64_t limit_bytes) {
  if (!ctx) return GBMC_ERR_ARG;
  ctx->mem_limit = (size_t)limit_bytes;
  return GBMC_OK;
}

gbmc_status gbmc_mem_info(const gbmc_ctx* ctx, uint64_t* held_bytes, uint64_t* limit_bytes) {
  if (!ctx || !held_bytes || !limit_bytes) return GBMC_ERR_ARG;
  *held_bytes = ctx->mem_used;
  *limit_bytes = ctx->mem_limit;
  return GBMC_OK;
}

static gbmc_status upload_tables(gbmc_ctx* ctx) {
  if (ctx->host_only) return GBMC_OK;
  // until the new blob is on the device the context has no usable materials
  // (a failed upload leaves them unset: gbmc_set_materials again)
  const bool had = ctx->have_mat;
  ctx->have_mat = false;
  CK(cudaSetDevice(ctx->device));
  gbmc_status s = dalloc(ctx, &ctx->d_tab, ctx->T.data.size() + 4);
  if (s != GBMC_OK) return s;
  CK(cudaMemcpy(ctx->d_tab, ctx->T.data.data(), ctx->T.data.size() * sizeof(float), cudaMemcpyHostToDevice));
  ctx->have_mat = had;
  return GBMC_OK;
}

gbmc_status gbmc_set_materials(gbmc_ctx* ctx, const gbmc_material* mats, int n_mat,
                               const gbmc_transport* tp, double e_max) {
  if (!ctx || !mats || !tp) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (n_mat < 1 || n_mat > GBMC_MAX_MAT) return fail(ctx, GBMC_ERR_ARG, "n_mat out of range");
  if (!(e_max > 0.02 && e_max <= 1000.0)) return fail(ctx, GBMC_ERR_ARG, "e_max out of range");
  const bool tp_ok = tp->eabs_g >= 1e-3 && tp->eabs_e >= 1e-3 && tp->wcc >= 1e-3 && tp->wcr >= 1e-3 &&
                     tp->c1 > 0.0 && tp->step_frac > 0.0 && tp->step_frac < 1.0 && tp->step_vox > 0.0;
  if (!tp_ok) return fail(ctx, GBMC_ERR_ARG, "transport parameters out of range");
  std::vector<gbmc_material> m(mats, mats + n_mat);
  for (auto& x : m) {
    if (x.n_el < 1 || x.n_el > GBMC_MAX_EL || !(x.I_eV > 0.0)) return fail(ctx, GBMC_ERR_ARG, "bad material");
    double s = 0.0;
    for (int i = 0; i < x.n_el; ++i) {
      if (x.Z[i] < 1 || x.Z[i] > 100 || !(x.A[i] > 0.0) || !(x.w[i] >= 0.0)) return fail(ctx, GBMC_ERR_ARG, "bad element");
      s += x.w[i];
    }
    if (!(s > 0.0)) return fail(ctx, GBMC_ERR_ARG, "mass fractions sum to zero");
    for (int i = 0; i < x.n_el; ++i) x.w[i] /= s;
  }
  ctx->mats = m;
  ctx->tp = *tp;
  build_tables(ctx->T, ctx->mats.data(), n_mat, *tp, e_max * 1.001, 384, 512);
  ctx->have_maj = false;   // new materials: the majorant follows the phantom again
  if (ctx->have_ph) build_majorant(ctx->T, ctx->rho_max);
  ctx->have_mat = true;
  return upload_tables(ctx);
}

gbmc_status gbmc_load_phantom(gbmc_ctx* ctx, int nx, int ny, int nz, double dx, double dy, double dz,
                              const uint8_t* mat, const float* rho, int ptr_kind) {
  if (!ctx || !mat || !rho) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (!ctx->have_mat) return fail(ctx, GBMC_ERR_STATE, "gbmc_set_materials first");
  if (nx < 1 || ny < 1 || nz < 1 || !(dx > 0) || !(dy > 0) || !(dz > 0))
    return fail(ctx, GBMC_ERR_ARG, "bad grid");
  if (ptr_kind != GBMC_PTR_HOST && ptr_kind != GBMC_PTR_DEVICE) return fail(ctx, GBMC_ERR_ARG, "bad ptr_kind");
  const int64_t nvox = (int64_t)nx * ny * nz;
  if (nvox >= ((int64_t)1 << 31)) return fail(ctx, GBMC_ERR_ARG, "grid too large (>= 2^31 voxels)");
  CK(cudaSetDevice(ctx->device));
  if (ctx->last_stream) CK(cudaStreamSynchronize(ctx->last_stream));   // runs read the old phantom
  const int n_mat = (int)ctx->mats.size();
  gbmc_status s;
  // the phantom and its tally buffers keep their device memory when the voxel
  // count is unchanged (loading phantom after phantom then allocates nothing);
  // until the new phantom is in place and valid the context has none
  const bool same = ctx->d_mat && ctx->nvox_alloc == nvox;
  ctx->have_ph = false;
  if (!same) {
    ctx->nvox_alloc = 0;
    if ((s = dalloc(ctx, &ctx->d_mat, (size_t)nvox + 16)) != GBMC_OK) return s;
    if ((s = dalloc(ctx, &ctx->d_rho, (size_t)nvox + 4)) != GBMC_OK) return s;
  }
  const cudaMemcpyKind kind = ptr_kind == GBMC_PTR_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpy(ctx->d_mat, mat, nvox, kind));
  CK(cudaMemcpy(ctx->d_rho, rho, nvox * sizeof(float), kind));
  // validated on the device: material ids below n_mat, finite positive
  // densities, and each material's largest density (for the majorant)
  if (!ctx->d_valid) CK(cudaMalloc((void**)&ctx->d_valid, sizeof(unsigned int) * (1 + GBMC_MAX_MAT)));
  CK(cudaMemset(ctx->d_valid, 0, sizeof(unsigned int) * (1 + GBMC_MAX_MAT)));
  CK(launch_validate_phantom(ctx->d_mat, ctx->d_rho, nvox, n_mat, ctx->d_valid,
                             reinterpret_cast<float*>(ctx->d_valid + 1), 0));
  unsigned int hb[1 + GBMC_MAX_MAT];
  CK(cudaMemcpy(hb, ctx->d_valid, sizeof hb, cudaMemcpyDeviceToHost));
  if (hb[0]) return fail(ctx, GBMC_ERR_ARG, "phantom voxel with bad material id or density");
  double rmax[GBMC_MAX_MAT] = {};
  for (int m = 0; m < n_mat; ++m) { float f; std::memcpy(&f, &hb[1 + m], 4); rmax[m] = f; }
  for (int m = 0; m < n_mat; ++m)
    if (ctx->have_maj && rmax[m] > ctx->rho_maj[m])
      return fail(ctx, GBMC_ERR_ARG, "phantom density above the fixed majorant density of its material");
  ctx->nx = nx; ctx->ny = ny; ctx->nz = nz; ctx->dx = dx; ctx->dy = dy; ctx->dz = dz;
  ctx->nvox = nvox;
  for (int m = 0; m < GBMC_MAX_MAT; ++m) ctx->rho_max[m] = m < n_mat ? rmax[m] : 0.0;
  build_majorant(ctx->T, ctx->have_maj ? ctx->rho_maj : ctx->rho_max);
  if ((s = upload_tables(ctx)) != GBMC_OK) return s;
  ctx->tile_stride = (nvox + 3) & ~(int64_t)3;
  if (!same) {
    const size_t ntile = (size_t)ctx->tile_stride * (size_t)ctx->opt.n_batches;
    if ((s = dalloc(ctx, &ctx->d_tile, ntile)) != GBMC_OK) return s;
    if ((s = dalloc(ctx, &ctx->d_s1, (size_t)ctx->tile_stride)) != GBMC_OK) return s;
    if ((s = dalloc(ctx, &ctx->d_s2, (size_t)ctx->tile_stride)) != GBMC_OK) return s;
    if ((s = dalloc(ctx, &ctx->d_inv_n, (size_t)ctx->opt.n_batches)) != GBMC_OK) return s;
    if ((s = dalloc(ctx, &ctx->d_out, 2 * (size_t)nvox)) != GBMC_OK) return s;
    ctx->nvox_alloc = nvox;
  }
  ctx->have_ph = true;
  return gbmc_reset_tally(ctx);   // clears the tiles and the FP64 sums
}

gbmc_status gbmc_build_alias(const double* weights, int n, float* prob, int* alias) {
  if (!weights || !prob || !alias || n < 1) return GBMC_ERR_ARG;
  double tot = 0.0;
  for (int i = 0; i < n; ++i) {
    if (!(weights[i] >= 0.0) || !std::isfinite(weights[i])) return GBMC_ERR_ARG;
    tot += weights[i];
  }
  if (!(tot > 0.0)) return GBMC_ERR_ARG;
  // Vose's construction: scaled weights n w_i / sum; small/large work lists
  std::vector<double> q(n);
  std::vector<int> small, large;
  for (int i = 0; i < n; ++i) {
    q[i] = weights[i] * n / tot;
    (q[i] < 1.0 ? small : large).push_back(i);
  }
  for (int i = 0; i < n; ++i) { prob[i] = 1.0f; alias[i] = i; }
  while (!small.empty() && !large.empty()) {
    const int s = small.back(); small.pop_back();
    const int l = large.back();
    prob[s] = (float)q[s];
    alias[s] = l;
    q[l] -= 1.0 - q[s];
    if (q[l] < 1.0) { large.pop_back(); small.push_back(l); }
  }
  for (int i : large) { prob[i] = 1.0f; alias[i] = i; }
  for (int i : small) { prob[i] = 1.0f; alias[i] = i; }   // round-off leftovers
  return GBMC_OK;
}

// validate a source against the tables and build its alias table: fb holds
// prob[n] then edges[n + 1] (floats), al the alias indices
static gbmc_status prepare_source(gbmc_ctx* ctx, const gbmc_source* src, std::vector<float>& fb,
                                  std::vector<int>& al) {
  if (src->particle < 0 || src->particle > 2 || src->shape < 0 || src->shape > 1)
    return fail(ctx, GBMC_ERR_ARG, "bad source particle/shape");
  if (src->n_bins < 0 || src->n_bins > GBMC_MAX_BINS) return fail(ctx, GBMC_ERR_ARG, "bad n_bins");
  const double emax = ctx->T.emax;
  fb.clear();
  al.clear();
  if (src->n_bins > 0) {
    if (!src->edges || !src->weights) return fail(ctx, GBMC_ERR_ARG, "null bins");
    const int n = src->n_bins;
    for (int i = 0; i < n; ++i)
      if (!(src->edges[i + 1] > src->edges[i])) return fail(ctx, GBMC_ERR_ARG, "edges not increasing");
    if (!(src->edges[0] > 0.0) || src->edges[n] > emax) return fail(ctx, GBMC_ERR_ARG, "spectrum outside table range");
    fb.resize(2 * n + 1);
    al.resize(n);
    if (gbmc_build_alias(src->weights, n, fb.data(), al.data()) != GBMC_OK)
      return fail(ctx, GBMC_ERR_ARG, "bad bin weights");
    for (int i = 0; i <= n; ++i) fb[n + i] = (float)src->edges[i];
  } else if (!(src->energy > 0.0) || src->energy > emax) {
    return fail(ctx, GBMC_ERR_ARG, "source energy outside table range");
  }
  return GBMC_OK;
}

gbmc_status gbmc_set_source(gbmc_ctx* ctx, const gbmc_source* src) {
  if (!ctx || !src) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (!ctx->have_mat) return fail(ctx, GBMC_ERR_STATE, "gbmc_set_materials first");
  std::vector<float> fb;
  std::vector<int> al;
  gbmc_status s = prepare_source(ctx, src, fb, al);
  if (s != GBMC_OK) return s;
  CK(cudaSetDevice(ctx->device));
  ctx->have_src = false;   // until the new source's alias table is in place
  if ((s = dalloc(ctx, &ctx->d_bins, fb.size())) != GBMC_OK) return s;
  if ((s = dalloc(ctx, &ctx->d_alias, al.size())) != GBMC_OK) return s;
  if (!fb.empty()) {
    CK(cudaMemcpy(ctx->d_bins, fb.data(), fb.size() * 4, cudaMemcpyHostToDevice));
    CK(cudaMemcpy(ctx->d_alias, al.data(), al.size() * 4, cudaMemcpyHostToDevice));
  }
  ctx->src = *src;
  ctx->src.edges = nullptr;
  ctx->src.weights = nullptr;
  ctx->have_src = true;
  return GBMC_OK;
}

// A pencil beam's coordinate as the device stores it (FP32), chosen so that
// the device's own FP32 locate (floor(x * (1/d)), geometry of Sec. 4.2.2)
// puts it in the voxel that the exact coordinate is in: floor(x0 / d) in FP64,
// the tie-break for a point on a plane with no motion across it. A decimal
// position on a voxel plane (7.2 cm on a 3 mm grid) is not representable in
// FP32, and its nearest float can fall on either side of the plane; the
// nudge is at most a few ulp (1e-7 cm), and makes the beam enter the same
// voxel column as the FP64 computation.
static float pencil_coord(double x0, double d, int n) {
  const double f64 = x0 / d;
  if (!(f64 >= 0.0) || f64 >= (double)n) return (float)x0;   // outside: nothing to match
  const int want = (int)std::floor(f64);
  const float id = (float)(1.0 / d);
  float x = (float)x0;
  for (int it = 0; it < 64; ++it) {
    const int got = (int)std::floor(x * id);
    if (got == want) break;
    x = std::nextafter(x, got < want ? INFINITY : -INFINITY);
  }
  return x;
}

static bool vr_on(const gbmc_vr& v) {
  return v.f_inel != 1.0 || v.f_brems != 1.0 || v.n_split_brems != 1;
}

static DevProblem make_problem(gbmc_ctx* ctx, uint64_t seed) {
  DevProblem P;
  std::memset(&P, 0, sizeof P);
  P.job.nx = ctx->nx; P.job.ny = ctx->ny; P.job.nz = ctx->nz; P.job.nxy = ctx->nx * ctx->ny;
  P.job.inv_nx = 1.0f / (float)ctx->nx; P.job.inv_nxy = 1.0f / (float)P.job.nxy;
  P.job.dx = (float)ctx->dx; P.job.dy = (float)ctx->dy; P.job.dz = (float)ctx->dz;
  P.job.idx = (float)(1.0 / ctx->dx); P.job.idy = (float)(1.0 / ctx->dy); P.job.idz = (float)(1.0 / ctx->dz);
  P.job.dmin = (float)std::min(ctx->dx, std::min(ctx->dy, ctx->dz));
  P.job.mat = ctx->d_mat; P.job.rho = ctx->d_rho;
  const Tables& T = ctx->T;
  P.tab = ctx->d_tab;
  P.tab_g_floats = tab_region_g(T.n_mat, T.nE);
  P.tab_e_off = tab_off_e(T.n_mat, T.nE);
  P.tab_e_floats = (int)T.data.size() - P.tab_e_off;
  for (int m = 0; m < GBMC_MAX_MAT; ++m)
    P.off_el[m] = (m < T.n_mat && T.off_el[m] >= 0) ? T.off_el[m] - P.tab_e_off : -1;
  P.n_mat = T.n_mat; P.nE = T.nE; P.nR = T.nR; P.nA = T.nA;
  P.lg0 = T.lg0; P.inv_d = T.inv_d;
  for (int m = 0; m < GBMC_MAX_MAT; ++m)
    for (int s = 0; s < 2; ++s) { P.lr0[m][s] = T.lr0[m][s]; P.inv_dr[m][s] = T.inv_dr[m][s]; }
  P.la0 = T.la0; P.inv_da = T.inv_da;
  P.off_major = T.off_major; P.off_soft = T.off_soft - P.tab_e_off;
  P.off_mpar = T.off_mpar - P.tab_e_off;
  for (int m = 0; m < GBMC_MAX_MAT; ++m) P.mats[m] = T.dmat[m];
  P.eabs_g = (float)ctx->tp.eabs_g; P.eabs_e = (float)ctx->tp.eabs_e;
  P.wcc = (float)ctx->tp.wcc; P.wcr = (float)ctx->tp.wcr;
  P.step_keep = (float)(1.0 - ctx->tp.step_frac);
  P.lg_keep = (float)std::log2(1.0 - ctx->tp.step_frac);
  P.lg_eabs_e = (float)std::log2(ctx->tp.eabs_e);
  P.vr_fi = (float)ctx->vr.f_inel; P.vr_fb = (float)ctx->vr.f_brems;
  P.vr_wlo = (float)ctx->vr.w_lo; P.vr_whi = (float)ctx->vr.w_hi;
  P.vr_split = ctx->vr.n_split_brems;
  P.vr_on = vr_on(ctx->vr) ? 1 : 0;
  P.job.step_len = (float)(ctx->tp.step_vox * std::min(ctx->dx, std::min(ctx->dy, ctx->dz)));
  P.job.particle = ctx->src.particle; P.job.shape = ctx->src.shape; P.job.n_bins = ctx->src.n_bins;
  P.job.x0 = (float)ctx->src.x0; P.job.y0 = (float)ctx->src.y0;
  if (ctx->src.shape == 0) {
    P.job.x0 = pencil_coord(ctx->src.x0, ctx->dx, ctx->nx);
    P.job.y0 = pencil_coord(ctx->src.y0, ctx->dy, ctx->ny);
  }
  P.job.hx = (float)ctx->src.hx; P.job.hy = (float)ctx->src.hy; P.job.energy = (float)ctx->src.energy;
  P.job.bin_prob = ctx->d_bins;
  P.job.bin_edges = ctx->d_bins ? ctx->d_bins + ctx->src.n_bins : nullptr;
  P.job.bin_alias = ctx->d_alias;
  P.job.keys = philox_keys((uint32_t)seed, (uint32_t)(seed >> 32));   // job id 0
  P.job.tile = ctx->d_tile;
  P.job.tile_stride = ctx->tile_stride;
  P.job.run_first = 0; P.job.run_n = 1; P.job.run_k = 1;
  P.counters = ctx->d_counters; P.ledger = ctx->d_ledger; P.err = ctx->d_err;
  return P;
}

static gbmc_status ready(gbmc_ctx* ctx) {
  if (!ctx) return GBMC_ERR_ARG;
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (!ctx->have_mat || !ctx->have_ph || !ctx->have_src)
    return fail(ctx, GBMC_ERR_STATE, "materials, phantom and source must be set before running");
  return GBMC_OK;
}

// one wave of resident blocks: blocks_per_sm (default: what the kernel's
// register budget lets stay resident, `resident`) blocks per SM
static int full_grid(gbmc_ctx* ctx, int64_t items, int resident = 2) {
  const int bps = ctx->opt.blocks_per_sm > 0 ? std::min(ctx->opt.blocks_per_sm, resident) : resident;
  const int64_t full = (int64_t)ctx->sm_count * bps;
  const int64_t need = (items + ctx->opt.block - 1) / ctx->opt.block;
  return (int)std::max<int64_t>(1, std::min(full, need));
}

// time one launch with two pool events on the run's stream (opt.timing)
#define TIMED(call, list)                                                  \
  do {                                                                     \
    int a_ = -1, b_ = -1;                                                  \
    if (ctx->opt.timing) {                                                 \
      CK(pool_event(ctx, &a_)); CK(pool_event(ctx, &b_));                  \
      CK(cudaEventRecord(ctx->ev_pool[a_], s));                            \
    }                                                                      \
    CK(call);                                                              \
    if (ctx->opt.timing) {                                                 \
      CK(cudaEventRecord(ctx->ev_pool[b_], s));                            \
      ctx->list.push_back({a_, b_});                                       \
    }                                                                      \
  } while (0)

// queue storage: 5 queues (photon/charged x in/out, deferred charged events)
// of cap particles, each record kQueueFields 4-byte words in four arrays of
// 16-byte field groups (the device side lays them out: ring_queue)
static gbmc_status ensure_queues(gbmc_ctx* ctx) {
  const int cap = ctx->opt.queue_cap > 0 ? ctx->opt.queue_cap : kDefaultQueueCap;
  if (ctx->d_qmem && ctx->q_cap == cap) return GBMC_OK;
  const size_t per = (size_t)cap;
  gbmc_status st = dalloc(ctx, &ctx->d_qmem, per * kQueueFields * 5);
  if (st != GBMC_OK) return st;
  // counters: appends (photons, charged, deferred), spare, work claims (photon, charged)
  if (!ctx->d_qcnt) {
    CK(cudaMalloc((void**)&ctx->d_qcnt, 8 * sizeof(unsigned int)));
    CK(cudaMemset(ctx->d_qcnt, 0, 8 * sizeof(unsigned int)));
  }
  if (!ctx->h_qcnt) CK(cudaMallocHost((void**)&ctx->h_qcnt, 4 * sizeof(unsigned int)));
  ctx->q_cap = cap;
  return GBMC_OK;
}

// wavefront run: queues of photons and charged particles, refilled with new
// primaries up to a target population, until every history is finished. The
// pass sizes are decided on the device (k_pass_ctl), and a run's passes are
// the body of a CUDA-graph while loop whose condition the control kernel sets:
// the host submits the whole run as one graph launch and returns without
// waiting (the loop ends on the device when the control kernel reports the
// run done, or after its pass cap, flagged). The instantiated graph is kept
// and launched again while the run's launch parameters are unchanged. With
// per-launch timing on, passes are launched one by one instead (the state is
// read after each, and kernels without work are not launched), so that every
// timed launch is a pass with work.

// the bytes of every launch parameter of the pass loop: the cached graph is
// reused only when they are identical
static void key_bytes(std::vector<unsigned char>& k, const void* v, size_t n) {
  const unsigned char* b = static_cast<const unsigned char*>(v);
  k.insert(k.end(), b, b + n);
}
#define key_add(k, v) key_bytes(k, &(v), sizeof(v))

static constexpr size_t kGraphCache = 4;   // pass loops kept (e.g. the adjoint's two replays)

static gbmc_status build_pass_graph(gbmc_ctx* ctx, const DevProblem& P, const WfRing& R, const PassCtl& c,
                                    int g_ph, int mb_ph, int g_ch, int blk_ch, int mb_ch, int g_kn,
                                    int g_dr, const float* wv,
                                    cudaGraphExec_t* out) {
  cudaGraph_t graph = nullptr;
  CK(cudaGraphCreate(&graph, 0));
  cudaGraphConditionalHandle h = 0;
  cudaError_t e = cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault);
  cudaGraphNodeParams cp = {};
  cp.type = cudaGraphNodeTypeConditional;
  cp.conditional.handle = h;
  cp.conditional.type = cudaGraphCondTypeWhile;
  cp.conditional.size = 1;
  cudaGraphNode_t node = nullptr;
  if (e == cudaSuccess) e = cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &cp);
  if (e == cudaSuccess) {
    // the loop body: one pass (photon, charged, knock kernels) and its control
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    // The photon kernel is a branch of its own, beside the charged kernel and
    // its deferred events: the two read different input queues and append to
    // the output queues through atomic counters only, so they can run at once,
    // and each fills the SMs that the other's tail leaves idle. The drain
    // kernel (which works only when the other three do not) and the control
    // kernel follow both.
    cudaStream_t cs = ctx->cap_stream, cs2 = ctx->cap_stream2;
    cudaEvent_t fork = nullptr, join = nullptr;
    e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join, cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t ce = cudaEventRecord(fork, cs);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs2, fork, 0);
      if (ce == cudaSuccess)
        ce = launch_wavefront_pass(P, true, R, ctx->d_pass, g_ph, ctx->opt.block, mb_ph, wv, cs2);
      if (ce == cudaSuccess) ce = cudaEventRecord(join, cs2);
      if (ce == cudaSuccess)
        ce = launch_wavefront_pass(P, false, R, ctx->d_pass, g_ch, blk_ch, mb_ch, wv, cs);
      if (ce == cudaSuccess) ce = launch_knock_pass(P, R, ctx->d_pass, g_kn, ctx->opt.block, wv, cs);
      if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cs, join, 0);
      if (ce == cudaSuccess) ce = launch_drain_pass(P, R, ctx->d_pass, g_dr, wv, cs);
      if (ce == cudaSuccess) ce = launch_pass_ctl(c, ctx->d_pass, ctx->d_qcnt, P.err, 0, ctx->d_loop, cs, h, 1);
      cudaGraph_t out = nullptr;
      const cudaError_t ee = cudaStreamEndCapture(cs, &out);
      e = ce != cudaSuccess ? ce : ee;
    }
    if (fork) cudaEventDestroy(fork);
    if (join) cudaEventDestroy(join);
  }
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "wavefront pass-loop graph");
  *out = exec;
  return GBMC_OK;
}

static gbmc_status run_wavefront(gbmc_ctx* ctx, DevProblem& P, cudaStream_t s,
                                 const float* wv = nullptr) {
  gbmc_status st = ensure_queues(ctx);
  if (st != GBMC_OK) return st;
  if (!ctx->d_pass) CK(cudaMalloc((void**)&ctx->d_pass, sizeof(PassState)));
  if (!ctx->h_pass) CK(cudaMallocHost((void**)&ctx->h_pass, sizeof(PassState)));
  if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
  if (!ctx->cap_stream2) CK(cudaStreamCreateWithFlags(&ctx->cap_stream2, cudaStreamNonBlocking));
  const int cap = ctx->q_cap;
  PassCtl c;
  if (P.jobs) {              // batched: primaries per class over the jobs
    c.n_prim[0] = ctx->batch_prim[0];
    c.n_prim[1] = ctx->batch_prim[1];
  } else {
    const int cls = (P.job.particle == GBMC_PHOTON) ? 0 : 1;
    c.n_prim[cls] = P.job.run_n;
    c.n_prim[cls ^ 1] = 0;
  }
  c.target = std::min<int64_t>(cap, std::max<int64_t>(1024, ctx->opt.pass_target > 0 ? ctx->opt.pass_target : cap / 2));
  c.drain = (int64_t)ctx->sm_count * 512;   // below this: the drain pass ends the run
  c.cap = cap;
  c.budget_g = ctx->opt.photon_budget;
  c.budget_e = std::min(ctx->opt.charged_budget, kCapEsteps - 1);
  c.max_passes = 1 << 20;   // far above any run's passes (2^32 histories: ~1e4)
  const WfRing R{ctx->d_qmem, ctx->d_qcnt, cap};
  const int bps = ctx->opt.blocks_per_sm;
  const int g_ph = full_grid(ctx, INT64_MAX / 2, bps >= 3 ? 3 : 2), mb_ph = bps > 0 ? bps : 2;
  // the charged kernel: one block per SM holding the threads of bps_ch blocks
  const int mb_ch = bps > 0 ? std::min(bps, 3) : 3;
  const int g_ch = ctx->sm_count, blk_ch = ctx->opt.block * mb_ch;
  const int g_kn = full_grid(ctx, INT64_MAX / 2, 3);
  const int g_dr = 2 * ctx->sm_count;   // the drain kernel: 2 blocks of 256 per SM
  CK(cudaMemsetAsync(ctx->d_pass, 0, sizeof(PassState), s));
  CK(launch_pass_ctl(c, ctx->d_pass, ctx->d_qcnt, P.err, 1, ctx->d_loop, s));
  ++ctx->n_kernels;
  if (ctx->opt.timing) {
    PassState& h = *ctx->h_pass;
    for (int pass = 0; pass < c.max_passes + 1; ++pass) {
      CK(cudaMemcpyAsync(&h, ctx->d_pass, sizeof(PassState), cudaMemcpyDeviceToHost, s));
      CK(cudaStreamSynchronize(s));
      if (h.done) break;
      const int n_ph = h.n_in[0] + h.n_new[0];
      const int n_ch = h.n_in[1] + h.n_new[1];
      if (h.drain) {
        TIMED(launch_drain_pass(P, R, ctx->d_pass, g_dr, wv, s), ev_drain);
        ++ctx->n_kernels;
      } else if (n_ph > 0) {
        TIMED(launch_wavefront_pass(P, true, R, ctx->d_pass, g_ph, ctx->opt.block, mb_ph, wv, s), ev_photon);
        ++ctx->n_kernels;
      }
      if (n_ch > 0 && !h.drain) {
        TIMED(launch_wavefront_pass(P, false, R, ctx->d_pass, g_ch, blk_ch, mb_ch, wv, s),
              ev_transport);
        TIMED(launch_knock_pass(P, R, ctx->d_pass, g_kn, ctx->opt.block, wv, s), ev_photon);
        ctx->n_kernels += 2;
      }
      CK(launch_pass_ctl(c, ctx->d_pass, ctx->d_qcnt, P.err, 0, ctx->d_loop, s));
      ++ctx->n_kernels;
    }
    if (!h.done) return fail(ctx, GBMC_ERR_DEVICE_LIMIT, "wavefront pass limit reached");
    return GBMC_OK;
  }
  std::vector<unsigned char> key;   // P is zero-filled before its fields are set
  key_add(key, P); key_add(key, R.qmem); key_add(key, R.cnt); key_add(key, R.cap);
  key_add(key, c); key_add(key, wv);
  key_add(key, g_ph); key_add(key, mb_ph); key_add(key, g_ch); key_add(key, mb_ch);
  key_add(key, g_kn); const int blk = ctx->opt.block;
  key_add(key, blk); key_add(key, blk_ch); key_add(key, g_dr);
  auto& cache = ctx->wf_graphs;
  size_t hit = 0;
  while (hit < cache.size() && cache[hit].first != key) ++hit;
  if (hit == cache.size()) {
    cudaGraphExec_t exec = nullptr;
    if ((st = build_pass_graph(ctx, P, R, c, g_ph, mb_ph, g_ch, blk_ch, mb_ch, g_kn, g_dr, wv, &exec)) !=
        GBMC_OK)
      return st;
    if (cache.size() == kGraphCache) {
      cudaGraphExecDestroy(cache.back().second);
      cache.pop_back();
    }
    cache.insert(cache.begin(), {key, exec});
  } else if (hit > 0) {
    std::rotate(cache.begin(), cache.begin() + hit, cache.begin() + hit + 1);
  }
  CK(cudaGraphLaunch(cache.front().second, s));
  ++ctx->graph_launches;
  return GBMC_OK;
}

gbmc_status gbmc_run(gbmc_ctx* ctx, uint64_t n_hist, uint64_t seed, uint64_t first_hist,
                     void* cuda_stream) {
  gbmc_status st = ready(ctx);
  if (st != GBMC_OK) return st;
  if (n_hist == 0) return GBMC_OK;
  if (first_hist + n_hist > ((uint64_t)1 << 32)) return fail(ctx, GBMC_ERR_ARG, "history ids must be < 2^32");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  DevProblem P = make_problem(ctx, seed);
  const uint64_t Kmax = (uint64_t)ctx->opt.n_batches;
  const uint64_t K = std::min<uint64_t>(Kmax, n_hist);   // every batch non-empty
  P.job.run_first = (uint32_t)first_hist;
  P.job.run_n = n_hist;
  P.job.run_k = (int)K;
  std::vector<double> inv_n(K);
  for (uint64_t k = 0; k < K; ++k) {
    const uint64_t a = (uint64_t)(((unsigned __int128)n_hist * k) / K);
    const uint64_t b = (uint64_t)(((unsigned __int128)n_hist * (k + 1)) / K);
    inv_n[k] = 1.0 / (double)(b - a);
  }
  if (ctx->opt.timing && (!ctx->ev_transport.empty() || !ctx->ev_flush.empty() || !ctx->ev_photon.empty())) {
    CK(cudaStreamSynchronize(ctx->last_stream));
    CK(fold_timings(ctx));
  }
  CK(cudaMemcpyAsync(ctx->d_inv_n, inv_n.data(), K * sizeof(double), cudaMemcpyHostToDevice, s));
  CK(cudaEventRecord(ctx->ev0, s));
  if (ctx->opt.kernel == GBMC_KERNEL_PLAIN) {
    TIMED(launch_plain(P, full_grid(ctx, (int64_t)n_hist), ctx->opt.block, s, ctx->opt.ledger_check != 0),
          ev_transport);
    ++ctx->n_kernels;
  } else {
    st = run_wavefront(ctx, P, s);
    if (st != GBMC_OK) return st;
  }
  TIMED(launch_flush_tiles(ctx->d_tile, ctx->tile_stride, (int)K, ctx->d_inv_n, ctx->d_s1, ctx->d_s2,
                           ctx->d_ledger + 1, ctx->sm_count, s), ev_flush);
  ++ctx->n_kernels;
  CK(cudaEventRecord(ctx->ev1, s));
  ctx->timed = true;
  ctx->n_hist += n_hist;
  ctx->k_batches += K;
  ctx->last_stream = s;
  return GBMC_OK;
}

static gbmc_status check_flags(gbmc_ctx* ctx) {
  unsigned int e = 0;
  CK(cudaMemcpy(&e, ctx->d_err, 4, cudaMemcpyDeviceToHost));
  if (e & E_BOUNDS)
    return fail(ctx, GBMC_ERR_BOUNDS, "checked build: an index out of range was caught (flags " +
                                          std::to_string(e) + ")");
  if (e & E_STACK) return fail(ctx, GBMC_ERR_STACK, "a per-thread secondary stack overflowed");
  if (e) return fail(ctx, GBMC_ERR_DEVICE_LIMIT, "a bounded device loop gave up (flags " + std::to_string(e) + ")");
  return GBMC_OK;
}

static gbmc_status read_tally(gbmc_ctx* ctx, double* mean, double* var, int ptr_kind, int dose) {
  gbmc_status st = ready(ctx);
  if (st != GBMC_OK) return st;
  if (!mean) return fail(ctx, GBMC_ERR_ARG, "null output");
  if (ctx->n_hist == 0) return fail(ctx, GBMC_ERR_STATE, "no histories run");
  CK(cudaSetDevice(ctx->device));
  CK(cudaStreamSynchronize(ctx->last_stream));
  const double vol = ctx->dx * ctx->dy * ctx->dz;
  double* dm = (ptr_kind == GBMC_PTR_DEVICE) ? mean : ctx->d_out;
  double* dv = var ? ((ptr_kind == GBMC_PTR_DEVICE) ? var : ctx->d_out + ctx->nvox) : nullptr;
  CK(launch_finalize(ctx->d_s1, ctx->d_s2, ctx->d_rho, ctx->nvox, (double)ctx->n_hist,
                     (double)ctx->k_batches, vol, dose, dm, dv, ctx->last_stream));
  if (ptr_kind == GBMC_PTR_HOST) {
    CK(cudaMemcpyAsync(mean, dm, ctx->nvox * sizeof(double), cudaMemcpyDeviceToHost, ctx->last_stream));
    if (var) CK(cudaMemcpyAsync(var, dv, ctx->nvox * sizeof(double), cudaMemcpyDeviceToHost, ctx->last_stream));
  } else if (ptr_kind != GBMC_PTR_DEVICE) {
    return fail(ctx, GBMC_ERR_ARG, "bad ptr_kind");
  }
  CK(cudaStreamSynchronize(ctx->last_stream));
  return check_flags(ctx);
}

gbmc_status gbmc_get_dose(gbmc_ctx* ctx, double* dose, double* var, int ptr_kind) {
  return read_tally(ctx, dose, var, ptr_kind, 1);
}

gbmc_status gbmc_get_edep(gbmc_ctx* ctx, double* mean, double* var, int ptr_kind) {
  return read_tally(ctx, mean, var, ptr_kind, 0);
}

gbmc_status gbmc_get_stats(gbmc_ctx* ctx, gbmc_stats* out) {
  if (!ctx || !out) return GBMC_ERR_ARG;
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  CK(cudaSetDevice(ctx->device));
  if (ctx->last_stream || ctx->timed) CK(cudaStreamSynchronize(ctx->last_stream));
  std::memset(out, 0, sizeof *out);
  unsigned long long c[NCOUNT];
  double l[6];
  unsigned int e = 0;
  CK(cudaMemcpy(c, ctx->d_counters, sizeof c, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(l, ctx->d_ledger, sizeof l, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(&e, ctx->d_err, 4, cudaMemcpyDeviceToHost));
  out->n_hist = ctx->n_hist + ctx->batch_hist; out->n_batches = ctx->k_batches + ctx->batch_k;
  out->n_tent = c[C_TENT]; out->n_real = c[C_REAL]; out->n_e_steps = c[C_ESTEP];
  out->n_cross = c[C_CROSS]; out->n_hard = c[C_HARD]; out->n_particles = c[C_PART];
  out->e_src = l[0]; out->e_dep = l[1]; out->e_esc = l[2]; out->e_pair_net = l[3];
  out->max_ledger_rel = l[4];
  out->n_ledger_checked = (uint64_t)l[5];
  out->error_flags = e;
  if (ctx->timed) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
    out->last_run_ms = ms;
  }
  CK(fold_timings(ctx));
  out->transport_ms = ctx->transport_ms;
  out->flush_ms = ctx->flush_ms;
  out->n_transport_launches = ctx->n_transport;
  out->n_flush_launches = ctx->n_flush;
  out->photon_ms = ctx->photon_ms;
  out->n_photon_launches = ctx->n_photon;
  out->drain_ms = ctx->drain_ms;
  out->n_drain_launches = ctx->n_drain;
  unsigned long long loop[2];
  CK(cudaMemcpy(loop, ctx->d_loop, sizeof loop, cudaMemcpyDeviceToHost));
  out->n_kernel_launches = ctx->n_kernels + 5 * loop[0];   // each graph loop iteration: 5 kernels
  out->n_passes = loop[1];
  out->n_graph_launches = ctx->graph_launches;
  return check_flags(ctx);
}

gbmc_status gbmc_reset_tally(gbmc_ctx* ctx) {
  if (!ctx) return GBMC_ERR_ARG;
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  CK(cudaSetDevice(ctx->device));
  if (ctx->last_stream) CK(cudaStreamSynchronize(ctx->last_stream));
  CK(cudaDeviceSynchronize());
  if (ctx->nvox) {
    CK(cudaMemset(ctx->d_tile, 0, (size_t)ctx->tile_stride * ctx->opt.n_batches * sizeof(float)));
    CK(cudaMemset(ctx->d_s1, 0, ctx->tile_stride * sizeof(double)));
    CK(cudaMemset(ctx->d_s2, 0, ctx->tile_stride * sizeof(double)));
  }
  CK(cudaMemset(ctx->d_counters, 0, sizeof(unsigned long long) * NCOUNT));
  CK(cudaMemset(ctx->d_ledger, 0, sizeof(double) * 6));
  CK(cudaMemset(ctx->d_err, 0, sizeof(unsigned int)));
  ctx->n_hist = 0;
  ctx->k_batches = 0;
  ctx->timed = false;
  ctx->ev_transport.clear();
  ctx->ev_flush.clear();
  ctx->ev_photon.clear();
  ctx->ev_drain.clear();
  ctx->ev_used = 0;
  ctx->transport_ms = ctx->flush_ms = ctx->photon_ms = ctx->drain_ms = 0.0;
  CK(cudaMemset(ctx->d_loop, 0, 2 * sizeof(unsigned long long)));
  ctx->n_kernels = 0; ctx->graph_launches = 0;
  ctx->batch_hist = 0; ctx->batch_k = 0;
  ctx->n_transport = ctx->n_flush = ctx->n_photon = ctx->n_drain = 0;
  return GBMC_OK;
}

gbmc_status gbmc_get_moments(gbmc_ctx* ctx, double* s1, double* s2, uint64_t* n_hist,
                             uint64_t* n_batches, int ptr_kind) {
  if (!ctx) return GBMC_ERR_ARG;
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (!ctx->have_ph) return fail(ctx, GBMC_ERR_STATE, "no phantom loaded");
  if (!s1 || !s2 || !n_hist || !n_batches) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (ptr_kind != GBMC_PTR_HOST && ptr_kind != GBMC_PTR_DEVICE) return fail(ctx, GBMC_ERR_ARG, "bad ptr_kind");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->last_stream;
  CK(cudaStreamSynchronize(s));
  const cudaMemcpyKind kind = ptr_kind == GBMC_PTR_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
  CK(cudaMemcpyAsync(s1, ctx->d_s1, ctx->nvox * sizeof(double), kind, s));
  CK(cudaMemcpyAsync(s2, ctx->d_s2, ctx->nvox * sizeof(double), kind, s));
  CK(cudaStreamSynchronize(s));
  *n_hist = ctx->n_hist;
  *n_batches = ctx->k_batches;
  return check_flags(ctx);
}

gbmc_status gbmc_add_moments(gbmc_ctx* ctx, const double* s1, const double* s2, uint64_t n_hist,
                             uint64_t n_batches, int ptr_kind) {
  if (!ctx) return GBMC_ERR_ARG;
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (!ctx->have_ph) return fail(ctx, GBMC_ERR_STATE, "no phantom loaded");
  if (!s1 || !s2) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (ptr_kind != GBMC_PTR_HOST && ptr_kind != GBMC_PTR_DEVICE) return fail(ctx, GBMC_ERR_ARG, "bad ptr_kind");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = ctx->last_stream;
  const double* a = s1;
  const double* b = s2;
  if (ptr_kind == GBMC_PTR_HOST) {   // staged through the read-back scratch (2 nvox doubles)
    CK(cudaMemcpyAsync(ctx->d_out, s1, ctx->nvox * sizeof(double), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(ctx->d_out + ctx->nvox, s2, ctx->nvox * sizeof(double), cudaMemcpyHostToDevice, s));
    a = ctx->d_out;
    b = ctx->d_out + ctx->nvox;
  }
  CK(launch_add_moments(ctx->d_s1, ctx->d_s2, a, b, ctx->nvox, s));
  CK(cudaStreamSynchronize(s));
  ctx->n_hist += n_hist;
  ctx->k_batches += n_batches;
  return GBMC_OK;
}

gbmc_status gbmc_run_batch(gbmc_ctx* ctx, const gbmc_job* jobs, int n_jobs, void* cuda_stream) {
  if (!ctx || !jobs || n_jobs < 1 || n_jobs > 65535) return fail(ctx, GBMC_ERR_ARG, "1 <= n_jobs <= 65535 jobs");
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (!ctx->have_mat) return fail(ctx, GBMC_ERR_STATE, "gbmc_set_materials first");
  CK(cudaSetDevice(ctx->device));
  if (ctx->n_hist) CK(cudaStreamSynchronize(ctx->last_stream));   // runs share queues and counters
  cudaStream_t s = (cudaStream_t)cuda_stream;
  const int n_mat = (int)ctx->mats.size();
  gbmc_status st;
  // host-side argument checks first (nothing is touched before they pass)
  for (int j = 0; j < n_jobs; ++j) {
    const gbmc_job& J = jobs[j];
    if (J.nx < 1 || J.ny < 1 || J.nz < 1 || !(J.dx > 0) || !(J.dy > 0) || !(J.dz > 0) || !J.mat || !J.rho)
      return fail(ctx, GBMC_ERR_ARG, "job " + std::to_string(j) + ": bad grid or null phantom");
    if ((int64_t)J.nx * J.ny * J.nz >= ((int64_t)1 << 31)) return fail(ctx, GBMC_ERR_ARG, "job grid too large");
    if (J.n_hist == 0 || J.first_hist + J.n_hist > ((uint64_t)1 << 32))
      return fail(ctx, GBMC_ERR_ARG, "job " + std::to_string(j) + ": need 0 < n_hist, ids < 2^32");
  }
  // the job buffers of the last batched run are kept when every job has the
  // same voxel count and batch count (repeated runs of the same jobs then
  // allocate nothing); otherwise they are released and allocated anew
  // (a batched run that failed part-way leaves its job buffers partly
  // allocated: it is never reused, and its doses cannot be read)
  bool reuse = ctx->batch_ready && (int)ctx->batch.size() == n_jobs;
  ctx->batch_ready = false;
  for (int j = 0; j < n_jobs && reuse; ++j) {
    const gbmc_job& J = jobs[j];
    const int64_t nvox = (int64_t)J.nx * J.ny * J.nz;
    const int K = (int)std::min<uint64_t>((uint64_t)ctx->opt.n_batches, J.n_hist);
    reuse = ctx->batch[j].nvox == nvox && ctx->batch[j].K == K;
  }
  if (!reuse) {
    free_batch(ctx);
    ctx->batch.resize(n_jobs);
  }
  // phantoms: copied to the device and validated there (material ids below
  // n_mat, finite positive densities, per-material maximum density), one
  // kernel per job, one read-back for all jobs
  const int vw = 1 + GBMC_MAX_MAT;
  unsigned int* d_valid = nullptr;
  CK(cudaMalloc((void**)&d_valid, sizeof(unsigned int) * vw * (size_t)n_jobs));
  cudaError_t ve = cudaMemsetAsync(d_valid, 0, sizeof(unsigned int) * vw * (size_t)n_jobs, s);
  for (int j = 0; j < n_jobs && ve == cudaSuccess; ++j) {
    const gbmc_job& J = jobs[j];
    BatchJob& B = ctx->batch[j];
    const int64_t nvox = (int64_t)J.nx * J.ny * J.nz;
    if (!reuse) {
      if ((st = dalloc(ctx, &B.d_mat, (size_t)nvox)) != GBMC_OK) { cudaFree(d_valid); return st; }
      if ((st = dalloc(ctx, &B.d_rho, (size_t)nvox)) != GBMC_OK) { cudaFree(d_valid); return st; }
    }
    ve = cudaMemcpyAsync(B.d_mat, J.mat, (size_t)nvox, cudaMemcpyHostToDevice, s);
    if (ve == cudaSuccess) ve = cudaMemcpyAsync(B.d_rho, J.rho, (size_t)nvox * sizeof(float), cudaMemcpyHostToDevice, s);
    if (ve == cudaSuccess)
      ve = launch_validate_phantom(B.d_mat, B.d_rho, nvox, n_mat, d_valid + (size_t)vw * j,
                                   reinterpret_cast<float*>(d_valid + (size_t)vw * j + 1), s);
  }
  std::vector<unsigned int> hv((size_t)vw * n_jobs);
  if (ve == cudaSuccess) ve = cudaMemcpyAsync(hv.data(), d_valid, hv.size() * sizeof(unsigned int), cudaMemcpyDeviceToHost, s);
  if (ve == cudaSuccess) ve = cudaStreamSynchronize(s);
  cudaFree(d_valid);
  if (ve != cudaSuccess) { free_batch(ctx); return cuda_fail(ctx, ve, "batched phantom upload"); }
  std::vector<DevJob> dj(n_jobs);
  std::vector<uint64_t> cf[2] = {{0}, {0}};
  std::vector<int> cj[2];
  std::vector<float> fb, maj(ctx->T.nE);
  std::vector<int> al;
  std::vector<double> inv_n;
  int64_t max_vox = 0;
  for (int j = 0; j < n_jobs; ++j) {
    const gbmc_job& J = jobs[j];
    BatchJob& B = ctx->batch[j];
    const int64_t nvox = (int64_t)J.nx * J.ny * J.nz;
    if (hv[(size_t)vw * j]) {
      free_batch(ctx);
      return fail(ctx, GBMC_ERR_ARG, "job " + std::to_string(j) + ": bad material id or density");
    }
    double rmax[GBMC_MAX_MAT] = {};
    for (int m = 0; m < n_mat; ++m) {
      float f;
      std::memcpy(&f, &hv[(size_t)vw * j + 1 + m], 4);
      rmax[m] = f;
    }
    if ((st = prepare_source(ctx, &J.src, fb, al)) != GBMC_OK) { free_batch(ctx); return st; }
    majorant_table(ctx->T, rmax, maj.data());
    B.nvox = nvox;
    B.stride = (nvox + 3) & ~(int64_t)3;
    B.vol = J.dx * J.dy * J.dz;
    B.n_hist = J.n_hist;
    B.K = (int)std::min<uint64_t>((uint64_t)ctx->opt.n_batches, J.n_hist);
    if ((st = upload_keep(ctx, &B.d_major, maj.data(), maj.size(), reuse)) != GBMC_OK) return st;
    const bool same_bins = reuse && B.n_bins == J.src.n_bins;
    if (!fb.empty()) {
      if ((st = upload_keep(ctx, &B.d_bins, fb.data(), fb.size(), same_bins)) != GBMC_OK) return st;
      if ((st = upload_keep(ctx, &B.d_alias, al.data(), al.size(), same_bins)) != GBMC_OK) return st;
    } else {
      if ((st = dalloc(ctx, &B.d_bins, 0)) != GBMC_OK) return st;
      if ((st = dalloc(ctx, &B.d_alias, 0)) != GBMC_OK) return st;
    }
    B.n_bins = J.src.n_bins;
    if (!reuse) {
      if ((st = dalloc(ctx, &B.d_tile, (size_t)B.stride * B.K)) != GBMC_OK) return st;
      if ((st = dalloc(ctx, &B.d_s12, 2 * (size_t)B.stride)) != GBMC_OK) return st;
    }
    CK(cudaMemsetAsync(B.d_tile, 0, (size_t)B.stride * B.K * sizeof(float), s));
    CK(cudaMemsetAsync(B.d_s12, 0, 2 * (size_t)B.stride * sizeof(double), s));
    inv_n.assign(B.K, 0.0);
    for (int k = 0; k < B.K; ++k) {
      const uint64_t a = (uint64_t)(((unsigned __int128)J.n_hist * k) / B.K);
      const uint64_t b = (uint64_t)(((unsigned __int128)J.n_hist * (k + 1)) / B.K);
      inv_n[k] = 1.0 / (double)(b - a);
    }
    if ((st = upload_keep(ctx, &B.d_inv_n, inv_n.data(), inv_n.size(), reuse)) != GBMC_OK) return st;
    DevJob& D = dj[j];
    std::memset(&D, 0, sizeof D);
    D.nx = J.nx; D.ny = J.ny; D.nz = J.nz; D.nxy = J.nx * J.ny;
    D.inv_nx = 1.0f / (float)J.nx; D.inv_nxy = 1.0f / (float)D.nxy;
    D.dx = (float)J.dx; D.dy = (float)J.dy; D.dz = (float)J.dz;
    D.idx = (float)(1.0 / J.dx); D.idy = (float)(1.0 / J.dy); D.idz = (float)(1.0 / J.dz);
    D.dmin = (float)std::min(J.dx, std::min(J.dy, J.dz));
    D.step_len = (float)(ctx->tp.step_vox * std::min(J.dx, std::min(J.dy, J.dz)));
    D.mat = B.d_mat; D.rho = B.d_rho; D.major = B.d_major;
    D.particle = J.src.particle; D.shape = J.src.shape; D.n_bins = J.src.n_bins;
    D.x0 = (float)J.src.x0; D.y0 = (float)J.src.y0; D.hx = (float)J.src.hx; D.hy = (float)J.src.hy;
    if (J.src.shape == 0) {
      D.x0 = pencil_coord(J.src.x0, J.dx, J.nx);
      D.y0 = pencil_coord(J.src.y0, J.dy, J.ny);
    }
    D.energy = (float)J.src.energy;
    D.bin_prob = B.d_bins;
    D.bin_edges = B.d_bins ? B.d_bins + J.src.n_bins : nullptr;
    D.bin_alias = B.d_alias;
    D.keys = philox_keys((uint32_t)J.seed, (uint32_t)(J.seed >> 32) ^ (uint32_t)j);
    D.run_first = (uint32_t)J.first_hist; D.run_n = J.n_hist; D.run_k = B.K;
    D.tile = B.d_tile; D.tile_stride = B.stride;
    const int cls = (J.src.particle == GBMC_PHOTON) ? 0 : 1;
    cj[cls].push_back(j);
    cf[cls].push_back(cf[cls].back() + J.n_hist);
    max_vox = std::max(max_vox, nvox);
  }
  std::vector<uint64_t> cfa(cf[0]);
  cfa.insert(cfa.end(), cf[1].begin(), cf[1].end());
  std::vector<int> cja(cj[0]);
  cja.insert(cja.end(), cj[1].begin(), cj[1].end());
  // the job table and class prefixes keep their buffers when the jobs (and so
  // their classes) are the same shape as the last run's
  const bool same_cls = reuse && ctx->batch_ncls[0] == (int)cj[0].size() && ctx->batch_ncls[1] == (int)cj[1].size();
  if ((st = upload_keep(ctx, &ctx->d_jobs, dj.data(), dj.size(), reuse)) != GBMC_OK) return st;
  if ((st = upload_keep(ctx, &ctx->d_cls_first, cfa.data(), cfa.size(), same_cls)) != GBMC_OK) return st;
  if ((st = upload_keep(ctx, &ctx->d_cls_job, cja.data(), std::max<size_t>(cja.size(), 1), same_cls)) != GBMC_OK)
    return st;
  ctx->batch_ncls[0] = (int)cj[0].size();
  ctx->batch_ncls[1] = (int)cj[1].size();
  if (!(reuse && ctx->d_bout && ctx->bout_len == max_vox))
    if ((st = dalloc(ctx, &ctx->d_bout, 2 * (size_t)max_vox)) != GBMC_OK) return st;
  ctx->bout_len = max_vox;
  DevProblem P = make_problem(ctx, 0);
  P.jobs = ctx->d_jobs;
  P.n_jobs = n_jobs;
  P.cls_first[0] = ctx->d_cls_first;
  P.cls_first[1] = ctx->d_cls_first + cf[0].size();
  P.cls_job[0] = ctx->d_cls_job;
  P.cls_job[1] = ctx->d_cls_job + cj[0].size();
  P.n_cls[0] = (int)cj[0].size();
  P.n_cls[1] = (int)cj[1].size();
  ctx->batch_prim[0] = cf[0].back();
  ctx->batch_prim[1] = cf[1].back();
  CK(cudaEventRecord(ctx->ev0, s));
  if ((st = run_wavefront(ctx, P, s)) != GBMC_OK) return st;
  for (int j = 0; j < n_jobs; ++j) {
    BatchJob& B = ctx->batch[j];
    CK(launch_flush_tiles(B.d_tile, B.stride, B.K, B.d_inv_n, B.d_s12, B.d_s12 + B.stride,
                          ctx->d_ledger + 1, ctx->sm_count, s));
    ++ctx->n_kernels;
  }
  CK(cudaEventRecord(ctx->ev1, s));
  ctx->timed = true;
  for (const BatchJob& B : ctx->batch) { ctx->batch_hist += B.n_hist; ctx->batch_k += (uint64_t)B.K; }
  CK(cudaStreamSynchronize(s));
  ctx->last_stream = s;
  ctx->batch_ready = true;
  return check_flags(ctx);
}

gbmc_status gbmc_get_job_dose(gbmc_ctx* ctx, int job, double* dose, double* var, int ptr_kind) {
  if (!ctx || !dose) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (job < 0 || job >= (int)ctx->batch.size()) return fail(ctx, GBMC_ERR_ARG, "no such job in the last batched run");
  if (!ctx->batch_ready) return fail(ctx, GBMC_ERR_STATE, "the last batched run did not complete");
  if (ptr_kind != GBMC_PTR_HOST && ptr_kind != GBMC_PTR_DEVICE) return fail(ctx, GBMC_ERR_ARG, "bad ptr_kind");
  CK(cudaSetDevice(ctx->device));
  const BatchJob& B = ctx->batch[job];
  cudaStream_t s = ctx->last_stream;
  double* dm = (ptr_kind == GBMC_PTR_DEVICE) ? dose : ctx->d_bout;
  double* dv = var ? ((ptr_kind == GBMC_PTR_DEVICE) ? var : ctx->d_bout + B.nvox) : nullptr;
  CK(launch_finalize(B.d_s12, B.d_s12 + B.stride, B.d_rho, B.nvox, (double)B.n_hist, (double)B.K,
                     B.vol, 1, dm, dv, s));
  if (ptr_kind == GBMC_PTR_HOST) {
    CK(cudaMemcpyAsync(dose, dm, B.nvox * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (var) CK(cudaMemcpyAsync(var, dv, B.nvox * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaStreamSynchronize(s));
  return GBMC_OK;
}

// device time of one trial: a single run of n histories, or the batch with
// every job's histories scaled to n in total (same seeds each trial)
static gbmc_status autotune_trial(gbmc_ctx* ctx, const std::vector<gbmc_job>& jobs, uint64_t n,
                                  uint64_t seed, void* stream, double* ms) {
  gbmc_status st;
  if (jobs.empty()) {
    if ((st = gbmc_run(ctx, n, seed, 0, stream)) != GBMC_OK) return st;
  } else {
    if ((st = gbmc_run_batch(ctx, jobs.data(), (int)jobs.size(), stream)) != GBMC_OK) return st;
  }
  CK(cudaEventSynchronize(ctx->ev1));
  float f = 0.f;
  CK(cudaEventElapsedTime(&f, ctx->ev0, ctx->ev1));
  *ms = f;
  return GBMC_OK;
}

gbmc_status gbmc_autotune(gbmc_ctx* ctx, const gbmc_job* jobs, int n_jobs, uint64_t n_trial,
                          uint64_t seed, void* cuda_stream, gbmc_options* chosen) {
  if (!ctx) return GBMC_ERR_ARG;
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (ctx->opt.kernel != GBMC_KERNEL_WAVEFRONT) return fail(ctx, GBMC_ERR_STATE, "autotune tunes the wavefront kernels");
  if (n_trial == 0 || n_jobs < 0 || (n_jobs > 0 && !jobs)) return fail(ctx, GBMC_ERR_ARG, "bad trial size or jobs");
  gbmc_status st;
  if (n_jobs == 0 && (st = ready(ctx)) != GBMC_OK) return st;
  std::vector<gbmc_job> tj(jobs, jobs + n_jobs);
  if (n_jobs) {
    uint64_t tot = 0;
    for (const gbmc_job& j : tj) tot += j.n_hist;
    for (gbmc_job& j : tj)
      j.n_hist = std::max<uint64_t>(1, (uint64_t)((unsigned __int128)j.n_hist * n_trial / std::max<uint64_t>(tot, 1)));
  }
  const int cap = ctx->opt.queue_cap > 0 ? ctx->opt.queue_cap : kDefaultQueueCap;
  const gbmc_options start = ctx->opt;
  gbmc_options best = start;
  if (best.pass_target == 0) best.pass_target = cap / 2;
  // candidates per option (coordinate search, two sweeps); a trial time is the
  // better of two runs of the same histories. Block shape: threads per block
  // and resident blocks per SM (0 = each kernel's own default; 2 and 3 also
  // pick the photon kernel variant compiled for that occupancy)
  const int n_opt = 5;
  const int cand[n_opt][3] = {{8, 16, 32}, {4, 8, 16}, {cap / 8, cap / 4, cap / 2},
                              {128, 256, 256}, {0, 2, 3}};
  auto trial = [&](const gbmc_options& o, double* t) -> gbmc_status {
    ctx->opt = o;
    double a = 0.0, b = 0.0;
    gbmc_status r = autotune_trial(ctx, tj, n_trial, seed, cuda_stream, &a);
    if (r == GBMC_OK) r = autotune_trial(ctx, tj, n_trial, seed, cuda_stream, &b);
    *t = std::min(a, b);
    return r;
  };
  double t_best = 0.0;
  if ((st = trial(best, &t_best)) != GBMC_OK) { ctx->opt = start; return st; }
  for (int sweep = 0; sweep < 2; ++sweep)
    for (int p = 0; p < n_opt; ++p)
      for (int v : cand[p]) {
        gbmc_options o = best;
        int* field = p == 0 ? &o.charged_budget : p == 1 ? &o.photon_budget : p == 2 ? &o.pass_target
                   : p == 3 ? &o.block : &o.blocks_per_sm;
        if (*field == v) continue;
        *field = v;
        double t = 0.0;
        if ((st = trial(o, &t)) != GBMC_OK) { ctx->opt = start; return st; }
        if (t < 0.98 * t_best) { best = o; t_best = t; }
      }
  ctx->opt = best;
  if ((st = gbmc_reset_tally(ctx)) != GBMC_OK) return st;
  if (chosen) *chosen = best;
  return GBMC_OK;
}

gbmc_status gbmc_set_majorant(gbmc_ctx* ctx, const double* rho_maj, int n_mat) {
  if (!ctx) return GBMC_ERR_ARG;
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (!ctx->have_mat) return fail(ctx, GBMC_ERR_STATE, "gbmc_set_materials first");
  if (!rho_maj) {
    ctx->have_maj = false;
  } else {
    if (n_mat != (int)ctx->mats.size()) return fail(ctx, GBMC_ERR_ARG, "one density per material");
    for (int m = 0; m < n_mat; ++m) {
      if (!(rho_maj[m] > 0.0) || !std::isfinite(rho_maj[m]))
        return fail(ctx, GBMC_ERR_ARG, "majorant densities must be finite and positive");
      if (ctx->have_ph && rho_maj[m] < ctx->rho_max[m])
        return fail(ctx, GBMC_ERR_ARG, "majorant density below the phantom's maximum");
    }
    for (int m = 0; m < GBMC_MAX_MAT; ++m) ctx->rho_maj[m] = m < n_mat ? rho_maj[m] : 0.0;
    ctx->have_maj = true;
  }
  if (!ctx->have_ph) return GBMC_OK;
  CK(cudaSetDevice(ctx->device));
  build_majorant(ctx->T, ctx->have_maj ? ctx->rho_maj : ctx->rho_max);
  return upload_tables(ctx);
}

gbmc_status gbmc_set_vr(gbmc_ctx* ctx, const gbmc_vr* vr) {
  if (!ctx) return GBMC_ERR_ARG;
  if (!vr) {
    ctx->vr = gbmc_vr{1.0, 1.0, 0.0, 0.0, 1};
    return GBMC_OK;
  }
  const bool ok = vr->f_inel >= 1.0 && vr->f_inel <= 1e6 && vr->f_brems >= 1.0 && vr->f_brems <= 1e6 &&
                  vr->w_lo >= 0.0 && vr->w_hi >= vr->w_lo && std::isfinite(vr->w_lo) &&
                  vr->n_split_brems >= 1 && vr->n_split_brems <= 64;
  if (!ok) return fail(ctx, GBMC_ERR_ARG, "variance-reduction parameters out of range");
  ctx->vr = *vr;
  if (!std::isfinite(ctx->vr.w_hi)) ctx->vr.w_hi = 3.0e38;
  return GBMC_OK;
}

gbmc_status gbmc_adjoint(gbmc_ctx* ctx, const double* dL_dD, int g_ptr_kind, uint64_t n_hist,
                         uint64_t seed, uint64_t first_hist, double* grad, double* var,
                         int out_ptr_kind, void* cuda_stream) {
  gbmc_status st = ready(ctx);
  if (st != GBMC_OK) return st;
  if (vr_on(ctx->vr)) return fail(ctx, GBMC_ERR_STATE, "the adjoint runs analog histories: switch variance reduction off");
  if (!dL_dD || !grad) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (n_hist == 0) return fail(ctx, GBMC_ERR_ARG, "n_hist must be positive");
  if (first_hist + n_hist > ((uint64_t)1 << 32)) return fail(ctx, GBMC_ERR_ARG, "history ids must be < 2^32");
  if ((g_ptr_kind != GBMC_PTR_HOST && g_ptr_kind != GBMC_PTR_DEVICE) ||
      (out_ptr_kind != GBMC_PTR_HOST && out_ptr_kind != GBMC_PTR_DEVICE))
    return fail(ctx, GBMC_ERR_ARG, "bad ptr_kind");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (ctx->n_hist) CK(cudaStreamSynchronize(ctx->last_stream));   // runs share the tiles
  const int64_t nvox = ctx->nvox, stride = ctx->tile_stride;
  // scratch: S1 | S2 | counters (NCOUNT) | ledger (4) | err, all 8-byte slots
  if (ctx->adj_stride != stride) {
    if ((st = dalloc(ctx, &ctx->d_adj, 2 * (size_t)stride + NCOUNT + 4 + 1)) != GBMC_OK) return st;
    if ((st = dalloc(ctx, &ctx->d_wv, (size_t)stride)) != GBMC_OK) return st;
    ctx->adj_stride = stride;
  }
  double* s1 = ctx->d_adj;
  double* s2 = s1 + stride;
  unsigned long long* counters = reinterpret_cast<unsigned long long*>(s2 + stride);
  double* ledger = reinterpret_cast<double*>(counters + NCOUNT);
  unsigned int* err = reinterpret_cast<unsigned int*>(ledger + 4);
  CK(cudaMemsetAsync(ctx->d_adj, 0, (2 * (size_t)stride + NCOUNT + 4 + 1) * sizeof(double), s));
  // the tiles are clear between runs (every flush clears them)
  const double* g = dL_dD;
  if (g_ptr_kind == GBMC_PTR_HOST) {
    CK(cudaMemcpyAsync(ctx->d_out, dL_dD, nvox * sizeof(double), cudaMemcpyHostToDevice, s));
    g = ctx->d_out;
  }
  const double vol = ctx->dx * ctx->dy * ctx->dz;
  CK(launch_adjoint_weights(g, ctx->d_rho, nvox, vol, ctx->d_wv, s));
  DevProblem P = make_problem(ctx, seed);
  P.counters = counters; P.ledger = ledger; P.err = err;
  // the plain kernel holds G_h in a register per history; the wavefront keeps
  // it in a per-history buffer, so its runs go in chunks of at most 2^26
  // histories (each chunk is a run of its own batches, like repeated gbmc_run)
  const bool wf = (ctx->opt.kernel == GBMC_KERNEL_WAVEFRONT);
  const uint64_t chunk = wf ? std::min<uint64_t>(n_hist, (uint64_t)1 << 26) : n_hist;
  if (wf && ctx->gbuf_len < chunk) {
    if ((st = dalloc(ctx, &ctx->d_gbuf, (size_t)chunk)) != GBMC_OK) return st;
    ctx->gbuf_len = chunk;
  }
  uint64_t k_total = 0;
  std::vector<double> inv_n;
  for (uint64_t off = 0; off < n_hist; off += chunk) {
    const uint64_t c = std::min<uint64_t>(chunk, n_hist - off);
    const uint64_t K = std::min<uint64_t>((uint64_t)ctx->opt.n_batches, c);
    P.job.run_first = (uint32_t)(first_hist + off);
    P.job.run_n = c;
    P.job.run_k = (int)K;
    inv_n.assign(K, 0.0);
    for (uint64_t k = 0; k < K; ++k) {
      const uint64_t a = (uint64_t)(((unsigned __int128)c * k) / K);
      const uint64_t b = (uint64_t)(((unsigned __int128)c * (k + 1)) / K);
      inv_n[k] = 1.0 / (double)(b - a);
    }
    CK(cudaMemcpyAsync(ctx->d_inv_n, inv_n.data(), K * sizeof(double), cudaMemcpyHostToDevice, s));
    if (!wf) {
      CK(launch_adjoint(P, ctx->d_wv, full_grid(ctx, (int64_t)c), ctx->opt.block, s));
    } else {
      P.gbuf = ctx->d_gbuf;
      CK(cudaMemsetAsync(ctx->d_gbuf, 0, c * sizeof(float), s));
      P.mode = M_G_SUM;
      if ((st = run_wavefront(ctx, P, s, ctx->d_wv)) != GBMC_OK) return st;
      P.mode = M_SCATTER;
      if ((st = run_wavefront(ctx, P, s, ctx->d_wv)) != GBMC_OK) return st;
    }
    CK(launch_flush_tiles(ctx->d_tile, stride, (int)K, ctx->d_inv_n, s1, s2, ledger + 1,
                          ctx->sm_count, s));
    k_total += K;
  }
  const uint64_t K = k_total;
  double* dm = (out_ptr_kind == GBMC_PTR_DEVICE) ? grad : ctx->d_out;
  double* dv = var ? ((out_ptr_kind == GBMC_PTR_DEVICE) ? var : ctx->d_out + nvox) : nullptr;
  CK(launch_finalize(s1, s2, ctx->d_rho, nvox, (double)n_hist, (double)K, vol, 0, dm, dv, s));
  if (out_ptr_kind == GBMC_PTR_HOST) {
    CK(cudaMemcpyAsync(grad, dm, nvox * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (var) CK(cudaMemcpyAsync(var, dv, nvox * sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  unsigned int e = 0;
  CK(cudaMemcpyAsync(&e, err, 4, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e & E_BOUNDS)
    return fail(ctx, GBMC_ERR_BOUNDS, "checked build: an index out of range was caught (flags " +
                                          std::to_string(e) + ")");
  if (e & E_STACK) return fail(ctx, GBMC_ERR_STACK, "a per-thread secondary stack overflowed");
  if (e) return fail(ctx, GBMC_ERR_DEVICE_LIMIT, "a bounded device loop gave up (flags " + std::to_string(e) + ")");
  return GBMC_OK;
}

gbmc_status gbmc_philox_fill(int device, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                             uint32_t k0, uint32_t k1, uint32_t* out, int n) {
  if (!out || n < 1) return GBMC_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return GBMC_ERR_CUDA;
  uint32_t* d = nullptr;
  if (cudaMalloc((void**)&d, (size_t)n * 16) != cudaSuccess) return GBMC_ERR_OOM;
  cudaError_t e = launch_philox_fill(c0, c1, c2, c3, k0, k1, d, n, 0);
  if (e == cudaSuccess) e = cudaMemcpy(out, d, (size_t)n * 16, cudaMemcpyDeviceToHost);
  cudaFree(d);
  return e == cudaSuccess ? GBMC_OK : GBMC_ERR_CUDA;
}

gbmc_status gbmc_first_interactions(gbmc_ctx* ctx, uint64_t seed, uint64_t first_hist, int n,
                                    double* xyz, int* type) {
  gbmc_status st = ready(ctx);
  if (st != GBMC_OK) return st;
  if (n < 1 || !xyz || !type) return fail(ctx, GBMC_ERR_ARG, "bad output");
  if (ctx->src.particle != GBMC_PHOTON) return fail(ctx, GBMC_ERR_STATE, "photon source required");
  CK(cudaSetDevice(ctx->device));
  DevProblem P = make_problem(ctx, seed);
  P.job.run_first = (uint32_t)first_hist;
  P.job.run_n = (uint64_t)n;
  P.job.run_k = 1;
  float* dx = nullptr;
  int* dt = nullptr;
  CK(cudaMalloc((void**)&dx, (size_t)n * 12));
  CK(cudaMalloc((void**)&dt, (size_t)n * 4));
  cudaError_t e = launch_first_interactions(P, (uint32_t)first_hist, n, dx, dt, 0);
  std::vector<float> hx((size_t)3 * n);
  if (e == cudaSuccess) e = cudaMemcpy(hx.data(), dx, (size_t)n * 12, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(type, dt, (size_t)n * 4, cudaMemcpyDeviceToHost);
  cudaFree(dx);
  cudaFree(dt);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "first_interactions");
  for (size_t i = 0; i < hx.size(); ++i) xyz[i] = hx[i];
  return GBMC_OK;
}

gbmc_status gbmc_table_eval(gbmc_ctx* ctx, int q, int m, const double* x, int n, double* out) {
  if (!ctx || !x || !out || n < 0) return GBMC_ERR_ARG;
  if (!ctx->have_mat) return fail(ctx, GBMC_ERR_STATE, "gbmc_set_materials first");
  const Tables& T = ctx->T;
  if (q < 100 && (q < 0 || q >= Q_RINV_E || m < 0 || m >= T.n_mat)) return fail(ctx, GBMC_ERR_ARG, "bad quantity");
  if ((q == GBMC_Q_SIG_HARD_E || q == GBMC_Q_SIG_HARD_P) && (m < 0 || m >= T.n_mat))
    return fail(ctx, GBMC_ERR_ARG, "bad material");
  if ((q == GBMC_Q_RANGE_INV_E || q == GBMC_Q_RANGE_INV_P) && (m < 0 || m >= T.n_mat))
    return fail(ctx, GBMC_ERR_ARG, "bad material");
  for (int i = 0; i < n; ++i) {
    const float xv = (float)x[i];
    double v;
    if (q < 100) {
      const GridPos g = grid_pos(log2f(xv), T.lg0, T.inv_d, T.nE);
      const float* t = T.data.data() + tab_off(q, m, T.n_mat, T.nE);
      v = (q == Q_XC) ? lerp_tab(t, g) : exp2_tab(t, g);
    } else if (q == GBMC_Q_MAJORANT) {
      const GridPos g = grid_pos(log2f(xv), T.lg0, T.inv_d, T.nE);
      v = exp2_tab(T.data.data() + T.off_major, g);
    } else if (q == GBMC_Q_RANGE_INV_E || q == GBMC_Q_RANGE_INV_P) {
      const int s = q == GBMC_Q_RANGE_INV_P;
      const GridPos g = grid_pos(log2f(xv), T.lr0[m][s], T.inv_dr[m][s], T.nR);
      v = exp2_tab(T.data.data() + tab_off(s ? Q_RINV_P : Q_RINV_E, m, T.n_mat, T.nE), g);
    } else if (q == GBMC_Q_SIG_HARD_E || q == GBMC_Q_SIG_HARD_P) {
      const GridPos g = grid_pos(log2f(xv), T.lg0, T.inv_d, T.nE);
      v = exp2_tab(T.data.data() + tab_off(q == GBMC_Q_SIG_HARD_P ? Q_SIG_H_P : Q_SIG_H_E, m, T.n_mat, T.nE), g);
    } else if (q == GBMC_Q_SOFT_APRIME) {
      const GridPos g = grid_pos(log2f(xv / (1.0f - xv)), T.la0, T.inv_da, T.nA);
      v = exp2_tab(T.data.data() + T.off_soft, g);
    } else {
      return fail(ctx, GBMC_ERR_ARG, "bad quantity");
    }
    out[i] = v;
  }
  return GBMC_OK;
}


}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free run: per-call scratch in a file-scope device array.
// ---------------------------------------------------------------------------

// Scratch of gbmc_run_noalloc: [batch tiles | 1/n_k | counters | ledger | flags].
// Device code never names it; host code passes its device address (looked up
// once per device with cudaGetSymbolAddress) to the kernels.
static __device__ __align__(256) float g_noalloc_scratch[GBMC_NOALLOC_MAX_FLOATS];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
float* g_noalloc_ptr[kMaxDevices] = {};
int64_t g_noalloc_err_off[kMaxDevices];   // flag word of the last call per device (floats; -1 none)
bool g_noalloc_init = false;

// device address of the scratch array on `device` (which must be current):
// looked up on every call outside a stream capture (the query is cheap and
// allocates nothing, and a device reset moves the array), and taken from the
// last lookup inside one
cudaError_t noalloc_scratch(int device, cudaStream_t s, float** out) {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_init) {
    for (int d = 0; d < kMaxDevices; ++d) g_noalloc_err_off[d] = -1;
    g_noalloc_init = true;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t e = cudaStreamIsCapturing(s, &cs);
  if (e != cudaSuccess) return e;
  if (cs == cudaStreamCaptureStatusNone || !g_noalloc_ptr[device]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = static_cast<float*>(p);
  }
  *out = g_noalloc_ptr[device];
  return cudaSuccess;
}

// true if p is device memory of `device` (or managed memory)
bool is_device_ptr(const void* p, int device) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();   // clear the sticky-free error of an unknown pointer
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == device;
}
}  // namespace

extern "C" gbmc_status gbmc_run_noalloc(gbmc_ctx* ctx, uint64_t n_hist, uint64_t seed,
                                        uint64_t first_hist, int n_batches, double* sum,
                                        double* sum2, void* cuda_stream) {
  gbmc_status st = ready(ctx);
  if (st != GBMC_OK) return st;
  if (!sum || !sum2) return fail(ctx, GBMC_ERR_ARG, "null output buffer");
  if (n_batches < 2 || n_batches > GBMC_NOALLOC_MAX_BATCHES)
    return fail(ctx, GBMC_ERR_ARG, "n_batches outside 2..GBMC_NOALLOC_MAX_BATCHES");
  if (n_hist == 0) return GBMC_OK;
  if (first_hist + n_hist > ((uint64_t)1 << 32)) return fail(ctx, GBMC_ERR_ARG, "history ids must be < 2^32");
  if (ctx->device >= kMaxDevices) return fail(ctx, GBMC_ERR_ARG, "device index too large");
  const int K = (int)std::min<uint64_t>((uint64_t)n_batches, n_hist);
  // layout in floats: tiles, then 1/n_k (doubles), counters (u64), ledger
  // (doubles) and the flag word, each 2-float aligned
  const int64_t stride = ctx->tile_stride;
  const int64_t off_inv = (int64_t)K * stride;
  const int64_t off_cnt = off_inv + 2 * (int64_t)K;
  const int64_t off_led = off_cnt + 2 * (int64_t)NCOUNT;
  const int64_t off_err = off_led + 2 * 4;
  const int64_t used = off_err + 2;
  if (used > (int64_t)GBMC_NOALLOC_MAX_FLOATS)
    return fail(ctx, GBMC_ERR_ARG, "phantom x batches exceed the allocation-free scratch (" +
                                       std::to_string(GBMC_NOALLOC_MAX_FLOATS) + " floats)");
  CK(cudaSetDevice(ctx->device));
  if (!is_device_ptr(sum, ctx->device) || !is_device_ptr(sum2, ctx->device))
    return fail(ctx, GBMC_ERR_ARG, "sum and sum2 must be device memory of the context's device");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  float* base = nullptr;
  CK(noalloc_scratch(ctx->device, s, &base));
  CK(cudaMemsetAsync(base, 0, (size_t)used * sizeof(float), s));   // tiles, counters, ledger start at 0
  double* inv_n = reinterpret_cast<double*>(base + off_inv);
  CK(launch_batch_weights(inv_n, n_hist, K, s));
  DevProblem P = make_problem(ctx, seed);
  P.job.run_first = (uint32_t)first_hist;
  P.job.run_n = n_hist;
  P.job.run_k = K;
  P.job.tile = base;
  P.job.tile_stride = stride;
  P.counters = reinterpret_cast<unsigned long long*>(base + off_cnt);
  P.ledger = reinterpret_cast<double*>(base + off_led);
  P.err = reinterpret_cast<unsigned int*>(base + off_err);
  CK(launch_plain(P, full_grid(ctx, (int64_t)n_hist), ctx->opt.block, s));
  CK(launch_flush_tiles_scalar(base, stride, ctx->nvox, K, inv_n, sum, sum2, P.ledger + 1,
                               ctx->sm_count, s));
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    g_noalloc_err_off[ctx->device] = off_err;
  }
  return GBMC_OK;
}

extern "C" gbmc_status gbmc_noalloc_flags(gbmc_ctx* ctx, void* cuda_stream, uint32_t* flags) {
  if (!ctx || !flags) return fail(ctx, GBMC_ERR_ARG, "null argument");
  if (ctx->host_only) return fail(ctx, GBMC_ERR_STATE, "host-only context");
  if (ctx->device >= kMaxDevices) return fail(ctx, GBMC_ERR_ARG, "device index too large");
  int64_t off = -1;
  float* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (g_noalloc_init) off = g_noalloc_err_off[ctx->device];
    base = g_noalloc_ptr[ctx->device];
  }
  if (off < 0 || !base) return fail(ctx, GBMC_ERR_STATE, "no allocation-free run on this device");
  CK(cudaSetDevice(ctx->device));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CK(cudaStreamSynchronize(s));
  CK(cudaMemcpy(flags, base + off, sizeof(uint32_t), cudaMemcpyDeviceToHost));
  return GBMC_OK;
}

