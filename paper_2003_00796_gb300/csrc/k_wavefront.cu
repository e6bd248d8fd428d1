// k_wavefront.cu -- wavefront (event-queue) transport: the per-thread stack of
// the paper's history loop (Sec. 4.1; per-type stacks of Sec. 5.2) becomes
// structure-of-arrays queues in global memory, one per particle type. Each
// pass runs two kernels:
//   photon kernel:  every queued photon (plus newly issued primaries when the
//                   source emits photons) flies by Woodcock tracking to its
//                   next real interactions (at most max_real per pass);
//   charged kernel: every queued e-/e+ (plus primaries of an electron or
//                   positron source) takes at most max_steps class II steps.
// Survivors and secondaries are appended to the output queues of their type
// with warp-aggregated atomics, so that a warp works on one particle type at a
// time (the SIMT divergence of the one-history-per-thread kernel comes mostly
// from lanes running photon and electron code side by side). Charged particles
// whose next event makes a secondary (hard inelastic, hard bremsstrahlung,
// annihilation) are sorted into a third queue and handled by a small knock
// kernel in the same pass, so the charged kernel holds only the steps and the
// elastic events that make up most of the work. Particles carry
// their own random-stream position, so the histories are exactly those of the
// plain kernel; each particle scores into the tile of its batch.
#include "gbmc_internal.h"
#include "transport.cuh"

namespace gb {

// stage one table region (the photon or the charged one) into shared memory;
// the regions start on 16-byte boundaries
__device__ __forceinline__ void wf_stage(const float* src_f, int n, float* stab) {
  const int n4 = n >> 2;
  const float4* src = reinterpret_cast<const float4*>(src_f);
  float4* dst = reinterpret_cast<float4*>(stab);
  for (int i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = __ldg(src + i);
  for (int i = (n4 << 2) + threadIdx.x; i < n; i += blockDim.x) stab[i] = __ldg(src_f + i);
  __syncthreads();
}

// shared memory of a wavefront kernel: its table region (none for the knock kernel)
inline size_t wf_smem_bytes(const DevProblem& P, int kind) {   // 0 photon, 1 charged, 2 knock
  const int n = kind == 0 ? P.tab_g_floats : kind == 1 ? P.tab_e_floats : 0;
  return ((size_t)n * 4 + 15) & ~(size_t)15;
}

// a record in four 16-byte vector accesses; the weight is used only by the
// weighted kernels (vr), the others take 1. An input queue is only read
// while a kernel runs (the read-only path is safe)
__device__ __forceinline__ void wf_load(const Queue& q, int i, Particle& c, bool vr) {
  const float4 a = __ldg(q.pos + i), b = __ldg(q.dir + i), d = __ldg(q.st + i);
  const uint4 h = __ldg(q.id + i);
  c.x = a.x; c.y = a.y; c.z = a.z; c.u = a.w;
  c.v = b.x; c.w = b.y; c.E = b.z; c.meta = __float_as_uint(b.w);
  c.path_lo = h.x; c.path_hi = h.y; c.hist = h.z; c.nchild = h.w;
  c.n = __float_as_uint(d.x); c.vox = __float_as_int(d.y); c.r = d.z;
  c.wt = vr ? d.w : 1.0f;
}

__device__ __forceinline__ void wf_store(const Queue& q, int i, const Particle& c, bool vr) {
  q.pos[i] = make_float4(c.x, c.y, c.z, c.u);
  q.dir[i] = make_float4(c.v, c.w, c.E, __uint_as_float(c.meta));
  q.id[i] = make_uint4(c.path_lo, c.path_hi, c.hist, c.nchild);
  q.st[i] = make_float4(__uint_as_float(c.n), __int_as_float(c.vox), c.r, vr ? c.wt : 1.0f);
}

// appends to the photon or charged output queue; lanes that push together are
// grouped by target queue and take consecutive slots with one atomic per group
struct QueueSink {
  Queue g, e, k;
  unsigned int* cnt;   // [0] photons out, [1] charged out, [2] deferred events
  int cap;
  // queue q: 0 photon, 1 charged, 2 deferred charged events
  __device__ __forceinline__ void append(Track& t, const Particle& c, int q, int vox) {
    const unsigned mask = __activemask();
    const unsigned same = __match_any_sync(mask, q);
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(same) - 1;
    const unsigned rank = __popc(same & ((1u << lane) - 1u));
    unsigned base = 0;
    if (lane == leader) base = atomicAdd(cnt + q, (unsigned)__popc(same));
    base = __shfl_sync(same, base, leader);
    const unsigned slot = base + rank;
    if (slot < (unsigned)cap) {
      wf_store(q == 0 ? g : (q == 1 ? e : k), (int)slot, c, t.vr);
    } else {  // queue full: scored where it was made, flagged
      t.err |= E_QUEUE;
      score(t, vox, c.E * c.wt);
    }
  }
  __device__ __forceinline__ void push(Track& t, const Particle& c, int vox) {
    append(t, c, ((c.meta & 3u) == GBMC_PHOTON) ? 0 : 1, vox);
  }
};

__device__ __forceinline__ void wf_init(Track& t, const DevProblem& P, const float* tab_g,
                                        const float* tab_e, int mode) {
  t.P = &P; t.J = &P.job; t.tab_g = tab_g; t.tab_e = tab_e;
  t.tile = P.job.tile; t.pa = nullptr; t.pe = 0.0f;
  t.c_tent = t.c_real = t.c_estep = t.c_cross = t.c_hard = t.c_part = 0;
  t.l_src = t.l_esc = t.l_pair = 0.0;
  t.err = 0;
  t.mode = mode; t.wv = nullptr; t.G = 0.0f;
  t.check = false; t.l_dep = 0.0;
  t.vr = false;
}

// every lane of the warp reaches this point (blocks are whole warps); the
// warp is reconverged before the full-mask reductions
__device__ __forceinline__ void wf_commit(Track& t) {
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
    if (l[0] != 0.0) atomicAdd(P.ledger + 0, l[0]);
    if (l[1] != 0.0) atomicAdd(P.ledger + 2, l[1]);
    if (l[2] != 0.0) atomicAdd(P.ledger + 3, l[2]);
    if (e) atomicOr(P.err, e);
  }
}

// queue q of the five in one allocation (photon in/out, charged in/out by
// the pass parity, deferred events): field group g (16 bytes per record) at
// qmem + (16 q + 4 g) cap floats, 16-byte aligned
__device__ __forceinline__ Queue ring_queue(float* qmem, int q, int cap) {
  float* b = qmem + (size_t)q * kQueueFields * (size_t)cap;
  const size_t c = (size_t)cap;
  Queue Q;
  Q.pos = reinterpret_cast<float4*>(b);
  Q.dir = reinterpret_cast<float4*>(b + 4 * c);
  Q.id = reinterpret_cast<uint4*>(b + 8 * c);
  Q.st = reinterpret_cast<float4*>(b + 12 * c);
  return Q;
}

__device__ __forceinline__ QueueSink ring_sink(const WfRing& R, int cur) {
  QueueSink k;
  k.g = ring_queue(R.qmem, 0 + (cur ^ 1), R.cap);
  k.e = ring_queue(R.qmem, 2 + (cur ^ 1), R.cap);
  k.k = ring_queue(R.qmem, 4, R.cap);
  k.cnt = R.cnt;
  k.cap = R.cap;
  return k;
}

// Dynamic work claiming by warps: a warp takes chunks of up to kClaimChunk
// consecutive items of the pass from a per-kernel counter and hands them to
// its lanes in order as they need one. Lanes that refill together load
// neighbouring queue records, and the work balances across warps (a fixed
// per-thread share leaves warps with long particles running alone at the end).
// Every lane of the warp must call it (it is warp-synchronous); it returns the
// lane's new item, or -1.
constexpr int kClaimChunk = 64;

struct WarpClaim {
  int next = 0, end = 0;       // the warp's current chunk (uniform across the warp)
  bool done = false;           // the pass's items are all handed out
  int chunk = kClaimChunk;     // items per claim: smaller when the pass is small, so
                               // that its items spread over all warps of the grid
};

__device__ __forceinline__ int claim_chunk(int total) {
  const int warps = (int)(gridDim.x * blockDim.x) >> 5;
  return max(4, min(kClaimChunk, total / (4 * max(warps, 1))));
}

__device__ __forceinline__ int warp_claim(WarpClaim& w, bool need_one, int total, unsigned int* counter) {
  const unsigned full = 0xffffffffu;
  const unsigned need = __ballot_sync(full, need_one);
  if (need == 0 || w.done) return -1;
  const int lane = threadIdx.x & 31;
  const int rank = __popc(need & ((1u << lane) - 1u));
  const int k = __popc(need);
  int got = 0, mine = -1;
  for (int guard = 0; guard < 32 && got < k; ++guard) {
    if (w.next >= w.end) {
      int b = 0;
      if (lane == 0) b = (int)atomicAdd(counter, (unsigned)w.chunk);
      b = __shfl_sync(full, b, 0);
      if (b >= total) { w.done = true; break; }
      w.next = b;
      w.end = min(b + w.chunk, total);
    }
    const int take = min(k - got, w.end - w.next);
    if (need_one && rank >= got && rank < got + take) mine = w.next + (rank - got);
    got += take;
    w.next += take;
  }
  return mine;
}

// class-wide primary number gi of class cls -> job and history id (batched run)
__device__ __forceinline__ int job_of_primary(const DevProblem& P, int cls, uint64_t gi, uint32_t& hist,
                                              uint32_t& err) {
  const uint64_t* f = P.cls_first[cls];
  int lo = 0, hi = P.n_cls[cls];   // f[lo] <= gi < f[hi]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(f + mid) <= gi) lo = mid; else hi = mid;
  }
  const int j = chk(__ldg(P.cls_job[cls] + lo), P.n_jobs, err);
  hist = P.jobs[j].run_first + (uint32_t)(gi - __ldg(f + lo));
  return j;
}

template <bool BATCHED>
__device__ __forceinline__ void issue_primary(Track& t, const DevProblem& P, int cls, uint64_t gi, Live& p) {
  if (BATCHED) {
    uint32_t hist;
    const int j = job_of_primary(P, cls, gi, hist, t.err);
    t.J = P.jobs + j;
    primary(t, hist, p);
    p.job = j;
  } else {
    primary(t, P.job.run_first + (uint32_t)gi, p);
  }
}

// One pass over a queue of one particle type, its sizes read from the pass
// state the control kernel wrote. Items [0, n_in) come from the input queue;
// items [n_in, n_in + n_new) are new primaries, numbered prim0 + (i - n_in)
// within their particle class. PHOTON selects the photon or the charged physics.
// MODE: TALLY for transport; G_SUM and SCATTER are the adjoint's two replays
// (deposit weights in `wv`; the weights pointer is unused for TALLY)
// BATCHED: particles of several jobs share the queues; each carries its job,
// and new primaries are numbered over the jobs of their class
// VR: weighted particles (interaction forcing, splitting; transport only)
// MINB: resident threads per SM in units of 256. The photon kernel runs MINB
// blocks of 256 per SM; the charged kernel one block of 256 MINB threads per
// SM, so that its tables (about three times the photon region) are staged
// once per SM and the shared memory they leave free serves as L1 cache for
// the phantom and queue reads
template <bool PHOTON, int MINB, int MODE, bool BATCHED, bool VR>
__global__ void __launch_bounds__(PHOTON ? 256 : 256 * MINB, PHOTON ? MINB : 1)
    k_wf(const DevProblem P, const WfRing R, const PassState* __restrict__ ps,
         const float* __restrict__ wv) {
  if (ps->drain) return;   // the run's last pass belongs to the drain kernel
  const int cur = ps->cur;
  const int cls = PHOTON ? 0 : 1;
  const int n_in = ps->n_in[cls];
  const int n_new = ps->n_new[cls];
  const uint64_t prim0 = ps->prim0[cls];
  const int budget = PHOTON ? ps->budget_g : ps->budget_e;
  const int total = n_in + n_new;
  if ((int)(blockIdx.x * blockDim.x) >= total) return;   // no work for this block
  const Queue in = ring_queue(R.qmem, PHOTON ? cur : 2 + cur, R.cap);
  QueueSink out = ring_sink(R, cur);
  extern __shared__ float4 smem4[];
  float* stab = reinterpret_cast<float*>(smem4);
  if (PHOTON) wf_stage(P.tab, P.tab_g_floats, stab);
  else wf_stage(P.tab + P.tab_e_off, P.tab_e_floats, stab);
  Track t;
  wf_init(t, P, PHOTON ? stab : nullptr, PHOTON ? nullptr : stab, MODE);
  t.vr = VR;
  t.wv = wv;
  if (PHOTON) {
    // lock-step over Woodcock flights: each lane takes one flight per
    // iteration and the next photon when its own is done or out of budget.
    // A lane whose flight ends in a real collision holds it until at least
    // half of the warp's busy lanes hold one, and then they all carry out
    // their interactions together: the interaction code (type choice,
    // sampling, rotation, secondaries) is several flights long, and run by a
    // few lanes at a time it would leave the rest of the warp idle
    Live p;
    PhotonXs xs;
    PhotonHit hit;
    bool have = false, held = false;
    int nreal = 0, flights = 0;
    WarpClaim wc;
    wc.chunk = claim_chunk(total);
    unsigned int* claim = R.cnt + 4 + cls;
    for (int it = 0; it < (1 << 26); ++it) {
      const int i = warp_claim(wc, !have, total, claim);
      if (!__any_sync(0xffffffffu, have || i >= 0)) break;   // the warp's work is done
      if (i >= 0) {
        if (i < n_in) {
          Particle c;
          wf_load(in, chk(i, R.cap, t.err), c, VR);
          live_from(p, c);
          if (BATCHED) t.J = P.jobs + chk(p.job, P.n_jobs, t.err);
        } else {
          issue_primary<BATCHED>(t, P, cls, prim0 + (uint64_t)(i - n_in), p);
          t.l_src += p.E;
          ++t.c_part;
        }
        set_batch(t, p.batch);
        if (p.rng.n == 0 && p.path != 0) ++t.c_part;   // a secondary starts
        g_load(t, p.rng.hist);
        xs.lastE = -1.0f;
        have = true;
        nreal = 0;
        flights = 0;
      }
      if (have && !held) {
        const int st = photon_fly(t, p, xs, hit);
        ++flights;
        if (st == PH_DEAD) {
          have = false;
          g_release(t, p.rng.hist);
        } else if (st == PH_REAL) {
          held = true;
        } else if (flights >= kCapWoodcock) {   // runaway: flagged, energy counted as escaped
          t.err |= E_WOODCOCK;
          t.l_esc += (double)(p.E * p.wt);
          have = false;
          g_release(t, p.rng.hist);
        }
      }
      const unsigned n_held = __popc(__ballot_sync(0xffffffffu, held));
      const unsigned n_busy = __popc(__ballot_sync(0xffffffffu, have));
      if (held && 2u * n_held >= n_busy) {
        held = false;
        const int st = photon_interact(t, out, p, xs, hit);
        if (st == PH_DEAD) {
          have = false;
          g_release(t, p.rng.hist);
        } else if (++nreal >= budget) {
          have = false;
          g_release(t, p.rng.hist);
          Particle c;
          particle_from(c, p);
          out.append(t, c, 0, p.vox >= 0 ? p.vox : 0);
        }
      }
    }
    if (have || !wc.done) t.err |= E_WOODCOCK;   // iteration guard hit (not reached in practice)
  } else {
    // lock-step: each lane holds one particle and takes one step per
    // iteration, taking the next particle when its own is done, deferred or
    // out of budget, so that the warp runs the step code together
    Live p;
    Cell cell;
    bool have = false;
    int left = 0;
    WarpClaim wc;
    wc.chunk = claim_chunk(total);
    unsigned int* claim = R.cnt + 4 + cls;
    for (int it = 0; it < (1 << 24); ++it) {
      const int i = warp_claim(wc, !have, total, claim);
      if (!__any_sync(0xffffffffu, have || i >= 0)) break;   // the warp's work is done
      if (i >= 0) {
        if (i < n_in) {
          Particle c;
          wf_load(in, chk(i, R.cap, t.err), c, VR);
          live_from(p, c);
          if (BATCHED) t.J = P.jobs + chk(p.job, P.n_jobs, t.err);
        } else {
          issue_primary<BATCHED>(t, P, cls, prim0 + (uint64_t)(i - n_in), p);
          t.l_src += p.E;
          ++t.c_part;
        }
        set_batch(t, p.batch);
        if (p.rng.n == 0 && p.path != 0) ++t.c_part;   // a secondary starts
        if (!charged_begin(t, p, cell)) continue;
        g_load(t, p.rng.hist);
        have = true;
        left = min(budget, kCapEsteps);
      }
      if (!have) continue;
      const int st = charged_step<QueueSink, true>(t, out, p, cell);
      if (st == CT_ALIVE && --left > 0) continue;
      if (st == CT_ALIVE && left <= 0 && budget >= kCapEsteps) {   // no budget: a runaway
        t.err |= E_ESTEP;
        score(t, cell.v, p.E * p.wt);
        have = false;
        g_release(t, p.rng.hist);
        continue;
      }
      have = false;
      g_release(t, p.rng.hist);
      if (st != CT_DEAD) {
        p.vox = cell.v;
        Particle c;
        particle_from(c, p);
        out.append(t, c, st == CT_DEFERRED ? 2 : 1, cell.v);
      }
    }
    if (have || !wc.done) t.err |= E_ESTEP;   // iteration guard hit (not reached in practice)
  }
  wf_commit(t);
}

// The deferred events of charged particles (hard inelastic collisions, hard
// bremsstrahlung, positron annihilation), recorded by the charged kernel of the
// same pass; their count is read from the device. Keeping the secondary-making
// code out of the charged kernel keeps that kernel's instruction footprint small.
template <int MODE, bool BATCHED, bool VR>
__global__ void __launch_bounds__(256) k_knock(const DevProblem P, const WfRing R,
                                               const PassState* __restrict__ ps,
                                               const float* __restrict__ wv) {
  const int n_in = (int)min(R.cnt[2], (unsigned)R.cap);
  if ((int)(blockIdx.x * blockDim.x) >= n_in) return;
  const Queue in = ring_queue(R.qmem, 4, R.cap);
  QueueSink out = ring_sink(R, ps->cur);
  Track t;   // the deferred events need no tables
  wf_init(t, P, nullptr, nullptr, MODE);
  t.vr = VR;
  t.wv = wv;
  const int stride = gridDim.x * blockDim.x;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_in; i += stride) {
    Particle c;
    wf_load(in, chk(i, R.cap, t.err), c, VR);
    Live p;
    live_from(p, c);
    if (BATCHED) t.J = P.jobs + chk(p.job, P.n_jobs, t.err);
    set_batch(t, p.batch);
    g_load(t, p.rng.hist);
    const bool alive = knock(t, out, p);
    g_release(t, p.rng.hist);
    if (alive) {
      Particle d;
      particle_from(d, p);
      out.append(t, d, 1, p.vox);
    }
  }
  wf_commit(t);
}

// The run's last pass. Once every primary has been issued and fewer particles
// than the drain threshold are in flight, passes would each take the few
// particles left only as far as their next deferred event, and a run of long
// tracks (20 MeV electrons make a deferred event every few tens of steps)
// would end in dozens of passes, each as long as its slowest particle with the
// GPU nearly idle. Instead the control kernel marks the pass as the drain: the
// photon, charged and knock kernels do nothing, and this kernel runs every
// remaining particle -- the queued charged particles and photons and the run's
// last primaries -- with all of its secondaries to the end, the secondaries on
// a per-thread stack (deferred events sampled in place) as in the plain
// kernel. A particle's random stream travels with it, so the histories are
// unchanged: the run still replays the plain kernel's histories. Items are
// claimed one at a time (each is a whole subtree), charged particles first.
constexpr int kDrainStack = 48;

template <int MODE, bool BATCHED, bool VR>
__global__ void __launch_bounds__(256, 2) k_drain(const DevProblem P, const WfRing R,
                                                  const PassState* __restrict__ ps,
                                                  const float* __restrict__ wv) {
  if (!ps->drain) return;
  const int cur = ps->cur;
  const int e_in = ps->n_in[1], g_in = ps->n_in[0];
  const int e_end = e_in + ps->n_new[1];
  const int total = e_end + g_in + ps->n_new[0];
  if ((int)(blockIdx.x * blockDim.x) >= total) return;
  extern __shared__ float4 smem4[];
  float* stab = reinterpret_cast<float*>(smem4);
  wf_stage(P.tab, P.tab_e_off + P.tab_e_floats, stab);
  Track t;
  wf_init(t, P, stab, stab + P.tab_e_off, MODE);
  t.vr = VR;
  t.wv = wv;
  const Queue qg = ring_queue(R.qmem, cur, R.cap);
  const Queue qe = ring_queue(R.qmem, 2 + cur, R.cap);
  StackSink<kDrainStack> st;
  unsigned int* claim = R.cnt + 6;
  for (int it = 0; it < (1 << 26); ++it) {
    const int i = (int)atomicAdd(claim, 1u);
    if (i >= total) break;
    const bool photon = i >= e_end;
    const int cls = photon ? 0 : 1;
    const int k = photon ? i - e_end : i;
    const int n_in = photon ? g_in : e_in;
    Live p;
    if (k < n_in) {
      Particle c;
      wf_load(photon ? qg : qe, chk(k, R.cap, t.err), c, VR);
      live_from(p, c);
      if (BATCHED) t.J = P.jobs + chk(p.job, P.n_jobs, t.err);
    } else {
      issue_primary<BATCHED>(t, P, cls, ps->prim0[cls] + (uint64_t)(k - n_in), p);
      t.l_src += p.E;
      ++t.c_part;
    }
    set_batch(t, p.batch);
    if (p.rng.n == 0 && p.path != 0) ++t.c_part;   // a secondary starts
    const uint32_t hist = p.rng.hist;
    g_load(t, hist);
    if (photon) photon_track(t, st, p, 1 << 30);
    else charged_track(t, st, p, kCapEsteps);
    // its secondaries (and theirs) belong to the same history
    for (int g = 0; g < (1 << 20) && st.sp > 0; ++g) {
      live_from(p, st.s[--st.sp]);
      if (!VR) p.wt = 1.0f;
      track_to_death(t, st, p);
    }
    g_release(t, hist);
  }
  wf_commit(t);
}

size_t drain_smem_bytes(const DevProblem& P) {
  return ((size_t)(P.tab_e_off + P.tab_e_floats) * 4 + 15) & ~(size_t)15;
}

cudaError_t launch_drain_pass(const DevProblem& P, const WfRing& R, const PassState* ps, int grid,
                              const float* wv, cudaStream_t s) {
  const size_t smem = drain_smem_bytes(P);
  auto kern = P.jobs ? (P.vr_on ? k_drain<M_TALLY, true, true> : k_drain<M_TALLY, true, false>)
            : P.mode == M_G_SUM ? k_drain<M_G_SUM, false, false>
            : P.mode == M_SCATTER ? k_drain<M_SCATTER, false, false>
            : P.vr_on ? k_drain<M_TALLY, false, true> : k_drain<M_TALLY, false, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, smem, s>>>(P, R, ps, wv);
  return cudaGetLastError();
}

cudaError_t launch_knock_pass(const DevProblem& P, const WfRing& R, const PassState* ps, int grid,
                              int block, const float* wv, cudaStream_t s) {
  const size_t smem = wf_smem_bytes(P, 2);
  auto kern = P.jobs ? (P.vr_on ? k_knock<M_TALLY, true, true> : k_knock<M_TALLY, true, false>)
            : P.mode == M_G_SUM ? k_knock<M_G_SUM, false, false>
            : P.mode == M_SCATTER ? k_knock<M_SCATTER, false, false>
            : P.vr_on ? k_knock<M_TALLY, false, true> : k_knock<M_TALLY, false, false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(P, R, ps, wv);
  return cudaGetLastError();
}

cudaError_t launch_wavefront_pass(const DevProblem& P, bool photon, const WfRing& R,
                                  const PassState* ps, int grid, int block, int min_blocks,
                                  const float* wv, cudaStream_t s) {
  const size_t smem = wf_smem_bytes(P, photon ? 0 : 1);
  // both kernels have a variant compiled for 768 resident threads per SM
  // (register cap 80) and one for 512 (cap 128), chosen by min_blocks; the
  // adjoint's replays, batched runs and the weighted (variance-reduction)
  // variants use the default occupancy variants only
  auto kern =
      P.jobs ? (P.vr_on ? (photon ? k_wf<true, 2, M_TALLY, true, true> : k_wf<false, 3, M_TALLY, true, true>)
                        : (photon ? k_wf<true, 2, M_TALLY, true, false> : k_wf<false, 3, M_TALLY, true, false>))
      : P.mode == M_G_SUM ? (photon ? k_wf<true, 2, M_G_SUM, false, false> : k_wf<false, 3, M_G_SUM, false, false>)
      : P.mode == M_SCATTER ? (photon ? k_wf<true, 2, M_SCATTER, false, false>
                                      : k_wf<false, 3, M_SCATTER, false, false>)
      : P.vr_on ? (photon ? k_wf<true, 2, M_TALLY, false, true> : k_wf<false, 3, M_TALLY, false, true>)
      : photon ? (min_blocks >= 3 ? k_wf<true, 3, M_TALLY, false, false> : k_wf<true, 2, M_TALLY, false, false>)
               : (min_blocks >= 3 ? k_wf<false, 3, M_TALLY, false, false> : k_wf<false, 2, M_TALLY, false, false>);
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  kern<<<grid, block, smem, s>>>(P, R, ps, wv);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Pass control on the device: after each pass (and once before the first),
// one thread turns the pass's output counts into the next pass's sizes and
// budgets, tops the population up with new primaries, swaps the queue parity
// and clears the counters. No host round trip between passes: a run's passes
// are the body of a CUDA-graph while loop whose condition this kernel sets
// (in_graph: 1 while passes remain, 0 when the run is done), so the host
// submits a run once and never waits on it. Bounded: after max_passes the run
// stops with an error flag. loop[0] counts the executions inside the graph
// (loop iterations, 5 kernels each), loop[1] the passes scheduled with work.
// ---------------------------------------------------------------------------
__global__ void k_pass_ctl(const PassCtl c, PassState* __restrict__ ps, unsigned int* __restrict__ cnt,
                           unsigned int* __restrict__ err, int first, cudaGraphConditionalHandle h,
                           int in_graph, unsigned long long* __restrict__ loop) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  PassState st = *ps;
  int64_t ng = 0, ne = 0;
  if (!first) {
    ng = min(cnt[0], (unsigned)c.cap);
    ne = min(cnt[1], (unsigned)c.cap);
    st.cur ^= 1;
    // how much a pass multiplied its particles into one output queue
    const int64_t done_in = (int64_t)st.n_in[0] + st.n_new[0] + st.n_in[1] + st.n_new[1];
    if (done_in > 0) st.growth = fmaxf(st.growth, (float)max(ng, ne) / (float)done_in);
  } else {
    st.growth = 0.0f;
  }
  cnt[0] = 0; cnt[1] = 0; cnt[2] = 0;
  cnt[4] = 0; cnt[5] = 0; cnt[6] = 0;   // the transport kernels' work-claim counters
  st.busy = 0;
  st.drain = 0;
  st.n_in[0] = 0; st.n_in[1] = 0;
  st.n_new[0] = 0; st.n_new[1] = 0;
  if (!st.done) {
    const int64_t pop = ng + ne;
    const int64_t left_g = (int64_t)(c.n_prim[0] - st.issued[0]);
    const int64_t left_e = (int64_t)(c.n_prim[1] - st.issued[1]);
    const int64_t left = left_g + left_e;
    // queue room: the next pass's particles times the largest growth seen so
    // far (4 before any pass has run) must fit 85 % of a queue, else a
    // photon-rich workload (many tracked Compton electrons per photon and
    // pass) overflows the output queues
    const float g = st.passes == 0 ? 4.0f : fmaxf(st.growth, 1.0f);
    const int64_t room = (int64_t)(0.85f * (float)c.cap / g) - pop;
    int64_t n_new = min(min(max(c.target - pop, (int64_t)0), max(room, (int64_t)0)), left);
    // progress: with nothing in flight some primaries always go out (a
    // queue too small for the growth then overflows, flagged, instead of
    // ending the run with primaries left)
    if (pop == 0 && n_new == 0) n_new = min(left, (int64_t)max(1, c.cap / 8));
    // new primaries split between the classes by what each has left
    int64_t ng_new = left > 0 ? min(left_g, (int64_t)(((unsigned __int128)n_new * (uint64_t)left_g) /
                                                      (uint64_t)left)) : 0;
    int64_t ne_new = min(left_e, n_new - ng_new);
    ng_new = min(left_g, n_new - ne_new);
    ng_new = min(ng_new, (int64_t)c.cap - ng);
    ne_new = min(ne_new, (int64_t)c.cap - ne);
    if (pop == 0 && ng_new + ne_new == 0) {
      st.done = 1;
    } else if (st.passes >= c.max_passes) {
      st.done = 1;
      atomicOr(err, (unsigned)E_PASSES);
    } else {
      // the last pass: every primary issued and few particles left -- the
      // drain kernel runs them all to the end
      // (never the first pass, so that every run also goes through the
      // photon, charged and knock kernels)
      st.drain = st.passes > 0 && (pop + ng_new + ne_new) < c.drain && ng_new == left_g && ne_new == left_e;
      st.budget_g = c.budget_g;
      st.budget_e = c.budget_e;
      st.prim0[0] = st.issued[0];
      st.prim0[1] = st.issued[1];
      st.issued[0] += (uint64_t)ng_new;
      st.issued[1] += (uint64_t)ne_new;
      st.n_in[0] = (int)ng;
      st.n_in[1] = (int)ne;
      st.n_new[0] = (int)ng_new;
      st.n_new[1] = (int)ne_new;
      st.busy = 1;
      st.passes += 1;
      loop[1] += 1;
    }
  }
  *ps = st;
  if (in_graph) {
    loop[0] += 1;
    cudaGraphSetConditional(h, st.done ? 0u : 1u);
  }
}

cudaError_t launch_pass_ctl(const PassCtl& c, PassState* ps, unsigned int* cnt, unsigned int* err,
                            int first, unsigned long long* loop, cudaStream_t s,
                            cudaGraphConditionalHandle h, int in_graph) {
  k_pass_ctl<<<1, 32, 0, s>>>(c, ps, cnt, err, first, h, in_graph, loop);
  return cudaGetLastError();
}

}  // namespace gb
