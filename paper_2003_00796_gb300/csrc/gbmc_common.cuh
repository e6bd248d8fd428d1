// gbmc_common.cuh -- data layout, random numbers and table interpolation shared
// by the kernels and the host side of the library.
//
// Everything here is the library's own code; the CPU oracle is a separate
// implementation of the same physics reading and shares none of it.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/gbmc.h"

#if defined(__CUDACC__)
#define GB_HD __host__ __device__ __forceinline__
#define GB_D __device__ __forceinline__
#else
#define GB_HD inline
#define GB_D inline
#endif

namespace gb {

// ---------------------------------------------------------------------------
// Physical constants (CODATA) in the units of the library: MeV, cm, g.
// ---------------------------------------------------------------------------
constexpr double kMec2 = 0.51099895;
constexpr double kRe = 2.8179403262e-13;
constexpr double kAlpha = 1.0 / 137.035999084;
constexpr double kNa = 6.02214076e23;
constexpr double kPi = 3.14159265358979323846;
constexpr double kPeConst = 4.0e-32;   // photoelectric: sigma = K Z^4 / E^3, cm^2 MeV^3

constexpr float kMec2f = 0.51099895f;

// ---------------------------------------------------------------------------
// Table layout. Per material m and quantity q the table holds nE values on a
// uniform log2(E) grid; value = log2(quantity) except Q_XC (raw 1 - mu_c).
// Zero quantities (below a threshold) are stored as kLog2Zero.
// ---------------------------------------------------------------------------
enum TabQ {
  Q_MU_TOT = 0, Q_MU_CO, Q_MU_PE, Q_MU_RAY,      // photon, cm^2/g
  Q_SIG_EL, Q_SIG_INEL_E, Q_SIG_INEL_P, Q_SIG_BR, // hard event xs, cm^2/g
  Q_SIG1, Q_XC,                                   // soft transport xs; cut deflection
  Q_R_E, Q_R_P,                                   // CSDA range (+offset), g/cm^2
  Q_RINV_E, Q_RINV_P,                             // log2 E on a log2 r grid
  Q_SIG_H_E, Q_SIG_H_P,                           // hard el + inel + brems (e-, e+), cm^2/g
  NQ
};
constexpr float kLog2Zero = -140.0f;

// per-material parameters staged with the charged tables (shared memory, so
// that lanes on different materials read them without serialising): log2 r
// grid of the inverse range (e-, e+), element count, element CDF rows, and
// the screening constants of hard elastic events
enum MatPar {
  MP_LR0_E = 0, MP_INVDR_E, MP_LR0_P, MP_INVDR_P, MP_NEL, MP_OFF_EL,
  MP_EL_CA = 6, MP_EL_CB = MP_EL_CA + GBMC_MAX_EL, MP_STRIDE = MP_EL_CB + GBMC_MAX_EL
};

struct DevMat {
  int n_el;
  float ray_w[GBMC_MAX_EL];     // n_i Z_i^2 (per gram, scaled)
  float ray_iqz2[GBMC_MAX_EL];  // 1 / q_Z^2 (mc units)
  float el_w[GBMC_MAX_EL];      // n_i Z_i (Z_i + 1) (scaled)
  float el_cA[GBMC_MAX_EL];     // A = cA / p^2 * (1.13 + cB / beta^2)
  float el_cB[GBMC_MAX_EL];
};

struct Particle {      // a particle waiting on a stack or in a queue
  float x, y, z, u, v, w, E;
  uint32_t meta;       // type (bits 0-1) | deferred event (bits 2-3) | batch (bits 4-15)
                       // | job << 16
  uint32_t path_lo, path_hi, hist, nchild;
  uint32_t n;          // next draw of the particle's stream
  int vox;             // charged: voxel tracked by the DDA, -1 = locate
  float r;             // charged: residual range in the current material, < 0 = unset
  float wt;            // statistical weight (1 without variance reduction)
};

// structure-of-arrays particle queue (wavefront kernels): the record's 16
// words in four arrays of 16-byte field groups, so that a lane moves a
// record with four vector loads or stores, and lanes that take consecutive
// items touch consecutive 16-byte slots of each array:
//   pos = (x, y, z, u), dir = (v, w, E, meta), id = (path_lo, path_hi, hist,
//   nchild), st = (n, vox, r, wt)
struct Queue {
  float4* pos;
  float4* dir;
  uint4* id;
  float4* st;
};
constexpr int kQueueFields = 16;   // 4-byte words per record

// the ten round keys of Philox4x32-10 (k[2r], k[2r+1] for round r): the key
// schedule adds the Weyl constants once per run instead of once per block
struct PhiloxKeys { uint32_t k[20]; };

// what a deposit and a tentative photon collision do: the transport's tally,
// or one of the adjoint's two replays (see Track in transport.cuh)
enum TrackMode { M_TALLY = 0, M_G_SUM = 1, M_SCATTER = 2 };

// One transport job: a phantom, a source and a run of histories with its
// batch tiles. A single run has one (DevProblem::job); a batched run keeps an
// array of them in device memory and each particle carries its job's index.
struct DevJob {
  // phantom
  int nx, ny, nz, nxy;
  float inv_nx, inv_nxy;       // 1 / nx, 1 / (nx ny): a voxel index's coordinates
  float dx, dy, dz, idx, idy, idz, dmin;
  float step_len;              // class II step bound: step_vox voxel widths (times density)
  const uint8_t* mat;
  const float* rho;
  const float* major;          // photon majorant (log2, per energy node) in global memory;
                               // nullptr: the one staged with the tables
  // source
  int particle, shape, n_bins;
  float x0, y0, hx, hy, energy;
  const float* bin_prob;
  const int* bin_alias;
  const float* bin_edges;
  // rng key
  PhiloxKeys keys;             // round keys of (lo32(seed), hi32(seed) ^ job)
  // run: histories [run_first, run_first + run_n) in run_k batches
  uint32_t run_first;
  uint64_t run_n;
  int run_k;
  // tally: FP32 batch tiles, run_k tiles of tile_stride floats
  float* tile;
  int64_t tile_stride;
};

struct DevProblem {
  // tables
  const float* tab;            // global copy of the blob (two regions, see tab_off_e)
  int tab_g_floats;            // photon region: [0, tab_g_floats)
  int tab_e_off, tab_e_floats; // charged region: [tab_e_off, tab_e_off + tab_e_floats)
  int n_mat, nE, nR, nA;
  float lg0, inv_d;            // log2 E grid
  float lr0[GBMC_MAX_MAT][2], inv_dr[GBMC_MAX_MAT][2];  // log2 r grids
  float la0, inv_da;           // logit2(mbar) grid of the soft A' table
  int off_major;               // majorant, within the photon region
  int off_soft;                // soft A' table, within the charged region
  int off_mpar;                // per-material parameters (MatPar), within the charged region
  DevMat mats[GBMC_MAX_MAT];
  int off_el[GBMC_MAX_MAT];    // element CDF rows of material m within the charged
                               // region (-1: single element)
  // transport
  float eabs_g, eabs_e, wcc, wcr, step_keep;
  float lg_keep, lg_eabs_e;    // log2 of step_keep and of eabs_e
  // variance reduction: interaction forcing factors of hard inelastic
  // collisions and hard bremsstrahlung for e+- with weight in [vr_wlo, vr_whi],
  // and the number of copies of each bremsstrahlung photon (1, 1, 1: off)
  float vr_fi, vr_fb, vr_wlo, vr_whi;
  int vr_split;
  int vr_on;                   // any of them active: the weighted kernels run
  // the job of a single run
  DevJob job;
  // batched run: jobs[n_jobs]; primaries of particle class c (0 photon,
  // 1 charged) are numbered over the class's jobs in order: job
  // cls_job[c][k] owns primaries [cls_first[c][k], cls_first[c][k + 1])
  const DevJob* jobs;
  int n_jobs;
  const uint64_t* cls_first[2];
  const int* cls_job[2];
  int n_cls[2];
  // bookkeeping
  unsigned long long* counters;  // NCOUNT
  double* ledger;              // e_src, e_dep, e_esc, e_pair_net
  unsigned int* err;
  // adjoint on the wavefront path: G_h of the run's histories (index h - job.run_first)
  float* gbuf;
  int mode;                    // tracking mode of the run's kernels (host dispatch)
};

constexpr int kCapWoodcock = 1 << 20;   // tentative collisions per photon flight
constexpr int kCapEsteps = 1 << 17;     // steps per charged particle
constexpr int kCapDda = 1 << 16;        // voxel crossings per charged segment
constexpr int kCapReject = 1 << 12;     // rejection-sampling trials

enum Counter { C_TENT = 0, C_REAL, C_ESTEP, C_CROSS, C_HARD, C_PART, NCOUNT };
enum ErrBit { E_STACK = 1u, E_WOODCOCK = 2u, E_ESTEP = 4u, E_DDA = 8u, E_REJECT = 16u, E_QUEUE = 32u,
              E_PASSES = 64u, E_BOUNDS = 128u };

// Checked build (the same sources compiled with -DGBMC_CHECKED into
// libgbmc_checked.so): every voxel, material, batch, job, queue-slot, alias-bin,
// element and adjoint-buffer index is tested against its bound before it is
// used. An index out of range records E_BOUNDS in the thread's error word
// and is replaced by 0, so that the run ends with GBMC_ERR_BOUNDS instead of
// touching memory out of range. In the default build kChecked is false, the
// tests fold away and the generated code is that of the unchecked sources.
#ifdef GBMC_CHECKED
constexpr bool kChecked = true;
#else
constexpr bool kChecked = false;
#endif

// i if 0 <= i < n, else 0 with E_BOUNDS recorded
GB_D int chk(int i, int64_t n, uint32_t& err) {
  if (kChecked && !(i >= 0 && (int64_t)i < n)) { err |= E_BOUNDS; return 0; }
  return i;
}

// the same for an unsigned 32-bit offset
GB_D uint32_t chk_u(uint32_t i, uint64_t n, uint32_t& err) {
  if (kChecked && !((uint64_t)i < n)) { err |= E_BOUNDS; return 0u; }
  return i;
}

// an invariant of the transport state (checked build only): false records E_BOUNDS
GB_D bool chk_true(bool ok, uint32_t& err) {
  if (kChecked && !ok) { err |= E_BOUNDS; return false; }
  return true;
}

// wavefront queues: five SoA queues of cap particles in one allocation
// (photon in/out, charged in/out by pass parity, deferred charged events)
// and their counters: appends (photons out, charged out, deferred) at 0-2,
// the photon, charged and drain kernels' work claims at 4-6
struct WfRing {
  float* qmem;
  unsigned int* cnt;
  int cap;
};

// what a wavefront pass does, written on the device by the pass-control kernel;
// primaries are counted per particle class (0 photon, 1 charged)
struct PassState {
  int n_in[2];                 // queued photons, charged particles
  int n_new[2];                // primaries issued in this pass, per class
  int cur;                     // parity of the input queues
  int budget_g, budget_e;      // real photon events / class II steps per particle
  int done, busy, passes;
  int drain;                   // the run's last pass: every particle runs to the end (k_drain)
  uint64_t prim0[2];           // class-wide number of the pass's first new primary
  uint64_t issued[2];          // primaries issued so far, per class
  float growth;                // largest (queue output / particles processed) of a pass so far
};

// the run's constants for the pass control
struct PassCtl {
  uint64_t n_prim[2];          // primaries of each class in the run
  int64_t target, drain;
  int cap, budget_g, budget_e, max_passes;
};

// The table blob has two regions, each staged into shared memory only by the
// kernels that need it:
//   photon region at 0: Q_MU_* of every material (4 n_mat nE), then the photon
//     majorant (nE);
//   charged region at tab_off_e(): the other quantities, the soft A' table
//     (nA), then the element CDF rows of hard elastic events.
GB_HD int tab_region_g(int n_mat, int nE) { return (4 * n_mat + 1) * nE; }
GB_HD int tab_off_e(int n_mat, int nE) { return (tab_region_g(n_mat, nE) + 3) & ~3; }

// offset of quantity q of material m within its region
GB_HD int tab_rel(int q, int m, int n_mat, int nE) {
  return q < Q_SIG_EL ? (q * n_mat + m) * nE : ((q - Q_SIG_EL) * n_mat + m) * nE;
}

// offset of quantity q of material m in the blob
GB_HD int tab_off(int q, int m, int n_mat, int nE) {
  return (q < Q_SIG_EL ? 0 : tab_off_e(n_mat, nE)) + tab_rel(q, m, n_mat, nE);
}

// blob size before the element CDF rows
inline size_t tab_size_floats(int n_mat, int nE, int nR, int nA) {
  (void)nR;
  return (size_t)tab_off_e(n_mat, nE) + (size_t)(NQ - Q_SIG_EL) * n_mat * nE + nA;
}

// ---------------------------------------------------------------------------
// Interpolation on a uniform grid: position (i, f) of x, value of a table.
// ---------------------------------------------------------------------------
struct GridPos { int i; float f; };

GB_HD GridPos grid_pos(float lx, float l0, float inv_d, int n) {
  float t = (lx - l0) * inv_d;
  t = fminf(fmaxf(t, 0.0f), (float)(n - 1) - 1e-3f);
  int i = (int)t;
  GridPos p; p.i = i; p.f = t - (float)i;
  return p;
}

GB_HD float lerp_tab(const float* t, GridPos p) {
  const float a = t[p.i], b = t[p.i + 1];
  return fmaf(p.f, b - a, a);
}

GB_HD float exp2_tab(const float* t, GridPos p) { return exp2f(lerp_tab(t, p)); }

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11)
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

GB_HD PhiloxKeys philox_keys(uint32_t k0, uint32_t k1) {
  PhiloxKeys K;
  for (int r = 0; r < 10; ++r) {
    K.k[2 * r] = k0;
    K.k[2 * r + 1] = k1;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return K;
}

GB_HD U4 philox4x32_10(U4 c, const PhiloxKeys& K) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // each product as one 32 x 32 -> 64-bit multiply (high and low words)
    const uint64_t p0 = (uint64_t)0xD2511F53u * c.x, p1 = (uint64_t)0xCD9E8D57u * c.z;
    const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    U4 n;
    n.x = hi1 ^ c.y ^ K.k[2 * r];
    n.y = lo1;
    n.z = hi0 ^ c.w ^ K.k[2 * r + 1];
    n.w = lo0;
    c = n;
  }
  return c;
}

// child path: splitmix64 finaliser of parent + ordinal * golden gamma
GB_HD uint64_t child_path(uint64_t parent, uint32_t ordinal) {
  uint64_t z = parent + (uint64_t)ordinal * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// uniform in (0,1): ((w >> 9) + 0.5) * 2^-23, exact in binary32
GB_HD float word_to_uniform(uint32_t w) {
  return ((float)(w >> 9) + 0.5f) * (1.0f / 8388608.0f);
}

// -ln u for u in (0,1), never negative: the device code is built with
// approximate (MUFU) logarithms, whose absolute error can push ln u above 0
// for u within a few ulp of 1
GB_HD float neg_log(float u) { return fmaxf(-logf(u), 0.0f); }

// A particle's random stream: draw n is word n % 4 of
// Philox(counter = (hist, path_lo, path_hi, n / 4), key).
struct Rng {
  uint32_t hist, plo, phi, n;
  uint32_t blk;            // block held in w[], 0xffffffff = none
  uint32_t w0, w1, w2, w3;
};

GB_HD void rng_init(Rng& r, uint32_t hist, uint64_t path, uint32_t n) {
  r.hist = hist; r.plo = (uint32_t)path; r.phi = (uint32_t)(path >> 32); r.n = n;
  r.blk = 0xffffffffu;
}

GB_HD float rng_draw(Rng& r, const PhiloxKeys& K) {
  const uint32_t b = r.n >> 2;
  if (b != r.blk) {
    U4 c; c.x = r.hist; c.y = r.plo; c.z = r.phi; c.w = b;
    const U4 o = philox4x32_10(c, K);
    r.w0 = o.x; r.w1 = o.y; r.w2 = o.z; r.w3 = o.w; r.blk = b;
  }
  const uint32_t s = r.n & 3u;
  const uint32_t w = (s == 0) ? r.w0 : (s == 1) ? r.w1 : (s == 2) ? r.w2 : r.w3;
  ++r.n;
  return word_to_uniform(w);
}

// Fixed-slot draws: a photon flight takes one whole block, a class II step
// two, starting at the next block boundary (draw index n rounded up to a
// multiple of 4); n moves past them and the first block's index is returned.
GB_HD uint32_t rng_take_blocks(Rng& r, uint32_t k) {
  const uint32_t b = (r.n + 3u) >> 2;
  r.n = (b + k) << 2;
  return b;
}

GB_HD U4 rng_block(const Rng& r, uint32_t b, const PhiloxKeys& K) {
  U4 c; c.x = r.hist; c.y = r.plo; c.z = r.phi; c.w = b;
  return philox4x32_10(c, K);
}

}  // namespace gb
