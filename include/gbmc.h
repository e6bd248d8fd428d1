/*
 * gbmc.h -- C ABI of the GB300 (sm_103a) voxel dose Monte Carlo library.
 *
 * The library runs the data-parallel history loop of PenRed (arXiv 2003.00796,
 * Sec. 4.1 and Fig. "flowTally": sample a primary, then JUMP / STEP / KNOCK for
 * it and its secondaries, scoring energy into a tally) for photons, electrons
 * and positrons in a voxelised phantom (Sec. 4.2.2), with the tally's mean and
 * standard deviation per voxel (Sec. 4.2.3, Eq. 1-3).
 *
 * Conventions (all entry points):
 *  - Every call returns a gbmc_status; nothing throws across the ABI.
 *    gbmc_last_error() gives a human-readable message for the last failure.
 *  - Inputs are copied by the library (the caller keeps ownership of every
 *    pointer passed in). Outputs go to caller buffers of the documented size.
 *  - ptr_kind: GBMC_PTR_HOST for host memory, GBMC_PTR_DEVICE for device
 *    memory on the context's device (e.g. a torch CUDA tensor's data_ptr).
 *  - A context is bound to one device and is not thread-safe: use one context
 *    per host thread. gbmc_run is asynchronous on the given CUDA stream
 *    (NULL = legacy default stream); the getters synchronise that stream.
 *  - Device-side loops are bounded; a bound that is hit retires the particle,
 *    sets an error flag and makes gbmc_run / gbmc_get_stats report
 *    GBMC_ERR_DEVICE_LIMIT (the context stays usable).
 *  - Layout of voxel arrays: C order [iz][iy][ix], nx*ny*nz elements; the
 *    grid occupies [0, nx dx] x [0, ny dy] x [0, nz dz] cm, vacuum outside.
 */
#ifndef GBMC_H
#define GBMC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gbmc_ctx gbmc_ctx;

typedef enum {
  GBMC_OK = 0,
  GBMC_ERR_ARG = 1,          /* invalid argument (null, size, NaN/negative density, ...) */
  GBMC_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  GBMC_ERR_OOM = 3,          /* device allocation failed */
  GBMC_ERR_STATE = 4,        /* call out of order (e.g. run before load_phantom) */
  GBMC_ERR_DEVICE_LIMIT = 5, /* a bounded device loop gave up (see gbmc_stats.error_flags) */
  GBMC_ERR_STACK = 6,        /* a per-thread secondary stack overflowed */
  GBMC_ERR_BOUNDS = 7        /* checked build only: an index out of range was caught */
} gbmc_status;

enum { GBMC_PTR_HOST = 0, GBMC_PTR_DEVICE = 1 };
enum { GBMC_PHOTON = 0, GBMC_ELECTRON = 1, GBMC_POSITRON = 2 };
enum { GBMC_KERNEL_PLAIN = 0, GBMC_KERNEL_WAVEFRONT = 1 };

#define GBMC_MAX_MAT 4
#define GBMC_MAX_EL 8
#define GBMC_MAX_BINS 256
/* Largest number of batches per run (gbmc_options.n_batches): a particle
 * record carries its history's batch in a few bits, and the flush keeps the
 * batch weights 1/n_k in shared memory. */
#define GBMC_MAX_BATCHES 1024

/* A material as element mass fractions (Sec. 5: PENELOPE material files are
 * replaced by this closed-form description). */
typedef struct {
  int n_el;                  /* 1..GBMC_MAX_EL */
  int Z[GBMC_MAX_EL];        /* atomic numbers */
  double A[GBMC_MAX_EL];     /* atomic weights, g/mol */
  double w[GBMC_MAX_EL];     /* mass fractions (normalised by the library) */
  double I_eV;               /* mean excitation energy for the Bethe formula */
} gbmc_material;

/* Transport parameters (the E_abs, C1, C2, W_cc, W_cr set of Sec. 5.2). */
typedef struct {
  double eabs_g;             /* photon absorption energy, MeV */
  double eabs_e;             /* electron/positron absorption energy, MeV */
  double wcc;                /* hard inelastic cut-off, MeV */
  double wcr;                /* hard bremsstrahlung cut-off, MeV */
  double c1;                 /* hard elastic mfp = max(lambda_el, c1 lambda_1) */
  double step_frac;          /* max fractional CSDA energy loss per step (C2-like) */
  double step_vox;           /* max step, in voxel widths */
} gbmc_transport;

/* Primary state sampler (Sec. 4.2.1): position on the z = 0 face, direction
 * +z, energy mono or binned. */
typedef struct {
  int particle;              /* GBMC_PHOTON / GBMC_ELECTRON / GBMC_POSITRON */
  int shape;                 /* 0: pencil at (x0, y0); 1: uniform rectangle */
  double x0, y0;             /* cm */
  double hx, hy;             /* rectangle half widths, cm */
  double energy;             /* MeV, when n_bins == 0 */
  int n_bins;                /* 0 or 1..GBMC_MAX_BINS */
  const double* edges;       /* n_bins + 1 increasing bin edges, MeV (host) */
  const double* weights;     /* n_bins non-negative bin weights (host) */
} gbmc_source;

typedef struct {
  int kernel;                /* GBMC_KERNEL_PLAIN or GBMC_KERNEL_WAVEFRONT */
  int n_batches;             /* batches per gbmc_run for the variance (2..GBMC_MAX_BATCHES;
                                0 = 40); others make gbmc_create return GBMC_ERR_ARG */
  int block;                 /* threads per block (0 = library default) */
  int blocks_per_sm;         /* grid = blocks_per_sm * SMs, capped per kernel at what its
                                registers keep resident (0 = per kernel: 3 for the charged
                                and knock kernels, 2 for the photon and plain kernels;
                                >= 3 also selects the photon kernel compiled for 3). The
                                charged kernel runs the same threads per SM as one block
                                (block * its blocks per SM threads, one block per SM), so
                                that its tables are staged once per SM */
  int stack_cap;             /* per-thread secondary stack capacity of the plain and drain
                                kernels: fixed at 48 records when the kernels are compiled;
                                0 or 48, other values return GBMC_ERR_ARG */
  int queue_cap;             /* wavefront queue capacity in particles (0 = 2^24: five
                                queues of 64-byte records, 5.4 GB); the run's last pass
                                (the drain) runs the particles left to the end on per-thread
                                stacks of 48 records instead of queues */
  int timing;                /* 1: time every transport and flush launch with CUDA
                                events on the run's stream (gbmc_stats *_ms fields) */
  int photon_budget;         /* wavefront: real photon interactions per photon per
                                pass (0 = 16) */
  int charged_budget;        /* wavefront: class II steps per e-/e+ per pass (0 = 32) */
  int pass_target;           /* wavefront: particles in flight that new primaries top
                                the queues up to each pass (0 = queue_cap / 2); fewer
                                while the largest queue growth a pass has shown says
                                they would overflow 85 % of a queue */
  int ledger_check;          /* plain kernel only (GBMC_ERR_ARG with the wavefront
                                kernel): 1 checks every history's energy ledger in
                                FP64 (source = deposits + escapes + 2mc^2 (pairs -
                                annihilations)); the largest relative residual is in
                                gbmc_stats.max_ledger_rel */
} gbmc_options;

/* Event counters and the energy ledger, summed over all gbmc_run and
 * gbmc_run_batch calls since the last gbmc_reset_tally. */
typedef struct {
  uint64_t n_hist, n_batches;
  uint64_t n_tent;           /* photon Woodcock tentative collisions */
  uint64_t n_real;           /* photon real interactions */
  uint64_t n_e_steps;        /* charged-particle steps */
  uint64_t n_cross;          /* charged-particle voxel crossings */
  uint64_t n_hard;           /* charged-particle hard events (incl. delta) */
  uint64_t n_particles;      /* particles tracked (primaries + secondaries) */
  double e_src, e_dep, e_esc;  /* MeV: source, deposited, escaped */
  double e_pair_net;         /* MeV: 2mc^2 (n_pair - n_annih) */
  uint32_t error_flags;      /* bit 0 stack overflow, 1 Woodcock cap, 2 e-step cap,
                                3 DDA cap, 4 rejection cap, 5 queue overflow,
                                6 wavefront pass cap, 7 index out of range (checked
                                build only, GBMC_FLAG_BOUNDS) */
  uint32_t reserved;
  double last_run_ms;        /* device time of the last gbmc_run (all launches) */
  double transport_ms;       /* summed device time of the charged-particle (wavefront) or
                                plain transport launches (timing = 1) */
  double flush_ms;           /* summed device time of flush launches (timing = 1) */
  uint64_t n_transport_launches, n_flush_launches;
  double photon_ms;          /* summed device time of wavefront photon launches (timing = 1) */
  uint64_t n_photon_launches;
  uint64_t n_kernel_launches;  /* every kernel the library launched for gbmc_run, including
                                the ones run by the wavefront pass loop's CUDA graph */
  uint64_t n_passes;         /* wavefront passes with work */
  uint64_t n_graph_launches; /* CUDA-graph launches of the wavefront pass loop (one per
                                wavefront run: the loop over passes runs on the device) */
  double max_ledger_rel;     /* ledger_check: largest |residual| / source energy of a history */
  uint64_t n_ledger_checked; /* ledger_check: histories checked */
  double drain_ms;           /* summed device time of the wavefront's drain launches, the
                                run's last pass (timing = 1) */
  uint64_t n_drain_launches;
} gbmc_stats;

/* Create a context on `device` (Sec. 4.1: one simulation object holding the
 * configured geometry, materials, source and tallies; Sec. 4.3: one per worker,
 * here one per GPU and host thread). opt may be NULL (defaults); out-of-range
 * options return GBMC_ERR_ARG and leave *out NULL. device < 0 makes a host-only
 * context (tables and host helpers, no GPU). Release it with gbmc_destroy. */
gbmc_status gbmc_create(gbmc_ctx** out, int device, const gbmc_options* opt);

/* Device-memory limit of a context. The paper has no counterpart (PenRed runs
 * in host memory); it is for programs that share one GPU between several
 * contexts or other work and give each a budget. Every problem-sized device
 * buffer of the context (tables, phantom, batch tiles and tally sums, the
 * wavefront queues, the buffers of batched jobs and of the adjoint) comes from
 * one allocator, which counts the bytes it holds. limit_bytes caps that count
 * (0 = no limit, the default); an allocation that would pass it fails as a
 * failed cudaMalloc does: GBMC_ERR_OOM, nothing allocated, and the context
 * usable (the call can be repeated after a higher limit, or with a smaller
 * problem). A failed call leaves the state it was building unset -- materials
 * (gbmc_set_materials again), phantom, source, or the batched run whose job
 * doses then cannot be read -- and runs refuse it with GBMC_ERR_STATE.
 * Lowering the limit frees nothing. Small fixed buffers (counters, error
 * word, pass state) are not counted. gbmc_mem_info returns the bytes held and
 * the limit. NULL arguments: GBMC_ERR_ARG. */
gbmc_status gbmc_set_mem_limit(gbmc_ctx* ctx, uint64_t limit_bytes);
gbmc_status gbmc_mem_info(const gbmc_ctx* ctx, uint64_t* held_bytes, uint64_t* limit_bytes);

/* Set materials (n_mat <= GBMC_MAX_MAT; material index = phantom id) and
 * transport parameters, and build the FP32 log-energy tables from the closed
 * forms in FP64 on the host (e_max: largest energy to tabulate, MeV). */
gbmc_status gbmc_set_materials(gbmc_ctx* ctx, const gbmc_material* mats, int n_mat,
                               const gbmc_transport* tp, double e_max);

/* Load the voxel phantom: mat[v] < n_mat, rho[v] finite and > 0 (g/cm^3).
 * Requires gbmc_set_materials first (the photon majorant needs both). */
gbmc_status gbmc_load_phantom(gbmc_ctx* ctx, int nx, int ny, int nz,
                              double dx, double dy, double dz,
                              const uint8_t* mat, const float* rho, int ptr_kind);

/* Set the primary source. Energies must lie in (eabs, e_max]. */
gbmc_status gbmc_set_source(gbmc_ctx* ctx, const gbmc_source* src);

/* Run histories [first_hist, first_hist + n_hist) (history ids < 2^32) with
 * Philox seed `seed` and job id 0, in opt.n_batches batches, adding to the
 * tally: the history loop of Sec. 4.1 (sample a primary, then JUMP / STEP /
 * KNOCK for it and every secondary), the histories split into batches as the
 * paper splits them among threads (Sec. 4.3, Eq. 3). Calls with disjoint id
 * ranges add up. Asynchronous on `cuda_stream` (a cudaStream_t or NULL): the
 * call enqueues the work and returns without waiting (the wavefront kernel's
 * pass loop is one CUDA-graph launch whose while loop is driven by a device
 * control kernel; with opt.timing the passes are launched and read back one
 * by one, and the call returns when they are done); the getters synchronise.
 * Errors of the device-side loop bounds are reported by the next getter. */
gbmc_status gbmc_run(gbmc_ctx* ctx, uint64_t n_hist, uint64_t seed, uint64_t first_hist,
                     void* cuda_stream);

/* Dose per voxel in MeV/g per primary history, and the variance of that mean
 * (the tally of Sec. 4.2.3: mean over histories as in Eq. 1, its uncertainty
 * from the batch means, the GPU form of Eq. 2-3). Each array has nx*ny*nz
 * doubles (caller-owned, on host or device by ptr_kind); var may be NULL.
 * Synchronises the last run's stream; GBMC_ERR_STATE before any history. */
gbmc_status gbmc_get_dose(gbmc_ctx* ctx, double* dose, double* var, int ptr_kind);

/* Raw tally: mean energy per history per voxel (MeV) and its variance. */
gbmc_status gbmc_get_edep(gbmc_ctx* ctx, double* mean, double* var, int ptr_kind);

/* Event counters of the history loop (Sec. 4.1: the JUMP / STEP / KNOCK
 * events that take 80-90 % of the run time), the energy ledger and the device
 * times, summed since the last reset. Synchronises the last run's stream;
 * returns GBMC_ERR_DEVICE_LIMIT / GBMC_ERR_STACK if a device loop bound or a
 * secondary stack overflowed (out is filled all the same). */
gbmc_status gbmc_get_stats(gbmc_ctx* ctx, gbmc_stats* out);

/* Zero the tally (Sec. 4.2.3: the tally's accumulators, as a new simulation
 * starts them), the batch count and the statistics. Synchronises the device. */
gbmc_status gbmc_reset_tally(gbmc_ctx* ctx);

/* Tally moments, for combining runs made elsewhere (Sec. 4.3: workers and MPI
 * processes meet only at the end, where their counters are summed, Eq. 3).
 * Per voxel S1 = sum_k B_k (MeV) and S2 = sum_k B_k^2 / n_k over every batch
 * k of the tally (B_k: energy deposited by the n_k histories of batch k), with
 * the tally's history and batch counts. Mean energy per history = S1 / N and
 * its variance (S2 - N mean^2) / (N (K - 1)); moments of several tallies add.
 *   gbmc_get_moments copies S1 and S2 (nx*ny*nz doubles each, caller-owned,
 *   host or device by ptr_kind) and the counts; synchronises the last run.
 *   gbmc_add_moments adds the given S1, S2 and counts to the tally, so that
 *   gbmc_get_dose / gbmc_get_edep then report the combined estimate. A
 *   multi-GPU run: every rank gets its moments, an all-reduce sums them,
 *   every rank resets its tally and adds the sums.
 * GBMC_ERR_STATE without a phantom; null arrays or counts -> GBMC_ERR_ARG. */
gbmc_status gbmc_get_moments(gbmc_ctx* ctx, double* s1, double* s2, uint64_t* n_hist,
                             uint64_t* n_batches, int ptr_kind);
gbmc_status gbmc_add_moments(gbmc_ctx* ctx, const double* s1, const double* s2, uint64_t n_hist,
                             uint64_t n_batches, int ptr_kind);

/* One job of a batched run: its own phantom, source and histories. */
typedef struct {
  int nx, ny, nz;            /* voxels per axis */
  double dx, dy, dz;         /* voxel size, cm */
  const uint8_t* mat;        /* host, nx*ny*nz material ids (< the context's n_mat) */
  const float* rho;          /* host, nx*ny*nz densities, g/cm^3 (finite, > 0) */
  gbmc_source src;           /* primary source (max energy within the tables' range) */
  uint64_t n_hist;           /* histories [first_hist, first_hist + n_hist), ids < 2^32 */
  uint64_t first_hist;
  uint64_t seed;             /* Philox seed; the key's job id is the job's index */
} gbmc_job;

/* Batched run (many beams and phantoms of uneven size in one run): every job
 * of jobs[n_jobs] (1 <= n_jobs <= 65535) is transported by the same wavefront
 * pass loop (Sec. 4.1 history loop; the jobs' particles share the queues and
 * each carries its job; new primaries are claimed job by job on the device,
 * the GPU form of the dynamic work assignment of Sec. 4.3), submitted as one
 * CUDA-graph launch whose while loop runs the passes until all jobs are done.
 * Materials and transport settings are the context's (gbmc_set_materials,
 * whose e_max must cover every job's source); each job has its own phantom,
 * photon majorant, source, Philox key (seed, job id = index), and
 * min(opt.n_batches, n_hist) batches. The library copies the inputs (the
 * phantoms are validated on the device: material ids below the context's
 * material count, finite positive densities); a job's device memory is about
 * nvox * (5 + 4 * batches + 16) bytes and is kept for the next batched run,
 * which reuses it when every job has the same voxel and batch counts. Results
 * (gbmc_get_job_dose) stay until the next gbmc_run_batch; the run does not
 * touch the single-run tally. Synchronous: returns when every job is done.
 * Each job's histories are those of a single run with the same phantom,
 * source, seed and job id (the same random numbers for the same particles; a
 * rare particle can round differently in FP32 depending on which kernel
 * finishes it). */
gbmc_status gbmc_run_batch(gbmc_ctx* ctx, const gbmc_job* jobs, int n_jobs, void* cuda_stream);

/* Dose (MeV/g per history) and variance of the mean of job `job` of the last
 * batched run; arrays of that job's nx*ny*nz doubles; var may be NULL. */
gbmc_status gbmc_get_job_dose(gbmc_ctx* ctx, int job, double* dose, double* var, int ptr_kind);

/* Autotuner of the wavefront options (opt.kernel must be WAVEFRONT): times
 * trial runs of the same histories -- a single run of n_trial histories of the
 * loaded phantom and source (jobs = NULL), or the batch `jobs` with every
 * job's histories scaled to n_trial in total -- over the class II step budget
 * {8, 16, 32}, the photon event budget {4, 8, 16}, the pass target (queue
 * depth) {cap/8, cap/4, cap/2}, and the block shape: threads per block
 * {128, 256} and resident blocks per SM {per-kernel default, 2, 3}; one option
 * at a time in two sweeps, keeping a change when it is more than 2 % faster.
 * Stores the choice in the context's options and copies it to `chosen` (may
 * be NULL). The tally and statistics are reset afterwards (and, with jobs,
 * the last batched run is replaced). The paper's counterpart is the
 * user-chosen thread count of Sec. 6.1-6.2. */
gbmc_status gbmc_autotune(gbmc_ctx* ctx, const gbmc_job* jobs, int n_jobs, uint64_t n_trial,
                          uint64_t seed, void* cuda_stream, gbmc_options* chosen);

/* Fix the photon majorant (Woodcock tracking, Sec. 4.2.2 geometry) from the
 * given per-material densities rho_maj[n_mat] (g/cm^3) instead of the loaded
 * phantom's maxima, so that it does not move when densities are perturbed
 * (finite differences, gradients). n_mat must equal the material count and
 * every value must be >= that material's largest phantom density (else
 * GBMC_ERR_ARG; a later gbmc_load_phantom that violates it fails the same
 * way). rho_maj = NULL returns to the phantom's maxima; gbmc_set_materials
 * also resets it. */
gbmc_status gbmc_set_majorant(gbmc_ctx* ctx, const double* rho_maj, int n_mat);

/* Variance reduction (Sec. 5.2 runs its 40 keV electron example with hard
 * bremsstrahlung and hard inelastic collisions forced by factors 2000 and 200
 * and bremsstrahlung photons split in two). Every particle carries a weight
 * (primaries 1); deposits and escapes are weighted.
 *   Interaction forcing: for an electron or positron whose weight lies in
 *   [w_lo, w_hi], the hard inelastic and hard bremsstrahlung cross sections
 *   are multiplied by f_inel and f_brems. At such an event the secondary
 *   carries the particle's weight divided by the factor, and the particle
 *   takes the energy loss and deflection with probability 1 / factor (one
 *   more uniform, drawn after the event's own samples).
 *   Splitting: each bremsstrahlung photon is emitted as n_split_brems copies
 *   of 1 / n_split_brems of its weight; copy 0 takes the stream of the
 *   particle's next child, copy k >= 1 the child stream of ordinal 2^31 + k
 *   of copy 0's path, so every other stream of the history is the one of
 *   the run without splitting.
 * Unbiased: the dose and its variance estimate keep their meaning; the energy
 * ledger holds per history without forcing and in expectation with it.
 * vr = NULL (or factors 1, n_split_brems 1) switches it off. Values:
 * f_inel, f_brems in [1, 1e6], 0 <= w_lo <= w_hi, n_split_brems in [1, 64],
 * else GBMC_ERR_ARG. gbmc_adjoint refuses (GBMC_ERR_STATE) while it is on.
 * Applies to every later run, batched runs included. */
typedef struct {
  double f_inel, f_brems;    /* forcing factors (>= 1) */
  double w_lo, w_hi;         /* weight window of forced particles */
  int n_split_brems;         /* copies of each bremsstrahlung photon (>= 1) */
} gbmc_vr;
gbmc_status gbmc_set_vr(gbmc_ctx* ctx, const gbmc_vr* vr);

/* Path-replay adjoint: dL/drho_v per voxel (MeV/g per history per g/cm^3 of
 * density, times the units of L) for a given dL_dD[nx*ny*nz] = dL/dD_v (D the
 * dose of gbmc_get_dose), by the likelihood-ratio (score-function) estimator
 * of the derivative of the dose tally (Sec. 4.2.3, Eq. 1); the paper does not
 * differentiate its method, this is the estimator stated here:
 *   per history h: G_h = sum_v g_v q_hv / (rho_v V), q_hv its deposits;
 *   c_hv = G_h S_hv - g_v q_hv / (rho_v^2 V), with S_hv summing over h's
 *   tentative photon collisions in v the score 1/rho_v (real) or
 *   -kappa / (mbar - rho_v kappa) (virtual; kappa the mass attenuation of the
 *   voxel's material, mbar the majorant);  dL/drho_v = E_h[c_hv].
 * Each history of [first_hist, first_hist + n_hist) is run twice from its
 * Philox key (first summing G_h, then scattering c_hv), in opt.n_batches
 * batches; grad gets the mean and var (may be NULL) the variance of that mean.
 * opt.kernel picks the replay kernels: PLAIN keeps G_h in a register per
 * history; WAVEFRONT runs both replays as wavefront runs with G_h in a
 * per-history device buffer (4 bytes per history, in chunks of 2^26
 * histories, each chunk with its own batches). Both give the same histories.
 * Exact when only photon flights depend on density (charged particles
 * absorbed where they are made: eabs_e above the source energy); with
 * charged transport the density dependence of electron steps is left out.
 * Use a fixed majorant (gbmc_set_majorant) when comparing with perturbed
 * runs. dL_dD is read from host or device memory (g_ptr_kind), grad/var are
 * written to out_ptr_kind memory. Synchronous: returns when the result is
 * in place. Does not touch the dose tally. */
gbmc_status gbmc_adjoint(gbmc_ctx* ctx, const double* dL_dD, int g_ptr_kind, uint64_t n_hist,
                         uint64_t seed, uint64_t first_hist, double* grad, double* var,
                         int out_ptr_kind, void* cuda_stream);

/* Message of the last failed call on ctx (C ABI plumbing; the paper has no
 * counterpart). The string is owned by the context and valid until the next
 * call on it. */
const char* gbmc_last_error(const gbmc_ctx* ctx);

/* Free the context and all its device memory (the counterpart of
 * gbmc_create; the paper's simulation objects end with the program). NULL is
 * ignored. Waits for nothing: synchronise the context's streams first. */
void gbmc_destroy(gbmc_ctx* ctx);

/* ---- helpers for tests (same library, same code paths) ------------------ */

/* Fill out[4*n] with Philox4x32-10 words for counters (c0 + i, c1, c2, c3),
 * key (k0, k1), computed by the device Philox (GPU). */
gbmc_status gbmc_philox_fill(int device, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                             uint32_t k0, uint32_t k1, uint32_t* out, int n);

/* First real interaction of each primary photon (Woodcock + type choice of
 * the device code): xyz[3n] positions, type[n] 1 Compton 2 PE 3 Rayleigh 4 pair,
 * 0 none (escaped). Runs on the context's device. */
gbmc_status gbmc_first_interactions(gbmc_ctx* ctx, uint64_t seed, uint64_t first_hist,
                                    int n, double* xyz, int* type);

/* Walker alias table of n weights (host only, no GPU): prob[n] in [0,1],
 * alias[n] in [0,n). Bin j is drawn as j = floor(u n) kept with probability
 * prob[j], else alias[j]. */
gbmc_status gbmc_build_alias(const double* weights, int n, float* prob, int* alias);

/* Evaluate the library's FP32 table interpolation on the host (no GPU):
 * quantity q (see gbmc_table_quantity), material m, at energies E[n]. */
enum {
  GBMC_Q_MU_TOTAL = 0, GBMC_Q_MU_COMPTON, GBMC_Q_MU_PE, GBMC_Q_MU_RAYLEIGH,
  GBMC_Q_SIG_EL_HARD, GBMC_Q_SIG_INEL_E, GBMC_Q_SIG_INEL_P, GBMC_Q_SIG_BREMS,
  GBMC_Q_SIG1_SOFT, GBMC_Q_XC, GBMC_Q_RANGE_E, GBMC_Q_RANGE_P,
  GBMC_Q_MAJORANT = 100, GBMC_Q_RANGE_INV_E = 101, GBMC_Q_RANGE_INV_P = 102,
  GBMC_Q_SOFT_APRIME = 103,
  GBMC_Q_SIG_HARD_E = 104, GBMC_Q_SIG_HARD_P = 105   /* hard el + inel + brems, the step majorant's table */
};
gbmc_status gbmc_table_eval(gbmc_ctx* ctx, int q, int m, const double* x, int n, double* out);

/* ---- checked build --------------------------------------------------------
 * The same sources compiled with GBMC_CHECKED defined give a second library,
 * libgbmc_checked.so, with this same ABI. Its kernels test every voxel,
 * material, batch, job, queue-slot, alias-bin, element-count and adjoint-buffer
 * index against its bound (and the DDA's running voxel index against its
 * coordinates) before the access. An index out of range sets bit
 * GBMC_FLAG_BOUNDS of gbmc_stats.error_flags, is replaced by 0 so that no
 * memory outside the buffer is touched, and makes the run's status
 * GBMC_ERR_BOUNDS. It stands in for a device memory checker. The paper's
 * counterpart is a design rule, not a tool: its threads share read-only
 * geometry (constant STEP and LOCATE) and keep private tallies, so that races
 * cannot arise (Sec. 4.3); the kernels here follow the same rule, and the
 * checked build tests the indices that rule leaves open. The checks cost time; results
 * are otherwise those of libgbmc.so (the same histories and event counts). In
 * libgbmc.so the checks compile to nothing.
 *
 * gbmc_build_checked returns 1 in the checked library, 0 in the default one.
 * gbmc_check_index runs the checked build's index test on `device` for n
 * pairs (idx[i], bound[i]) (host arrays) and returns, per pair, the index the
 * kernels would use (out[i]) and the error bits it recorded (flags[i]):
 * idx[i] and 0 when 0 <= idx[i] < bound[i] or in the default library, else 0
 * and GBMC_FLAG_BOUNDS. It reads and writes only its own small buffers
 * (allocated and freed by the call). GBMC_ERR_ARG for null arrays or n < 0. */
#define GBMC_FLAG_BOUNDS 128u
int gbmc_build_checked(void);
gbmc_status gbmc_check_index(int device, const int* idx, const int64_t* bound, int n, int* out,
                             uint32_t* flags);

/* ---- measured pipe peaks (roofline denominators) --------------------------
 * The paper has no counterpart: it reports CPU run times only. The transport
 * kernels are bound by instruction issue on the FP32/INT32 pipes and the
 * special-function unit, and their tally by float atomics resolved in L2 (no
 * dense contraction, working set on chip), so their roofline is the measured
 * throughput of those pipes. gbmc_probe_peak runs one probe kernel on `device`
 * (8 blocks of 256 threads per SM, 8 independent chains per thread, iters
 * rounds of 4 operations per chain; the atomic probe: one add to a
 * pseudo-random word of a 32 MB buffer per thread and operation), timed with
 * CUDA events after one warm-up launch, and returns the operations executed
 * (*ops, thread-level) and the time of the timed launch (*ms); the rate is
 * ops / ms. Allocates and frees a small device buffer. */
enum {
  GBMC_PROBE_FFMA = 0,       /* fma.rn.f32 */
  GBMC_PROBE_IMAD = 1,       /* mad.lo.u32 */
  GBMC_PROBE_LG2 = 2,        /* lg2.approx.ftz.f32 */
  GBMC_PROBE_EX2 = 3,        /* ex2.approx.ftz.f32 */
  GBMC_PROBE_SIN = 4,        /* sin.approx.ftz.f32 */
  GBMC_PROBE_L2_ATOMIC = 5   /* float atomicAdd without return (RED), L2-resident */
};
gbmc_status gbmc_probe_peak(int device, int kind, int iters, double* ops, double* ms);

/* ---- allocation-free run --------------------------------------------------
 * The paper has no counterpart of this entry point; it exists for callers that
 * must not allocate device memory while histories run: a program that fixes
 * its device-memory budget at start-up, or one that keeps its streams
 * overlapping (cudaMalloc and cudaFree synchronise the device). Every other
 * run path allocates its batch tiles and queues with cudaMalloc.
 *
 * Runs histories [first_hist, first_hist + n_hist) with the plain kernel on a
 * context whose materials, phantom and source are already set (those calls
 * allocate; this one does not), in n_batches batches (2..GBMC_NOALLOC_MAX_BATCHES),
 * and ADDS per voxel the batch sums S1 += sum_k B_k and S2 += sum_k B_k^2 / n_k
 * (B_k: energy deposited in batch k, MeV; n_k: its history count) into `sum`
 * and `sum2`, caller-owned device buffers of nx*ny*nz doubles (zero them before
 * the first call). Mean energy per history = S1 / N and its variance
 * (S2 - N mean^2) / (N (K - 1)) over all calls' N histories and K batches.
 * The context's own tally and statistics are not touched.
 *
 * Scratch: a file-scope device array of GBMC_NOALLOC_MAX_FLOATS floats holds
 * the FP32 batch tiles (n_batches * nx*ny*nz rounded up to 4), the batch
 * weights and the event counters. Sizes beyond it return GBMC_ERR_ARG. Every
 * GPU that loads the library holds the array until the process exits. The
 * array is cleared at the start of each call; all calls share it, so calls
 * whose work overlaps on the GPU (different streams, or different contexts on
 * the same device without ordering) race and corrupt each other's results.
 * The first call on a device looks up the array's device address with that
 * device current; make that first call before any stream capture. Later calls
 * made outside a stream capture look the address up again (a cheap query that
 * allocates nothing), so a device reset between calls is harmless; a call
 * inside a capture uses the address found by the last call outside one.
 * `sum` and `sum2` must be device memory (checked with
 * cudaPointerGetAttributes, which allocates nothing; anything else returns
 * GBMC_ERR_ARG). Asynchronous on `cuda_stream`. The device-side loop-bound
 * and stack-overflow flags of the call go to the scratch array; read them
 * with gbmc_noalloc_flags. */
#define GBMC_NOALLOC_MAX_FLOATS (1 << 22)
#define GBMC_NOALLOC_MAX_BATCHES GBMC_MAX_BATCHES
gbmc_status gbmc_run_noalloc(gbmc_ctx* ctx, uint64_t n_hist, uint64_t seed, uint64_t first_hist,
                             int n_batches, double* sum, double* sum2, void* cuda_stream);

/* Error flags (the bits of gbmc_stats.error_flags: a secondary stack that
 * overflowed, a device loop bound that was hit) of the last gbmc_run_noalloc
 * call on the context's device, copied into *flags (host memory) after
 * synchronising `cuda_stream`, the stream that call ran on. 0 means the
 * call's result is complete. Allocates nothing; GBMC_ERR_STATE if no
 * allocation-free call has run on the device. */
gbmc_status gbmc_noalloc_flags(gbmc_ctx* ctx, void* cuda_stream, uint32_t* flags);

#ifdef __cplusplus
}
#endif
#endif
