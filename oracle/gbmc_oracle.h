/*
 * gbmc_oracle.h -- FP64 CPU oracle for voxel dose Monte Carlo.
 *
 * TEST INFRASTRUCTURE ONLY. This is the plain, serial (optionally
 * thread-per-batch) reference implementation that the GPU library is checked
 * against. Only the test-suite, the smoke check and the benchmark's CPU
 * baseline may load it; the product path never does. It shares no code with
 * the CUDA library: both are written independently from the same physics
 * reading.
 *
 * Method structure follows the paper (PenRed): per history, sample the
 * primary state (Sec. 4.2.1), then loop JUMP / STEP / KNOCK over the particle
 * and its secondaries (Sec. 4.1, Fig. "flowTally"), scoring energy into a
 * voxel tally (Sec. 4.2.3) whose mean and standard deviation follow Eq. 1-2
 * (history by history) and Eq. 3 (per-thread counters summed). The paper
 * prints no interaction physics; the closed-form physics set implemented here
 * (Klein-Nishina, Z^4/E^3 photoelectric, form-factor Rayleigh, Bethe-Heitler
 * pair, Bethe stopping, Moller, Rossi-Greisen bremsstrahlung, screened
 * Rutherford elastic, class II random-hinge stepping) is the contract that
 * both engines implement.
 */
#ifndef GBMC_ORACLE_H
#define GBMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define OR_MAX_EL 8
#define OR_MAX_MAT 8

typedef struct {
  int n_el;
  int Z[OR_MAX_EL];
  double A[OR_MAX_EL];   /* g/mol */
  double w[OR_MAX_EL];   /* mass fractions */
  double I_eV;           /* mean excitation energy */
} or_material;

typedef struct {
  double eabs_g, eabs_e;  /* absorption energies, MeV */
  double wcc, wcr;        /* hard inelastic / bremsstrahlung cut-offs, MeV */
  double c1;              /* hard elastic mfp = max(lambda_el, c1 * lambda_1) */
  double step_frac;       /* max fractional CSDA loss per step */
  double step_vox;        /* max step in voxel widths */
} or_transport;

typedef struct {
  int particle;           /* 0 photon, 1 electron, 2 positron */
  int shape;              /* 0 pencil, 1 uniform rectangle on z = 0 */
  double x0, y0, hx, hy;  /* cm */
  double energy;          /* MeV, used when n_bins == 0 */
  int n_bins;
  const double* edges;    /* n_bins + 1 */
  const double* weights;  /* n_bins */
} or_source;

typedef struct {
  int nx, ny, nz;
  double dx, dy, dz;
  const uint8_t* mat;     /* [iz][iy][ix] */
  const float* rho;       /* g/cm^3 */
} or_phantom;

typedef struct {
  /* tallies, all nvox doubles, accumulated (caller zeroes them) */
  double* sum_q;    /* Eq. 1: sum over histories of q_{h,v} (MeV) */
  double* sum_q2;   /* Eq. 1: sum over histories of q_{h,v}^2 */
  double* batch_s1; /* sum over batches of B_{k,v} */
  double* batch_s2; /* sum over batches of B_{k,v}^2 / n_k */
} or_tally;

typedef struct {
  uint64_t n_hist, n_batches;
  uint64_t n_tent, n_real, n_compton, n_pe, n_rayleigh, n_pair;
  uint64_t n_e_steps, n_cross, n_hard_el, n_hard_inel, n_hard_br, n_delta;
  uint64_t n_annih, n_escape, n_particles;
  double e_src, e_dep, e_esc, max_ledger_rel;
  double e_path;           /* mass thickness travelled by e+- (g/cm^2) */
  double e_path_absorbed;  /* ... by e+- that ended below eabs_e */
  uint64_t n_e_absorbed;   /* e+- that ended below eabs_e */
  /* instrumented runs only (or_problem_set_instrument): compensators of the
   * hard-event counts, i.e. the integrals over every e+- step's travelled
   * mass thickness of the hard elastic, inelastic and bremsstrahlung cross
   * sections at the CSDA energy (forcing factors applied), and of the step
   * majorant; E[n_hard_el] = E[i_el], ..., E[n_delta] = E[i_hat - i_el -
   * i_inel - i_br]. */
  double i_el, i_inel, i_br, i_hat;
} or_stats;

/* ---- random numbers ---------------------------------------------------- */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint64_t or_mix64(uint64_t parent_path, uint64_t ordinal);
double or_uniform(uint64_t seed, uint32_t job, uint32_t hist, uint64_t path, uint32_t n);

/* ---- cross sections (mass units, cm^2/g) -------------------------------- */
double or_sigma_kn(double k);                              /* per electron, cm^2 */
double or_rayleigh_I(double b);
double or_mu_compton(const or_material* m, double E);
double or_mu_pe(const or_material* m, double E);
double or_mu_rayleigh(const or_material* m, double E);
double or_mu_pair(const or_material* m, double E);
double or_mu_total(const or_material* m, double E);
double or_electron_density(const or_material* m);          /* e/g */
double or_s_col(const or_material* m, int positron, double T);       /* MeV cm^2/g */
double or_s_restricted(const or_material* m, int positron, double T, double wcc, double wcr);
double or_sig_inel(const or_material* m, int positron, double T, double wcc); /* cm^2/g */
double or_inv_x0(const or_material* m);                     /* 1/X0, cm^2/g */
double or_sig_brems(const or_material* m, double T, double wcr);
double or_sig_el_hard(const or_material* m, double T, double c1);
double or_el_xc(const or_material* m, double T, double c1);      /* 1 - mu_c */
double or_sig1_soft(const or_material* m, double T, double c1);
double or_soft_aprime(double mbar);                         /* solves G(A') = mbar */

/* ---- ranges (need an initialised problem: material index) ------------- */
typedef struct or_problem or_problem;
or_problem* or_problem_create(const or_material* mats, int n_mat, const or_transport* tp,
                              const or_phantom* ph, const or_source* src);
void or_problem_destroy(or_problem* p);
double or_range(const or_problem* p, int mat, int positron, double T);   /* g/cm^2 */
double or_range_inv(const or_problem* p, int mat, int positron, double r);

/* ---- samplers: n independent samples, sample i uses stream (seed, 0, i, 0) */
void or_sample_compton(double k, int n, uint64_t seed, double* eps, double* cost);
void or_sample_rayleigh(const or_material* m, double E, int n, uint64_t seed, double* cost);
void or_sample_pair_split(int n, uint64_t seed, double* x);
void or_sample_moller(double T, double wcc, int n, uint64_t seed, double* W);
void or_sample_el_hard(const or_material* m, double T, double c1, int n, uint64_t seed, double* cost);
void or_sample_soft(double aprime, int n, uint64_t seed, double* cost);
void or_sample_source_energy(const or_source* s, int n, uint64_t seed, double* E);
/* Compton kinematics of the transport: scattered photon and electron directions */
void or_compton_kinematics(double E, double eps, double cost, double phi, const double u[3], double u1[3],
                           double pe[3]);
/* positrons at rest: the two annihilation photons (directions, energies) */
void or_sample_annihilation(int n, uint64_t seed, double* d1, double* d2, double* E1, double* E2);

/* ---- geometry: voxel chord lengths of a straight segment (DDA) --------- */
int or_ray_chords(const or_phantom* ph, const double x[3], const double u[3], double length,
                  int max_out, int64_t* vox, double* len);

/* ---- transport run ---------------------------------------------------- */
/* Histories [first_hist, first_hist + n_hist) split into n_batches batches
 * (batch k: [first + floor(kN/K), first + floor((k+1)N/K))); n_threads >= 1
 * workers each take whole batches (Eq. 3). Returns 0 on success. */
int or_run(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
           uint64_t n_hist, int n_batches, int n_threads, or_tally* tally, or_stats* stats);

/* Per-history trace for cross-engine checks: for each history, the position
 * (x,y,z) and type (1 Compton, 2 PE, 3 Rayleigh, 4 pair, 0 none) of the
 * primary photon's first real interaction. */
int or_first_interactions(const or_problem* p, uint64_t seed, uint32_t job,
                          uint64_t first_hist, uint64_t n_hist, double* xyz, int* type);

/* The same for the k-th (k >= 1) real interaction of the primary photon,
 * with the photon's energy just before it in E (may be NULL; 0 where the
 * photon left or was absorbed before its k-th interaction). */
int or_nth_interactions(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
                        uint64_t n_hist, int k, double* xyz, double* E, int* type);

/* Accumulate the hard-event compensators of or_stats (slow: test use). */
int or_problem_set_instrument(or_problem* p, int on);

/* Two-body kinematics of a hard inelastic collision (Moller / positron) as
 * the transport applies it: a particle of kinetic energy T along u[3] gives
 * W to an electron at rest; up = its new direction, ud = the electron's,
 * azimuths phi and phi + pi. */
void or_binary_collision(double T, double W, double phi, const double u[3], double up[3],
                         double ud[3]);

/* Per-atom screened Rutherford (Wentzel) elastic DCS dsigma/dmu, cm^2. */
double or_elastic_dcs(int Z, double T, double mu);

/* ---- fixed photon majorant and the dose gradient ----------------------- */
/* Build the photon majorant from the given per-material densities instead of
 * the phantom's maxima (each must be >= the maximum; returns 1 otherwise), so
 * that it stays fixed when densities are perturbed. */
int or_problem_set_majorant(or_problem* p, const double* rho_maj);

/* Variance reduction (Sec. 5.2 runs its 40 keV electron example with hard
 * bremsstrahlung and hard inelastic collisions forced by factors 2000 and 200
 * and bremsstrahlung photons split in two). Interaction forcing: for an
 * electron or positron whose weight lies in [w_lo, w_hi], the hard inelastic
 * and hard bremsstrahlung cross sections are multiplied by f_inel, f_brems;
 * at such an event the secondary carries the particle's weight divided by the
 * factor, and the particle itself takes the energy loss (and deflection) with
 * probability 1 / factor, drawn after the event's own samples. Splitting:
 * every bremsstrahlung photon is emitted as n_split_brems copies, each of
 * 1 / n_split_brems of its weight; copy 0 takes the stream of the parent's
 * next child, copy k >= 1 the child stream of ordinal 2^31 + k of copy 0's
 * path (the parent's child count does not see the copies). Deposits and
 * escapes are weighted. Default: factors 1, window [0, inf), no splitting.
 * Returns 0, or 1 for out-of-range values (factors >= 1, 0 <= w_lo <= w_hi,
 * 1 <= n_split_brems <= 64). or_adjoint refuses (returns 5) a problem with
 * variance reduction. */
typedef struct {
  double f_inel, f_brems;
  double w_lo, w_hi;
  int n_split_brems;
} or_vr;
int or_problem_set_vr(or_problem* p, const or_vr* vr);

/* Likelihood-ratio estimate of dL/drho per voxel given g = dL/dD (D in MeV/g
 * per history), over [first_hist, first_hist + n_hist) in n_batches batches:
 * adds the batch sums of the per-history contributions to s1 and s2
 * (s1 = sum_k B_k, s2 = sum_k B_k^2 / n_k). Only the photon Woodcock
 * acceptance and the explicit 1/rho of the dose are differentiated.
 * g == NULL gives the score alone (G_h = 1, no explicit term), whose mean is 0. */
int or_adjoint(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
               uint64_t n_hist, int n_batches, const double* g, double* s1, double* s2,
               or_stats* stats);

/* Test functionals with closed forms: per voxel, sums over histories of
 * G_h S_hv and its square for G_h = 1{the primary photon's first real
 * interaction is in voxel target} (target < 0: it leaves without one), S_hv
 * from the primary's flights up to that interaction. */
int or_lr_primary(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
                  uint64_t n_hist, int64_t target, double* s1, double* s2);

#ifdef __cplusplus
}
#endif
#endif
