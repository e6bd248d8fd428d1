/*
 * gbmc_oracle.c -- FP64 CPU oracle for voxel dose Monte Carlo.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg, never by the product path. Shares no code with
 * the CUDA library.
 *
 * Readability over speed: cross sections are evaluated from their closed forms
 * at every use (no interpolation tables), ranges are Gauss-Legendre integrals
 * of 1/S, and every sampler is the textbook algorithm it names. Function
 * comments cite the paper passage (section / equation) whose role the function
 * plays; the physics formulas themselves are not in the paper and are the
 * closed-form set listed in gbmc_oracle.h.
 *
 * Random numbers: every particle owns a Philox4x32-10 stream (Salmon et al.,
 * SC'11) with key (lo32(seed), hi32(seed) ^ job) and counter
 * (history, lo32(path), hi32(path), n / 4); draw n is word n % 4, mapped to
 * u = ((word >> 9) + 0.5) * 2^-23, which lies strictly inside (0, 1) and is
 * exactly representable in binary32. A primary has path 0; the c-th secondary
 * (c = 0, 1, ...) of a particle with path P gets path mix64(P, c + 1) where
 * mix64 is the splitmix64 finaliser of P + (c + 1) * 0x9E3779B97F4A7C15.
 * This replaces the RANECU seeds of Sec. 4.3 and makes each particle's random
 * numbers independent of the order in which particles are processed.
 */
#include "gbmc_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

/* CODATA constants */
#define MEC2 0.51099895          /* MeV */
#define RE 2.8179403262e-13      /* cm */
#define ALPHA (1.0 / 137.035999084)
#define NAVO 6.02214076e23
#define PI 3.14159265358979323846
#define K_PE 4.0e-32             /* photoelectric constant, cm^2 MeV^3 */

/* ======================================================================= */
/* Philox4x32-10 and particle streams (replaces RANECU, Sec. 4.3)          */
/* ======================================================================= */

static void philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  uint32_t n0 = hi1 ^ c[1] ^ k[0];
  uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
}

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    if (r > 0) { k[0] += 0x9E3779B9u; k[1] += 0xBB67AE85u; }
    philox_round(c, k);
  }
  memcpy(out, c, sizeof c);
}

uint64_t or_mix64(uint64_t parent_path, uint64_t ordinal) {
  uint64_t z = parent_path + ordinal * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

static double word_to_u(uint32_t w) {
  return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0);
}

typedef struct {
  uint32_t key[2];
  uint32_t hist;
  uint64_t path;
  uint32_t n;          /* next draw index */
  uint32_t nchild;     /* secondaries created so far */
  uint32_t cached_block;
  int have_cache;
  uint32_t cache[4];
} stream_t;

static void stream_init(stream_t* s, uint64_t seed, uint32_t job, uint32_t hist, uint64_t path) {
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32) ^ job;
  s->hist = hist; s->path = path; s->n = 0; s->nchild = 0; s->have_cache = 0;
}

static double draw(stream_t* s) {
  const uint32_t blk = s->n >> 2;
  if (!s->have_cache || s->cached_block != blk) {
    uint32_t ctr[4] = {s->hist, (uint32_t)s->path, (uint32_t)(s->path >> 32), blk};
    or_philox4x32_10(ctr, s->key, s->cache);
    s->cached_block = blk; s->have_cache = 1;
  }
  return word_to_u(s->cache[s->n++ & 3u]);
}

/* a child stream: path derived from the parent's path and its child count */
static void stream_child(stream_t* parent, stream_t* child) {
  child->key[0] = parent->key[0]; child->key[1] = parent->key[1];
  child->hist = parent->hist;
  child->path = or_mix64(parent->path, (uint64_t)parent->nchild + 1u);
  parent->nchild++;
  child->n = 0; child->nchild = 0; child->have_cache = 0;
}

/* the stream of copy k >= 1 of a split particle: derived from the first
 * copy's path with child ordinal 2^31 + k, an ordinal no particle reaches by
 * its own children, so the parent's child count -- and every other stream of
 * the history -- is the same as without splitting */
static void stream_split(const stream_t* first, uint32_t k, stream_t* copy) {
  copy->key[0] = first->key[0]; copy->key[1] = first->key[1];
  copy->hist = first->hist;
  copy->path = or_mix64(first->path, 0x80000000ull + k);
  copy->n = 0; copy->nchild = 0; copy->have_cache = 0;
}

double or_uniform(uint64_t seed, uint32_t job, uint32_t hist, uint64_t path, uint32_t n) {
  stream_t s; stream_init(&s, seed, job, hist, path); s.n = n;
  return draw(&s);
}

/* ======================================================================= */
/* Gauss-Legendre nodes (a library-style quadrature primitive)            */
/* ======================================================================= */

#define GL_N 32
#define GL8_N 8
static double gl_x[GL_N], gl_w[GL_N], gl8_x[GL8_N], gl8_w[GL8_N];
static pthread_once_t gl_once = PTHREAD_ONCE_INIT;

/* n-point Gauss-Legendre nodes and weights on [-1, 1] (Newton on P_n) */
static void gl_nodes(int n, double* xs, double* ws) {
  for (int i = 0; i < n; ++i) {
    double x = cos(PI * (i + 0.75) / (n + 0.5)), dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * x * p1 - (j - 1.0) * p0) / j;
        p0 = p1; p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    xs[i] = x;
    ws[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

static void gl_init(void) {
  gl_nodes(GL_N, gl_x, gl_w);
  gl_nodes(GL8_N, gl8_x, gl8_w);
}

/* ======================================================================= */
/* Materials                                                               */
/* ======================================================================= */

static double atoms_per_gram(const or_material* m, int i) { return NAVO * m->w[i] / m->A[i]; }

double or_electron_density(const or_material* m) {
  double ne = 0.0;
  for (int i = 0; i < m->n_el; ++i) ne += atoms_per_gram(m, i) * m->Z[i];
  return ne;
}

/* ======================================================================= */
/* Photon cross sections (KNOCK physics; closed forms)                    */
/* ======================================================================= */

/* Klein-Nishina total cross section per free electron, k = E / mc^2. */
double or_sigma_kn(double k) {
  const double a = 1.0 + 2.0 * k, l = log(a);
  const double t1 = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / a - l / k);
  const double t2 = l / (2.0 * k);
  const double t3 = (1.0 + 3.0 * k) / (a * a);
  return 2.0 * PI * RE * RE * (t1 + t2 - t3);
}

double or_mu_compton(const or_material* m, double E) {
  return or_electron_density(m) * or_sigma_kn(E / MEC2);
}

/* photoelectric: sigma_atom = K_pe Z^4 / E^3 */
double or_mu_pe(const or_material* m, double E) {
  double s = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double z = m->Z[i];
    s += atoms_per_gram(m, i) * K_PE * z * z * z * z;
  }
  return s / (E * E * E);
}

/* Thomas-Fermi screening momentum (units of mc) */
static double rayleigh_qz(int Z) { return ALPHA / 0.885 * cbrt((double)Z); }
static double rayleigh_b(double k, int Z) { double q = rayleigh_qz(Z); return 2.0 * k * k / (q * q); }

/* I(b) = int_0^2 (1 + (1-t)^2) / (1 + b t)^2 dt by composite Gauss-Legendre in
 * v = ln(1 + b t), where dt / (1 + b t)^2 = exp(-v) dv / b and the integrand
 * (1 + (1 - t(v))^2) exp(-v) / b is smooth on [0, ln(1 + 2b)]. */
double or_rayleigh_I(double b) {
  pthread_once(&gl_once, gl_init);
  if (b < 1e-300) return 8.0 / 3.0;
  const double V = log1p(2.0 * b);
  const int np = 1 + (int)(V / 0.25);
  const double h = V / np;
  double acc = 0.0;
  for (int j = 0; j < np; ++j) {
    for (int i = 0; i < GL8_N; ++i) {
      const double v = h * (j + 0.5 * (gl8_x[i] + 1.0));
      const double t = expm1(v) / b;
      acc += gl8_w[i] * 0.5 * h * (1.0 + (1.0 - t) * (1.0 - t)) * exp(-v);
    }
  }
  return acc / b;
}

double or_mu_rayleigh(const or_material* m, double E) {
  const double k = E / MEC2;
  double s = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double z = m->Z[i];
    s += atoms_per_gram(m, i) * PI * RE * RE * z * z * or_rayleigh_I(rayleigh_b(k, m->Z[i]));
  }
  return s;
}

/* pair (nuclear + triplet folded as Z(Z+1)), k > 2 */
double or_mu_pair(const or_material* m, double E) {
  const double k = E / MEC2;
  if (k <= 2.0) return 0.0;
  const double r = (k - 2.0) / k;
  const double f = fmax(2.0 * PI / 3.0 * r * r * r, 28.0 / 9.0 * log(2.0 * k) - 218.0 / 27.0);
  double s = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double z = m->Z[i];
    s += atoms_per_gram(m, i) * ALPHA * RE * RE * z * (z + 1.0) * f;
  }
  return s;
}

double or_mu_total(const or_material* m, double E) {
  return or_mu_compton(m, E) + or_mu_pe(m, E) + or_mu_rayleigh(m, E) + or_mu_pair(m, E);
}

/* ======================================================================= */
/* Electron / positron cross sections and stopping powers                 */
/* ======================================================================= */

static double beta2_of(double tau) { return tau * (tau + 2.0) / ((tau + 1.0) * (tau + 1.0)); }

/* Bethe collision stopping power (ICRU 37 form), no density effect. */
double or_s_col(const or_material* m, int positron, double T) {
  const double tau = T / MEC2, b2 = beta2_of(tau), ne = or_electron_density(m);
  /* I-value of the mixture: the single I of the material */
  const double Ir = m->I_eV * 1e-6 / MEC2;
  double F;
  if (!positron) {
    F = 1.0 - b2 + (tau * tau / 8.0 - (2.0 * tau + 1.0) * log(2.0)) / ((tau + 1.0) * (tau + 1.0));
  } else {
    const double y = tau + 2.0;
    F = 2.0 * log(2.0) - b2 / 12.0 * (23.0 + 14.0 / y + 10.0 / (y * y) + 4.0 / (y * y * y));
  }
  const double L = log(tau * tau * (tau + 2.0) / (2.0 * Ir * Ir));
  return 2.0 * PI * RE * RE * MEC2 * ne / b2 * (L + F);
}

/* Moller: energy-loss integral and number of hard collisions above wcc.
 * DCS per electron: dsigma/dW = K/T^2 f(eps), eps = W/T,
 * f = 1/eps^2 + 1/(1-eps)^2 + a - b/(eps(1-eps)), K = 2 pi re^2 mc^2 / beta^2. */
static void moller_parts(double T, double wcc, double* n_hard, double* w_hard) {
  *n_hard = 0.0; *w_hard = 0.0;
  if (T <= 2.0 * wcc) return;
  const double tau = T / MEC2, b2 = beta2_of(tau);
  const double K = 2.0 * PI * RE * RE * MEC2 / b2;
  const double a = (tau / (tau + 1.0)) * (tau / (tau + 1.0));
  const double b = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
  const double ec = wcc / T;
  /* number: int_ec^1/2 f deps */
  const double nn = (1.0 / ec - 2.0) + (2.0 - 1.0 / (1.0 - ec)) + a * (0.5 - ec)
                    - b * log((1.0 - ec) / ec);
  /* loss: int_ec^1/2 eps f deps, antiderivative
   * H = ln eps + 1/(1-eps) + ln(1-eps) + a eps^2/2 + b ln(1-eps) */
#define H_(e) (log(e) + 1.0 / (1.0 - (e)) + log(1.0 - (e)) + a * (e) * (e) / 2.0 + b * log(1.0 - (e)))
  const double ww = H_(0.5) - H_(ec);
#undef H_
  *n_hard = K / T * nn;
  *w_hard = K * ww;
}

/* positron hard inelastic: free 1/W^2 DCS on [wcc, T] (a reading: the paper gives no
 * positron collision law, and Bhabha structure is not part of this physics set) */
static void bhabha_parts(double T, double wcc, double* n_hard, double* w_hard) {
  *n_hard = 0.0; *w_hard = 0.0;
  if (T <= wcc) return;
  const double tau = T / MEC2, b2 = beta2_of(tau);
  const double K = 2.0 * PI * RE * RE * MEC2 / b2;
  *n_hard = K * (1.0 / wcc - 1.0 / T);
  *w_hard = K * log(T / wcc);
}

double or_sig_inel(const or_material* m, int positron, double T, double wcc) {
  double n, w;
  if (positron) bhabha_parts(T, wcc, &n, &w); else moller_parts(T, wcc, &n, &w);
  return or_electron_density(m) * n;
}

/* Rossi-Greisen radiation length: 1/X0 = 4 alpha re^2 sum_i (NA w_i/A_i) Z(Z+1) ln(183 Z^-1/3) */
double or_inv_x0(const or_material* m) {
  double s = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double z = m->Z[i];
    s += atoms_per_gram(m, i) * z * (z + 1.0) * log(183.0 / cbrt(z));
  }
  return 4.0 * ALPHA * RE * RE * s;
}

/* hard bremsstrahlung, N dsigma/dW = 1/(X0 W) on (0, T] */
double or_sig_brems(const or_material* m, double T, double wcr) {
  if (T <= wcr) return 0.0;
  return or_inv_x0(m) * log(T / wcr);
}

double or_s_restricted(const or_material* m, int positron, double T, double wcc, double wcr) {
  double n, w;
  if (positron) bhabha_parts(T, wcc, &n, &w); else moller_parts(T, wcc, &n, &w);
  const double scol = or_s_col(m, positron, T) - or_electron_density(m) * w;
  const double srad = or_inv_x0(m) * fmin(T, wcr);
  return scol + srad;
}

/* screened Rutherford (Wentzel) per atom: dsigma/dmu = 2 pi C / (1 - mu + 2A)^2 */
static void wentzel_params(int Z, double T, double* C, double* A) {
  const double tau = T / MEC2, b2 = beta2_of(tau), p2 = tau * (tau + 2.0);
  const double f = (tau + 1.0) / p2;
  const double z = Z;
  *C = z * (z + 1.0) * RE * RE * f * f;
  const double s = ALPHA * cbrt(z) / (0.885 * sqrt(p2));
  *A = 0.25 * s * s * (1.13 + 3.76 * (ALPHA * z) * (ALPHA * z) / b2);
}

/* total elastic and first transport cross sections (mass units) */
static void elastic_totals(const or_material* m, double T, double* sel, double* s1) {
  *sel = 0.0; *s1 = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double C, A; wentzel_params(m->Z[i], T, &C, &A);
    const double n = atoms_per_gram(m, i);
    *sel += n * PI * C / (A * (1.0 + A));
    *s1 += n * 2.0 * PI * C * (log1p(1.0 / A) - 1.0 / (1.0 + A));
  }
}

/* hard elastic cross section above deflection x = 1 - mu >= xc */
static double el_hard_above(const or_material* m, double T, double xc) {
  double s = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double C, A; wentzel_params(m->Z[i], T, &C, &A);
    s += atoms_per_gram(m, i) * 2.0 * PI * C * (2.0 - xc) / ((xc + 2.0 * A) * (2.0 + 2.0 * A));
  }
  return s;
}

/* hard elastic cross section: the mean free path between hard events is
 * max(lambda_el, C1 lambda_1), i.e. sigma_h = min(sigma_el, sigma_1 / C1) */
double or_sig_el_hard(const or_material* m, double T, double c1) {
  double sel, s1; elastic_totals(m, T, &sel, &s1);
  return fmin(sel, s1 / c1);
}

/* cut-off deflection xc = 1 - mu_c at which the hard cross section equals
 * or_sig_el_hard (bisection; 0 when every elastic event is hard) */
double or_el_xc(const or_material* m, double T, double c1) {
  double sel, s1; elastic_totals(m, T, &sel, &s1);
  if (sel <= s1 / c1) return 0.0;
  const double target = s1 / c1;
  double lo = 0.0, hi = 2.0;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (el_hard_above(m, T, mid) > target) lo = mid; else hi = mid;
    if (hi - lo <= 1e-15 * hi) break;
  }
  return 0.5 * (lo + hi);
}

/* soft first transport cross section: int over 0 <= 1 - mu < xc of (1 - mu) dsigma */
double or_sig1_soft(const or_material* m, double T, double c1) {
  const double xc = or_el_xc(m, T, c1);
  if (xc <= 0.0) return 0.0;
  double s = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double C, A; wentzel_params(m->Z[i], T, &C, &A);
    s += atoms_per_gram(m, i) * 2.0 * PI * C * (log1p(xc / (2.0 * A)) - xc / (xc + 2.0 * A));
  }
  return s;
}

/* G(A) = 2A[(1+A) ln(1+1/A) - 1] = 1 - <mu> of the Wentzel law on [-1, 1] */
static double soft_G(double A) {
  if (A < 1e3) return 2.0 * A * ((1.0 + A) * log1p(1.0 / A) - 1.0);
  /* large A: G = 2 sum_{n>=1} (-1)^(n+1) y^(n-1) / (n (n+1)), y = 1/A */
  const double y = 1.0 / A;
  double g = 0.0, yp = 1.0;
  for (int n = 1; n <= 8; ++n) {
    g += ((n & 1) ? 1.0 : -1.0) * yp / (n * (n + 1.0));
    yp *= y;
  }
  return 2.0 * g;
}

double or_soft_aprime(double mbar) {
  /* bisection in ln A, then Newton polish */
  double lo = -80.0, hi = 40.0;
  for (int it = 0; it < 200; ++it) {
    double mid = 0.5 * (lo + hi);
    if (soft_G(exp(mid)) < mbar) lo = mid; else hi = mid;
    if (hi - lo < 1e-13) break;
  }
  double A = exp(0.5 * (lo + hi));
  for (int it = 0; it < 3; ++it) {
    double L = log1p(1.0 / A);
    double d = 2.0 * ((1.0 + 2.0 * A) * L - 2.0);
    if (d <= 0.0) break;
    double An = A - (soft_G(A) - mbar) / d;
    if (!(An > 0.0)) break;
    A = An;
  }
  return A;
}

/* ======================================================================= */
/* Problem: materials, phantom, source, range integrals                   */
/* ======================================================================= */

#define RG_N 2048
#define RG_EMIN 1e-3
#define RG_EMAX 100.0

struct or_problem {
  int n_mat;
  or_material mats[OR_MAX_MAT];
  or_transport tp;
  or_phantom ph;
  or_source src;
  double* src_cdf;                   /* spectrum cumulative weights */
  double rho_max[OR_MAX_MAT];        /* largest density of each material */
  double ne[OR_MAX_MAT], inv_x0[OR_MAX_MAT];
  double rg_lnE[RG_N];
  double rg_R[OR_MAX_MAT][2][RG_N];  /* cumulative range at grid nodes */
  double dmin;
  or_vr vr;                          /* variance reduction (off: factors 1) */
  int instrument;                    /* accumulate the hard-event compensators (pins) */
};

/* restricted stopping power with the material constants (electron density,
 * 1/X0) taken from the problem instead of recomputed */
static double s_r(const or_problem* p, int m, int pos, double T) {
  const or_material* mat = &p->mats[m];
  const double tau = T / MEC2, b2 = beta2_of(tau), ne = p->ne[m];
  const double Ir = mat->I_eV * 1e-6 / MEC2;
  double F;
  if (!pos) {
    F = 1.0 - b2 + (tau * tau / 8.0 - (2.0 * tau + 1.0) * log(2.0)) / ((tau + 1.0) * (tau + 1.0));
  } else {
    const double y = tau + 2.0;
    F = 2.0 * log(2.0) - b2 / 12.0 * (23.0 + 14.0 / y + 10.0 / (y * y) + 4.0 / (y * y * y));
  }
  const double L = log(tau * tau * (tau + 2.0) / (2.0 * Ir * Ir));
  double n, w;
  if (pos) bhabha_parts(T, p->tp.wcc, &n, &w); else moller_parts(T, p->tp.wcc, &n, &w);
  return 2.0 * PI * RE * RE * MEC2 * ne / b2 * (L + F) - ne * w + p->inv_x0[m] * fmin(T, p->tp.wcr);
}

/* int_{Ea}^{Eb} dT / S_r(T), Gauss-Legendre in ln T */
static double range_piece(const or_problem* p, int m, int pos, double Ea, double Eb) {
  const double la = log(Ea), lb = log(Eb), h = 0.5 * (lb - la), c = 0.5 * (lb + la);
  double acc = 0.0;
  for (int i = 0; i < GL8_N; ++i) {
    double T = exp(c + h * gl8_x[i]);
    acc += gl8_w[i] * T / s_r(p, m, pos, T);
  }
  return h * acc;
}

double or_range(const or_problem* p, int m, int pos, double T) {
  if (T <= RG_EMIN) return 0.0;
  double x = (log(T) - p->rg_lnE[0]) / (p->rg_lnE[1] - p->rg_lnE[0]);
  int i = (int)floor(x);
  if (i >= RG_N - 1) i = RG_N - 2;
  if (i < 0) i = 0;
  const double Ei = exp(p->rg_lnE[i]);
  return p->rg_R[m][pos][i] + range_piece(p, m, pos, Ei, T);
}

double or_range_inv(const or_problem* p, int m, int pos, double r) {
  if (r <= 0.0) return RG_EMIN;
  const double* R = p->rg_R[m][pos];
  int lo = 0, hi = RG_N - 1;
  if (r >= R[hi]) return exp(p->rg_lnE[hi]);
  while (hi - lo > 1) { int mid = (lo + hi) / 2; if (R[mid] <= r) lo = mid; else hi = mid; }
  const double Enode = exp(p->rg_lnE[lo]);
  double a = Enode, b = exp(p->rg_lnE[hi]);
  double T = a + (b - a) * (r - R[lo]) / (R[hi] - R[lo]);
  for (int it = 0; it < 60; ++it) {
    double f = R[lo] + range_piece(p, m, pos, Enode, T) - r;
    if (f > 0.0) b = T; else a = T;
    double Tn = T - f * s_r(p, m, pos, T);
    if (!(Tn > a && Tn < b)) Tn = 0.5 * (a + b);
    if (fabs(Tn - T) <= 1e-14 * T) { T = Tn; break; }
    T = Tn;
  }
  return T;
}

or_problem* or_problem_create(const or_material* mats, int n_mat, const or_transport* tp,
                              const or_phantom* ph, const or_source* src) {
  pthread_once(&gl_once, gl_init);
  if (n_mat < 1 || n_mat > OR_MAX_MAT) return NULL;
  or_problem* p = (or_problem*)calloc(1, sizeof(or_problem));
  p->n_mat = n_mat;
  memcpy(p->mats, mats, sizeof(or_material) * n_mat);
  p->tp = *tp;
  p->vr.f_inel = p->vr.f_brems = 1.0;
  p->vr.w_lo = 0.0; p->vr.w_hi = INFINITY;
  p->vr.n_split_brems = 1;
  if (ph) p->ph = *ph;
  if (src) {
    p->src = *src;
    if (src->n_bins > 0) {
      p->src_cdf = (double*)malloc(sizeof(double) * (src->n_bins + 1));
      p->src_cdf[0] = 0.0;
      for (int i = 0; i < src->n_bins; ++i) p->src_cdf[i + 1] = p->src_cdf[i] + src->weights[i];
    }
  }
  for (int m = 0; m < n_mat; ++m) {
    p->rho_max[m] = 0.0;
    p->ne[m] = or_electron_density(&p->mats[m]);
    p->inv_x0[m] = or_inv_x0(&p->mats[m]);
  }
  if (ph && ph->mat) {
    const int64_t nv = (int64_t)ph->nx * ph->ny * ph->nz;
    for (int64_t v = 0; v < nv; ++v) {
      int m = ph->mat[v];
      if (m < n_mat && ph->rho[v] > p->rho_max[m]) p->rho_max[m] = ph->rho[v];
    }
    p->dmin = fmin(ph->dx, fmin(ph->dy, ph->dz));
  }
  for (int i = 0; i < RG_N; ++i)
    p->rg_lnE[i] = log(RG_EMIN) + (log(RG_EMAX) - log(RG_EMIN)) * i / (RG_N - 1);
  for (int m = 0; m < n_mat; ++m)
    for (int pos = 0; pos < 2; ++pos) {
      p->rg_R[m][pos][0] = 0.0;
      for (int i = 1; i < RG_N; ++i)
        p->rg_R[m][pos][i] = p->rg_R[m][pos][i - 1] +
            range_piece(p, m, pos, exp(p->rg_lnE[i - 1]), exp(p->rg_lnE[i]));
    }
  return p;
}

void or_problem_destroy(or_problem* p) {
  if (!p) return;
  free(p->src_cdf);
  free(p);
}

/* ======================================================================= */
/* Geometry: LOCATE and voxel-boundary stepping (Sec. 4.2.2)              */
/* ======================================================================= */

/* index along one axis; a point on a plane belongs to the voxel the direction
 * enters, floor when the direction component is zero; -1/-2 outside */
static int locate_axis(double x, double u, double d, int n) {
  double f = x / d;
  double fl = floor(f);
  int i = (int)fl;
  if (f == fl && u < 0.0) i -= 1;
  if (f < 0.0 || i < 0 || i >= n) return -1;
  return i;
}

static int64_t locate(const or_phantom* ph, const double x[3], const double u[3]) {
  int ix = locate_axis(x[0], u[0], ph->dx, ph->nx);
  int iy = locate_axis(x[1], u[1], ph->dy, ph->ny);
  int iz = locate_axis(x[2], u[2], ph->dz, ph->nz);
  if (ix < 0 || iy < 0 || iz < 0) return -1;
  return ((int64_t)iz * ph->ny + iy) * ph->nx + ix;
}

static void vox_ijk(const or_phantom* ph, int64_t v, int ijk[3]) {
  ijk[0] = (int)(v % ph->nx);
  ijk[1] = (int)((v / ph->nx) % ph->ny);
  ijk[2] = (int)(v / ((int64_t)ph->nx * ph->ny));
}

/* distance to the exit face of voxel ijk along u; axis of that face */
static double face_distance(const or_phantom* ph, const int ijk[3], const double x[3],
                            const double u[3], int* axis, double* face) {
  const double d3[3] = {ph->dx, ph->dy, ph->dz};
  double best = INFINITY; *axis = -1; *face = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (u[a] == 0.0) continue;
    double f = (u[a] > 0.0) ? (ijk[a] + 1) * d3[a] : ijk[a] * d3[a];
    double t = (f - x[a]) / u[a];
    if (t < 0.0) t = 0.0;
    if (t < best) { best = t; *axis = a; *face = f; }
  }
  return best;
}

int or_ray_chords(const or_phantom* ph, const double x0[3], const double u[3], double length,
                  int max_out, int64_t* vox, double* len) {
  double x[3] = {x0[0], x0[1], x0[2]};
  int64_t v = locate(ph, x, u);
  int n = 0;
  double left = length;
  while (v >= 0 && left > 0.0 && n < max_out) {
    int ijk[3]; vox_ijk(ph, v, ijk);
    int axis; double face;
    double d = face_distance(ph, ijk, x, u, &axis, &face);
    if (d >= left) { vox[n] = v; len[n] = left; ++n; break; }
    vox[n] = v; len[n] = d; ++n;
    for (int a = 0; a < 3; ++a) x[a] += d * u[a];
    x[axis] = face;
    left -= d;
    ijk[axis] += (u[axis] > 0.0) ? 1 : -1;
    const int nn[3] = {ph->nx, ph->ny, ph->nz};
    if (ijk[axis] < 0 || ijk[axis] >= nn[axis]) break;
    v = ((int64_t)ijk[2] * ph->ny + ijk[1]) * ph->nx + ijk[0];
  }
  return n;
}

/* ======================================================================= */
/* Direction rotation                                                     */
/* ======================================================================= */

static void rotate(double u[3], double cost, double phi) {
  if (cost > 1.0) cost = 1.0;
  if (cost < -1.0) cost = -1.0;
  const double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
  const double cp = cos(phi), sp = sin(phi);
  const double ux = u[0], uy = u[1], uz = u[2];
  const double s2 = ux * ux + uy * uy;
  if (s2 > 1e-20) {
    const double s = sqrt(s2);
    u[0] = ux * cost + sint * (ux * uz * cp - uy * sp) / s;
    u[1] = uy * cost + sint * (uy * uz * cp + ux * sp) / s;
    u[2] = uz * cost - sint * cp * s;
  } else {
    u[0] = sint * cp;
    u[1] = sint * sp;
    u[2] = (uz >= 0.0 ? 1.0 : -1.0) * cost;
  }
  const double nrm = 1.0 / sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  u[0] *= nrm; u[1] *= nrm; u[2] *= nrm;
}

/* ======================================================================= */
/* Samplers (the KNOCK routines of Sec. 4.1)                              */
/* ======================================================================= */

/* Klein-Nishina by Butcher & Messel (1960) decomposition; returns eps = E'/E */
/* Compton kinematics: the photon of energy E along u leaves with eps E at
 * polar cosine cost and azimuth phi (u is turned in place); the electron,
 * with the energy E - eps E, moves along the momentum the photon lost,
 * E u_before - eps E u_after (momentum conservation, units of 1/c) */
static void compton_kinematics(double E, double eps, double cost, double phi, double u[3], double pe[3]) {
  const double E1 = eps * E;
  double u0[3] = {u[0], u[1], u[2]};
  rotate(u, cost, phi);
  double pn = 0.0;
  for (int a = 0; a < 3; ++a) { pe[a] = E * u0[a] - E1 * u[a]; pn += pe[a] * pe[a]; }
  pn = sqrt(pn);
  if (pn > 0.0) for (int a = 0; a < 3; ++a) pe[a] /= pn;
  else memcpy(pe, u0, 3 * sizeof(double));
}

/* test hook: compton_kinematics on a copy of u (u1 = the scattered photon's
 * direction, pe = the electron's) */
void or_compton_kinematics(double E, double eps, double cost, double phi, const double u[3], double u1[3],
                           double pe[3]) {
  memcpy(u1, u, 3 * sizeof(double));
  compton_kinematics(E, eps, cost, phi, u1, pe);
}

static double sample_compton(stream_t* s, double k, double* cost) {
  const double e0 = 1.0 / (1.0 + 2.0 * k);
  const double a1 = log(1.0 + 2.0 * k), a2 = 0.5 * (1.0 - e0 * e0);
  for (;;) {
    const double u1 = draw(s), u2 = draw(s), u3 = draw(s);
    double eps;
    if (u1 * (a1 + a2) < a1) eps = exp(-a1 * u2);
    else eps = sqrt(e0 * e0 + (1.0 - e0 * e0) * u2);
    const double t = (1.0 - eps) / (k * eps);
    const double sin2 = t * (2.0 - t);
    const double g = 1.0 - eps * sin2 / (1.0 + eps * eps);
    if (u3 <= g) { *cost = 1.0 - t; return eps; }
  }
}

/* Rayleigh: composition over elements of the envelopes 1/(1+b t)^2, each with
 * weight n_i Z_i^2 * 2/(1+2b_i), then rejection with (1 + cos^2)/2. */
static double sample_rayleigh(stream_t* s, const or_material* m, double E) {
  const double k = E / MEC2;
  double wsum = 0.0, w[OR_MAX_EL], b[OR_MAX_EL];
  for (int i = 0; i < m->n_el; ++i) {
    b[i] = rayleigh_b(k, m->Z[i]);
    double z = m->Z[i];
    w[i] = atoms_per_gram(m, i) * z * z * 2.0 / (1.0 + 2.0 * b[i]);
    wsum += w[i];
  }
  for (;;) {
    const double u1 = draw(s), u2 = draw(s), u3 = draw(s);
    double c = u1 * wsum; int i = 0;
    while (i < m->n_el - 1 && c >= w[i]) { c -= w[i]; ++i; }
    const double t = 2.0 * u2 / (1.0 + 2.0 * b[i] * (1.0 - u2));
    if (u3 <= 0.5 * (1.0 + (1.0 - t) * (1.0 - t))) return 1.0 - t;
  }
}

/* pair split x = T-/(E - 2mc^2) with p(x) ~ x^2 + (1-x)^2 + (2/3)x(1-x):
 * inverse of F(x) = (9x - 6x^2 + 4x^3)/7 by safeguarded Newton in FP64 */
static double pair_split_from_u(double u) {
  double lo = 0.0, hi = 1.0, x = u;
  for (int it = 0; it < 100; ++it) {
    double f = (9.0 * x - 6.0 * x * x + 4.0 * x * x * x) / 7.0 - u;
    if (f > 0.0) hi = x; else lo = x;
    double d = (9.0 - 12.0 * x + 12.0 * x * x) / 7.0;
    double xn = x - f / d;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    if (fabs(xn - x) < 1e-16) { x = xn; break; }
    x = xn;
  }
  return x;
}

/* Moller: eps from the 1/eps^2 envelope on [wcc/T, 1/2], rejection */
static double sample_moller(stream_t* s, double T, double wcc) {
  const double tau = T / MEC2;
  const double a = (tau / (tau + 1.0)) * (tau / (tau + 1.0));
  const double b = (2.0 * tau + 1.0) / ((tau + 1.0) * (tau + 1.0));
  const double ec = wcc / T, gmax = 2.0 + 0.25 * a;
  for (;;) {
    const double u1 = draw(s), u2 = draw(s);
    const double eps = ec / (1.0 - u1 * (1.0 - 2.0 * ec));
    const double r = eps / (1.0 - eps);
    const double g = 1.0 + r * r + a * eps * eps - b * r;
    if (u2 * gmax <= g) return eps * T;
  }
}

static double sample_bhabha(stream_t* s, double T, double wcc) {
  const double u = draw(s);
  return wcc / (1.0 - u * (1.0 - wcc / T));
}

/* hard elastic: element by partial cross section, then exact inversion */
static double sample_el_hard_u(const or_material* m, double T, double c1, double u1, double u2) {
  const double xc = or_el_xc(m, T, c1);
  double w[OR_MAX_EL], Av[OR_MAX_EL], wsum = 0.0;
  for (int i = 0; i < m->n_el; ++i) {
    double C, A; wentzel_params(m->Z[i], T, &C, &A);
    Av[i] = A;
    w[i] = atoms_per_gram(m, i) * C * (1.0 / (xc + 2.0 * A) - 1.0 / (2.0 + 2.0 * A));
    wsum += w[i];
  }
  double c = u1 * wsum; int i = 0;
  while (i < m->n_el - 1 && c >= w[i]) { c -= w[i]; ++i; }
  const double A = Av[i];
  const double D = 1.0 / (xc + 2.0 * A) - 1.0 / (2.0 + 2.0 * A);
  const double x = 1.0 / (1.0 / (xc + 2.0 * A) - u2 * D) - 2.0 * A;
  return 1.0 - x;
}

static double sample_el_hard(stream_t* s, const or_material* m, double T, double c1) {
  const double u1 = draw(s), u2 = draw(s);
  return sample_el_hard_u(m, T, c1, u1, u2);
}

/* soft deflection: Wentzel-shaped law with parameter A' on [-1, 1] */
static double soft_mu(double aprime, double u) {
  return 1.0 - 2.0 * aprime * u / (1.0 + aprime - u);
}

#define SOFT_MMIN 1e-9
#define SOFT_MMAX 0.9999

static double sample_soft_u(double mbar, double u) {
  if (mbar < SOFT_MMIN) return 1.0;
  if (mbar > SOFT_MMAX) return 2.0 * u - 1.0;
  return soft_mu(or_soft_aprime(mbar), u);
}

/* ---- sampler entry points for distribution tests ---- */
/* The draws of one class II step come from two whole blocks of the particle's
 * stream, in fixed slots: the step starts at the next block boundary (draw
 * index rounded up to a multiple of 4); block b holds the hard distance, the
 * hinge position, the soft deflection and its azimuth, block b+1 the event
 * type, the element, the hard elastic angle and its azimuth. Words a step
 * does not use are skipped; the stream continues after the two blocks. */
static void take_blocks(stream_t* s, uint32_t nblk, double* u) {
  const uint32_t b = (s->n + 3u) >> 2;
  for (uint32_t k = 0; k < nblk; ++k) {
    uint32_t ctr[4] = {s->hist, (uint32_t)s->path, (uint32_t)(s->path >> 32), b + k};
    uint32_t o[4];
    or_philox4x32_10(ctr, s->key, o);
    for (int j = 0; j < 4; ++j) u[4 * k + j] = word_to_u(o[j]);
  }
  s->n = (b + nblk) << 2;
}

static void step_words(stream_t* s, double u[8]) { take_blocks(s, 2, u); }

/* A photon flight (Woodcock step) takes one whole block the same way: the
 * flight distance, the real/virtual test, the interaction type, and the
 * azimuth of a Compton or Rayleigh event (or the pair energy split). The
 * rejection samplers continue from the stream after it. */
static void flight_words(stream_t* s, double u[4]) { take_blocks(s, 1, u); }

void or_sample_compton(double k, int n, uint64_t seed, double* eps, double* cost) {
  for (int i = 0; i < n; ++i) {
    stream_t s; stream_init(&s, seed, 0, (uint32_t)i, 0);
    double c; double e = sample_compton(&s, k, &c);
    if (eps) eps[i] = e;
    if (cost) cost[i] = c;
  }
}
void or_sample_rayleigh(const or_material* m, double E, int n, uint64_t seed, double* cost) {
  for (int i = 0; i < n; ++i) {
    stream_t s; stream_init(&s, seed, 0, (uint32_t)i, 0);
    cost[i] = sample_rayleigh(&s, m, E);
  }
}
void or_sample_pair_split(int n, uint64_t seed, double* x) {
  for (int i = 0; i < n; ++i) {
    stream_t s; stream_init(&s, seed, 0, (uint32_t)i, 0);
    x[i] = pair_split_from_u(draw(&s));
  }
}
void or_sample_moller(double T, double wcc, int n, uint64_t seed, double* W) {
  for (int i = 0; i < n; ++i) {
    stream_t s; stream_init(&s, seed, 0, (uint32_t)i, 0);
    W[i] = sample_moller(&s, T, wcc);
  }
}
void or_sample_el_hard(const or_material* m, double T, double c1, int n, uint64_t seed, double* cost) {
  for (int i = 0; i < n; ++i) {
    stream_t s; stream_init(&s, seed, 0, (uint32_t)i, 0);
    cost[i] = sample_el_hard(&s, m, T, c1);
  }
}
void or_sample_soft(double aprime, int n, uint64_t seed, double* cost) {
  for (int i = 0; i < n; ++i) {
    stream_t s; stream_init(&s, seed, 0, (uint32_t)i, 0);
    cost[i] = soft_mu(aprime, draw(&s));
  }
}

/* primary energy: inverse CDF over the bins, uniform within the bin */
static double source_energy(const or_problem* p, stream_t* s) {
  const or_source* src = &p->src;
  if (src->n_bins <= 0) return src->energy;
  const double u = draw(s), v = draw(s);
  const double c = u * p->src_cdf[src->n_bins];
  int i = 0;
  while (i < src->n_bins - 1 && p->src_cdf[i + 1] <= c) ++i;
  return src->edges[i] + (src->edges[i + 1] - src->edges[i]) * v;
}

void or_sample_source_energy(const or_source* src, int n, uint64_t seed, double* E) {
  or_material dummy; memset(&dummy, 0, sizeof dummy);
  dummy.n_el = 1; dummy.Z[0] = 1; dummy.A[0] = 1.0; dummy.w[0] = 1.0; dummy.I_eV = 10.0;
  or_transport tp; memset(&tp, 0, sizeof tp); tp.wcc = tp.wcr = 0.01;
  or_problem* p = or_problem_create(&dummy, 1, &tp, NULL, src);
  for (int i = 0; i < n; ++i) {
    stream_t s; stream_init(&s, seed, 0, (uint32_t)i, 0);
    E[i] = source_energy(p, &s);
  }
  or_problem_destroy(p);
}

/* ======================================================================= */
/* Transport (the history loop of Fig. "flowTally")                       */
/* ======================================================================= */

enum { PT_PHOTON = 0, PT_ELECTRON = 1, PT_POSITRON = 2 };

typedef struct {
  int type;
  double x[3], u[3], E;
  double wt;               /* statistical weight (1 without variance reduction) */
  stream_t rs;
} particle;

typedef struct {
  const or_problem* p;
  uint64_t seed; uint32_t job;
  /* per-history scratch tally */
  double* hq; int64_t* touched; int64_t n_touched;
  /* stack of secondaries (Sec. 5: independent stacks -> here one LIFO) */
  particle* stack; int n_stack, cap_stack;
  /* ledger (weighted: deposits, escapes, pair productions, annihilations) */
  double dep, esc, w_pair, w_annih;
  or_stats st;
  /* interaction trace: the tr_k-th real interaction of the primary photon */
  int trace; double tr_xyz[3]; int tr_type; int tr_k, tr_count; double tr_E;
  /* adjoint: the history's tentative photon collisions (voxel, score term) */
  int adj; int64_t* col_v; double* col_s; int64_t n_col, cap_col;
} worker;

/* the likelihood-ratio score term of one tentative photon collision in voxel v
 * (density rho, material attenuation kappa, majorant mbar): the collision is
 * real with probability rho kappa / mbar, so d/drho of the log probability of
 * what happened is 1/rho if it was real and -kappa/(mbar - rho kappa) if it
 * was virtual */
static void record_collision(worker* w, int64_t v, int real, double rho, double kappa, double mbar) {
  if (w->n_col == w->cap_col) {
    w->cap_col = w->cap_col ? 2 * w->cap_col : 256;
    w->col_v = (int64_t*)realloc(w->col_v, sizeof(int64_t) * w->cap_col);
    w->col_s = (double*)realloc(w->col_s, sizeof(double) * w->cap_col);
  }
  w->col_v[w->n_col] = v;
  w->col_s[w->n_col] = real ? 1.0 / rho : -kappa / (mbar - rho * kappa);
  w->n_col++;
}

static void deposit(worker* w, int64_t v, double e) {
  if (v < 0 || e == 0.0) return;
  if (w->hq[v] == 0.0) w->touched[w->n_touched++] = v;
  w->hq[v] += e;
  w->dep += e;
  /* a voxel whose running sum returns to exactly 0 would be listed twice;
   * deposits are positive so it cannot */
}

static void push(worker* w, const particle* q) {
  if (w->n_stack == w->cap_stack) {
    w->cap_stack = w->cap_stack ? 2 * w->cap_stack : 64;
    w->stack = (particle*)realloc(w->stack, sizeof(particle) * w->cap_stack);
  }
  w->stack[w->n_stack++] = *q;
}

/* create a secondary of `parent` at the parent's position, with its weight */
static void make_child(particle* parent, particle* c, int type, double E, const double u[3]) {
  c->type = type; c->E = E; c->wt = parent->wt;
  memcpy(c->x, parent->x, sizeof c->x);
  memcpy(c->u, u, sizeof c->u);
  stream_child(&parent->rs, &c->rs);
}

/* positron at rest: two back-to-back photons, isotropic */
static void annihilate(worker* w, particle* e) {
  const double cost = 2.0 * draw(&e->rs) - 1.0;
  const double phi = 2.0 * PI * draw(&e->rs);
  const double sint = sqrt(fmax(0.0, 1.0 - cost * cost));
  double d1[3] = {sint * cos(phi), sint * sin(phi), cost};
  double d2[3] = {-d1[0], -d1[1], -d1[2]};
  particle g1, g2;
  make_child(e, &g1, PT_PHOTON, MEC2, d1);
  make_child(e, &g2, PT_PHOTON, MEC2, d2);
  push(w, &g1); push(w, &g2);
  w->w_annih += e->wt; w->st.n_annih++;
}

/* test hook: the two photons of n positrons annihilating at rest at the
 * origin, positron i on the primary stream of history i under `seed`: unit
 * directions d1[3n], d2[3n] and energies E1[n], E2[n] (MeV), as annihilate()
 * pushes them */
void or_sample_annihilation(int n, uint64_t seed, double* d1, double* d2, double* E1, double* E2) {
  worker w;
  memset(&w, 0, sizeof w);
  for (int i = 0; i < n; ++i) {
    particle e;
    memset(&e, 0, sizeof e);
    e.type = PT_POSITRON;
    e.wt = 1.0;
    stream_init(&e.rs, seed, 0, (uint32_t)i, 0);
    w.n_stack = 0;
    annihilate(&w, &e);
    memcpy(d1 + 3 * (size_t)i, w.stack[0].u, sizeof w.stack[0].u);
    memcpy(d2 + 3 * (size_t)i, w.stack[1].u, sizeof w.stack[1].u);
    E1[i] = w.stack[0].E;
    E2[i] = w.stack[1].E;
  }
  free(w.stack);
}

/* charged particle of weight wt created at an interaction in voxel v:
 * absorbed at once below eabs_e (and a positron then annihilates), else
 * queued */
static void emit_charged(worker* w, particle* parent, int type, double T, const double u[3], int64_t v,
                         double wt) {
  particle c;
  make_child(parent, &c, type, T, u);
  c.wt = wt;
  if (T < w->p->tp.eabs_e) {
    deposit(w, v, T * wt);
    if (type == PT_POSITRON) annihilate(w, &c);
  } else {
    push(w, &c);
  }
}

/* photon of total weight wt created at an interaction in voxel v, as n_split
 * copies of weight wt / n_split (copy 0 is the parent's next child, copies
 * k >= 1 take split streams of copy 0): deposited at once below eabs_g, else
 * queued */
static void emit_photon(worker* w, particle* parent, double E, const double u[3], int64_t v, double wt,
                        int n_split) {
  particle c;
  make_child(parent, &c, PT_PHOTON, E, u);
  c.wt = wt / n_split;
  for (int k = 0; k < n_split; ++k) {
    particle ck = c;
    if (k > 0) stream_split(&c.rs, (uint32_t)k, &ck.rs);
    if (E < w->p->tp.eabs_g) deposit(w, v, E * ck.wt);
    else push(w, &ck);
  }
}

/* photon: Woodcock free flight (JUMP + STEP) and interaction (KNOCK) */
static void track_photon(worker* w, particle* g) {
  const or_problem* p = w->p;
  const or_phantom* ph = &p->ph;
  double E = -1.0, mbar = 0.0, mu_m[OR_MAX_MAT];
  for (;;) {
    if (g->E != E) {
      E = g->E;
      mbar = 0.0;
      for (int m = 0; m < p->n_mat; ++m) {
        mu_m[m] = or_mu_total(&p->mats[m], E);
        if (p->rho_max[m] > 0.0) mbar = fmax(mbar, p->rho_max[m] * mu_m[m]);
      }
    }
    double fu[4];
    flight_words(&g->rs, fu);
    const double s = -log(fu[0]) / mbar;
    for (int a = 0; a < 3; ++a) g->x[a] += s * g->u[a];
    const int64_t v = locate(ph, g->x, g->u);
    w->st.n_tent++;
    if (v < 0) { w->esc += g->E * g->wt; w->st.n_escape++; return; }
    const int mi = ph->mat[v];
    const double mu_v = ph->rho[v] * mu_m[mi];
    const int real = !(fu[1] * mbar >= mu_v);
    if (w->adj) record_collision(w, v, real, ph->rho[v], mu_m[mi], mbar);
    if (!real) continue;   /* virtual collision */
    w->st.n_real++;
    const or_material* mat = &p->mats[mi];
    const double pc = or_mu_compton(mat, E), pp = or_mu_pe(mat, E);
    const double pr = or_mu_rayleigh(mat, E), pq = or_mu_pair(mat, E);
    const double c = fu[2] * (pc + pp + pr + pq);
    int type = (c < pc) ? 1 : (c < pc + pp) ? 2 : (c < pc + pp + pr) ? 3 : 4;
    if (w->trace && ++w->tr_count == w->tr_k) {
      w->tr_type = type; w->tr_E = E; memcpy(w->tr_xyz, g->x, sizeof w->tr_xyz);
      return;   /* a trace needs nothing after the traced interaction */
    }
    if (type == 1) {                       /* Compton */
      w->st.n_compton++;
      double cost;
      const double k = E / MEC2;
      const double eps = sample_compton(&g->rs, k, &cost);
      const double phi = 2.0 * PI * fu[3];
      const double E1 = eps * E, Te = E - E1;
      double pe[3];
      compton_kinematics(E, eps, cost, phi, g->u, pe);
      emit_charged(w, g, PT_ELECTRON, Te, pe, v, g->wt);
      g->E = E1;
      if (E1 < p->tp.eabs_g) { deposit(w, v, E1 * g->wt); return; }
    } else if (type == 2) {                /* photoelectric */
      w->st.n_pe++;
      emit_charged(w, g, PT_ELECTRON, E, g->u, v, g->wt);
      return;
    } else if (type == 3) {                /* Rayleigh */
      w->st.n_rayleigh++;
      const double cost = sample_rayleigh(&g->rs, mat, E);
      const double phi = 2.0 * PI * fu[3];
      rotate(g->u, cost, phi);
    } else {                               /* pair */
      w->st.n_pair++;
      const double x = pair_split_from_u(fu[3]);
      const double Tk = E - 2.0 * MEC2;
      const double Tm = x * Tk, Tp = Tk - Tm;
      w->w_pair += g->wt;
      emit_charged(w, g, PT_ELECTRON, Tm, g->u, v, g->wt);
      emit_charged(w, g, PT_POSITRON, Tp, g->u, v, g->wt);
      return;
    }
  }
}

/* hard-event partial cross sections (mass units) of material m at T */
static void hard_xs(const or_problem* p, int m, int pos, double T, double* sel, double* sin_, double* sbr) {
  const or_material* mat = &p->mats[m];
  *sel = or_sig_el_hard(mat, T, p->tp.c1);
  *sin_ = or_sig_inel(mat, pos, T, p->tp.wcc);
  *sbr = or_sig_brems(mat, T, p->tp.wcr);
}

typedef struct {
  int64_t v; int ijk[3];
  double r;      /* residual range R_m(T) of the current material */
  int m;
  double path;   /* mass thickness travelled by this particle */
} ctrack;

enum { MV_OK = 0, MV_EXIT = 1, MV_MAT = 2 };

/* STEP for charged particles: move through mass thickness `mass` along u,
 * voxel by voxel (DDA), losing energy by the CSDA range relation and
 * depositing each voxel's share where it is lost. Stops at a material change
 * (particle placed in the new voxel) or at the phantom surface. */
static int move_mass(worker* w, particle* e, ctrack* t, double mass) {
  const or_problem* p = w->p;
  const or_phantom* ph = &p->ph;
  const int pos = (e->type == PT_POSITRON);
  const int nn[3] = {ph->nx, ph->ny, ph->nz};
  double left = mass;
  for (;;) {
    const double rho = ph->rho[t->v];
    int axis; double face;
    const double d = face_distance(ph, t->ijk, e->x, e->u, &axis, &face);
    const double mf = rho * d;
    double mm;
    int crossed = 0;
    if (left <= mf) {
      mm = left;
      const double dd = left / rho;
      for (int a = 0; a < 3; ++a) e->x[a] += dd * e->u[a];
    } else {
      mm = mf;
      for (int a = 0; a < 3; ++a) e->x[a] += d * e->u[a];
      e->x[axis] = face;
      crossed = 1;
    }
    /* CSDA loss over mm in this voxel */
    t->r -= mm;
    double Tn = (t->r > 0.0) ? or_range_inv(p, t->m, pos, t->r) : 0.0;
    if (Tn > e->E) Tn = e->E;
    deposit(w, t->v, (e->E - Tn) * e->wt);
    e->E = Tn;
    left -= mm;
    w->st.e_path += mm;
    t->path += mm;
    if (!crossed) return MV_OK;
    w->st.n_cross++;
    t->ijk[axis] += (e->u[axis] > 0.0) ? 1 : -1;
    if (t->ijk[axis] < 0 || t->ijk[axis] >= nn[axis]) { t->v = -1; return MV_EXIT; }
    t->v = ((int64_t)t->ijk[2] * ph->ny + t->ijk[1]) * ph->nx + t->ijk[0];
    if (ph->mat[t->v] != t->m) return MV_MAT;
  }
}

static void absorb_charged(worker* w, particle* e, int64_t v) {
  w->st.n_e_absorbed++;
  deposit(w, v, e->E * e->wt);
  e->E = 0.0;
  if (e->type == PT_POSITRON) annihilate(w, e);
}

/* two-body kinematics of a hard inelastic collision with a free electron at
 * rest: a particle of kinetic energy T moving along u gives W to the
 * electron; both polar cosines follow from energy and momentum conservation,
 * the two azimuths are opposite (phi and phi + pi). up: the particle's new
 * direction, ud: the electron's. */
static void binary_collision(double T, double W, double phi, const double u[3], double up[3],
                             double ud[3]) {
  const double Tp = T - W;
  const double cp = sqrt(fmin(1.0, (Tp / T) * (T + 2.0 * MEC2) / (Tp + 2.0 * MEC2)));
  const double cd = sqrt(fmin(1.0, (W / T) * (T + 2.0 * MEC2) / (W + 2.0 * MEC2)));
  memcpy(ud, u, 3 * sizeof(double));
  rotate(ud, cd, phi + PI);
  memcpy(up, u, 3 * sizeof(double));
  rotate(up, cp, phi);
}

void or_binary_collision(double T, double W, double phi, const double u[3], double up[3], double ud[3]) {
  binary_collision(T, W, phi, u, up, ud);
}

/* per-atom elastic DCS dsigma/dmu of the screened Rutherford (Wentzel) law */
double or_elastic_dcs(int Z, double T, double mu) {
  double C, A; wentzel_params(Z, T, &C, &A);
  const double d = 1.0 - mu + 2.0 * A;
  return 2.0 * PI * C / (d * d);
}

/* instrumented runs: the compensators of the hard-event counts over the mass
 * thickness m that a step travelled from residual range R0 in material mat:
 * per event type the integral of its (forcing-scaled) cross section at the
 * CSDA energy R^-1(R0 - s), 0 <= s <= m, and the majorant times m (the rate
 * of hard samples); 8-point Gauss-Legendre. The counts minus their
 * compensators have mean zero, whatever the tracks do. */
static void hard_compensators(worker* w, int mat, int pos, double R0, double m, double smaj,
                              double fi, double fb) {
  if (!w->p->instrument || !(m > 0.0)) return;
  const double h = 0.5 * m;
  double a_el = 0.0, a_in = 0.0, a_br = 0.0;
  for (int i = 0; i < GL8_N; ++i) {
    const double E = or_range_inv(w->p, mat, pos, R0 - h * (1.0 + gl8_x[i]));
    double sel, sin_, sbr;
    hard_xs(w->p, mat, pos, E, &sel, &sin_, &sbr);
    a_el += gl8_w[i] * sel; a_in += gl8_w[i] * sin_; a_br += gl8_w[i] * sbr;
  }
  w->st.i_el += h * a_el;
  w->st.i_inel += fi * h * a_in;
  w->st.i_br += fb * h * a_br;
  w->st.i_hat += smaj * m;
}

/* electron / positron: class II mixed simulation with a random hinge */
static void track_charged(worker* w, particle* e) {
  const or_problem* p = w->p;
  const or_phantom* ph = &p->ph;
  const or_transport* tp = &p->tp;
  const int pos = (e->type == PT_POSITRON);
  /* interaction forcing: for a particle whose weight lies in the window, the
   * hard inelastic and hard bremsstrahlung cross sections are multiplied by
   * their forcing factors (the weight of a particle never changes) */
  const int forced = (e->wt >= p->vr.w_lo && e->wt <= p->vr.w_hi);
  const double fi = forced ? p->vr.f_inel : 1.0, fb = forced ? p->vr.f_brems : 1.0;
  ctrack t;
  t.path = 0.0;
  t.v = locate(ph, e->x, e->u);
  if (t.v < 0) { w->esc += e->E * e->wt; w->st.n_escape++; return; }
  vox_ijk(ph, t.v, t.ijk);
  for (;;) {
    if (e->E <= tp->eabs_e) { w->st.e_path_absorbed += t.path; absorb_charged(w, e, t.v); return; }
    w->st.n_e_steps++;
    double su[8];
    step_words(&e->rs, su);
    t.m = ph->mat[t.v];
    const double T0 = e->E;
    const double rho = ph->rho[t.v];
    const double R0 = or_range(p, t.m, pos, T0);
    t.r = R0;
    /* step control: CSDA loss <= step_frac of T (or down to eabs), and at most
     * step_vox voxel widths at the current density */
    double Tlo = (1.0 - tp->step_frac) * T0;
    int final = 0;
    if (Tlo <= tp->eabs_e) { Tlo = tp->eabs_e; final = 1; }
    double tmax = R0 - or_range(p, t.m, pos, Tlo);
    const double tgeo = tp->step_vox * p->dmin * rho;
    if (tgeo < tmax) { tmax = tgeo; final = 0; }
    const double Tend = or_range_inv(p, t.m, pos, R0 - tmax);
    double a1, a2, a3, b1, b2, b3;
    hard_xs(p, t.m, pos, T0, &a1, &a2, &a3);
    hard_xs(p, t.m, pos, Tend, &b1, &b2, &b3);
    const double smaj = fmax(a1 + fi * a2 + fb * a3, b1 + fi * b2 + fb * b3);
    const double th = (smaj > 0.0) ? -log(su[0]) / smaj : INFINITY;
    int hard = 0;
    double tstep = tmax;
    if (th < tmax) { tstep = th; hard = 1; }
    const double tau = su[1] * tstep;
    const double path0 = t.path;
    int st = move_mass(w, e, &t, tau);
    if (st != MV_OK) hard_compensators(w, t.m, pos, R0, t.path - path0, smaj, fi, fb);
    if (st == MV_EXIT) { w->esc += e->E * e->wt; w->st.n_escape++; return; }
    if (st == MV_MAT) continue;
    /* hinge: soft deflection for the whole step, at the step's initial energy */
    const double mbar = -expm1(-tstep * or_sig1_soft(&p->mats[t.m], T0, tp->c1));
    const double mu = sample_soft_u(mbar, su[2]);
    const double phi = 2.0 * PI * su[3];
    rotate(e->u, mu, phi);
    st = move_mass(w, e, &t, tstep - tau);
    hard_compensators(w, t.m, pos, R0, t.path - path0, smaj, fi, fb);
    if (st == MV_EXIT) { w->esc += e->E * e->wt; w->st.n_escape++; return; }
    if (st == MV_MAT) continue;
    if (!hard) {
      if (final) { w->st.e_path_absorbed += t.path; absorb_charged(w, e, t.v); return; }
      continue;
    }
    /* hard event (or delta) at the current energy */
    double sel, sin_, sbr;
    hard_xs(p, t.m, pos, e->E, &sel, &sin_, &sbr);
    sin_ *= fi; sbr *= fb;
    const double c = su[4] * smaj;
    if (c < sel) {
      w->st.n_hard_el++;
      const double cost = sample_el_hard_u(&p->mats[t.m], e->E, tp->c1, su[5], su[6]);
      const double ph2 = 2.0 * PI * su[7];
      rotate(e->u, cost, ph2);
    } else if (c < sel + sin_) {
      w->st.n_hard_inel++;
      const double T = e->E;
      const double W = pos ? sample_bhabha(&e->rs, T, tp->wcc) : sample_moller(&e->rs, T, tp->wcc);
      const double ph2 = 2.0 * PI * draw(&e->rs);
      double up[3], ud[3];
      binary_collision(T, W, ph2, e->u, up, ud);
      /* forced event: the delta ray carries weight wt / fi, and the primary
       * takes the loss and the deflection with probability 1 / fi */
      const int apply = (fi == 1.0) || (draw(&e->rs) * fi < 1.0);
      if (apply) {
        memcpy(e->u, up, sizeof up);
        e->E = T - W;
      }
      emit_charged(w, e, PT_ELECTRON, W, ud, t.v, e->wt / fi);
    } else if (c < sel + sin_ + sbr) {
      w->st.n_hard_br++;
      const double T = e->E;
      const double W = tp->wcr * exp(draw(&e->rs) * log(T / tp->wcr));
      /* forced emission: the photon carries weight wt / fb and the electron
       * loses W with probability 1 / fb; the photon is emitted as n_split
       * copies of weight wt / (fb n_split), each with its own stream */
      const int apply = (fb == 1.0) || (draw(&e->rs) * fb < 1.0);
      if (apply) e->E = T - W;
      emit_photon(w, e, W, e->u, t.v, e->wt / fb, p->vr.n_split_brems);
    } else {
      w->st.n_delta++;
    }
  }
}

/* sample the primary state (Sec. 4.2.1) */
static void primary(worker* w, uint32_t hist, particle* q) {
  const or_problem* p = w->p;
  const or_source* src = &p->src;
  stream_init(&q->rs, w->seed, w->job, hist, 0);
  q->type = src->particle;
  q->wt = 1.0;
  double x = src->x0, y = src->y0;
  if (src->shape == 1) {
    x = src->x0 - src->hx + 2.0 * src->hx * draw(&q->rs);
    y = src->y0 - src->hy + 2.0 * src->hy * draw(&q->rs);
  }
  q->x[0] = x; q->x[1] = y; q->x[2] = 0.0;
  q->u[0] = 0.0; q->u[1] = 0.0; q->u[2] = 1.0;
  q->E = source_energy(p, &q->rs);
}

static void run_history(worker* w, uint32_t hist) {
  particle q;
  primary(w, hist, &q);
  const double esrc = q.E;
  w->dep = 0.0; w->esc = 0.0; w->w_pair = 0.0; w->w_annih = 0.0;
  w->n_stack = 0;
  push(w, &q);
  while (w->n_stack > 0) {
    particle c = w->stack[--w->n_stack];
    w->st.n_particles++;
    if (c.type == PT_PHOTON) track_photon(w, &c);
    else track_charged(w, &c);
  }
  /* energy ledger: E_src + 2mc^2 n_annih = deposits + escapes + 2mc^2 n_pair
   * (weighted; exact per history unless interactions are forced, where it
   * holds in expectation only) */
  const double lhs = esrc + 2.0 * MEC2 * w->w_annih;
  const double rhs = w->dep + w->esc + 2.0 * MEC2 * w->w_pair;
  const double rel = fabs(lhs - rhs) / esrc;
  if (rel > w->st.max_ledger_rel) w->st.max_ledger_rel = rel;
  w->st.e_src += esrc; w->st.e_dep += w->dep; w->st.e_esc += w->esc;
  w->st.n_hist++;
}

/* ======================================================================= */
/* Runs: batches, threads, Eq. 1-3 estimators                             */
/* ======================================================================= */

typedef struct {
  const or_problem* p;
  uint64_t seed; uint32_t job; uint64_t first, n; int K;
  int tid, nthreads;
  int64_t nvox;
  double *sq, *sq2, *s1, *s2;   /* thread-private tallies */
  or_stats st;
  int err;
} job_t;

static void* worker_main(void* arg) {
  job_t* J = (job_t*)arg;
  worker w; memset(&w, 0, sizeof w);
  w.p = J->p; w.seed = J->seed; w.job = J->job;
  w.hq = (double*)calloc(J->nvox, sizeof(double));
  w.touched = (int64_t*)malloc(sizeof(int64_t) * J->nvox);
  double* bt = (double*)calloc(J->nvox, sizeof(double));
  int64_t* btouched = (int64_t*)malloc(sizeof(int64_t) * J->nvox);
  char* bflag = (char*)calloc(J->nvox, 1);
  if (!w.hq || !w.touched || !bt || !btouched || !bflag) { J->err = 1; goto done; }
  for (int k = J->tid; k < J->K; k += J->nthreads) {
    const uint64_t h0 = J->first + (uint64_t)((unsigned __int128)J->n * k / J->K);
    const uint64_t h1 = J->first + (uint64_t)((unsigned __int128)J->n * (k + 1) / J->K);
    if (h1 == h0) continue;
    int64_t nbt = 0;
    for (uint64_t h = h0; h < h1; ++h) {
      w.n_touched = 0;
      run_history(&w, (uint32_t)h);
      for (int64_t i = 0; i < w.n_touched; ++i) {
        const int64_t v = w.touched[i];
        const double q = w.hq[v];
        J->sq[v] += q;
        J->sq2[v] += q * q;
        if (!bflag[v]) { bflag[v] = 1; btouched[nbt++] = v; }
        bt[v] += q;
        w.hq[v] = 0.0;
      }
    }
    const double nk = (double)(h1 - h0);
    for (int64_t i = 0; i < nbt; ++i) {
      const int64_t v = btouched[i];
      J->s1[v] += bt[v];
      J->s2[v] += bt[v] * bt[v] / nk;
      bt[v] = 0.0; bflag[v] = 0;
    }
    w.st.n_batches++;
  }
done:
  J->st = w.st;
  free(w.hq); free(w.touched); free(w.stack); free(bt); free(btouched); free(bflag);
  return NULL;
}

static void add_stats(or_stats* a, const or_stats* b) {
  a->n_hist += b->n_hist; a->n_batches += b->n_batches;
  a->n_tent += b->n_tent; a->n_real += b->n_real; a->n_compton += b->n_compton;
  a->n_pe += b->n_pe; a->n_rayleigh += b->n_rayleigh; a->n_pair += b->n_pair;
  a->n_e_steps += b->n_e_steps; a->n_cross += b->n_cross; a->n_hard_el += b->n_hard_el;
  a->n_hard_inel += b->n_hard_inel; a->n_hard_br += b->n_hard_br; a->n_delta += b->n_delta;
  a->n_annih += b->n_annih; a->n_escape += b->n_escape; a->n_particles += b->n_particles;
  a->e_src += b->e_src; a->e_dep += b->e_dep; a->e_esc += b->e_esc; a->e_path += b->e_path;
  a->e_path_absorbed += b->e_path_absorbed; a->n_e_absorbed += b->n_e_absorbed;
  a->i_el += b->i_el; a->i_inel += b->i_inel; a->i_br += b->i_br; a->i_hat += b->i_hat;
  if (b->max_ledger_rel > a->max_ledger_rel) a->max_ledger_rel = b->max_ledger_rel;
}

int or_run(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
           uint64_t n_hist, int n_batches, int n_threads, or_tally* tally, or_stats* stats) {
  if (!p || !tally || n_batches < 1 || n_threads < 1) return 1;
  if (first_hist + n_hist > 0x100000000ull) return 2;   /* 32-bit history counter */
  const int64_t nvox = (int64_t)p->ph.nx * p->ph.ny * p->ph.nz;
  if (n_threads > n_batches) n_threads = n_batches;
  job_t* J = (job_t*)calloc(n_threads, sizeof(job_t));
  pthread_t* th = (pthread_t*)calloc(n_threads, sizeof(pthread_t));
  int err = 0;
  for (int t = 0; t < n_threads; ++t) {
    J[t].p = p; J[t].seed = seed; J[t].job = job; J[t].first = first_hist; J[t].n = n_hist;
    J[t].K = n_batches; J[t].tid = t; J[t].nthreads = n_threads; J[t].nvox = nvox;
    if (n_threads == 1) {
      J[t].sq = tally->sum_q; J[t].sq2 = tally->sum_q2; J[t].s1 = tally->batch_s1; J[t].s2 = tally->batch_s2;
    } else {
      J[t].sq = (double*)calloc(nvox, sizeof(double));
      J[t].sq2 = (double*)calloc(nvox, sizeof(double));
      J[t].s1 = (double*)calloc(nvox, sizeof(double));
      J[t].s2 = (double*)calloc(nvox, sizeof(double));
      if (!J[t].sq || !J[t].sq2 || !J[t].s1 || !J[t].s2) err = 3;
    }
  }
  if (!err) {
    if (n_threads == 1) worker_main(&J[0]);
    else {
      for (int t = 0; t < n_threads; ++t) pthread_create(&th[t], NULL, worker_main, &J[t]);
      for (int t = 0; t < n_threads; ++t) pthread_join(th[t], NULL);
      /* Eq. 3: the per-thread counters are summed */
      for (int t = 0; t < n_threads; ++t)
        for (int64_t v = 0; v < nvox; ++v) {
          tally->sum_q[v] += J[t].sq[v]; tally->sum_q2[v] += J[t].sq2[v];
          tally->batch_s1[v] += J[t].s1[v]; tally->batch_s2[v] += J[t].s2[v];
        }
    }
    if (stats) for (int t = 0; t < n_threads; ++t) { add_stats(stats, &J[t].st); if (J[t].err) err = 4; }
  }
  if (n_threads > 1)
    for (int t = 0; t < n_threads; ++t) { free(J[t].sq); free(J[t].sq2); free(J[t].s1); free(J[t].s2); }
  free(J); free(th);
  return err;
}

int or_nth_interactions(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
                        uint64_t n_hist, int k, double* xyz, double* E, int* type) {
  if (k < 1) return 1;
  const int64_t nvox = (int64_t)p->ph.nx * p->ph.ny * p->ph.nz;
  worker w; memset(&w, 0, sizeof w);
  w.p = p; w.seed = seed; w.job = job;
  w.hq = (double*)calloc(nvox, sizeof(double));
  w.touched = (int64_t*)malloc(sizeof(int64_t) * nvox);
  for (uint64_t i = 0; i < n_hist; ++i) {
    particle q;
    primary(&w, (uint32_t)(first_hist + i), &q);
    w.trace = 1; w.tr_type = 0; w.tr_k = k; w.tr_count = 0; w.tr_E = 0.0;
    w.n_stack = 0; w.n_touched = 0;
    if (q.type == PT_PHOTON) track_photon(&w, &q);
    type[i] = w.tr_type;
    if (E) E[i] = w.tr_type ? w.tr_E : 0.0;
    for (int a = 0; a < 3; ++a) xyz[3 * i + a] = w.tr_type ? w.tr_xyz[a] : 0.0;
    for (int64_t j = 0; j < w.n_touched; ++j) w.hq[w.touched[j]] = 0.0;
  }
  free(w.hq); free(w.touched); free(w.stack);
  return 0;
}

int or_first_interactions(const or_problem* p, uint64_t seed, uint32_t job,
                          uint64_t first_hist, uint64_t n_hist, double* xyz, int* type) {
  return or_nth_interactions(p, seed, job, first_hist, n_hist, 1, xyz, NULL, type);
}

int or_problem_set_instrument(or_problem* p, int on) {
  p->instrument = on ? 1 : 0;
  return 0;
}

/* ======================================================================= */
/* Fixed majorant and the likelihood-ratio gradient of the dose           */
/* ======================================================================= */

int or_problem_set_vr(or_problem* p, const or_vr* vr) {
  if (!p || !vr) return 1;
  if (!(vr->f_inel >= 1.0) || !(vr->f_brems >= 1.0) || !(vr->w_lo >= 0.0) || !(vr->w_hi >= vr->w_lo) ||
      vr->n_split_brems < 1 || vr->n_split_brems > 64)
    return 1;
  p->vr = *vr;
  return 0;
}

static int vr_active(const or_problem* p) {
  return p->vr.f_inel != 1.0 || p->vr.f_brems != 1.0 || p->vr.n_split_brems != 1;
}

int or_problem_set_majorant(or_problem* p, const double* rho_maj) {
  for (int m = 0; m < p->n_mat; ++m)
    if (!(rho_maj[m] >= p->rho_max[m])) return 1;   /* acceptance would exceed 1 */
  for (int m = 0; m < p->n_mat; ++m) p->rho_max[m] = rho_maj[m];
  return 0;
}

/* The estimator, written out per history h (photon Woodcock flights only carry
 * the density dependence that it differentiates; charged steps are held fixed):
 *   D_u            = E_h[q_hu] / (rho_u V_u)                 (dose, MeV/g)
 *   G_h            = sum_u g_u q_hu / (rho_u V_u)            (g = dL/dD)
 *   S_hv           = sum of the score terms of h's tentative collisions in v
 *   c_hv           = G_h S_hv - g_v q_hv / (rho_v^2 V_v)
 *   dL/drho_v      = E_h[c_hv]
 * c is summed per batch like the dose tally (s1 = sum_k B_k, s2 = sum_k B_k^2/n_k). */
int or_adjoint(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
               uint64_t n_hist, int n_batches, const double* g, double* s1, double* s2,
               or_stats* stats) {
  if (!p || !s1 || !s2 || n_batches < 1) return 1;
  if (first_hist + n_hist > 0x100000000ull) return 2;
  if (vr_active(p)) return 5;   /* the estimator is written for analog histories */
  const or_phantom* ph = &p->ph;
  const int64_t nvox = (int64_t)ph->nx * ph->ny * ph->nz;
  const double V = ph->dx * ph->dy * ph->dz;
  worker w; memset(&w, 0, sizeof w);
  w.p = p; w.seed = seed; w.job = job; w.adj = 1;
  w.hq = (double*)calloc(nvox, sizeof(double));
  w.touched = (int64_t*)malloc(sizeof(int64_t) * nvox);
  double* c = (double*)calloc(nvox, sizeof(double));     /* c_hv of the current history */
  double* bt = (double*)calloc(nvox, sizeof(double));    /* batch sums */
  if (!w.hq || !w.touched || !c || !bt) { free(w.hq); free(w.touched); free(c); free(bt); return 3; }
  for (int k = 0; k < n_batches; ++k) {
    const uint64_t h0 = first_hist + (uint64_t)((unsigned __int128)n_hist * k / n_batches);
    const uint64_t h1 = first_hist + (uint64_t)((unsigned __int128)n_hist * (k + 1) / n_batches);
    if (h1 == h0) continue;
    for (uint64_t h = h0; h < h1; ++h) {
      w.n_touched = 0; w.n_col = 0;
      run_history(&w, (uint32_t)h);
      /* g == NULL: G_h = 1 and no explicit term, i.e. the score alone (mean 0) */
      double G = g ? 0.0 : 1.0;
      if (g)
        for (int64_t i = 0; i < w.n_touched; ++i) {
          const int64_t v = w.touched[i];
          G += g[v] * w.hq[v] / (ph->rho[v] * V);
        }
      for (int64_t i = 0; i < w.n_col; ++i) c[w.col_v[i]] += G * w.col_s[i];
      for (int64_t i = 0; i < w.n_touched; ++i) {
        const int64_t v = w.touched[i];
        if (g) c[v] -= g[v] * w.hq[v] / (ph->rho[v] * ph->rho[v] * V);
        w.hq[v] = 0.0;
      }
      /* move c into the batch sum (every voxel c touched is a collision or a deposit voxel) */
      for (int64_t i = 0; i < w.n_col; ++i) { bt[w.col_v[i]] += c[w.col_v[i]]; c[w.col_v[i]] = 0.0; }
      for (int64_t i = 0; i < w.n_touched; ++i) { bt[w.touched[i]] += c[w.touched[i]]; c[w.touched[i]] = 0.0; }
    }
    const double nk = (double)(h1 - h0);
    for (int64_t v = 0; v < nvox; ++v) {
      s1[v] += bt[v];
      s2[v] += bt[v] * bt[v] / nk;
      bt[v] = 0.0;
    }
    w.st.n_batches++;
  }
  if (stats) add_stats(stats, &w.st);
  free(w.hq); free(w.touched); free(w.stack); free(w.col_v); free(w.col_s); free(c); free(bt);
  return 0;
}

/* Test functionals with closed-form derivatives, on the primary photon's
 * flights up to its first real interaction: G_h = 1 if that interaction is in
 * voxel `target` (target < 0: if the primary leaves without one). Adds per
 * voxel the sums over histories of G_h S_hv and (G_h S_hv)^2, S_hv from those
 * flights' tentative collisions (a virtual term is negative, a real one
 * positive); their mean is dP/drho_v of the event G_h = 1. */
int or_lr_primary(const or_problem* p, uint64_t seed, uint32_t job, uint64_t first_hist,
                  uint64_t n_hist, int64_t target, double* s1, double* s2) {
  if (!p || !s1 || !s2) return 1;
  const int64_t nvox = (int64_t)p->ph.nx * p->ph.ny * p->ph.nz;
  worker w; memset(&w, 0, sizeof w);
  w.p = p; w.seed = seed; w.job = job; w.adj = 1;
  w.hq = (double*)calloc(nvox, sizeof(double));
  w.touched = (int64_t*)malloc(sizeof(int64_t) * nvox);
  double* c = (double*)calloc(nvox, sizeof(double));
  if (!w.hq || !w.touched || !c) { free(w.hq); free(w.touched); free(c); return 3; }
  for (uint64_t i = 0; i < n_hist; ++i) {
    particle q;
    primary(&w, (uint32_t)(first_hist + i), &q);
    if (q.type != PT_PHOTON) continue;
    w.n_col = 0; w.n_touched = 0; w.n_stack = 0;
    track_photon(&w, &q);
    for (int64_t j = 0; j < w.n_touched; ++j) w.hq[w.touched[j]] = 0.0;
    /* the primary's flights end at its first real collision (the first
     * positive score term) or at its escape */
    int64_t end = 0, where = -1;
    while (end < w.n_col && !(w.col_s[end] > 0.0)) ++end;
    if (end < w.n_col) { where = w.col_v[end]; ++end; }
    if (where != target) continue;
    for (int64_t j = 0; j < end; ++j) c[w.col_v[j]] += w.col_s[j];
    for (int64_t j = 0; j < end; ++j) {
      const int64_t v = w.col_v[j];
      if (c[v] != 0.0) { s1[v] += c[v]; s2[v] += c[v] * c[v]; c[v] = 0.0; }
    }
  }
  free(w.hq); free(w.touched); free(w.stack); free(w.col_v); free(w.col_s); free(c);
  return 0;
}
