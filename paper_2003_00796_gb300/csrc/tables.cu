// tables.cu -- host-side FP64 closed-form physics and the FP32 tables the
// kernels interpolate (the KNOCK / JUMP data of Sec. 4.1; the paper's material
// files are replaced by closed forms, see the library header).
//
// Independent of the CPU oracle: different numerical routes are used on
// purpose (closed-form Rayleigh integral with a series near b = 0, composite
// Simpson ranges, bisection inverses), so that parity tests compare two
// implementations rather than one.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "gbmc_internal.h"

namespace gb {
namespace host {

static double apg(const gbmc_material& m, int i) { return kNa * m.w[i] / m.A[i]; }

double electron_density(const gbmc_material& m) {
  double s = 0.0;
  for (int i = 0; i < m.n_el; ++i) s += apg(m, i) * m.Z[i];
  return s;
}

// Klein-Nishina total per electron
double sigma_kn(double k) {
  const double q = 1.0 + 2.0 * k, lq = std::log(q);
  const double a = (1.0 + k) / (k * k) * (2.0 * (1.0 + k) / q - lq / k);
  return 2.0 * kPi * kRe * kRe * (a + lq / (2.0 * k) - (1.0 + 3.0 * k) / (q * q));
}

// I(b) = int_0^2 (1 + (1-t)^2) / (1 + b t)^2 dt, closed form; series for small b
double rayleigh_int(double b) {
  if (b < 0.02) {
    // I = sum_n (-1)^n (n+1) b^n m_n, m_n = int_0^2 (1 + (1-t)^2) t^n dt
    double s = 0.0, bn = 1.0;
    for (int n = 0; n < 16; ++n) {
      const double p = std::pow(2.0, n + 1);
      const double mn = 2.0 * p / (n + 1) - 4.0 * p / (n + 2) + 4.0 * p / (n + 3);
      s += ((n & 1) ? -1.0 : 1.0) * (n + 1) * bn * mn;
      bn *= b;
    }
    return s;
  }
  const double U = 1.0 + 2.0 * b, c = 1.0 + b, lU = std::log1p(2.0 * b);
  return (2.0 * b / U + (c * c * 2.0 * b / U - 2.0 * c * lU + 2.0 * b) / (b * b)) / b;
}

static double qz2(int Z) { const double q = kAlpha / 0.885 * std::cbrt((double)Z); return q * q; }

void photon_xs(const gbmc_material& m, double E, double* co, double* pe, double* ray, double* pair) {
  const double k = E / kMec2;
  *co = electron_density(m) * sigma_kn(k);
  double spe = 0.0, sray = 0.0, spair = 0.0;
  for (int i = 0; i < m.n_el; ++i) {
    const double Z = m.Z[i], n = apg(m, i);
    spe += n * kPeConst * Z * Z * Z * Z;
    sray += n * kPi * kRe * kRe * Z * Z * rayleigh_int(2.0 * k * k / qz2(m.Z[i]));
    if (k > 2.0) {
      const double r = (k - 2.0) / k;
      const double f = std::max(2.0 * kPi / 3.0 * r * r * r, 28.0 / 9.0 * std::log(2.0 * k) - 218.0 / 27.0);
      spair += n * kAlpha * kRe * kRe * Z * (Z + 1.0) * f;
    }
  }
  *pe = spe / (E * E * E);
  *ray = sray;
  *pair = spair;
}

// --- charged particles ----------------------------------------------------

struct ElKin { double tau, b2, p2; };
static ElKin kin(double T) { ElKin k; k.tau = T / kMec2; k.p2 = k.tau * (k.tau + 2.0); k.b2 = k.p2 / ((k.tau + 1.0) * (k.tau + 1.0)); return k; }

double s_col(const gbmc_material& m, bool pos, double T) {
  const ElKin k = kin(T);
  const double ir = m.I_eV * 1e-6 / kMec2;
  const double t = k.tau;
  double F;
  if (!pos) {
    F = 1.0 - k.b2 + (t * t / 8.0 - (2.0 * t + 1.0) * std::log(2.0)) / ((t + 1.0) * (t + 1.0));
  } else {
    const double y = t + 2.0;
    F = 2.0 * std::log(2.0) - k.b2 / 12.0 * (23.0 + 14.0 / y + 10.0 / (y * y) + 4.0 / (y * y * y));
  }
  return 2.0 * kPi * kRe * kRe * kMec2 * electron_density(m) / k.b2 *
         (std::log(t * t * (t + 2.0) / (2.0 * ir * ir)) + F);
}

// hard inelastic: number (per g) and energy-loss integral (MeV per g) above wcc
void hard_inel(const gbmc_material& m, bool pos, double T, double wcc, double* num, double* loss) {
  *num = 0.0; *loss = 0.0;
  const ElKin k = kin(T);
  const double K = 2.0 * kPi * kRe * kRe * kMec2 / k.b2 * electron_density(m);
  if (!pos) {
    if (T <= 2.0 * wcc) return;
    const double a = (k.tau / (k.tau + 1.0)) * (k.tau / (k.tau + 1.0));
    const double b = (2.0 * k.tau + 1.0) / ((k.tau + 1.0) * (k.tau + 1.0));
    const double e = wcc / T;
    // int_e^1/2 [1/x^2 + 1/(1-x)^2 + a - b/(x(1-x))] dx
    *num = K / T * (1.0 / e - 1.0 / (1.0 - e) + a * (0.5 - e) - b * std::log((1.0 - e) / e));
    // int_e^1/2 x [..] dx, antiderivative ln x + 1/(1-x) + (1+b) ln(1-x) + a x^2/2
    auto H = [&](double x) { return std::log(x) + 1.0 / (1.0 - x) + (1.0 + b) * std::log1p(-x) + 0.5 * a * x * x; };
    *loss = K * (H(0.5) - H(e));
  } else {
    if (T <= wcc) return;
    *num = K * (1.0 / wcc - 1.0 / T);
    *loss = K * std::log(T / wcc);
  }
}

double inv_x0(const gbmc_material& m) {
  double s = 0.0;
  for (int i = 0; i < m.n_el; ++i) {
    const double Z = m.Z[i];
    s += apg(m, i) * Z * (Z + 1.0) * std::log(183.0 / std::cbrt(Z));
  }
  return 4.0 * kAlpha * kRe * kRe * s;
}

double s_restricted(const gbmc_material& m, bool pos, double T, double wcc, double wcr) {
  double n, l;
  hard_inel(m, pos, T, wcc, &n, &l);
  return s_col(m, pos, T) - l + inv_x0(m) * std::min(T, wcr);
}

// screened Rutherford parameters per atom: dsigma/dmu = 2 pi C/(1 - mu + 2A)^2
static void wentzel(int Zi, double T, double* C, double* A) {
  const ElKin k = kin(T);
  const double Z = Zi;
  const double f = (k.tau + 1.0) / k.p2;
  *C = Z * (Z + 1.0) * kRe * kRe * f * f;
  const double s = kAlpha * std::cbrt(Z) / 0.885;
  *A = 0.25 * s * s / k.p2 * (1.13 + 3.76 * (kAlpha * Z) * (kAlpha * Z) / k.b2);
}

// hard-elastic count above cut deflection xc (per g)
static double el_above(const gbmc_material& m, double T, double xc) {
  double s = 0.0;
  for (int i = 0; i < m.n_el; ++i) {
    double C, A; wentzel(m.Z[i], T, &C, &A);
    s += apg(m, i) * 2.0 * kPi * C * (2.0 - xc) / ((xc + 2.0 * A) * (2.0 + 2.0 * A));
  }
  return s;
}

// hard elastic xs = min(sigma_el, sigma_1 / c1), its cut xc, and the soft
// first transport xs below the cut
void elastic(const gbmc_material& m, double T, double c1, double* hard, double* xc, double* soft1) {
  double sel = 0.0, s1 = 0.0;
  for (int i = 0; i < m.n_el; ++i) {
    double C, A; wentzel(m.Z[i], T, &C, &A);
    const double n = apg(m, i);
    sel += n * kPi * C / (A * (1.0 + A));
    s1 += n * 2.0 * kPi * C * (std::log1p(1.0 / A) - 1.0 / (1.0 + A));
  }
  if (sel <= s1 / c1) { *hard = sel; *xc = 0.0; *soft1 = 0.0; return; }
  *hard = s1 / c1;
  double lo = 0.0, hi = 2.0;
  for (int it = 0; it < 120; ++it) {
    const double mid = 0.5 * (lo + hi);
    (el_above(m, T, mid) > *hard ? lo : hi) = mid;
  }
  *xc = 0.5 * (lo + hi);
  double s = 0.0;
  for (int i = 0; i < m.n_el; ++i) {
    double C, A; wentzel(m.Z[i], T, &C, &A);
    const double y = *xc / (2.0 * A);
    s += apg(m, i) * 2.0 * kPi * C * (std::log1p(y) - y / (1.0 + y));
  }
  *soft1 = s;
}

// 1 - <mu> of the Wentzel law with parameter A on [-1, 1]
static double wentzel_mean(double A) {
  if (A > 500.0) {  // series in y = 1/A
    const double y = 1.0 / A;
    return 1.0 - y / 3.0 + y * y / 6.0 - y * y * y / 10.0 + y * y * y * y / 15.0;
  }
  return 2.0 * A * ((1.0 + A) * std::log1p(1.0 / A) - 1.0);
}

double soft_aprime(double mbar) {
  double lo = std::log(1e-14), hi = std::log(1e6);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    (wentzel_mean(std::exp(mid)) < mbar ? lo : hi) = mid;
  }
  return std::exp(0.5 * (lo + hi));
}

}  // namespace host

// ---------------------------------------------------------------------------
// Table construction
// ---------------------------------------------------------------------------

static float lg2(double v) { return v > 0.0 ? (float)std::log2(v) : kLog2Zero; }

// Range with an offset: R'(E) = Emin / S(Emin) + int_Emin^E dE/S, by composite
// Simpson in ln E on a fine grid; values at the fine nodes.
struct FineRange {
  std::vector<double> lnE, R;
  double eval(double E) const {   // interpolation of ln R' in ln E (cubic-free, fine grid)
    const double x = (std::log(E) - lnE[0]) / (lnE[1] - lnE[0]);
    int i = (int)std::floor(x);
    i = std::max(0, std::min(i, (int)lnE.size() - 2));
    const double f = x - i;
    return std::exp(std::log(R[i]) * (1.0 - f) + std::log(R[i + 1]) * f);
  }
};

static FineRange build_range(const gbmc_material& m, bool pos, const gbmc_transport& tp,
                             double emin, double emax) {
  const int nf = 8192, sub = 8;
  FineRange fr;
  fr.lnE.resize(nf); fr.R.resize(nf);
  const double l0 = std::log(emin), l1 = std::log(emax), h = (l1 - l0) / (nf - 1);
  auto g = [&](double l) { const double E = std::exp(l); return E / host::s_restricted(m, pos, E, tp.wcc, tp.wcr); };
  fr.lnE[0] = l0;
  fr.R[0] = emin / host::s_restricted(m, pos, emin, tp.wcc, tp.wcr);
  for (int i = 1; i < nf; ++i) {
    const double a = l0 + h * (i - 1), hs = h / sub;
    double acc = g(a) + g(a + h);
    for (int j = 1; j < sub; ++j) acc += (j & 1 ? 4.0 : 2.0) * g(a + j * hs);
    fr.lnE[i] = l0 + h * i;
    fr.R[i] = fr.R[i - 1] + acc * hs / 3.0;
  }
  return fr;
}

// photon energy (MeV) at which the pair cross section's two branches meet:
// the threshold form (2 pi / 3) ((k - 2) / k)^3 and the asymptotic form
// (28 / 9) ln 2k - 218 / 27 cross at one k for every element (bisection in
// FP64). The attenuation table has a kink there; a grid node placed on it
// keeps the log-log interpolation error at the smooth-function level.
static double pair_kink_energy() {
  auto g = [](double k) {
    const double r = (k - 2.0) / k;
    return 2.0 * kPi / 3.0 * r * r * r - (28.0 / 9.0 * std::log(2.0 * k) - 218.0 / 27.0);
  };
  double a = 4.0, b = 40.0;   // g(a) > 0 > g(b)
  for (int it = 0; it < 200; ++it) {
    const double m = 0.5 * (a + b);
    (g(m) > 0.0 ? a : b) = m;
  }
  return 0.5 * (a + b) * kMec2;
}

bool build_tables(Tables& T, const gbmc_material* mats, int n_mat, const gbmc_transport& tp,
                  double emax, int nE, int nA) {
  T.n_mat = n_mat; T.nE = nE; T.nR = nE; T.nA = nA;
  T.emin = 1e-3; T.emax = emax;
  // uniform log2 E grid from emin, its spacing widened (at most by one part in
  // the number of nodes below the kink) so that a node falls on the pair kink
  double dl = (std::log2(emax) - std::log2(T.emin)) / (nE - 1);
  const double lk = std::log2(pair_kink_energy()) - std::log2(T.emin);
  if (lk > 4.0 * dl && lk < (nE - 2) * dl) dl = lk / std::floor(lk / dl);
  T.lg0 = (float)std::log2(T.emin);
  T.inv_d = (float)(1.0 / dl);
  T.data.assign(tab_size_floats(n_mat, nE, nE, nA), 0.0f);
  T.mu_tot.assign((size_t)n_mat * nE, 0.0);
  for (int m = 0; m < n_mat; ++m) {
    const gbmc_material& M = mats[m];
    for (int i = 0; i < nE; ++i) {
      const double E = std::exp2(std::log2(T.emin) + dl * i);
      double co, pe, ray, pair;
      host::photon_xs(M, E, &co, &pe, &ray, &pair);
      const double tot = co + pe + ray + pair;
      T.mu_tot[(size_t)m * nE + i] = tot;
      T.data[tab_off(Q_MU_TOT, m, n_mat, nE) + i] = lg2(tot);
      T.data[tab_off(Q_MU_CO, m, n_mat, nE) + i] = lg2(co);
      T.data[tab_off(Q_MU_PE, m, n_mat, nE) + i] = lg2(pe);
      T.data[tab_off(Q_MU_RAY, m, n_mat, nE) + i] = lg2(ray);
      double hard, xc, soft1;
      host::elastic(M, E, tp.c1, &hard, &xc, &soft1);
      T.data[tab_off(Q_SIG_EL, m, n_mat, nE) + i] = lg2(hard);
      T.data[tab_off(Q_XC, m, n_mat, nE) + i] = (float)xc;
      T.data[tab_off(Q_SIG1, m, n_mat, nE) + i] = lg2(soft1);
      double n_e, n_p, l;
      host::hard_inel(M, false, E, tp.wcc, &n_e, &l);
      T.data[tab_off(Q_SIG_INEL_E, m, n_mat, nE) + i] = lg2(n_e);
      host::hard_inel(M, true, E, tp.wcc, &n_p, &l);
      T.data[tab_off(Q_SIG_INEL_P, m, n_mat, nE) + i] = lg2(n_p);
      const double br = E > tp.wcr ? host::inv_x0(M) * std::log(E / tp.wcr) : 0.0;
      T.data[tab_off(Q_SIG_BR, m, n_mat, nE) + i] = lg2(br);
      // the summed hard cross section: between nodes its log-linear
      // interpolation is never below the sum of the parts' log-linear
      // interpolations (Hoelder: sum a^(1-f) b^f <= (sum a)^(1-f) (sum b)^f),
      // so it bounds them for the step majorant; 3e-5 in log2 covers FP32
      // rounding
      T.data[tab_off(Q_SIG_H_E, m, n_mat, nE) + i] = lg2(hard + n_e + br) + 3e-5f;
      T.data[tab_off(Q_SIG_H_P, m, n_mat, nE) + i] = lg2(hard + n_p + br) + 3e-5f;
    }
    for (int s = 0; s < 2; ++s) {
      const FineRange fr = build_range(M, s == 1, tp, T.emin, std::exp2(std::log2(T.emin) + dl * (nE - 1)));
      const int qR = s ? Q_R_P : Q_R_E, qI = s ? Q_RINV_P : Q_RINV_E;
      for (int i = 0; i < nE; ++i) {
        const double E = std::exp2(std::log2(T.emin) + dl * i);
        T.data[tab_off(qR, m, n_mat, nE) + i] = (float)std::log2(fr.eval(E));
      }
      // inverse: log2 E on a uniform log2 r grid
      const double r0 = std::log2(fr.R.front()), r1 = std::log2(fr.R.back());
      T.lr0[m][s] = (float)r0;
      T.inv_dr[m][s] = (float)((nE - 1) / (r1 - r0));
      for (int j = 0; j < nE; ++j) {
        const double r = std::exp2(r0 + (r1 - r0) * j / (nE - 1));
        // find E with R'(E) = r on the fine grid, then refine by bisection
        int lo = 0, hi = (int)fr.R.size() - 1;
        while (hi - lo > 1) { const int mid = (lo + hi) / 2; (fr.R[mid] <= r ? lo : hi) = mid; }
        double a = fr.lnE[lo], b = fr.lnE[hi];
        for (int it = 0; it < 80; ++it) {
          const double mid = 0.5 * (a + b);
          (fr.eval(std::exp(mid)) <= r ? a : b) = mid;
        }
        T.data[tab_off(qI, m, n_mat, nE) + j] = (float)(0.5 * (a + b) / std::log(2.0));
      }
    }
  }
  // soft-deflection A'(mbar) on a uniform grid of y = log2(mbar / (1 - mbar)),
  // where log2 A' is close to linear at both ends (A' ~ mbar at small mbar,
  // A' ~ 1 / (3 (1 - mbar)) as mbar -> 1)
  auto logit2 = [](double x) { return std::log2(x / (1.0 - x)); };
  const double ya = logit2(1e-9), yb = logit2(0.9999);
  T.la0 = (float)ya;
  T.inv_da = (float)((nA - 1) / (yb - ya));
  T.off_major = 4 * n_mat * nE;
  T.off_soft = tab_off_e(n_mat, nE) + (NQ - Q_SIG_EL) * n_mat * nE;
  for (int j = 0; j < nA; ++j) {
    const double y = ya + (yb - ya) * j / (nA - 1);
    const double mb = 1.0 / (1.0 + std::exp2(-y));
    T.data[T.off_soft + j] = (float)std::log2(host::soft_aprime(mb));
  }
  // per-element sampling data
  for (int m = 0; m < n_mat; ++m) {
    DevMat& d = T.dmat[m];
    std::memset(&d, 0, sizeof d);
    const gbmc_material& M = mats[m];
    d.n_el = M.n_el;
    for (int i = 0; i < M.n_el; ++i) {
      const double Z = M.Z[i], n = kNa * M.w[i] / M.A[i];
      d.ray_w[i] = (float)(n * Z * Z * 1e-22);
      d.ray_iqz2[i] = (float)(1.0 / (std::pow(kAlpha / 0.885, 2) * std::pow(Z, 2.0 / 3.0)));
      d.el_w[i] = (float)(n * Z * (Z + 1.0) * 1e-22);
      const double s = kAlpha * std::cbrt(Z) / 0.885;
      d.el_cA[i] = (float)(0.25 * s * s);
      d.el_cB[i] = (float)(3.76 * (kAlpha * Z) * (kAlpha * Z));
    }
  }
  // which element a hard elastic event is on: cumulative probabilities of
  // elements 0 .. n_el - 2 at the energy nodes, P_i(E) = sum_{j<=i} w_j / sum w,
  // w_j = n_j C_j / ((xc + 2 A_j)(2 + 2 A_j)), the partial hard cross sections
  // above the cut xc(E) (staged with the charged region)
  T.n_staged = (int)T.data.size();
  for (int m = 0; m < n_mat; ++m) {
    const gbmc_material& M = mats[m];
    if (M.n_el < 2) { T.off_el[m] = -1; continue; }
    T.off_el[m] = (int)T.data.size();
    T.data.resize(T.data.size() + (size_t)(M.n_el - 1) * nE, 0.0f);
    for (int k = 0; k < nE; ++k) {
      const double E = std::exp2(std::log2(T.emin) + dl * k);
      double hard, xc, soft1;
      host::elastic(M, E, tp.c1, &hard, &xc, &soft1);
      double w[GBMC_MAX_EL], sum = 0.0;
      for (int j = 0; j < M.n_el; ++j) {
        double C, A; host::wentzel(M.Z[j], E, &C, &A);
        w[j] = host::apg(M, j) * C / ((xc + 2.0 * A) * (2.0 + 2.0 * A));
        sum += w[j];
      }
      double c = 0.0;
      for (int j = 0; j + 1 < M.n_el; ++j) {
        c += w[j];
        T.data[T.off_el[m] + (size_t)j * nE + k] = (float)(c / sum);
      }
    }
  }
  // per-material parameters (MatPar), offsets relative to the charged region
  T.off_mpar = (int)T.data.size();
  T.data.resize(T.data.size() + (size_t)MP_STRIDE * n_mat, 0.0f);
  const int e0 = tab_off_e(n_mat, nE);
  for (int m = 0; m < n_mat; ++m) {
    float* mp = T.data.data() + T.off_mpar + (size_t)m * MP_STRIDE;
    mp[MP_LR0_E] = T.lr0[m][0]; mp[MP_INVDR_E] = T.inv_dr[m][0];
    mp[MP_LR0_P] = T.lr0[m][1]; mp[MP_INVDR_P] = T.inv_dr[m][1];
    mp[MP_NEL] = (float)mats[m].n_el;
    mp[MP_OFF_EL] = T.off_el[m] >= 0 ? (float)(T.off_el[m] - e0) : -1.0f;
    for (int i = 0; i < mats[m].n_el; ++i) {
      mp[MP_EL_CA + i] = T.dmat[m].el_cA[i];
      mp[MP_EL_CB + i] = T.dmat[m].el_cB[i];
    }
  }
  return true;
}

// photon majorant per energy node, log2 of max_m rho_max[m] mu_m(E). Between
// nodes its log-linear interpolation is at least every material's (the
// interpolation of a maximum bounds the maximum of the interpolations), so
// the margin only has to cover FP32 rounding of the lookups: 1e-5
void majorant_table(const Tables& T, const double* rho_max, float* out) {
  for (int i = 0; i < T.nE; ++i) {
    double mb = 0.0;
    for (int m = 0; m < T.n_mat; ++m)
      mb = std::max(mb, rho_max[m] * T.mu_tot[(size_t)m * T.nE + i]);
    out[i] = lg2(mb * (1.0 + 1e-5));
  }
}

void build_majorant(Tables& T, const double* rho_max) {
  majorant_table(T, rho_max, T.data.data() + T.off_major);
}

}  // namespace gb
