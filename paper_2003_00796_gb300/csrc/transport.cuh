// transport.cuh -- device physics of one particle: photon Woodcock flight and
// interactions, class II electron/positron steps with a random hinge and a
// voxel DDA, primary sampling, scoring. Used by the plain kernel and by the
// wavefront kernels.
//
// Paper roles: JUMP / STEP / KNOCK of Sec. 4.1; primary state samplers of
// Sec. 4.2.1; LOCATE / STEP of the voxel geometry of Sec. 4.2.2; tally scoring
// of Sec. 4.2.3. The physics is the closed-form set documented in gbmc.h's
// companion design notes (FP32 stepping and sampling; FP64 for the pair split).
#pragma once

#include "gbmc_common.cuh"

namespace gb {

constexpr int kCapWoodcock = 1 << 20;   // tentative collisions per photon flight
constexpr int kCapEsteps = 1 << 17;     // steps per charged particle
constexpr int kCapDda = 1 << 16;        // voxel crossings per charged segment
constexpr int kCapReject = 1 << 12;     // rejection-sampling trials

// ---------------------------------------------------------------------------
// Per-thread tracking context
// ---------------------------------------------------------------------------
struct Track {
  const DevProblem* P;
  const float* tab;          // tables staged in shared memory
  // pending deposit (consecutive deposits into one voxel are merged)
  int pv;
  float pe;
  // counters and ledger
  uint32_t c_tent, c_real, c_estep, c_cross, c_hard, c_part;
  double l_src, l_esc, l_pair;
  uint32_t err;
};

// the particle being tracked (registers)
struct Live {
  float x, y, z, u, v, w, E;
  int type;
  uint64_t path;
  uint32_t nchild;
  Rng rng;
};

GB_D float rnd(Track& t, Live& p) { return rng_draw(p.rng, t.P->key0, t.P->key1); }

GB_D void score_flush(Track& t) {
  if (t.pv >= 0 && t.pe > 0.0f) atomicAdd(t.P->tile + t.pv, t.pe);
  t.pv = -1;
  t.pe = 0.0f;
}

GB_D void score(Track& t, int v, float e) {
  if (!(e > 0.0f)) return;
  if (v == t.pv) { t.pe += e; return; }
  score_flush(t);
  t.pv = v;
  t.pe = e;
}

GB_D const float* tq(const Track& t, int q, int m) {
  return t.tab + tab_off(q, m, t.P->n_mat, t.P->nE);
}

GB_D GridPos egrid(const Track& t, float E) {
  return grid_pos(log2f(E), t.P->lg0, t.P->inv_d, t.P->nE);
}

// ---------------------------------------------------------------------------
// Geometry (Sec. 4.2.2 LOCATE): a point on a plane belongs to the voxel its
// direction enters; floor when that direction component is zero.
// ---------------------------------------------------------------------------
GB_D int locate_axis(float x, float u, float id, int n) {
  const float f = x * id;
  const float fl = floorf(f);
  int i = (int)fl;
  if (f == fl && u < 0.0f) i -= 1;
  return (f < 0.0f || i < 0 || i >= n) ? -1 : i;
}

GB_D int locate(const DevProblem& P, float x, float y, float z, float u, float v, float w,
                int& ix, int& iy, int& iz) {
  ix = locate_axis(x, u, P.idx, P.nx);
  iy = locate_axis(y, v, P.idy, P.ny);
  iz = locate_axis(z, w, P.idz, P.nz);
  if ((ix | iy | iz) < 0) return -1;
  return iz * P.nxy + iy * P.nx + ix;
}

// rotate direction by polar cosine cost and azimuth (cos phi, sin phi)
GB_D void rotate(float& u, float& v, float& w, float cost, float cp, float sp) {
  cost = fminf(1.0f, fmaxf(-1.0f, cost));
  const float sint = sqrtf(fmaxf(0.0f, 1.0f - cost * cost));
  const float s2 = u * u + v * v;
  float nu, nv, nw;
  if (s2 > 1e-10f) {
    const float s = sqrtf(s2), is = 1.0f / s;
    nu = u * cost + sint * (u * w * cp - v * sp) * is;
    nv = v * cost + sint * (v * w * cp + u * sp) * is;
    nw = w * cost - sint * cp * s;
  } else {
    nu = sint * cp;
    nv = sint * sp;
    nw = (w >= 0.0f ? 1.0f : -1.0f) * cost;
  }
  const float r = rsqrtf(nu * nu + nv * nv + nw * nw);
  u = nu * r; v = nv * r; w = nw * r;
}

// ---------------------------------------------------------------------------
// Secondaries
// ---------------------------------------------------------------------------
struct Stack {
  Particle* s;
  int sp, cap;
};

GB_D void make_child(const Live& parent, uint32_t ordinal, Particle& c, int type, float E,
                     float u, float v, float w) {
  c.x = parent.x; c.y = parent.y; c.z = parent.z;
  c.u = u; c.v = v; c.w = w; c.E = E; c.type = type;
  const uint64_t path = child_path(parent.path, ordinal);
  c.path_lo = (uint32_t)path; c.path_hi = (uint32_t)(path >> 32);
  c.hist = parent.rng.hist; c.nchild = 0;
}

GB_D void push(Track& t, Stack& st, const Particle& c, int vox) {
  if (st.sp < st.cap) {
    st.s[st.sp++] = c;
  } else {
    // overflow: the particle is scored where it was made and flagged
    t.err |= E_STACK;
    score(t, vox, c.E);
  }
}

GB_D void live_from(Live& p, const Particle& c) {
  p.x = c.x; p.y = c.y; p.z = c.z; p.u = c.u; p.v = c.v; p.w = c.w; p.E = c.E;
  p.type = c.type;
  p.path = ((uint64_t)c.path_hi << 32) | c.path_lo;
  p.nchild = c.nchild;
  rng_init(p.rng, c.hist, p.path, 0);
}

// positron at rest: two back-to-back isotropic 0.511 MeV photons
GB_D void annihilate(Track& t, Stack& st, Live& e, int vox) {
  const float cost = 2.0f * rnd(t, e) - 1.0f;
  float sp, cp;
  sincospif(2.0f * rnd(t, e), &sp, &cp);
  const float sint = sqrtf(fmaxf(0.0f, 1.0f - cost * cost));
  Particle g;
  make_child(e, ++e.nchild, g, GBMC_PHOTON, kMec2f, sint * cp, sint * sp, cost);
  push(t, st, g, vox);
  make_child(e, ++e.nchild, g, GBMC_PHOTON, kMec2f, -sint * cp, -sint * sp, -cost);
  push(t, st, g, vox);
  t.l_pair -= 2.0 * kMec2;
}

// charged secondary made at an interaction in voxel vox
GB_D void emit_charged(Track& t, Stack& st, Live& parent, int type, float T, float u, float v,
                       float w, int vox) {
  Particle c;
  make_child(parent, ++parent.nchild, c, type, T, u, v, w);
  if (T < t.P->eabs_e) {
    score(t, vox, T);
    if (type == GBMC_POSITRON) {
      Live q;
      live_from(q, c);
      annihilate(t, st, q, vox);
    }
  } else {
    push(t, st, c, vox);
  }
}

GB_D void emit_photon(Track& t, Stack& st, Live& parent, float E, int vox) {
  Particle c;
  make_child(parent, ++parent.nchild, c, GBMC_PHOTON, E, parent.u, parent.v, parent.w);
  if (E < t.P->eabs_g) score(t, vox, E);
  else push(t, st, c, vox);
}

// ---------------------------------------------------------------------------
// Photon KNOCK samplers
// ---------------------------------------------------------------------------

// Klein-Nishina, Butcher & Messel decomposition; returns eps = E'/E
GB_D float sample_compton(Track& t, Live& p, float k, float& cost) {
  const float e0 = 1.0f / (1.0f + 2.0f * k);
  const float a1 = log1pf(2.0f * k), a2 = 0.5f * (1.0f - e0 * e0);
  float eps = 1.0f, tt = 0.0f;
  for (int it = 0; it < kCapReject; ++it) {
    const float u1 = rnd(t, p), u2 = rnd(t, p), u3 = rnd(t, p);
    eps = (u1 * (a1 + a2) < a1) ? expf(-a1 * u2) : sqrtf(fmaf(1.0f - e0 * e0, u2, e0 * e0));
    tt = (1.0f - eps) / (k * eps);
    const float sin2 = tt * (2.0f - tt);
    const float g = 1.0f - eps * sin2 / (1.0f + eps * eps);
    if (u3 <= g) { cost = 1.0f - tt; return eps; }
  }
  t.err |= E_REJECT;
  cost = 1.0f - tt;
  return eps;
}

// Rayleigh: composition over elements of 1/(1 + b t)^2, rejection (1 + cos^2)/2
GB_D float sample_rayleigh(Track& t, Live& p, const DevMat& M, float E) {
  const float k = E / kMec2f, k2 = 2.0f * k * k;
  float wsum = 0.0f;
#pragma unroll
  for (int i = 0; i < GBMC_MAX_EL; ++i)
    if (i < M.n_el) wsum += M.ray_w[i] * 2.0f / (1.0f + 2.0f * k2 * M.ray_iqz2[i]);
  float tt = 0.0f;
  for (int it = 0; it < kCapReject; ++it) {
    const float u1 = rnd(t, p), u2 = rnd(t, p), u3 = rnd(t, p);
    float c = u1 * wsum, b = 0.0f;
#pragma unroll
    for (int i = 0; i < GBMC_MAX_EL; ++i) {
      if (i < M.n_el) {
        const float bi = k2 * M.ray_iqz2[i];
        const float wi = M.ray_w[i] * 2.0f / (1.0f + 2.0f * bi);
        if (b == 0.0f && (c < wi || i == M.n_el - 1)) b = fmaxf(bi, 1e-30f);
        c -= wi;
      }
    }
    tt = 2.0f * u2 / (1.0f + 2.0f * b * (1.0f - u2));
    if (u3 <= 0.5f * (1.0f + (1.0f - tt) * (1.0f - tt))) return 1.0f - tt;
  }
  t.err |= E_REJECT;
  return 1.0f - tt;
}

// pair split x = T-/(E - 2mc^2): inverse of (9x - 6x^2 + 4x^3)/7 in FP64
GB_D double pair_split(double u) {
  double lo = 0.0, hi = 1.0, x = u;
  for (int it = 0; it < 64; ++it) {
    const double f = (x * (9.0 + x * (-6.0 + 4.0 * x))) / 7.0 - u;
    if (f > 0.0) hi = x; else lo = x;
    const double d = (9.0 + x * (-12.0 + 12.0 * x)) / 7.0;
    double xn = x - f / d;
    if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
    const bool done = fabs(xn - x) < 1e-15;
    x = xn;
    if (done) break;
  }
  return x;
}

// ---------------------------------------------------------------------------
// Photon: Woodcock flight and interaction. Returns when the photon dies.
// ---------------------------------------------------------------------------
GB_D void photon_track(Track& t, Stack& st, Live& p) {
  const DevProblem& P = *t.P;
  float lastE = -1.0f, mbar = 1.0f, mu0 = 0.f, mu1 = 0.f, mu2 = 0.f, mu3 = 0.f;
  GridPos gp;
  gp.i = 0; gp.f = 0.0f;
  for (int it = 0; it < kCapWoodcock; ++it) {
    if (p.E != lastE) {
      lastE = p.E;
      gp = egrid(t, p.E);
      mbar = exp2_tab(t.tab + P.off_major, gp);
      mu0 = exp2_tab(tq(t, Q_MU_TOT, 0), gp);
      if (P.n_mat > 1) mu1 = exp2_tab(tq(t, Q_MU_TOT, 1), gp);
      if (P.n_mat > 2) mu2 = exp2_tab(tq(t, Q_MU_TOT, 2), gp);
      if (P.n_mat > 3) mu3 = exp2_tab(tq(t, Q_MU_TOT, 3), gp);
    }
    const float s = -logf(rnd(t, p)) / mbar;
    p.x = fmaf(s, p.u, p.x);
    p.y = fmaf(s, p.v, p.y);
    p.z = fmaf(s, p.w, p.z);
    int ix, iy, iz;
    const int vox = locate(P, p.x, p.y, p.z, p.u, p.v, p.w, ix, iy, iz);
    ++t.c_tent;
    if (vox < 0) { t.l_esc += p.E; return; }
    const int m = __ldg(P.mat + vox);
    const float rho = __ldg(P.rho + vox);
    const float mum = (m == 0) ? mu0 : (m == 1) ? mu1 : (m == 2) ? mu2 : mu3;
    if (rnd(t, p) * mbar >= rho * mum) continue;          // virtual collision
    ++t.c_real;
    const float co = exp2_tab(tq(t, Q_MU_CO, m), gp);
    const float pe = exp2_tab(tq(t, Q_MU_PE, m), gp);
    const float ray = exp2_tab(tq(t, Q_MU_RAY, m), gp);
    const float c = rnd(t, p) * mum;
    if (c < co) {                                         // Compton
      float cost;
      const float k = p.E / kMec2f;
      const float eps = sample_compton(t, p, k, cost);
      float sp, cp;
      sincospif(2.0f * rnd(t, p), &sp, &cp);
      const float E0 = p.E, E1 = eps * E0, Te = E0 - E1;
      const float u0 = p.u, v0 = p.v, w0 = p.w;
      rotate(p.u, p.v, p.w, cost, cp, sp);
      float eu = E0 * u0 - E1 * p.u, ev = E0 * v0 - E1 * p.v, ew = E0 * w0 - E1 * p.w;
      const float n2 = eu * eu + ev * ev + ew * ew;
      if (n2 > 0.0f) { const float r = rsqrtf(n2); eu *= r; ev *= r; ew *= r; }
      else { eu = u0; ev = v0; ew = w0; }
      emit_charged(t, st, p, GBMC_ELECTRON, Te, eu, ev, ew, vox);
      p.E = E1;
      if (E1 < P.eabs_g) { score(t, vox, E1); return; }
    } else if (c < co + pe) {                             // photoelectric
      emit_charged(t, st, p, GBMC_ELECTRON, p.E, p.u, p.v, p.w, vox);
      return;
    } else if (c < co + pe + ray || p.E <= 2.0f * kMec2f) {  // Rayleigh
      const float cost = sample_rayleigh(t, p, P.mats[m], p.E);
      float sp, cp;
      sincospif(2.0f * rnd(t, p), &sp, &cp);
      rotate(p.u, p.v, p.w, cost, cp, sp);
    } else {                                              // pair
      const double x = pair_split((double)rnd(t, p));
      const double Tk = (double)p.E - 2.0 * kMec2;
      const double Tm = x * Tk;
      const float fTm = (float)Tm, fTp = (float)(Tk - Tm);
      t.l_pair += 2.0 * kMec2;
      emit_charged(t, st, p, GBMC_ELECTRON, fTm, p.u, p.v, p.w, vox);
      emit_charged(t, st, p, GBMC_POSITRON, fTp, p.u, p.v, p.w, vox);
      return;
    }
  }
  t.err |= E_WOODCOCK;
  t.l_esc += p.E;
}

// ---------------------------------------------------------------------------
// Charged particles: class II mixed simulation with a random hinge
// ---------------------------------------------------------------------------
struct Cell {          // voxel tracked by the DDA
  int ix, iy, iz, v;
  float rho;
};

GB_D float rinv(const Track& t, int m, int s, float r) {
  const DevProblem& P = *t.P;
  const GridPos g = grid_pos(log2f(r), P.lr0[m][s], P.inv_dr[m][s], P.nR);
  return exp2_tab(tq(t, s ? Q_RINV_P : Q_RINV_E, m), g);
}

enum { MV_OK = 0, MV_EXIT = 1, MV_MAT = 2 };

// move through mass thickness `mass`, voxel by voxel, losing energy by the
// CSDA range relation (residual range r) and scoring each voxel's share
GB_D int move_mass(Track& t, Live& p, Cell& c, float mass, float& r, int m, int s) {
  const DevProblem& P = *t.P;
  const float iu = 1.0f / p.u, iv = 1.0f / p.v, iw = 1.0f / p.w;
  float left = mass;
  for (int it = 0; it < kCapDda; ++it) {
    // distance to the exit face of the current voxel
    const float fx = (p.u > 0.0f) ? (float)(c.ix + 1) * P.dx : (float)c.ix * P.dx;
    const float fy = (p.v > 0.0f) ? (float)(c.iy + 1) * P.dy : (float)c.iy * P.dy;
    const float fz = (p.w > 0.0f) ? (float)(c.iz + 1) * P.dz : (float)c.iz * P.dz;
    const float tx = (p.u != 0.0f) ? (fx - p.x) * iu : INFINITY;
    const float ty = (p.v != 0.0f) ? (fy - p.y) * iv : INFINITY;
    const float tz = (p.w != 0.0f) ? (fz - p.z) * iw : INFINITY;
    int axis = 0;
    float d = tx;
    if (ty < d) { d = ty; axis = 1; }
    if (tz < d) { d = tz; axis = 2; }
    d = fmaxf(d, 0.0f);
    const float mf = c.rho * d;
    float mm;
    bool crossed;
    if (left <= mf) {
      mm = left;
      const float dd = left / c.rho;
      p.x = fmaf(dd, p.u, p.x); p.y = fmaf(dd, p.v, p.y); p.z = fmaf(dd, p.w, p.z);
      crossed = false;
    } else {
      mm = mf;
      p.x = fmaf(d, p.u, p.x); p.y = fmaf(d, p.v, p.y); p.z = fmaf(d, p.w, p.z);
      if (axis == 0) p.x = fx; else if (axis == 1) p.y = fy; else p.z = fz;
      crossed = true;
    }
    // CSDA loss over mm in this voxel
    r -= mm;
    float Tn = rinv(t, m, s, fmaxf(r, 1e-30f));
    Tn = fminf(Tn, p.E);
    score(t, c.v, p.E - Tn);
    p.E = Tn;
    left -= mm;
    if (!crossed) return MV_OK;
    ++t.c_cross;
    if (axis == 0) {
      c.ix += (p.u > 0.0f) ? 1 : -1;
      if (c.ix < 0 || c.ix >= P.nx) return MV_EXIT;
      c.v += (p.u > 0.0f) ? 1 : -1;
    } else if (axis == 1) {
      c.iy += (p.v > 0.0f) ? 1 : -1;
      if (c.iy < 0 || c.iy >= P.ny) return MV_EXIT;
      c.v += (p.v > 0.0f) ? P.nx : -P.nx;
    } else {
      c.iz += (p.w > 0.0f) ? 1 : -1;
      if (c.iz < 0 || c.iz >= P.nz) return MV_EXIT;
      c.v += (p.w > 0.0f) ? P.nxy : -P.nxy;
    }
    c.rho = __ldg(P.rho + c.v);
    if ((int)__ldg(P.mat + c.v) != m) return MV_MAT;
  }
  t.err |= E_DDA;
  return MV_OK;
}

GB_D float soft_mu(const Track& t, float mbar, float u) {
  if (mbar < 1e-9f) return 1.0f;
  if (mbar > 0.9999f) return 2.0f * u - 1.0f;
  const DevProblem& P = *t.P;
  const GridPos g = grid_pos(log2f(mbar / (1.0f - mbar)), P.la0, P.inv_da, P.nA);
  const float A = exp2_tab(t.tab + P.off_soft, g);
  return 1.0f - 2.0f * A * u / (1.0f + A - u);
}

GB_D float hard_sum(const Track& t, int m, int s, GridPos g) {
  return exp2_tab(tq(t, Q_SIG_EL, m), g) + exp2_tab(tq(t, s ? Q_SIG_INEL_P : Q_SIG_INEL_E, m), g) +
         exp2_tab(tq(t, Q_SIG_BR, m), g);
}

// hard elastic: element by partial hard cross section, then exact inversion
GB_D float sample_el_hard(Track& t, Live& p, const DevMat& M, float T, float xc) {
  const float tau = T / kMec2f, p2 = tau * (tau + 2.0f);
  const float b2 = p2 / ((tau + 1.0f) * (tau + 1.0f));
  const float ip2 = 1.0f / p2, ib2 = 1.0f / b2;
  float wsum = 0.0f;
#pragma unroll
  for (int i = 0; i < GBMC_MAX_EL; ++i) {
    if (i < M.n_el) {
      const float A = M.el_cA[i] * ip2 * (1.13f + M.el_cB[i] * ib2);
      wsum += M.el_w[i] * (2.0f - xc) / ((xc + 2.0f * A) * (2.0f + 2.0f * A));
    }
  }
  const float u1 = rnd(t, p), u2 = rnd(t, p);
  float c = u1 * wsum, Asel = 0.0f;
  bool found = false;
#pragma unroll
  for (int i = 0; i < GBMC_MAX_EL; ++i) {
    if (i < M.n_el && !found) {
      const float A = M.el_cA[i] * ip2 * (1.13f + M.el_cB[i] * ib2);
      const float wi = M.el_w[i] * (2.0f - xc) / ((xc + 2.0f * A) * (2.0f + 2.0f * A));
      if (c < wi || i == M.n_el - 1) { Asel = A; found = true; }
      c -= wi;
    }
  }
  const float a = 1.0f / (xc + 2.0f * Asel), D = a - 1.0f / (2.0f + 2.0f * Asel);
  const float x = 1.0f / (a - u2 * D) - 2.0f * Asel;
  return 1.0f - x;
}

// Moller energy transfer, rejection from the 1/eps^2 envelope on [wcc/T, 1/2]
GB_D float sample_moller(Track& t, Live& p, float T, float wcc) {
  const float tau = T / kMec2f;
  const float a = (tau / (tau + 1.0f)) * (tau / (tau + 1.0f));
  const float b = (2.0f * tau + 1.0f) / ((tau + 1.0f) * (tau + 1.0f));
  const float ec = wcc / T, gmax = 2.0f + 0.25f * a;
  float eps = ec;
  for (int it = 0; it < kCapReject; ++it) {
    const float u1 = rnd(t, p), u2 = rnd(t, p);
    eps = ec / (1.0f - u1 * (1.0f - 2.0f * ec));
    const float r = eps / (1.0f - eps);
    const float g = 1.0f + r * r + a * eps * eps - b * r;
    if (u2 * gmax <= g) return eps * T;
  }
  t.err |= E_REJECT;
  return eps * T;
}

GB_D void absorb_charged(Track& t, Stack& st, Live& e, int vox) {
  score(t, vox, e.E);
  e.E = 0.0f;
  if (e.type == GBMC_POSITRON) annihilate(t, st, e, vox);
}

GB_D void charged_track(Track& t, Stack& st, Live& e) {
  const DevProblem& P = *t.P;
  const int s = (e.type == GBMC_POSITRON) ? 1 : 0;
  Cell c;
  c.v = locate(P, e.x, e.y, e.z, e.u, e.v, e.w, c.ix, c.iy, c.iz);
  if (c.v < 0) { t.l_esc += e.E; return; }
  c.rho = __ldg(P.rho + c.v);
  for (int it = 0; it < kCapEsteps; ++it) {
    if (e.E <= P.eabs_e) { absorb_charged(t, st, e, c.v); return; }
    ++t.c_estep;
    const int m = __ldg(P.mat + c.v);
    const float T0 = e.E;
    const GridPos g0 = egrid(t, T0);
    const float* Rt = tq(t, s ? Q_R_P : Q_R_E, m);
    const float R0 = exp2_tab(Rt, g0);
    float Tlo = P.step_keep * T0;
    bool final = false;
    if (Tlo <= P.eabs_e) { Tlo = P.eabs_e; final = true; }
    float tmax = fmaxf(R0 - exp2_tab(Rt, egrid(t, Tlo)), 0.0f);
    const float tgeo = P.step_len * c.rho;
    if (tgeo < tmax) { tmax = tgeo; final = false; }
    const float Tend = rinv(t, m, s, R0 - tmax);
    const float smaj = fmaxf(hard_sum(t, m, s, g0), hard_sum(t, m, s, egrid(t, Tend)));
    const float u1 = rnd(t, e);
    const float th = (smaj > 0.0f) ? -logf(u1) / smaj : INFINITY;
    const bool hard = th < tmax;
    const float tstep = hard ? th : tmax;
    const float tau = rnd(t, e) * tstep;
    float r = R0;
    int mv = move_mass(t, e, c, tau, r, m, s);
    if (mv == MV_EXIT) { t.l_esc += e.E; return; }
    if (mv == MV_MAT) continue;
    // hinge: soft deflection for the whole step at the step's initial energy
    const float sig1 = exp2_tab(tq(t, Q_SIG1, m), g0);
    const float mbar = -expm1f(-tstep * sig1);
    const float mu = soft_mu(t, mbar, rnd(t, e));
    float sp, cp;
    sincospif(2.0f * rnd(t, e), &sp, &cp);
    rotate(e.u, e.v, e.w, mu, cp, sp);
    mv = move_mass(t, e, c, tstep - tau, r, m, s);
    if (mv == MV_EXIT) { t.l_esc += e.E; return; }
    if (mv == MV_MAT) continue;
    if (!hard) {
      if (final) { absorb_charged(t, st, e, c.v); return; }
      continue;
    }
    // hard event (or delta) at the current energy
    ++t.c_hard;
    const GridPos gn = egrid(t, e.E);
    const float sel = exp2_tab(tq(t, Q_SIG_EL, m), gn);
    // below their thresholds the tables hold a denormal "zero": never select
    const bool inel_ok = e.E > (s ? P.wcc : 2.0f * P.wcc);
    const float sin_ = inel_ok ? exp2_tab(tq(t, s ? Q_SIG_INEL_P : Q_SIG_INEL_E, m), gn) : 0.0f;
    const float sbr = (e.E > P.wcr) ? exp2_tab(tq(t, Q_SIG_BR, m), gn) : 0.0f;
    const float cc = rnd(t, e) * smaj;
    if (cc < sel) {
      const float xc = lerp_tab(tq(t, Q_XC, m), gn);
      const float cost = sample_el_hard(t, e, P.mats[m], e.E, xc);
      float sp2, cp2;
      sincospif(2.0f * rnd(t, e), &sp2, &cp2);
      rotate(e.u, e.v, e.w, cost, cp2, sp2);
    } else if (cc < sel + sin_) {
      const float T = e.E;
      float W;
      if (s) W = P.wcc / (1.0f - rnd(t, e) * (1.0f - P.wcc / T));
      else W = sample_moller(t, e, T, P.wcc);
      const float Tp = T - W;
      const float k2 = T + 2.0f * kMec2f;
      const float cpri = sqrtf(fminf(1.0f, (Tp / T) * k2 / (Tp + 2.0f * kMec2f)));
      const float cdel = sqrtf(fminf(1.0f, (W / T) * k2 / (W + 2.0f * kMec2f)));
      float sp2, cp2;
      sincospif(2.0f * rnd(t, e), &sp2, &cp2);
      float du = e.u, dv = e.v, dw = e.w;
      rotate(du, dv, dw, cdel, -cp2, -sp2);
      rotate(e.u, e.v, e.w, cpri, cp2, sp2);
      e.E = Tp;
      emit_charged(t, st, e, GBMC_ELECTRON, W, du, dv, dw, c.v);
    } else if (cc < sel + sin_ + sbr) {
      const float T = e.E;
      const float W = P.wcr * expf(rnd(t, e) * logf(T / P.wcr));
      e.E = T - W;
      emit_photon(t, st, e, W, c.v);
    }
  }
  t.err |= E_ESTEP;
  score(t, c.v, e.E);
}

// ---------------------------------------------------------------------------
// Primary state (Sec. 4.2.1)
// ---------------------------------------------------------------------------
GB_D void primary(const Track& t, uint32_t hist, Live& p) {
  const DevProblem& P = *t.P;
  p.type = P.particle;
  p.path = 0;
  p.nchild = 0;
  rng_init(p.rng, hist, 0, 0);
  float x = P.x0, y = P.y0;
  if (P.shape == 1) {
    x = P.x0 - P.hx + 2.0f * P.hx * rng_draw(p.rng, P.key0, P.key1);
    y = P.y0 - P.hy + 2.0f * P.hy * rng_draw(p.rng, P.key0, P.key1);
  }
  p.x = x; p.y = y; p.z = 0.0f;
  p.u = 0.0f; p.v = 0.0f; p.w = 1.0f;
  if (P.n_bins > 0) {
    const float a = rng_draw(p.rng, P.key0, P.key1), b = rng_draw(p.rng, P.key0, P.key1);
    const float xa = a * (float)P.n_bins;
    int j = min((int)xa, P.n_bins - 1);
    if (xa - (float)j >= __ldg(P.bin_prob + j)) j = __ldg(P.bin_alias + j);
    const float lo = __ldg(P.bin_edges + j), hi = __ldg(P.bin_edges + j + 1);
    p.E = fmaf(hi - lo, b, lo);
  } else {
    p.E = P.energy;
  }
}

}  // namespace gb
