// transport.cuh -- device physics of one particle: photon Woodcock flight and
// interactions, class II electron/positron steps with a random hinge and a
// voxel DDA, primary sampling, scoring. Shared by the plain kernel (secondaries
// on a per-thread stack) and the wavefront kernels (secondaries appended to
// global SoA queues): the secondary sink is a template parameter.
//
// Paper roles: JUMP / STEP / KNOCK of Sec. 4.1; primary state samplers of
// Sec. 4.2.1; LOCATE / STEP of the voxel geometry of Sec. 4.2.2; tally scoring
// of Sec. 4.2.3. FP32 stepping and sampling; FP64 for the pair split.
//
// Small deflections are carried as x = 1 - cos(theta) (or sin^2 in closed
// form) all the way into the rotation, so that angles below ~3e-4 rad, which
// binary32 cannot represent as a cosine, are not lost.
#pragma once

#include "gbmc_common.cuh"

namespace gb {

// ---------------------------------------------------------------------------
// Per-thread tracking context
// ---------------------------------------------------------------------------
// What a deposit and a tentative photon collision do (the adjoint replays a
// history twice with the same random numbers; forward kernels keep TALLY,
// which the compiler folds away):
//   TALLY:   deposit e in voxel v -> batch tile[v] += e
//   G_SUM:   deposit -> G += e w_v, w_v = g_v / (rho_v V) (g = dL/dD)
//   SCATTER: deposit -> tile[v] -= e w_v / rho_v (the explicit d(1/rho) term);
//            tentative collision in v -> tile[v] += G * (1/rho_v if real,
//            -kappa / (mbar - rho_v kappa) if virtual), the likelihood-ratio
//            score of the Woodcock acceptance
// (the TrackMode values are in gbmc_common.cuh, for the host's dispatch)
struct Track {
  const DevProblem* P;
  const float* tab_g;        // photon table region staged in shared memory (or null)
  const float* tab_e;        // charged table region staged in shared memory (or null)
  float* tile;               // batch tile of the particle being tracked
  float* pa;                 // pending deposit address (merged deposits)
  float pe;
  uint32_t c_tent, c_real, c_estep, c_cross, c_hard, c_part;
  double l_src, l_esc, l_pair;
  uint32_t err;
  const DevJob* J;           // the job of the particle being tracked
  int mode;                  // TrackMode
  bool check;                // per-history energy ledger (plain kernel, checked runs)
  bool vr;                   // weighted particles (a compile-time constant of each kernel:
                             // without variance reduction every weight is 1 and folds away)
  double l_dep;              // checked runs: energy scored so far
  const float* wv;           // adjoint: w_v per voxel
  float G;                   // adjoint: sum of e w_v over the history
};

// the particle being tracked (registers)
struct Live {
  float x, y, z, u, v, w, E;
  int type;
  int batch;                 // batch of its history within its job (< 4096)
  int job;                   // job of a batched run (0 for a single run)
  int pending;               // charged: deferred event (0 none, 1 hard inelastic, 2 hard
                             // bremsstrahlung, 3 annihilation at rest)
  int vox;                   // charged: voxel tracked by the DDA (-1 = locate)
  float r;                   // charged: residual range R(E) in the current material (< 0 = unset)
  float wt;                  // statistical weight
  uint64_t path;
  uint32_t nchild;
  Rng rng;
};

GB_D float rnd(Track& t, Live& p) { return rng_draw(p.rng, t.J->keys); }

GB_D void score_flush(Track& t) {
  if (t.pa && t.pe != 0.0f) atomicAdd(t.pa, t.pe);
  t.pa = nullptr;
  t.pe = 0.0f;
}

GB_D void score(Track& t, int v, float e) {
  if (!(e > 0.0f)) return;
  v = chk(v, (int64_t)t.J->nxy * t.J->nz, t.err);
  if (t.check) t.l_dep += (double)e;
  if (t.mode == M_G_SUM) { t.G = fmaf(e, __ldg(t.wv + v), t.G); return; }
  if (t.mode == M_SCATTER) e *= -__ldg(t.wv + v) / __ldg(t.J->rho + v);
  float* a = t.tile + v;
  if (a == t.pa) { t.pe += e; return; }
  score_flush(t);
  t.pa = a;
  t.pe = e;
}

// adjoint on the wavefront path, where a history's particles meet in
// different lanes and passes: G_h lives in P.gbuf. A particle takes it when a
// lane picks the particle up (SCATTER) and adds its deposits' share back when
// the lane lets the particle go (G_SUM).
GB_D void g_load(Track& t, uint32_t hist) {
  t.G = (t.mode == M_SCATTER) ? __ldg(t.P->gbuf + chk_u(hist - t.J->run_first, t.J->run_n, t.err)) : 0.0f;
}

GB_D void g_release(Track& t, uint32_t hist) {
  if (t.mode == M_G_SUM && t.G != 0.0f)
    atomicAdd(t.P->gbuf + chk_u(hist - t.J->run_first, t.J->run_n, t.err), t.G);
  t.G = 0.0f;
}

GB_D void set_batch(Track& t, int batch) {
  t.tile = t.J->tile + (int64_t)chk(batch, t.J->run_k, t.err) * t.J->tile_stride;
}

GB_D const float* tq(const Track& t, int q, int m) {
  return (q < Q_SIG_EL ? t.tab_g : t.tab_e) + tab_rel(q, m, t.P->n_mat, t.P->nE);
}

GB_D GridPos egrid(const Track& t, float E) {
  return grid_pos(log2f(E), t.P->lg0, t.P->inv_d, t.P->nE);
}

// history id -> batch: largest k with floor(k N / K) <= i, i = h - first
GB_D int batch_of(const DevJob& J, uint32_t hist) {
  const uint64_t i = (uint64_t)(hist - J.run_first);
  return (int)(((i + 1) * (uint64_t)J.run_k - 1) / J.run_n);
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

GB_D int locate(const DevJob& J, float x, float y, float z, float u, float v, float w,
                int& ix, int& iy, int& iz) {
  ix = locate_axis(x, u, J.idx, J.nx);
  iy = locate_axis(y, v, J.idy, J.ny);
  iz = locate_axis(z, w, J.idz, J.nz);
  if ((ix | iy | iz) < 0) return -1;
  return iz * J.nxy + iy * J.nx + ix;
}

// sine and cosine of the azimuth 2 pi u: the hardware sine/cosine of the
// reduced angle pi (2u - 1) in (-pi, pi), where their absolute error is about
// 2^-21, negated (the angle is 2 pi u - pi)
GB_D void azimuth(float u, float& sp, float& cp) {
  float s, c;
  __sincosf(3.14159265f * (2.0f * u - 1.0f), &s, &c);
  sp = -s;
  cp = -c;
}

// rotate direction by polar angle (cos, sin) and azimuth (cos phi, sin phi)
GB_D void rotate(float& u, float& v, float& w, float cost, float sint, float cp, float sp) {
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

// rotation from x = 1 - cos(theta), exact for small angles
GB_D void rotate_x(float& u, float& v, float& w, float x, float cp, float sp) {
  x = fminf(fmaxf(x, 0.0f), 2.0f);
  rotate(u, v, w, 1.0f - x, sqrtf(x * (2.0f - x)), cp, sp);
}

// rotation from sin^2(theta) given in closed form (forward hemisphere)
GB_D void rotate_s2(float& u, float& v, float& w, float sin2, float cp, float sp) {
  sin2 = fminf(fmaxf(sin2, 0.0f), 1.0f);
  rotate(u, v, w, sqrtf(1.0f - sin2), sqrtf(sin2), cp, sp);
}

// ---------------------------------------------------------------------------
// Secondaries: every particle created goes to a sink (a per-thread stack or a
// global queue); the child's stream is derived from the parent's path.
// ---------------------------------------------------------------------------
GB_D void make_child(const Live& parent, uint32_t ordinal, Particle& c, int type, float E,
                     float u, float v, float w) {
  c.x = parent.x; c.y = parent.y; c.z = parent.z;
  c.u = u; c.v = v; c.w = w; c.E = E;
  c.meta = (uint32_t)type | ((uint32_t)parent.batch << 4) | ((uint32_t)parent.job << 16);
  const uint64_t path = child_path(parent.path, ordinal);
  c.path_lo = (uint32_t)path; c.path_hi = (uint32_t)(path >> 32);
  c.hist = parent.rng.hist; c.nchild = 0; c.n = 0; c.vox = -1; c.r = -1.0f;
  c.wt = parent.wt;
}

GB_D void live_from(Live& p, const Particle& c) {
  p.x = c.x; p.y = c.y; p.z = c.z; p.u = c.u; p.v = c.v; p.w = c.w; p.E = c.E;
  p.type = (int)(c.meta & 3u);
  p.pending = (int)((c.meta >> 2) & 3u);
  p.batch = (int)((c.meta >> 4) & 0xfffu);
  p.job = (int)(c.meta >> 16);
  p.vox = c.vox;
  p.r = c.r;
  p.wt = c.wt;
  p.path = ((uint64_t)c.path_hi << 32) | c.path_lo;
  p.nchild = c.nchild;
  rng_init(p.rng, c.hist, p.path, c.n);
}

GB_D void particle_from(Particle& c, const Live& p) {
  c.x = p.x; c.y = p.y; c.z = p.z; c.u = p.u; c.v = p.v; c.w = p.w; c.E = p.E;
  c.meta = (uint32_t)p.type | ((uint32_t)p.pending << 2) | ((uint32_t)p.batch << 4) |
           ((uint32_t)p.job << 16);
  c.path_lo = (uint32_t)p.path; c.path_hi = (uint32_t)(p.path >> 32);
  c.hist = p.rng.hist; c.nchild = p.nchild; c.n = p.rng.n; c.vox = p.vox; c.r = p.r;
  c.wt = p.wt;
}

// positron at rest: two back-to-back isotropic 0.511 MeV photons
template <class Sink>
GB_D void annihilate(Track& t, Sink& sk, Live& e, int vox) {
  const float cost = 2.0f * rnd(t, e) - 1.0f;
  float sp, cp;
  azimuth(rnd(t, e), sp, cp);
  const float sint = sqrtf(fmaxf(0.0f, 1.0f - cost * cost));
  Particle g;
  make_child(e, ++e.nchild, g, GBMC_PHOTON, kMec2f, sint * cp, sint * sp, cost);
  sk.push(t, g, vox);
  make_child(e, ++e.nchild, g, GBMC_PHOTON, kMec2f, -sint * cp, -sint * sp, -cost);
  sk.push(t, g, vox);
  t.l_pair -= 2.0 * kMec2 * e.wt;
}

// a secondary made at an interaction in voxel vox: below its absorption
// energy it is scored on the spot (a positron then annihilates there),
// otherwise it goes to the sink
template <class Sink>
GB_D void emit(Track& t, Sink& sk, const Particle& c, int vox) {
  const int type = (int)(c.meta & 3u);
  const float cut = (type == GBMC_PHOTON) ? t.P->eabs_g : t.P->eabs_e;
  if (c.E < cut) {
    score(t, vox, c.E * c.wt);
    if (type == GBMC_POSITRON) {
      Live q;
      live_from(q, c);
      annihilate(t, sk, q, vox);
    }
  } else {
    sk.push(t, c, vox);
  }
}

// ---------------------------------------------------------------------------
// Photon KNOCK samplers
// ---------------------------------------------------------------------------

// Klein-Nishina, Butcher & Messel decomposition; returns eps = E'/E and
// x = 1 - cos(theta)
GB_D float sample_compton(Track& t, Live& p, float k, float& x) {
  const float e0 = 1.0f / (1.0f + 2.0f * k);
  const float a1 = log1pf(2.0f * k), a2 = 0.5f * (1.0f - e0 * e0);
  float eps = 1.0f, tt = 0.0f;
  for (int it = 0; it < kCapReject; ++it) {
    const float u1 = rnd(t, p), u2 = rnd(t, p), u3 = rnd(t, p);
    eps = (u1 * (a1 + a2) < a1) ? expf(-a1 * u2) : sqrtf(fmaf(1.0f - e0 * e0, u2, e0 * e0));
    tt = (1.0f - eps) / (k * eps);
    const float sin2 = tt * (2.0f - tt);
    const float g = 1.0f - eps * sin2 / (1.0f + eps * eps);
    if (u3 <= g) { x = tt; return eps; }
  }
  t.err |= E_REJECT;
  x = tt;
  return eps;
}

// Rayleigh: composition over elements of 1/(1 + b t)^2, rejection (1 + cos^2)/2;
// returns t = 1 - cos(theta)
GB_D float sample_rayleigh(Track& t, Live& p, const DevMat& M, float E) {
  const float k = E / kMec2f, k2 = 2.0f * k * k;
  float wsum = 0.0f;
#pragma unroll 1
  for (int i = 0; i < M.n_el; ++i) wsum += M.ray_w[i] * 2.0f / (1.0f + 2.0f * k2 * M.ray_iqz2[i]);
  float tt = 0.0f;
  for (int it = 0; it < kCapReject; ++it) {
    const float u1 = rnd(t, p), u2 = rnd(t, p), u3 = rnd(t, p);
    float c = u1 * wsum, b = 0.0f;
#pragma unroll 1
    for (int i = 0; i < M.n_el; ++i) {
      const float bi = k2 * M.ray_iqz2[i];
      const float wi = M.ray_w[i] * 2.0f / (1.0f + 2.0f * bi);
      if (c < wi || i == M.n_el - 1) { b = bi; break; }
      c -= wi;
    }
    tt = 2.0f * u2 / (1.0f + 2.0f * b * (1.0f - u2));
    if (u3 <= 0.5f * (1.0f + (1.0f - tt) * (1.0f - tt))) return tt;
  }
  t.err |= E_REJECT;
  return tt;
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
// Photon: Woodcock flight and interactions
// ---------------------------------------------------------------------------
// majorant and per-material attenuation at the photon's current energy,
// looked up again only when the energy changes
struct PhotonXs {
  float lastE = -1.0f, mbar = 1.0f, mu0 = 0.f, mu1 = 0.f, mu2 = 0.f, mu3 = 0.f;
  GridPos gp;
};

GB_D void photon_xs(const Track& t, float E, PhotonXs& xs) {
  const DevProblem& P = *t.P;
  xs.lastE = E;
  xs.gp = egrid(t, E);
  // the majorant of a batched run's job lives in global memory (per job)
  const float* maj = t.J->major;
  xs.mbar = maj ? exp2f(fmaf(xs.gp.f, __ldg(maj + xs.gp.i + 1) - __ldg(maj + xs.gp.i), __ldg(maj + xs.gp.i)))
                : exp2_tab(t.tab_g + P.off_major, xs.gp);
  xs.mu0 = exp2_tab(tq(t, Q_MU_TOT, 0), xs.gp);
  if (P.n_mat > 1) xs.mu1 = exp2_tab(tq(t, Q_MU_TOT, 1), xs.gp);
  if (P.n_mat > 2) xs.mu2 = exp2_tab(tq(t, Q_MU_TOT, 2), xs.gp);
  if (P.n_mat > 3) xs.mu3 = exp2_tab(tq(t, Q_MU_TOT, 3), xs.gp);
}

enum { PH_VIRTUAL = 0, PH_REAL = 1, PH_DEAD = 2 };

// a real collision found by a flight and not yet carried out: its voxel,
// material, attenuation and the flight block's two remaining words
struct PhotonHit {
  int vox, m;
  float mum;
  uint32_t wz, ww;
};

// One Woodcock flight (Sec. 4.2.2) to the next tentative collision. Returns
// PH_VIRTUAL (virtual collision), PH_DEAD (escaped) or PH_REAL (a real
// collision, described in h, for photon_interact).
GB_D int photon_fly(Track& t, Live& p, PhotonXs& xs, PhotonHit& h) {
  const DevJob& J = *t.J;
  if (p.E != xs.lastE) photon_xs(t, p.E, xs);
  // the flight's draws: one whole Philox block in fixed slots (distance,
  // real/virtual, interaction type, azimuth or pair split); rejection
  // samplers continue from the stream after it
  const U4 wb = rng_block(p.rng, rng_take_blocks(p.rng, 1u), J.keys);
  const float s = neg_log(word_to_uniform(wb.x)) / xs.mbar;
  p.x = fmaf(s, p.u, p.x);
  p.y = fmaf(s, p.v, p.y);
  p.z = fmaf(s, p.w, p.z);
  int ix, iy, iz;
  int vox = locate(J, p.x, p.y, p.z, p.u, p.v, p.w, ix, iy, iz);
  ++t.c_tent;
  if (vox < 0) { t.l_esc += (double)(p.E * p.wt); return PH_DEAD; }
  vox = chk(vox, (int64_t)J.nxy * J.nz, t.err);
  const int m = chk(__ldg(J.mat + vox), t.P->n_mat, t.err);
  const float rho = __ldg(J.rho + vox);
  const float mum = (m == 0) ? xs.mu0 : (m == 1) ? xs.mu1 : (m == 2) ? xs.mu2 : xs.mu3;
  const bool real = !(word_to_uniform(wb.y) * xs.mbar >= rho * mum);
  if (t.mode == M_SCATTER)
    atomicAdd(t.tile + vox, t.G * (real ? 1.0f / rho : -mum / (xs.mbar - rho * mum)));
  if (!real) return PH_VIRTUAL;
  ++t.c_real;
  h.vox = vox; h.m = m; h.mum = mum; h.wz = wb.z; h.ww = wb.w;
  return PH_REAL;
}

// The interaction of a real collision found by photon_fly (the photon has not
// moved since). Returns PH_REAL (the photon survived) or PH_DEAD (absorbed or
// converted).
template <class Sink>
GB_D int photon_interact(Track& t, Sink& sk, Live& p, const PhotonXs& xs, const PhotonHit& h) {
  const DevProblem& P = *t.P;
  const int vox = h.vox, m = h.m;
  const float mum = h.mum;
  const GridPos gp = xs.gp;
  const float co = exp2_tab(tq(t, Q_MU_CO, m), gp);
  const float pe = exp2_tab(tq(t, Q_MU_PE, m), gp);
  const float ray = exp2_tab(tq(t, Q_MU_RAY, m), gp);
  const float c = word_to_uniform(h.wz) * mum;
  Particle sec[2];
  int nsec = 0;
  bool dead = false;
  if (c < co) {                                         // Compton
    float x;
    const float k = p.E / kMec2f;
    const float eps = sample_compton(t, p, k, x);
    float sp, cp;
    azimuth(word_to_uniform(h.ww), sp, cp);
    const float E0 = p.E, E1 = eps * E0, Te = E0 - E1;
    const float u0 = p.u, v0 = p.v, w0 = p.w;
    rotate_x(p.u, p.v, p.w, x, cp, sp);
    float eu = E0 * u0 - E1 * p.u, ev = E0 * v0 - E1 * p.v, ew = E0 * w0 - E1 * p.w;
    const float n2 = eu * eu + ev * ev + ew * ew;
    if (n2 > 0.0f) { const float r = rsqrtf(n2); eu *= r; ev *= r; ew *= r; }
    else { eu = u0; ev = v0; ew = w0; }
    make_child(p, ++p.nchild, sec[nsec++], GBMC_ELECTRON, Te, eu, ev, ew);
    p.E = E1;
    if (E1 < P.eabs_g) { score(t, vox, E1 * p.wt); dead = true; }
  } else if (c < co + pe) {                             // photoelectric
    make_child(p, ++p.nchild, sec[nsec++], GBMC_ELECTRON, p.E, p.u, p.v, p.w);
    dead = true;
  } else if (c < co + pe + ray || p.E <= 2.0f * kMec2f) {  // Rayleigh
    const float x = sample_rayleigh(t, p, P.mats[m], p.E);
    float sp, cp;
    azimuth(word_to_uniform(h.ww), sp, cp);
    rotate_x(p.u, p.v, p.w, x, cp, sp);
  } else {                                              // pair
    const double xsplit = pair_split((double)word_to_uniform(h.ww));
    const double Tk = (double)p.E - 2.0 * kMec2;
    const double Tm = xsplit * Tk;
    const float fTm = (float)Tm, fTp = (float)(Tk - Tm);
    t.l_pair += 2.0 * kMec2 * p.wt;
    make_child(p, ++p.nchild, sec[nsec++], GBMC_ELECTRON, fTm, p.u, p.v, p.w);
    make_child(p, ++p.nchild, sec[nsec++], GBMC_POSITRON, fTp, p.u, p.v, p.w);
    dead = true;
  }
#pragma unroll 1
  for (int j = 0; j < nsec; ++j) emit(t, sk, sec[j], vox);
  return dead ? PH_DEAD : PH_REAL;
}

// One flight and, if the collision is real, its interaction.
template <class Sink>
GB_D int photon_flight(Track& t, Sink& sk, Live& p, PhotonXs& xs) {
  PhotonHit h;
  const int st = photon_fly(t, p, xs, h);
  return st == PH_REAL ? photon_interact(t, sk, p, xs, h) : st;
}

// Tracks a photon through at most max_real real interactions; returns true
// if it is still alive after them.
template <class Sink>
GB_D bool photon_track(Track& t, Sink& sk, Live& p, int max_real) {
  PhotonXs xs;
  int nreal = 0;
  for (int it = 0; it < kCapWoodcock; ++it) {
    const int st = photon_flight(t, sk, p, xs);
    if (st == PH_DEAD) return false;
    if (st == PH_REAL && ++nreal >= max_real) return true;
  }
  t.err |= E_WOODCOCK;
  t.l_esc += (double)(p.E * p.wt);
  return false;
}

// ---------------------------------------------------------------------------
// Charged particles: class II mixed simulation with a random hinge
// ---------------------------------------------------------------------------
struct Cell {          // voxel tracked by the DDA, with its density and material
  int ix, iy, iz, v;
  float rho;
  int m;
};

// material m's parameter block in the staged charged tables
GB_D const float* mpar(const Track& t, int m) { return t.tab_e + t.P->off_mpar + m * MP_STRIDE; }

GB_D float rinv(const Track& t, int m, int s, float r) {
  const DevProblem& P = *t.P;
  const float* mp = mpar(t, m) + 2 * s;
  const GridPos g = grid_pos(log2f(r), mp[MP_LR0_E], mp[MP_INVDR_E], P.nR);
  return exp2_tab(tq(t, s ? Q_RINV_P : Q_RINV_E, m), g);
}

enum { MV_OK = 0, MV_EXIT = 1, MV_MAT = 2 };

// move through mass thickness `mass`, voxel by voxel, losing energy by the
// CSDA range relation (residual range r) and scoring each voxel's share.
// The loss of the last piece, which ends inside a voxel, is left to the
// caller (r is reduced, p.E is not): the particle's energy is settled once per
// voxel -- at each crossing, and by the caller at the end of the step -- so
// that the hinge segment of a step that stays in one voxel takes no R^-1
// lookup (the hinge deflection uses the step's initial energy)
GB_D int move_mass(Track& t, Live& p, Cell& c, float mass, float& r, int m, int s) {
  const DevJob& J = *t.J;
  const float iu = 1.0f / p.u, iv = 1.0f / p.v, iw = 1.0f / p.w;
  float left = mass;
  for (int it = 0; it < kCapDda; ++it) {
    const float fx = (p.u > 0.0f) ? (float)(c.ix + 1) * J.dx : (float)c.ix * J.dx;
    const float fy = (p.v > 0.0f) ? (float)(c.iy + 1) * J.dy : (float)c.iy * J.dy;
    const float fz = (p.w > 0.0f) ? (float)(c.iz + 1) * J.dz : (float)c.iz * J.dz;
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
    r -= mm;
    left -= mm;
    if (!crossed) return MV_OK;
    float Tn = rinv(t, m, s, fmaxf(r, 1e-30f));
    Tn = fminf(Tn, p.E);
    score(t, c.v, (p.E - Tn) * p.wt);
    p.E = Tn;
    ++t.c_cross;
    if (axis == 0) {
      c.ix += (p.u > 0.0f) ? 1 : -1;
      if (c.ix < 0 || c.ix >= J.nx) return MV_EXIT;
      c.v += (p.u > 0.0f) ? 1 : -1;
    } else if (axis == 1) {
      c.iy += (p.v > 0.0f) ? 1 : -1;
      if (c.iy < 0 || c.iy >= J.ny) return MV_EXIT;
      c.v += (p.v > 0.0f) ? J.nx : -J.nx;
    } else {
      c.iz += (p.w > 0.0f) ? 1 : -1;
      if (c.iz < 0 || c.iz >= J.nz) return MV_EXIT;
      c.v += (p.w > 0.0f) ? J.nxy : -J.nxy;
    }
    // the DDA's running index and its coordinates name the same voxel
    chk_true(c.v == c.iz * J.nxy + c.iy * J.nx + c.ix, t.err);
    c.v = chk(c.v, (int64_t)J.nxy * J.nz, t.err);
    c.rho = __ldg(J.rho + c.v);
    c.m = chk(__ldg(J.mat + c.v), t.P->n_mat, t.err);
    if (c.m != m) return MV_MAT;
  }
  t.err |= E_DDA;
  return MV_OK;
}

// 1 - e^-x for x >= 0: the Taylor polynomial x - x^2/2 + x^3/6 below 1/64
// (relative error under x^3/24 < 2e-7), else 1 - 2^(-x log2 e)
GB_D float one_minus_exp_neg(float x) {
  if (x < 0.015625f) return x * fmaf(x, fmaf(x, 0.16666667f, -0.5f), 1.0f);
  return 1.0f - exp2f(-1.44269504f * x);
}

// soft deflection: returns x = 1 - mu of the Wentzel-shaped law with 1-<mu> = mbar
GB_D float soft_x(const Track& t, float mbar, float u) {
  if (mbar < 1e-9f) return 0.0f;
  if (mbar > 0.9999f) return 2.0f * (1.0f - u);
  const DevProblem& P = *t.P;
  const GridPos g = grid_pos(log2f(mbar / (1.0f - mbar)), P.la0, P.inv_da, P.nA);
  const float A = exp2_tab(t.tab_e + P.off_soft, g);
  return 2.0f * A * u / (1.0f + A - u);
}

// hard-event mass attenuation coefficient, the inelastic and bremsstrahlung
// parts multiplied by their forcing factors (1 without forcing, where the sum
// is exactly the unforced one)
GB_D float hard_sum(const Track& t, int m, int s, GridPos g, float fi, float fb) {
  // without forcing (analog kernels, or a particle outside the forcing
  // window): the summed table, one lookup instead of three, and the same
  // majorant as an analog run
  if (!t.vr || (fi == 1.0f && fb == 1.0f)) return exp2_tab(tq(t, s ? Q_SIG_H_P : Q_SIG_H_E, m), g);
  return exp2_tab(tq(t, Q_SIG_EL, m), g) + fi * exp2_tab(tq(t, s ? Q_SIG_INEL_P : Q_SIG_INEL_E, m), g) +
         fb * exp2_tab(tq(t, Q_SIG_BR, m), g);
}

// interaction forcing factors (inelastic, bremsstrahlung) of a charged
// particle of weight wt: the configured ones inside the weight window, else 1
GB_D void forcing(const Track& t, float wt, float& fi, float& fb) {
  const DevProblem& P = *t.P;
  if (!t.vr) { fi = fb = 1.0f; return; }
  const bool in = wt >= P.vr_wlo && wt <= P.vr_whi;
  fi = in ? P.vr_fi : 1.0f;
  fb = in ? P.vr_fb : 1.0f;
}

// hard elastic: the element from its tabulated cumulative probability at the
// energy node position gn (u1), then exact inversion of its screened
// Rutherford law above the cut xc (u2); returns x = 1 - mu
GB_D float sample_el_hard(Track& t, int m, float T, float xc, GridPos gn, float u1, float u2) {
  const DevProblem& P = *t.P;
  const float* mp = mpar(t, m);
  const int n_el = chk_true((int)mp[MP_NEL] <= GBMC_MAX_EL, t.err) ? (int)mp[MP_NEL] : 1;
  int i = 0;
  if (n_el > 1) {
    const float* cdf = t.tab_e + (int)mp[MP_OFF_EL];   // staged with the charged tables
    const int last = n_el - 1;
#pragma unroll 1
    for (; i < last; ++i) {
      const float* row = cdf + i * P.nE + gn.i;
      if (u1 < fmaf(gn.f, row[1] - row[0], row[0])) break;
    }
  }
  const float tau = T / kMec2f, p2 = tau * (tau + 2.0f);
  const float b2 = p2 / ((tau + 1.0f) * (tau + 1.0f));
  const float A = mp[MP_EL_CA + i] / p2 * (1.13f + mp[MP_EL_CB + i] / b2);
  const float a = 1.0f / (xc + 2.0f * A), D = a - 1.0f / (2.0f + 2.0f * A);
  return 1.0f / (a - u2 * D) - 2.0f * A;
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

template <class Sink>
GB_D void absorb_charged(Track& t, Sink& sk, Live& e, int vox) {
  score(t, vox, e.E * e.wt);
  e.E = 0.0f;
  if (e.type == GBMC_POSITRON) annihilate(t, sk, e, vox);
}

// hard inelastic collision (Moller / free 1/W^2 positron law) or hard
// bremsstrahlung emission at the current energy: one secondary, emitted here.
// Interaction forcing (factor f > 1): the secondary carries weight wt / f and
// the particle takes the loss and deflection with probability 1 / f, decided
// by one more draw after the event's own. Bremsstrahlung splitting: the photon
// goes out as vr_split copies of 1 / vr_split of its weight; copy k >= 1 takes
// the stream of child ordinal 2^31 + k of copy 0's path, so the particle's own
// child count -- and every other stream of the history -- is unchanged.
template <class Sink>
GB_D void knock_secondary(Track& t, Sink& sk, Live& e, bool inelastic, int vox) {
  const DevProblem& P = *t.P;
  const int s = (e.type == GBMC_POSITRON) ? 1 : 0;
  const float T = e.E;
  float fi, fb;
  forcing(t, e.wt, fi, fb);
  Particle sec;
  if (inelastic) {
    float W;
    if (s) W = P.wcc / (1.0f - rnd(t, e) * (1.0f - P.wcc / T));
    else W = sample_moller(t, e, T, P.wcc);
    const float Tp = T - W;
    // two-body kinematics, sin^2 in closed form (no cancellation):
    // sin^2 = 2 mc^2 (T - T') / (T (T' + 2 mc^2)) for the outgoing T'
    const float m2 = 2.0f * kMec2f;
    const float s2p = m2 * W / (T * (Tp + m2));
    const float s2d = m2 * Tp / (T * (W + m2));
    float sp2, cp2;
    azimuth(rnd(t, e), sp2, cp2);
    float du = e.u, dv = e.v, dw = e.w;
    rotate_s2(du, dv, dw, s2d, -cp2, -sp2);
    const bool apply = (fi == 1.0f) || (rnd(t, e) * fi < 1.0f);
    if (apply) {
      rotate_s2(e.u, e.v, e.w, s2p, cp2, sp2);
      e.E = Tp;
      e.r = -1.0f;
    }
    make_child(e, ++e.nchild, sec, GBMC_ELECTRON, W, du, dv, dw);
    sec.wt = e.wt / fi;
    emit(t, sk, sec, vox);
  } else {
    const float W = fminf(P.wcr * expf(rnd(t, e) * logf(T / P.wcr)), T);
    const bool apply = (fb == 1.0f) || (rnd(t, e) * fb < 1.0f);
    if (apply) {
      e.E = T - W;
      e.r = -1.0f;
    }
    make_child(e, ++e.nchild, sec, GBMC_PHOTON, W, e.u, e.v, e.w);
    const int ns = t.vr ? P.vr_split : 1;
    sec.wt = e.wt / fb / (float)ns;
    const uint64_t path0 = ((uint64_t)sec.path_hi << 32) | sec.path_lo;
    emit(t, sk, sec, vox);
#pragma unroll 1
    for (int k = 1; k < ns; ++k) {
      const uint64_t pk = child_path(path0, 0x80000000u + (uint32_t)k);
      sec.path_lo = (uint32_t)pk;
      sec.path_hi = (uint32_t)(pk >> 32);
      emit(t, sk, sec, vox);
    }
  }
}

// the deferred event of a charged particle (wavefront "knock" pass); returns
// true if the particle continues
template <class Sink>
GB_D bool knock(Track& t, Sink& sk, Live& e) {
  const int ev = e.pending;
  e.pending = 0;
  if (ev == 3) {                 // positron at rest (its kinetic energy is already scored)
    annihilate(t, sk, e, e.vox);
    return false;
  }
  knock_secondary(t, sk, e, ev == 1, e.vox);
  return true;
}

enum { CT_DEAD = 0, CT_ALIVE = 1, CT_DEFERRED = 2 };

// Start (or resume) a charged particle: its DDA cell from the tracked voxel,
// or by LOCATE for a new particle. Returns false if it starts outside.
GB_D bool charged_begin(Track& t, Live& e, Cell& c) {
  const DevJob& J = *t.J;
  if (e.vox >= 0) {
    // the voxel's coordinates: quotients estimated in FP32 (off by at most
    // one for any phantom side below 2^22), then made exact by integer
    // correction (loops that end for any index: the remainder moves toward
    // [0, divisor) by one divisor per turn)
    c.v = e.vox;
    int iz = min(max((int)((float)c.v * J.inv_nxy), 0), J.nz - 1);
    int rem = c.v - iz * J.nxy;
    while (rem < 0) { --iz; rem += J.nxy; }
    while (rem >= J.nxy) { ++iz; rem -= J.nxy; }
    int iy = min(max((int)((float)rem * J.inv_nx), 0), J.ny - 1);
    int ix = rem - iy * J.nx;
    while (ix < 0) { --iy; ix += J.nx; }
    while (ix >= J.nx) { ++iy; ix -= J.nx; }
    c.iz = iz; c.iy = iy; c.ix = ix;
  } else {
    c.v = locate(J, e.x, e.y, e.z, e.u, e.v, e.w, c.ix, c.iy, c.iz);
    if (c.v < 0) { t.l_esc += (double)(e.E * e.wt); return false; }
  }
  c.v = chk(c.v, (int64_t)J.nxy * J.nz, t.err);
  c.rho = __ldg(J.rho + c.v);
  c.m = chk(__ldg(J.mat + c.v), t.P->n_mat, t.err);
  return true;
}

// One class II step. Returns CT_ALIVE if the particle goes on (its tracked
// voxel kept in c), CT_DEAD if it was absorbed or left the phantom, and --
// with DEFER -- CT_DEFERRED when a hard inelastic or bremsstrahlung event, or
// a positron annihilation, is due: the event is recorded in e.pending for the
// knock pass, the stream position already past the event-type draw.
template <class Sink, bool DEFER = false>
GB_D int charged_step(Track& t, Sink& sk, Live& e, Cell& c) {
  const DevProblem& P = *t.P;
  const DevJob& J = *t.J;
  const int s = (e.type == GBMC_POSITRON) ? 1 : 0;
  if (e.E <= P.eabs_e) {
    if (DEFER && e.type == GBMC_POSITRON) {
      score(t, c.v, e.E * e.wt);
      e.E = 0.0f;
      e.pending = 3;
      e.vox = c.v;
      return CT_DEFERRED;
    }
    absorb_charged(t, sk, e, c.v);
    return CT_DEAD;
  }
  ++t.c_estep;
  // the step's draws come from two whole Philox blocks in fixed slots:
  // block b: hard distance, hinge position, soft deflection, soft azimuth;
  // block b+1 (hard events only): event type, element, elastic angle, azimuth
  const uint32_t b = rng_take_blocks(e.rng, 2u);
  const U4 w1 = rng_block(e.rng, b, J.keys);
  const int m = c.m;
  const float T0 = e.E;
  const float lT0 = log2f(T0);
  const GridPos g0 = grid_pos(lT0, P.lg0, P.inv_d, P.nE);
  const float* Rt = tq(t, s ? Q_R_P : Q_R_E, m);
  // the residual range is carried from step to step (the energy is always
  // R^-1 of it), so the table round trip R^-1(R(E)) -- not exact in FP32 --
  // is taken only after a material change or a discrete energy loss
  const float R0 = (e.r > 0.0f) ? e.r : exp2_tab(Rt, g0);
  // log2 of the step's lowest energy from log2 T0 (no second logarithm)
  const bool final0 = P.step_keep * T0 <= P.eabs_e;
  const float lTlo = final0 ? P.lg_eabs_e : lT0 + P.lg_keep;
  bool final = final0;
  float tmax = fmaxf(R0 - exp2_tab(Rt, grid_pos(lTlo, P.lg0, P.inv_d, P.nE)), 0.0f);
  const float tgeo = J.step_len * c.rho;
  if (tgeo < tmax) { tmax = tgeo; final = false; }
  // the end energy enters only through its grid position: the inverse-range
  // table holds log2 E, used as is
  const GridPos gend =
      grid_pos(lerp_tab(tq(t, s ? Q_RINV_P : Q_RINV_E, m),
                        grid_pos(log2f(R0 - tmax), mpar(t, m)[MP_LR0_E + 2 * s],
                                 mpar(t, m)[MP_INVDR_E + 2 * s], P.nR)),
               P.lg0, P.inv_d, P.nE);
  float fi, fb;
  forcing(t, e.wt, fi, fb);
  const float smaj = fmaxf(hard_sum(t, m, s, g0, fi, fb), hard_sum(t, m, s, gend, fi, fb));
  const float u1 = word_to_uniform(w1.x);
  const float th = (smaj > 0.0f) ? neg_log(u1) / smaj : INFINITY;
  const bool hard = th < tmax;
  const float tstep = hard ? th : tmax;
  const float tau = word_to_uniform(w1.y) * tstep;
  float r = R0;
  int mv = MV_OK;
  // two segments, tau before the hinge and tstep - tau after it
#pragma unroll 1
  for (int seg = 0; seg < 2; ++seg) {
    mv = move_mass(t, e, c, seg == 0 ? tau : tstep - tau, r, m, s);
    if (mv != MV_OK || seg == 1) break;
    // hinge: soft deflection for the whole step at the step's initial energy
    const float sig1 = exp2_tab(tq(t, Q_SIG1, m), g0);
    const float mbar = one_minus_exp_neg(tstep * sig1);
    const float xs = soft_x(t, mbar, word_to_uniform(w1.z));
    float sp, cp;
    azimuth(word_to_uniform(w1.w), sp, cp);
    rotate_x(e.u, e.v, e.w, xs, cp, sp);
  }
  if (mv == MV_EXIT) { t.l_esc += (double)(e.E * e.wt); return CT_DEAD; }
  if (mv == MV_MAT) { e.r = -1.0f; return CT_ALIVE; }
  {  // the loss in the voxel where the step ended
    float Tn = rinv(t, m, s, fmaxf(r, 1e-30f));
    Tn = fminf(Tn, e.E);
    score(t, c.v, (e.E - Tn) * e.wt);
    e.E = Tn;
  }
  e.r = r;
  if (!hard) {
    if (final) {
      if (DEFER && e.type == GBMC_POSITRON) {
        score(t, c.v, e.E * e.wt);
        e.E = 0.0f;
        e.pending = 3;
        e.vox = c.v;
        return CT_DEFERRED;
      }
      absorb_charged(t, sk, e, c.v);
      return CT_DEAD;
    }
    return CT_ALIVE;
  }
  // hard event (or delta) at the current energy
  ++t.c_hard;
  const GridPos gn = egrid(t, e.E);
  const float sel = exp2_tab(tq(t, Q_SIG_EL, m), gn);
  // below their thresholds the tables hold a denormal "zero": never select
  const bool inel_ok = e.E > (s ? P.wcc : 2.0f * P.wcc);
  const float sin_ = inel_ok ? fi * exp2_tab(tq(t, s ? Q_SIG_INEL_P : Q_SIG_INEL_E, m), gn) : 0.0f;
  const float sbr = (e.E > P.wcr) ? fb * exp2_tab(tq(t, Q_SIG_BR, m), gn) : 0.0f;
  const U4 w2 = rng_block(e.rng, b + 1u, J.keys);
  const float cc = word_to_uniform(w2.x) * smaj;
  if (cc < sel) {
    const float xc = lerp_tab(tq(t, Q_XC, m), gn);
    const float x = sample_el_hard(t, m, e.E, xc, gn, word_to_uniform(w2.y), word_to_uniform(w2.z));
    float sp2, cp2;
    azimuth(word_to_uniform(w2.w), sp2, cp2);
    rotate_x(e.u, e.v, e.w, x, cp2, sp2);
  } else if (cc < sel + sin_ + sbr) {
    // a hard inelastic collision or a hard bremsstrahlung emission: one
    // secondary of energy W
    const bool inel = cc < sel + sin_;
    if (DEFER) {
      e.pending = inel ? 1 : 2;
      e.vox = c.v;
      return CT_DEFERRED;
    }
    knock_secondary(t, sk, e, inel, c.v);
  }
  return CT_ALIVE;
}

// Runs at most max_steps steps (plain kernel: no budget). Returns CT_ALIVE if
// the particle is still moving after them (tracked voxel kept in e.vox).
template <class Sink, bool DEFER = false>
GB_D int charged_track(Track& t, Sink& sk, Live& e, int max_steps) {
  Cell c;
  if (!charged_begin(t, e, c)) return CT_DEAD;
  const int cap = min(max_steps, kCapEsteps);
  for (int it = 0; it < cap; ++it) {
    const int st = charged_step<Sink, DEFER>(t, sk, e, c);
    if (st != CT_ALIVE) return st;
  }
  if (max_steps < kCapEsteps) {  // step budget of this pass used up
    e.vox = c.v;
    return CT_ALIVE;
  }
  t.err |= E_ESTEP;
  score(t, c.v, e.E * e.wt);
  return CT_DEAD;
}

// ---------------------------------------------------------------------------
// Primary state (Sec. 4.2.1)
// ---------------------------------------------------------------------------
GB_D void primary(Track& t, uint32_t hist, Live& p) {
  const DevJob& J = *t.J;
  p.type = J.particle;
  p.batch = batch_of(J, hist);
  p.job = 0;
  p.pending = 0;
  p.vox = -1;
  p.r = -1.0f;
  p.wt = 1.0f;
  p.path = 0;
  p.nchild = 0;
  rng_init(p.rng, hist, 0, 0);
  float x = J.x0, y = J.y0;
  if (J.shape == 1) {
    x = J.x0 - J.hx + 2.0f * J.hx * rng_draw(p.rng, J.keys);
    y = J.y0 - J.hy + 2.0f * J.hy * rng_draw(p.rng, J.keys);
  }
  p.x = x; p.y = y; p.z = 0.0f;
  p.u = 0.0f; p.v = 0.0f; p.w = 1.0f;
  if (J.n_bins > 0) {
    const float a = rng_draw(p.rng, J.keys), b = rng_draw(p.rng, J.keys);
    const float xa = a * (float)J.n_bins;
    int j = min((int)xa, J.n_bins - 1);
    if (xa - (float)j >= __ldg(J.bin_prob + j)) j = chk(__ldg(J.bin_alias + j), J.n_bins, t.err);
    const float lo = __ldg(J.bin_edges + j), hi = __ldg(J.bin_edges + j + 1);
    p.E = fmaf(hi - lo, b, lo);
  } else {
    p.E = J.energy;
  }
}

// secondaries on a per-thread stack in local memory (the plain kernel, and
// the wavefront's drain of a run's last particles)
template <int CAP>
struct StackSink {
  Particle s[CAP];
  int sp = 0;
  __device__ __forceinline__ void push(Track& t, const Particle& c, int vox) {
    if (sp < CAP) {
      s[sp++] = c;
    } else {  // overflow: scored where it was made, flagged
      t.err |= E_STACK;
      score(t, vox, c.E * c.wt);
    }
  }
};

// run the rest of a particle's life (plain kernel: no step budget)
template <class Sink>
GB_D void track_to_death(Track& t, Sink& sk, Live& p) {
  set_batch(t, p.batch);
  ++t.c_part;
  if (p.type == GBMC_PHOTON) photon_track(t, sk, p, 1 << 30);
  else charged_track(t, sk, p, kCapEsteps);
}

}  // namespace gb
