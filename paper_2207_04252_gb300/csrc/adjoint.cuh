// Discrete adjoint of the FP64 RK2 step (reverse stage kernels).
//
// The step map E^n -> E^{n+1} at a fixed dt is differentiated as written:
// limiter branches, the wave pattern and sampling of the exact Riemann
// solution, the dust upwinding and the positivity fallback are held at the
// branch the forward values take; the star pressure's derivative follows from
// the implicit function theorem at the converged p*.  For one stage
//     Y = E_base + tau (G(E_in) - R0) / V,    E_out = D(Y)   (drag),
// a cotangent lambda_out on E_out gives mu = D'(Y)^T lambda_out on Y and on
// E_base, the weighted cotangent mu' = tau / V mu on G, and
// G'(E_in)^T mu' = sum over faces (flux part) + V S'(E_in)^T mu' (sources).
//
// Kernels:
//   adj_point_kernel  drag and source adjoints per cell, writes mu', the
//                     cotangent of E^n and the d/dSt block partials;
//   adj_flux_kernel   flux part of G'^T mu' along one axis, accumulated into
//                     the cotangent of the stage input.
// A line of L lanes along the axis owns T = L - 4 cells: lane p holds cell
// c = c0 - 2 + p, reconstructs it (gas: the conservative departures, or the
// primitive ones with RC = RECON_PRIM), solves the face below it (once per tile),
// back-propagates the face cotangent to both face states, passes the lower
// one down by a shuffle, back-propagates its own reconstruction and passes
// the neighbour contributions up and down by shuffles; every sum has a fixed
// order, so the result is deterministic.
#pragma once
#include "stage_full.cuh"

namespace rossbi {

// ------------------------------------------------------------------ forward-mode number, 6 tangents
// Tangents with respect to the primitive face states (rho_L, u_L, p_L, rho_R, u_R, p_R).
struct J6 {
  double v;
  double d[6];
};

__device__ __forceinline__ J6 jc(double v) {
  J6 r;
  r.v = v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = 0.0;
  return r;
}
__device__ __forceinline__ J6 jv(double v, int k) {
  J6 r = jc(v);
  r.d[k] = 1.0;
  return r;
}
__device__ __forceinline__ J6 operator+(const J6& a, const J6& b) {
  J6 r;
  r.v = a.v + b.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = a.d[q] + b.d[q];
  return r;
}
__device__ __forceinline__ J6 operator-(const J6& a, const J6& b) {
  J6 r;
  r.v = a.v - b.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = a.d[q] - b.d[q];
  return r;
}
__device__ __forceinline__ J6 operator*(const J6& a, const J6& b) {
  J6 r;
  r.v = a.v * b.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = a.d[q] * b.v + a.v * b.d[q];
  return r;
}
__device__ __forceinline__ J6 operator/(const J6& a, const J6& b) {
  J6 r;
  r.v = a.v / b.v;
  const double ib = 1.0 / b.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = (a.d[q] - r.v * b.d[q]) * ib;
  return r;
}
__device__ __forceinline__ J6 operator+(const J6& a, double b) {
  J6 r = a;
  r.v = a.v + b;
  return r;
}
__device__ __forceinline__ J6 operator-(const J6& a, double b) {
  J6 r = a;
  r.v = a.v - b;
  return r;
}
__device__ __forceinline__ J6 operator*(const J6& a, double b) {
  J6 r;
  r.v = a.v * b;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = a.d[q] * b;
  return r;
}
__device__ __forceinline__ J6 operator*(double a, const J6& b) {
  J6 r;
  r.v = a * b.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = a * b.d[q];
  return r;
}
__device__ __forceinline__ J6 operator/(const J6& a, double b) {
  J6 r;
  r.v = a.v / b;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = a.d[q] / b;
  return r;
}
__device__ __forceinline__ J6 operator/(double a, const J6& b) {
  J6 r;
  r.v = a / b.v;
  const double s = -r.v / b.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = s * b.d[q];
  return r;
}
__device__ __forceinline__ J6 jsqrt(const J6& a) {
  J6 r;
  r.v = sqrt(a.v);
  const double s = 0.5 / r.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = s * a.d[q];
  return r;
}
__device__ __forceinline__ J6 jpow(const J6& a, double e) {
  J6 r;
  r.v = pow(a.v, e);
  const double s = e * r.v / a.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = s * a.d[q];
  return r;
}

// a^e with its value v given (computed elsewhere, e.g. as a polynomial).
__device__ __forceinline__ J6 jpow_v(const J6& a, double e, double v) {
  J6 r;
  r.v = v;
  const double s = e * v / a.v;
#pragma unroll
  for (int q = 0; q < 6; ++q) r.d[q] = s * a.d[q];
  return r;
}

// ------------------------------------------------------------------ Riemann solution and its Jacobian
struct JSide {
  J6 rho, u, p, c;
};

// f_K(p) at a fixed p (its tangent: the partials in the side's state) and the
// value of df_K/dp; the value arithmetic is that of pressure_fn.
// G75 (gamma = 7/5): zK = (p / p_K)^(1/7) is given.
template <bool G75>
__device__ __forceinline__ void pressure_fn_jac(double g, const JSide& K, double p, J6& f, double& fd, double zK) {
  if (p <= K.p.v) {
    const J6 prat = jc(p) / K.p;
    const J6 e = G75 ? jpow_v(prat, 1.0 / 7.0, zK) : jpow(prat, (g - 1.0) / (2.0 * g));
    f = 2.0 * K.c / (g - 1.0) * (e - 1.0);
    fd = e.v / (prat.v * K.rho.v * K.c.v);
  } else {
    const J6 A = 2.0 / ((g + 1.0) * K.rho);
    const J6 B = (g - 1.0) / (g + 1.0) * K.p;
    const J6 q = jsqrt(A / (B + p));
    f = (jc(p) - K.p) * q;
    fd = (1.0 - 0.5 * (p - K.p.v) / (B.v + p)) * q.v;
  }
}

template <bool G75>
__device__ __forceinline__ void fan_jac(double g, const JSide& K, double sgn, J6& rho, J6& u, J6& p) {
  const J6 cf = 2.0 / (g + 1.0) * (K.c + sgn * 0.5 * (g - 1.0) * K.u);
  u = sgn * cf;
  const J6 ratio = cf / K.c;
  if (G75) {  // exponents 5 and 7
    const double r = ratio.v, r2 = r * r, r5 = r2 * r2 * r;
    rho = K.rho * jpow_v(ratio, 5.0, r5);
    p = K.p * jpow_v(ratio, 7.0, r5 * r2);
  } else {
    rho = K.rho * jpow(ratio, 2.0 / (g - 1.0));
    p = K.p * jpow(ratio, 2.0 * g / (g - 1.0));
  }
}

// The face state of riemann_face (riemann_face_g75 for G75) together with its
// Jacobian in the six primitive inputs.  Branch decisions are taken on the
// same values; for gamma = 7/5 the powers come from z = (p/p_L)^(1/7) as in
// the forward solver.
template <bool G75>
__device__ __noinline__ int riemann_jac(double g, double rl, double ul, double pl, double rr, double ur, double pr,
                                        J6& rho, J6& u, J6& p, unsigned& status) {
  const JSide L{jv(rl, 0), jv(ul, 1), jv(pl, 2), jsqrt(g * jv(pl, 2) / jv(rl, 0))};
  const JSide R{jv(rr, 3), jv(ur, 4), jv(pr, 5), jsqrt(g * jv(pr, 5) / jv(rr, 3))};
  const double cl = L.c.v, cr = R.c.v;
  if (2.0 / (g - 1.0) * (cl + cr) <= ur - ul) {  // vacuum
    const double sl_star = ul + 2.0 * cl / (g - 1.0);
    const double sr_star = ur - 2.0 * cr / (g - 1.0);
    if (0.0 <= sl_star) {
      if (0.0 <= ul - cl) { rho = L.rho; u = L.u; p = L.p; }
      else fan_jac<G75>(g, L, 1.0, rho, u, p);
      return -1;
    }
    if (0.0 >= sr_star) {
      if (0.0 >= ur + cr) { rho = R.rho; u = R.u; p = R.p; }
      else fan_jac<G75>(g, R, -1.0, rho, u, p);
      return 1;
    }
    rho = u = p = jc(0.0);
    return 0;
  }
  // Newton on the star pressure, values only (same arithmetic as the forward)
  const RSide Lv{rl, ul, pl, cl}, Rv{rr, ur, pr, cr};
  const double pfloor = 1e-8 * fmin(pl, pr);
  double ps = fmax(pfloor, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (cl + cr));
  bool conv = false;
  double zl = 0.0, zr = 0.0;
  if (G75) {
    const double k = root7(pl / pr);
    double z = root7(ps / pl);
    double fl, fdl, fr, fdr, step;
    conv = newton_z_g75(Lv, Rv, ur - ul, pfloor, k, ps, z, fl, fdl, fr, fdr, step);  // the forward's iteration
    zl = z;
    zr = z * k;
  } else {
    for (int it = 0; it < 100; ++it) {
      double fl, fdl, fr, fdr;
      pressure_fn(g, Lv, ps, fl, fdl);
      pressure_fn(g, Rv, ps, fr, fdr);
      const double pn = fmax(pfloor, ps - (fl + fr + ur - ul) / (fdl + fdr));
      const double change = 2.0 * fabs(pn - ps) / (pn + ps);
      ps = pn;
      if (change <= 1e-12) { conv = true; break; }
    }
  }
  if (!conv) status |= STATUS_RIEMANN;
  // implicit function theorem: f_L(p*) + f_R(p*) + u_R - u_L = 0
  J6 FL, FR;
  double dl, dr;
  pressure_fn_jac<G75>(g, L, ps, FL, dl, zl);
  pressure_fn_jac<G75>(g, R, ps, FR, dr, zr);
  J6 PS = jc(ps);
  if (ps == pfloor) {
    PS = 1e-8 * (pl <= pr ? L.p : R.p);
  } else {
    const double iD = -1.0 / (dl + dr);
#pragma unroll
    for (int q = 0; q < 6; ++q) PS.d[q] = (FL.d[q] + FR.d[q] + R.u.d[q] - L.u.d[q]) * iD;
  }
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    FL.d[q] += dl * PS.d[q];
    FR.d[q] += dr * PS.d[q];
  }
  const J6 US = 0.5 * (L.u + R.u) + 0.5 * (FR - FL);
  if (0.0 <= US.v) {
    if (ps <= pl) {
      if (0.0 <= ul - cl) { rho = L.rho; u = L.u; p = L.p; return -1; }
      const J6 ratio = PS / L.p;
      if (0.0 > US.v - cl * (G75 ? zl : pow(ratio.v, (g - 1.0) / (2.0 * g)))) {
        if (G75) {
          const double z2 = zl * zl;
          rho = L.rho * jpow_v(ratio, 5.0 / 7.0, z2 * z2 * zl);
        } else {
          rho = L.rho * jpow(ratio, 1.0 / g);
        }
        u = US; p = PS; return -1;
      }
      fan_jac<G75>(g, L, 1.0, rho, u, p);
      return -1;
    }
    const J6 ratio = PS / L.p;
    if (0.0 <= ul - cl * sqrt((g + 1.0) / (2.0 * g) * ratio.v + (g - 1.0) / (2.0 * g))) {
      rho = L.rho; u = L.u; p = L.p; return -1;
    }
    const double g6 = (g - 1.0) / (g + 1.0);
    rho = L.rho * (ratio + g6) / (ratio * g6 + 1.0); u = US; p = PS;
    return -1;
  }
  if (ps > pr) {
    const J6 ratio = PS / R.p;
    if (0.0 >= ur + cr * sqrt((g + 1.0) / (2.0 * g) * ratio.v + (g - 1.0) / (2.0 * g))) {
      rho = R.rho; u = R.u; p = R.p; return 1;
    }
    const double g6 = (g - 1.0) / (g + 1.0);
    rho = R.rho * (ratio + g6) / (ratio * g6 + 1.0); u = US; p = PS;
    return 1;
  }
  if (0.0 >= ur + cr) { rho = R.rho; u = R.u; p = R.p; return 1; }
  const J6 ratio = PS / R.p;
  if (0.0 <= US.v + cr * (G75 ? zr : pow(ratio.v, (g - 1.0) / (2.0 * g)))) {
    if (G75) {
      const double z2 = zr * zr;
      rho = R.rho * jpow_v(ratio, 5.0 / 7.0, z2 * z2 * zr);
    } else {
      rho = R.rho * jpow(ratio, 1.0 / g);
    }
    u = US; p = PS; return 1;
  }
  fan_jac<G75>(g, R, -1.0, rho, u, p);
  return 1;
}

// ------------------------------------------------------------------ face flux adjoints
// Cotangents of the primitive face states (u, v, w, P, rho in the field
// slots) for a cotangent Fb on the gas flux gas_face_flux<D>(WL, WR).
template <int D>
__device__ __noinline__ void gas_flux_vjp(double g, const double* WL, const double* WR, const double* Fb, double* WLb,
                                          double* WRb, unsigned& status) {
  constexpr int n = Axes<D>::n, t1 = Axes<D>::t1, t2 = Axes<D>::t2;
#pragma unroll
  for (int f = 0; f < 5; ++f) WLb[f] = WRb[f] = 0.0;
  const double rl = WL[RHO], rr = WR[RHO], pl = WL[EN], pr = WR[EN];
  if (!(rl > 0.0) || !(rr > 0.0) || !(pl > 0.0) || !(pr > 0.0)) return;  // zero flux
  J6 Rs, Us, Ps;
  const int side = g == 1.4 ? riemann_jac<true>(g, rl, WL[n], pl, rr, WR[n], pr, Rs, Us, Ps, status)
                            : riemann_jac<false>(g, rl, WL[n], pl, rr, WR[n], pr, Rs, Us, Ps, status);
  double ut1 = 0.0, ut2 = 0.0;
  if (side < 0) { ut1 = WL[t1]; ut2 = WL[t2]; }
  else if (side > 0) { ut1 = WR[t1]; ut2 = WR[t2]; }
  const double rho = Rs.v, u = Us.v, p = Ps.v;
  const double m = rho * u;
  const double K = 0.5 * (u * u + ut1 * ut1 + ut2 * ut2);
  const double H = rho * K + p / (g - 1.0) + p;
  const double FE = Fb[EN];
  // F = (m, m u + p, m ut1, m ut2, H u) in (RHO, n, t1, t2, EN)
  const double mb = Fb[RHO] + Fb[n] * u + Fb[t1] * ut1 + Fb[t2] * ut2;
  const double ub = Fb[n] * m + FE * (H + u * rho * u) + mb * rho;
  const double rb = FE * u * K + mb * u;
  const double pb = Fb[n] + FE * u * (1.0 / (g - 1.0) + 1.0);
  const double ut1b = Fb[t1] * m + FE * u * rho * ut1;
  const double ut2b = Fb[t2] * m + FE * u * rho * ut2;
  double w[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) w[q] = rb * Rs.d[q] + ub * Us.d[q] + pb * Ps.d[q];
  WLb[RHO] = w[0];
  WLb[n] = w[1];
  WLb[EN] = w[2];
  WRb[RHO] = w[3];
  WRb[n] = w[4];
  WRb[EN] = w[5];
  if (side < 0) {
    WLb[t1] = ut1b;
    WLb[t2] = ut2b;
  } else if (side > 0) {
    WRb[t1] = ut1b;
    WRb[t2] = ut2b;
  }
}

// Cotangents of the dust face primitives (u, v, w, rho_d) for a cotangent Fb
// (dust order: momenta 0..2, mass 3) on dust_kinetic_flux<D>(WL, WR).
template <int D>
__device__ __forceinline__ void dust_flux_vjp(const double* WL, const double* WR, const double* Fb, double* WLb,
                                              double* WRb) {
  constexpr int n = Axes<D>::n, t1 = Axes<D>::t1, t2 = Axes<D>::t2;
  const double ml = WL[3] * (WL[n] > 0.0 ? WL[n] : 0.0);
  const double mr = WR[3] * (WR[n] < 0.0 ? WR[n] : 0.0);
  const double mlb = Fb[3] + Fb[n] * WL[n] + Fb[t1] * WL[t1] + Fb[t2] * WL[t2];
  const double mrb = Fb[3] + Fb[n] * WR[n] + Fb[t1] * WR[t1] + Fb[t2] * WR[t2];
  WLb[3] = 0.0;
  WRb[3] = 0.0;
  WLb[n] = Fb[n] * ml;
  WLb[t1] = Fb[t1] * ml;
  WLb[t2] = Fb[t2] * ml;
  WRb[n] = Fb[n] * mr;
  WRb[t1] = Fb[t1] * mr;
  WRb[t2] = Fb[t2] * mr;
  if (WL[n] > 0.0) {
    WLb[3] += mlb * WL[n];
    WLb[n] += mlb * WL[3];
  }
  if (WR[n] < 0.0) {
    WRb[3] += mrb * WR[n];
    WRb[n] += mrb * WR[3];
  }
}

// ------------------------------------------------------------------ reconstruction adjoint
// Cotangents (bm, b0, bp) of the three cell deviations for cotangents gm, gp
// on the face values qm, qp of parabola(em, e0, ep, w); branches of the
// forward values.
__device__ __forceinline__ void parabola_vjp(double em, double e0, double ep, const double* w, double gm, double gp,
                                             double& bm, double& b0, double& bp) {
  const double sm = (e0 - em) * w[0];
  const double sp = (ep - e0) * w[1];
  const double s = minmod(sm, sp);
  const double a = (sp - sm) * w[2];
  const double b = (sp * w[3] + sm * w[4]) * w[2];
  double ab = 0.0, bb = 0.0, sb = 0.0;
  {
    const double A = w[5] * (a * w[5] + b), B = s * w[7];
    if (A * B > 0.0) {
      if (fabs(A) < fabs(B)) { ab += gm * w[5] * w[5]; bb += gm * w[5]; }
      else sb += gm * w[7];
    }
  }
  {
    const double A = w[6] * (a * w[6] + b), B = s * w[8];
    if (A * B > 0.0) {
      if (fabs(A) < fabs(B)) { ab += gp * w[6] * w[6]; bb += gp * w[6]; }
      else sb += gp * w[8];
    }
  }
  double smb = -ab * w[2] + bb * w[4] * w[2];
  double spb = ab * w[2] + bb * w[3] * w[2];
  if (sm * sp > 0.0) {
    if (fabs(sm) < fabs(sp)) smb += sb;
    else spb += sb;
  }
  bm = -smb * w[0];
  bp = spb * w[1];
  b0 = gm + gp + smb * w[0] - spb * w[1];
}

// ------------------------------------------------------------------ drag and source adjoints
// Cotangent li of the drag input U (pre-drag state) for a cotangent lo of its
// output (apply_drag over tau); returns lo . dD/dSt.
__device__ __forceinline__ double drag_vjp(const DevGrid& g, int i, const double* U, const double* lo, double* li,
                                           double tau, const DragArgs& d) {
#pragma unroll
  for (int f = 0; f < 9; ++f) li[f] = lo[f];
  const double rg = U[RHO], rd = U[DRHO];
  if (!(rd > 0.0) || !(rg > 0.0)) return 0.0;
  double ts, cs = 0.0;
  bool stokes_regime = false;  // drag law 2 above r_p = 9 lambda / 4 (the forward's branch)
  if (d.law == 0) {
    if (g.geom == GEOM_CYL) {
      const double r = g.rc[i + GH];
      ts = d.stokes / sqrt(g.gm / (r * r * r));
    } else {
      ts = d.stokes;
    }
  } else {
    cs = sqrt(g.gamma * gas_pressure(g.gamma, U[MU], U[MV], U[MW], U[EN], rg) / rg);
    ts = d.rhos_rp / (rg * cs);
    stokes_regime = d.law == 2 && d.kappa * rg > 2.25;
    if (stokes_regime) ts = ts * ((4.0 / 9.0) * (d.kappa * rg));
  }
  const double kk = tau * (1.0 + rd / rg) / ts;
  const double mu = rg * rd / (rg + rd);
  const double relax = kk / (1.0 + kk);
  const double K = mu * relax;
  const double e = lo[EN];
  double Kb = 0.0, rgb = 0.0, rdb = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double vg = U[MU + c] / rg;
    const double vd = U[DMU + c] / rd;
    const double dv = vd - vg;
    const double X = mu * dv * relax;
    const double ugp = U[MU + c] + X;
    const double dE = 0.5 * X * (ugp / rg + vg);
    const double Xb = lo[MU + c] - lo[DMU + c] + e * ugp / rg;
    li[MU + c] += e * X / rg;
    rgb -= e * dE / rg;
    Kb += Xb * dv;
    const double dvb = Xb * K;
    li[DMU + c] += dvb / rd;
    rdb -= dvb * vd / rd;
    li[MU + c] -= dvb / rg;
    rgb += dvb * vg / rg;
  }
  const double mub = Kb * relax;
  const double relaxb = Kb * mu;
  const double kkb = relaxb / ((1.0 + kk) * (1.0 + kk));
  const double s = rg + rd;
  rgb += mub * rd * rd / (s * s);
  rdb += mub * rg * rg / (s * s);
  rdb += kkb * tau / (rg * ts);
  rgb -= kkb * tau * rd / (rg * rg * ts);
  const double tsb = -kkb * kk / ts;
  if (d.law == 1 || d.law == 2) {
    // t_s = rhos_rp / (rho_g c_s), c_s = sqrt(gamma P / rho_g); in the Stokes
    // regime t_s = (4/9) kappa rhos_rp / c_s, with no explicit rho_g
    if (!stokes_regime) rgb -= tsb * ts / rg;
    const double csb = -tsb * ts / cs;
    const double Pb = csb * g.gamma / (2.0 * cs * rg);
    rgb -= csb * cs / (2.0 * rg);
    const double gm1 = g.gamma - 1.0;
    li[EN] += Pb * gm1;
    double k2 = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double v = U[MU + c] / rg;
      li[MU + c] -= Pb * gm1 * v;
      k2 += v * v;
    }
    rgb += Pb * gm1 * 0.5 * k2;
  }
  li[RHO] += rgb;
  li[DRHO] += rdb;
  return tsb * ts / d.stokes;  // t_s is proportional to St in every law
}

// out += s S'(U)^T for the App. B sources at a cell (cylindrical only).
__device__ __forceinline__ void sources_vjp(const DevGrid& g, int i, int k, const double* U, const double* s,
                                            double* out) {
  const double r = g.rc[i + GH];
  const double z = g.x0[2] + (k + 0.5) * g.dx[2];
  const double R2 = r * r + z * z;
  const double R3 = R2 * sqrt(R2);
  const double fr = -g.gm * r / R3, fz = -g.gm * z / R3;
  const double Om = g.omega;
  const double A1 = fr + Om * Om * r;
  const double gm1 = g.gamma - 1.0;
  {
    const double ir = 1.0 / U[RHO];
    const double u = U[MU] * ir, v = U[MV] * ir, w = U[MW] * ir;
    out[MU] += s[MU] * (-gm1 * u / r) + s[MV] * (-v / r - 2.0 * Om) + s[EN] * A1;
    out[MV] += s[MU] * (2.0 * v / r + 2.0 * Om - gm1 * v / r) + s[MV] * (-u / r);
    out[MW] += s[MU] * (-gm1 * w / r) + s[EN] * fz;
    out[EN] += s[MU] * gm1 / r;
    out[RHO] += s[MU] * (-v * v / r + gm1 * 0.5 * (u * u + v * v + w * w) / r + A1) + s[MV] * (u * v / r) + s[MW] * fz;
  }
  if (g.nf > 5 && U[DRHO] > 0.0) {
    const double ir = 1.0 / U[DRHO];
    const double u = U[DMU] * ir, v = U[DMV] * ir;
    out[DMU] += s[DMV] * (-v / r - 2.0 * Om);
    out[DMV] += s[DMU] * (2.0 * v / r + 2.0 * Om) + s[DMV] * (-u / r);
    out[DRHO] += s[DMU] * (-v * v / r + A1) + s[DMV] * (u * v / r) + s[DMW] * fz;
  }
}

// ------------------------------------------------------------------ kernels
struct AdjPointArgs {
  DevGrid g;
  const double* Y[9];      // pre-drag stage output
  const double* lout[9];   // cotangent of the stage output
  const double* Ein[9];    // stage input (the sources are evaluated on it)
  double* M[9];            // out: mu' = tau / V mu
  double* lam_n[9];        // cotangent of E^n: written in stage 2, accumulated in stage 1
  double* lam_in[9];       // stage 2: cotangent of E*, written (stage 1: unused)
  double tau;
  DragArgs drag;
  int stage2;
  double* partials;        // [gridDim.x] block sums of lambda_out . dD/dSt
  double* ind_partials;    // indirect gravity on: [2][gridDim.x] block sums of dJ/dA, dJ/dB (without X_ref)
};

constexpr int ADJ_PT_NT = 256;

template <int NF>
__global__ void __launch_bounds__(ADJ_PT_NT) adj_point_kernel(const AdjPointArgs a) {
  __shared__ double red[ADJ_PT_NT / 32];
  const DevGrid& g = a.g;
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  double dst = 0.0;
  double pa = 0.0, pb = 0.0;  // indirect gravity: cotangents of A_disc, B_disc (over X_ref)
  for (size_t lin = blockIdx.x * (size_t)ADJ_PT_NT + threadIdx.x; lin < ncell; lin += (size_t)gridDim.x * ADJ_PT_NT) {
    const int gi = (int)(lin % g.nr);
    const int gk = (int)(lin / ((size_t)g.nr * g.nth));
    double lo[9], mu[9], U[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) lo[f] = U[f] = 0.0;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      lo[f] = a.lout[f][lin];
      U[f] = a.Y[f][lin];
    }
    if (NF == 9) {
      dst += drag_vjp(g, gi, U, lo, mu, a.tau, a.drag);
    } else {
#pragma unroll
      for (int f = 0; f < 9; ++f) mu[f] = lo[f];
    }
    const double iv = g.ivol[gi];
    double src[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) src[f] = 0.0;
    if (g.geom == GEOM_CYL) {
      double E[9], s[9];
#pragma unroll
      for (int f = 0; f < 9; ++f) {
        E[f] = f < NF ? a.Ein[f][lin] : 0.0;
        s[f] = a.tau * mu[f];
      }
      sources_vjp(g, gi, gk, E, s, src);
      if (g.damp_k) {  // wave-killing zones: d(-V k E'_f)/dE_f = -V k
        const double kd = g.damp_k[(size_t)gk * g.nr + gi];
#pragma unroll
        for (int f = 0; f < 5; ++f) src[f] -= kd * s[f];
      }
      if (g.x_ind != 0.0) {
        // indirect gravity, S = -(rho gr, rho gt, 0, m_u gr + m_v gt) and
        // -(rho_d gr, rho_d gt, 0) for dust: its local part at fixed
        // (gr, gt), and P = dJ/dgr, Q = dJ/dgt, which reach A and B through
        // gr = X (A c + B s), gt = X (-A s + B c)
        const int gj = (int)((lin / g.nr) % g.nth);
        const double gr = g.ind_g[gj], gt = g.ind_g[g.nth + gj];
        src[RHO] -= s[MU] * gr + s[MV] * gt;
        src[MU] -= s[EN] * gr;
        src[MV] -= s[EN] * gt;
        double P = -(s[MU] * E[RHO] + s[EN] * E[MU]);
        double Q = -(s[MV] * E[RHO] + s[EN] * E[MV]);
        if (NF == 9 && E[DRHO] > 0.0) {
          src[DRHO] -= s[DMU] * gr + s[DMV] * gt;
          P -= s[DMU] * E[DRHO];
          Q -= s[DMV] * E[DRHO];
        }
        const double c = g.ind_cs[gj], sn = g.ind_cs[g.nth + gj];
        pa += P * c - Q * sn;
        pb += P * sn + Q * c;
      }
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      a.M[f][lin] = a.tau * iv * mu[f];
      if (a.stage2) {
        a.lam_n[f][lin] = mu[f];
        a.lam_in[f][lin] = src[f];
      } else {
        a.lam_n[f][lin] += mu[f] + src[f];
      }
    }
  }
  const double t = block_sum<ADJ_PT_NT>(dst, red);
  if (threadIdx.x == 0) a.partials[blockIdx.x] = t;
  if (g.x_ind != 0.0) {
    const double ta = block_sum<ADJ_PT_NT>(pa, red);
    const double tb = block_sum<ADJ_PT_NT>(pb, red);
    if (threadIdx.x == 0) {
      a.ind_partials[blockIdx.x] = ta;
      a.ind_partials[gridDim.x + blockIdx.x] = tb;
    }
  }
}

// The cotangent that reaches the stage input through the disc moments:
// A = sum w (rho - rho_0 + rho_d) cos(theta), B likewise with sin, so
// lam[RHO] and lam[DRHO] gain X_ref w (dA cos(theta_j) + dB sin(theta_j)),
// (dA, dB) the reduced point-kernel partials; w = V r / R^3 [nz][nr].
static __global__ void __launch_bounds__(ADJ_PT_NT) adj_indirect_bcast_kernel(const DevGrid g, const double* w,
                                                                       const double* dAB, double* lam_rho,
                                                                       double* lam_drho) {
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  const double dA = g.x_ind * dAB[0], dB = g.x_ind * dAB[1];
  for (size_t lin = blockIdx.x * (size_t)ADJ_PT_NT + threadIdx.x; lin < ncell; lin += (size_t)gridDim.x * ADJ_PT_NT) {
    const int i = (int)(lin % g.nr);
    const size_t jk = lin / g.nr;
    const int j = (int)(jk % g.nth), k = (int)(jk / g.nth);
    const double v = w[(size_t)k * g.nr + i] * (dA * g.ind_cs[j] + dB * g.ind_cs[g.nth + j]);
    lam_rho[lin] += v;
    if (lam_drho) lam_drho[lin] += v;
  }
}

struct AdjFluxArgs {
  DevGrid g;
  const double* E[9];      // stage input state (full)
  const double* M[9];      // mu'
  double* lam[9];          // += flux part of G'(E)^T mu'
  unsigned* status;
};

// Shared memory of adj_flux_kernel in doubles.
template <int NF, int L, int NL>
constexpr size_t adj_flux_smem_doubles() {
  return (size_t)NF * ((L + 2) + L) * (NL + 1);
}

template <int NF, int D, int L, int NL, int RC>
__global__ void __launch_bounds__(L * NL, 1) adj_flux_kernel(const AdjFluxArgs a) {
  constexpr int T = L - 4;      // cells per line owned by a block
  constexpr int PE = T + 6;     // staged E': cells c0 - 3 .. c0 + T + 2
  constexpr int PM = T + 4;     // staged mu': cells c0 - 2 .. c0 + T + 1
  constexpr int NLP = NL + 1;   // padded line stride
  constexpr int NT = L * NL;
  constexpr unsigned FULL = 0xffffffffu;
  static_assert(L <= 32 && (32 % L) == 0, "a line must fit a warp");
  extern __shared__ double smem[];
  double* sE = smem;
  double* sM = smem + (size_t)NF * PE * NLP;
  const DevGrid& g = a.g;
  const int nd = D == 0 ? g.nr : (D == 1 ? g.nth : g.nz);
  const int na = D == 0 ? g.nth : g.nr;                  // fastest transverse extent
  const int nlines = D == 0 ? g.nth * g.nz : (D == 1 ? g.nr * g.nz : g.nr * g.nth);
  const int ntiles = (nd + T - 1) / T;
  const int c0 = (blockIdx.x % ntiles) * T;
  const int line0 = (blockIdx.x / ntiles) * NL;
  const bool periodic = g.bc_lo[D] == BC_PERIODIC;
  auto cell_of = [&](int line, int cd, int c[3]) {
    const int ta = line % na, tb = line / na;
    c[0] = D == 0 ? cd : ta;
    c[1] = D == 1 ? cd : (D == 0 ? ta : tb);
    c[2] = D == 2 ? cd : tb;
  };

  for (int idx = threadIdx.x; idx < PE * NL; idx += NT) {
    const int pos = D == 0 ? idx % PE : idx / NL;
    const int l = D == 0 ? idx / PE : idx % NL;
    const int line = line0 + l;
    double* dst = sE + pos * NLP + l;
    int c[3];
    cell_of(line, c0 - 3 + pos, c);
    if (line >= nlines || !resolve_cell(g, c)) {
#pragma unroll
      for (int f = 0; f < NF; ++f) dst[(size_t)f * PE * NLP] = 0.0;
      continue;
    }
    const size_t lin = ((size_t)c[2] * g.nth + c[1]) * g.nr + c[0];
    double U[5], W[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) U[f] = a.E[f][lin];
    if (RC == RECON_PRIM) gas_prim(g.gamma, U, W);
    const double* e0 = RC == RECON_PRIM ? g.w0c : g.e0c;
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const double v = RC == RECON_PRIM ? W[f] : U[f];
      dst[(size_t)f * PE * NLP] = g.has_eq ? v - e0[((size_t)f * g.nz + c[2]) * g.nr + c[0]] : v;
    }
#pragma unroll
    for (int f = 5; f < NF; ++f) dst[(size_t)f * PE * NLP] = a.E[f][lin];
  }
  for (int idx = threadIdx.x; idx < PM * NL; idx += NT) {
    const int pos = D == 0 ? idx % PM : idx / NL;
    const int l = D == 0 ? idx / PM : idx % NL;
    const int line = line0 + l;
    double* dst = sM + pos * NLP + l;
    int cd = c0 - 2 + pos;
    bool ok = line < nlines;
    if (cd < 0 || cd >= nd) {
      if (periodic) {
        cd %= nd;
        if (cd < 0) cd += nd;
      } else {
        ok = false;  // no cell: faces beyond the domain carry no cotangent
      }
    }
    if (!ok) {
#pragma unroll
      for (int f = 0; f < NF; ++f) dst[(size_t)f * PM * NLP] = 0.0;
      continue;
    }
    int c[3];
    cell_of(line, cd, c);
    const size_t lin = ((size_t)c[2] * g.nth + c[1]) * g.nr + c[0];
#pragma unroll
    for (int f = 0; f < NF; ++f) dst[(size_t)f * PM * NLP] = a.M[f][lin];
  }
  __syncthreads();

  const int p = threadIdx.x % L, l = threadIdx.x / L;
  const int line = line0 + l;
  const bool line_ok = line < nlines;
  const int c = c0 - 2 + p;
  int cc[3];
  cell_of(line_ok ? line : 0, c, cc);
  const int gi = cc[0], gk = cc[2];
  const int ci = clampi(gi, 0, g.nr - 1), ck = clampi(gk, 0, g.nz - 1);
  const double gam = g.gamma;
  unsigned status = 0;
  auto sv = [&](int f, int q) -> double { return sE[((size_t)f * PE + q) * NLP + l]; };
  auto sm = [&](int f, int q) -> double { return sM[((size_t)f * PM + q) * NLP + l]; };
  // equilibrium on a face: conservative, or primitive with RC = RECON_PRIM
  auto eq_face = [&](int f, int fd) -> double {
    if (!g.has_eq) return 0.0;
    const double* tc = RC == RECON_PRIM ? g.w0c : g.e0c;
    const double* tr = RC == RECON_PRIM ? g.w0r : g.e0r;
    const double* tz = RC == RECON_PRIM ? g.w0z : g.e0z;
    if (D == 0) return tr[((size_t)f * g.nz + ck) * (g.nr + 1) + clampi(fd, 0, g.nr)];
    if (D == 1) return tc[((size_t)f * g.nz + ck) * g.nr + ci];
    return tz[((size_t)f * (g.nz + 1) + clampi(fd, 0, g.nz)) * g.nr + ci];
  };
  double w[9];
  parabola_weights<double, D>(g.rcoef, gi, g.nr, g.dx[D], w);

  // ---- forward reconstruction of this lane's cell
  double qm[5], qp[5];
  bool shaped = false;
#pragma unroll
  for (int f = 0; f < 5; ++f) shaped |= parabola(sv(f, p), sv(f, p + 1), sv(f, p + 2), w, qm[f], qp[f]);
  bool fallback = false;
  if (shaped && line_ok) {
    if (RC == RECON_PRIM) {
      fallback = !(eq_face(RHO, c) + qm[RHO] > 0.0 && eq_face(RHO, c + 1) + qp[RHO] > 0.0 &&
                   eq_face(EN, c) + qm[EN] > 0.0 && eq_face(EN, c + 1) + qp[EN] > 0.0);
    } else {
      double Um[5], Up[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        Um[f] = eq_face(f, c) + qm[f];
        Up[f] = eq_face(f, c + 1) + qp[f];
      }
      double Wm[5], Wp[5];  // the forward's test, on the same converted states
      gas_prim(gam, Um, Wm);
      gas_prim(gam, Up, Wp);
      fallback = !(Um[RHO] > 0.0 && Up[RHO] > 0.0 && Wm[EN] > 0.0 && Wp[EN] > 0.0);
    }
    if (fallback) {
#pragma unroll
      for (int f = 0; f < 5; ++f) qm[f] = qp[f] = sv(f, p + 1);
    }
  }
  double dm[4], dp[4], pm[4], p0[4], pp[4];
  if (NF == 9) {
    pm[3] = sv(8, p);
    p0[3] = sv(8, p + 1);
    pp[3] = sv(8, p + 2);
    const double im = pm[3] > 0.0 ? 1.0 / pm[3] : 0.0;
    const double i0 = p0[3] > 0.0 ? 1.0 / p0[3] : 0.0;
    const double ip = pp[3] > 0.0 ? 1.0 / pp[3] : 0.0;
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      pm[q] = sv(5 + q, p) * im;
      p0[q] = sv(5 + q, p + 1) * i0;
      pp[q] = sv(5 + q, p + 2) * ip;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) parabola(pm[q], p0[q], pp[q], w, dm[q], dp[q]);
  }

  // ---- the face below this cell: cotangents of its two states
  const bool has_face = line_ok && p >= 1;
  const double area = D == 0 ? g.area_r[clampi(c, 0, g.nr)] : (D == 1 ? g.area_t[ci] : g.area_z[ci]);
  double Fb[9];
#pragma unroll
  for (int f = 0; f < NF; ++f) Fb[f] = has_face ? area * (sm(f, p) - sm(f, p > 0 ? p - 1 : 0)) : 0.0;
  double ULb[5], URb[5];
  {
    double UL[5], UR[5];
#pragma unroll
    for (int f = 0; f < 5; ++f) {
      const double ql = __shfl_up_sync(FULL, qp[f], 1, L);
      const double e0 = eq_face(f, c);
      UL[f] = e0 + ql;
      UR[f] = e0 + qm[f];
    }
    if (has_face && RC == RECON_PRIM) {
      gas_flux_vjp<D>(gam, UL, UR, Fb, ULb, URb, status);
    } else if (has_face) {  // conservative face states: through W = gas_prim(U)
      double WL[5], WR[5], WLb[5], WRb[5];
      gas_prim(gam, UL, WL);
      gas_prim(gam, UR, WR);
      gas_flux_vjp<D>(gam, WL, WR, Fb, WLb, WRb, status);
      gas_prim_vjp(gam, UL, WLb, ULb);
      gas_prim_vjp(gam, UR, WRb, URb);
    } else {
#pragma unroll
      for (int f = 0; f < 5; ++f) ULb[f] = URb[f] = 0.0;
    }
  }
  double WLb[4], WRb[4];
  if (NF == 9) {
    double WL[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) WL[q] = __shfl_up_sync(FULL, dp[q], 1, L);
    if (has_face) {
      dust_flux_vjp<D>(WL, dm, Fb + 5, WLb, WRb);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) WLb[q] = WRb[q] = 0.0;
    }
  }

  // ---- cotangents of this cell's face values: lower from its own face, upper from the lane above
  double tm[9], t0[9], tp[9];  // contributions to cells c - 1, c, c + 1
#pragma unroll
  for (int f = 0; f < 5; ++f) {
    const double up = __shfl_down_sync(FULL, ULb[f], 1, L);
    const double gpf = p < L - 1 ? up : 0.0;
    if (fallback) {
      tm[f] = tp[f] = 0.0;
      t0[f] = URb[f] + gpf;
    } else {
      parabola_vjp(sv(f, p), sv(f, p + 1), sv(f, p + 2), w, URb[f], gpf, tm[f], t0[f], tp[f]);
    }
  }
  if (NF == 9) {
    double bm[4], b0[4], bp[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const double up = __shfl_down_sync(FULL, WLb[q], 1, L);
      parabola_vjp(pm[q], p0[q], pp[q], w, WRb[q], p < L - 1 ? up : 0.0, bm[q], b0[q], bp[q]);
    }
    // primitives (u, v, w, rho_d) back to the conservative dust fields of each cell
    auto back = [&](const double* b, const double* prim, double* t) {
      const double inv = prim[3] > 0.0 ? 1.0 / prim[3] : 0.0;  // prim[3] is the density itself
      double rb = b[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        t[5 + q] = b[q] * inv;
        rb -= b[q] * prim[q] * inv;
      }
      t[8] = rb;
    };
    back(bm, pm, tm);
    back(b0, p0, t0);
    back(bp, pp, tp);
  }
  double tot[9];
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double from_above = __shfl_down_sync(FULL, tm[f], 1, L);
    const double from_below = __shfl_up_sync(FULL, tp[f], 1, L);
    tot[f] = t0[f] + (p < L - 1 ? from_above : 0.0) + (p > 0 ? from_below : 0.0);
  }
  // zero-gradient ghosts copy the edge cell: fold their cotangents into it
  const bool out_lo = g.bc_lo[D] == BC_OUTFLOW, out_hi = g.bc_hi[D] == BC_OUTFLOW;
  if (out_lo || out_hi) {
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double u1 = __shfl_up_sync(FULL, tot[f], 1, L), u2 = __shfl_up_sync(FULL, tot[f], 2, L);
      const double d1 = __shfl_down_sync(FULL, tot[f], 1, L), d2 = __shfl_down_sync(FULL, tot[f], 2, L);
      if (out_lo && c == 0 && p >= 2) tot[f] += u1 + u2;
      if (out_hi && c == nd - 1 && p + 2 < L) tot[f] += d1 + d2;
    }
  }
  if (line_ok && p >= 2 && p < T + 2 && c < nd) {
    const size_t lin = ((size_t)cc[2] * g.nth + cc[1]) * g.nr + cc[0];
    if (RC == RECON_PRIM) {  // gas: primitive-deviation cotangents back to the conservative fields
      double U[5], Ub[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) U[f] = a.E[f][lin];
      gas_prim_vjp(gam, U, tot, Ub);
#pragma unroll
      for (int f = 0; f < 5; ++f) a.lam[f][lin] += Ub[f];
    } else {
#pragma unroll
      for (int f = 0; f < 5; ++f) a.lam[f][lin] += tot[f];
    }
#pragma unroll
    for (int f = 5; f < NF; ++f) a.lam[f][lin] += tot[f];
  }
  if (status) atomicOr(a.status, status);
}

struct Fields9 {
  double* p[9];
};

// Stage-1 drag on its own: out = D(Y) over tau (E* from the pre-drag state).
static __global__ void __launch_bounds__(ADJ_PT_NT) drag_only_kernel(DevGrid g, const Fields9 Y, const Fields9 out,
                                                             double tau, DragArgs d) {
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  for (size_t lin = blockIdx.x * (size_t)ADJ_PT_NT + threadIdx.x; lin < ncell; lin += (size_t)gridDim.x * ADJ_PT_NT) {
    double U[9];
#pragma unroll
    for (int f = 0; f < 9; ++f) U[f] = Y.p[f][lin];
    apply_drag<true, 1>(g, (int)(lin % g.nr), U, tau, d);
#pragma unroll
    for (int f = 0; f < 9; ++f) out.p[f][lin] = U[f];
  }
}

// Fixed-order sum of the d/dSt block partials of both stages; adds the
// result to this call's slot [0] and to the running total [1].
static __global__ void __launch_bounds__(512) adj_dst_reduce_kernel(const double* partials, int n, double* slots) {
  __shared__ double red[512 / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < n; b += 512) v += partials[b];
  v = block_sum<512>(v, red);
  if (threadIdx.x == 0) {
    slots[0] = v;
    slots[1] += v;
  }
}

}  // namespace rossbi
