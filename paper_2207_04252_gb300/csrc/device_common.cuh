// Device-side data structures and per-cell / per-face physics of the RoSSBi3D
// step (arXiv:2207.04252).  Included by the kernel translation units only.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace rossbi {

// Conservative variables in App. B order, then the dust fluid; dust species
// s occupies fields 5 + 4 s .. 8 + 4 s in the same order (species 0 is DMU ..
// DRHO).
enum { MU = 0, MV = 1, MW = 2, EN = 3, RHO = 4, DMU = 5, DMV = 6, DMW = 7, DRHO = 8 };
constexpr int ND_MAX = 4;                 // dust species
constexpr int NF_MAX = 5 + 4 * ND_MAX;    // conservative fields
enum { GEOM_BOX = 0, GEOM_CYL = 1 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_EQUILIBRIUM = 2 };
enum { STATUS_NONPHYSICAL = 1u, STATUS_RIEMANN = 2u };
// Gas reconstruction (Sect. 2.7): the paper's component-wise parabola on the
// conservative departures E' = E - E0 of App. B's variables, or the parabola
// on the departures of the primitive variables (rho, u, v, w, P).
enum { RECON_CONS = 0, RECON_PRIM = 1 };

constexpr int GH = 2;   // ghost offset of the axis-0 coordinate tables
constexpr int RCW = 10; // parabola weights per axis-0 cell (9 used)

// Grid data the kernels read.  Passed by value as a kernel parameter; the
// pointers are device tables owned by the host runtime.
struct DevGrid {
  int geom, nr, nth, nz, nf, has_eq;
  int recon;             // RECON_CONS or RECON_PRIM
  int bc_lo[3], bc_hi[3];
  double gamma, gm, omega, cfl;
  double x0[3], dx[3];   // uniform axes 1, 2 (and axis 0 of the Box): origin, spacing
  const double* rc;      // axis-0 cell centres,  index i + GH, i in [-GH, nr + GH)
  const double* rf;      // axis-0 lower faces,   index i + GH, i in [-GH, nr + GH]
  const double* rcoef;   // axis-0 parabola weights for cells i in [-1, nr]: RCW per cell at (i + 1) * RCW
  const double* vol;     // V(i)
  const double* ivol;    // 1 / V(i)
  const double* area_r;  // A of the axis-0 face i - 1/2, i in [0, nr]
  const double* area_t;  // A of an axis-1 face of a cell with radial index i
  const double* area_z;  // A of an axis-2 face of a cell with radial index i
  const double* maxA;    // largest face area of a cell with radial index i
  const double* e0c;     // equilibrium gas state at centres   [5][nz][nr]
  const double* e0r;     // equilibrium gas state at r faces   [5][nz][nr + 1]
  const double* e0z;     // equilibrium gas state at z faces   [5][nz + 1][nr]
  const double* w0c;     // equilibrium primitive gas state (u, v, w, P, rho in the
  const double* w0r;     //   field slots MU, MV, MW, EN, RHO) at centres, r faces and
  const double* w0z;     //   z faces, same layouts as e0c / e0r / e0z
  const double* r0;      // balanced residual G(E0)            [5][nz][nr]
  // indirect gravity (Sect. 2.10): X_ref (0 = off); cos / sin of the
  // axis-1 cell centres [2][nth]; and, for the stage's input state, the
  // gradient of the indirect potential in (r, theta) components at each
  // axis-1 index [2][nth], in double and in float
  double x_ind;
  const double* ind_cs;
  const double* ind_g;
  const float* ind_gf;
  // damping zones (Sect. 2.4; the de Val-Borro et al. 2006 relaxation): the
  // rate of the radial wave-killing zones plus that of the vertical damped
  // boundary at each cell centre [nz][nr], in double and in float, or null
  const double* damp_k;
  const float* damp_kf;
  // dust species s has the Stokes number St x st_factor[s] (st_factor[0] = 1)
  double st_factor[ND_MAX];
};

__host__ __device__ constexpr int pow2ceil(int v) {
  int p = 1;
  while (p < v) p <<= 1;
  return p;
}

// Normal / transverse momentum fields for a face normal to axis D.
template <int D> struct Axes;
template <> struct Axes<0> { static constexpr int n = MU, t1 = MV, t2 = MW; };
template <> struct Axes<1> { static constexpr int n = MV, t1 = MU, t2 = MW; };
template <> struct Axes<2> { static constexpr int n = MW, t1 = MU, t2 = MV; };

// ------------------------------------------------------------------ Riemann
// Exact solution of the 1D Riemann problem (Sect. 2.6; the paper takes the
// solver of Toro, ch. 4), sampled on the face (x/t = 0).  Newton iteration on
// the star pressure from the primitive-variable estimate, then the wave
// pattern decides which state sits on the face.
struct RSide {
  double rho, u, p, c;
};

__device__ __forceinline__ void pressure_fn(double g, const RSide& K, double p, double& f, double& fd) {
  if (p <= K.p) {  // rarefaction branch
    const double prat = p / K.p;
    const double e = pow(prat, (g - 1.0) / (2.0 * g));
    f = 2.0 * K.c / (g - 1.0) * (e - 1.0);
    fd = e / (prat * K.rho * K.c);
  } else {         // shock branch
    const double A = 2.0 / ((g + 1.0) * K.rho);
    const double B = (g - 1.0) / (g + 1.0) * K.p;
    const double q = sqrt(A / (B + p));
    f = (p - K.p) * q;
    fd = (1.0 - 0.5 * (p - K.p) / (B + p)) * q;
  }
}

// Fan state at x/t = 0 inside a left (sgn = +1) or right (sgn = -1) rarefaction.
__device__ __forceinline__ void fan_state(double g, const RSide& K, double sgn, double& rho, double& u, double& p) {
  const double cf = 2.0 / (g + 1.0) * (K.c + sgn * 0.5 * (g - 1.0) * K.u);
  u = sgn * cf;
  const double ratio = cf / K.c;
  rho = K.rho * pow(ratio, 2.0 / (g - 1.0));
  p = K.p * pow(ratio, 2.0 * g / (g - 1.0));
}

// Returns the face state (rho, u_n, p) and the side (-1 left, +1 right, 0 vacuum)
// whose transverse velocity is carried.
__device__ __forceinline__ int riemann_face(double g, double rl, double ul, double pl, double rr, double ur, double pr,
                                            double& rho, double& u, double& p, unsigned& status) {
  const RSide L{rl, ul, pl, sqrt(g * pl / rl)};
  const RSide R{rr, ur, pr, sqrt(g * pr / rr)};
  if (2.0 / (g - 1.0) * (L.c + R.c) <= ur - ul) {  // the waves open a vacuum
    const double sl_star = ul + 2.0 * L.c / (g - 1.0);
    const double sr_star = ur - 2.0 * R.c / (g - 1.0);
    if (0.0 <= sl_star) {
      if (0.0 <= ul - L.c) { rho = rl; u = ul; p = pl; }
      else fan_state(g, L, 1.0, rho, u, p);
      return -1;
    }
    if (0.0 >= sr_star) {
      if (0.0 >= ur + R.c) { rho = rr; u = ur; p = pr; }
      else fan_state(g, R, -1.0, rho, u, p);
      return 1;
    }
    rho = u = p = 0.0;
    return 0;
  }
  const double pfloor = 1e-8 * fmin(pl, pr);
  double ps = fmax(pfloor, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (L.c + R.c));
  double fl, fdl, fr, fdr, step = 0.0;
  bool conv = false;
  for (int it = 0; it < 100; ++it) {
    pressure_fn(g, L, ps, fl, fdl);
    pressure_fn(g, R, ps, fr, fdr);
    const double pn = fmax(pfloor, ps - (fl + fr + ur - ul) / (fdl + fdr));
    const double change = 2.0 * fabs(pn - ps) / (pn + ps);
    step = pn - ps;
    ps = pn;
    if (change <= 1e-12) { conv = true; break; }
  }
  if (!conv) status |= STATUS_RIEMANN;
  // f_K at the converged p* from the last evaluation, one Newton step away:
  // the neglected second-order term is below rounding once the change is
  // under 1e-12
  fl += fdl * step;
  fr += fdr * step;
  const double us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  if (0.0 <= us) {  // face lies left of the contact
    if (ps <= pl) {
      if (0.0 <= ul - L.c) { rho = rl; u = ul; p = pl; return -1; }
      const double ratio = ps / pl;
      if (0.0 > us - L.c * pow(ratio, (g - 1.0) / (2.0 * g))) {
        rho = rl * pow(ratio, 1.0 / g); u = us; p = ps; return -1;
      }
      fan_state(g, L, 1.0, rho, u, p);
      return -1;
    }
    const double ratio = ps / pl;
    if (0.0 <= ul - L.c * sqrt((g + 1.0) / (2.0 * g) * ratio + (g - 1.0) / (2.0 * g))) {
      rho = rl; u = ul; p = pl; return -1;
    }
    const double g6 = (g - 1.0) / (g + 1.0);
    rho = rl * (ratio + g6) / (ratio * g6 + 1.0); u = us; p = ps;
    return -1;
  }
  if (ps > pr) {  // right shock
    const double ratio = ps / pr;
    if (0.0 >= ur + R.c * sqrt((g + 1.0) / (2.0 * g) * ratio + (g - 1.0) / (2.0 * g))) {
      rho = rr; u = ur; p = pr; return 1;
    }
    const double g6 = (g - 1.0) / (g + 1.0);
    rho = rr * (ratio + g6) / (ratio * g6 + 1.0); u = us; p = ps;
    return 1;
  }
  if (0.0 >= ur + R.c) { rho = rr; u = ur; p = pr; return 1; }
  const double ratio = ps / pr;
  if (0.0 <= us + R.c * pow(ratio, (g - 1.0) / (2.0 * g))) {
    rho = rr * pow(ratio, 1.0 / g); u = us; p = ps; return 1;
  }
  fan_state(g, R, -1.0, rho, u, p);
  return 1;
}

// The same solver for gamma = 7/5.  With z_K = (p / p_K)^(1/7) the pressure
// functions, the star density behind a rarefaction and the fan state are
// polynomials in z (exponents (gamma-1)/(2 gamma) = 1/7, 1/gamma = 5/7 ... in
// units of 1/7).  Newton runs on z_L (p = p_L z_L^7, z_R = z_L k with
// k = (p_L / p_R)^(1/7)), so a face takes two powers instead of two per
// iteration; the iterates, the stopping test on p and the sampling are those
// of riemann_face.
// Side constants of the gamma = 7/5 pressure functions, formed once per face:
// 1/(rho c), the shock coefficients A = 2/((gamma+1) rho) (as sqrt(A) and
// 1/A) and B = (gamma-1)/(gamma+1) p_K.
struct RSideZ {
  double irc, sqA, iA, B;
};
__device__ __forceinline__ RSideZ side_z(const RSide& K) {
  RSideZ s;
  s.irc = 1.0 / (K.rho * K.c);
  s.iA = 1.2 * K.rho;
  s.sqA = rsqrt(s.iA);
  s.B = K.p * (1.0 / 6.0);
  return s;
}

// Pressure function of side K at p = p_K z^7 (iz = 1/z): rarefaction
// f = 5 c (z - 1), df/dp = 1 / (rho c z^6); shock f = (p - p_K) q with
// q = sqrt(A / (B + p)), df/dp = (1 - (p - p_K) / (2 (B + p))) q, where
// (p - p_K)/(B + p) = (p - p_K) q^2 / A: no division.
__device__ __forceinline__ void pressure_fn_z(const RSide& K, const RSideZ& S, double p, double z, double iz,
                                              double& f, double& fd) {
  if (z <= 1.0) {
    const double i3 = iz * iz * iz;
    f = 5.0 * K.c * (z - 1.0);
    fd = S.irc * i3 * i3;
  } else {
    const double q = S.sqA * rsqrt(S.B + p);
    const double dp = p - K.p;
    f = dp * q;
    fd = (1.0 - 0.5 * dp * q * q * S.iA) * q;
  }
}

// Newton on z_L = (p / p_L)^(1/7) (p = p_L z_L^7, z_R = z_L k with
// k = (p_L / p_R)^(1/7)) from the start ps, z; on return ps, z are the last
// iterate, f*, fd* the pressure functions at the one before and step the last
// change of p.  The stopping test 2 |dp| <= 1e-12 (p_new + p_old) is that of
// riemann_face without its division.
__device__ __forceinline__ bool newton_z_g75(const RSide& L, const RSide& R, double du, double pfloor, double k,
                                             double& ps, double& z, double& fl, double& fdl, double& fr,
                                             double& fdr, double& step) {
  const RSideZ SL = side_z(L), SR = side_z(R);
  const double ik = 1.0 / k;
  for (int it = 0; it < 100; ++it) {
    const double iz = 1.0 / z;
    pressure_fn_z(L, SL, ps, z, iz, fl, fdl);
    pressure_fn_z(R, SR, ps, z * k, iz * ik, fr, fdr);
    // Newton on z_L: dp/dz_L = 7 p / z_L
    double zn = z - (fl + fr + du) * z / (7.0 * ps * (fdl + fdr));
    double z2 = zn * zn, z7 = z2 * z2 * z2 * zn;
    double pn = L.p * z7;
    if (!(pn >= pfloor)) {
      pn = pfloor;
      zn = pow(pfloor / L.p, 1.0 / 7.0);
    }
    step = pn - ps;
    const bool done = 2.0 * fabs(step) <= 1e-12 * (pn + ps);
    ps = pn;
    z = zn;
    if (done) return true;
  }
  return false;
}

// y^(1/7).  Near 1 (|y - 1| <= 2^-10, the common case of smooth flow, where
// p* and the two side pressures differ little) the binomial series of
// (1 + x)^(1/7) to x^5, whose truncation is below 2e-20 relative, saves
// GB300's narrow FP64 pipe a logarithm and an exponential; pow elsewhere.
__device__ __forceinline__ double root7(double y) {
  const double x = y - 1.0;
  if (fabs(x) <= 0.0009765625) {
    return 1.0 + x * (0.14285714285714285714 +           // 1/7
                      x * (-0.061224489795918367347 +    // -3/49
                           x * (0.037900874635568513120 +   // 13/343
                                x * (-0.027072053311120366514 +  // -65/2401
                                     x * 0.020884155411435413816))));  // 351/16807
  }
  return pow(y, 1.0 / 7.0);
}

__device__ __forceinline__ void fan_state_g75(const RSide& K, double sgn, double& rho, double& u, double& p) {
  const double cf = (K.c + sgn * 0.2 * K.u) / 1.2;
  u = sgn * cf;
  const double r = cf / K.c, r2 = r * r, r5 = r2 * r2 * r;
  rho = K.rho * r5;
  p = K.p * r5 * r2;
}

__device__ __forceinline__ int riemann_face_g75(double rl, double ul, double pl, double rr, double ur, double pr,
                                                double& rho, double& u, double& p, unsigned& status) {
  constexpr double g = 1.4;
  const RSide L{rl, ul, pl, sqrt(g * pl / rl)};
  const RSide R{rr, ur, pr, sqrt(g * pr / rr)};
  if (5.0 * (L.c + R.c) <= ur - ul) {  // the waves open a vacuum
    const double sl_star = ul + 5.0 * L.c;
    const double sr_star = ur - 5.0 * R.c;
    if (0.0 <= sl_star) {
      if (0.0 <= ul - L.c) { rho = rl; u = ul; p = pl; }
      else fan_state_g75(L, 1.0, rho, u, p);
      return -1;
    }
    if (0.0 >= sr_star) {
      if (0.0 >= ur + R.c) { rho = rr; u = ur; p = pr; }
      else fan_state_g75(R, -1.0, rho, u, p);
      return 1;
    }
    rho = u = p = 0.0;
    return 0;
  }
  const double pfloor = 1e-8 * fmin(pl, pr);
  double ps = fmax(pfloor, 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (L.c + R.c));
  const double k = root7(pl / pr);
  double z = root7(ps / pl);
  double fl, fdl, fr, fdr, step = 0.0;
  if (!newton_z_g75(L, R, ur - ul, pfloor, k, ps, z, fl, fdl, fr, fdr, step)) status |= STATUS_RIEMANN;
  fl += fdl * step;  // f_K at the converged p*, one Newton step from the last evaluation
  fr += fdr * step;
  const double us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  if (0.0 <= us) {  // face lies left of the contact
    if (ps <= pl) {
      if (0.0 <= ul - L.c) { rho = rl; u = ul; p = pl; return -1; }
      if (0.0 > us - L.c * z) {
        const double z2 = z * z;
        rho = rl * z2 * z2 * z; u = us; p = ps; return -1;
      }
      fan_state_g75(L, 1.0, rho, u, p);
      return -1;
    }
    const double ratio = ps / pl;
    if (0.0 <= ul - L.c * sqrt((g + 1.0) / (2.0 * g) * ratio + (g - 1.0) / (2.0 * g))) {
      rho = rl; u = ul; p = pl; return -1;
    }
    const double g6 = (g - 1.0) / (g + 1.0);
    rho = rl * (ratio + g6) / (ratio * g6 + 1.0); u = us; p = ps;
    return -1;
  }
  if (ps > pr) {  // right shock
    const double ratio = ps / pr;
    if (0.0 >= ur + R.c * sqrt((g + 1.0) / (2.0 * g) * ratio + (g - 1.0) / (2.0 * g))) {
      rho = rr; u = ur; p = pr; return 1;
    }
    const double g6 = (g - 1.0) / (g + 1.0);
    rho = rr * (ratio + g6) / (ratio * g6 + 1.0); u = us; p = ps;
    return 1;
  }
  if (0.0 >= ur + R.c) { rho = rr; u = ur; p = pr; return 1; }
  const double zr = z * k;
  if (0.0 <= us + R.c * zr) {
    const double z2 = zr * zr;
    rho = rr * z2 * z2 * zr; u = us; p = ps; return 1;
  }
  fan_state_g75(R, -1.0, rho, u, p);
  return 1;
}

__device__ __forceinline__ double gas_pressure(double g, double mu, double mv, double mw, double en, double rho) {
  return (g - 1.0) * (en - 0.5 * (mu * mu + mv * mv + mw * mw) / rho);
}

// Primitive gas state (u, v, w, P, rho), in the field slots MU, MV, MW, EN,
// RHO, of a conservative gas state.
__device__ __forceinline__ void gas_prim(double g, const double* U, double* W) {
  const double ir = 1.0 / U[RHO];  // one division: GB300's FP64 divide is a multi-instruction sequence
  W[MU] = U[MU] * ir;
  W[MV] = U[MV] * ir;
  W[MW] = U[MW] * ir;
  W[EN] = (g - 1.0) * (U[EN] - 0.5 * (U[MU] * U[MU] + U[MV] * U[MV] + U[MW] * U[MW]) * ir);
  W[RHO] = U[RHO];
}

// Cotangent Ub of the conservative gas state U for a cotangent Wb of its
// primitive state W = gas_prim(U) (the transpose of the conversion's
// Jacobian at U).
__device__ __forceinline__ void gas_prim_vjp(double g, const double* U, const double* Wb, double* Ub) {
  const double ir = 1.0 / U[RHO], gm1 = g - 1.0;
  const double v0 = U[MU] * ir, v1 = U[MV] * ir, v2 = U[MW] * ir;
  const double bP = Wb[EN];
  Ub[MU] = Wb[MU] * ir - gm1 * bP * v0;
  Ub[MV] = Wb[MV] * ir - gm1 * bP * v1;
  Ub[MW] = Wb[MW] * ir - gm1 * bP * v2;
  Ub[EN] = gm1 * bP;
  Ub[RHO] = Wb[RHO] - (Wb[MU] * v0 + Wb[MV] * v1 + Wb[MW] * v2) * ir + gm1 * bP * 0.5 * (v0 * v0 + v1 * v1 + v2 * v2);
}

// Gas flux F(E*) through a face normal to axis D from the reconstructed left
// and right primitive states (App. B flux vector; energy flux (E + P) u_n).
template <int D>
__device__ __forceinline__ void gas_face_flux(double g, const double* WL, const double* WR, double* F,
                                              unsigned& status) {
  constexpr int n = Axes<D>::n, t1 = Axes<D>::t1, t2 = Axes<D>::t2;
  const double rl = WL[RHO], rr = WR[RHO], pl = WL[EN], pr = WR[EN];
  if (!(rl > 0.0) || !(rr > 0.0) || !(pl > 0.0) || !(pr > 0.0)) {
    status |= STATUS_NONPHYSICAL;
#pragma unroll
    for (int f = 0; f < 5; ++f) F[f] = 0.0;
    return;
  }
  double rho, u, p;
  const int side = g == 1.4 ? riemann_face_g75(rl, WL[n], pl, rr, WR[n], pr, rho, u, p, status)
                            : riemann_face(g, rl, WL[n], pl, rr, WR[n], pr, rho, u, p, status);
  double ut1 = 0.0, ut2 = 0.0;
  if (side < 0) { ut1 = WL[t1]; ut2 = WL[t2]; }
  else if (side > 0) { ut1 = WR[t1]; ut2 = WR[t2]; }
  const double m = rho * u;
  F[RHO] = m;
  F[n] = m * u + p;
  F[t1] = m * ut1;
  F[t2] = m * ut2;
  F[EN] = (0.5 * rho * (u * u + ut1 * ut1 + ut2 * ut2) + p / (g - 1.0) + p) * u;
}

// Flux of the pressureless dust fluid (Sect. 2.9 "adapted" solver) by kinetic
// flux-vector splitting (Bouchut, Jin & Li 2003): the matter moving right
// crosses from the left face state, the matter moving left from the right one.
// WL, WR hold face primitives (u, v, w, rho_d); F the dust fluxes in the
// order (rho_d u, rho_d v, rho_d w, rho_d) for a face normal to axis D.
template <int D, class T>
__device__ __forceinline__ void dust_kinetic_flux(const T* WL, const T* WR, T* F) {
  constexpr int n = Axes<D>::n, t1 = Axes<D>::t1, t2 = Axes<D>::t2;  // 0..2 in the dust block
  const T ml = WL[3] * (WL[n] > T(0) ? WL[n] : T(0));
  const T mr = WR[3] * (WR[n] < T(0) ? WR[n] : T(0));
  F[3] = ml + mr;
  F[n] = ml * WL[n] + mr * WR[n];
  F[t1] = ml * WL[t1] + mr * WR[t1];
  F[t2] = ml * WL[t2] + mr * WR[t2];
}

// ------------------------------------------------------------------ sources
// App. B sources per unit volume at the cell centre: geometric terms,
// stellar gravity (Sect. 2.1), the rotating-frame Coriolis / centrifugal
// terms and, when switched on, the indirect gravity of Sect. 2.10 (force
// -grad Phi_ind on gas and dust, and its work on the gas); the Box has none.
// XT = false compiles the optional terms out.
template <bool XT>
__device__ __forceinline__ void cell_sources(const DevGrid& g, int i, int j, int k, const double* U, double* S) {
  const double r = g.rc[i + GH];
  const double z = g.x0[2] + (k + 0.5) * g.dx[2];
  const double R2 = r * r + z * z;
  const double R3 = R2 * sqrt(R2);
  const double fr = -g.gm * r / R3, fz = -g.gm * z / R3;
  const double Om = g.omega;
  {
    const double rho = U[RHO];
    const double ir = 1.0 / rho;
    const double u = U[MU] * ir, v = U[MV] * ir, w = U[MW] * ir;
    const double P = gas_pressure(g.gamma, U[MU], U[MV], U[MW], U[EN], rho);
    S[MU] = rho * v * v / r + P / r + rho * fr + 2.0 * Om * rho * v + rho * Om * Om * r;
    S[MV] = -rho * u * v / r - 2.0 * Om * rho * u;
    S[MW] = rho * fz;
    S[EN] = rho * u * (fr + Om * Om * r) + rho * w * fz;
    S[RHO] = 0.0;
  }
  for (int b = 5; b < g.nf; b += 4) {  // each dust species
    const double rho = U[b + 3];
    if (rho > 0.0) {
      const double ir = 1.0 / rho;
      const double u = U[b] * ir, v = U[b + 1] * ir;
      S[b] = rho * v * v / r + rho * fr + 2.0 * Om * rho * v + rho * Om * Om * r;
      S[b + 1] = -rho * u * v / r - 2.0 * Om * rho * u;
      S[b + 2] = rho * fz;
    } else {
      S[b] = S[b + 1] = S[b + 2] = 0.0;
    }
    S[b + 3] = 0.0;
  }
  if (XT && g.x_ind != 0.0) {
    const double gr = g.ind_g[j], gt = g.ind_g[g.nth + j];  // grad Phi_ind, (r, theta)
    const double rho = U[RHO];
    const double ir = 1.0 / rho;
    S[MU] -= rho * gr;
    S[MV] -= rho * gt;
    S[EN] -= rho * (U[MU] * ir * gr + U[MV] * ir * gt);
    for (int b = 5; b < g.nf; b += 4) {
      if (U[b + 3] > 0.0) {
        S[b] -= U[b + 3] * gr;
        S[b + 1] -= U[b + 3] * gt;
      }
    }
  }
}

// ------------------------------------------------------------------ drag
struct DragArgs {
  double stokes;
  double rhos_rp;  // Epstein constant rho_s r_p (drag laws 1 and 2)
  int law;
  double kappa;    // drag law 2: r_p / lambda_0, the mean free path being lambda_0 / rho_g
};

// Stopping time of dust species s (Stokes number St x st_factor[s]) in a cell
// of radial index i with gas state U (Sect. 2.9): drag law 0 t_s = St /
// Omega_K(r) (the Box: St); laws 1 and 2 Epstein t_s = rho_s r_p /
// (rho_g c_s), rho_s r_p proportional to St; law 2 (compiled in with XT) adds
// the Stokes regime of Sect. 2.9: above r_p = 9 lambda / 4 the Epstein time
// grows by (4/9) r_p / lambda.
template <bool XT>
__device__ __forceinline__ double stopping_time(const DevGrid& g, int i, const double* U, const DragArgs& d, int s) {
  const double rg = U[RHO];
  if (d.law == 0) {
    const double st = d.stokes * g.st_factor[s];
    if (g.geom == GEOM_CYL) {
      const double r = g.rc[i + GH];
      return st / sqrt(g.gm / (r * r * r));
    }
    return st;
  }
  const double cs = sqrt(g.gamma * gas_pressure(g.gamma, U[MU], U[MV], U[MW], U[EN], rg) / rg);
  double ts = d.rhos_rp * g.st_factor[s] / (rg * cs);
  if (XT && d.law == 2 && d.kappa * rg > 2.25) ts = ts * ((4.0 / 9.0) * (d.kappa * rg));
  return ts;
}

// Semi-implicit drag over a stage of length tau (Sect. 2.9 drag law).  One
// dust species: the relative gas-dust velocity relaxes by
// 1 / (1 + tau (1 + eps) / t_s) at fixed barycentric velocity.  ND > 1
// species: the backward-Euler system of the gas coupled to each species
// (no dust-dust exchange) in closed form, v_g' = (rho_g v_g + sum rho_k w_k
// v_k) / (rho_g + sum rho_k w_k), v_k' = (v_k + a_k v_g') / (1 + a_k), with
// a_k = tau / t_k and w_k = a_k / (1 + a_k).  The gas energy gains the work
// done on the gas in both.
template <bool XT, int ND>
__device__ __forceinline__ void apply_drag(const DevGrid& g, int i, double* U, double tau, const DragArgs& d) {
  const double rg = U[RHO];
  if constexpr (ND == 1) {
    const double rd = U[DRHO];
    if (!(rd > 0.0) || !(rg > 0.0)) return;
    const double ts = stopping_time<XT>(g, i, U, d, 0);
    const double kk = tau * (1.0 + rd / rg) / ts;
    const double mu = rg * rd / (rg + rd);
    const double relax = kk / (1.0 + kk);
    double dE = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const double vg = U[MU + c] / rg;
      const double X = mu * (U[DMU + c] / rd - vg) * relax;
      U[MU + c] += X;
      U[DMU + c] -= X;
      dE += 0.5 * X * (U[MU + c] / rg + vg);
    }
    U[EN] += dE;
  } else {
  if (!(rg > 0.0)) return;
  double a[ND], num[3], den = rg;
#pragma unroll
  for (int c = 0; c < 3; ++c) num[c] = U[MU + c];
#pragma unroll
  for (int s = 0; s < ND; ++s) {
    const int b = 5 + 4 * s;
    a[s] = 0.0;
    if (!(U[b + 3] > 0.0)) continue;
    a[s] = tau / stopping_time<XT>(g, i, U, d, s);
    const double w = a[s] / (1.0 + a[s]);
    den += U[b + 3] * w;
#pragma unroll
    for (int c = 0; c < 3; ++c) num[c] += U[b + c] * w;
  }
  double dE = 0.0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const double vg_ex = U[MU + c] / rg;
    const double vg = num[c] / den;
#pragma unroll
    for (int s = 0; s < ND; ++s) {
      const int b = 5 + 4 * s;
      if (!(U[b + 3] > 0.0)) continue;
      U[b + c] = U[b + 3] * ((U[b + c] / U[b + 3] + a[s] * vg) / (1.0 + a[s]));
    }
    U[MU + c] = rg * vg;
    dE += 0.5 * rg * (vg * vg - vg_ex * vg_ex);
  }
  U[EN] += dE;
  }
}

// ------------------------------------------------------------------ CFL
// Sect. 2.5, Eq. (cfl condition) for one cell of radial index i.
__device__ __forceinline__ double cell_dt(const DevGrid& g, int i, const double* U) {
  const double rho = U[RHO];
  const double vel = sqrt(U[MU] * U[MU] + U[MV] * U[MV] + U[MW] * U[MW]) / rho;
  const double cs = sqrt(g.gamma * gas_pressure(g.gamma, U[MU], U[MV], U[MW], U[EN], rho) / rho);
  const double V = g.vol[i], A = g.maxA[i];
  double dt = g.cfl * V / ((vel + cs) * A);
  for (int b = 5; b < g.nf; b += 4) {
    if (!(U[b + 3] > 0.0)) continue;
    const double vd = sqrt(U[b] * U[b] + U[b + 1] * U[b + 1] + U[b + 2] * U[b + 2]) / U[b + 3];
    if (vd > 0.0) dt = fmin(dt, g.cfl * V / (vd * A));
  }
  return dt;
}

__device__ __forceinline__ bool cell_nonphysical(const DevGrid& g, const double* U) {
  const double P = gas_pressure(g.gamma, U[MU], U[MV], U[MW], U[EN], U[RHO]);
  bool bad = !(U[RHO] > 0.0) || !(P > 0.0);
  for (int b = 5; b < g.nf; b += 4) bad |= !(U[b + 3] >= 0.0);
  return bad;
}

// Positive doubles order like their bit patterns, so a 64-bit integer
// atomicMin of the bits is an exact, order-independent minimum.
__device__ __forceinline__ void atomic_min_pos_double(unsigned long long* slot, double v) {
  atomicMin(slot, (unsigned long long)__double_as_longlong(v));
}

}  // namespace rossbi
