// Fused RK2 stage kernel of the perturbation forms (state E' = E - E0).
//
// Same tiling and sweeps as the FP64 full-state kernel, but every quantity is
// formed as an exact algebraic difference from the equilibrium state E0
// (App. A), so that the balanced right-hand side G(E0 + E') - G(E0) of Sect.
// 2.8 is computed without ever forming the large equilibrium terms (the
// Keplerian centrifugal and gravity terms are O(rho v_K^2 / r), the
// perturbations 1e-4 of that and less):
//   - the parabola and limiter of Sect. 2.7 act on the conservative
//     departures E' themselves (the state), and the face state E0 + q is
//     turned into primitive perturbations about the face equilibrium,
//     rho = rho0 + rho', du = (m' - rho' u0)/rho,
//     dP = (gamma-1)(E' - [rho' |u0|^2/2 + rho u0.du + rho |du|^2/2]);
//     with RC = RECON_PRIM the same conversion is applied to each cell and
//     the parabola acts on the primitive perturbations instead;
//   - the exact Riemann solver (Sect. 2.6) iterates on dp* = p* - p0 with
//     the pressure functions written in p/p_K - 1 (log1p / expm1 for the
//     rarefaction powers), samples the wave pattern on full values and returns
//     the face-state perturbation; near-sonic fans use the FP64-derived
//     u0 -/+ c0 of the face;
//   - fluxes are differences F(W0 + dW) - F(W0) expanded by hand;
//   - sources use the FP64-derived equilibrium coefficient
//     C_r = f_r + Omega^2 r + v0^2/r + 2 Omega v0 = (1/rho0) dP0/dr.
// The Riemann problem falls back to the FP64 full-state solver on vacuum
// generation, strong rarefaction (p* < p_K / 10) or slow Newton convergence;
// the fallbacks are counted.
#pragma once
#include "stage_full.cuh"

namespace rossbi {

template <class T>
struct PertTables {
  const T* cen;    // [8][nz][nr]   rho0, v0, p0, C_r, f_z, f_r + Omega^2 r, 2 v0/r + 2 Omega, 1/r
  const T* fr;     // [5][nz][nr+1] rho0, v0, p0, c0, h0 on r faces   (h0 = E0 + p0)
  const T* fz;     // [5][nz+1][nr] same on z faces
  const T* ft;     // [7][nz][nr]   same on theta faces (= centres), then v0 - c0, v0 + c0
  const T* rcoef;  // axis-0 parabola weights, RCW per cell as DevGrid::rcoef
  const T* vol;
  const T* ivol;
  const T* area_r;
  const T* area_t;
  const T* area_z;
  const T* maxA;
  const T* omk;    // Omega_K at the cell-centre radius (constant-St drag)
  unsigned long long* fallbacks;  // count of FP64 fallback Riemann faces
};

// One state element global -> shared by an asynchronous copy (cp.async with
// the L1-allocating .ca policy: the halo cells are read again by the
// neighbouring tiles), and the wait for all of a thread's copies.
template <class T>
__device__ __forceinline__ void cp_async_elem(T* smem, const T* gmem) {
  static_assert(sizeof(T) == 4 || sizeof(T) == 8, "4- or 8-byte elements");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <class T> struct Math;
template <> struct Math<float> {
  static __device__ __forceinline__ float log1p_(float x) { return log1pf(x); }
  static __device__ __forceinline__ float expm1_(float x) { return expm1f(x); }
  static __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
  static __device__ __forceinline__ float abs_(float x) { return fabsf(x); }
  static constexpr float eps = 1.1920929e-7f;
  static constexpr int max_iter = 24;
};
template <> struct Math<double> {
  static __device__ __forceinline__ double log1p_(double x) { return log1p(x); }
  static __device__ __forceinline__ double expm1_(double x) { return expm1(x); }
  static __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }
  static __device__ __forceinline__ double abs_(double x) { return fabs(x); }
  static constexpr double eps = 2.220446049250313e-16;
  static constexpr int max_iter = 60;
};

// (1 + x)^a - 1, accurate for small x.
template <class T>
__device__ __forceinline__ T pow1pm1(T x, T a) {
  return Math<T>::expm1_(a * Math<T>::log1p_(x));
}
// sqrt(1 + t) - 1, accurate for small t.
template <class T>
__device__ __forceinline__ T sqrt1pm1(T t) {
  return t / (Math<T>::sqrt_(T(1) + t) + T(1));
}

// Powers of the exact solver, (1 + x)^a - 1 for the exponents it needs.
// Generic gamma: log1p / expm1.
template <class T>
struct PowGeneric {
  static constexpr bool series = false;
  static __device__ __forceinline__ T rar(T x, T g) { return pow1pm1(x, (g - T(1)) / (T(2) * g)); }
  static __device__ __forceinline__ T dens(T x, T g, T) { return pow1pm1(x, T(1) / g); }
  static __device__ __forceinline__ T fan_rho(T y, T g) { return pow1pm1(y, T(2) / (g - T(1))); }
  static __device__ __forceinline__ T fan_p(T y, T g) { return pow1pm1(y, T(2) * g / (g - T(1))); }
};
// gamma = 7/5 in float: with z = (1 + x)^(1/7), z^7 - 1 = (z - 1)(1 + z + ... + z^6)
// gives (1 + x)^(1/7) - 1 = x / sum z^k, accurate to a few times the error of
// the hardware log2 / exp2 estimate of z; (1 + x)^(5/7) - 1 = (z - 1)(1 + z +
// z^2 + z^3 + z^4); the fan exponents 5 and 7 are exact polynomials.
struct PowG75 {
  // Near p = p_K (|x| <= xs, x = p/p_K - 1) the pressure function of a side
  // is f = (c/gamma) x S(x) and f' = T(x)/(rho c), with S, T the Taylor
  // series of the rarefaction branch (x <= 0: S = ((1+x)^(1/7) - 1)/(x/7),
  // T = (1+x)^(-6/7)) or the shock branch (x > 0: S = (1 + 6x/7)^(-1/2),
  // T = (1 + 6x/7)^(-3/2) (1 + 3x/7)) to x^4; the branches agree to x^2 (f is
  // C^2 at p_K).  Truncation at |x| = 1/32: 4e-9 relative in f, 2.2e-8 in f'.
  static constexpr bool series = true;
  static constexpr float xs = 0.03125f;
  static constexpr float inv_gamma = 0.714285714f;
  static constexpr float beta = 0.142857143f;  // (gamma - 1) / (2 gamma)
  static __device__ __forceinline__ void pressure_series(float x, float& S, float& Td) {
    const bool rar = x <= 0.0f;
    const float s2 = rar ? 0.265306122f : 0.275510204f;    // 13/49 | 27/98
    const float s3 = rar ? -0.189504373f : -0.196793003f;  // -65/343 | -135/686
    const float s4 = rar ? 0.146189088f : 0.147594752f;    // 351/2401 | 2835/19208
    const float t2 = rar ? 0.795918367f : 0.826530612f;    // 39/49 | 81/98
    const float t3 = rar ? -0.758017493f : -0.787172012f;  // -260/343 | -270/343
    const float t4 = rar ? 0.730945440f : 0.737973761f;    // 1755/2401 | 14175/19208
    S = 1.0f + x * (-0.428571429f + x * (s2 + x * (s3 + x * s4)));
    Td = 1.0f + x * (-0.857142857f + x * (t2 + x * (t3 + x * t4)));
  }
  static __device__ __forceinline__ float rar(float x, float) {
    const float z = exp2f(__log2f(1.0f + x) * 0.142857142857f);
    const float s = 1.0f + z * (1.0f + z * (1.0f + z * (1.0f + z * (1.0f + z * (1.0f + z)))));
    return __fdividef(x, s);
  }
  static __device__ __forceinline__ float dens(float, float, float r) {
    const float z = 1.0f + r;
    return r * (1.0f + z * (1.0f + z * (1.0f + z * (1.0f + z))));
  }
  static __device__ __forceinline__ float fan_rho(float y, float) {
    return y * (5.0f + y * (10.0f + y * (10.0f + y * (5.0f + y))));
  }
  static __device__ __forceinline__ float fan_p(float y, float) {
    return y * (7.0f + y * (21.0f + y * (35.0f + y * (35.0f + y * (21.0f + y * (7.0f + y))))));
  }
};

// Face equilibrium in the frame of a face normal to axis D.
template <class T>
struct PFace {
  T rho, un, ut1, ut2, p, c, h, un_mc, un_pc;
};

// Perturbation of one side of a face, with the full values the wave pattern needs.
template <class T>
struct PSide {
  T drho, dun, dut1, dut2, dp;  // perturbations
  T rho, un, p, c, dc;          // full values and c - c0
};

// Face primitive perturbations (du, dv, dw, dP, drho in the field slots MU,
// MV, MW, EN, RHO) about the face equilibrium, in the frame of axis D, with
// the full values the wave pattern needs.  Returns false if the full state is
// not physical.
template <class T, int D>
__device__ __forceinline__ bool pert_side(T g, const PFace<T>& W0, const T* q, bool has_eq, PSide<T>& s) {
  const T dur = q[MU], dvt = q[MV], dwz = q[MW], dp = q[EN];
  const T rho = W0.rho + q[RHO];
  s.drho = q[RHO];
  s.dp = dp;
  s.dun = D == 0 ? dur : (D == 1 ? dvt : dwz);
  s.dut1 = D == 0 ? dvt : dur;
  s.dut2 = D == 2 ? dvt : dwz;
  s.rho = rho;
  s.p = W0.p + dp;
  s.un = W0.un + s.dun;
  if (!(rho > T(0)) || !(s.p > T(0))) return false;
  s.c = Math<T>::sqrt_(g * s.p / rho);
  if (has_eq) {
    s.dc = W0.c * sqrt1pm1((dp * W0.rho - W0.p * q[RHO]) / (W0.p * rho));
  } else {
    s.dc = s.c;
  }
  return true;
}

// Reciprocals of a side that the series form of its pressure function uses.
template <class T>
struct PSideInv {
  T ip, cg, irc;  // 1/p, c/gamma, 1/(rho c)
};

// Pressure function of side K at trial p = p0 + d, in perturbation form.
template <class T, class P>
__device__ __forceinline__ void pert_pressure_fn(T g, const PSide<T>& K, const PSideInv<T>& I, T p, T d, T& f,
                                                 T& fd) {
  const T dpk = d - K.dp;  // p - p_K
  if constexpr (P::series) {
    const T x = dpk * I.ip;
    if (Math<T>::abs_(x) <= P::xs) {
      T S, Td;
      P::pressure_series(x, S, Td);
      f = I.cg * x * S;
      fd = I.irc * Td;
      return;
    }
  }
  if (dpk <= T(0)) {
    const T x = dpk / K.p;
    const T r = P::rar(x, g);  // (p/p_K)^((g-1)/2g) - 1
    f = T(2) * K.c / (g - T(1)) * r;
    fd = (T(1) + r) / ((T(1) + x) * K.rho * K.c);
  } else {
    const T A = T(2) / ((g + T(1)) * K.rho);
    const T B = (g - T(1)) / (g + T(1)) * K.p;
    const T q = Math<T>::sqrt_(A / (B + p));
    f = dpk * q;
    fd = (T(1) - T(0.5) * dpk / (B + p)) * q;
  }
}

template <class T, class P>
__device__ __forceinline__ void fan_pert(T g, const PFace<T>& W0, const PSide<T>& K, bool left, T& drho, T& dun,
                                         T& dp) {
  const T g6 = (g - T(1)) / (g + T(1));
  if (left) {  // (u_L - c_L) = (u0 - c0) + du_L - dc_L
    const T y = g6 * (W0.un_mc + K.dun - K.dc) / K.c;
    drho = K.drho + K.rho * P::fan_rho(y, g);
    dp = K.dp + K.p * P::fan_p(y, g);
    dun = -W0.un_mc + K.dc + K.c * y;
  } else {     // (-u_R - c_R) = -(u0 + c0) - du_R - dc_R
    const T y = g6 * (-W0.un_pc - K.dun - K.dc) / K.c;
    drho = K.drho + K.rho * P::fan_rho(y, g);
    dp = K.dp + K.p * P::fan_p(y, g);
    dun = -W0.un_pc - K.dc - K.c * y;
  }
}

// Perturbation of the face state of the exact Riemann solution.  Returns
// 0 on success, 1 when the caller must use the FP64 full-state solver.
template <class T, class P>
__device__ __forceinline__ int pert_riemann(T g, const PFace<T>& W0, const PSide<T>& L, const PSide<T>& R, T& drho,
                                            T& dun, T& dp, int& side) {
  if (T(2) / (g - T(1)) * (L.c + R.c) <= R.un - L.un) return 1;  // vacuum generation
  const T du = R.dun - L.dun;
  const T floor_p = T(1e-8) * fmin(L.p, R.p);
  T d = T(0.5) * (L.dp + R.dp) - T(0.125) * du * (L.rho + R.rho) * (L.c + R.c);  // PVRS in dp
  if (W0.p + d < floor_p) d = floor_p - W0.p;
  const T scale = Math<T>::abs_(L.dp) + Math<T>::abs_(R.dp) + (L.rho * L.c + R.rho * R.c) * Math<T>::abs_(du);
  PSideInv<T> IL{}, IR{};
  if constexpr (P::series) {
    IL.ip = T(1) / L.p;
    IR.ip = T(1) / R.p;
    IL.cg = L.c * P::inv_gamma;
    IR.cg = R.c * P::inv_gamma;
    IL.irc = T(1) / (L.rho * L.c);
    IR.irc = T(1) / (R.rho * R.c);
  }
  T fl, fdl, fr, fdr, step = T(0);
  bool conv = false;
  for (int it = 0; it < Math<T>::max_iter; ++it) {
    const T p = W0.p + d;
    pert_pressure_fn<T, P>(g, L, IL, p, d, fl, fdl);
    pert_pressure_fn<T, P>(g, R, IR, p, d, fr, fdr);
    T dn = d - (fl + fr + du) / (fdl + fdr);
    if (W0.p + dn < floor_p) dn = floor_p - W0.p;
    step = dn - d;
    const T change = Math<T>::abs_(step);
    d = dn;
    if (change <= T(8) * Math<T>::eps * (scale + Math<T>::abs_(d))) {
      conv = true;
      break;
    }
  }
  if (!conv) return 1;
  const T ps = W0.p + d;
  if (ps < T(0.1) * fmin(L.p, R.p)) return 1;  // strong rarefaction: near vacuum
  // p*/p_K - 1 and the rarefaction power (p*/p_K)^((g-1)/2g) - 1 of a side,
  // from the series near p_K
  auto rel = [&](T dpk, T pk, const PSideInv<T>& I) -> T {
    if constexpr (P::series) return dpk * I.ip;
    else return dpk / pk;
  };
  auto rar = [&](T x) -> T {
    if constexpr (P::series) {
      if (Math<T>::abs_(x) <= P::xs) {
        T S, Td;
        P::pressure_series(x, S, Td);
        return P::beta * x * S;
      }
    }
    return P::rar(x, g);
  };
  // f_K at the converged p* from the last evaluation, one (converged) Newton
  // step away; the second-order remainder is below rounding
  fl += fdl * step;
  fr += fdr * step;
  const T dus = T(0.5) * (L.dun + R.dun) + T(0.5) * (fr - fl);
  const T us = W0.un + dus;
  const T g6 = (g - T(1)) / (g + T(1));
  if (us >= T(0)) {
    side = -1;
    const T x = rel(d - L.dp, L.p, IL);  // p*/p_L - 1
    if (d <= L.dp) {
      if (L.un - L.c >= T(0)) { drho = L.drho; dun = L.dun; dp = L.dp; return 0; }
      const T r = rar(x);
      const T cs = L.c * (T(1) + r);
      if (us - cs < T(0)) { drho = L.drho + L.rho * P::dens(x, g, r); dun = dus; dp = d; return 0; }
      fan_pert<T, P>(g, W0, L, true, drho, dun, dp);
      return 0;
    }
    if (L.un - L.c * Math<T>::sqrt_(T(1) + (g + T(1)) / (T(2) * g) * x) >= T(0)) {
      drho = L.drho; dun = L.dun; dp = L.dp; return 0;
    }
    drho = L.drho + L.rho * x * (T(1) - g6) / (T(1) + g6 * (T(1) + x));
    dun = dus;
    dp = d;
    return 0;
  }
  side = 1;
  const T x = rel(d - R.dp, R.p, IR);  // p*/p_R - 1
  if (d > R.dp) {
    if (R.un + R.c * Math<T>::sqrt_(T(1) + (g + T(1)) / (T(2) * g) * x) <= T(0)) {
      drho = R.drho; dun = R.dun; dp = R.dp; return 0;
    }
    drho = R.drho + R.rho * x * (T(1) - g6) / (T(1) + g6 * (T(1) + x));
    dun = dus;
    dp = d;
    return 0;
  }
  if (R.un + R.c <= T(0)) { drho = R.drho; dun = R.dun; dp = R.dp; return 0; }
  const T r = rar(x);
  const T cs = R.c * (T(1) + r);
  if (us + cs > T(0)) { drho = R.drho + R.rho * P::dens(x, g, r); dun = dus; dp = d; return 0; }
  fan_pert<T, P>(g, W0, R, false, drho, dun, dp);
  return 0;
}

// F(W0 + dW) - F(W0) through a face (App. B flux components, energy flux
// (E + P) u_n), written without forming the equilibrium flux.  F is in face
// order: mass, normal momentum, transverse momenta t1, t2, energy.
template <class T>
__device__ __forceinline__ void pert_flux(T g, const PFace<T>& W0, T drho, T dun, T dut1, T dut2, T dp, T* F) {
  const T un = W0.un + dun, ut1 = W0.ut1 + dut1, ut2 = W0.ut2 + dut2;
  const T dmass = drho * un + W0.rho * dun;
  const T m0 = W0.rho * W0.un;
  F[0] = dmass;
  F[1] = dmass * un + m0 * dun + dp;
  F[2] = dmass * ut1 + m0 * dut1;
  F[3] = dmass * ut2 + m0 * dut2;
  const T du2 = dun * (T(2) * W0.un + dun) + dut1 * (T(2) * W0.ut1 + dut1) + dut2 * (T(2) * W0.ut2 + dut2);
  const T dh = T(0.5) * drho * (un * un + ut1 * ut1 + ut2 * ut2) + T(0.5) * W0.rho * du2 + g / (g - T(1)) * dp;
  F[4] = dh * un + W0.h * dun;
}

// Face state perturbation of a Riemann solve, the side whose transverse
// velocity it carries (-1 left, +1 right, 0 vacuum) and status bits.
template <class T>
struct PStar {
  T drho, dun, dp;
  int side;
  unsigned status;
};

// FP64 full-state solver on W0 + dW for the faces the perturbation solver
// hands back; kept out of line so the common path stays small.  Arguments
// and result by value: a pointer or reference into the caller's frame would
// keep the caller's face states in local memory.
template <class T>
__device__ __noinline__ PStar<T> pert_fallback_fp64(T g, const PFace<T> W0, const PSide<T> L, const PSide<T> R) {
  const double rl = (double)W0.rho + (double)L.drho, rr = (double)W0.rho + (double)R.drho;
  const double ul = (double)W0.un + (double)L.dun, ur = (double)W0.un + (double)R.dun;
  const double pl = (double)W0.p + (double)L.dp, pr = (double)W0.p + (double)R.dp;
  double rho, u, p;
  PStar<T> o;
  o.status = 0;
  o.side = riemann_face((double)g, rl, ul, pl, rr, ur, pr, rho, u, p, o.status);
  o.drho = (T)(rho - (double)W0.rho);
  o.dun = (T)(u - (double)W0.un);
  o.dp = (T)(p - (double)W0.p);
  return o;
}

// Face-order gas flux perturbation (as pert_flux), status bits and whether
// the FP64 fallback solved the face.
template <class T>
struct PFlux {
  T F[5];
  unsigned status, fallback;
};

// Gas flux perturbation through a face from the primitive perturbations of
// its two reconstructed states (already checked physical).  One out-of-line
// copy serves the three sweep directions; arguments and result by value.
template <class T, class P>
__device__ __noinline__ PFlux<T> pert_face_flux(T g, const PFace<T> W0, const PSide<T> L, const PSide<T> R) {
  PFlux<T> o;
  o.status = 0;
  o.fallback = 0;
  PStar<T> st;
  st.side = 0;
  if (pert_riemann<T, P>(g, W0, L, R, st.drho, st.dun, st.dp, st.side) != 0) {
    o.fallback = 1;
    st = pert_fallback_fp64(g, W0, L, R);
    o.status = st.status;
  }
  T dut1 = T(0), dut2 = T(0);
  if (st.side < 0) { dut1 = L.dut1; dut2 = L.dut2; }
  else if (st.side > 0) { dut1 = R.dut1; dut2 = R.dut2; }
  else { dut1 = -W0.ut1; dut2 = -W0.ut2; }  // vacuum: no transverse motion
  pert_flux<T>(g, W0, st.drho, st.dun, dut1, dut2, st.dp, o.F);
  return o;
}

template <class T>
__device__ __forceinline__ PSide<T> shfl_up_side(const PSide<T>& s, int width) {
  constexpr unsigned FULL = 0xffffffffu;
  PSide<T> o;
  o.drho = __shfl_up_sync(FULL, s.drho, 1, width);
  o.dun = __shfl_up_sync(FULL, s.dun, 1, width);
  o.dut1 = __shfl_up_sync(FULL, s.dut1, 1, width);
  o.dut2 = __shfl_up_sync(FULL, s.dut2, 1, width);
  o.dp = __shfl_up_sync(FULL, s.dp, 1, width);
  o.rho = __shfl_up_sync(FULL, s.rho, 1, width);
  o.un = __shfl_up_sync(FULL, s.un, 1, width);
  o.p = __shfl_up_sync(FULL, s.p, 1, width);
  o.c = __shfl_up_sync(FULL, s.c, 1, width);
  o.dc = __shfl_up_sync(FULL, s.dc, 1, width);
  return o;
}

template <class T>
struct PertArgs {
  DevGrid g;          // geometry, sizes, boundary conditions, double tables
  PertTables<T> t;
  const T* in[NF_MAX];
  const T* base[NF_MAX];
  T* out[NF_MAX];
  double dt_host;
  const unsigned long long* dt_dev;
  double tau_frac;
  DragArgs drag;
  int stage2;
  double* partials;  // stage 2: [nf + 1][gridDim.x] block sums of V*E', then block dt minima
  unsigned* status;
  int tiles_r, tiles_z;  // tile counts along r and z (block -> tile: r fastest, then z, then theta)
  // the grid's and the drag's parameters in the state precision, converted
  // once on the host (GB300's FP64 pipe is narrow: per-use conversions of the
  // double originals cost latency in the float kernel)
  T gam, om, cfl, dx1, dx2, stokes, rhos_rp, kappa;
  T st_factor[ND_MAX];  // Stokes-number factor of each dust species
};

// Primitive perturbations (du, dv, dw, dP, drho in the field slots MU, MV,
// MW, EN, RHO) of the conservative departure q about an equilibrium state of
// density rho0 and azimuthal velocity v0 (r and z velocities zero):
// rho = rho0 + rho', du = (m' - rho' u0)/rho,
// dP = (gamma-1)(E' - [rho' |u0|^2/2 + rho u0.du + rho |du|^2/2]).
template <class T>
__device__ __forceinline__ void face_prim(T g, T rho0, T v0, const T* q, T* w) {
  const T rho = rho0 + q[RHO];
  const T ir = T(1) / rho;
  const T du = q[MU] * ir, dv = (q[MV] - q[RHO] * v0) * ir, dw = q[MW] * ir;
  const T dke = T(0.5) * q[RHO] * v0 * v0 + rho * v0 * dv + T(0.5) * rho * (du * du + dv * dv + dw * dw);
  w[MU] = du;
  w[MV] = dv;
  w[MW] = dw;
  w[EN] = (g - T(1)) * (q[EN] - dke);
  w[RHO] = q[RHO];
}

template <class T, int D>
__device__ __forceinline__ PFace<T> face_eq(const PertTables<T>& t, const DevGrid& g, int ci, int ck, int fd,
                                            T& v0) {
  PFace<T> W;
  if (!g.has_eq) {
    W.rho = W.un = W.ut1 = W.ut2 = W.p = W.c = W.h = W.un_mc = W.un_pc = T(0);
    v0 = T(0);
    return W;
  }
  if (D == 1) {
    const size_t s = (size_t)g.nz * g.nr, o = (size_t)ck * g.nr + ci;
    W.rho = t.ft[o];
    v0 = t.ft[s + o];
    W.p = t.ft[2 * s + o];
    W.c = t.ft[3 * s + o];
    W.h = t.ft[4 * s + o];
    W.un_mc = t.ft[5 * s + o];
    W.un_pc = t.ft[6 * s + o];
    W.un = v0;
    W.ut1 = W.ut2 = T(0);
    return W;
  }
  const T* tab;
  size_t s, o;
  if (D == 0) {
    tab = t.fr;
    s = (size_t)g.nz * (g.nr + 1);
    o = (size_t)ck * (g.nr + 1) + clampi(fd, 0, g.nr);
  } else {
    tab = t.fz;
    s = (size_t)(g.nz + 1) * g.nr;
    o = (size_t)clampi(fd, 0, g.nz) * g.nr + ci;
  }
  W.rho = tab[o];
  v0 = tab[s + o];
  W.p = tab[2 * s + o];
  W.c = tab[3 * s + o];
  W.h = tab[4 * s + o];
  W.un = T(0);
  W.un_mc = -W.c;
  W.un_pc = W.c;
  W.ut1 = D == 0 ? v0 : T(0);  // r face: t1 = theta;  z face: t1 = r, t2 = theta
  W.ut2 = D == 2 ? v0 : T(0);
  return W;
}

// One 32-lane chunk of the sweep along axis D: items base .. base + 31 (whole
// lines of L lanes).  The flux divergence of the chunk's cells is written to
// sG (ACC: added to it).
template <class T, int NF, int TR, int TT, int TZ, int NT, int D, class P, int RC, bool ACC>
__device__ __forceinline__ void sweep_pert_chunk(const PertArgs<T>& a, const T* sE, T* sG, int i0, int j0, int k0,
                                                 int base, unsigned& status, unsigned& nfallback) {
  constexpr int BX = TR + 4, BY = TT + 4, BZ = TZ + 4, BOX = BX * BY * BZ, NCORE = TR * TT * TZ;
  constexpr int TD = D == 0 ? TR : (D == 1 ? TT : TZ);
  constexpr int L = pow2ceil(TD + 2);
  static_assert(L <= 32, "line does not fit a warp");
  constexpr int NA = D == 0 ? TT : TR;
  constexpr int NB = D == 2 ? TT : TZ;
  constexpr int ITEMS = NA * NB * L;
  constexpr int STRIDE = D == 0 ? 1 : (D == 1 ? BX : BX * BY);
  constexpr unsigned FULL = 0xffffffffu;
  const DevGrid& g = a.g;
  const T gam = a.gam;
  const bool has_eq = g.has_eq != 0;
  const int lane = threadIdx.x & 31;
  {
    const int item = base + lane;
    const bool valid = item < ITEMS;
    const int line = valid ? item / L : 0;
    const int c = item % L - 1;
    const int ta = line % NA, tb = line / NA;
    const int x = D == 0 ? c : ta;
    const int y = D == 1 ? c : (D == 0 ? ta : tb);
    const int z = D == 2 ? c : tb;
    const int gi = i0 + x, gj = j0 + y, gk = k0 + z;
    const bool line_ok = valid && (D == 0 ? (gj < g.nth && gk < g.nz)
                                          : (D == 1 ? (gi < g.nr && gk < g.nz) : (gi < g.nr && gj < g.nth)));
    const int gd = D == 0 ? gi : (D == 1 ? gj : gk);
    const int nd = D == 0 ? g.nr : (D == 1 ? g.nth : g.nz);
    const bool do_recon = line_ok && c <= TD && gd <= nd;
    const bool do_face = do_recon && c >= 0;
    const bool do_acc = line_ok && c >= 0 && c < TD && gd < nd;
    const int sidx = do_recon ? ((z + 2) * BY + (y + 2)) * BX + (x + 2) : (2 * BY + 2) * BX + 2;
    T w[9];
    parabola_weights<T, D>(a.t.rcoef, gi, g.nr, D == 1 ? a.dx1 : a.dx2, w);
    const int ci = clampi(gi, 0, g.nr - 1), ck = clampi(gk, 0, g.nz - 1);
    T area = T(0);
    if (do_face) area = D == 0 ? a.t.area_r[clampi(gi, 0, g.nr)] : (D == 1 ? a.t.area_t[ci] : a.t.area_z[ci]);
    {
      T qm[5], qp[5];
      bool shaped = false;
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        const T* s = sE + f * BOX + sidx;
        shaped |= parabola(s[-STRIDE], s[0], s[STRIDE], w, qm[f], qp[f]);
      }
      // both face states, used for the positivity check of Sect. 2.7's
      // reconstruction and then by the two faces' solvers
      T v0m, v0p;
      const PFace<T> Wm = face_eq<T, D>(a.t, g, ci, ck, gd, v0m);
      const PFace<T> Wp = face_eq<T, D>(a.t, g, ci, ck, gd + 1, v0p);
      PSide<T> sm, sp;
      bool ok;
      if (RC == RECON_PRIM) {
        ok = pert_side<T, D>(gam, Wm, qm, has_eq, sm) & pert_side<T, D>(gam, Wp, qp, has_eq, sp);
        if (!ok && shaped) {  // positivity fallback: flat reconstruction of the gas fields
#pragma unroll
          for (int f = 0; f < 5; ++f) qm[f] = qp[f] = sE[f * BOX + sidx];
          ok = pert_side<T, D>(gam, Wm, qm, has_eq, sm) & pert_side<T, D>(gam, Wp, qp, has_eq, sp);
        }
      } else {
        // conservative face departures -> primitive perturbations about the
        // face equilibrium (rho0, v0 of that face)
        T pm[5], pp[5];
        face_prim<T>(gam, Wm.rho, v0m, qm, pm);
        face_prim<T>(gam, Wp.rho, v0p, qp, pp);
        ok = pert_side<T, D>(gam, Wm, pm, has_eq, sm) & pert_side<T, D>(gam, Wp, pp, has_eq, sp);
        if (!ok && shaped) {  // positivity fallback: flat reconstruction of the gas fields
#pragma unroll
          for (int f = 0; f < 5; ++f) qm[f] = qp[f] = sE[f * BOX + sidx];
          face_prim<T>(gam, Wm.rho, v0m, qm, pm);
          face_prim<T>(gam, Wp.rho, v0p, qp, pp);
          ok = pert_side<T, D>(gam, Wm, pm, has_eq, sm) & pert_side<T, D>(gam, Wp, pp, has_eq, sp);
        }
      }
      T F[5];
      {
        const PSide<T> sl = shfl_up_side(sp, L);  // upper face state of the lower neighbour
        const bool okl = __shfl_up_sync(FULL, ok ? 1 : 0, 1, L) != 0;
        if (do_face) {
          if (ok && okl) {
            const PFlux<T> ff = pert_face_flux<T, P>(gam, Wm, sl, sm);
            status |= ff.status;
            nfallback += ff.fallback;
            F[RHO] = ff.F[0] * area;
            F[Axes<D>::n] = ff.F[1] * area;
            F[Axes<D>::t1] = ff.F[2] * area;
            F[Axes<D>::t2] = ff.F[3] * area;
            F[EN] = ff.F[4] * area;
          } else {
            status |= STATUS_NONPHYSICAL;
#pragma unroll
            for (int f = 0; f < 5; ++f) F[f] = T(0);
          }
        } else {
#pragma unroll
          for (int f = 0; f < 5; ++f) F[f] = T(0);
        }
      }
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        const T Fu = __shfl_down_sync(FULL, F[f], 1, L);
        if (do_acc) {
          T* dst = sG + f * NCORE + (z * TT + y) * TR + x;
          if (ACC) *dst += F[f] - Fu;
          else *dst = F[f] - Fu;
        }
      }
    }
#pragma unroll 1
    for (int b = 5; b < NF; b += 4) {  // each dust species: primitive reconstruction, kinetic flux
      T qm[4], qp[4];
      dust_recon<T, BOX, STRIDE>(sE, sidx, b, w, qm, qp);
      T F[4];
      {
        T WL[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) WL[f] = __shfl_up_sync(FULL, qp[f], 1, L);
        if (do_face) {
          dust_kinetic_flux<D>(WL, qm, F);
#pragma unroll
          for (int f = 0; f < 4; ++f) F[f] *= area;
        } else {
#pragma unroll
          for (int f = 0; f < 4; ++f) F[f] = T(0);
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const T Fu = __shfl_down_sync(FULL, F[f], 1, L);
        if (do_acc) {
          T* dst = sG + (b + f) * NCORE + (z * TT + y) * TR + x;
          if (ACC) *dst += F[f] - Fu;
          else *dst = F[f] - Fu;
        }
      }
    }
  }
}

// Items (lanes) of the sweep along axis D of a TR x TT x TZ tile.
template <int TR, int TT, int TZ, int D>
__host__ __device__ constexpr int sweep_items() {
  return (D == 0 ? TT * TZ : (D == 1 ? TR * TZ : TR * TT)) * pow2ceil((D == 0 ? TR : (D == 1 ? TT : TZ)) + 2);
}

// The whole sweep along axis D, chunks spread over the block's warps.
template <class T, int NF, int TR, int TT, int TZ, int NT, int D, class P, int RC, bool ACC>
__device__ __forceinline__ void sweep_pert(const PertArgs<T>& a, const T* sE, T* sG, int i0, int j0, int k0,
                                           unsigned& status, unsigned& nfallback) {
  constexpr int CH = (sweep_items<TR, TT, TZ, D>() + 31) / 32;
  for (int ch = threadIdx.x >> 5; ch < CH; ch += NT / 32)
    sweep_pert_chunk<T, NF, TR, TT, TZ, NT, D, P, RC, ACC>(a, sE, sG, i0, j0, k0, ch * 32, status, nfallback);
}

// Dynamic shared memory of stage_pert_kernel: the staged tile and halo, and
// the accumulator of the flux divergence.  (A second accumulator, which let
// the r and theta sweeps share one pool of chunks without a barrier between
// them, measured 15 % slower on the FP32 bench grid: 101 KB per block leaves
// two blocks per SM too little L1 for the face solver's stack.)
template <class T, int NF, int TR, int TT, int TZ>
__host__ __device__ constexpr size_t pert_smem_bytes() {
  return (size_t)NF * ((TR + 4) * (TT + 4) * (TZ + 4) + TR * TT * TZ) * sizeof(T);
}

// Cell-centre equilibrium coefficients.
template <class T>
struct PCell {
  T rho0, v0, p0, Cr, fz, gr, cor, ir;
};

template <class T>
__device__ __forceinline__ PCell<T> cell_eq(const PertTables<T>& t, const DevGrid& g, int i, int k) {
  PCell<T> c;
  if (!g.has_eq) {
    c.rho0 = c.v0 = c.p0 = c.Cr = c.fz = c.gr = c.cor = c.ir = T(0);
    return c;
  }
  const size_t s = (size_t)g.nz * g.nr, o = (size_t)k * g.nr + i;
  c.rho0 = t.cen[o];
  c.v0 = t.cen[s + o];
  c.p0 = t.cen[2 * s + o];
  c.Cr = t.cen[3 * s + o];
  c.fz = t.cen[4 * s + o];
  c.gr = t.cen[5 * s + o];
  c.cor = t.cen[6 * s + o];
  c.ir = t.cen[7 * s + o];
  return c;
}

// Primitive perturbations at a cell centre: rho, (du, dv, dw), dp.
template <class T>
__device__ __forceinline__ void cell_prim(T g, const PCell<T>& c, const T* q, T& rho, T& du, T& dv, T& dw, T& dp) {
  rho = c.rho0 + q[RHO];
  const T ir = T(1) / rho;
  du = q[MU] * ir;
  dv = (q[MV] - q[RHO] * c.v0) * ir;
  dw = q[MW] * ir;
  const T dke = T(0.5) * q[RHO] * c.v0 * c.v0 + rho * c.v0 * dv + T(0.5) * rho * (du * du + dv * dv + dw * dw);
  dp = (g - T(1)) * (q[EN] - dke);
}

// Source perturbation S(E0 + E') - S(E0) per unit volume (App. B sources,
// stellar gravity, rotating frame), cylindrical geometry, plus the whole
// indirect-gravity source of Sect. 2.10 when it is on (the equilibrium's
// residual carries none).
// q: the staged cell, primitive gas perturbations (du, dv, dw, dP, drho) in
// slots 0..4 and the conservative dust fields in slots 5..8.
template <class T, int NF, bool XT>
__device__ __forceinline__ void pert_sources(const PertArgs<T>& a, const PCell<T>& c, int j, const T* q, T* S) {
  const DevGrid& g = a.g;
  const T Om = a.om;
  const T rho = c.rho0 + q[RHO], du = q[MU], dv = q[MV], dw = q[MW], dp = q[EN];
  const T v = c.v0 + dv;
  S[MU] = q[RHO] * c.Cr + rho * dv * c.cor + rho * dv * dv * c.ir + dp * c.ir;
  S[MV] = -rho * du * (v * c.ir + T(2) * Om);
  S[MW] = q[RHO] * c.fz;
  S[EN] = rho * du * c.gr + rho * dw * c.fz;
  S[RHO] = T(0);
#pragma unroll
  for (int b = 5; b < NF; b += 4) {  // each dust species
    const T rd = q[b + 3];
    if (rd > T(0)) {
      const T ird = T(1) / rd;
      const T dvd = (q[b + 1] - rd * c.v0) * ird;  // v_d - v0
      const T vd = c.v0 + dvd;
      S[b] = rd * (c.Cr + dvd * c.cor + dvd * dvd * c.ir);
      S[b + 1] = -q[b] * (vd * c.ir + T(2) * Om);
      S[b + 2] = rd * c.fz;
    } else {
      S[b] = S[b + 1] = S[b + 2] = T(0);
    }
    S[b + 3] = T(0);
  }
  if (XT && g.x_ind != 0.0) {
    T gr, gt;  // grad Phi_ind, (r, theta), tabulated per axis-1 index in the state precision
    if constexpr (sizeof(T) == 4) {
      gr = g.ind_gf[j];
      gt = g.ind_gf[g.nth + j];
    } else {
      gr = g.ind_g[j];
      gt = g.ind_g[g.nth + j];
    }
    S[MU] -= rho * gr;
    S[MV] -= rho * gt;
    S[EN] -= rho * (du * gr + v * gt);
#pragma unroll
    for (int b = 5; b < NF; b += 4) {
      if (q[b + 3] > T(0)) {
        S[b] -= q[b + 3] * gr;
        S[b + 1] -= q[b + 3] * gt;
      }
    }
  }
}

// Stopping time of dust species s in a perturbation-form cell (as
// stopping_time of the full-state kernel; gas density rg, pressure p0 + dp).
template <class T, bool XT>
__device__ __forceinline__ T pert_stopping_time(const PertArgs<T>& a, const PCell<T>& c, int i, T rg, T dp, int s) {
  if (a.drag.law == 0) {
    const T st = a.stokes * a.st_factor[s];
    return a.g.geom == GEOM_CYL ? st / a.t.omk[i] : st;
  }
  const T cs = Math<T>::sqrt_(a.gam * (c.p0 + dp) / rg);
  T ts = a.rhos_rp * a.st_factor[s] / (rg * cs);
  if (XT && a.drag.law == 2) {  // Stokes regime of Sect. 2.9 above r_p = 9 lambda / 4
    const T x = a.kappa * rg;
    if (x > T(2.25)) ts = ts * (T(4.0 / 9.0) * x);
  }
  return ts;
}

// Semi-implicit drag on a perturbation-form cell state (the closed forms of
// apply_drag; the gas velocity is u0 + du).  Several species: the gas
// velocity moves by D = sum rho_k w_k (v_k - v_g) / (rho_g + sum rho_k w_k)
// and species k by w_k (D - (v_k - v_g)), w_k = a_k / (1 + a_k), every
// quantity a difference of velocities, never the large u0 itself.
template <class T, int NF, bool XT>
__device__ __forceinline__ void pert_drag(const PertArgs<T>& a, const PCell<T>& c, int i, T* q, T tau) {
  const T gam = a.gam;
  T rg, du, dv, dw, dp;
  cell_prim(gam, c, q, rg, du, dv, dw, dp);
  const T u0[3] = {T(0), c.v0, T(0)};
  const T dug[3] = {du, dv, dw};
  if constexpr (NF == 9) {
    const T rd = q[DRHO];
    if (!(rd > T(0)) || !(rg > T(0))) return;
    const T ts = pert_stopping_time<T, XT>(a, c, i, rg, dp, 0);
    const T kk = tau * (T(1) + rd / rg) / ts;
    const T mu = rg * rd / (rg + rd);
    const T relax = kk / (T(1) + kk);
    const T ird = T(1) / rd;
    T dE = T(0);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T dvd = (q[DMU + k] - rd * u0[k]) * ird;  // v_d - u0
      const T X = mu * (dvd - dug[k]) * relax;
      const T vg_ex = u0[k] + dug[k];
      q[MU + k] += X;
      q[DMU + k] -= X;
      dE += T(0.5) * X * (T(2) * vg_ex + X / rg);
    }
    q[EN] += dE;
  } else {
  constexpr int ND = (NF - 5) / 4;
  if (!(rg > T(0))) return;
  T wk[ND], den = rg, num[3] = {T(0), T(0), T(0)};
#pragma unroll
  for (int s = 0; s < ND; ++s) {
    const int b = 5 + 4 * s;
    wk[s] = T(0);
    const T rd = q[b + 3];
    if (!(rd > T(0))) continue;
    const T ak = tau / pert_stopping_time<T, XT>(a, c, i, rg, dp, s);
    wk[s] = ak / (T(1) + ak);
    den += rd * wk[s];
    const T ird = T(1) / rd;
#pragma unroll
    for (int k = 0; k < 3; ++k) num[k] += rd * wk[s] * ((q[b + k] - rd * u0[k]) * ird - dug[k]);
  }
  T dE = T(0);
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const T D = num[k] / den;  // v_g' - v_g
#pragma unroll
    for (int s = 0; s < ND; ++s) {
      const int b = 5 + 4 * s;
      const T rd = q[b + 3];
      if (!(rd > T(0))) continue;
      const T rel = (q[b + k] - rd * u0[k]) / rd - dug[k];  // v_k - v_g
      q[b + k] += rd * wk[s] * (D - rel);
    }
    q[MU + k] += rg * D;
    dE += T(0.5) * rg * D * (T(2) * (u0[k] + dug[k]) + D);
  }
  q[EN] += dE;
  }
}

template <class T, int NF>
__device__ __forceinline__ T pert_cell_dt(const PertArgs<T>& a, const PCell<T>& c, int i, const T* q, bool& bad) {
  const PertTables<T>& t = a.t;
  const T gam = a.gam;
  T rho, du, dv, dw, dp;
  cell_prim(gam, c, q, rho, du, dv, dw, dp);
  const T p = c.p0 + dp;
  bad = !(rho > T(0)) || !(p > T(0));
  const T v = c.v0 + dv;
  const T vel = Math<T>::sqrt_(du * du + v * v + dw * dw);
  const T cs = Math<T>::sqrt_(gam * p / rho);
  const T V = t.vol[i], A = t.maxA[i], cfl = a.cfl;
  T dt = cfl * V / ((vel + cs) * A);
#pragma unroll
  for (int b = 5; b < NF; b += 4) {
    if (q[b + 3] > T(0)) {
      const T vd = Math<T>::sqrt_(q[b] * q[b] + q[b + 1] * q[b + 1] + q[b + 2] * q[b + 2]) / q[b + 3];
      if (vd > T(0)) dt = fmin(dt, cfl * V / (vd * A));
    }
    bad |= !(q[b + 3] >= T(0));
  }
  return dt;
}

// XT: the optional terms (indirect gravity, wave-killing zones) are compiled
// in; the plain instantiation carries none of their code.
template <class T, int NF, int TR, int TT, int TZ, int NT, int MINB, class P, bool XT, int RC>
__global__ void __launch_bounds__(NT, MINB) stage_pert_kernel(const PertArgs<T> a) {
  constexpr int BX = TR + 4, BY = TT + 4, BZ = TZ + 4, BOX = BX * BY * BZ, NCORE = TR * TT * TZ;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sE = reinterpret_cast<T*>(smem_raw);
  T* sG = sE + NF * BOX;
  const DevGrid& g = a.g;
  const int tile = blockIdx.x;
  // r fastest, then z, then theta: the tiles whose halos a tile re-reads
  // (its r, z and theta neighbours) run at most tiles_r x tiles_z blocks
  // apart, so the re-reads hit in L2
  const int i0 = (tile % a.tiles_r) * TR;
  const int k0 = ((tile / a.tiles_r) % a.tiles_z) * TZ;
  const int j0 = (tile / (a.tiles_r * a.tiles_z)) * TT;
  unsigned status = 0, nfallback = 0;

  if constexpr (RC == RECON_CONS) {
    // the conservative departures are staged as they are stored: each cell's
    // fields go global -> shared by asynchronous copies (cp.async, no
    // registers), all of a thread's cells in flight at once; equilibrium
    // ghosts are zero departures
    for (int idx = threadIdx.x; idx < BOX; idx += NT) {
      const int x = idx % BX - 2, y = (idx / BX) % BY - 2, z = idx / (BX * BY) - 2;
      const int outside = (x < 0 || x >= TR) + (y < 0 || y >= TT) + (z < 0 || z >= TZ);
      if (outside > 1) continue;  // edge and corner cells of the box: no sweep reads them
      int c[3] = {i0 + x, j0 + y, k0 + z};
      if (!resolve_cell(g, c)) {
#pragma unroll
        for (int f = 0; f < NF; ++f) sE[f * BOX + idx] = T(0);
      } else {
        const size_t lin = ((size_t)c[2] * g.nth + c[1]) * g.nr + c[0];
#pragma unroll
        for (int f = 0; f < NF; ++f) cp_async_elem<T>(sE + f * BOX + idx, a.in[f] + lin);
      }
    }
    cp_async_wait_all();
  } else {
  // staging in batches of CH cells per thread: every load of a batch is
  // issued before any of them is used (memory-level parallelism)
    constexpr int NIT = (BOX + NT - 1) / NT;
    constexpr int CH = 2;
    for (int it0 = 0; it0 < NIT; it0 += CH) {
      T v[CH][NF], e0[CH][3];
      int st[CH];  // 0: nothing, 1: equilibrium ghost (zero), 2: loaded
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int idx = threadIdx.x + (it0 + u) * NT;
        st[u] = 0;
        if (it0 + u < NIT && idx < BOX) {
          const int x = idx % BX - 2, y = (idx / BX) % BY - 2, z = idx / (BX * BY) - 2;
          const int outside = (x < 0 || x >= TR) + (y < 0 || y >= TT) + (z < 0 || z >= TZ);
          if (outside <= 1) {
            int c[3] = {i0 + x, j0 + y, k0 + z};
            if (!resolve_cell(g, c)) {
              st[u] = 1;
            } else {
              st[u] = 2;
              const size_t lin = ((size_t)c[2] * g.nth + c[1]) * g.nr + c[0];
#pragma unroll
              for (int f = 0; f < NF; ++f) v[u][f] = a.in[f][lin];
              if (RC == RECON_PRIM && g.has_eq) {
                const size_t sz = (size_t)g.nz * g.nr, o = (size_t)c[2] * g.nr + c[0];
                e0[u][0] = a.t.cen[o];
                e0[u][1] = a.t.cen[sz + o];
                e0[u][2] = a.t.cen[2 * sz + o];
              } else {
                e0[u][0] = e0[u][1] = e0[u][2] = T(0);
              }
            }
          }
        }
      }
#pragma unroll
      for (int u = 0; u < CH; ++u) {
        const int idx = threadIdx.x + (it0 + u) * NT;
        if (st[u] == 1) {
#pragma unroll
          for (int f = 0; f < NF; ++f) sE[f * BOX + idx] = T(0);
        } else if (st[u] == 2 && RC == RECON_CONS) {  // the state is E' itself
#pragma unroll
          for (int f = 0; f < NF; ++f) sE[f * BOX + idx] = v[u][f];
        } else if (st[u] == 2) {
          PCell<T> ce;
          ce.rho0 = e0[u][0];
          ce.v0 = e0[u][1];
          ce.p0 = e0[u][2];
          T rho, du, dv, dw, dp;
          cell_prim(a.gam, ce, v[u], rho, du, dv, dw, dp);
          sE[MU * BOX + idx] = du;
          sE[MV * BOX + idx] = dv;
          sE[MW * BOX + idx] = dw;
          sE[EN * BOX + idx] = dp;
          sE[RHO * BOX + idx] = v[u][RHO];
#pragma unroll
          for (int f = 5; f < NF; ++f) sE[f * BOX + idx] = v[u][f];
        }
      }
    }
  }
  __syncthreads();
  sweep_pert<T, NF, TR, TT, TZ, NT, 0, P, RC, false>(a, sE, sG, i0, j0, k0, status, nfallback);
  __syncthreads();
  sweep_pert<T, NF, TR, TT, TZ, NT, 1, P, RC, true>(a, sE, sG, i0, j0, k0, status, nfallback);
  __syncthreads();
  sweep_pert<T, NF, TR, TT, TZ, NT, 2, P, RC, true>(a, sE, sG, i0, j0, k0, status, nfallback);
  __syncthreads();

  const T tau = (T)(a.tau_frac * (a.dt_dev ? __longlong_as_double((long long)*a.dt_dev) : a.dt_host));
  T dtmin = T(INFINITY);
  double sums[NF];  // the conservation partials of V E', in FP64 from the first product
#pragma unroll
  for (int f = 0; f < NF; ++f) sums[f] = 0.0;
  for (int cidx = threadIdx.x; cidx < NCORE; cidx += NT) {
    const int x = cidx % TR, y = (cidx / TR) % TT, z = cidx / (TR * TT);
    const int gi = i0 + x, gj = j0 + y, gk = k0 + z;
    if (gi >= g.nr || gj >= g.nth || gk >= g.nz) continue;
    const size_t lin = ((size_t)gk * g.nth + gj) * g.nr + gi;
    const PCell<T> ce = cell_eq(a.t, g, gi, gk);
    const int sidx = ((z + 2) * BY + (y + 2)) * BX + (x + 2);
    T q[NF], G[NF];  // q: primitive gas perturbations, conservative dust
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      q[f] = sE[f * BOX + sidx];
      G[f] = sG[f * NCORE + cidx];
    }
    if (RC == RECON_CONS) {  // the staged gas departures are conservative
      T qc[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) qc[f] = q[f];
      face_prim<T>(a.gam, ce.rho0, ce.v0, qc, q);
    }
    if (g.geom == GEOM_CYL) {
      T S[NF];
      pert_sources<T, NF, XT>(a, ce, gj, q, S);
      const T V = a.t.vol[gi];
#pragma unroll
      for (int f = 0; f < NF; ++f) G[f] += V * S[f];
    }
    if (XT && g.damp_k) {  // wave-killing zones: the gas departures E' relax towards 0
      T kd;
      if constexpr (sizeof(T) == 4) kd = g.damp_kf[(size_t)gk * g.nr + gi];
      else kd = g.damp_k[(size_t)gk * g.nr + gi];
      if (kd != T(0)) {
        const T V = a.t.vol[gi];
#pragma unroll
        for (int f = 0; f < 5; ++f) G[f] -= V * kd * a.in[f][lin];
      }
    }
    const T iv = a.t.ivol[gi];
    T E[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      // stage 1 updates its own input, whose raw values are staged
      const T b = !a.stage2 && (RC == RECON_CONS || f >= 5) ? sE[f * BOX + sidx] : a.base[f][lin];
      E[f] = b + tau * G[f] * iv;
    }
    if constexpr (NF > 5) pert_drag<T, NF, XT>(a, ce, gi, E, tau);
#pragma unroll
    for (int f = 0; f < NF; ++f) a.out[f][lin] = E[f];
    bool bad_in = false;
    if (a.stage2) {
      bool bad = false;
      dtmin = fmin(dtmin, pert_cell_dt<T, NF>(a, ce, gi, E, bad));
      if (bad) status |= STATUS_NONPHYSICAL;
      const double V = g.vol[gi];
#pragma unroll
      for (int f = 0; f < NF; ++f) sums[f] += V * (double)E[f];
    } else {
      bad_in = !(ce.rho0 + q[RHO] > T(0)) || !(ce.p0 + q[EN] > T(0));
#pragma unroll
      for (int b = 5; b < NF; b += 4) bad_in |= !(q[b + 3] >= T(0));
      if (bad_in) status |= STATUS_NONPHYSICAL;
    }
  }
  if (a.stage2) {
    // the block's sums in FP64: each thread's partials to shared memory (the
    // staging area, free once every thread is past the epilogue), then NF x 8
    // threads add 32 of them each and 8-lane shuffles finish; the CFL minimum,
    // exact in any precision, stays in the state's
    constexpr int NW = NT / 32, SEG = NT / 8;
    static_assert(NT % 8 == 0 && NF * 8 <= NT, "reduction layout");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dtmin = fmin(dtmin, __shfl_xor_sync(0xffffffffu, dtmin, o));
    __syncthreads();
    double* red = reinterpret_cast<double*>(smem_raw);  // [NF][NT] partials, then [NW] minima
#pragma unroll
    for (int f = 0; f < NF; ++f) red[f * NT + threadIdx.x] = sums[f];
    if (lane == 0) red[NF * NT + warp] = (double)dtmin;
    __syncthreads();
    if (threadIdx.x < NF * 8) {
      const int f = threadIdx.x >> 3, seg = threadIdx.x & 7;
      const double* src = red + f * NT + seg * SEG;
      double acc = 0.0;
#pragma unroll 8
      for (int u = 0; u < SEG; ++u) acc += src[u];
      const unsigned grp = 0xffu << (lane & 24);  // this 8-lane group (all of it active)
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) acc += __shfl_down_sync(grp, acc, o, 8);
      if (seg == 0) a.partials[(size_t)f * gridDim.x + blockIdx.x] = acc;
    }
    if (threadIdx.x == NT - 1) {
      double m = red[NF * NT];
      for (int w = 1; w < NW; ++w) m = fmin(m, red[NF * NT + w]);
      a.partials[(size_t)NF * gridDim.x + blockIdx.x] = m;
    }
  }
  if (status) atomicOr(a.status, status);
  if (nfallback) atomicAdd(a.t.fallbacks, (unsigned long long)nfallback);
}

// CFL of a perturbation-form state (Sect. 2.5), block minimum into *slot.
template <class T, int NF>
__global__ void pert_cfl_kernel(const PertArgs<T> a, unsigned long long* slot) {
  __shared__ double red[256 / 32];
  const DevGrid& g = a.g;
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  double m = INFINITY;
  unsigned status = 0;
  for (size_t lin = blockIdx.x * (size_t)256 + threadIdx.x; lin < ncell; lin += (size_t)gridDim.x * 256) {
    T q[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) q[f] = a.in[f][lin];
    const int i = (int)(lin % g.nr), k = (int)(lin / ((size_t)g.nr * g.nth));
    bool bad = false;
    m = fmin(m, (double)pert_cell_dt<T, NF>(a, cell_eq(a.t, g, i, k), i, q, bad));
    if (bad) status |= STATUS_NONPHYSICAL;
  }
  m = block_min<256>(m, red);
  if (threadIdx.x == 0) atomic_min_pos_double(slot, m);
  if (status) atomicOr(a.status, status);
}

// Per-block FP64 partial sums of V * E'_f.
template <class T, int NF>
__global__ void pert_sums_kernel(const PertArgs<T> a, double* partials) {
  __shared__ double red[256 / 32];
  const DevGrid& g = a.g;
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  double s[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) s[f] = 0.0;
  for (size_t lin = blockIdx.x * (size_t)256 + threadIdx.x; lin < ncell; lin += (size_t)gridDim.x * 256) {
    const double V = g.vol[lin % g.nr];
#pragma unroll
    for (int f = 0; f < NF; ++f) s[f] += V * (double)a.in[f][lin];
  }
#pragma unroll
  for (int f = 0; f < NF; ++f) {
    const double t = block_sum<256>(s[f], red);
    if (threadIdx.x == 0) partials[(size_t)f * gridDim.x + blockIdx.x] = t;
  }
}

}  // namespace rossbi
