// RoSSBi3D hot-path oracle: TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU restatement of one time step of the RoSSBi3D method
// (Rendon Restrepo, Barge & Vavrik, arXiv:2207.04252).  Only the test suite,
// the smoke check and bench.py's CPU-baseline leg may load this library.  It
// shares no code, header, table or constant with the CUDA library; the two are
// compared on identical seeded inputs.
//
// Every cell is updated on its own: the six face fluxes of a cell are computed
// from scratch for that cell (each face is therefore evaluated twice per
// stage, once for each neighbour, with identical inputs and identical code, so
// the scheme stays conservative).  No blocking, fusion or reordering.
//
// Section numbers refer to the paper.  "Toro" is E. F. Toro, Riemann Solvers
// and Numerical Methods for Fluid Dynamics, ch. 4, which Sect. 2.6 names as the
// source of the exact Riemann solver.
//
// Readings of the paper that this file takes (the paper is silent or garbled):
//  R1  cell centre in r is the geometric mean of its face radii (log mesh).
//  R2  reconstruction (Sect. 2.7 on the conservative vector E of App. B): the
//      parabola acts component-wise on the departures E'_p = E_p - E0_p of the
//      five conservative gas variables (rho u, rho v, rho w, E, rho); a face
//      state is the face equilibrium E0 plus the interpolated departure.  This
//      is the default.  The MinMod limiter (Sect. 2.7 names the limiter only):
//      each face deviation of the parabola, d = q - E'_i, is limited to
//      minmod(d, s h), where s is the minmod of the two one-sided slopes and
//      h = +-min(2|x_face - x_i|, |x_neighbour - x_i|) on that side: the
//      curvature is reduced only where the parabola would leave the interval
//      of the neighbouring cell values, the result is flat at an extremum, and
//      it depends continuously on the data.  If a reconstructed gas face state
//      has rho<=0 or P<=0, all gas departures of that cell are used flat in
//      that direction.
//      Option 2 (a departure in one component): the same on the departures
//      of rho, rho u, rho v, rho w and of the pressure P(E) - P(E0) instead
//      of the energy; the face energy is P / (gamma - 1) + |m|^2 / 2 rho of
//      the face pressure, momenta and density.  Without the energy, the face
//      pressure is no longer a difference of reconstructed terms O(Mach^2)
//      larger than itself: the epicycle oscillates as it should and the
//      vortex's rounding-level drift stays at 1e-13.
//      Option 1 (a departure from the paper, kept for comparison): the same
//      parabola and limiter on the departures of the PRIMITIVE gas variables
//      (rho, u, v, w, P) from the equilibrium primitives, the face state being
//      the face equilibrium primitives plus the interpolated departure.  In a
//      fast rotating frame the conservative face pressure P = (gamma - 1)
//      (E - |m|^2 / 2 rho) is a difference of terms O(Mach^2) larger than P,
//      so the conservative form is sensitive there; the primitive form is not.
//  R3  the energy flux is (E+P)u_n (App. B prints rho(E+P)u, which is not
//      dimensionally consistent with the governing equations of Sect. 2.1).
//  R4  the RK2 update is E + dt*G/V (Sect. 2.5 prints a*V*dt*G; the compact
//      form V dE/dt = G of Sect. 2.2 fixes the 1/V).
//  R5  the dust ("adapted" solver, Sect. 2.9) is reconstructed in primitive
//      variables (rho_d and the velocity, same limiter) in both gas modes, a
//      departure from the component-wise E'_p of Sect. 2.7: the dust has no
//      pressure to keep rho_d away from zero, and the dust velocity of
//      interpolated momentum and density is unbounded near dust vacuum.  Its
//      face flux is the kinetic flux-vector splitting of pressureless gas
//      dynamics (Bouchut, Jin & Li 2003): rho_L max(u_L,0)(1,u_L,...) +
//      rho_R min(u_R,0)(1,u_R,...), which carries delta shocks by
//      accumulating mass.  Option 1 (oracle only): the velocity is used flat
//      in a cell where rho_d is a local maximum along the axis and the
//      velocity component along it decreases across the cell (a converging
//      flow piling up mass: a delta shock's spike).  With the velocity
//      parabola such a spike takes at its faces the interpolated velocity of
//      the converging streams, which points back into it, and it falls
//      behind the delta-shock speed of the pressureless Riemann problem (by
//      20 cells of 400 at t = 0.3 in the delta-shock pin); with option 1 it
//      moves at that speed to within a cell.  Flattening at every extremum
//      instead stalls the outflow of a density minimum in a diverging flow
//      and does not converge on a smooth one.
//  R6  rotating frame of angular speed Omega_f: Coriolis 2 Omega_f rho v e_r -
//      2 Omega_f rho u e_theta and centrifugal rho Omega_f^2 r e_r; the stored
//      azimuthal velocity is frame-relative.
//  R7  semi-implicit drag: after the explicit stage update, a closed-form
//      backward-Euler relaxation of the gas-dust relative velocity over the
//      stage length, conserving total momentum; the gas energy changes by the
//      work of the drag on the gas (no frictional heating).  This couples gas
//      and dust at first order in time (backward Euler, and the drag split
//      from the transport after each stage).  Option 1 (oracle only): Strang
//      splitting, half a step of trapezoidal drag before and after the RK2
//      step of the other terms, second order (the dusty-wave pin).
//  R8  equilibrium exponent uses c_iso^2 = P/rho (App. A writes c_s^2).
//  R9  Newton on p* stops when the relative change is <= 1e-12 (the error
//      left after that step is far below round-off); PVRS start, floored at
//      1e-8 min(pL, pR).
//  R10 CFL uses the frame-relative speed; a dust cell adds cfl V/(|v_d| maxA).
//  R16 indirect gravity (Sect. 2.10): A_disc and B_disc are sums over the
//      cells of the stage's input state, each cell a point mass at its
//      centre; the mass is the gas density's departure from the equilibrium
//      (an axisymmetric disc exerts no net pull, so its own A and B vanish)
//      plus the dust density.  As in the paper the vertical component is
//      dropped, and the constant in front (X_ref) is a parameter (the
//      gravitational constant in code units, 0 = off).  The force per unit
//      mass is -grad Phi_ind on gas and dust; the gas energy gains the work
//      rho (u, v).(-grad Phi_ind).  The equilibrium's residual R0 carries no
//      indirect term.
//  R17 wave-killing zones (Sect. 2.4 names radial wave-killing boundaries
//      without giving them; the form is that of de Val-Borro et al. 2006,
//      MNRAS 370, 529): in r < r_ein and r > r_eout the gas departures
//      relax towards the equilibrium, dE'/dt = -E' R(r) / tau, with R the
//      parabola that is 1 at the domain boundary and 0 (with zero slope) at
//      the zone's edge, and tau = f x the Keplerian orbital period at that
//      boundary.  It is a term of G, so it acts inside every RK stage; the
//      five conservative gas departures relax at one rate; dust is left
//      alone.  The edges and f are parameters.  Parity unpinned for the
//      profile and the constants, which come from the cited work: the pins
//      check the structure (local, linear, gas-only, the parabola through
//      its end conditions, the period) and the equilibrium.
//  R21 vertical sheared damped boundary (Sect. 2.4 names it, after the works
//      it cites, with no formula): the ghost cells beyond z = +-z_max carry
//      the sheared equilibrium flow (E' = 0, the equilibrium boundary of
//      Sect. 2.4), and in |z| > z_e the five conservative gas departures
//      relax towards it as in R17, dE'/dt = -E' R(z) / tau(r), with R the
//      parabola that is 1 at |z| = z_max and 0 (zero slope) at |z| = z_e, and
//      tau = f x the Keplerian orbital period at the cell's radius.  Its rate
//      adds to R17's radial one.  Parity unpinned for the profile and the
//      constants, as for R17.
//  R19 Stokes regime (Sect. 2.9, drag law 2): the Epstein stopping time of
//      law 1 applies while r_p <= 9 lambda / 4; above, t_s = (4/9)(r_p/lambda)
//      t_E (continuous at the switch).  The mean free path is lambda =
//      lambda_0 / rho_g (Sect. 2.9: mu m_u / (sigma_eff rho)), and
//      kappa = r_p / lambda_0 is a parameter; rho_s r_p is fixed, as for
//      law 1, so that the Epstein stopping time gives St at r = 1, z = 0.
//  R20 several dust species (Sect. 5.4 names the multi-fluid approach): N
//      pressureless dust fluids, species s in fields 5 + 4 s .. 8 + 4 s, each
//      reconstructed, fluxed and sourced as the single dust fluid (R5) and
//      coupled to the gas only, by its own drag (Stokes number St x f_s); the
//      semi-implicit drag solves the coupled backward-Euler system in closed
//      form (one species keeps the closed form of R7).
//  R22 Rossby-wave-instability disc (Sect. 4.3 adds a radial Gaussian density
//      bump to the stationary solution without saying how it is balanced):
//      the bump is part of the equilibrium E0.  rho and P are scaled by
//      s = 1 + delta G(r), G = exp(-(r - r0)^2 / (2 Delta_r^2)), at the
//      equilibrium temperature, and v_theta0 follows from radial balance with
//      the bumped pressure, so the bumped disc is itself a stationary
//      solution (of the equations, and of the balanced scheme of Sect. 2.8
//      exactly) and the run evolves only the seeded v_r of mode m.
//
// Parity unpinned (readings checked only for their properties and for
// self-consistency, since the paper gives no formula or value to test them
// against): the exact MinMod rule of R2 (pinned: exact on quadratics, flat at
// extrema, no new extrema, Lipschitz; second-order convergence on smooth
// waves), the dust flux of R5 (pinned: its case table, conservation, and the
// delta-shock and smooth-compression solutions of pressureless gas), the drag
// integrator of R7 (pinned: its closed form, the exponential limit, and its
// first-order convergence to the dusty acoustic wave), the vortex initial
// condition (a recipe of the workloads; its velocity is pinned against the
// recipe's stream function), and the wave-killing profile and constants of
// R17 (pinned: its structure).
//
// Tangent-linear mode (the paper has none; it pins the GPU adjoint).  The
// numeric core is written for a scalar type T and also instantiated with a
// dual number (value + one tangent): every branch is taken on the values, so
// the tangent is the derivative of the branch taken, at a fixed dt.  The
// star pressure's tangent is not carried through the Newton iterates but set
// by the implicit function theorem at the converged p*:
// dp* = -(df_L + df_R + du_R - du_L) / (f_L'(p*) + f_R'(p*)).
#include <cmath>
#include <cstdint>
#include <cstring>
#include <vector>
#include <unordered_map>
#include <array>
#include <algorithm>

namespace orc {

using std::sqrt;
using std::pow;
using std::exp;
using std::fabs;

enum { GEOM_BOX = 0, GEOM_CYL = 1 };
enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_EQUILIBRIUM = 2 };
// Conservative variables in the order of App. B: (rho u, rho v, rho w, E, rho),
// followed by the dust fluid (rho_d u_d, rho_d v_d, rho_d w_d, rho_d).
enum { MU = 0, MV = 1, MW = 2, EN = 3, RHO = 4, DMU = 5, DMV = 6, DMW = 7, DRHO = 8 };
enum { ST_NONPHYSICAL = 1, ST_RIEMANN = 2 };
// Reconstruction of the gas (reading R2): conservative departures (Sect. 2.7
// on App. B's E, the default), primitive departures (option 1), or the
// conservative ones with the pressure departure in place of the energy one
// (option 2).
enum { RECON_CONSERVATIVE = 0, RECON_PRIMITIVE = 1, RECON_PRESSURE = 2 };
// Dust reconstruction (reading R5): the parabola on rho_d and each velocity
// component (the default, as the kernels have it), or option 1, the same with
// the velocity used flat in a cell where rho_d is a local maximum and the
// flow converges along the axis.
enum { DUST_RECON_PARABOLA = 0, DUST_RECON_FLAT_AT_SPIKES = 1 };
// Drag integration (reading R7): backward Euler in closed form after each
// RK2 stage (the default, as the kernels have it), or option 1, Strang
// splitting: half a step of trapezoidal (Crank-Nicolson) drag before and after
// an RK2 step of the other terms.
enum { DRAG_IN_STAGES = 0, DRAG_STRANG_TRAPEZOIDAL = 1 };
// Dust species s occupies fields 5 + 4 s .. 8 + 4 s (rho_d u_d, rho_d v_d,
// rho_d w_d, rho_d); species 0 is the single dust fluid above.
static const int ND_MAX = 4, NFMAX = 5 + 4 * ND_MAX;

struct Desc {
  int geometry, nr, nth, nz;
  double x0[3], x1[3];
  int bc_lo[3], bc_hi[3];
  double gamma, gm, omega_frame, cfl;
  int n_dust;
};

static const int NG = 3;  // ghost layers kept in the coordinate tables

struct Oracle {
  Desc d;
  int n[3];
  int nf;
  long ncell;
  std::vector<double> xc[3], xf[3];  // centre / lower face of cell c at [c + NG]
  bool has_eq = false;
  double sigma0 = 0, beta_sigma = 0, T0 = 0, beta_T = 0;
  double bump_delta = 0, bump_r0 = 1, bump_width = 0;  // radial density bump of reading R22
  // equilibrium conservative gas state (5 values) at centres, r faces and z faces,
  // over the index ranges extended by NG ghosts
  std::vector<double> e0c, e0r, e0z;
  std::vector<double> r0;  // balanced-scheme residual G(E0), nf x ncell
  double x_ind = 0.0;      // X_ref of the indirect-gravity term (Sect. 2.10), 0 = off
  bool damp = false;       // wave-killing zones of reading R17
  double damp_ein = 0.0, damp_eout = 0.0, damp_tau_in = 0.0, damp_tau_out = 0.0;
  bool damp_z = false;     // vertical sheared damped boundary of reading R21
  double damp_ze = 0.0, damp_zf = 0.0;
  double kappa = 0.0;      // r_p / lambda_0 of the Stokes regime (reading R19)
  int nd = 0;              // dust species
  int recon = RECON_CONSERVATIVE;  // gas reconstruction (reading R2)
  int dust_recon = DUST_RECON_PARABOLA;  // dust reconstruction (reading R5)
  int drag_scheme = DRAG_IN_STAGES;      // drag integration (reading R7)
  double st_factor[ND_MAX] = {1.0, 1.0, 1.0, 1.0};  // St_k = St x st_factor[k] (reading R20)
  int status = 0;
  long newton_iters = 0, riemann_calls = 0;
};

// ---------------------------------------------------------------- geometry
// Sect. 2.3: logarithmic spacing in r, uniform in theta and z.  The Box option
// (Sect. 2.11, Table of options) is uniform in x, y, z.
static double face_coord(const Oracle& o, int ax, int c) {
  if (o.d.geometry == GEOM_CYL && ax == 0)
    return o.d.x0[0] * pow(o.d.x1[0] / o.d.x0[0], (double)c / o.n[0]);
  return o.d.x0[ax] + (o.d.x1[ax] - o.d.x0[ax]) * c / o.n[ax];
}
static double centre_coord(const Oracle& o, int ax, int c) {
  if (o.d.geometry == GEOM_CYL && ax == 0) return sqrt(face_coord(o, 0, c) * face_coord(o, 0, c + 1));
  return 0.5 * (face_coord(o, ax, c) + face_coord(o, ax, c + 1));
}
static inline double XC(const Oracle& o, int ax, int c) { return o.xc[ax][c + NG]; }
static inline double XF(const Oracle& o, int ax, int c) { return o.xf[ax][c + NG]; }

struct Metric {
  double V, A_lo[3], A_hi[3], maxA;
};
// Sect. 2.2: cell volume and face areas of the finite-volume cell.
static Metric metric(const Oracle& o, int i) {
  Metric m;
  const double dy = (o.d.x1[1] - o.d.x0[1]) / o.n[1];
  const double dz = (o.d.x1[2] - o.d.x0[2]) / o.n[2];
  if (o.d.geometry == GEOM_CYL) {
    const double rm = XF(o, 0, i), rp = XF(o, 0, i + 1);
    m.V = 0.5 * (rp * rp - rm * rm) * dy * dz;
    m.A_lo[0] = rm * dy * dz;
    m.A_hi[0] = rp * dy * dz;
    m.A_lo[1] = m.A_hi[1] = (rp - rm) * dz;
    m.A_lo[2] = m.A_hi[2] = 0.5 * (rp * rp - rm * rm) * dy;
    m.maxA = std::max(m.A_hi[0], std::max(m.A_hi[1], m.A_hi[2]));
  } else {
    const double dx = (o.d.x1[0] - o.d.x0[0]) / o.n[0];
    m.V = dx * dy * dz;
    m.A_lo[0] = m.A_hi[0] = dy * dz;
    m.A_lo[1] = m.A_hi[1] = dx * dz;
    m.A_lo[2] = m.A_hi[2] = dx * dy;
    m.maxA = std::max(m.A_hi[0], std::max(m.A_hi[1], m.A_hi[2]));
  }
  return m;
}

// ---------------------------------------------------------------- equilibrium
// App. A: axisymmetric, locally isothermal gas in Keplerian rotation and
// vertical hydrostatic balance; code units GM = gm, k_B/(mu m_u) = 1.
static void eq_prim(const Oracle& o, double r, double z, double& rho, double& vth, double& p) {
  const double gm = o.d.gm;
  const double cs2 = o.T0 * pow(r, o.beta_T);     // T(r) = c_iso^2
  const double omk = sqrt(gm / (r * r * r));      // Omega_K(r)
  const double H = sqrt(2.0 * cs2) / omk;         // H = sqrt(2/gamma) c_s / Omega_K, c_s^2 = gamma c_iso^2
  const double R = sqrt(r * r + z * z);
  const double g = 1.0 / R - 1.0 / r;
  rho = o.sigma0 * pow(r, o.beta_sigma) / (sqrt(M_PI) * H) * exp(gm / cs2 * g);
  p = cs2 * rho;
  // d ln P0 / dr, differentiated by hand from the expressions above
  double dlnp = (o.beta_T + o.beta_sigma - 0.5 * (o.beta_T + 3.0)) / r +
                      gm / cs2 * (-o.beta_T * g / r - r / (R * R * R) + 1.0 / (r * r));
  // Sect. 4.3 (reading R22): a radial Gaussian density bump at r0 of width
  // Delta_r, rho and P both scaled by s = 1 + delta G(r) (the temperature
  // kept, so vertical balance holds unchanged); d ln P / dr gains s'/s
  if (o.bump_delta != 0.0) {
    const double x = (r - o.bump_r0) / o.bump_width;
    const double G = exp(-0.5 * x * x);
    const double s = 1.0 + o.bump_delta * G;
    rho *= s;
    p *= s;
    dlnp += o.bump_delta * G * (-x / o.bump_width) / s;
  }
  // v_theta0^2 = -r f_star,r + (r/rho) dP/dr
  vth = sqrt(gm * r * r / (R * R * R) + r * cs2 * dlnp);
}
// Conservative equilibrium state in the rotating frame (reading R6).
static void eq_cons(const Oracle& o, double r, double z, double U[5]) {
  double rho, vth, p;
  eq_prim(o, r, z, rho, vth, p);
  const double v = vth - o.d.omega_frame * r;
  U[MU] = 0.0;
  U[MV] = rho * v;
  U[MW] = 0.0;
  U[EN] = 0.5 * rho * v * v + p / (o.d.gamma - 1.0);
  U[RHO] = rho;
}
static inline const double* E0C(const Oracle& o, int i, int k) {
  return &o.e0c[((size_t)(k + NG) * (o.n[0] + 2 * NG) + (i + NG)) * 5];
}
static inline const double* E0R(const Oracle& o, int iface, int k) {
  return &o.e0r[((size_t)(k + NG) * (o.n[0] + 2 * NG + 1) + (iface + NG)) * 5];
}
static inline const double* E0Z(const Oracle& o, int i, int kface) {
  return &o.e0z[((size_t)(kface + NG) * (o.n[0] + 2 * NG) + (i + NG)) * 5];
}

// ---------------------------------------------------------------- scalar types
// The numeric core below is written once for a scalar type T: double for the
// oracle itself, Dual (value + one tangent) for its tangent-linear mode.
// Every branch is decided on the value, so the tangent is the derivative of
// the branch that was taken.
struct Dual {
  double v, d;
  Dual(double v_ = 0.0, double d_ = 0.0) : v(v_), d(d_) {}
};
static inline Dual operator+(Dual a, Dual b) { return Dual(a.v + b.v, a.d + b.d); }
static inline Dual operator-(Dual a, Dual b) { return Dual(a.v - b.v, a.d - b.d); }
static inline Dual operator*(Dual a, Dual b) { return Dual(a.v * b.v, a.d * b.v + a.v * b.d); }
static inline Dual operator/(Dual a, Dual b) { return Dual(a.v / b.v, (a.d * b.v - a.v * b.d) / (b.v * b.v)); }
static inline Dual operator-(Dual a) { return Dual(-a.v, -a.d); }
static inline Dual operator+(Dual a, double b) { return Dual(a.v + b, a.d); }
static inline Dual operator+(double a, Dual b) { return Dual(a + b.v, b.d); }
static inline Dual operator-(Dual a, double b) { return Dual(a.v - b, a.d); }
static inline Dual operator-(double a, Dual b) { return Dual(a - b.v, -b.d); }
static inline Dual operator*(Dual a, double b) { return Dual(a.v * b, a.d * b); }
static inline Dual operator*(double a, Dual b) { return Dual(a * b.v, a * b.d); }
static inline Dual operator/(Dual a, double b) { return Dual(a.v / b, a.d / b); }
static inline Dual operator/(double a, Dual b) { return Dual(a / b.v, -a * b.d / (b.v * b.v)); }
static inline Dual& operator+=(Dual& a, Dual b) { a = a + b; return a; }
static inline Dual& operator-=(Dual& a, Dual b) { a = a - b; return a; }
static inline bool operator<(Dual a, Dual b) { return a.v < b.v; }
static inline bool operator<=(Dual a, Dual b) { return a.v <= b.v; }
static inline bool operator>(Dual a, Dual b) { return a.v > b.v; }
static inline bool operator>=(Dual a, Dual b) { return a.v >= b.v; }
static inline bool operator!=(Dual a, Dual b) { return a.v != b.v; }
static inline Dual sqrt(Dual a) {
  const double r = std::sqrt(a.v);
  return Dual(r, a.d / (2.0 * r));
}
static inline Dual pow(Dual a, double e) {
  const double r = std::pow(a.v, e);
  return Dual(r, e * std::pow(a.v, e - 1.0) * a.d);
}
static inline Dual fabs(Dual a) { return a.v < 0.0 ? -a : a; }
static inline double val(double x) { return x; }
static inline double val(Dual x) { return x.v; }
template <class T> static inline T tmin(T a, T b) { return b < a ? b : a; }

// ---------------------------------------------------------------- state access
template <class T>
struct ArrAccT {
  using value_type = T;
  const T* E;
  long ncell;
  T get(int f, long lin) const { return E[(size_t)f * ncell + lin]; }
};
using ArrAcc = ArrAccT<double>;

// Deviation E' = E - E0 (Sect. 2.7) of field f at cell (i, j, k); at most one
// index may lie outside the domain, where the ghost rule of Sect. 2.4 applies:
// equilibrium ghosts carry E' = 0, periodic ghosts wrap, outflow ghosts copy
// the nearest interior deviation.
template <class Acc>
static typename Acc::value_type dev(const Oracle& o, const Acc& E, int f, int i, int j, int k) {
  using T = typename Acc::value_type;
  int c[3] = {i, j, k};
  for (int ax = 0; ax < 3; ++ax) {
    if (c[ax] >= 0 && c[ax] < o.n[ax]) continue;
    const int bc = c[ax] < 0 ? o.d.bc_lo[ax] : o.d.bc_hi[ax];
    if (bc == BC_EQUILIBRIUM) return T(0.0);
    if (bc == BC_PERIODIC)
      c[ax] = ((c[ax] % o.n[ax]) + o.n[ax]) % o.n[ax];
    else
      c[ax] = c[ax] < 0 ? 0 : o.n[ax] - 1;
  }
  const long lin = ((long)c[2] * o.n[1] + c[1]) * o.n[0] + c[0];
  T e = E.get(f, lin);
  if (f < 5 && o.has_eq) e -= E0C(o, c[0], c[2])[f];
  return e;
}

template <class T>
static inline T pressure(double g, const T* U);

// Pressure departure P(E) - P(E0) of cell (i, j, k) under the same ghost
// rule as dev() (reading R2, option 2); without an equilibrium, P(E).
template <class Acc>
static typename Acc::value_type pdev(const Oracle& o, const Acc& E, int i, int j, int k) {
  using T = typename Acc::value_type;
  int c[3] = {i, j, k};
  for (int ax = 0; ax < 3; ++ax) {
    if (c[ax] >= 0 && c[ax] < o.n[ax]) continue;
    const int bc = c[ax] < 0 ? o.d.bc_lo[ax] : o.d.bc_hi[ax];
    if (bc == BC_EQUILIBRIUM) return T(0.0);
    if (bc == BC_PERIODIC)
      c[ax] = ((c[ax] % o.n[ax]) + o.n[ax]) % o.n[ax];
    else
      c[ax] = c[ax] < 0 ? 0 : o.n[ax] - 1;
  }
  const long lin = ((long)c[2] * o.n[1] + c[1]) * o.n[0] + c[0];
  T U[5];
  for (int f = 0; f < 5; ++f) U[f] = E.get(f, lin);
  if (!o.has_eq) return pressure(o.d.gamma, U);
  const double* U0 = E0C(o, c[0], c[2]);
  return pressure(o.d.gamma, U) - pressure(o.d.gamma, U0);
}

// ---------------------------------------------------------------- reconstruction
template <class T>
static inline T minmod(T a, T b) {
  if (a * b <= 0.0) return T(0.0);
  return fabs(a) < fabs(b) ? a : b;
}
// Sect. 2.7: the parabola through the three cell values of E' at the centre
// coordinates xm < x0 < xp, evaluated at the faces fm, fp of the middle cell,
// with the paper's coefficients a, b and the slopes nabla E'(i) = sm,
// nabla E'(i+1) = sp; then the MinMod limiter of reading R2.  Returns false
// when the result is flat.
template <class T>
static bool parabola(T em, T e0, T ep, double xm, double x0, double xp, double fm, double fp, T& qm, T& qp) {
  const T sm = (e0 - em) / (x0 - xm);
  const T sp = (ep - e0) / (xp - x0);
  const T s = minmod(sm, sp);
  const T a = (sp - sm) / (xp - xm);
  const T b = (sp * (x0 - xm) + sm * (xp - x0)) / (xp - xm);
  const double dm = fm - x0, dp = fp - x0;
  const double hm = -std::min(-2.0 * dm, x0 - xm), hp = std::min(2.0 * dp, xp - x0);
  qm = e0 + minmod(a * dm * dm + b * dm, s * hm);
  qp = e0 + minmod(a * dp * dp + b * dp, s * hp);
  return s != 0.0;
}

template <class T>
static inline T pressure(double g, const T* U) {
  return (g - 1.0) * (U[EN] - 0.5 * (U[MU] * U[MU] + U[MV] * U[MV] + U[MW] * U[MW]) / U[RHO]);
}

// Equilibrium gas state (5 values) on face `fc` (the lower face of cell fc)
// along axis ax, for a cell with radial index i and vertical index k.
static void eq_face(const Oracle& o, int ax, int i, int k, int fc, double e0[5]) {
  if (!o.has_eq) {
    for (int f = 0; f < 5; ++f) e0[f] = 0.0;
    return;
  }
  const double* s = ax == 0 ? E0R(o, fc, k) : ax == 1 ? E0C(o, i, k) : E0Z(o, i, fc);
  for (int f = 0; f < 5; ++f) e0[f] = s[f];
}

// Primitive gas state (u, v, w, P, rho), in the field slots MU, MV, MW, EN,
// RHO, of a conservative state, and back.
template <class T>
static void prim_of(double g, const T* U, T* W) {
  for (int q = 0; q < 3; ++q) W[MU + q] = U[MU + q] / U[RHO];
  W[EN] = pressure(g, U);
  W[RHO] = U[RHO];
}
template <class T>
static void cons_of(double g, const T* W, T* U) {
  U[RHO] = W[RHO];
  for (int q = 0; q < 3; ++q) U[MU + q] = W[RHO] * W[MU + q];
  U[EN] = W[EN] / (g - 1.0) + 0.5 * W[RHO] * (W[MU] * W[MU] + W[MV] * W[MV] + W[MW] * W[MW]);
}

// Primitive deviations (u', v', w', P', rho') of cell (i, j, k), stored in the
// field slots MU, MV, MW, EN, RHO: the cell's primitive state minus the
// equilibrium primitive state at the cell (reading R2).  Ghost rule of
// Sect. 2.4 as in dev(): equilibrium ghosts carry zero deviation, periodic
// ghosts wrap, outflow ghosts copy the nearest interior deviation.
template <class Acc, class T = typename Acc::value_type>
static void prim_dev(const Oracle& o, const Acc& E, int i, int j, int k, T d[5]) {
  int c[3] = {i, j, k};
  for (int ax = 0; ax < 3; ++ax) {
    if (c[ax] >= 0 && c[ax] < o.n[ax]) continue;
    const int bc = c[ax] < 0 ? o.d.bc_lo[ax] : o.d.bc_hi[ax];
    if (bc == BC_EQUILIBRIUM) {
      for (int f = 0; f < 5; ++f) d[f] = T(0.0);
      return;
    }
    if (bc == BC_PERIODIC)
      c[ax] = ((c[ax] % o.n[ax]) + o.n[ax]) % o.n[ax];
    else
      c[ax] = c[ax] < 0 ? 0 : o.n[ax] - 1;
  }
  const long lin = ((long)c[2] * o.n[1] + c[1]) * o.n[0] + c[0];
  T U[5];
  for (int f = 0; f < 5; ++f) U[f] = E.get(f, lin);
  double W0[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
  if (o.has_eq) prim_of(o.d.gamma, E0C(o, c[0], c[2]), W0);
  for (int q = 0; q < 3; ++q) d[MU + q] = U[MU + q] / U[RHO] - W0[MU + q];
  d[EN] = pressure(o.d.gamma, U) - W0[EN];
  d[RHO] = U[RHO] - W0[RHO];
}

// Face deviations q- (lower face) and q+ (upper face) of cell `cell` along ax,
// as conservative face states minus the conservative face equilibrium.  Gas
// (Sect. 2.7, reading R2): by default the parabola + MinMod on each of the
// five conservative departures E'_p; with the primitive option, on the
// primitive departures, face primitives = face equilibrium primitives +
// deviation.  In both, if either face has rho <= 0 or P <= 0 the cell's gas
// departures are used flat.  Dust: reading R5.
template <class Acc, class T = typename Acc::value_type>
static void recon(const Oracle& o, const Acc& E, int ax, const int cell[3], T qm[NFMAX], T qp[NFMAX]) {
  int cm[3] = {cell[0], cell[1], cell[2]}, cp[3] = {cell[0], cell[1], cell[2]};
  cm[ax] -= 1;
  cp[ax] += 1;
  const int c = cell[ax];
  const double xm = XC(o, ax, c - 1), x0 = XC(o, ax, c), xp = XC(o, ax, c + 1);
  const double fm = XF(o, ax, c), fp = XF(o, ax, c + 1);
  double e0m[5], e0p[5];
  eq_face(o, ax, cell[0], cell[2], c, e0m);
  eq_face(o, ax, cell[0], cell[2], c + 1, e0p);
  if (o.recon == RECON_CONSERVATIVE || o.recon == RECON_PRESSURE) {
    T em[5], ec[5], ep[5];
    bool gas_shaped = false;
    for (int f = 0; f < 5; ++f) {
      em[f] = dev(o, E, f, cm[0], cm[1], cm[2]);
      ec[f] = dev(o, E, f, cell[0], cell[1], cell[2]);
      ep[f] = dev(o, E, f, cp[0], cp[1], cp[2]);
      if (o.recon == RECON_PRESSURE && f == EN) continue;
      gas_shaped |= parabola(em[f], ec[f], ep[f], xm, x0, xp, fm, fp, qm[f], qp[f]);
    }
    if (o.recon == RECON_PRESSURE) {
      // option 2 of reading R2: the pressure departure is reconstructed in
      // place of the energy one; the face energy follows from the face
      // pressure, momenta and density
      T pqm, pqp;
      gas_shaped |= parabola(pdev(o, E, cm[0], cm[1], cm[2]), pdev(o, E, cell[0], cell[1], cell[2]),
                             pdev(o, E, cp[0], cp[1], cp[2]), xm, x0, xp, fm, fp, pqm, pqp);
      auto energy = [&](const double* e0f, T* q, T pq) {
        T U[5];
        for (int f = 0; f < 5; ++f) U[f] = e0f[f] + q[f];
        const T P = (o.has_eq ? pressure(o.d.gamma, e0f) : 0.0) + pq;
        q[EN] = P / (o.d.gamma - 1.0) + 0.5 * (U[MU] * U[MU] + U[MV] * U[MV] + U[MW] * U[MW]) / U[RHO] - e0f[EN];
      };
      energy(e0m, qm, pqm);
      energy(e0p, qp, pqp);
    }
    if (gas_shaped) {  // positivity of both gas face states
      T Um[5], Up[5];
      for (int f = 0; f < 5; ++f) {
        Um[f] = e0m[f] + qm[f];
        Up[f] = e0p[f] + qp[f];
      }
      if (!(Um[RHO] > 0.0 && Up[RHO] > 0.0 && pressure(o.d.gamma, Um) > 0.0 && pressure(o.d.gamma, Up) > 0.0))
        for (int f = 0; f < 5; ++f) qm[f] = qp[f] = ec[f];
    }
  } else {
    T dm[5], d0[5], dp[5], wm[5], wp[5];
    prim_dev(o, E, cm[0], cm[1], cm[2], dm);
    prim_dev(o, E, cell[0], cell[1], cell[2], d0);
    prim_dev(o, E, cp[0], cp[1], cp[2], dp);
    bool gas_shaped = false;
    for (int f = 0; f < 5; ++f) gas_shaped |= parabola(dm[f], d0[f], dp[f], xm, x0, xp, fm, fp, wm[f], wp[f]);
    double W0m[5] = {0, 0, 0, 0, 0}, W0p[5] = {0, 0, 0, 0, 0};
    if (o.has_eq) {
      prim_of(o.d.gamma, e0m, W0m);
      prim_of(o.d.gamma, e0p, W0p);
    }
    T Wm[5], Wp[5];
    for (int f = 0; f < 5; ++f) {
      Wm[f] = W0m[f] + wm[f];
      Wp[f] = W0p[f] + wp[f];
    }
    if (gas_shaped && !(Wm[RHO] > 0.0 && Wp[RHO] > 0.0 && Wm[EN] > 0.0 && Wp[EN] > 0.0)) {
      for (int f = 0; f < 5; ++f) {  // positivity of both gas face states
        Wm[f] = W0m[f] + d0[f];
        Wp[f] = W0p[f] + d0[f];
      }
    }
    T Um[5], Up[5];
    cons_of(o.d.gamma, Wm, Um);
    cons_of(o.d.gamma, Wp, Up);
    for (int f = 0; f < 5; ++f) {
      qm[f] = Um[f] - e0m[f];
      qp[f] = Up[f] - e0p[f];
    }
  }
  for (int s = 0; s < o.nd; ++s) {  // R5: dust in primitive variables (rho_d, u_d, v_d, w_d), per species
    const int b = 5 + 4 * s;
    T pm[4], p0[4], pp[4], qmw[4], qpw[4];
    pm[3] = dev(o, E, b + 3, cm[0], cm[1], cm[2]);
    p0[3] = dev(o, E, b + 3, cell[0], cell[1], cell[2]);
    pp[3] = dev(o, E, b + 3, cp[0], cp[1], cp[2]);
    for (int q = 0; q < 3; ++q) {
      pm[q] = pm[3] > 0.0 ? dev(o, E, b + q, cm[0], cm[1], cm[2]) / pm[3] : T(0.0);
      p0[q] = p0[3] > 0.0 ? dev(o, E, b + q, cell[0], cell[1], cell[2]) / p0[3] : T(0.0);
      pp[q] = pp[3] > 0.0 ? dev(o, E, b + q, cp[0], cp[1], cp[2]) / pp[3] : T(0.0);
    }
    for (int q = 0; q < 4; ++q) parabola(pm[q], p0[q], pp[q], xm, x0, xp, fm, fp, qmw[q], qpw[q]);
    // option 1: where rho_d is a local maximum and the flow converges along
    // the axis (a delta shock's spike) the cell's own velocity is carried to
    // both faces, so that the spike's mass leaves it at the spike's speed
    // instead of the interpolated one
    if (o.dust_recon == DUST_RECON_FLAT_AT_SPIKES && p0[3] > pm[3] && p0[3] > pp[3] && pm[ax] > pp[ax])
      for (int q = 0; q < 3; ++q) qmw[q] = qpw[q] = p0[q];
    qm[b + 3] = qmw[3];
    qp[b + 3] = qpw[3];
    for (int q = 0; q < 3; ++q) {
      qm[b + q] = qmw[3] * qmw[q];
      qp[b + q] = qpw[3] * qpw[q];
    }
  }
}

// ---------------------------------------------------------------- exact Riemann solver (Toro)
template <class T>
struct Side {
  T rho, u, p, c;
};
// Pressure function f_K(p) of the star-region pressure and its derivative
// (Toro ch. 4.2-4.3): rarefaction branch for p <= p_K, shock branch above.
template <class T>
static void prefun(double g, const Side<T>& K, T p, T& f, T& fd) {
  if (p <= K.p) {  // rarefaction
    const T prat = p / K.p;
    f = 2.0 * K.c / (g - 1.0) * (pow(prat, (g - 1.0) / (2.0 * g)) - 1.0);
    fd = 1.0 / (K.rho * K.c) * pow(prat, -(g + 1.0) / (2.0 * g));
  } else {  // shock
    const T A = 2.0 / ((g + 1.0) * K.rho);
    const T B = (g - 1.0) / (g + 1.0) * K.p;
    const T q = sqrt(A / (B + p));
    f = (p - K.p) * q;
    fd = (1.0 - 0.5 * (p - K.p) / (B + p)) * q;
  }
}

template <class T>
struct RiemannResult {
  T rho, u, p;        // state at x/t = S
  int side;           // -1: left of the contact, +1: right, 0: vacuum
  T pstar, ustar;
  int iters;
  bool converged, vacuum;
};

template <class T>
static void fan_left(double g, const Side<T>& L, double S, T& rho, T& u, T& p) {
  const T c = 2.0 / (g + 1.0) * (L.c + 0.5 * (g - 1.0) * (L.u - S));
  u = 2.0 / (g + 1.0) * (L.c + 0.5 * (g - 1.0) * L.u + S);
  rho = L.rho * pow(c / L.c, 2.0 / (g - 1.0));
  p = L.p * pow(c / L.c, 2.0 * g / (g - 1.0));
}
template <class T>
static void fan_right(double g, const Side<T>& R, double S, T& rho, T& u, T& p) {
  const T c = 2.0 / (g + 1.0) * (R.c - 0.5 * (g - 1.0) * (R.u - S));
  u = 2.0 / (g + 1.0) * (-R.c + 0.5 * (g - 1.0) * R.u + S);
  rho = R.rho * pow(c / R.c, 2.0 / (g - 1.0));
  p = R.p * pow(c / R.c, 2.0 * g / (g - 1.0));
}

// Tangent of the star pressure.  The converged p* is a function of the two
// states through f_L(p*) + f_R(p*) + u_R - u_L = 0, so by the implicit
// function theorem dp* = -(df_L + df_R + du_R - du_L) / (f_L' + f_R') at p*,
// the partials taken with p held fixed; this replaces the tangent carried
// through the Newton iterates.  A p* held at the floor follows the floor.
static inline void star_tangent(double, const Side<double>&, const Side<double>&, double, double, double, double&) {}
static void star_tangent(double g, const Side<Dual>& L, const Side<Dual>& R, Dual ul, Dual ur, Dual floor_p, Dual& p) {
  if (p.v == floor_p.v) {
    p.d = floor_p.d;
    return;
  }
  Dual fl, fdl, fr, fdr;
  const Dual p0(p.v, 0.0);
  prefun(g, L, p0, fl, fdl);
  prefun(g, R, p0, fr, fdr);
  p.d = -(fl.d + fr.d + ur.d - ul.d) / (fdl.v + fdr.v);
}

// Sect. 2.6 / Toro ch. 4: exact solution of the Riemann problem between the
// primitive states L and R, sampled at x/t = S.
template <class T>
static RiemannResult<T> riemann(double g, T rl, T ul, T pl, T rr, T ur, T pr, double S) {
  RiemannResult<T> out{};
  const Side<T> L{rl, ul, pl, sqrt(g * pl / rl)};
  const Side<T> R{rr, ur, pr, sqrt(g * pr / rr)};
  if (2.0 / (g - 1.0) * (L.c + R.c) <= R.u - L.u) {  // vacuum generated (Toro 4.6)
    out.vacuum = true;
    out.converged = true;
    const T sl_star = L.u + 2.0 * L.c / (g - 1.0);
    const T sr_star = R.u - 2.0 * R.c / (g - 1.0);
    out.pstar = T(0.0);
    out.ustar = T(0.0);
    if (S <= sl_star) {
      out.side = -1;
      if (S <= L.u - L.c) { out.rho = L.rho; out.u = L.u; out.p = L.p; }
      else fan_left(g, L, S, out.rho, out.u, out.p);
    } else if (S >= sr_star) {
      out.side = 1;
      if (S >= R.u + R.c) { out.rho = R.rho; out.u = R.u; out.p = R.p; }
      else fan_right(g, R, S, out.rho, out.u, out.p);
    } else {
      out.side = 0;
      out.rho = out.u = out.p = T(0.0);
    }
    return out;
  }
  // Newton iteration on the star pressure (reading R9)
  const T floor_p = 1e-8 * tmin(pl, pr);
  T p = 0.5 * (pl + pr) - 0.125 * (ur - ul) * (rl + rr) * (L.c + R.c);  // PVRS
  if (p < floor_p) p = floor_p;
  T fl, fdl, fr, fdr;
  int it = 0;
  bool conv = false;
  for (it = 1; it <= 100; ++it) {
    prefun(g, L, p, fl, fdl);
    prefun(g, R, p, fr, fdr);
    T pn = p - (fl + fr + ur - ul) / (fdl + fdr);
    if (pn < floor_p) pn = floor_p;
    const double change = 2.0 * std::fabs(val(pn) - val(p)) / (val(pn) + val(p));
    p = pn;
    if (change <= 1e-12) {
      conv = true;
      break;
    }
  }
  star_tangent(g, L, R, ul, ur, floor_p, p);
  prefun(g, L, p, fl, fdl);
  prefun(g, R, p, fr, fdr);
  const T us = 0.5 * (ul + ur) + 0.5 * (fr - fl);
  out.pstar = p;
  out.ustar = us;
  out.iters = it;
  out.converged = conv;
  // sampling (Toro 4.5)
  if (S <= us) {
    out.side = -1;
    if (p <= pl) {  // left rarefaction
      const T shl = ul - L.c;
      if (S <= shl) { out.rho = rl; out.u = ul; out.p = pl; }
      else {
        const T cml = L.c * pow(p / pl, (g - 1.0) / (2.0 * g));
        const T stl = us - cml;
        if (S > stl) { out.rho = rl * pow(p / pl, 1.0 / g); out.u = us; out.p = p; }
        else fan_left(g, L, S, out.rho, out.u, out.p);
      }
    } else {  // left shock
      const T pml = p / pl;
      const T sl = ul - L.c * sqrt((g + 1.0) / (2.0 * g) * pml + (g - 1.0) / (2.0 * g));
      if (S <= sl) { out.rho = rl; out.u = ul; out.p = pl; }
      else {
        const double g6 = (g - 1.0) / (g + 1.0);
        out.rho = rl * (pml + g6) / (pml * g6 + 1.0);
        out.u = us;
        out.p = p;
      }
    }
  } else {
    out.side = 1;
    if (p > pr) {  // right shock
      const T pmr = p / pr;
      const T sr = ur + R.c * sqrt((g + 1.0) / (2.0 * g) * pmr + (g - 1.0) / (2.0 * g));
      if (S >= sr) { out.rho = rr; out.u = ur; out.p = pr; }
      else {
        const double g6 = (g - 1.0) / (g + 1.0);
        out.rho = rr * (pmr + g6) / (pmr * g6 + 1.0);
        out.u = us;
        out.p = p;
      }
    } else {  // right rarefaction
      const T shr = ur + R.c;
      if (S >= shr) { out.rho = rr; out.u = ur; out.p = pr; }
      else {
        const T cmr = R.c * pow(p / pr, (g - 1.0) / (2.0 * g));
        const T str = us + cmr;
        if (S <= str) { out.rho = rr * pow(p / pr, 1.0 / g); out.u = us; out.p = p; }
        else fan_right(g, R, S, out.rho, out.u, out.p);
      }
    }
  }
  return out;
}

static inline void axes(int ax, int& n, int& t1, int& t2) {
  if (ax == 0) { n = MU; t1 = MV; t2 = MW; }
  else if (ax == 1) { n = MV; t1 = MU; t2 = MW; }
  else { n = MW; t1 = MU; t2 = MV; }
}

// Sect. 2.6: flux F(E*) of the exact Riemann solution at the face, from the
// reconstructed left and right conservative gas states.  Flux components of
// App. B with the energy flux of reading R3.
template <class T>
static void gas_flux(Oracle& o, int ax, const T UL[5], const T UR[5], T F[5]) {
  const double g = o.d.gamma;
  int n, t1, t2;
  axes(ax, n, t1, t2);
  for (int f = 0; f < 5; ++f) F[f] = T(0.0);
  const T rl = UL[RHO], rr = UR[RHO];
  if (!(rl > 0.0) || !(rr > 0.0)) { o.status |= ST_NONPHYSICAL; return; }
  const T pl = pressure(g, UL), pr = pressure(g, UR);
  if (!(pl > 0.0) || !(pr > 0.0)) { o.status |= ST_NONPHYSICAL; return; }
  const RiemannResult<T> s = riemann(g, rl, UL[n] / rl, pl, rr, UR[n] / rr, pr, 0.0);
  o.riemann_calls++;
  o.newton_iters += s.iters;
  if (!s.converged) o.status |= ST_RIEMANN;
  T ut1 = T(0.0), ut2 = T(0.0);
  if (s.side < 0) { ut1 = UL[t1] / rl; ut2 = UL[t2] / rl; }
  else if (s.side > 0) { ut1 = UR[t1] / rr; ut2 = UR[t2] / rr; }
  const T m = s.rho * s.u;
  F[RHO] = m;
  F[n] = m * s.u + s.p;
  F[t1] = m * ut1;
  F[t2] = m * ut2;
  F[EN] = (0.5 * s.rho * (s.u * s.u + ut1 * ut1 + ut2 * ut2) + s.p / (g - 1.0) + s.p) * s.u;
}

// Sect. 2.9 / reading R5: kinetic flux-vector splitting of the pressureless
// dust fluid: what moves right leaves the left state, what moves left leaves
// the right state.
template <class T>
static void dust_flux(int ax, const T* UL, const T* UR, T* F, int b = 5) {  // b: the species' first field
  int n, t1, t2;
  axes(ax, n, t1, t2);
  n += b; t1 += b; t2 += b;
  const int drho = b + 3;
  const T rl = UL[drho], rr = UR[drho];
  T Fs[4] = {T(0.0), T(0.0), T(0.0), T(0.0)};
  if (rl > 0.0) {
    const T ul = UL[n] / rl;
    const T m = rl * (ul > 0.0 ? ul : T(0.0));
    Fs[0] += m; Fs[1] += m * ul; Fs[2] += m * (UL[t1] / rl); Fs[3] += m * (UL[t2] / rl);
  }
  if (rr > 0.0) {
    const T ur = UR[n] / rr;
    const T m = rr * (ur < 0.0 ? ur : T(0.0));
    Fs[0] += m; Fs[1] += m * ur; Fs[2] += m * (UR[t1] / rr); Fs[3] += m * (UR[t2] / rr);
  }
  F[drho] = Fs[0];
  F[n] = Fs[1];
  F[t1] = Fs[2];
  F[t2] = Fs[3];
}

// ---------------------------------------------------------------- sources
// App. B source vector in cylindrical coordinates, with stellar gravity
// (Sect. 2.1) and the rotating-frame terms of reading R6; per unit volume,
// at the cell centre.  gind = X_ref (A_disc, B_disc) of Sect. 2.10 (reading
// R16), or null.  The Box has no source terms.
template <class T>
static void sources(const Oracle& o, int i, int j, int k, const T* U, const T* gind, T* S) {
  for (int f = 0; f < o.nf; ++f) S[f] = T(0.0);
  if (o.d.geometry != GEOM_CYL) return;
  const double r = XC(o, 0, i), z = XC(o, 2, k);
  const double R2 = r * r + z * z;
  const double R3 = R2 * std::sqrt(R2);
  const double fr = -o.d.gm * r / R3, fz = -o.d.gm * z / R3;
  const double Om = o.d.omega_frame;
  // gradient of the indirect potential, (r, theta) components at this cell
  T dphi_r(0.0), dphi_t(0.0);
  if (gind) {
    const double th = XC(o, 1, j);
    dphi_r = gind[0] * std::cos(th) + gind[1] * std::sin(th);
    dphi_t = -gind[0] * std::sin(th) + gind[1] * std::cos(th);
  }
  {
    const T rho = U[RHO];
    const T u = U[MU] / rho, v = U[MV] / rho, w = U[MW] / rho;
    const T P = pressure(o.d.gamma, U);
    S[MU] = rho * v * v / r + P / r + rho * fr + 2.0 * Om * rho * v + rho * Om * Om * r;
    S[MV] = -rho * u * v / r - 2.0 * Om * rho * u;
    S[MW] = rho * fz;
    S[EN] = rho * u * (fr + Om * Om * r) + rho * w * fz;
    S[RHO] = T(0.0);
    if (gind) {
      S[MU] -= rho * dphi_r;
      S[MV] -= rho * dphi_t;
      S[EN] -= rho * (u * dphi_r + v * dphi_t);
    }
  }
  for (int sp = 0; sp < o.nd; ++sp) {
    const int b = 5 + 4 * sp;
    if (!(U[b + 3] > 0.0)) continue;
    const T rho = U[b + 3];
    const T u = U[b] / rho, v = U[b + 1] / rho;
    S[b] = rho * v * v / r + rho * fr + 2.0 * Om * rho * v + rho * Om * Om * r;
    S[b + 1] = -rho * u * v / r - 2.0 * Om * rho * u;
    S[b + 2] = rho * fz;
    S[b + 3] = T(0.0);
    if (gind) {
      S[b] -= rho * dphi_r;
      S[b + 1] -= rho * dphi_t;
    }
  }
}

// Sect. 2.10: X_ref (A_disc, B_disc), the integrals of r' cos(theta') / R'^3
// and r' sin(theta') / R'^3 over the disc mass, as sums over cells of mass
// V (rho - rho_0 + rho_d) at the centre (reading R16).  Zero when off.
template <class Acc, class T = typename Acc::value_type>
static void indirect_moments(const Oracle& o, const Acc& E, T gind[2]) {
  gind[0] = gind[1] = T(0.0);
  if (o.x_ind == 0.0 || o.d.geometry != GEOM_CYL) return;
  T A(0.0), B(0.0);
  for (long lin = 0; lin < o.ncell; ++lin) {
    const int i = (int)(lin % o.n[0]);
    const int j = (int)((lin / o.n[0]) % o.n[1]);
    const int k = (int)(lin / ((long)o.n[0] * o.n[1]));
    const double r = XC(o, 0, i), th = XC(o, 1, j), z = XC(o, 2, k);
    const double R2 = r * r + z * z;
    T dm = E.get(RHO, lin);
    if (o.has_eq) dm = dm - E0C(o, i, k)[RHO];
    for (int sp = 0; sp < o.nd; ++sp) dm += E.get(5 + 4 * sp + 3, lin);
    dm = dm * metric(o, i).V;
    A += dm * (r * std::cos(th) / (R2 * std::sqrt(R2)));
    B += dm * (r * std::sin(th) / (R2 * std::sqrt(R2)));
  }
  gind[0] = o.x_ind * A;
  gind[1] = o.x_ind * B;
}

// Reading R17: relaxation rate R(r) / tau of the wave-killing zones at the
// centre of radial cell i (0 in the interior), plus reading R21's vertical
// rate at the centre of cell (i, k).
static double damping_rate(const Oracle& o, int i, int k) {
  double rate = 0.0;
  const double r = XC(o, 0, i);
  if (o.damp) {
    const double rin = o.d.x0[0], rout = o.d.x1[0];
    if (r < o.damp_ein) {
      const double x = (o.damp_ein - r) / (o.damp_ein - rin);
      rate = x * x / o.damp_tau_in;
    } else if (r > o.damp_eout) {
      const double x = (r - o.damp_eout) / (rout - o.damp_eout);
      rate = x * x / o.damp_tau_out;
    }
  }
  if (o.damp_z) {
    const double az = std::fabs(XC(o, 2, k)), zmax = o.d.x1[2];
    if (az > o.damp_ze) {
      const double x = (az - o.damp_ze) / (zmax - o.damp_ze);
      const double tau = o.damp_zf * 2.0 * M_PI / std::sqrt(o.d.gm / (r * r * r));
      rate += x * x / tau;
    }
  }
  return rate;
}

// ---------------------------------------------------------------- G(E) per cell
// Sect. 2.2, Eq. (compact form): G = S V - sum_faces A F.n, for one cell.
template <class Acc, class T = typename Acc::value_type>
static void G_cell(Oracle& o, const Acc& E, int i, int j, int k, T G[NFMAX], const T* gind = nullptr) {
  const Metric m = metric(o, i);
  for (int f = 0; f < o.nf; ++f) G[f] = T(0.0);
  const int cell[3] = {i, j, k};
  for (int ax = 0; ax < 3; ++ax) {
    T qm_c[NFMAX], qp_c[NFMAX], qm_m[NFMAX], qp_m[NFMAX], qm_p[NFMAX], qp_p[NFMAX];
    int cm[3] = {i, j, k}, cp[3] = {i, j, k};
    cm[ax] -= 1;
    cp[ax] += 1;
    recon(o, E, ax, cm, qm_m, qp_m);
    recon(o, E, ax, cell, qm_c, qp_c);
    recon(o, E, ax, cp, qm_p, qp_p);
    const int c = cell[ax];
    for (int side = 0; side < 2; ++side) {
      const int fc = side == 0 ? c : c + 1;        // face index (lower face of cell fc)
      const T* ql = side == 0 ? qp_m : qp_c;       // left state of the face
      const T* qr = side == 0 ? qm_c : qm_p;       // right state of the face
      double e0[5];
      T UL[NFMAX], UR[NFMAX], F[NFMAX];
      eq_face(o, ax, i, k, fc, e0);
      for (int f = 0; f < 5; ++f) { UL[f] = e0[f] + ql[f]; UR[f] = e0[f] + qr[f]; }
      for (int f = 5; f < o.nf; ++f) { UL[f] = ql[f]; UR[f] = qr[f]; }
      gas_flux(o, ax, UL, UR, F);
      for (int sp = 0; sp < o.nd; ++sp) dust_flux(ax, UL, UR, F, 5 + 4 * sp);
      const double A = side == 0 ? m.A_lo[ax] : m.A_hi[ax];
      for (int f = 0; f < o.nf; ++f) G[f] += side == 0 ? A * F[f] : -A * F[f];
    }
  }
  T U[NFMAX], S[NFMAX];
  for (int f = 0; f < NFMAX; ++f) U[f] = T(0.0);
  const long lin = ((long)k * o.n[1] + j) * o.n[0] + i;
  for (int f = 0; f < o.nf; ++f) U[f] = E.get(f, lin);
  if (!(U[RHO] > 0.0) || !(pressure(o.d.gamma, U) > 0.0)) o.status |= ST_NONPHYSICAL;
  for (int sp = 0; sp < o.nd; ++sp)
    if (U[5 + 4 * sp + 3] < 0.0) o.status |= ST_NONPHYSICAL;
  sources(o, i, j, k, U, gind, S);
  for (int f = 0; f < o.nf; ++f) G[f] += m.V * S[f];
  const double kd = damping_rate(o, i, k);  // readings R17, R21
  if (kd != 0.0)
    for (int f = 0; f < 5; ++f) G[f] -= m.V * kd * (U[f] - (o.has_eq ? E0C(o, i, k)[f] : 0.0));
}

// ---------------------------------------------------------------- drag
template <class T>
struct DustParamsT {
  T stokes;
  int drag_law;  // 0: constant Stokes number St = t_s Omega_K(r); 1: Epstein, St fixed at (r=1, z=0);
                 // 2: Epstein with the Stokes regime above r_p = 9 lambda / 4 (reading R19)
};
using DustParams = DustParamsT<double>;
// Sect. 2.9 stopping time of dust species `sp` (Stokes number St x
// st_factor[sp]) in a cell of radial index i with gas state U.
template <class T>
static T stopping_time(const Oracle& o, int i, const T* U, const DustParamsT<T>& dp, int sp) {
  const T st = sp == 0 ? dp.stokes : dp.stokes * o.st_factor[sp];
  const T rg = U[RHO];
  if (dp.drag_law == 0)
    return o.d.geometry == GEOM_CYL ? st / std::sqrt(o.d.gm / std::pow(XC(o, 0, i), 3)) : st;
  // Epstein t_s = rho_s r_p / (rho_g c_s), with rho_s r_p fixed so that St holds at r = 1, z = 0
  double rho1, vth1, p1;
  eq_prim(o, 1.0, 0.0, rho1, vth1, p1);
  const T rhos_rp = st * rho1 * std::sqrt(o.d.gamma * p1 / rho1) / std::sqrt(o.d.gm);
  const T cs = sqrt(o.d.gamma * pressure(o.d.gamma, U) / rg);
  T ts = rhos_rp / (rg * cs);
  // r_p / lambda = kappa rho_g; the Stokes regime lengthens t_s by (4/9) r_p / lambda
  if (dp.drag_law == 2 && o.kappa * rg > 2.25) ts = ts * ((4.0 / 9.0) * (o.kappa * rg));
  return ts;
}

// Sect. 2.9 drag law with the semi-implicit integration of reading R7.  One
// species: the relative velocity relaxes in closed form at a fixed
// barycentric velocity.  Several (reading R20): the backward-Euler system
// rho_g v_g' = rho_g v_g + sum_k rho_k (v_k' - v_g') a_k,
// v_k' = v_k - (v_k' - v_g') a_k (a_k = tau / t_k, no dust-dust exchange) is
// solved in closed form, v_k' - v_g' = (v_k - v_g') / (1 + a_k); the gas
// energy gains the work of the drag on the gas in both.
template <class T>
static void drag(const Oracle& o, int i, T* U, double tau, const DustParamsT<T>& dp, double theta = 1.0) {
  if (o.nd == 0) return;
  const T rg = U[RHO];
  if (o.nd > 1) {
    if (!(rg > 0.0)) return;
    T a[ND_MAX], num[3], den = rg;
    for (int c = 0; c < 3; ++c) num[c] = U[MU + c];
    for (int sp = 0; sp < o.nd; ++sp) {
      const int b = 5 + 4 * sp;
      a[sp] = T(0.0);
      if (!(U[b + 3] > 0.0)) continue;
      a[sp] = theta * tau / stopping_time(o, i, U, dp, sp);
      const T w = a[sp] / (1.0 + a[sp]);
      den += U[b + 3] * w;
      for (int c = 0; c < 3; ++c) num[c] += U[b + c] * w;  // rho_k v_k a_k / (1 + a_k)
    }
    // backward Euler over theta tau; the theta-method's step is then
    // v' = (v_BE - (1 - theta) v) / theta (trapezoidal for theta = 1/2)
    T dE = T(0.0);
    for (int c = 0; c < 3; ++c) {
      const T vg_ex = U[MU + c] / rg;
      const T vg = (num[c] / den - (1.0 - theta) * vg_ex) / theta;
      for (int sp = 0; sp < o.nd; ++sp) {
        const int b = 5 + 4 * sp;
        if (!(U[b + 3] > 0.0)) continue;
        const T vk = U[b + c] / U[b + 3];
        U[b + c] = U[b + 3] * (((vk + a[sp] * (num[c] / den)) / (1.0 + a[sp]) - (1.0 - theta) * vk) / theta);
      }
      U[MU + c] = rg * vg;
      dE += 0.5 * rg * (vg * vg - vg_ex * vg_ex);
    }
    U[EN] += dE;
    return;
  }
  const T rd = U[DRHO];
  if (!(rd > 0.0) || !(rg > 0.0)) return;
  const T ts = stopping_time(o, i, U, dp, 0);
  const T eps = rd / rg;
  const T kk = tau * (1.0 + eps) / ts;
  const T mu = rg * rd / (rg + rd);
  T dE = T(0.0);
  for (int c = 0; c < 3; ++c) {
    const T vg_ex = U[MU + c] / rg;
    const T vd_ex = U[DMU + c] / rd;
    const T X = mu * (vd_ex - vg_ex) * (kk / (1.0 + theta * kk));  // theta-method; 1 = backward Euler
    U[MU + c] += X;
    U[DMU + c] -= X;
    dE += 0.5 * X * (U[MU + c] / rg + vg_ex);
  }
  U[EN] += dE;
}

// One RK stage at one cell: Eout = Ebase + tau G(Ein)/V, then drag (Sect. 2.5).
template <class Acc, class T = typename Acc::value_type>
static void stage_cell(Oracle& o, const Acc& Ein, const T* Ebase, long lin, double tau, const DustParamsT<T>& dp,
                       T out[NFMAX], const T* gind = nullptr) {
  const int i = (int)(lin % o.n[0]);
  const int j = (int)((lin / o.n[0]) % o.n[1]);
  const int k = (int)(lin / ((long)o.n[0] * o.n[1]));
  T G[NFMAX];
  G_cell(o, Ein, i, j, k, G, gind);
  if (!o.r0.empty())
    for (int f = 0; f < o.nf; ++f) G[f] -= o.r0[(size_t)f * o.ncell + lin];  // Sect. 2.8 balanced scheme
  const double V = metric(o, i).V;
  for (int f = 0; f < o.nf; ++f) out[f] = Ebase[(size_t)f * o.ncell + lin] + tau * G[f] / V;
  if (o.drag_scheme == DRAG_IN_STAGES) drag(o, i, out, tau, dp);
}

// Option 1 of reading R7: half a step of trapezoidal drag on every cell.
template <class T>
static void half_drag_all(const Oracle& o, T* E, double dt, const DustParamsT<T>& dp) {
  T U[NFMAX];
  for (long lin = 0; lin < o.ncell; ++lin) {
    for (int f = 0; f < o.nf; ++f) U[f] = E[(size_t)f * o.ncell + lin];
    drag(o, (int)(lin % o.n[0]), U, 0.5 * dt, dp, 0.5);
    for (int f = 0; f < o.nf; ++f) E[(size_t)f * o.ncell + lin] = U[f];
  }
}

template <class T>
static void stage_all(Oracle& o, const T* Ein, const T* Ebase, T* Eout, double tau, const DustParamsT<T>& dp) {
  const ArrAccT<T> A{Ein, o.ncell};
  T out[NFMAX], gind[2];
  indirect_moments(o, A, gind);
  const bool ind = o.x_ind != 0.0 && o.d.geometry == GEOM_CYL;
  for (long lin = 0; lin < o.ncell; ++lin) {
    stage_cell(o, A, Ebase, lin, tau, dp, out, ind ? gind : nullptr);
    for (int f = 0; f < o.nf; ++f) Eout[(size_t)f * o.ncell + lin] = out[f];
  }
}

// Stage-1 state E* evaluated lazily, one cell at a time, for sampled checks.
struct LazyStageAcc {
  using value_type = double;
  Oracle* o;
  const double* En;
  double tau;
  DustParams dp;
  mutable std::unordered_map<long, std::array<double, NFMAX>> cache;
  double get(int f, long lin) const {
    auto it = cache.find(lin);
    if (it == cache.end()) {
      std::array<double, NFMAX> v{};
      const ArrAcc A{En, o->ncell};
      stage_cell(*o, A, En, lin, tau, dp, v.data());
      it = cache.emplace(lin, v).first;
    }
    return it->second[f];
  }
};

static double cell_dt(const Oracle& o, const double* U, int i) {
  const Metric m = metric(o, i);
  const double rho = U[RHO];
  const double vel = sqrt(U[MU] * U[MU] + U[MV] * U[MV] + U[MW] * U[MW]) / rho;
  const double cs = sqrt(o.d.gamma * pressure(o.d.gamma, U) / rho);
  double dt = o.d.cfl * m.V / ((vel + cs) * m.maxA);  // Sect. 2.5, Eq. (cfl condition)
  for (int sp = 0; sp < o.nd; ++sp) {
    const int b = 5 + 4 * sp;
    if (!(U[b + 3] > 0.0)) continue;
    const double vd = sqrt(U[b] * U[b] + U[b + 1] * U[b + 1] + U[b + 2] * U[b + 2]) / U[b + 3];
    if (vd > 0.0) dt = std::min(dt, o.d.cfl * m.V / (vd * m.maxA));
  }
  return dt;
}

static void build_tables(Oracle& o) {
  const int nrx = o.n[0] + 2 * NG, nzx = o.n[2] + 2 * NG;
  o.e0c.assign((size_t)nzx * nrx * 5, 0.0);
  o.e0r.assign((size_t)nzx * (nrx + 1) * 5, 0.0);
  o.e0z.assign((size_t)(nzx + 1) * nrx * 5, 0.0);
  if (!o.has_eq) return;
  for (int k = -NG; k < o.n[2] + NG; ++k)
    for (int i = -NG; i < o.n[0] + NG; ++i)
      eq_cons(o, XC(o, 0, i), XC(o, 2, k), &o.e0c[((size_t)(k + NG) * nrx + (i + NG)) * 5]);
  for (int k = -NG; k < o.n[2] + NG; ++k)
    for (int i = -NG; i <= o.n[0] + NG; ++i)
      eq_cons(o, XF(o, 0, i), XC(o, 2, k), &o.e0r[((size_t)(k + NG) * (nrx + 1) + (i + NG)) * 5]);
  for (int k = -NG; k <= o.n[2] + NG; ++k)
    for (int i = -NG; i < o.n[0] + NG; ++i)
      eq_cons(o, XC(o, 0, i), XF(o, 2, k), &o.e0z[((size_t)(k + NG) * nrx + (i + NG)) * 5]);
}

static void equilibrium_state(const Oracle& o, double* E) {
  for (long lin = 0; lin < o.ncell; ++lin) {
    const int i = (int)(lin % o.n[0]);
    const int k = (int)(lin / ((long)o.n[0] * o.n[1]));
    for (int f = 0; f < o.nf; ++f) E[(size_t)f * o.ncell + lin] = (f < 5 && o.has_eq) ? E0C(o, i, k)[f] : 0.0;
  }
}

}  // namespace orc

using namespace orc;

extern "C" {

void* orc_create(const Desc* d) {
  Oracle* o = new Oracle();
  o->d = *d;
  o->n[0] = d->nr;
  o->n[1] = d->nth;
  o->n[2] = d->nz;
  o->nd = std::max(0, std::min(d->n_dust, ND_MAX));
  o->nf = 5 + 4 * o->nd;
  o->ncell = (long)d->nr * d->nth * d->nz;
  for (int ax = 0; ax < 3; ++ax) {
    o->xc[ax].resize(o->n[ax] + 2 * NG);
    o->xf[ax].resize(o->n[ax] + 2 * NG + 1);
    for (int c = -NG; c < o->n[ax] + NG; ++c) o->xc[ax][c + NG] = centre_coord(*o, ax, c);
    for (int c = -NG; c <= o->n[ax] + NG; ++c) o->xf[ax][c + NG] = face_coord(*o, ax, c);
  }
  build_tables(*o);
  return o;
}

void orc_destroy(void* h) { delete (Oracle*)h; }

int orc_nfields(void* h) { return ((Oracle*)h)->nf; }

// Sets the disc equilibrium (App. A) and runs the empty run of Sect. 2.8.
// disc = {sigma0, beta_sigma, T0, beta_T, bump_delta, bump_r0, bump_width}
// (bump_delta = 0: no bump), or NULL for no equilibrium.
int orc_set_equilibrium(void* h, const double* disc) {
  Oracle& o = *(Oracle*)h;
  o.has_eq = disc != nullptr;
  if (disc) {
    o.sigma0 = disc[0];
    o.beta_sigma = disc[1];
    o.T0 = disc[2];
    o.beta_T = disc[3];
    o.bump_delta = disc[4];
    o.bump_r0 = disc[5];
    o.bump_width = disc[6];
  }
  build_tables(o);
  o.r0.clear();
  if (!o.has_eq) return 0;
  std::vector<double> E0((size_t)o.nf * o.ncell), R((size_t)o.nf * o.ncell);
  equilibrium_state(o, E0.data());
  const ArrAcc A{E0.data(), o.ncell};
  double G[NFMAX];
  for (long lin = 0; lin < o.ncell; ++lin) {
    const int i = (int)(lin % o.n[0]);
    const int j = (int)((lin / o.n[0]) % o.n[1]);
    const int k = (int)(lin / ((long)o.n[0] * o.n[1]));
    G_cell(o, A, i, j, k, G);
    for (int f = 0; f < o.nf; ++f) R[(size_t)f * o.ncell + lin] = G[f];
  }
  o.r0.swap(R);
  const int st = o.status;
  o.status = 0;
  return st;
}

void orc_equilibrium_state(void* h, double* E) { equilibrium_state(*(Oracle*)h, E); }

void orc_eq_prim(void* h, double r, double z, double* out) {
  eq_prim(*(Oracle*)h, r, z, out[0], out[1], out[2]);
}

void orc_coords(void* h, int ax, double* centres, double* faces) {
  const Oracle& o = *(Oracle*)h;
  for (int c = 0; c < o.n[ax] + 2 * NG; ++c) centres[c] = o.xc[ax][c];
  for (int c = 0; c <= o.n[ax] + 2 * NG; ++c) faces[c] = o.xf[ax][c];
}

void orc_metric(void* h, int i, double* out /* V, A_lo[3], A_hi[3], maxA */) {
  const Metric m = metric(*(Oracle*)h, i);
  out[0] = m.V;
  for (int a = 0; a < 3; ++a) { out[1 + a] = m.A_lo[a]; out[4 + a] = m.A_hi[a]; }
  out[7] = m.maxA;
}

// Balanced right-hand side G(E) - R0 for every cell (no drag).
int orc_rhs(void* h, const double* E, double* G) {
  Oracle& o = *(Oracle*)h;
  const ArrAcc A{E, o.ncell};
  double g[NFMAX], gind[2];
  indirect_moments(o, A, gind);
  const bool ind = o.x_ind != 0.0 && o.d.geometry == GEOM_CYL;
  for (long lin = 0; lin < o.ncell; ++lin) {
    const int i = (int)(lin % o.n[0]);
    const int j = (int)((lin / o.n[0]) % o.n[1]);
    const int k = (int)(lin / ((long)o.n[0] * o.n[1]));
    G_cell(o, A, i, j, k, g, ind ? gind : nullptr);
    for (int f = 0; f < o.nf; ++f)
      G[(size_t)f * o.ncell + lin] = g[f] - (o.r0.empty() ? 0.0 : o.r0[(size_t)f * o.ncell + lin]);
  }
  const int st = o.status;
  o.status = 0;
  return st;
}

int orc_stage(void* h, const double* Ein, const double* Ebase, double* Eout, double tau, double stokes, int law) {
  Oracle& o = *(Oracle*)h;
  stage_all(o, Ein, Ebase, Eout, tau, DustParams{stokes, law});
  const int st = o.status;
  o.status = 0;
  return st;
}

// Sect. 2.5: midpoint RK2, E^{n+1} = E^n + dt G(E^n + dt/2 G(E^n)/V)/V, in place.
int orc_step(void* h, double* E, double dt, double stokes, int law) {
  Oracle& o = *(Oracle*)h;
  const DustParams dp{stokes, law};
  std::vector<double> Es((size_t)o.nf * o.ncell), En((size_t)o.nf * o.ncell);
  if (o.drag_scheme == DRAG_STRANG_TRAPEZOIDAL) half_drag_all(o, E, dt, dp);
  stage_all(o, E, E, Es.data(), 0.5 * dt, dp);
  stage_all(o, Es.data(), E, En.data(), dt, dp);
  if (o.drag_scheme == DRAG_STRANG_TRAPEZOIDAL) half_drag_all(o, En.data(), dt, dp);
  std::memcpy(E, En.data(), sizeof(double) * En.size());
  const int st = o.status;
  o.status = 0;
  return st;
}

// Tangent-linear step: E^{n+1} and its directional derivative dE^{n+1} along
// the direction (dE^n, dSt) in state and Stokes number, at a fixed dt; every
// branch (limiter, Riemann wave pattern, sampling, positivity) is the one the
// values take.  E and dE are updated in place.
int orc_step_tlm(void* h, double* E, double* dE, double dt, double stokes, double dstokes, int law) {
  Oracle& o = *(Oracle*)h;
  const DustParamsT<Dual> dp{Dual(stokes, dstokes), law};
  const size_t n = (size_t)o.nf * o.ncell;
  std::vector<Dual> X(n), Es(n), En(n);
  for (size_t q = 0; q < n; ++q) X[q] = Dual(E[q], dE[q]);
  if (o.drag_scheme == DRAG_STRANG_TRAPEZOIDAL) half_drag_all(o, X.data(), dt, dp);
  stage_all(o, X.data(), X.data(), Es.data(), 0.5 * dt, dp);
  stage_all(o, Es.data(), X.data(), En.data(), dt, dp);
  if (o.drag_scheme == DRAG_STRANG_TRAPEZOIDAL) half_drag_all(o, En.data(), dt, dp);
  for (size_t q = 0; q < n; ++q) {
    E[q] = En[q].v;
    dE[q] = En[q].d;
  }
  const int st = o.status;
  o.status = 0;
  return st;
}

// One RK2 step evaluated only at the listed cells (linear indices); out is
// ncells x nf.  E* is evaluated lazily on the neighbourhood the stencil needs.
int orc_step_sampled(void* h, const double* E, double dt, double stokes, int law, const long* cells, long ncells,
                     double* out) {
  Oracle& o = *(Oracle*)h;
  if (o.x_ind != 0.0) return -1;  // the indirect term needs the whole of E*
  if (o.drag_scheme != DRAG_IN_STAGES) return -1;  // sampled steps follow the default drag
  const DustParams dp{stokes, law};
  LazyStageAcc S{&o, E, 0.5 * dt, dp, {}};
  for (long s = 0; s < ncells; ++s) stage_cell(o, S, E, cells[s], dt, dp, out + (size_t)s * o.nf);
  const int st = o.status;
  o.status = 0;
  return st;
}

double orc_cfl_dt(void* h, const double* E) {
  const Oracle& o = *(Oracle*)h;
  double dt = INFINITY, U[NFMAX];
  for (long lin = 0; lin < o.ncell; ++lin) {
    for (int f = 0; f < o.nf; ++f) U[f] = E[(size_t)f * o.ncell + lin];
    dt = std::min(dt, cell_dt(o, U, (int)(lin % o.n[0])));
  }
  return dt;
}

void orc_sums(void* h, const double* E, double* sums) {
  const Oracle& o = *(Oracle*)h;
  for (int f = 0; f < o.nf; ++f) {
    double s = 0.0;
    for (long lin = 0; lin < o.ncell; ++lin) s += metric(o, (int)(lin % o.n[0])).V * E[(size_t)f * o.ncell + lin];
    sums[f] = s;
  }
}

// X_ref of the indirect-gravity term of Sect. 2.10 (reading R16); 0 = off.
void orc_set_indirect(void* h, double x_ref) { ((Oracle*)h)->x_ind = x_ref; }

// X_ref (A_disc, B_disc) of the state E (zero when off or on the Box).
void orc_indirect(void* h, const double* E, double* out) {
  const Oracle& o = *(Oracle*)h;
  indirect_moments(o, ArrAcc{E, o.ncell}, out);
}

// Wave-killing zones of reading R17: edges r_ein (inner zone r < r_ein) and
// r_eout (outer zone r > r_eout), tau = f x the orbital period 2 pi / Omega_K
// at each boundary; f <= 0 switches them off.  Cylindrical grids only.
int orc_set_damping(void* h, double r_ein, double r_eout, double f) {
  Oracle& o = *(Oracle*)h;
  o.damp = false;
  if (!(f > 0.0)) return 0;
  const double rin = o.d.x0[0], rout = o.d.x1[0];
  if (o.d.geometry != GEOM_CYL || !(r_ein > rin) || !(r_eout < rout) || !(r_ein <= r_eout)) return 1;
  o.damp = true;
  o.damp_ein = r_ein;
  o.damp_eout = r_eout;
  o.damp_tau_in = f * 2.0 * M_PI / std::sqrt(o.d.gm / (rin * rin * rin));
  o.damp_tau_out = f * 2.0 * M_PI / std::sqrt(o.d.gm / (rout * rout * rout));
  return 0;
}

// Vertical sheared damped boundary of reading R21: |z| > z_edge relaxes the
// gas departures with tau = f x the local orbital period; f <= 0 switches it
// off.  Cylindrical grids symmetric about z = 0 only.
int orc_set_vertical_damping(void* h, double z_edge, double f) {
  Oracle& o = *(Oracle*)h;
  o.damp_z = false;
  if (!(f > 0.0)) return 0;
  if (o.d.geometry != GEOM_CYL || !(o.d.x0[2] == -o.d.x1[2]) || !(z_edge >= 0.0) || !(z_edge < o.d.x1[2])) return 1;
  o.damp_z = true;
  o.damp_ze = z_edge;
  o.damp_zf = f;
  return 0;
}

// Relaxation rate of the damping zones (readings R17, R21) at cell (i, k).
double orc_damping_rate(void* h, int i, int k) { return damping_rate(*(Oracle*)h, i, k); }

// App. B source vector per unit volume of the state U (nf values) at the
// centre of cell (i, j, k), without the indirect term.
void orc_sources(void* h, int i, int j, int k, const double* U, double* S) {
  const Oracle& o = *(Oracle*)h;
  double u[NFMAX] = {0}, s[NFMAX];
  for (int f = 0; f < o.nf; ++f) u[f] = U[f];
  sources(o, i, j, k, u, (const double*)nullptr, s);
  for (int f = 0; f < o.nf; ++f) S[f] = s[f];
}

// Stokes-number factors of the dust species (reading R20): species k has
// St x f[k]; species 0 always has St itself.
void orc_set_species_stokes(void* h, const double* f, int n) {
  Oracle& o = *(Oracle*)h;
  for (int k = 1; k < n && k < ND_MAX; ++k) o.st_factor[k] = f[k];
}

// Gas reconstruction of reading R2: 0 = conservative departures (Sect. 2.7
// on App. B's E; the default), 1 = primitive departures, 2 = the pressure
// departure in place of the energy one.
int orc_set_recon(void* h, int mode) {
  if (mode != RECON_CONSERVATIVE && mode != RECON_PRIMITIVE && mode != RECON_PRESSURE) return 1;
  ((Oracle*)h)->recon = mode;
  return 0;
}

// Dust reconstruction of reading R5: 0 = the parabola on rho_d and the
// velocity (the default), 1 = the velocity flat at a converging density
// maximum.
int orc_set_dust_recon(void* h, int mode) {
  if (mode != DUST_RECON_PARABOLA && mode != DUST_RECON_FLAT_AT_SPIKES) return 1;
  ((Oracle*)h)->dust_recon = mode;
  return 0;
}

// Drag integration of reading R7: 0 = backward Euler after each RK2 stage
// (the default), 1 = Strang splitting with trapezoidal half steps.
int orc_set_drag_scheme(void* h, int mode) {
  if (mode != DRAG_IN_STAGES && mode != DRAG_STRANG_TRAPEZOIDAL) return 1;
  ((Oracle*)h)->drag_scheme = mode;
  return 0;
}

// Reconstructed face states of cell (i, j, k) along axis ax: the full
// conservative states (E0 + q) on its lower (Um) and upper (Up) faces, nf
// values each (dust: the reconstructed dust fields).
void orc_recon_faces(void* h, const double* E, int ax, int i, int j, int k, double* Um, double* Up) {
  const Oracle& o = *(Oracle*)h;
  const ArrAcc A{E, o.ncell};
  const int cell[3] = {i, j, k};
  double qm[NFMAX], qp[NFMAX], e0m[5], e0p[5];
  recon(o, A, ax, cell, qm, qp);
  eq_face(o, ax, i, k, cell[ax], e0m);
  eq_face(o, ax, i, k, cell[ax] + 1, e0p);
  for (int f = 0; f < o.nf; ++f) {
    Um[f] = f < 5 ? e0m[f] + qm[f] : qm[f];
    Up[f] = f < 5 ? e0p[f] + qp[f] : qp[f];
  }
}

// kappa = r_p / lambda_0 of the Stokes regime of drag law 2 (reading R19);
// kappa <= 0 keeps every cell in the Epstein regime.
void orc_set_stokes_regime(void* h, double kappa) { ((Oracle*)h)->kappa = kappa; }

void orc_counters(void* h, long* out) {
  const Oracle& o = *(Oracle*)h;
  out[0] = o.riemann_calls;
  out[1] = o.newton_iters;
}

// ---- single-function entry points used by the pins ----
int orc_riemann(double gamma, const double* WL, const double* WR, double S, double* W, double* star) {
  const RiemannResult r = riemann(gamma, WL[0], WL[1], WL[2], WR[0], WR[1], WR[2], S);
  W[0] = r.rho;
  W[1] = r.u;
  W[2] = r.p;
  star[0] = r.pstar;
  star[1] = r.ustar;
  star[2] = r.iters;
  star[3] = r.converged ? 1.0 : 0.0;
  star[4] = r.side;
  return r.vacuum ? 1 : 0;
}

int orc_parabola(double em, double e0, double ep, double xm, double x0, double xp, double fm, double fp,
                 double* q) {
  return parabola(em, e0, ep, xm, x0, xp, fm, fp, q[0], q[1]) ? 1 : 0;
}

void orc_gas_flux(void* h, int ax, const double* UL, const double* UR, double* F) {
  gas_flux(*(Oracle*)h, ax, UL, UR, F);
}

// UL, UR, F: the four dust fields (rho_d u_d, rho_d v_d, rho_d w_d, rho_d).
void orc_dust_flux(int ax, const double* UL, const double* UR, double* F) {
  double F9[NFMAX] = {0}, L9[NFMAX] = {0}, R9[NFMAX] = {0};
  for (int f = 0; f < 4; ++f) { L9[5 + f] = UL[f]; R9[5 + f] = UR[f]; }
  dust_flux(ax, L9, R9, F9);
  for (int f = 5; f < 9; ++f) F[f - 5] = F9[f];
}

void orc_drag(void* h, int i, double* U, double tau, double stokes, int law) {
  drag(*(Oracle*)h, i, U, tau, DustParams{stokes, law});
}

int orc_status(void* h) {
  Oracle& o = *(Oracle*)h;
  const int st = o.status;
  o.status = 0;
  return st;
}

}  // extern "C"
