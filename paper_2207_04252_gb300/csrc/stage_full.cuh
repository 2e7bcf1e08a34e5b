// Fused RK2 stage kernel of the FP64 (full conservative state) form.
//
// One CTA owns a TR x TT x TZ tile of cells.  It stages the tile and a 2-deep
// halo along each axis into shared memory as deviations from the equilibrium
// (Sect. 2.7: the conservative departures E' = E - E0 of the gas, or with
// RC = RECON_PRIM the primitive departures u', v', w', P', rho'), then
// sweeps the three directions.  In a sweep, lines along the
// direction map onto groups of L = pow2(T + 2) lanes: lane p reconstructs cell
// p - 1 (parabola + MinMod), receives the upper face state of its lower
// neighbour by a shuffle, solves the exact Riemann problem on its lower face
// (Sect. 2.6) and the dust flux, and receives the flux of its upper face by a
// second shuffle, so each face is solved once per tile.  The flux divergence
// is accumulated in shared memory; the epilogue adds the sources (App. B),
// subtracts the balanced residual R0 (Sect. 2.8), applies the RK stage update
// (Sect. 2.5) and the semi-implicit drag (Sect. 2.9), and in stage 2 fuses the
// CFL minimum and the FP64 conservation partial sums of the new state.
#pragma once
#include "device_common.cuh"

namespace rossbi {

struct StageArgs {
  DevGrid g;
  const double* in[NF_MAX];    // stage input (stencil) state
  const double* base[NF_MAX];  // E^n, base of the update
  double* out[NF_MAX];         // updated state
  double* gout;            // mode 1: G(E) - R0 written here, [nf][ncell]
  double dt_host;
  const unsigned long long* dt_dev;  // if set, dt is read from this device slot
  double tau_frac;                   // 0.5 (stage 1) or 1.0 (stage 2)
  DragArgs drag;
  int stage2;                        // fuse CFL of the output and conservation partials
  double* partials;                  // stage 2: [nf + 1][gridDim.x] block sums of V*E, then block dt minima
  unsigned* status;
  int mode;                          // 0 update, 1 residual only (empty run)
  int tiles_r, tiles_z;  // tile counts along r and z (block -> tile: r fastest, then z, then theta)
};

template <class T>
__device__ __forceinline__ T minmod(T a, T b) {
  if (a * b <= T(0)) return T(0);
  return fabs(a) < fabs(b) ? a : b;
}

// Parabola through three deviations (Sect. 2.7) with the MinMod limiter: each
// face deviation is limited to minmod(deviation, s h), s the minmod slope and
// h the signed limiter reach of that side.  w = {1/(x0-xm), 1/(xp-x0),
// 1/(xp-xm), x0-xm, xp-x0, fm-x0, fp-x0, h-, h+}.  Returns false if flat.
template <class T>
__device__ __forceinline__ bool parabola(T em, T e0, T ep, const T* w, T& qm, T& qp) {
  const T sm = (e0 - em) * w[0];
  const T sp = (ep - e0) * w[1];
  const T s = minmod(sm, sp);
  const T a = (sp - sm) * w[2];
  const T b = (sp * w[3] + sm * w[4]) * w[2];
  qm = e0 + minmod(w[5] * (a * w[5] + b), s * w[7]);
  qp = e0 + minmod(w[6] * (a * w[6] + b), s * w[8]);
  return s != T(0);
}

// Parabola weights of a cell along axis D (axis 0 from the table, uniform axes closed form).
template <class T, int D>
__device__ __forceinline__ void parabola_weights(const T* rcoef, int gi, int nr, T h, T* w) {
  if (D == 0) {
    const int c = gi < -1 ? -1 : (gi > nr ? nr : gi);
    const T* cw = rcoef + (c + 1) * RCW;
#pragma unroll
    for (int q = 0; q < 9; ++q) w[q] = cw[q];
  } else {
    w[0] = w[1] = T(1) / h;
    w[2] = T(0.5) / h;
    w[3] = w[4] = h;
    w[5] = T(-0.5) * h;
    w[6] = T(0.5) * h;
    w[7] = -h;
    w[8] = h;
  }
}

// Primitive dust reconstruction (u, v, w, rho_d) of the cell at s (stride S
// along the sweep) from the conservative shared-memory fields b .. b + 3 of
// one dust species (momenta, then density).
template <class T, int BOX, int S>
__device__ __forceinline__ void dust_recon(const T* sE, int sidx, int b, const T* w, T* wm, T* wp) {
  T pm[4], p0[4], pp[4];
  const T* r = sE + (b + 3) * BOX + sidx;
  pm[3] = r[-S];
  p0[3] = r[0];
  pp[3] = r[S];
  const T im = pm[3] > T(0) ? T(1) / pm[3] : T(0);
  const T i0 = p0[3] > T(0) ? T(1) / p0[3] : T(0);
  const T ip = pp[3] > T(0) ? T(1) / pp[3] : T(0);
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const T* m = sE + (b + c) * BOX + sidx;
    pm[c] = m[-S] * im;
    p0[c] = m[0] * i0;
    pp[c] = m[S] * ip;
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) parabola(pm[q], p0[q], pp[q], w, wm[q], wp[q]);
}

// Ghost rule of Sect. 2.4 for a cell index possibly outside the domain.
// Returns false for an equilibrium ghost (E' = 0).
__device__ __forceinline__ bool resolve_cell(const DevGrid& g, int c[3]) {
  const int n[3] = {g.nr, g.nth, g.nz};
#pragma unroll
  for (int ax = 0; ax < 3; ++ax) {
    if (c[ax] >= 0 && c[ax] < n[ax]) continue;
    const int bc = c[ax] < 0 ? g.bc_lo[ax] : g.bc_hi[ax];
    if (bc == BC_EQUILIBRIUM) return false;
    if (bc == BC_PERIODIC) {
      c[ax] %= n[ax];
      if (c[ax] < 0) c[ax] += n[ax];
    } else {
      c[ax] = c[ax] < 0 ? 0 : n[ax] - 1;
    }
  }
  return true;
}

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

template <int NF, int TR, int TT, int TZ, int NT, int D, int RC>
__device__ __forceinline__ void sweep_full(const StageArgs& a, const double* sE, double* sG, int i0, int j0, int k0,
                                           unsigned& status) {
  constexpr int ZH = TZ == 1 ? 0 : 2;  // z halo (none in the flat one-z-cell tile)
  constexpr int BX = TR + 4, BY = TT + 4, BZ = TZ + 2 * ZH, BOX = BX * BY * BZ, NCORE = TR * TT * TZ;
  constexpr int TD = D == 0 ? TR : (D == 1 ? TT : TZ);
  constexpr int L = pow2ceil(TD + 2);
  static_assert(L <= 32, "line does not fit a warp");
  constexpr int NA = D == 0 ? TT : TR;
  constexpr int NB = D == 2 ? TT : TZ;
  constexpr int ITEMS = NA * NB * L;
  constexpr int STRIDE = D == 0 ? 1 : (D == 1 ? BX : BX * BY);
  constexpr int NW = NT / 32;
  constexpr unsigned FULL = 0xffffffffu;
  const DevGrid& g = a.g;
  const double gam = g.gamma;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int base = warp * 32; base < ITEMS; base += NW * 32) {
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
    const int sidx = do_recon ? ((z + ZH) * BY + (y + 2)) * BX + (x + 2) : (ZH * BY + 2) * BX + 2;

    // parabola weights of this cell along D
    double w[9];
    parabola_weights<double, D>(g.rcoef, gi, g.nr, g.dx[D], w);
    // equilibrium gas state (conservative, or primitive with RC = RECON_PRIM)
    // on the lower face of this cell (index along D = gd) and on its upper
    // face; table indices clamped
    const int ci = clampi(gi, 0, g.nr - 1), ck = clampi(gk, 0, g.nz - 1);
    auto eq_face = [&](int f, int fd) -> double {
      if (!g.has_eq) return 0.0;
      const double* tc = RC == RECON_PRIM ? g.w0c : g.e0c;
      const double* tr = RC == RECON_PRIM ? g.w0r : g.e0r;
      const double* tz = RC == RECON_PRIM ? g.w0z : g.e0z;
      if (D == 0) return tr[((size_t)f * g.nz + ck) * (g.nr + 1) + clampi(fd, 0, g.nr)];
      if (D == 1) return tc[((size_t)f * g.nz + ck) * g.nr + ci];
      return tz[((size_t)f * (g.nz + 1) + clampi(fd, 0, g.nz)) * g.nr + ci];
    };
    double area = 0.0;
    if (do_face) area = D == 0 ? g.area_r[clampi(gi, 0, g.nr)] : (D == 1 ? g.area_t[ci] : g.area_z[ci]);

    // ---------------- gas: departures in slots 0..4
    {
      double qm[5], qp[5];
      bool shaped = false;
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        const double* s = sE + f * BOX + sidx;
        shaped |= parabola(s[-STRIDE], s[0], s[STRIDE], w, qm[f], qp[f]);
      }
      double F[5];
      if (RC == RECON_PRIM) {
        if (shaped && do_recon) {  // positivity of both reconstructed face states
          const bool ok = eq_face(RHO, gd) + qm[RHO] > 0.0 && eq_face(RHO, gd + 1) + qp[RHO] > 0.0 &&
                          eq_face(EN, gd) + qm[EN] > 0.0 && eq_face(EN, gd + 1) + qp[EN] > 0.0;
          if (!ok) {
#pragma unroll
            for (int f = 0; f < 5; ++f) qm[f] = qp[f] = sE[f * BOX + sidx];
          }
        }
        double UL[5], UR[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          const double ql = __shfl_up_sync(FULL, qp[f], 1, L);
          const double w0 = do_face ? eq_face(f, gd) : 0.0;
          UL[f] = w0 + ql;
          UR[f] = w0 + qm[f];
        }
        if (do_face) {
          gas_face_flux<D>(gam, UL, UR, F, status);
#pragma unroll
          for (int f = 0; f < 5; ++f) F[f] *= area;
        } else {
#pragma unroll
          for (int f = 0; f < 5; ++f) F[f] = 0.0;
        }
      } else {
        // face states E0 + q on both faces of this cell (Sect. 2.7 on App. B's
        // E); flat departures if either is not physical
        double Um[5], Up[5];
#pragma unroll
        for (int f = 0; f < 5; ++f) {
          Um[f] = eq_face(f, gd) + qm[f];
          Up[f] = eq_face(f, gd + 1) + qp[f];
        }
        double WL[5], WR[5], WP[5];
        gas_prim(gam, Um, WR);  // right state of the lower face
        gas_prim(gam, Up, WP);  // left state of the upper face, for the lane above
        if (shaped && do_recon) {
          const bool ok = Um[RHO] > 0.0 && Up[RHO] > 0.0 && WR[EN] > 0.0 && WP[EN] > 0.0;
          if (!ok) {
#pragma unroll
            for (int f = 0; f < 5; ++f) {
              const double e = sE[f * BOX + sidx];
              Um[f] = eq_face(f, gd) + e;
              Up[f] = eq_face(f, gd + 1) + e;
            }
            gas_prim(gam, Um, WR);
            gas_prim(gam, Up, WP);
          }
        }
#pragma unroll
        for (int f = 0; f < 5; ++f) WL[f] = __shfl_up_sync(FULL, WP[f], 1, L);
        if (do_face) {
          gas_face_flux<D>(gam, WL, WR, F, status);
#pragma unroll
          for (int f = 0; f < 5; ++f) F[f] *= area;
        } else {
#pragma unroll
          for (int f = 0; f < 5; ++f) F[f] = 0.0;
        }
      }
#pragma unroll
      for (int f = 0; f < 5; ++f) {
        const double Fu = __shfl_down_sync(FULL, F[f], 1, L);
        if (do_acc) {
          double* dst = sG + f * NCORE + (z * TT + y) * TR + x;
          if (D == 0) *dst = F[f] - Fu;
          else *dst += F[f] - Fu;
        }
      }
    }
    // ---------------- dust: each species' fields b .. b + 3, primitive
    // reconstruction, kinetic flux
#pragma unroll 1
    for (int b = 5; b < NF; b += 4) {
      double qm[4], qp[4];
      dust_recon<double, BOX, STRIDE>(sE, sidx, b, w, qm, qp);
      double F[4];
      {
        double WL[4];
#pragma unroll
        for (int f = 0; f < 4; ++f) WL[f] = __shfl_up_sync(FULL, qp[f], 1, L);
        if (do_face) {
          dust_kinetic_flux<D>(WL, qm, F);
#pragma unroll
          for (int f = 0; f < 4; ++f) F[f] *= area;
        } else {
#pragma unroll
          for (int f = 0; f < 4; ++f) F[f] = 0.0;
        }
      }
#pragma unroll
      for (int f = 0; f < 4; ++f) {
        const double Fu = __shfl_down_sync(FULL, F[f], 1, L);
        if (do_acc) {
          double* dst = sG + (b + f) * NCORE + (z * TT + y) * TR + x;
          if (D == 0) *dst = F[f] - Fu;
          else *dst += F[f] - Fu;
        }
      }
    }
  }
}

template <int NT>
__device__ __forceinline__ double block_min(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double m = red[0];
  for (int q = 1; q < NT / 32; ++q) m = fmin(m, red[q]);
  __syncthreads();
  return m;
}

// Fixed-order block sum (deterministic for a fixed launch shape).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  double s = 0.0;
  for (int q = 0; q < NT / 32; ++q) s += red[q];
  __syncthreads();
  return s;
}

// XT: the optional terms (indirect gravity, wave-killing zones) are compiled
// in; the plain instantiation carries none of their code.
// TZ = 1 is the flat tile of a grid one z cell thick whose z boundaries are
// periodic or outflow: both z ghosts of the cell are the cell itself, its two
// z faces carry the same flux, and the z sweep, whose divergence is exactly
// zero, is skipped (as is the z halo).
template <int NF, int TR, int TT, int TZ, int NT, bool XT, int RC>
__global__ void __launch_bounds__(NT, 1) stage_full_kernel(const StageArgs a) {
  constexpr int ZH = TZ == 1 ? 0 : 2;
  constexpr int BX = TR + 4, BY = TT + 4, BZ = TZ + 2 * ZH, BOX = BX * BY * BZ, NCORE = TR * TT * TZ;
  extern __shared__ double smem[];
  double* sE = smem;
  double* sG = smem + NF * BOX;
  const DevGrid& g = a.g;
  const int tile = blockIdx.x;
  // r fastest, then z, then theta: the tiles whose halos a tile re-reads
  // (its r, z and theta neighbours) run at most tiles_r x tiles_z blocks
  // apart, so the re-reads hit in L2
  const int i0 = (tile % a.tiles_r) * TR;
  const int k0 = ((tile / a.tiles_r) % a.tiles_z) * TZ;
  const int j0 = (tile / (a.tiles_r * a.tiles_z)) * TT;
  unsigned status = 0;

  // tile + halo as deviations (corners are never read): the gas departures
  // E' = E - E0 (or, with RC = RECON_PRIM, the primitive departures
  // u', v', w', P', rho') in slots 0..4, the dust as it is
  for (int idx = threadIdx.x; idx < BOX; idx += NT) {
    const int x = idx % BX - 2, y = (idx / BX) % BY - 2, z = idx / (BX * BY) - ZH;
    const int outside = (x < 0 || x >= TR) + (y < 0 || y >= TT) + (z < 0 || z >= TZ);
    if (outside > 1) continue;
    int c[3] = {i0 + x, j0 + y, k0 + z};
    if (!resolve_cell(g, c)) {
#pragma unroll
      for (int f = 0; f < NF; ++f) sE[f * BOX + idx] = 0.0;
      continue;
    }
    const size_t lin = ((size_t)c[2] * g.nth + c[1]) * g.nr + c[0];
    const size_t e0o = (size_t)c[2] * g.nr + c[0], e0s = (size_t)g.nz * g.nr;
    if (RC == RECON_PRIM) {
      double U[5], W[5];
#pragma unroll
      for (int f = 0; f < 5; ++f) U[f] = a.in[f][lin];
      gas_prim(g.gamma, U, W);
#pragma unroll
      for (int f = 0; f < 5; ++f) sE[f * BOX + idx] = g.has_eq ? W[f] - g.w0c[f * e0s + e0o] : W[f];
    } else {
#pragma unroll
      for (int f = 0; f < 5; ++f) sE[f * BOX + idx] = g.has_eq ? a.in[f][lin] - g.e0c[f * e0s + e0o] : a.in[f][lin];
    }
#pragma unroll
    for (int f = 5; f < NF; ++f) sE[f * BOX + idx] = a.in[f][lin];
  }
  __syncthreads();
  sweep_full<NF, TR, TT, TZ, NT, 0, RC>(a, sE, sG, i0, j0, k0, status);
  __syncthreads();
  sweep_full<NF, TR, TT, TZ, NT, 1, RC>(a, sE, sG, i0, j0, k0, status);
  __syncthreads();
  if constexpr (TZ > 1) {
    sweep_full<NF, TR, TT, TZ, NT, 2, RC>(a, sE, sG, i0, j0, k0, status);
    __syncthreads();
  }

  const double tau = a.tau_frac * (a.dt_dev ? __longlong_as_double((long long)*a.dt_dev) : a.dt_host);
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  double dtmin = INFINITY;
  double sums[NF];
#pragma unroll
  for (int f = 0; f < NF; ++f) sums[f] = 0.0;
  for (int cidx = threadIdx.x; cidx < NCORE; cidx += NT) {
    const int x = cidx % TR, y = (cidx / TR) % TT, z = cidx / (TR * TT);
    const int gi = i0 + x, gj = j0 + y, gk = k0 + z;
    if (gi >= g.nr || gj >= g.nth || gk >= g.nz) continue;
    const size_t lin = ((size_t)gk * g.nth + gj) * g.nr + gi;
    double U[NF], G[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      U[f] = a.in[f][lin];
      G[f] = sG[f * NCORE + cidx];
    }
    if (cell_nonphysical(g, U)) status |= STATUS_NONPHYSICAL;
    if (g.geom == GEOM_CYL) {
      double S[NF];
      cell_sources<XT>(g, gi, gj, gk, U, S);
      const double V = g.vol[gi];
#pragma unroll
      for (int f = 0; f < NF; ++f) G[f] += V * S[f];
    }
    if (g.r0) {
#pragma unroll
      for (int f = 0; f < 5; ++f) G[f] -= g.r0[((size_t)f * g.nz + gk) * g.nr + gi];
    }
    if (XT && g.damp_k) {  // wave-killing zones: the gas departures relax towards E0
      const double kd = g.damp_k[(size_t)gk * g.nr + gi];
      if (kd != 0.0) {
        const double V = g.vol[gi];
#pragma unroll
        for (int f = 0; f < 5; ++f) G[f] -= V * kd * (U[f] - g.e0c[((size_t)f * g.nz + gk) * g.nr + gi]);
      }
    }
    if (a.mode == 1) {
#pragma unroll
      for (int f = 0; f < NF; ++f) a.gout[f * ncell + lin] = G[f];
      continue;
    }
    const double iv = g.ivol[gi];
    double E[NF];
#pragma unroll
    for (int f = 0; f < NF; ++f) E[f] = a.base[f][lin] + tau * G[f] * iv;
    if constexpr (NF > 5) apply_drag<XT, (NF - 5) / 4>(g, gi, E, tau, a.drag);
#pragma unroll
    for (int f = 0; f < NF; ++f) a.out[f][lin] = E[f];
    if (a.stage2) {
      dtmin = fmin(dtmin, cell_dt(g, gi, E));
      if (cell_nonphysical(g, E)) status |= STATUS_NONPHYSICAL;
      const double V = g.vol[gi];
#pragma unroll
      for (int f = 0; f < NF; ++f) sums[f] += V * E[f];
    }
  }
  if (a.mode == 0 && a.stage2) {
    double* red = smem;  // the staged tile is no longer needed
    const double m = block_min<NT>(dtmin, red);
    if (threadIdx.x == 0) a.partials[(size_t)NF * gridDim.x + blockIdx.x] = m;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const double s = block_sum<NT>(sums[f], red);
      if (threadIdx.x == 0) a.partials[(size_t)f * gridDim.x + blockIdx.x] = s;
    }
  }
  if (status) atomicOr(a.status, status);
}

}  // namespace rossbi
