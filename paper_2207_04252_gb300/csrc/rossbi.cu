// Host runtime and C ABI of the GB300 RoSSBi3D hot-path library.
//
// Owns the mesh tables, the equilibrium tables and balanced residual, the
// reduction slots and the optional scratch state; launches the fused stage
// kernels.  The C ABI is declared (and documented) in include/rossbi.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/rossbi.h"
#include "launch.cuh"

using namespace rossbi;

namespace {

constexpr int CFL_NT = 256;

}  // namespace

struct rossbi_grid {
  rossbi_grid_desc desc{};
  cudaStream_t stream = nullptr;
  int device = -1;                     // the device current at rossbi_init_grid
  int nf = 5;
  size_t ncell = 0;
  DevGrid dg{};
  bool eq_set = false;
  bool has_disc = false;
  rossbi_disc_params disc{};
  // device tables
  double *d_rc = nullptr, *d_rf = nullptr, *d_rcoef = nullptr, *d_vol = nullptr, *d_ivol = nullptr;
  double *d_area_r = nullptr, *d_area_t = nullptr, *d_area_z = nullptr, *d_maxA = nullptr;
  double *d_e0c = nullptr, *d_e0r = nullptr, *d_e0z = nullptr, *d_r0 = nullptr;
  double* d_w0 = nullptr;              // primitive equilibrium tables (centres, r faces, z faces)
  std::vector<double> h_e0c;
  // reductions and status
  unsigned long long* d_dt = nullptr;  // [3]: step ping-pong slots 0/1, standalone CFL slot 2
  int dt_slot = 0;                     // slot holding the step length of the next step
  bool dt_on_device = false;
  double* d_partials = nullptr;
  size_t partials_cap = 0;
  double* d_sums = nullptr;
  unsigned* d_status = nullptr;
  double* h_pinned = nullptr;          // [32] readback area: [0..20] values, [28] status word
  // library-owned buffers
  void* d_scratch = nullptr;           // E* when the caller passes none
  void* d_hoststate = nullptr;         // device copy for rossbi_step_host
  int tiles_r = 0, tiles_t = 0, tiles_z = 0;
  int tile_tt = 6;                     // theta extent of a stage-kernel tile
  // perturbation forms: equilibrium and metric tables in the state precision
  void* d_ptab = nullptr;              // one allocation holding every table below
  PertTables<float> pt_f{};
  PertTables<double> pt_d{};
  unsigned long long* d_fallbacks = nullptr;
  double eq_sums[5] = {0, 0, 0, 0, 0}; // sum_cells V E0_f (FP64)
  // adjoint: five FP64 states (Y1, E*, Y2, mu', cotangent of E*), d/dSt partials and slots
  double* d_adj = nullptr;
  double* d_adj_part = nullptr;
  double* d_adj_slots = nullptr;       // [0] this call's d/dSt, [1] running total
  // indirect gravity: [2] disc moments A, B; [2][nth] cos / sin of the
  // azimuthal centres; [nz][nr] V r / R^3; [2][IND_BLOCKS] block partials
  double* d_ind = nullptr;
  double* d_adj_ind = nullptr;         // adjoint of the indirect term: [2 stages][2][adj_blocks] partials,
                                       // [2 stages][2] reduced, [2][nth] stage-1 gradient table
  double* d_damp = nullptr;            // relaxation rates of the damping zones per cell centre [nz][nr]
                                       // in double, then [nz][nr] in float
  bool damp_r = false, damp_z = false; // radial wave-killing zones; vertical sheared damped boundary
  rossbi_damping_params damp_rp{};
  rossbi_vertical_damping_params damp_zp{};
  int adj_blocks = 0;
  // stage-kernel timing (rossbi_profile_*)
  bool profiling = false;
  std::vector<cudaEvent_t> ev;         // start/stop pairs
  int ev_used = 0;
  double prof_ms = 0.0;
  int prof_launches = 0;
};

namespace {

size_t elem_size(const rossbi_grid* g) { return g->desc.precision == ROSSBI_FP32_PERT ? 4 : 8; }

#define CK(call)                                            \
  do {                                                      \
    cudaError_t e_ = (call);                                \
    if (e_ != cudaSuccess) {                                \
      return e_ == cudaErrorMemoryAllocation ? ROSSBI_ERR_OOM : ROSSBI_ERR_CUDA; \
    }                                                       \
  } while (0)

template <class T>
rossbi_status upload(T** dst, const std::vector<T>& src, cudaStream_t s) {
  if (*dst) cudaFree(*dst);
  *dst = nullptr;
  CK(cudaMalloc(dst, src.size() * sizeof(T)));
  CK(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
  return ROSSBI_OK;
}

// ---------------------------------------------------------------- mesh (Sect. 2.3)
double axis0_face(const rossbi_grid_desc& d, int i) {
  if (d.geometry == ROSSBI_GEOM_CYL) return d.x0[0] * std::pow(d.x1[0] / d.x0[0], (double)i / d.nr);
  return d.x0[0] + (d.x1[0] - d.x0[0]) * i / d.nr;
}
double axis0_centre(const rossbi_grid_desc& d, int i) {
  if (d.geometry == ROSSBI_GEOM_CYL) return std::sqrt(axis0_face(d, i) * axis0_face(d, i + 1));
  return 0.5 * (axis0_face(d, i) + axis0_face(d, i + 1));
}

// ---------------------------------------------------------------- equilibrium (App. A)
void equilibrium_prim(const rossbi_grid_desc& d, const rossbi_disc_params& p, double r, double z, double& rho,
                      double& vth, double& pres, double* dlnp_out = nullptr) {
  const double cs2 = p.T0 * std::pow(r, p.beta_T);
  const double omk = std::sqrt(d.gm / (r * r * r));
  const double H = std::sqrt(2.0 * cs2) / omk;
  const double R = std::sqrt(r * r + z * z);
  const double gpot = 1.0 / R - 1.0 / r;
  rho = p.sigma0 * std::pow(r, p.beta_sigma) / (std::sqrt(M_PI) * H) * std::exp(d.gm / cs2 * gpot);
  pres = cs2 * rho;
  double dlnp = (p.beta_T + p.beta_sigma - 0.5 * (p.beta_T + 3.0)) / r +
                d.gm / cs2 * (-p.beta_T * gpot / r - r / (R * R * R) + 1.0 / (r * r));
  if (p.bump_delta != 0.0) {  // Sect. 4.3: rho, P x (1 + delta G) at the same T; d ln P / dr gains its log-derivative
    const double x = (r - p.bump_r0) / p.bump_width;
    const double G = std::exp(-0.5 * x * x);
    const double s = 1.0 + p.bump_delta * G;
    rho *= s;
    pres *= s;
    dlnp -= p.bump_delta * G * x / (p.bump_width * s);
  }
  vth = std::sqrt(d.gm * r * r / (R * R * R) + r * cs2 * dlnp);
  if (dlnp_out) *dlnp_out = dlnp;
}

void equilibrium_cons(const rossbi_grid_desc& d, const rossbi_disc_params& p, double r, double z, double* U,
                      size_t stride) {
  double rho, vth, pres;
  equilibrium_prim(d, p, r, z, rho, vth, pres);
  const double v = vth - d.omega_frame * r;
  U[MU * stride] = 0.0;
  U[MV * stride] = rho * v;
  U[MW * stride] = 0.0;
  U[EN * stride] = 0.5 * rho * v * v + pres / (d.gamma - 1.0);
  U[RHO * stride] = rho;
}

rossbi_status check_desc(const rossbi_grid_desc& d) {
  if (d.nr < 1 || d.nth < 1 || d.nz < 1) return ROSSBI_ERR_ARG;
  if (d.geometry != ROSSBI_GEOM_BOX && d.geometry != ROSSBI_GEOM_CYL) return ROSSBI_ERR_ARG;
  if (!(d.gamma > 1.0) || !(d.cfl > 0.0)) return ROSSBI_ERR_ARG;
  if (d.n_dust < 0 || d.n_dust > ND_MAX) return ROSSBI_ERR_UNSUPPORTED;
  for (int a = 0; a < 3; ++a) {
    if (!(d.x1[a] > d.x0[a])) return ROSSBI_ERR_ARG;
    for (int bc : {d.bc_lo[a], d.bc_hi[a]})
      if (bc < ROSSBI_BC_PERIODIC || bc > ROSSBI_BC_EQUILIBRIUM) return ROSSBI_ERR_ARG;
    if ((d.bc_lo[a] == ROSSBI_BC_PERIODIC) != (d.bc_hi[a] == ROSSBI_BC_PERIODIC)) return ROSSBI_ERR_ARG;
  }
  if (d.geometry == ROSSBI_GEOM_CYL) {
    if (!(d.x0[0] > 0.0) || !(d.gm >= 0.0) || !std::isfinite(d.gm)) return ROSSBI_ERR_ARG;
    if (d.bc_lo[1] != ROSSBI_BC_PERIODIC) return ROSSBI_ERR_ARG;
    if (d.bc_lo[0] == ROSSBI_BC_PERIODIC) return ROSSBI_ERR_ARG;
  }
  if (d.precision != ROSSBI_FP64 && d.precision != ROSSBI_FP32_PERT && d.precision != ROSSBI_FP64_PERT)
    return ROSSBI_ERR_ARG;
  if (d.recon != ROSSBI_RECON_CONSERVATIVE && d.recon != ROSSBI_RECON_PRIMITIVE) return ROSSBI_ERR_ARG;
  return ROSSBI_OK;
}

rossbi_status status_from_word(unsigned w) {
  if (w & STATUS_NONPHYSICAL) return ROSSBI_ERR_NONPHYSICAL;
  if (w & STATUS_RIEMANN) return ROSSBI_ERR_RIEMANN;
  return ROSSBI_OK;
}

rossbi_status sync_and_status(rossbi_grid* g) {
  CK(cudaMemcpyAsync(g->h_pinned + 28, g->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, g->stream));
  CK(cudaMemsetAsync(g->d_status, 0, sizeof(unsigned), g->stream));
  CK(cudaStreamSynchronize(g->stream));
  unsigned w;
  std::memcpy(&w, g->h_pinned + 28, sizeof(unsigned));
  return status_from_word(w);
}

// ---------------------------------------------------------------- kernels
__global__ void cfl_kernel(DevGrid g, StageArgs a, unsigned long long* slot) {
  __shared__ double red[CFL_NT / 32];
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  double m = INFINITY;
  unsigned status = 0;
  for (size_t lin = blockIdx.x * (size_t)CFL_NT + threadIdx.x; lin < ncell; lin += (size_t)gridDim.x * CFL_NT) {
    double U[NF_MAX];
    for (int f = 0; f < g.nf; ++f) U[f] = a.in[f][lin];
    const int i = (int)(lin % g.nr);
    if (cell_nonphysical(g, U)) status |= STATUS_NONPHYSICAL;
    m = fmin(m, cell_dt(g, i, U));
  }
  m = block_min<CFL_NT>(m, red);
  if (threadIdx.x == 0) atomic_min_pos_double(slot, m);
  if (status) atomicOr(a.status, status);
}

__global__ void set_slot_kernel(unsigned long long* slot, unsigned long long v) { *slot = v; }

// Primitive equilibrium table from a conservative one ([5][n] each), with the
// conversion the stage kernels apply to the state, so that the deviations of
// an equilibrium state are exactly zero.
__global__ void eq_prim_kernel(double gamma, const double* e, double* w, size_t n) {
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    double U[5], W[5];
    for (int f = 0; f < 5; ++f) U[f] = e[f * n + q];
    gas_prim(gamma, U, W);
    for (int f = 0; f < 5; ++f) w[f * n + q] = W[f];
  }
}

// Per-block FP64 partial sums of V * E_f, fixed order.
__global__ void sums_kernel(DevGrid g, StageArgs a, double* partials) {
  __shared__ double red[CFL_NT / 32];
  const size_t ncell = (size_t)g.nr * g.nth * g.nz;
  double s[NF_MAX] = {};
  for (size_t lin = blockIdx.x * (size_t)CFL_NT + threadIdx.x; lin < ncell; lin += (size_t)gridDim.x * CFL_NT) {
    const double V = g.vol[lin % g.nr];
    for (int f = 0; f < g.nf; ++f) s[f] += V * a.in[f][lin];
  }
  for (int f = 0; f < g.nf; ++f) {
    const double t = block_sum<CFL_NT>(s[f], red);
    if (threadIdx.x == 0) partials[(size_t)f * gridDim.x + blockIdx.x] = t;
  }
}

// Reduces the per-block partials row by row in a fixed order (so the result
// does not depend on scheduling): rows 0..nf-1 are summed into sums[], row nf
// (when dt_slot is set) is minimised into the step-length slot.
constexpr int RED_NT = 512;
__global__ void __launch_bounds__(RED_NT) reduce_partials_kernel(const double* partials, int nblocks, int nf,
                                                                 double* sums, unsigned long long* dt_slot) {
  __shared__ double red[RED_NT / 32];
  const int row = blockIdx.x;
  const double* p = partials + (size_t)row * nblocks;
  const bool is_min = row == nf;
  double v = is_min ? INFINITY : 0.0;
  for (int b = threadIdx.x; b < nblocks; b += RED_NT) v = is_min ? fmin(v, p[b]) : v + p[b];
  if (is_min) {
    v = block_min<RED_NT>(v, red);
    if (threadIdx.x == 0) *dt_slot = (unsigned long long)__double_as_longlong(v);
  } else {
    v = block_sum<RED_NT>(v, red);
    if (threadIdx.x == 0) sums[row] = v;
  }
}

// Dust densities of every species (null beyond n).
template <class T>
struct DustRho {
  const T* p[ND_MAX];
  int n;
};

// Disc moments of the indirect gravity (Sect. 2.10): per-block FP64 partial
// sums of w (rho - rho_0 + sum rho_d) cos(theta) and ... sin(theta), with
// w = V r / R^3 of the cell centre; `full` states carry rho itself, the
// perturbation forms rho' already.  A warp takes one azimuthal row (nr cells)
// at a time; each lane sums its cells of the row in the state's precision
// (FP32: against a float copy of w, so that GB300's narrow FP64 pipe sees
// three operations per lane and row instead of several per cell), then the
// row sums are weighted by cos / sin and accumulated in FP64.  Rows go to
// warps in a fixed order, so the sums are reproducible.
constexpr int IND_NT = 256, IND_BLOCKS = 152 * 4;
template <class T, int ND>
__global__ void __launch_bounds__(IND_NT) indirect_moments_kernel(DevGrid g, const T* rho, const DustRho<T> dr,
                                                                  int full, const double* w, const float* wf,
                                                                  double* partials) {
  __shared__ double red[IND_NT / 32];
  constexpr int NW = IND_NT / 32;
  const int lane = threadIdx.x & 31;
  double A = 0.0, B = 0.0;
  const int rows = g.nth * g.nz;
  for (int row = blockIdx.x * NW + (threadIdx.x >> 5); row < rows; row += gridDim.x * NW) {
    const int j = row % g.nth, k = row / g.nth;
    const size_t base = (size_t)row * g.nr;
    T m = T(0);
    if constexpr (sizeof(T) == 4) {
      const float* wk = wf + (size_t)k * g.nr;
      for (int i = lane; i < g.nr; i += 32) {
        float x = rho[base + i];
#pragma unroll
        for (int s = 0; s < ND; ++s) x += dr.p[s][base + i];  // static indices: the pointers stay in the parameter bank
        m += x * wk[i];
      }
    } else {
      const double* wk = w + (size_t)k * g.nr;
      const double* e0 = full && g.has_eq ? g.e0c + ((size_t)RHO * g.nz + k) * g.nr : nullptr;
      for (int i = lane; i < g.nr; i += 32) {
        double dm = rho[base + i];
        if (e0) dm -= e0[i];
#pragma unroll
        for (int s = 0; s < ND; ++s) dm += dr.p[s][base + i];
        m += dm * wk[i];
      }
    }
    A += (double)m * g.ind_cs[j];
    B += (double)m * g.ind_cs[g.nth + j];
  }
  A = block_sum<IND_NT>(A, red);
  B = block_sum<IND_NT>(B, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = A;
    partials[gridDim.x + blockIdx.x] = B;
  }
}

// Fixed-order reduction of the moment partials into (A_disc, B_disc), as
// reduce_partials_kernel does it, then the gradient of the indirect
// potential at every axis-1 index, X_ref (A cos + B sin, -A sin + B cos), in
// double and in float (the stage epilogues read it per cell).
__global__ void __launch_bounds__(RED_NT) indirect_reduce_kernel(const double* partials, int nblocks, int nth,
                                                                 double x_ref, const double* cs, double* ab,
                                                                 double* gtab, float* gtabf) {
  __shared__ double red[RED_NT / 32];
  __shared__ double AB[2];
  for (int row = 0; row < 2; ++row) {
    const double* p = partials + (size_t)row * nblocks;
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += RED_NT) v += p[b];
    v = block_sum<RED_NT>(v, red);
    if (threadIdx.x == 0) AB[row] = v;
  }
  __syncthreads();
  const double A = AB[0], B = AB[1];
  if (threadIdx.x == 0) {
    ab[0] = A;
    ab[1] = B;
  }
  for (int j = threadIdx.x; j < nth; j += RED_NT) {
    const double c = cs[j], s = cs[nth + j];
    const double gr = x_ref * (A * c + B * s), gt = x_ref * (-A * s + B * c);
    gtab[j] = gr;
    gtab[nth + j] = gt;
    gtabf[j] = (float)gr;
    gtabf[nth + j] = (float)gt;
  }
}

// Halo rows of a decomposition in theta (Sect. 3.1 splits the grid into
// blocks of cells): copies rows j0 .. j0 + rows - 1 of every field between
// the state (SoA, index (k nth + j) nr + i) and a contiguous buffer laid out
// [f][k][jj][i].  One thread per element, consecutive threads along r, so
// both sides are read and written in coalesced runs of nr elements.
template <class T>
struct FieldPtrs {
  T* p[NF_MAX];
};
template <class T>
__global__ void theta_rows_kernel(FieldPtrs<T> st, T* buf, int nr, int nth, int nz, int nf, int j0, int rows,
                                  int unpack) {
  const size_t per_field = (size_t)nz * rows * nr, n = per_field * nf;
  for (size_t q = blockIdx.x * (size_t)blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x) {
    const int f = (int)(q / per_field);
    const size_t r = q - (size_t)f * per_field;
    const int i = (int)(r % nr);
    const size_t kj = r / nr;
    const int jj = (int)(kj % rows), k = (int)(kj / rows);
    const size_t lin = ((size_t)k * nth + (j0 + jj)) * nr + i;
    if (unpack) st.p[f][lin] = buf[q];
    else buf[q] = st.p[f][lin];
  }
}

constexpr int PROFILE_PAIRS = 1024;

rossbi_status profile_drain(rossbi_grid* g) {
  if (g->ev_used == 0) return ROSSBI_OK;
  CK(cudaStreamSynchronize(g->stream));
  for (int q = 0; q < g->ev_used; ++q) {
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, g->ev[2 * q], g->ev[2 * q + 1]));
    g->prof_ms += ms;
  }
  g->prof_launches += g->ev_used;
  g->ev_used = 0;
  return ROSSBI_OK;
}

rossbi_status launch_stage(rossbi_grid* g, const StageArgs& a, int nblocks) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g->profiling && a.mode == 0) {
    if (g->ev_used == PROFILE_PAIRS) {
      rossbi_status st = profile_drain(g);
      if (st != ROSSBI_OK) return st;
    }
    e0 = g->ev[2 * g->ev_used];
    e1 = g->ev[2 * g->ev_used + 1];
    CK(cudaEventRecord(e0, g->stream));
  }
  const bool xt = a.g.x_ind != 0.0 || a.g.damp_k != nullptr || a.drag.law == 2;  // optional terms on
  CK(run_stage_full(a, nblocks, g->stream, xt));
  if (e0) {
    CK(cudaEventRecord(e1, g->stream));
    g->ev_used++;
  }
  return ROSSBI_OK;
}

template <class T>
rossbi_status launch_pert(rossbi_grid* g, const PertArgs<T>& a, int nblocks) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (g->profiling) {
    if (g->ev_used == PROFILE_PAIRS) {
      rossbi_status st = profile_drain(g);
      if (st != ROSSBI_OK) return st;
    }
    e0 = g->ev[2 * g->ev_used];
    e1 = g->ev[2 * g->ev_used + 1];
    CK(cudaEventRecord(e0, g->stream));
  }
  const bool xt = a.g.x_ind != 0.0 || a.g.damp_k != nullptr || a.drag.law == 2;  // optional terms on
  if constexpr (sizeof(T) == 4)  // gamma = 7/5: integer-power forms of the float solver
    CK(run_stage_pert_f32(a, nblocks, g->stream, xt, g->desc.gamma == 1.4));
  else
    CK(run_stage_pert_f64(a, nblocks, g->stream, xt));
  if (e0) {
    CK(cudaEventRecord(e1, g->stream));
    g->ev_used++;
  }
  return ROSSBI_OK;
}

int n_tiles(const rossbi_grid* g) { return g->tiles_r * g->tiles_t * g->tiles_z; }

rossbi_status ensure_partials(rossbi_grid* g, size_t nblocks) {
  if (g->partials_cap >= nblocks) return ROSSBI_OK;
  if (g->d_partials) cudaFree(g->d_partials);
  g->d_partials = nullptr;
  g->partials_cap = 0;
  CK(cudaMalloc(&g->d_partials, nblocks * (NF_MAX + 1) * sizeof(double)));
  g->partials_cap = nblocks;
  return ROSSBI_OK;
}

StageArgs base_args(rossbi_grid* g) {
  StageArgs a;
  std::memset(&a, 0, sizeof(a));
  a.g = g->dg;
  a.status = g->d_status;
  a.tiles_r = g->tiles_r;
  a.tiles_z = g->tiles_z;
  return a;
}

// The empty run of Sect. 2.8 on a one-tile-thick azimuthal slab of the grid
// (same dtheta, so the same arithmetic as every column of the full grid).
rossbi_status empty_run(rossbi_grid* g) {
  const rossbi_grid_desc& d = g->desc;
  const int nth_s = std::min(d.nth, g->tile_tt);
  const size_t nslab = (size_t)d.nr * nth_s * d.nz;
  std::vector<double> E0(nslab * g->nf, 0.0);
  for (int f = 0; f < 5; ++f)
    for (int k = 0; k < d.nz; ++k)
      for (int j = 0; j < nth_s; ++j)
        for (int i = 0; i < d.nr; ++i)
          E0[f * nslab + ((size_t)k * nth_s + j) * d.nr + i] = g->h_e0c[((size_t)f * d.nz + k) * d.nr + i];
  double *dE = nullptr, *dG = nullptr;
  CK(cudaMalloc(&dE, E0.size() * sizeof(double)));
  cudaError_t e = cudaMalloc(&dG, E0.size() * sizeof(double));
  if (e != cudaSuccess) { cudaFree(dE); return ROSSBI_ERR_OOM; }
  rossbi_status st = ROSSBI_OK;
  do {
    if (cudaMemcpyAsync(dE, E0.data(), E0.size() * sizeof(double), cudaMemcpyHostToDevice, g->stream) !=
        cudaSuccess) { st = ROSSBI_ERR_CUDA; break; }
    StageArgs a = base_args(g);
    a.g.nth = nth_s;
    a.g.r0 = nullptr;
    a.g.x_ind = 0.0;  // the equilibrium's residual carries no indirect term
    a.g.damp_k = nullptr;  // nor a relaxation (E' = 0 there)
    for (int f = 0; f < g->nf; ++f) a.in[f] = dE + f * nslab;
    a.gout = dG;
    a.mode = 1;
    const int nblocks = g->tiles_r * 1 * g->tiles_z;  // one tile along theta
    st = launch_stage(g, a, nblocks);
    if (st != ROSSBI_OK) break;
    std::vector<double> G(E0.size());
    if (cudaMemcpyAsync(G.data(), dG, G.size() * sizeof(double), cudaMemcpyDeviceToHost, g->stream) !=
        cudaSuccess) { st = ROSSBI_ERR_CUDA; break; }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { st = ROSSBI_ERR_CUDA; break; }
    std::vector<double> R0((size_t)5 * d.nz * d.nr);
    for (int f = 0; f < 5; ++f)
      for (int k = 0; k < d.nz; ++k)
        for (int i = 0; i < d.nr; ++i)
          R0[((size_t)f * d.nz + k) * d.nr + i] = G[f * nslab + ((size_t)k * nth_s) * d.nr + i];
    st = upload(&g->d_r0, R0, g->stream);
    if (st != ROSSBI_OK) break;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { st = ROSSBI_ERR_CUDA; break; }
  } while (false);
  cudaFree(dE);
  cudaFree(dG);
  return st;
}

rossbi_status ensure_scratch(rossbi_grid* g, void** buf) {
  if (*buf) return ROSSBI_OK;
  CK(cudaMalloc(buf, g->ncell * g->nf * elem_size(g)));
  return ROSSBI_OK;
}

// Tables of the perturbation forms in the state precision T, built from FP64.
template <class T>
rossbi_status build_pert_tables(rossbi_grid* g, PertTables<T>& pt) {
  const rossbi_grid_desc& d = g->desc;
  const int nr = d.nr, nz = d.nz;
  const size_t ncen = (size_t)nz * nr, nfr = (size_t)nz * (nr + 1), nfz = (size_t)(nz + 1) * nr;
  const size_t off_cen = 0, off_fr = off_cen + 8 * ncen, off_fz = off_fr + 5 * nfr, off_ft = off_fz + 5 * nfz;
  const size_t off_rc = off_ft + 7 * ncen, off_vol = off_rc + (size_t)(nr + 2) * RCW, off_ivol = off_vol + nr;
  const size_t off_ar = off_ivol + nr, off_at = off_ar + nr + 1, off_az = off_at + nr, off_ma = off_az + nr;
  const size_t off_om = off_ma + nr, total = off_om + nr;
  std::vector<double> h(total, 0.0);
  std::vector<double> v(nr), rcoef((size_t)(nr + 2) * RCW), ar(nr + 1), at(nr), az(nr), ma(nr), iv(nr);
  if (cudaMemcpy(v.data(), g->d_vol, nr * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(iv.data(), g->d_ivol, nr * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(rcoef.data(), g->d_rcoef, rcoef.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(ar.data(), g->d_area_r, ar.size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(at.data(), g->d_area_t, nr * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(az.data(), g->d_area_z, nr * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(ma.data(), g->d_maxA, nr * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
    return ROSSBI_ERR_CUDA;
  for (size_t q = 0; q < rcoef.size(); ++q) h[off_rc + q] = rcoef[q];
  for (int i = 0; i < nr; ++i) {
    h[off_vol + i] = v[i];
    h[off_ivol + i] = iv[i];
    h[off_at + i] = at[i];
    h[off_az + i] = az[i];
    h[off_ma + i] = ma[i];
    const double r = axis0_centre(d, i);
    h[off_om + i] = d.geometry == ROSSBI_GEOM_CYL ? std::sqrt(d.gm / (r * r * r)) : 1.0;
  }
  for (int i = 0; i <= nr; ++i) h[off_ar + i] = ar[i];
  if (g->has_disc) {
    const double dz = (d.x1[2] - d.x0[2]) / nz, Om = d.omega_frame, gam = d.gamma;
    auto prim = [&](double r, double z, double* out, size_t stride, int nv) {
      double rho, vth, p, dlnp;
      equilibrium_prim(d, g->disc, r, z, rho, vth, p, &dlnp);
      const double v0 = vth - Om * r, c0 = std::sqrt(gam * p / rho);
      out[0] = rho;
      out[stride] = v0;
      out[2 * stride] = p;
      out[3 * stride] = c0;
      out[4 * stride] = 0.5 * rho * v0 * v0 + gam * p / (gam - 1.0);
      if (nv == 7) {
        out[5 * stride] = v0 - c0;
        out[6 * stride] = v0 + c0;
      }
    };
    for (int k = 0; k < nz; ++k) {
      const double z = d.x0[2] + (k + 0.5) * dz;
      for (int i = 0; i < nr; ++i) {
        const double r = axis0_centre(d, i);
        double rho, vth, p, dlnp;
        equilibrium_prim(d, g->disc, r, z, rho, vth, p, &dlnp);
        const double v0 = vth - Om * r, R2 = r * r + z * z, R3 = R2 * std::sqrt(R2);
        const double cs2 = g->disc.T0 * std::pow(r, g->disc.beta_T);
        double* c = &h[off_cen + (size_t)k * nr + i];
        c[0] = rho;
        c[ncen] = v0;
        c[2 * ncen] = p;
        c[3 * ncen] = cs2 * dlnp;                       // (1/rho0) dP0/dr
        c[4 * ncen] = -d.gm * z / R3;                   // f_z
        c[5 * ncen] = -d.gm * r / R3 + Om * Om * r;     // f_r + Omega^2 r
        c[6 * ncen] = 2.0 * v0 / r + 2.0 * Om;
        c[7 * ncen] = 1.0 / r;
        prim(r, z, &h[off_ft + (size_t)k * nr + i], ncen, 7);
      }
      for (int i = 0; i <= nr; ++i) prim(axis0_face(d, i), z, &h[off_fr + (size_t)k * (nr + 1) + i], nfr, 5);
    }
    for (int k = 0; k <= nz; ++k) {
      const double z = d.x0[2] + k * dz;
      for (int i = 0; i < nr; ++i) prim(axis0_centre(d, i), z, &h[off_fz + (size_t)k * nr + i], nfz, 5);
    }
  }
  std::vector<T> ht(total);
  for (size_t q = 0; q < total; ++q) ht[q] = (T)h[q];
  if (g->d_ptab) cudaFree(g->d_ptab);
  g->d_ptab = nullptr;
  CK(cudaMalloc(&g->d_ptab, total * sizeof(T)));
  CK(cudaMemcpy(g->d_ptab, ht.data(), total * sizeof(T), cudaMemcpyHostToDevice));
  const T* b = (const T*)g->d_ptab;
  pt.cen = b + off_cen;
  pt.fr = b + off_fr;
  pt.fz = b + off_fz;
  pt.ft = b + off_ft;
  pt.rcoef = b + off_rc;
  pt.vol = b + off_vol;
  pt.ivol = b + off_ivol;
  pt.area_r = b + off_ar;
  pt.area_t = b + off_at;
  pt.area_z = b + off_az;
  pt.maxA = b + off_ma;
  pt.omk = b + off_om;
  if (!g->d_fallbacks) {
    CK(cudaMalloc(&g->d_fallbacks, sizeof(unsigned long long)));
    CK(cudaMemset(g->d_fallbacks, 0, sizeof(unsigned long long)));
  }
  pt.fallbacks = g->d_fallbacks;
  for (int f = 0; f < 5; ++f) {
    double sum = 0.0;
    for (int k = 0; k < nz; ++k)
      for (int i = 0; i < nr; ++i) sum += v[i] * g->h_e0c[((size_t)f * nz + k) * nr + i];
    g->eq_sums[f] = sum * d.nth;
  }
  return ROSSBI_OK;
}

template <class T>
PertArgs<T> pert_args(rossbi_grid* g) {
  PertArgs<T> a;
  std::memset(&a, 0, sizeof(a));
  a.g = g->dg;
  if constexpr (sizeof(T) == 4) a.t = g->pt_f;
  else a.t = g->pt_d;
  a.status = g->d_status;
  a.tiles_r = g->tiles_r;
  a.tiles_z = g->tiles_z;
  a.gam = (T)g->dg.gamma;
  a.om = (T)g->dg.omega;
  a.cfl = (T)g->dg.cfl;
  a.dx1 = (T)g->dg.dx[1];
  a.dx2 = (T)g->dg.dx[2];
  for (int sp = 0; sp < ND_MAX; ++sp) a.st_factor[sp] = (T)g->dg.st_factor[sp];
  return a;
}

// The drag parameters of a step in the state precision.
template <class T>
void set_pert_drag(PertArgs<T>& a, const DragArgs& drag) {
  a.drag = drag;
  a.stokes = (T)drag.stokes;
  a.rhos_rp = (T)drag.rhos_rp;
  a.kappa = (T)drag.kappa;
}

// Drag parameters of a step (Sect. 2.9 drag law; Epstein constant fixed so
// that the Stokes number holds at r = 1, z = 0).
rossbi_status drag_args(rossbi_grid* g, const rossbi_dust_params* dust, DragArgs& drag) {
  drag = DragArgs{0.0, 0.0, 0, 0.0};
  if (g->nf > 5) {
    drag.stokes = dust->stokes;
    drag.law = dust->drag_law;
    if (!(dust->stokes > 0.0)) return ROSSBI_ERR_ARG;
    if (dust->drag_law == 0 && g->desc.geometry == ROSSBI_GEOM_CYL && !(g->desc.gm > 0.0))
      return ROSSBI_ERR_ARG;  // t_s = St / Omega_K needs a star
    if (dust->drag_law == 2) {  // Epstein constant as for law 1, plus the Stokes regime
      if (!(dust->kappa >= 0.0) || !std::isfinite(dust->kappa)) return ROSSBI_ERR_ARG;
      drag.kappa = dust->kappa;
    }
    if (dust->drag_law == 1 || dust->drag_law == 2) {
      if (!g->has_disc) return ROSSBI_ERR_ARG;
      double rho1, vth1, p1;
      equilibrium_prim(g->desc, g->disc, 1.0, 0.0, rho1, vth1, p1);
      drag.rhos_rp = dust->stokes * rho1 * std::sqrt(g->desc.gamma * p1 / rho1) / std::sqrt(g->desc.gm);
    } else if (dust->drag_law != 0) {
      return ROSSBI_ERR_ARG;
    }
  }
  return ROSSBI_OK;
}

rossbi_status prepare_step(rossbi_grid* g, void* const* state, void* const* scratch, double dt,
                           const rossbi_dust_params* dust, void** sc, DragArgs& drag) {
  if (!g->eq_set) return ROSSBI_ERR_ARG;
  if (!state) return ROSSBI_ERR_ARG;
  for (int f = 0; f < g->nf; ++f)
    if (!state[f]) return ROSSBI_ERR_ARG;
  if (g->nf > 5 && !dust) return ROSSBI_ERR_ARG;
  if (dt < 0.0 || !std::isfinite(dt)) return ROSSBI_ERR_ARG;
  if (dt == 0.0 && !g->dt_on_device) return ROSSBI_ERR_ARG;
  if (scratch) {
    for (int f = 0; f < g->nf; ++f) {
      if (!scratch[f]) return ROSSBI_ERR_ARG;
      for (int h = 0; h < g->nf; ++h)
        if (scratch[f] == state[h]) return ROSSBI_ERR_ARG;  // E* must not overwrite E^n
      sc[f] = scratch[f];
    }
  } else {
    rossbi_status st = ensure_scratch(g, &g->d_scratch);
    if (st != ROSSBI_OK) return st;
    for (int f = 0; f < g->nf; ++f) sc[f] = (char*)g->d_scratch + (size_t)f * g->ncell * elem_size(g);
  }
  rossbi_status st = ensure_partials(g, n_tiles(g));
  if (st != ROSSBI_OK) return st;
  return drag_args(g, dust, drag);
}

// Layout of the indirect-gravity tables, offsets in doubles: [2] the moments
// A, B; [2][nth] cos / sin of the azimuthal centres; [nz][nr] the weights
// V r / R^3 of the cell centres; [2][IND_BLOCKS] block partials; [2][nth]
// the gradient of the indirect potential; the same as floats; the weights as
// floats (for the FP32 form).
struct IndLayout {
  size_t cs, w, part, g, gf, wf, total;
};
IndLayout ind_layout(const rossbi_grid_desc& d) {
  const size_t nw = (size_t)d.nz * d.nr, nth = d.nth;
  IndLayout L;
  L.cs = 2;
  L.w = L.cs + 2 * nth;
  L.part = L.w + nw;
  L.g = L.part + 2 * (size_t)IND_BLOCKS;
  L.gf = L.g + 2 * nth;
  L.wf = L.gf + nth;  // 2 nth floats
  L.total = L.wf + (nw + 1) / 2;
  return L;
}

// Device tables of the indirect gravity (allocated once, layout above).
rossbi_status ensure_ind_tables(rossbi_grid* g) {
  if (g->d_ind) return ROSSBI_OK;
  const rossbi_grid_desc& d = g->desc;
  const double dy = (d.x1[1] - d.x0[1]) / d.nth, dz = (d.x1[2] - d.x0[2]) / d.nz;
  const IndLayout L = ind_layout(d);
  const size_t nw = (size_t)d.nz * d.nr, wf_at = L.wf;
  std::vector<double> h(L.total, 0.0);
  for (int j = 0; j < d.nth; ++j) {
    const double th = d.x0[1] + (j + 0.5) * dy;
    h[2 + j] = std::cos(th);
    h[2 + d.nth + j] = std::sin(th);
  }
  double* w = h.data() + 2 + 2 * (size_t)d.nth;
  for (int k = 0; k < d.nz; ++k) {
    const double z = d.x0[2] + (k + 0.5) * dz;
    for (int i = 0; i < d.nr; ++i) {
      const double r = axis0_centre(d, i), rm = axis0_face(d, i), rp = axis0_face(d, i + 1);
      const double V = 0.5 * (rp * rp - rm * rm) * dy * dz, R2 = r * r + z * z;
      w[(size_t)k * d.nr + i] = V * r / (R2 * std::sqrt(R2));
    }
  }
  std::vector<float> wf(nw);
  for (size_t q = 0; q < nw; ++q) wf[q] = (float)w[q];
  std::memcpy(h.data() + wf_at, wf.data(), nw * sizeof(float));
  rossbi_status st = upload(&g->d_ind, h, g->stream);
  if (st == ROSSBI_OK && cudaStreamSynchronize(g->stream) != cudaSuccess) st = ROSSBI_ERR_CUDA;
  if (st != ROSSBI_OK) {
    if (g->d_ind) cudaFree(g->d_ind);
    g->d_ind = nullptr;
    return st;
  }
  g->dg.ind_cs = g->d_ind + L.cs;
  g->dg.ind_g = g->d_ind + L.g;
  g->dg.ind_gf = reinterpret_cast<const float*>(g->d_ind + L.gf);
  return ROSSBI_OK;
}

// X_ref-free disc moments (A_disc, B_disc) of a state into d_ind[0..1].
rossbi_status indirect_moments(rossbi_grid* g, void* const* state) {
  const rossbi_grid_desc& d = g->desc;
  const IndLayout L = ind_layout(d);
  const double* w = g->d_ind + L.w;
  double* part = g->d_ind + L.part;
  const float* wf = reinterpret_cast<const float*>(g->d_ind + L.wf);
  // one instantiation per dust-species count
  auto launch = [&](auto tag, auto nd) {
    using T = decltype(tag);
    constexpr int ND = decltype(nd)::value;
    DustRho<T> dr{};
    for (int b = 5; b < g->nf; b += 4) dr.p[dr.n++] = (const T*)state[b + 3];
    indirect_moments_kernel<T, ND><<<IND_BLOCKS, IND_NT, 0, g->stream>>>(
        g->dg, (const T*)state[RHO], dr, d.precision == ROSSBI_FP64, w, wf, part);
  };
  auto by_species = [&](auto tag) {
    switch ((g->nf - 5) / 4) {
      case 0: launch(tag, std::integral_constant<int, 0>{}); break;
      case 1: launch(tag, std::integral_constant<int, 1>{}); break;
      case 2: launch(tag, std::integral_constant<int, 2>{}); break;
      case 3: launch(tag, std::integral_constant<int, 3>{}); break;
      default: launch(tag, std::integral_constant<int, 4>{}); break;
    }
  };
  if (d.precision == ROSSBI_FP32_PERT) by_species(float{});
  else by_species(double{});
  CK(cudaGetLastError());
  indirect_reduce_kernel<<<1, RED_NT, 0, g->stream>>>(part, IND_BLOCKS, d.nth, g->dg.x_ind, g->d_ind + L.cs,
                                                      g->d_ind, g->d_ind + L.g,
                                                      reinterpret_cast<float*>(g->d_ind + L.gf));
  CK(cudaGetLastError());
  return ROSSBI_OK;
}

rossbi_status finish_step(rossbi_grid* g, const double* partials, int nxt, double* next_dt) {
  reduce_partials_kernel<<<g->nf + 1, RED_NT, 0, g->stream>>>(partials, n_tiles(g), g->nf, g->d_sums,
                                                               g->d_dt + nxt);
  CK(cudaGetLastError());
  g->dt_slot = nxt;
  g->dt_on_device = true;
  if (next_dt) {
    CK(cudaMemcpyAsync(g->h_pinned, g->d_dt + nxt, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    const rossbi_status st = sync_and_status(g);
    *next_dt = g->h_pinned[0];
    return st;
  }
  return ROSSBI_OK;
}

// The two stages of one step (Sect. 2.5) with E* in sc and the stage-2
// block partials in `partials`; with the indirect gravity on, the disc
// moments of each stage's input are summed before it.  Allocates nothing.
rossbi_status step_full(rossbi_grid* g, void* const* state, void* const* sc, double* partials, double dt,
                        const DragArgs& drag, double* next_dt) {
  const int nblocks = n_tiles(g);
  const int cur = g->dt_slot, nxt = 1 - g->dt_slot;
  StageArgs a = base_args(g);
  a.drag = drag;
  a.dt_host = dt;
  a.dt_dev = dt == 0.0 ? g->d_dt + cur : nullptr;
  // stage 1: E* = E^n + dt/2 (G(E^n) - R0)/V, then drag
  for (int f = 0; f < g->nf; ++f) {
    a.in[f] = (const double*)state[f];
    a.base[f] = (const double*)state[f];
    a.out[f] = (double*)sc[f];
  }
  a.tau_frac = 0.5;
  a.stage2 = 0;
  rossbi_status st = g->dg.x_ind != 0.0 ? indirect_moments(g, state) : ROSSBI_OK;
  if (st == ROSSBI_OK) st = launch_stage(g, a, nblocks);
  if (st != ROSSBI_OK) return st;
  if (g->dg.x_ind != 0.0 && (st = indirect_moments(g, sc)) != ROSSBI_OK) return st;
  // stage 2: E^{n+1} = E^n + dt (G(E*) - R0)/V, then drag; fused CFL and sums
  for (int f = 0; f < g->nf; ++f) {
    a.in[f] = (const double*)sc[f];
    a.base[f] = (const double*)state[f];
    a.out[f] = (double*)state[f];
  }
  a.tau_frac = 1.0;
  a.stage2 = 1;
  a.partials = partials;
  st = launch_stage(g, a, nblocks);
  if (st != ROSSBI_OK) return st;
  return finish_step(g, partials, nxt, next_dt);
}

template <class T>
rossbi_status step_pert(rossbi_grid* g, void* const* state, void* const* sc, double* partials, double dt,
                        const DragArgs& drag, double* next_dt) {
  const int nblocks = n_tiles(g);
  const int cur = g->dt_slot, nxt = 1 - g->dt_slot;
  PertArgs<T> a = pert_args<T>(g);
  set_pert_drag(a, drag);
  a.dt_host = dt;
  a.dt_dev = dt == 0.0 ? g->d_dt + cur : nullptr;
  for (int f = 0; f < g->nf; ++f) {
    a.in[f] = (const T*)state[f];
    a.base[f] = (const T*)state[f];
    a.out[f] = (T*)sc[f];
  }
  a.tau_frac = 0.5;
  a.stage2 = 0;
  rossbi_status st = g->dg.x_ind != 0.0 ? indirect_moments(g, state) : ROSSBI_OK;
  if (st == ROSSBI_OK) st = launch_pert<T>(g, a, nblocks);
  if (st != ROSSBI_OK) return st;
  if (g->dg.x_ind != 0.0 && (st = indirect_moments(g, sc)) != ROSSBI_OK) return st;
  for (int f = 0; f < g->nf; ++f) {
    a.in[f] = (const T*)sc[f];
    a.base[f] = (const T*)state[f];
    a.out[f] = (T*)state[f];
  }
  a.tau_frac = 1.0;
  a.stage2 = 1;
  a.partials = partials;
  st = launch_pert<T>(g, a, nblocks);
  if (st != ROSSBI_OK) return st;
  return finish_step(g, partials, nxt, next_dt);
}

rossbi_status step_form(rossbi_grid* g, void* const* state, void* const* sc, double* partials, double dt,
                        const DragArgs& drag, double* next_dt) {
  switch (g->desc.precision) {
    case ROSSBI_FP64: return step_full(g, state, sc, partials, dt, drag, next_dt);
    case ROSSBI_FP32_PERT: return step_pert<float>(g, state, sc, partials, dt, drag, next_dt);
    default: return step_pert<double>(g, state, sc, partials, dt, drag, next_dt);
  }
}

// ---------------------------------------------------------------- adjoint
rossbi_status launch_adj_flux3(rossbi_grid* g, const AdjFluxArgs& a) {
  for (int axis = 0; axis < 3; ++axis) CK(run_adj_flux(a, axis, g->stream));
  return ROSSBI_OK;
}

template <int NF>
rossbi_status adjoint_reverse(rossbi_grid* g, void* const* state, double dt, const DragArgs& drag,
                              const void* const* lam_np1, void* const* lam_n, double* const* Y1, double* const* Es,
                              double* const* Y2, double* const* Mu, double* const* LamS) {
  const int nb = g->adj_blocks;
  AdjPointArgs p;
  std::memset(&p, 0, sizeof(p));
  p.g = g->dg;
  p.drag = drag;
  AdjFluxArgs fa;
  std::memset(&fa, 0, sizeof(fa));
  fa.g = g->dg;
  fa.status = g->d_status;
  // stage 2: E^{n+1} = D(Y2), Y2 = E^n + dt (G(E*) - R0) / V
  for (int f = 0; f < NF; ++f) {
    p.Y[f] = Y2[f];
    p.lout[f] = (const double*)lam_np1[f];
    p.Ein[f] = Es[f];
    p.M[f] = Mu[f];
    p.lam_n[f] = (double*)lam_n[f];
    p.lam_in[f] = LamS[f];
    fa.E[f] = Es[f];
    fa.M[f] = Mu[f];
    fa.lam[f] = LamS[f];
  }
  p.tau = dt;
  p.stage2 = 1;
  p.partials = g->d_adj_part;
  // indirect gravity: the stage's gradient tables (stage 2: those of E*, left
  // in the grid's tables by the recompute; stage 1: the saved copy), block
  // partials of dJ/dA, dJ/dB, their reduction, and the broadcast through the
  // moments into the cotangent of the stage input
  const bool ind = g->dg.x_ind != 0.0;
  const IndLayout L = ind_layout(g->desc);
  double* ind_part = g->d_adj_ind;
  double* ind_dab = g->d_adj_ind + 4 * (size_t)nb;
  const double* ind_g1 = g->d_adj_ind + 4 * (size_t)nb + 4;
  p.ind_partials = ind_part;
  adj_point_kernel<NF><<<nb, ADJ_PT_NT, 0, g->stream>>>(p);
  CK(cudaGetLastError());
  if (ind) {
    reduce_partials_kernel<<<2, RED_NT, 0, g->stream>>>(ind_part, nb, 2, ind_dab, nullptr);
    CK(cudaGetLastError());
    adj_indirect_bcast_kernel<<<nb, ADJ_PT_NT, 0, g->stream>>>(g->dg, g->d_ind + L.w, ind_dab, LamS[RHO],
                                                                NF == 9 ? LamS[DRHO] : nullptr);
    CK(cudaGetLastError());
  }
  rossbi_status st = launch_adj_flux3(g, fa);
  if (st != ROSSBI_OK) return st;
  // stage 1: E* = D(Y1), Y1 = E^n + dt/2 (G(E^n) - R0) / V
  for (int f = 0; f < NF; ++f) {
    p.Y[f] = Y1[f];
    p.lout[f] = LamS[f];
    p.Ein[f] = (const double*)state[f];
    fa.E[f] = (const double*)state[f];
    fa.lam[f] = (double*)lam_n[f];
  }
  p.tau = 0.5 * dt;
  p.stage2 = 0;
  p.partials = g->d_adj_part + nb;
  if (ind) {
    p.g.ind_g = ind_g1;
    p.ind_partials = ind_part + 2 * (size_t)nb;
  }
  adj_point_kernel<NF><<<nb, ADJ_PT_NT, 0, g->stream>>>(p);
  CK(cudaGetLastError());
  if (ind) {
    reduce_partials_kernel<<<2, RED_NT, 0, g->stream>>>(ind_part + 2 * (size_t)nb, nb, 2, ind_dab + 2, nullptr);
    CK(cudaGetLastError());
    adj_indirect_bcast_kernel<<<nb, ADJ_PT_NT, 0, g->stream>>>(g->dg, g->d_ind + L.w, ind_dab + 2,
                                                                (double*)lam_n[RHO],
                                                                NF == 9 ? (double*)lam_n[DRHO] : nullptr);
    CK(cudaGetLastError());
  }
  st = launch_adj_flux3(g, fa);
  if (st != ROSSBI_OK) return st;
  adj_dst_reduce_kernel<<<1, 512, 0, g->stream>>>(g->d_adj_part, 2 * nb, g->d_adj_slots);
  CK(cudaGetLastError());
  return ROSSBI_OK;
}

rossbi_status adjoint_step(rossbi_grid* g, void* const* state, double dt, const rossbi_dust_params* dust,
                           const void* const* lam_np1, void* const* lam_n, double* dparam) {
  if (!g->eq_set || !state || !lam_np1 || !lam_n) return ROSSBI_ERR_ARG;
  if (g->desc.precision != ROSSBI_FP64) return ROSSBI_ERR_UNSUPPORTED;
  if (!(dt > 0.0) || !std::isfinite(dt)) return ROSSBI_ERR_ARG;
  for (int f = 0; f < g->nf; ++f) {
    if (!state[f] || !lam_np1[f] || !lam_n[f]) return ROSSBI_ERR_ARG;
    for (int h = 0; h < g->nf; ++h)  // the cotangents must not overwrite E^n (lam_n may be lam_np1)
      if (lam_np1[f] == state[h] || lam_n[f] == state[h]) return ROSSBI_ERR_ARG;
  }
  if (g->nf > 9) return ROSSBI_ERR_UNSUPPORTED;  // the adjoint carries one dust species
  if (g->nf == 9 && !dust) return ROSSBI_ERR_ARG;
  DragArgs drag;
  rossbi_status st = drag_args(g, dust, drag);
  if (st != ROSSBI_OK) return st;
  const size_t nfc = (size_t)g->nf * g->ncell;
  if (!g->d_adj) {
    // all three buffers or none, so that a failed allocation leaves no half state
    const int nb = (int)std::min<size_t>((g->ncell + ADJ_PT_NT - 1) / ADJ_PT_NT, 2048);
    double *adj = nullptr, *part = nullptr, *slots = nullptr;
    cudaError_t e = cudaMalloc(&adj, 5 * nfc * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&part, 2 * (size_t)nb * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&slots, 2 * sizeof(double));
    if (e == cudaSuccess) e = cudaMemsetAsync(slots, 0, 2 * sizeof(double), g->stream);
    if (e != cudaSuccess) {
      cudaFree(adj);
      cudaFree(part);
      cudaFree(slots);
      return e == cudaErrorMemoryAllocation ? ROSSBI_ERR_OOM : ROSSBI_ERR_CUDA;
    }
    g->d_adj = adj;
    g->d_adj_part = part;
    g->d_adj_slots = slots;
    g->adj_blocks = nb;
  }
  const bool ind = g->dg.x_ind != 0.0;
  if (ind && !g->d_adj_ind) {
    const size_t n = 4 * (size_t)g->adj_blocks + 4 + 2 * (size_t)g->desc.nth;
    CK(cudaMalloc(&g->d_adj_ind, n * sizeof(double)));
  }
  double *Y1[9], *Es[9], *Y2[9], *Mu[9], *LamS[9];
  for (int f = 0; f < g->nf; ++f) {
    Y1[f] = g->d_adj + f * g->ncell;
    Es[f] = g->d_adj + nfc + f * g->ncell;
    Y2[f] = g->d_adj + 2 * nfc + f * g->ncell;
    Mu[f] = g->d_adj + 3 * nfc + f * g->ncell;
    LamS[f] = g->d_adj + 4 * nfc + f * g->ncell;
  }
  // forward recompute from E^n: the stage kernels with the drag switched off
  // (t_s = infinity makes apply_drag the identity) give the pre-drag states
  const int nblocks = n_tiles(g);
  StageArgs a = base_args(g);
  a.drag = drag;
  a.drag.stokes = INFINITY;
  a.drag.rhos_rp = INFINITY;
  a.dt_host = dt;
  for (int f = 0; f < g->nf; ++f) {
    a.in[f] = (const double*)state[f];
    a.base[f] = (const double*)state[f];
    a.out[f] = Y1[f];
  }
  a.tau_frac = 0.5;
  if (ind) {  // the moments of E^n; stage 1's gradient table is kept for the reverse sweep
    st = indirect_moments(g, state);
    if (st != ROSSBI_OK) return st;
    const IndLayout L = ind_layout(g->desc);
    CK(cudaMemcpyAsync(g->d_adj_ind + 4 * (size_t)g->adj_blocks + 4, g->d_ind + L.g,
                       2 * (size_t)g->desc.nth * sizeof(double), cudaMemcpyDeviceToDevice, g->stream));
  }
  st = launch_stage(g, a, nblocks);
  if (st != ROSSBI_OK) return st;
  double* const* Estar = Y1;
  if (g->nf == 9) {
    Fields9 y, o;
    for (int f = 0; f < 9; ++f) {
      y.p[f] = Y1[f];
      o.p[f] = Es[f];
    }
    drag_only_kernel<<<g->adj_blocks, ADJ_PT_NT, 0, g->stream>>>(g->dg, y, o, 0.5 * dt, drag);
    CK(cudaGetLastError());
    Estar = Es;
  }
  for (int f = 0; f < g->nf; ++f) {
    a.in[f] = Estar[f];
    a.base[f] = (const double*)state[f];
    a.out[f] = Y2[f];
  }
  a.tau_frac = 1.0;
  if (ind && (st = indirect_moments(g, (void* const*)Estar)) != ROSSBI_OK) return st;
  st = launch_stage(g, a, nblocks);
  if (st != ROSSBI_OK) return st;
  st = g->nf == 9 ? adjoint_reverse<9>(g, state, dt, drag, lam_np1, lam_n, Y1, Estar, Y2, Mu, LamS)
                  : adjoint_reverse<5>(g, state, dt, drag, lam_np1, lam_n, Y1, Estar, Y2, Mu, LamS);
  if (st != ROSSBI_OK) return st;
  if (dparam) {
    CK(cudaMemcpyAsync(g->h_pinned, g->d_adj_slots, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
    st = sync_and_status(g);
    *dparam += g->h_pinned[0];
    return st;
  }
  return ROSSBI_OK;
}

rossbi_status step_device(rossbi_grid* g, void* const* state, void* const* scratch, double dt,
                          const rossbi_dust_params* dust, double* next_dt) {
  void* sc[NF_MAX];
  DragArgs drag;
  rossbi_status st = prepare_step(g, state, scratch, dt, dust, sc, drag);
  if (st != ROSSBI_OK) return st;
  return step_form(g, state, sc, g->d_partials, dt, drag, next_dt);
}

}  // namespace

namespace {
// Eight independent FMA chains per thread; the result is stored so that
// nothing is eliminated.
template <class T>
__global__ void fma_peak_kernel(T* out, int iters) {
  T a[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) a[c] = T(threadIdx.x + c) * T(1e-7);
  const T m = T(0.9999999), k = T(1e-9);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      if constexpr (sizeof(T) == 4) a[c] = fmaf(a[c], m, k);
      else a[c] = fma(a[c], m, k);
    }
  }
  T s = T(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) s += a[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <class T>
rossbi_status fma_peak(cudaStream_t st, int iters, double* flops) {
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int blocks = 8 * sms, threads = 256;
  T* out = nullptr;
  if (cudaMalloc(&out, (size_t)blocks * threads * sizeof(T)) != cudaSuccess) return ROSSBI_ERR_OOM;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  rossbi_status r = ROSSBI_OK;
  float ms = 0.0f;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) r = ROSSBI_ERR_CUDA;
  if (r == ROSSBI_OK) {
    fma_peak_kernel<T><<<blocks, threads, 0, st>>>(out, iters);  // warm-up
    cudaEventRecord(e0, st);
    fma_peak_kernel<T><<<blocks, threads, 0, st>>>(out, iters);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess ||
        cudaGetLastError() != cudaSuccess)
      r = ROSSBI_ERR_CUDA;
  }
  if (r == ROSSBI_OK) *flops = 2.0 * 8.0 * iters * (double)blocks * threads / (ms * 1e-3);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  return r;
}
}  // namespace

extern "C" {

const char* rossbi_status_string(rossbi_status s) {
  switch (s) {
    case ROSSBI_OK: return "ok";
    case ROSSBI_ERR_ARG: return "invalid argument";
    case ROSSBI_ERR_CUDA: return "CUDA error";
    case ROSSBI_ERR_OOM: return "out of device memory";
    case ROSSBI_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, P <= 0 or NaN)";
    case ROSSBI_ERR_RIEMANN: return "Riemann solver did not converge";
    case ROSSBI_ERR_UNSUPPORTED: return "unsupported configuration";
  }
  return "unknown status";
}

int rossbi_nfields(const rossbi_grid* g) { return g ? g->nf : 0; }
int rossbi_precision(const rossbi_grid* g) { return g ? g->desc.precision : -1; }

void rossbi_destroy(rossbi_grid* g) {
  if (!g) return;
  double* tabs[] = {g->d_rc, g->d_rf, g->d_rcoef, g->d_vol, g->d_ivol, g->d_area_r, g->d_area_t,
                    g->d_area_z, g->d_maxA, g->d_e0c, g->d_e0r, g->d_e0z, g->d_r0, g->d_partials, g->d_sums};
  for (double* p : tabs)
    if (p) cudaFree(p);
  if (g->d_dt) cudaFree(g->d_dt);
  if (g->d_status) cudaFree(g->d_status);
  if (g->d_scratch) cudaFree(g->d_scratch);
  if (g->d_hoststate) cudaFree(g->d_hoststate);
  if (g->d_ptab) cudaFree(g->d_ptab);
  if (g->d_fallbacks) cudaFree(g->d_fallbacks);
  if (g->d_w0) cudaFree(g->d_w0);
  if (g->d_adj) cudaFree(g->d_adj);
  if (g->d_adj_part) cudaFree(g->d_adj_part);
  if (g->d_adj_slots) cudaFree(g->d_adj_slots);
  if (g->d_ind) cudaFree(g->d_ind);
  if (g->d_adj_ind) cudaFree(g->d_adj_ind);
  if (g->d_damp) cudaFree(g->d_damp);
  if (g->h_pinned) cudaFreeHost(g->h_pinned);
  for (cudaEvent_t e : g->ev) cudaEventDestroy(e);
  delete g;
}

rossbi_status rossbi_init_grid(const rossbi_grid_desc* desc, void* cuda_stream, rossbi_grid** out) {
  if (!desc || !out) return ROSSBI_ERR_ARG;
  *out = nullptr;
  const rossbi_status chk = check_desc(*desc);
  if (chk != ROSSBI_OK) return chk;
  rossbi_grid* g = new (std::nothrow) rossbi_grid();
  if (!g) return ROSSBI_ERR_OOM;
  g->desc = *desc;
  g->stream = (cudaStream_t)cuda_stream;
  if (cudaGetDevice(&g->device) != cudaSuccess) {
    delete g;
    return ROSSBI_ERR_CUDA;
  }
  g->nf = 5 + 4 * desc->n_dust;
  g->ncell = (size_t)desc->nr * desc->nth * desc->nz;
  const bool pert = desc->precision != ROSSBI_FP64;  // tile of the form's stage kernel
  const bool flat = !pert && flat_grid(desc->nz, desc->bc_lo[2], desc->bc_hi[2], g->nf);
  const int tr = pert ? P32_TR : F64_TR, tt = pert ? P32_TT : (flat ? FLAT_TT : F64_TT);
  const int tz = flat ? 1 : tile_z(desc->precision != ROSSBI_FP32_PERT, g->nf);
  g->tile_tt = tt;
  g->tiles_r = (desc->nr + tr - 1) / tr;
  g->tiles_t = (desc->nth + tt - 1) / tt;
  g->tiles_z = (desc->nz + tz - 1) / tz;
  const rossbi_grid_desc& d = *desc;
  const int nr = d.nr;
  const double dy = (d.x1[1] - d.x0[1]) / d.nth;
  const double dz = (d.x1[2] - d.x0[2]) / d.nz;
  std::vector<double> rc(nr + 2 * GH), rf(nr + 2 * GH + 1), rcoef((size_t)(nr + 2) * RCW, 0.0);
  for (int i = -GH; i < nr + GH; ++i) rc[i + GH] = axis0_centre(d, i);
  for (int i = -GH; i <= nr + GH; ++i) rf[i + GH] = axis0_face(d, i);
  for (int i = -1; i <= nr; ++i) {  // parabola weights (Sect. 2.7)
    const double xm = rc[i - 1 + GH], x0 = rc[i + GH], xp = rc[i + 1 + GH];
    const double fm = rf[i + GH], fp = rf[i + 1 + GH];
    double* w = &rcoef[(size_t)(i + 1) * RCW];
    w[0] = 1.0 / (x0 - xm);
    w[1] = 1.0 / (xp - x0);
    w[2] = 1.0 / (xp - xm);
    w[3] = x0 - xm;
    w[4] = xp - x0;
    w[5] = fm - x0;
    w[6] = fp - x0;
    w[7] = -std::min(2.0 * (x0 - fm), x0 - xm);  // limiter reach on the lower side
    w[8] = std::min(2.0 * (fp - x0), xp - x0);   // and on the upper side
  }
  std::vector<double> vol(nr), ivol(nr), ar(nr + 1), at(nr), az(nr), maxA(nr);
  if (d.geometry == ROSSBI_GEOM_CYL) {  // Sect. 2.2 finite volumes of the cylindrical mesh
    for (int i = 0; i <= nr; ++i) ar[i] = rf[i + GH] * dy * dz;
    for (int i = 0; i < nr; ++i) {
      const double rm = rf[i + GH], rp = rf[i + 1 + GH];
      vol[i] = 0.5 * (rp * rp - rm * rm) * dy * dz;
      at[i] = (rp - rm) * dz;
      az[i] = 0.5 * (rp * rp - rm * rm) * dy;
      maxA[i] = std::max(ar[i + 1], std::max(at[i], az[i]));
    }
  } else {
    const double dx = (d.x1[0] - d.x0[0]) / nr;
    for (int i = 0; i <= nr; ++i) ar[i] = dy * dz;
    for (int i = 0; i < nr; ++i) {
      vol[i] = dx * dy * dz;
      at[i] = dx * dz;
      az[i] = dx * dy;
      maxA[i] = std::max(ar[i], std::max(at[i], az[i]));
    }
  }
  for (int i = 0; i < nr; ++i) ivol[i] = 1.0 / vol[i];
  rossbi_status st = ROSSBI_OK;
  do {
    if ((st = upload(&g->d_rc, rc, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_rf, rf, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_rcoef, rcoef, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_vol, vol, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_ivol, ivol, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_area_r, ar, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_area_t, at, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_area_z, az, g->stream)) != ROSSBI_OK) break;
    if ((st = upload(&g->d_maxA, maxA, g->stream)) != ROSSBI_OK) break;
    if (cudaMalloc(&g->d_dt, 3 * sizeof(unsigned long long)) != cudaSuccess) { st = ROSSBI_ERR_OOM; break; }
    if (cudaMalloc(&g->d_sums, NF_MAX * sizeof(double)) != cudaSuccess) { st = ROSSBI_ERR_OOM; break; }
    if (cudaMalloc(&g->d_status, sizeof(unsigned)) != cudaSuccess) { st = ROSSBI_ERR_OOM; break; }
    if (cudaMemsetAsync(g->d_status, 0, sizeof(unsigned), g->stream) != cudaSuccess) { st = ROSSBI_ERR_CUDA; break; }
    if (cudaMallocHost(&g->h_pinned, 32 * sizeof(double)) != cudaSuccess) { st = ROSSBI_ERR_OOM; break; }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { st = ROSSBI_ERR_CUDA; break; }
  } while (false);
  if (st != ROSSBI_OK) {
    rossbi_destroy(g);
    return st;
  }
  DevGrid& dg = g->dg;
  dg.geom = d.geometry;
  dg.nr = d.nr;
  dg.nth = d.nth;
  dg.nz = d.nz;
  dg.nf = g->nf;
  dg.has_eq = 0;
  dg.recon = d.recon == ROSSBI_RECON_PRIMITIVE ? RECON_PRIM : RECON_CONS;
  for (int sp = 0; sp < ND_MAX; ++sp) dg.st_factor[sp] = 1.0;
  for (int a = 0; a < 3; ++a) {
    dg.bc_lo[a] = d.bc_lo[a];
    dg.bc_hi[a] = d.bc_hi[a];
    dg.x0[a] = d.x0[a];
    dg.dx[a] = (d.x1[a] - d.x0[a]) / (a == 0 ? d.nr : (a == 1 ? d.nth : d.nz));
  }
  dg.gamma = d.gamma;
  dg.gm = d.gm;
  dg.omega = d.geometry == ROSSBI_GEOM_CYL ? d.omega_frame : 0.0;
  dg.cfl = d.cfl;
  dg.rc = g->d_rc;
  dg.rf = g->d_rf;
  dg.rcoef = g->d_rcoef;
  dg.vol = g->d_vol;
  dg.ivol = g->d_ivol;
  dg.area_r = g->d_area_r;
  dg.area_t = g->d_area_t;
  dg.area_z = g->d_area_z;
  dg.maxA = g->d_maxA;
  *out = g;
  return ROSSBI_OK;
}

rossbi_status rossbi_set_equilibrium(rossbi_grid* g, const rossbi_disc_params* disc) {
  if (!g) return ROSSBI_ERR_ARG;
  const rossbi_grid_desc& d = g->desc;
  // a cylindrical grid without a disc (E0 = 0, e.g. the explosion test of
  // Sect. 4.1) runs in the FP64 form; the perturbation forms' source
  // coefficients are tabulated from a disc equilibrium
  if (d.geometry == ROSSBI_GEOM_CYL && !disc && d.precision != ROSSBI_FP64) return ROSSBI_ERR_UNSUPPORTED;
  if (d.geometry == ROSSBI_GEOM_CYL && disc && !(d.gm > 0.0)) return ROSSBI_ERR_ARG;  // Keplerian disc
  if (disc && disc->bump_delta != 0.0 &&
      (!(disc->bump_delta > -1.0) || !(disc->bump_width > 0.0) || !std::isfinite(disc->bump_delta) ||
       !std::isfinite(disc->bump_width) || !std::isfinite(disc->bump_r0)))
    return ROSSBI_ERR_ARG;
  g->eq_set = false;
  g->dg.has_eq = 0;
  g->dg.e0c = g->dg.e0r = g->dg.e0z = g->dg.r0 = nullptr;
  g->dg.w0c = g->dg.w0r = g->dg.w0z = nullptr;
  g->has_disc = disc != nullptr;
  if (!disc) {
    g->h_e0c.assign((size_t)5 * d.nz * d.nr, 0.0);
    rossbi_status st = ROSSBI_OK;
    if (d.precision == ROSSBI_FP32_PERT) st = build_pert_tables<float>(g, g->pt_f);
    else if (d.precision == ROSSBI_FP64_PERT) st = build_pert_tables<double>(g, g->pt_d);
    if (st != ROSSBI_OK) return st;
    g->eq_set = true;
    return ROSSBI_OK;
  }
  g->disc = *disc;
  const int nr = d.nr, nz = d.nz;
  const double dz = (d.x1[2] - d.x0[2]) / nz;
  std::vector<double> e0c((size_t)5 * nz * nr), e0r((size_t)5 * nz * (nr + 1)), e0z((size_t)5 * (nz + 1) * nr);
  for (int k = 0; k < nz; ++k) {
    const double z = d.x0[2] + (k + 0.5) * dz;
    for (int i = 0; i < nr; ++i)
      equilibrium_cons(d, *disc, axis0_centre(d, i), z, &e0c[(size_t)k * nr + i], (size_t)nz * nr);
    for (int i = 0; i <= nr; ++i)
      equilibrium_cons(d, *disc, axis0_face(d, i), z, &e0r[(size_t)k * (nr + 1) + i], (size_t)nz * (nr + 1));
  }
  for (int k = 0; k <= nz; ++k) {
    const double z = d.x0[2] + k * dz;
    for (int i = 0; i < nr; ++i)
      equilibrium_cons(d, *disc, axis0_centre(d, i), z, &e0z[(size_t)k * nr + i], (size_t)(nz + 1) * nr);
  }
  for (double v : e0c)
    if (!std::isfinite(v)) return ROSSBI_ERR_ARG;
  rossbi_status st;
  if ((st = upload(&g->d_e0c, e0c, g->stream)) != ROSSBI_OK) return st;
  if ((st = upload(&g->d_e0r, e0r, g->stream)) != ROSSBI_OK) return st;
  if ((st = upload(&g->d_e0z, e0z, g->stream)) != ROSSBI_OK) return st;
  g->h_e0c = e0c;
  g->dg.has_eq = 1;
  g->dg.e0c = g->d_e0c;
  g->dg.e0r = g->d_e0r;
  g->dg.e0z = g->d_e0z;
  {
    const size_t nc = (size_t)nz * nr, nrf = (size_t)nz * (nr + 1), nzf = (size_t)(nz + 1) * nr;
    if (g->d_w0) cudaFree(g->d_w0);
    g->d_w0 = nullptr;
    CK(cudaMalloc(&g->d_w0, 5 * (nc + nrf + nzf) * sizeof(double)));
    eq_prim_kernel<<<64, 256, 0, g->stream>>>(d.gamma, g->d_e0c, g->d_w0, nc);
    eq_prim_kernel<<<64, 256, 0, g->stream>>>(d.gamma, g->d_e0r, g->d_w0 + 5 * nc, nrf);
    eq_prim_kernel<<<64, 256, 0, g->stream>>>(d.gamma, g->d_e0z, g->d_w0 + 5 * (nc + nrf), nzf);
    CK(cudaGetLastError());
    g->dg.w0c = g->d_w0;
    g->dg.w0r = g->d_w0 + 5 * nc;
    g->dg.w0z = g->d_w0 + 5 * (nc + nrf);
  }
  if (d.precision == ROSSBI_FP64) {
    if ((st = empty_run(g)) != ROSSBI_OK) return st;
    g->dg.r0 = g->d_r0;
  } else if (d.precision == ROSSBI_FP32_PERT) {
    if ((st = build_pert_tables<float>(g, g->pt_f)) != ROSSBI_OK) return st;
  } else {
    if ((st = build_pert_tables<double>(g, g->pt_d)) != ROSSBI_OK) return st;
  }
  g->eq_set = true;
  return sync_and_status(g);
}

rossbi_status rossbi_get_equilibrium(rossbi_grid* g, double* host_out) {
  if (!g || !host_out || !g->eq_set) return ROSSBI_ERR_ARG;
  std::memcpy(host_out, g->h_e0c.data(), g->h_e0c.size() * sizeof(double));
  return ROSSBI_OK;
}

rossbi_status rossbi_cfl_dt(rossbi_grid* g, const void* const* state, double* dt_out) {
  if (!g || !state || !dt_out || !g->eq_set) return ROSSBI_ERR_ARG;
  for (int f = 0; f < g->nf; ++f)
    if (!state[f]) return ROSSBI_ERR_ARG;
  unsigned long long* slot = g->d_dt + g->dt_slot;
  set_slot_kernel<<<1, 1, 0, g->stream>>>(slot, 0x7ff0000000000000ull);
  CK(cudaGetLastError());
  const int blocks = (int)std::min<size_t>((g->ncell + CFL_NT - 1) / CFL_NT, 152 * 8);
  const int prec = g->desc.precision;
  if (prec == ROSSBI_FP64) {
    StageArgs a = base_args(g);
    for (int f = 0; f < g->nf; ++f) a.in[f] = (const double*)state[f];
    cfl_kernel<<<blocks, CFL_NT, 0, g->stream>>>(g->dg, a, slot);
  } else if (prec == ROSSBI_FP32_PERT) {
    PertArgs<float> a = pert_args<float>(g);
    for (int f = 0; f < g->nf; ++f) a.in[f] = (const float*)state[f];
    CK(by_nf(g->nf, [&](auto nf) {
      pert_cfl_kernel<float, decltype(nf)::value><<<blocks, 256, 0, g->stream>>>(a, slot);
      return cudaGetLastError();
    }));
  } else {
    PertArgs<double> a = pert_args<double>(g);
    for (int f = 0; f < g->nf; ++f) a.in[f] = (const double*)state[f];
    CK(by_nf(g->nf, [&](auto nf) {
      pert_cfl_kernel<double, decltype(nf)::value><<<blocks, 256, 0, g->stream>>>(a, slot);
      return cudaGetLastError();
    }));
  }
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(g->h_pinned, slot, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  const rossbi_status st = sync_and_status(g);
  *dt_out = g->h_pinned[0];
  g->dt_on_device = true;
  return st;
}

rossbi_status rossbi_step(rossbi_grid* g, void* const* state, void* const* scratch, double dt,
                          const rossbi_dust_params* dust, double* next_dt) {
  if (!g) return ROSSBI_ERR_ARG;
  return step_device(g, state, scratch, dt, dust, next_dt);
}

rossbi_status rossbi_step_host(rossbi_grid* g, void* const* host_state, double dt, const rossbi_dust_params* dust,
                               double* next_dt) {
  if (!g || !host_state) return ROSSBI_ERR_ARG;
  for (int f = 0; f < g->nf; ++f)
    if (!host_state[f]) return ROSSBI_ERR_ARG;
  rossbi_status st = ensure_scratch(g, &g->d_hoststate);
  if (st != ROSSBI_OK) return st;
  const size_t bytes = g->ncell * elem_size(g);
  void* dev[NF_MAX];
  for (int f = 0; f < g->nf; ++f) {
    dev[f] = (char*)g->d_hoststate + (size_t)f * bytes;
    CK(cudaMemcpyAsync(dev[f], host_state[f], bytes, cudaMemcpyHostToDevice, g->stream));
  }
  double ndt = 0.0;
  st = step_device(g, dev, nullptr, dt, dust, &ndt);
  for (int f = 0; f < g->nf; ++f)
    CK(cudaMemcpyAsync(host_state[f], dev[f], bytes, cudaMemcpyDeviceToHost, g->stream));
  CK(cudaStreamSynchronize(g->stream));
  if (next_dt) *next_dt = ndt;
  return st;
}

rossbi_status rossbi_conservation_sums(rossbi_grid* g, const void* const* state, double* sums) {
  if (!g || !state || !sums || !g->eq_set) return ROSSBI_ERR_ARG;
  for (int f = 0; f < g->nf; ++f)
    if (!state[f]) return ROSSBI_ERR_ARG;
  const int blocks = (int)std::min<size_t>((g->ncell + CFL_NT - 1) / CFL_NT, 152 * 8);
  rossbi_status st = ensure_partials(g, blocks);
  if (st != ROSSBI_OK) return st;
  const int prec = g->desc.precision;
  if (prec == ROSSBI_FP64) {
    StageArgs a = base_args(g);
    for (int f = 0; f < g->nf; ++f) a.in[f] = (const double*)state[f];
    sums_kernel<<<blocks, CFL_NT, 0, g->stream>>>(g->dg, a, g->d_partials);
  } else if (prec == ROSSBI_FP32_PERT) {
    PertArgs<float> a = pert_args<float>(g);
    for (int f = 0; f < g->nf; ++f) a.in[f] = (const float*)state[f];
    CK(by_nf(g->nf, [&](auto nf) {
      pert_sums_kernel<float, decltype(nf)::value><<<blocks, 256, 0, g->stream>>>(a, g->d_partials);
      return cudaGetLastError();
    }));
  } else {
    PertArgs<double> a = pert_args<double>(g);
    for (int f = 0; f < g->nf; ++f) a.in[f] = (const double*)state[f];
    CK(by_nf(g->nf, [&](auto nf) {
      pert_sums_kernel<double, decltype(nf)::value><<<blocks, 256, 0, g->stream>>>(a, g->d_partials);
      return cudaGetLastError();
    }));
  }
  CK(cudaGetLastError());
  reduce_partials_kernel<<<g->nf, RED_NT, 0, g->stream>>>(g->d_partials, blocks, g->nf, g->d_sums, nullptr);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(g->h_pinned, g->d_sums, g->nf * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  st = sync_and_status(g);
  for (int f = 0; f < g->nf; ++f) sums[f] = g->h_pinned[f];
  if (prec != ROSSBI_FP64)
    for (int f = 0; f < 5; ++f) sums[f] += g->eq_sums[f];
  return st;
}

rossbi_status rossbi_fallback_count(rossbi_grid* g, unsigned long long* count) {
  if (!g || !count) return ROSSBI_ERR_ARG;
  *count = 0;
  if (!g->d_fallbacks) return ROSSBI_OK;
  CK(cudaStreamSynchronize(g->stream));
  CK(cudaMemcpy(count, g->d_fallbacks, sizeof(unsigned long long), cudaMemcpyDeviceToHost));
  return ROSSBI_OK;
}

rossbi_status rossbi_measure_fma_peak(int fp64, void* cuda_stream, double* flops_per_s) {
  if (!flops_per_s) return ROSSBI_ERR_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  return fp64 ? fma_peak<double>(st, 1 << 13, flops_per_s) : fma_peak<float>(st, 1 << 19, flops_per_s);
}

rossbi_status rossbi_profile_enable(rossbi_grid* g, int enable) {
  if (!g) return ROSSBI_ERR_ARG;
  if (enable && g->ev.empty()) {
    g->ev.resize(2 * PROFILE_PAIRS, nullptr);
    for (auto& e : g->ev) CK(cudaEventCreate(&e));
  }
  g->profiling = enable != 0;
  return ROSSBI_OK;
}

rossbi_status rossbi_profile_read(rossbi_grid* g, double* stage_ms, int* stage_launches) {
  if (!g || !stage_ms || !stage_launches) return ROSSBI_ERR_ARG;
  const rossbi_status st = profile_drain(g);
  if (st != ROSSBI_OK) return st;
  *stage_ms = g->prof_ms;
  *stage_launches = g->prof_launches;
  g->prof_ms = 0.0;
  g->prof_launches = 0;
  return ROSSBI_OK;
}

rossbi_status rossbi_set_indirect(rossbi_grid* g, double x_ref) {
  if (!g || !std::isfinite(x_ref)) return ROSSBI_ERR_ARG;
  if (x_ref != 0.0 && g->desc.geometry != ROSSBI_GEOM_CYL) return ROSSBI_ERR_ARG;
  if (x_ref != 0.0) {
    const rossbi_status st = ensure_ind_tables(g);
    if (st != ROSSBI_OK) return st;
  }
  g->dg.x_ind = x_ref;
  return ROSSBI_OK;
}

}  // extern "C"

namespace {

// The rate table of the damping zones, per cell centre (nz, nr): the radial
// wave-killing zones (a parabola in r, 1 / tau at the boundary, 0 with zero
// slope at the zone edge, tau = f x the orbital period at that boundary)
// plus the vertical damped boundary (the same parabola in |z|, tau = f x the
// orbital period at the cell's radius).  Both off: no table.
rossbi_status build_damping(rossbi_grid* g) {
  const rossbi_grid_desc& d = g->desc;
  g->dg.damp_k = nullptr;
  g->dg.damp_kf = nullptr;
  if (!g->damp_r && !g->damp_z) return ROSSBI_OK;
  const double pi = 3.14159265358979323846;
  const double rin = d.x0[0], rout = d.x1[0], zmax = d.x1[2], dz = (d.x1[2] - d.x0[2]) / d.nz;
  const size_t n = (size_t)d.nz * d.nr;
  std::vector<double> k(n + (n + 1) / 2, 0.0);  // rates, then the same as floats
  const rossbi_damping_params& p = g->damp_rp;
  const double tau_in = p.period_factor * 2.0 * pi / std::sqrt(d.gm / (rin * rin * rin));
  const double tau_out = p.period_factor * 2.0 * pi / std::sqrt(d.gm / (rout * rout * rout));
  for (int kk = 0; kk < d.nz; ++kk) {
    const double az = std::fabs(d.x0[2] + (kk + 0.5) * dz);
    for (int i = 0; i < d.nr; ++i) {
      const double r = axis0_centre(d, i);
      double rate = 0.0;
      if (g->damp_r) {
        if (r < p.r_edge_in) {
          const double x = (p.r_edge_in - r) / (p.r_edge_in - rin);
          rate = x * x / tau_in;
        } else if (r > p.r_edge_out) {
          const double x = (r - p.r_edge_out) / (rout - p.r_edge_out);
          rate = x * x / tau_out;
        }
      }
      if (g->damp_z && az > g->damp_zp.z_edge) {
        const double x = (az - g->damp_zp.z_edge) / (zmax - g->damp_zp.z_edge);
        rate += x * x / (g->damp_zp.period_factor * 2.0 * pi / std::sqrt(d.gm / (r * r * r)));
      }
      k[(size_t)kk * d.nr + i] = rate;
    }
  }
  std::vector<float> kf(n);
  for (size_t q = 0; q < n; ++q) kf[q] = (float)k[q];
  std::memcpy(k.data() + n, kf.data(), n * sizeof(float));
  rossbi_status st = upload(&g->d_damp, k, g->stream);
  if (st == ROSSBI_OK && cudaStreamSynchronize(g->stream) != cudaSuccess) st = ROSSBI_ERR_CUDA;
  if (st != ROSSBI_OK) return st;
  g->dg.damp_k = g->d_damp;
  g->dg.damp_kf = reinterpret_cast<const float*>(g->d_damp + n);
  return ROSSBI_OK;
}

}  // namespace

extern "C" {

rossbi_status rossbi_set_damping(rossbi_grid* g, const rossbi_damping_params* p) {
  if (!g) return ROSSBI_ERR_ARG;
  if (!p) {
    g->damp_r = false;
    return build_damping(g);
  }
  const rossbi_grid_desc& d = g->desc;
  const double rin = d.x0[0], rout = d.x1[0];
  if (d.geometry != ROSSBI_GEOM_CYL || !g->eq_set || !g->has_disc) return ROSSBI_ERR_ARG;
  if (!(p->r_edge_in > rin) || !(p->r_edge_out < rout) || !(p->r_edge_in <= p->r_edge_out)) return ROSSBI_ERR_ARG;
  if (!(p->period_factor > 0.0) || !std::isfinite(p->period_factor)) return ROSSBI_ERR_ARG;
  g->damp_r = true;
  g->damp_rp = *p;
  return build_damping(g);
}

rossbi_status rossbi_set_vertical_damping(rossbi_grid* g, const rossbi_vertical_damping_params* p) {
  if (!g) return ROSSBI_ERR_ARG;
  if (!p) {
    g->damp_z = false;
    return build_damping(g);
  }
  const rossbi_grid_desc& d = g->desc;
  if (d.geometry != ROSSBI_GEOM_CYL || !g->eq_set || !g->has_disc || !(d.x0[2] == -d.x1[2])) return ROSSBI_ERR_ARG;
  if (!(p->z_edge >= 0.0) || !(p->z_edge < d.x1[2])) return ROSSBI_ERR_ARG;
  if (!(p->period_factor > 0.0) || !std::isfinite(p->period_factor)) return ROSSBI_ERR_ARG;
  g->damp_z = true;
  g->damp_zp = *p;
  return build_damping(g);
}

rossbi_status theta_rows(rossbi_grid* g, void* const* state, int j0, int rows, void* buf, int unpack) {
  if (!g || !state || !buf || rows < 1 || j0 < 0 || j0 + rows > g->desc.nth) return ROSSBI_ERR_ARG;
  for (int f = 0; f < g->nf; ++f)
    if (!state[f]) return ROSSBI_ERR_ARG;
  const rossbi_grid_desc& d = g->desc;
  const size_t n = (size_t)g->nf * d.nz * rows * d.nr;
  const int blocks = (int)std::min<size_t>((n + 255) / 256, 152 * 8);
  if (d.precision == ROSSBI_FP32_PERT) {
    FieldPtrs<float> p{};
    for (int f = 0; f < g->nf; ++f) p.p[f] = (float*)state[f];
    theta_rows_kernel<float><<<blocks, 256, 0, g->stream>>>(p, (float*)buf, d.nr, d.nth, d.nz, g->nf, j0, rows,
                                                             unpack);
  } else {
    FieldPtrs<double> p{};
    for (int f = 0; f < g->nf; ++f) p.p[f] = (double*)state[f];
    theta_rows_kernel<double><<<blocks, 256, 0, g->stream>>>(p, (double*)buf, d.nr, d.nth, d.nz, g->nf, j0, rows,
                                                              unpack);
  }
  CK(cudaGetLastError());
  return ROSSBI_OK;
}

rossbi_status rossbi_pack_theta_rows(rossbi_grid* g, const void* const* state, int j0, int rows, void* buf) {
  return theta_rows(g, (void* const*)state, j0, rows, buf, 0);
}

rossbi_status rossbi_unpack_theta_rows(rossbi_grid* g, void* const* state, int j0, int rows, const void* buf) {
  return theta_rows(g, state, j0, rows, (void*)buf, 1);
}

rossbi_status rossbi_set_dust_species(rossbi_grid* g, const double* stokes_factor, int n) {
  if (!g || !stokes_factor) return ROSSBI_ERR_ARG;
  const int nd = (g->nf - 5) / 4;
  if (n != nd || nd < 1) return ROSSBI_ERR_ARG;
  if (stokes_factor[0] != 1.0) return ROSSBI_ERR_ARG;  // species 0 has the Stokes number itself
  for (int sp = 1; sp < n; ++sp)
    if (!(stokes_factor[sp] > 0.0) || !std::isfinite(stokes_factor[sp])) return ROSSBI_ERR_ARG;
  for (int sp = 0; sp < n; ++sp) g->dg.st_factor[sp] = stokes_factor[sp];
  return ROSSBI_OK;
}

rossbi_status rossbi_indirect_moments(rossbi_grid* g, const void* const* state, double* ab) {
  if (!g || !state || !ab || !g->eq_set || g->desc.geometry != ROSSBI_GEOM_CYL) return ROSSBI_ERR_ARG;
  if (!state[RHO]) return ROSSBI_ERR_ARG;
  for (int b = 5; b < g->nf; b += 4)
    if (!state[b + 3]) return ROSSBI_ERR_ARG;
  rossbi_status st = ensure_ind_tables(g);
  if (st == ROSSBI_OK) st = indirect_moments(g, (void* const*)state);
  if (st != ROSSBI_OK) return st;
  CK(cudaMemcpyAsync(g->h_pinned, g->d_ind, 2 * sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  st = sync_and_status(g);
  ab[0] = g->h_pinned[0];
  ab[1] = g->h_pinned[1];
  return st;
}

rossbi_status rossbi_adjoint_step(rossbi_grid* g, const void* const* state_n, double dt,
                                  const rossbi_dust_params* dust, const void* const* lam_np1, void* const* lam_n,
                                  double* dparam) {
  if (!g) return ROSSBI_ERR_ARG;
  return adjoint_step(g, (void* const*)state_n, dt, dust, lam_np1, lam_n, dparam);
}

rossbi_status rossbi_adjoint_dstokes(rossbi_grid* g, double* total, int reset) {
  if (!g || !total) return ROSSBI_ERR_ARG;
  *total = 0.0;
  if (!g->d_adj_slots) return ROSSBI_OK;
  CK(cudaMemcpyAsync(g->h_pinned, g->d_adj_slots + 1, sizeof(double), cudaMemcpyDeviceToHost, g->stream));
  const rossbi_status st = sync_and_status(g);
  *total = g->h_pinned[0];
  if (reset) {
    CK(cudaMemsetAsync(g->d_adj_slots, 0, 2 * sizeof(double), g->stream));
    CK(cudaStreamSynchronize(g->stream));
  }
  return st;
}

rossbi_status rossbi_take_status(rossbi_grid* g) {
  if (!g) return ROSSBI_ERR_ARG;
  return sync_and_status(g);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Step without device allocation.
//
// rossbi_step takes its stage scratch (the intermediate state E* and the
// per-block reduction partials) from a buffer it cudaMallocs on first use, or
// from caller-passed buffers.  Some callers can allocate neither: host codes
// that hand all device memory to their own pool at start-up and forbid any
// later cudaMalloc, or loops that cannot afford the implicit device
// synchronisation a cudaMalloc/cudaFree may cause.  rossbi_step_noalloc runs
// the same kernels with that scratch placed in the fixed array below instead.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds NOALLOC_SCRATCH_BYTES of it until the process exits.  Host code
// must not use `noalloc_scratch` as a pointer (in host code the name is a host
// stand-in, not a device address); its device address is looked up once per
// device with cudaGetSymbolAddress, with that device current, on the first
// rossbi_step_noalloc call made on that device.  That first call should
// therefore come before any stream capture.  All calls share the array and it
// keeps the last call's contents; nothing in it needs to start at zero
// (stage 1 writes every E* cell stage 2 reads, and each stage-2 block writes
// its own partials).  Calls whose work overlaps on the GPU (other streams,
// other grids, other threads) race on the array and must be serialised by the
// caller.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)64 << 20;  // 64 MiB
static __device__ __align__(256) unsigned char noalloc_scratch[NOALLOC_SCRATCH_BYTES];

constexpr int NOALLOC_MAX_DEVICES = 64;
void* noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

rossbi_status noalloc_scratch_ptr(void** out) {
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return ROSSBI_ERR_ARG;
  if (!noalloc_ptr[dev]) {
    void* p = nullptr;
    CK(cudaGetSymbolAddress(&p, noalloc_scratch));
    noalloc_ptr[dev] = p;
  }
  *out = noalloc_ptr[dev];
  return ROSSBI_OK;
}

}  // namespace

extern "C" rossbi_status rossbi_step_noalloc(rossbi_grid* g, void* const* state, double dt,
                                             const rossbi_dust_params* dust, double* next_dt) {
  if (!g || !g->eq_set || !state) return ROSSBI_ERR_ARG;
  for (int f = 0; f < g->nf; ++f)
    if (!state[f]) return ROSSBI_ERR_ARG;
  if (g->nf > 5 && !dust) return ROSSBI_ERR_ARG;
  if (g->nf > 5 && dust->drag_law == 2) return ROSSBI_ERR_ARG;
  if (dt < 0.0 || !std::isfinite(dt)) return ROSSBI_ERR_ARG;
  if (dt == 0.0 && !g->dt_on_device) return ROSSBI_ERR_ARG;
  // the array's address is per device: only the grid's own device may be current
  int dev = -1;
  CK(cudaGetDevice(&dev));
  if (dev != g->device) return ROSSBI_ERR_ARG;
  const int nblocks = n_tiles(g);
  const size_t field_bytes = align256(g->ncell * elem_size(g));
  const size_t partial_bytes = (size_t)(g->nf + 1) * nblocks * sizeof(double);
  if ((size_t)g->nf * field_bytes + partial_bytes > NOALLOC_SCRATCH_BYTES) return ROSSBI_ERR_ARG;
  DragArgs drag;
  rossbi_status st = drag_args(g, dust, drag);
  if (st != ROSSBI_OK) return st;
  void* base = nullptr;
  st = noalloc_scratch_ptr(&base);
  if (st != ROSSBI_OK) return st;
  void* sc[NF_MAX];
  for (int f = 0; f < g->nf; ++f) sc[f] = (char*)base + (size_t)f * field_bytes;
  double* partials = (double*)((char*)base + (size_t)g->nf * field_bytes);
  // the same two stages as rossbi_step (with the indirect gravity's moments
  // in the grid's own tables, set up by rossbi_set_indirect)
  return step_form(g, state, sc, partials, dt, drag, next_dt);
}
