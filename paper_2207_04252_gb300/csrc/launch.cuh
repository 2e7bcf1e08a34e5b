// Kernel launchers of the stage and adjoint-flux kernels, one translation
// unit per kernel family (compiled in parallel), called by the host runtime.
// Each dispatches on the field count, the optional-term switch and the gas
// reconstruction mode to one instantiation of its kernel template.
#pragma once
#include <cuda_runtime.h>

#include <type_traits>

#include "adjoint.cuh"
#include "stage_pert.cuh"

namespace rossbi {

// Tiles of the stage kernels: 14 x 6 x 6 cells, lines of 16 / 8 / 8 lanes.
constexpr int F64_TR = 14, F64_TT = 6, F64_TZ = 6, F64_NT = 192;
constexpr int P32_TR = 14, P32_TT = 6, P32_TZ = 6, P32_NT = 256, P32_MINB = 2;
// With more than one dust species the FP64-state kernels' staged 14 x 6 x 6
// tile with its halo (18 x 10 x 10 cells) no longer fits in shared memory
// (13 fields: 234 KB of the 227 KB a block may have): they take tiles two z
// cells thick (lines of 4 lanes in z; 13 fields: 127 KB, 21: 205 KB).
constexpr int THIN_TZ = 2;
constexpr int tile_z(bool fp64_state, int nf) { return fp64_state && nf > 9 ? THIN_TZ : 6; }

// The FP64 kernel's flat tile, 14 x 30 x 1 cells without a z halo or z
// sweep, for grids one z cell thick whose z boundaries are periodic or
// outflow (the cell's two z faces then carry the same flux), with at most
// one dust species: the cylindrical explosion of Sect. 4.1 runs on it.
constexpr int FLAT_TT = 30;
inline bool flat_grid(int nz, int bc_lo_z, int bc_hi_z, int nf) {
  return nz == 1 && bc_lo_z != BC_EQUILIBRIUM && bc_hi_z != BC_EQUILIBRIUM && nf <= 9;
}

// Calls f(std::integral_constant<int, NF>) for the field count nf (5 + 4 x
// the number of dust species, 0 .. 4).
template <class F>
cudaError_t by_nf(int nf, F&& f) {
  switch (nf) {
    case 5: return f(std::integral_constant<int, 5>{});
    case 9: return f(std::integral_constant<int, 9>{});
    case 13: return f(std::integral_constant<int, 13>{});
    case 17: return f(std::integral_constant<int, 17>{});
    case 21: return f(std::integral_constant<int, 21>{});
  }
  return cudaErrorInvalidValue;
}
// Adjoint flux kernel: lines of 16 lanes (12 owned cells), 16 lines per block.
constexpr int ADJ_L = 16, ADJ_NL = 16;

// Raises a kernel's dynamic shared-memory limit once per device (the
// attribute belongs to the current device's context); `done` is the calling
// site's own flag word, one bit per device id < 64.
template <class K>
cudaError_t set_smem_once(K kern, size_t smem, unsigned long long& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) done |= bit;
  return e;
}

// Each launcher is instantiated per gas reconstruction mode RC in a
// translation unit of its own (they compile in parallel).
// One launch of the FP64 stage kernel over nblocks tiles; xt selects the
// instantiation with the optional terms (indirect gravity, damping zones,
// Stokes drag regime).
template <int RC>
cudaError_t run_stage_full_rc(const StageArgs& a, int nblocks, cudaStream_t s, bool xt);
inline cudaError_t run_stage_full(const StageArgs& a, int nblocks, cudaStream_t s, bool xt) {
  return a.g.recon == RECON_PRIM ? run_stage_full_rc<RECON_PRIM>(a, nblocks, s, xt)
                                 : run_stage_full_rc<RECON_CONS>(a, nblocks, s, xt);
}
// One launch of the perturbation-form stage kernel (float or double); g75
// selects the gamma = 7/5 power forms of the float solver.
template <class P, int RC>
cudaError_t run_stage_pert_f32_rc(const PertArgs<float>& a, int nblocks, cudaStream_t s, bool xt);
inline cudaError_t run_stage_pert_f32(const PertArgs<float>& a, int nblocks, cudaStream_t s, bool xt, bool g75) {
  if (a.g.recon == RECON_PRIM)
    return g75 ? run_stage_pert_f32_rc<PowG75, RECON_PRIM>(a, nblocks, s, xt)
               : run_stage_pert_f32_rc<PowGeneric<float>, RECON_PRIM>(a, nblocks, s, xt);
  return g75 ? run_stage_pert_f32_rc<PowG75, RECON_CONS>(a, nblocks, s, xt)
             : run_stage_pert_f32_rc<PowGeneric<float>, RECON_CONS>(a, nblocks, s, xt);
}
template <int RC>
cudaError_t run_stage_pert_f64_rc(const PertArgs<double>& a, int nblocks, cudaStream_t s, bool xt);
inline cudaError_t run_stage_pert_f64(const PertArgs<double>& a, int nblocks, cudaStream_t s, bool xt) {
  return a.g.recon == RECON_PRIM ? run_stage_pert_f64_rc<RECON_PRIM>(a, nblocks, s, xt)
                                 : run_stage_pert_f64_rc<RECON_CONS>(a, nblocks, s, xt);
}
// One launch of the adjoint flux kernel along axis 0, 1 or 2.
cudaError_t run_adj_flux(const AdjFluxArgs& a, int axis, cudaStream_t s);

}  // namespace rossbi
