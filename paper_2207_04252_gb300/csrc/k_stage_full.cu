// Launcher of the FP64 stage kernel (stage_full.cuh) for one gas
// reconstruction mode: ROSSBI_RC, the conservative one unless the including
// translation unit chose another.
#include "launch.cuh"

#ifndef ROSSBI_RC
#define ROSSBI_RC RECON_CONS
#endif

namespace rossbi {
namespace {

template <int NF, int TT, int TZ, bool XT, int RC>
cudaError_t launch(const StageArgs& a, int nblocks, cudaStream_t s) {
  constexpr int BOX = (F64_TR + 4) * (TT + 4) * (TZ == 1 ? 1 : TZ + 4);
  constexpr int NCORE = F64_TR * TT * TZ;
  constexpr size_t smem = (size_t)NF * (BOX + NCORE) * sizeof(double);
  auto kern = stage_full_kernel<NF, F64_TR, TT, TZ, F64_NT, XT, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, F64_NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NF, int RC>
cudaError_t launch_x(const StageArgs& a, int nblocks, cudaStream_t s, bool xt) {
  if constexpr (NF <= 9) {
    if (flat_grid(a.g.nz, a.g.bc_lo[2], a.g.bc_hi[2], NF))
      return xt ? launch<NF, FLAT_TT, 1, true, RC>(a, nblocks, s) : launch<NF, FLAT_TT, 1, false, RC>(a, nblocks, s);
  }
  constexpr int TZ = tile_z(true, NF);
  return xt ? launch<NF, F64_TT, TZ, true, RC>(a, nblocks, s) : launch<NF, F64_TT, TZ, false, RC>(a, nblocks, s);
}

}  // namespace

template <int RC>
cudaError_t run_stage_full_rc(const StageArgs& a, int nblocks, cudaStream_t s, bool xt) {
  return by_nf(a.g.nf, [&](auto nf) { return launch_x<decltype(nf)::value, RC>(a, nblocks, s, xt); });
}

template cudaError_t run_stage_full_rc<ROSSBI_RC>(const StageArgs&, int, cudaStream_t, bool);

}  // namespace rossbi
