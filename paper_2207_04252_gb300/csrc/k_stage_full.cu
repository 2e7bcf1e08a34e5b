// Launcher of the FP64 stage kernel (stage_full.cuh).
#include "launch.cuh"

namespace rossbi {
namespace {

template <int NF, int TZ, bool XT, int RC>
cudaError_t launch(const StageArgs& a, int nblocks, cudaStream_t s) {
  constexpr int BOX = (F64_TR + 4) * (F64_TT + 4) * (TZ + 4);
  constexpr int NCORE = F64_TR * F64_TT * TZ;
  constexpr size_t smem = (size_t)NF * (BOX + NCORE) * sizeof(double);
  auto kern = stage_full_kernel<NF, F64_TR, F64_TT, TZ, F64_NT, XT, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, F64_NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NF, int RC>
cudaError_t launch_x(const StageArgs& a, int nblocks, cudaStream_t s, bool xt) {
  constexpr int TZ = tile_z(true, NF);
  return xt ? launch<NF, TZ, true, RC>(a, nblocks, s) : launch<NF, TZ, false, RC>(a, nblocks, s);
}

}  // namespace

cudaError_t run_stage_full(const StageArgs& a, int nblocks, cudaStream_t s, bool xt) {
  return by_nf(a.g.nf, [&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    return a.g.recon == RECON_PRIM ? launch_x<NF, RECON_PRIM>(a, nblocks, s, xt)
                                   : launch_x<NF, RECON_CONS>(a, nblocks, s, xt);
  });
}

}  // namespace rossbi
