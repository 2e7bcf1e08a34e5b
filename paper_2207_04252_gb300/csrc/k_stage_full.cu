// Launcher of the FP64 stage kernel (stage_full.cuh).
#include "launch.cuh"

namespace rossbi {
namespace {

template <int NF, bool XT, int RC>
cudaError_t launch(const StageArgs& a, int nblocks, cudaStream_t s) {
  constexpr int BOX = (F64_TR + 4) * (F64_TT + 4) * (F64_TZ + 4);
  constexpr int NCORE = F64_TR * F64_TT * F64_TZ;
  constexpr size_t smem = (size_t)NF * (BOX + NCORE) * sizeof(double);
  auto kern = stage_full_kernel<NF, F64_TR, F64_TT, F64_TZ, F64_NT, XT, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, F64_NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NF, int RC>
cudaError_t launch_x(const StageArgs& a, int nblocks, cudaStream_t s, bool xt) {
  return xt ? launch<NF, true, RC>(a, nblocks, s) : launch<NF, false, RC>(a, nblocks, s);
}

}  // namespace

cudaError_t run_stage_full(const StageArgs& a, int nblocks, cudaStream_t s, bool xt) {
  if (a.g.recon == RECON_PRIM)
    return a.g.nf == 9 ? launch_x<9, RECON_PRIM>(a, nblocks, s, xt) : launch_x<5, RECON_PRIM>(a, nblocks, s, xt);
  return a.g.nf == 9 ? launch_x<9, RECON_CONS>(a, nblocks, s, xt) : launch_x<5, RECON_CONS>(a, nblocks, s, xt);
}

}  // namespace rossbi
