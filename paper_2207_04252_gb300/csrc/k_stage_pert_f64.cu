// Launcher of the FP64 perturbation-form stage kernel (stage_pert.cuh).
#include "launch.cuh"

namespace rossbi {
namespace {

template <int NF, bool XT, int RC>
cudaError_t launch(const PertArgs<double>& a, int nblocks, cudaStream_t s) {
  constexpr int BOX = (P32_TR + 4) * (P32_TT + 4) * (P32_TZ + 4), NCORE = P32_TR * P32_TT * P32_TZ;
  constexpr size_t smem = (size_t)NF * (BOX + NCORE) * sizeof(double);
  auto kern = stage_pert_kernel<double, NF, P32_TR, P32_TT, P32_TZ, P32_NT, 1, PowGeneric<double>, XT, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, P32_NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NF, int RC>
cudaError_t launch_x(const PertArgs<double>& a, int nblocks, cudaStream_t s, bool xt) {
  return xt ? launch<NF, true, RC>(a, nblocks, s) : launch<NF, false, RC>(a, nblocks, s);
}

}  // namespace

cudaError_t run_stage_pert_f64(const PertArgs<double>& a, int nblocks, cudaStream_t s, bool xt) {
  if (a.g.recon == RECON_PRIM)
    return a.g.nf == 9 ? launch_x<9, RECON_PRIM>(a, nblocks, s, xt) : launch_x<5, RECON_PRIM>(a, nblocks, s, xt);
  return a.g.nf == 9 ? launch_x<9, RECON_CONS>(a, nblocks, s, xt) : launch_x<5, RECON_CONS>(a, nblocks, s, xt);
}

}  // namespace rossbi
