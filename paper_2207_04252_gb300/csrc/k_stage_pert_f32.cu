// Launcher of the FP32 perturbation-form stage kernel (stage_pert.cuh).
#include "launch.cuh"

namespace rossbi {
namespace {

template <int NF, class P, bool XT, int RC>
cudaError_t launch(const PertArgs<float>& a, int nblocks, cudaStream_t s) {
  constexpr int BOX = (P32_TR + 4) * (P32_TT + 4) * (P32_TZ + 4), NCORE = P32_TR * P32_TT * P32_TZ;
  constexpr size_t smem = (size_t)NF * (BOX + NCORE) * sizeof(float);
  auto kern = stage_pert_kernel<float, NF, P32_TR, P32_TT, P32_TZ, P32_NT, P32_MINB, P, XT, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, P32_NT, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NF, class P, int RC>
cudaError_t launch_x(const PertArgs<float>& a, int nblocks, cudaStream_t s, bool xt) {
  return xt ? launch<NF, P, true, RC>(a, nblocks, s) : launch<NF, P, false, RC>(a, nblocks, s);
}

template <class P, int RC>
cudaError_t launch_nf(const PertArgs<float>& a, int nblocks, cudaStream_t s, bool xt) {
  return a.g.nf == 9 ? launch_x<9, P, RC>(a, nblocks, s, xt) : launch_x<5, P, RC>(a, nblocks, s, xt);
}

}  // namespace

cudaError_t run_stage_pert_f32(const PertArgs<float>& a, int nblocks, cudaStream_t s, bool xt, bool g75) {
  if (a.g.recon == RECON_PRIM)
    return g75 ? launch_nf<PowG75, RECON_PRIM>(a, nblocks, s, xt)
               : launch_nf<PowGeneric<float>, RECON_PRIM>(a, nblocks, s, xt);
  return g75 ? launch_nf<PowG75, RECON_CONS>(a, nblocks, s, xt)
             : launch_nf<PowGeneric<float>, RECON_CONS>(a, nblocks, s, xt);
}

}  // namespace rossbi
