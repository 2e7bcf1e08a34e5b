// Launcher of the FP32 perturbation-form stage kernel (stage_pert.cuh) for
// gamma = 7/5 (the integer-power forms of the solver).
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

}  // namespace

template <class P>
cudaError_t run_stage_pert_f32_p(const PertArgs<float>& a, int nblocks, cudaStream_t s, bool xt) {
  return by_nf(a.g.nf, [&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    if (a.g.recon == RECON_PRIM)
      return xt ? launch<NF, P, true, RECON_PRIM>(a, nblocks, s) : launch<NF, P, false, RECON_PRIM>(a, nblocks, s);
    return xt ? launch<NF, P, true, RECON_CONS>(a, nblocks, s) : launch<NF, P, false, RECON_CONS>(a, nblocks, s);
  });
}

#ifndef ROSSBI_F32_GENERIC_GAMMA
template cudaError_t run_stage_pert_f32_p<PowG75>(const PertArgs<float>&, int, cudaStream_t, bool);
#else
template cudaError_t run_stage_pert_f32_p<PowGeneric<float>>(const PertArgs<float>&, int, cudaStream_t, bool);
#endif

}  // namespace rossbi
