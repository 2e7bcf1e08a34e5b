// Launcher of the FP32 perturbation-form stage kernel (stage_pert.cuh) for
// one power form of the solver (ROSSBI_POW: the gamma = 7/5 integer powers
// unless the including translation unit chose the general ones) and one gas
// reconstruction mode (ROSSBI_RC, conservative unless chosen otherwise).
#include "launch.cuh"

#ifndef ROSSBI_RC
#define ROSSBI_RC RECON_CONS
#endif
#ifndef ROSSBI_POW
#define ROSSBI_POW PowG75
#endif

namespace rossbi {
namespace {

template <int NF, class P, bool XT, int RC>
cudaError_t launch(const PertArgs<float>& a, int nblocks, cudaStream_t s) {
  constexpr size_t smem = pert_smem_bytes<float, NF, P32_TR, P32_TT, P32_TZ>();
  auto kern = stage_pert_kernel<float, NF, P32_TR, P32_TT, P32_TZ, P32_NT, P32_MINB, P, XT, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, P32_NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <class P, int RC>
cudaError_t run_stage_pert_f32_rc(const PertArgs<float>& a, int nblocks, cudaStream_t s, bool xt) {
  return by_nf(a.g.nf, [&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    return xt ? launch<NF, P, true, RC>(a, nblocks, s) : launch<NF, P, false, RC>(a, nblocks, s);
  });
}

template cudaError_t run_stage_pert_f32_rc<ROSSBI_POW, ROSSBI_RC>(const PertArgs<float>&, int, cudaStream_t, bool);

}  // namespace rossbi
