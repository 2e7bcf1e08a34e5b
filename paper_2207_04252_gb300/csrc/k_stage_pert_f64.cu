// Launcher of the FP64 perturbation-form stage kernel (stage_pert.cuh) for
// one gas reconstruction mode (ROSSBI_RC, conservative unless the including
// translation unit chose another).
#include "launch.cuh"

#ifndef ROSSBI_RC
#define ROSSBI_RC RECON_CONS
#endif

namespace rossbi {
namespace {

template <int NF, int TZ, bool XT, int RC>
cudaError_t launch(const PertArgs<double>& a, int nblocks, cudaStream_t s) {
  constexpr size_t smem = pert_smem_bytes<double, NF, P32_TR, P32_TT, TZ>();
  auto kern = stage_pert_kernel<double, NF, P32_TR, P32_TT, TZ, P32_NT, 1, PowGeneric<double>, XT, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  kern<<<nblocks, P32_NT, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace

template <int RC>
cudaError_t run_stage_pert_f64_rc(const PertArgs<double>& a, int nblocks, cudaStream_t s, bool xt) {
  return by_nf(a.g.nf, [&](auto nf) {
    constexpr int NF = decltype(nf)::value;
    constexpr int TZ = tile_z(true, NF);
    return xt ? launch<NF, TZ, true, RC>(a, nblocks, s) : launch<NF, TZ, false, RC>(a, nblocks, s);
  });
}

template cudaError_t run_stage_pert_f64_rc<ROSSBI_RC>(const PertArgs<double>&, int, cudaStream_t, bool);

}  // namespace rossbi
