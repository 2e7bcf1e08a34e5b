// Launcher of the adjoint flux kernel (adjoint.cuh).
#include "launch.cuh"

namespace rossbi {
namespace {

template <int NF, int D, int RC>
cudaError_t launch(const AdjFluxArgs& a, cudaStream_t s) {
  constexpr size_t smem = adj_flux_smem_doubles<NF, ADJ_L, ADJ_NL>() * sizeof(double);
  constexpr int T = ADJ_L - 4;
  auto kern = adj_flux_kernel<NF, D, ADJ_L, ADJ_NL, RC>;
  static unsigned long long done = 0;
  cudaError_t e = set_smem_once(kern, smem, done);
  if (e != cudaSuccess) return e;
  const DevGrid& g = a.g;
  const long nd = D == 0 ? g.nr : (D == 1 ? g.nth : g.nz);
  const long nlines = D == 0 ? (long)g.nth * g.nz : (D == 1 ? (long)g.nr * g.nz : (long)g.nr * g.nth);
  const long nblocks = ((nd + T - 1) / T) * ((nlines + ADJ_NL - 1) / ADJ_NL);
  kern<<<(unsigned)nblocks, ADJ_L * ADJ_NL, smem, s>>>(a);
  return cudaGetLastError();
}

template <int NF, int RC>
cudaError_t launch_axis(const AdjFluxArgs& a, int axis, cudaStream_t s) {
  if (axis == 0) return launch<NF, 0, RC>(a, s);
  if (axis == 1) return launch<NF, 1, RC>(a, s);
  return launch<NF, 2, RC>(a, s);
}

}  // namespace

cudaError_t run_adj_flux(const AdjFluxArgs& a, int axis, cudaStream_t s) {
  if (a.g.recon == RECON_PRIM)
    return a.g.nf == 9 ? launch_axis<9, RECON_PRIM>(a, axis, s) : launch_axis<5, RECON_PRIM>(a, axis, s);
  return a.g.nf == 9 ? launch_axis<9, RECON_CONS>(a, axis, s) : launch_axis<5, RECON_CONS>(a, axis, s);
}

}  // namespace rossbi
