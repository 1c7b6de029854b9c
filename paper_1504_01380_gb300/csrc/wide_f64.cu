// Wide windows of uneven tiles: forward-Euler heat and KS, F64 state.
#include "swept_wide.cuh"

namespace swept {
namespace {
template <class DT>
cudaError_t launch_wide_dt(int stencil, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring) {
  if (stencil == kHeat) {
    switch (K) {
      case 1: return launch_wk<kHeat, DT, 1, 2>(a, nreg, odd, s, ring);
      case 2: return launch_wk<kHeat, DT, 2, 3>(a, nreg, odd, s, ring);
      case 4: return launch_wk<kHeat, DT, 4, 5>(a, nreg, odd, s, ring);
      case 8: return launch_wk<kHeat, DT, 8, 9>(a, nreg, odd, s, ring);
      case 16: return launch_wk<kHeat, DT, 16, 17>(a, nreg, odd, s, ring);
      case 32: return launch_wk<kHeat, DT, 32, 33>(a, nreg, odd, s, ring);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (K) {
    case 2: return launch_wk<kKS, DT, 2, 4>(a, nreg, odd, s, ring);
    case 4: return launch_wk<kKS, DT, 4, 6>(a, nreg, odd, s, ring);
    case 8: return launch_wk<kKS, DT, 8, 10>(a, nreg, odd, s, ring);
    case 16: return launch_wk<kKS, DT, 16, 18>(a, nreg, odd, s, ring);
    case 32: return launch_wk<kKS, DT, 32, 34>(a, nreg, odd, s, ring);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace

cudaError_t launch_wide_f64(int stencil, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring) {
  return launch_wide_dt<F64>(stencil, K, a, nreg, odd, s, ring);
}
}  // namespace swept
