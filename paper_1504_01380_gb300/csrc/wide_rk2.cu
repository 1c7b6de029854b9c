// Wide windows of uneven tiles: two-stage Runge-Kutta heat and KS (FP64 pairs).
#include "swept_wide.cuh"

namespace swept {
cudaError_t launch_wide_rk2(int stencil, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s, int ring) {
  if (stencil == kHeatRK2) {
    switch (K) {
      case 1: return launch_wk<kHeatRK2, F64P, 1, 2>(a, nreg, odd, s, ring);
      case 2: return launch_wk<kHeatRK2, F64P, 2, 3>(a, nreg, odd, s, ring);
      case 4: return launch_wk<kHeatRK2, F64P, 4, 5>(a, nreg, odd, s, ring);
      case 8: return launch_wk<kHeatRK2, F64P, 8, 9>(a, nreg, odd, s, ring);
      case 16: return launch_wk<kHeatRK2, F64P, 16, 17>(a, nreg, odd, s, ring);
      case 32: return launch_wk<kHeatRK2, F64P, 32, 33>(a, nreg, odd, s, ring);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (K) {
    case 2: return launch_wk<kKSRK2, F64P, 2, 4>(a, nreg, odd, s, ring);
    case 4: return launch_wk<kKSRK2, F64P, 4, 6>(a, nreg, odd, s, ring);
    case 8: return launch_wk<kKSRK2, F64P, 8, 10>(a, nreg, odd, s, ring);
    case 16: return launch_wk<kKSRK2, F64P, 16, 18>(a, nreg, odd, s, ring);
    case 32: return launch_wk<kKSRK2, F64P, 32, 34>(a, nreg, odd, s, ring);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace swept
