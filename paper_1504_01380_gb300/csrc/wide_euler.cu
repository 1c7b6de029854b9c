// Wide windows of uneven tiles: Euler equations, FP64 (K <= 4) and compensated FP32 (K <= 8).
#include "swept_wide.cuh"

namespace swept {
cudaError_t launch_wide_euler(int dtype, int K, const StageArgs& a, int nreg, int odd, cudaStream_t s) {
  if (dtype == 0) {
    switch (K) {
      case 1: return launch_wk<kEuler, F64E, 1, 2>(a, nreg, odd, s);
      case 2: return launch_wk<kEuler, F64E, 2, 3>(a, nreg, odd, s);
      case 4: return launch_wk<kEuler, F64E, 4, 5>(a, nreg, odd, s);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (K) {
    case 1: return launch_wk<kEuler, F32CE, 1, 2>(a, nreg, odd, s);
    case 2: return launch_wk<kEuler, F32CE, 2, 3>(a, nreg, odd, s);
    case 4: return launch_wk<kEuler, F32CE, 4, 5>(a, nreg, odd, s);
    case 8: return launch_wk<kEuler, F32CE, 8, 9>(a, nreg, odd, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace swept
