// Instantiation of the swept stage and ring kernels: two-stage Runge-Kutta (heat), FP64 pairs.
#include "swept_ring.cuh"
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_heatrk2_f64(int K, const StageArgs& a, cudaStream_t s) {
  return launch_stage_dispatch<kHeatRK2, F64P>(K, a, s);
}
cudaError_t launch_ring_heatrk2_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s) {
  return launch_ring_dispatch<kHeatRK2, F64P>(K, a, nwarps, s);
}
}  // namespace swept
