// Instantiation of the swept stage and ring kernels: two-stage Runge-Kutta (ks), FP64 pairs.
#include "swept_ring.cuh"
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_ksrk2_f64(int K, const StageArgs& a, cudaStream_t s) {
  return launch_stage_dispatch<kKSRK2, F64P>(K, a, s);
}
cudaError_t launch_ring_ksrk2_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s) {
  return launch_ring_dispatch<kKSRK2, F64P>(K, a, nwarps, s);
}
}  // namespace swept
