// Instantiation of the swept stage and ring kernels for the transposed KS step (adjoint), FP64.
#include "swept_ring.cuh"
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_ksadj_f64(int K, const StageArgs& a, cudaStream_t s) {
  return launch_stage_dispatch<kKSAdj, F64>(K, a, s);
}
cudaError_t launch_ring_ksadj_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s) {
  return launch_ring_dispatch<kKSAdj, F64>(K, a, nwarps, s);
}
}  // namespace swept
