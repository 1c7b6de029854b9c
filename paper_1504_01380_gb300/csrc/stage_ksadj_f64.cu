// Instantiation of the swept stage kernel for the transposed KS step (adjoint), FP64.
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_ksadj_f64(int K, const StageArgs& a, cudaStream_t s) {
  return launch_stage_dispatch<kKSAdj, F64>(K, a, s);
}
}  // namespace swept
