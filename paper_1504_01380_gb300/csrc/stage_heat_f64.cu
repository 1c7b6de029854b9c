// Instantiation of the swept stage kernel: heat, f64.
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_heat_f64(int K, const StageArgs& a, cudaStream_t s) {
  return launch_stage_dispatch<kHeat, F64>(K, a, s);
}
}  // namespace swept
