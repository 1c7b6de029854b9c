// Instantiation of the swept stage and ring kernels: heat, plain binary32 (diagnostic precision).
#include "swept_ring.cuh"
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_heat_f32(int K, const StageArgs& a, cudaStream_t s) {
  return launch_stage_dispatch<kHeat, F32>(K, a, s);
}
cudaError_t launch_ring_heat_f32(int K, const StageArgs& a, int nwarps, cudaStream_t s) {
  return launch_ring_dispatch<kHeat, F32>(K, a, nwarps, s);
}
}  // namespace swept
