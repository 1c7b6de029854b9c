// Instantiation of the swept stage and ring kernels: Euler equations on the
// compensated FP32 state (point states of 12 floats, 48-byte edges).  Tile
// widths B = 32 .. 256: 2B edge elements per warp of shared memory (4 warps:
// 12, 25, 49, 98 KB) and 12K state registers per lane.
#include "swept_ring.cuh"
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_euler_f32c(int K, const StageArgs& a, cudaStream_t s) {
  switch (K) {
    case 1: return launch_stage_k<kEuler, F32CE, 1>(a, s);
    case 2: return launch_stage_k<kEuler, F32CE, 2>(a, s);
    case 4: return launch_stage_k<kEuler, F32CE, 4>(a, s);
    case 8: return launch_stage_k<kEuler, F32CE, 8>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_ring_euler_f32c(int K, const StageArgs& a, int nwarps, cudaStream_t s) {
  switch (K) {
    case 1: return launch_ring_k<kEuler, F32CE, 1>(a, nwarps, s);
    case 2: return launch_ring_k<kEuler, F32CE, 2>(a, nwarps, s);
    case 4: return launch_ring_k<kEuler, F32CE, 4>(a, nwarps, s);
    case 8: return launch_ring_k<kEuler, F32CE, 8>(a, nwarps, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace swept
