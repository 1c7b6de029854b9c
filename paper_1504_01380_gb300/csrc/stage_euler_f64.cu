// Instantiation of the swept stage and ring kernels: Euler equations of gas
// dynamics (FP64 point states of 9 values).  Tile widths B = 32, 64, 128:
// the 72-byte edge elements make 2B elements per warp of shared memory
// (4 warps: 18, 37, 74 KB), and the state takes 18K registers per lane.
#include "swept_ring.cuh"
#include "swept_stage.cuh"

namespace swept {
cudaError_t launch_stage_euler_f64(int K, const StageArgs& a, cudaStream_t s) {
  switch (K) {
    case 1: return launch_stage_k<kEuler, F64E, 1>(a, s);
    case 2: return launch_stage_k<kEuler, F64E, 2>(a, s);
    case 4: return launch_stage_k<kEuler, F64E, 4>(a, s);
    default: return cudaErrorInvalidValue;
  }
}
cudaError_t launch_ring_euler_f64(int K, const StageArgs& a, int nwarps, cudaStream_t s) {
  switch (K) {
    case 1: return launch_ring_k<kEuler, F64E, 1>(a, nwarps, s);
    case 2: return launch_ring_k<kEuler, F64E, 2>(a, nwarps, s);
    case 4: return launch_ring_k<kEuler, F64E, 4>(a, nwarps, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace swept
