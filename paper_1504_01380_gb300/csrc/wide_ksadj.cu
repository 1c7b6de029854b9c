// Wide windows of uneven tiles: the transposed KS step (the adjoint sweep), FP64.
#include "swept_wide.cuh"

namespace swept {
cudaError_t launch_wide_ksadj(int K, const StageArgs& a, int nreg, int odd, cudaStream_t s) {
  switch (K) {
    case 2: return launch_wk<kKSAdj, F64, 2, 4>(a, nreg, odd, s);
    case 4: return launch_wk<kKSAdj, F64, 4, 6>(a, nreg, odd, s);
    case 8: return launch_wk<kKSAdj, F64, 8, 10>(a, nreg, odd, s);
    case 16: return launch_wk<kKSAdj, F64, 16, 18>(a, nreg, odd, s);
    case 32: return launch_wk<kKSAdj, F64, 32, 34>(a, nreg, odd, s);
    default: return cudaErrorInvalidValue;
  }
}
}  // namespace swept
