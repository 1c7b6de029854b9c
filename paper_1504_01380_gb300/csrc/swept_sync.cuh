// Device-side synchronisation between warps of one persistent launch: flags
// published with release semantics and read with acquire semantics, and a
// bounded wait (a clock budget; no wait in this library is unbounded).
#pragma once

#include <cstdint>

namespace swept {

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Wait until *flag >= target (acquire), sleeping `nap` ns between polls.  False
// when the clock budget (cycles from t0) ran out or *status became nonzero.
__device__ __forceinline__ bool wait_ge(const int* flag, int target, long long t0, long long budget,
                                        const int* status = nullptr, unsigned nap = 256) {
  for (;;) {
    if (ld_acquire(flag) >= target) return true;
    if (clock64() - t0 > budget) return false;
    if (status && ld_acquire(status) != 0) return false;
    __nanosleep(nap);
  }
}

// Shape of stage s of an advance of q*H + rem levels (the schedule of
// swept_advance): (V-fill height, trapezoid height).
__host__ __device__ __forceinline__ void stage_shape(int s, int q, int rem, int H, int& hv, int& ht) {
  if (q == 0) {
    hv = s == 0 ? 0 : rem;
    ht = s == 0 ? rem : 0;
  } else if (s == 0) {
    hv = 0; ht = H;
  } else if (s < q) {
    hv = H; ht = H;
  } else if (s == q) {
    hv = H; ht = rem;
  } else {
    hv = rem; ht = 0;
  }
}

}  // namespace swept
