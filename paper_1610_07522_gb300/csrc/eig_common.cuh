// Device helpers shared by the two FP64 eigensolvers (cyclic Jacobi and the
// Householder / bisection / inverse-iteration solver): refined reciprocals
// and the bounded grid barrier of their cooperative kernels.
#pragma once

#include "sky_internal.cuh"

namespace sky {

// x^{-1/2} from an FP32 seed and two Newton steps in FP64, r <- r (3 - x r^2)/2
// (relative error 1e-7 -> 1e-14 -> rounding); x must lie in the FP32 range.
__device__ __forceinline__ double rsqrt_refined(double x) {
  double r = (double)rsqrtf((float)x);
  r = r * fma(-0.5 * x, r * r, 1.5);
  r = r * fma(-0.5 * x, r * r, 1.5);
  return r;
}

// 1/x from an FP32 seed and two Newton steps in FP64, r <- r (2 - x r);
// x must lie in the FP32 range.
__device__ __forceinline__ double rcp_refined(double x) {
  double r = (double)__frcp_rn((float)x);
  r = r * fma(-x, r, 2.0);
  r = r * fma(-x, r, 2.0);
  return r;
}

// Barrier over `count` blocks of a cooperative launch that share the arrival
// counter `bar` (reset before the launch): barrier number e completes when
// the counter reaches e * count.  Release-add to arrive, acquire loads to
// wait, with a bounded spin: on timeout it flags SKY_ETIMEOUT and returns
// false.  The whole grid is count = gridDim.x.
__device__ __forceinline__ bool blocks_barrier(unsigned* bar, unsigned& epoch, unsigned count,
                                               int* status, long long max_spins) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const unsigned target = epoch * count;
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(bar) : "memory");
    int ok = 1;
    long long spins = 0;
    for (;;) {
      unsigned v;
      asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(bar) : "memory");
      if ((int)(v - target) >= 0) break;
      if (++spins > max_spins || (*(volatile int*)status & SKY_STATUS_BIT(SKY_ETIMEOUT))) {
        flag_status(status, SKY_ETIMEOUT);
        ok = 0;
        break;
      }
      if (spins > 64) __nanosleep(32);
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}
__device__ __forceinline__ bool grid_barrier(unsigned* bar, unsigned& epoch, int* status,
                                             long long max_spins) {
  return blocks_barrier(bar, epoch, gridDim.x, status, max_spins);
}

// Problem of item w: the last b with off[b] <= w (off ascending, off[np] > w).
__device__ __forceinline__ int find_prob(const int* off, int np, int w) {
  int lo = 0, hi = np - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= w) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace sky
