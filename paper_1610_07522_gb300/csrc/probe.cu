// FMA-chain probe: the FP64 or FP32 fused multiply-add rate of the device,
// the denominator of the roofline fractions of the kernels bound by those
// pipes (the FP64 FFT line passes, h psi, the eigensolver).  Every thread
// runs 8 independent dependency chains a <- a * b + c (8 chains hide the FMA
// latency), so the pipe, not the latency, limits the rate; the result is
// stored only under a condition that never holds, which keeps the chains live.
#include "sky_internal.cuh"

namespace sky {
namespace {

constexpr int kChains = 8;

template <typename T>
__global__ void __launch_bounds__(256) k_fma_probe(int iters, T b, T c, T* sink) {
  T a[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) a[i] = (T)(threadIdx.x + 1) * (T)(i + 1) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < kChains; ++i) a[i] = fma(a[i], b, c);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) s += a[i];
  if (s == (T)-1.2345e-7) sink[blockIdx.x] = s;
}

}  // namespace
}  // namespace sky

using namespace sky;

extern "C" sky_status sky_fma_probe(int fp64, int blocks_per_sm, int iters, void* stream,
                                    double* flops) {
  if (!flops || blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1) return SKY_EINVAL;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return SKY_ECUDA;
  }
  const int blocks = blocks_per_sm * sms, threads = 256;
  cudaStream_t s = (cudaStream_t)stream;
  // b = 1 - 2^-20 and c small keep the chains finite for any iteration count;
  // the sink is never written (the condition above never holds), so a null
  // pointer is never dereferenced
  if (fp64)
    k_fma_probe<double><<<blocks, threads, 0, s>>>(iters, 1.0 - 0x1p-20, 1e-9, (double*)nullptr);
  else
    k_fma_probe<float><<<blocks, threads, 0, s>>>(iters, 1.0f - 0x1p-20f, 1e-9f, (float*)nullptr);
  note_launch();
  *flops = 2.0 * kChains * (double)iters * blocks * threads;
  return cudaGetLastError() == cudaSuccess ? SKY_OK : SKY_ECUDA;
}
