// probe.cu -- the FP32 peak for the roofline of the render kernels: a kernel
// of independent fused multiply-add chains that keeps every FP32 lane busy,
// timed by the caller.  It is a measurement, not part of the rendering path.
#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent chains per thread (covers the FMA latency)

__global__ void __launch_bounds__(kProbeThreads) fma_probe_kernel(float *out, int iters, float x) {
  // a <- a * y + x with |y| < 1 stays bounded; nothing lets the compiler
  // shorten the chains (no reassociation of FP arithmetic)
  const float y = 0.9999999f;
  float a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = x + (float)(threadIdx.x + k);
#pragma unroll 16  // 128 FMAs per loop test: the loop overhead stays under 3% of the issue slots
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = __fmaf_rn(a[k], y, x);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == -1.0f) out[blockIdx.x] = s;  // never true; keeps the chains live
}

int launch_fp32_probe(int blocks, int iters, float *out, double *flops, cudaStream_t s) {
  fma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.5f);
  *flops = 2.0 * kProbeChains * (double)iters * (double)kProbeThreads * (double)blocks;
  return 0;
}

}  // namespace hgs
