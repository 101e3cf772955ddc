// probe.cu -- peak rates for the roofline of the render kernels: kernels of
// independent dependency chains that keep one execution unit of every SM
// busy, timed by the caller.  They are measurements, not part of the
// rendering path.
//   FFMA   binary32 fused multiply-add (2 flops each)
//   FFMA2  the packed two-lane binary32 fused multiply-add of sm_100-class
//          GPUs (4 flops per instruction); the render kernels evaluate a
//          lane's two pixels with it
//   EX2    the special-function unit's base-2 exponential (one op each)
//   RCP    the special-function unit's reciprocal (one op each)
#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

constexpr int kProbeThreads = 256;
constexpr int kProbeChains = 8;  // independent chains per thread (covers the pipe latency)

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

__global__ void __launch_bounds__(kProbeThreads) fma2_probe_kernel(float *out, int iters, float x) {
  const float2 y = make_float2(0.9999999f, 0.9999998f), xx = make_float2(x, x);
  float2 a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = make_float2(x + (float)(threadIdx.x + k), x - (float)k);
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = __ffma2_rn(a[k], y, xx);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k].x + a[k].y;
  if (s == -1.0f) out[blockIdx.x] = s;
}

// EX2: a <- 2^(-a) keeps a in [0.5, 1] once it is there; each step is one
// special-function op (the negation is an operand modifier).  RCP: a <- 1/a
// + 1 converges to the golden ratio; each step is one special-function op and
// one add, so the issue slots allow twice the special-function rate the unit
// is expected to have and the special-function unit stays the bound (a bare
// chain of reciprocals can be shortened by the compiler, which pairs them).
__device__ __forceinline__ float probe_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float probe_rcp(float x) {
  float y;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

template <int KIND>
__global__ void __launch_bounds__(kProbeThreads) mufu_probe_kernel(float *out, int iters, float x) {
  float a[kProbeChains];
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) a[k] = 0.5f + 0.01f * (float)((threadIdx.x + k) & 31) + 0.0f * x;
#pragma unroll 16
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kProbeChains; ++k) a[k] = KIND == HGS_PROBE_EX2 ? probe_ex2(-a[k]) : __fadd_rn(probe_rcp(a[k]), 1.0f);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < kProbeChains; ++k) s += a[k];
  if (s == -1.0f) out[blockIdx.x] = s;
}

int launch_alu_probe(int kind, int blocks, int iters, float *out, double *ops, cudaStream_t s) {
  const double steps = (double)kProbeChains * (double)iters * (double)kProbeThreads * (double)blocks;
  switch (kind) {
    case HGS_PROBE_FFMA:
      fma_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.5f);
      *ops = 2.0 * steps;
      return 0;
    case HGS_PROBE_FFMA2:
      fma2_probe_kernel<<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.5f);
      *ops = 4.0 * steps;
      return 0;
    case HGS_PROBE_EX2:
      mufu_probe_kernel<HGS_PROBE_EX2><<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.5f);
      *ops = steps;
      return 0;
    case HGS_PROBE_RCP:
      mufu_probe_kernel<HGS_PROBE_RCP><<<blocks, kProbeThreads, 0, s>>>(out, iters, 0.5f);
      *ops = steps;
      return 0;
    default:
      return -1;
  }
}

}  // namespace hgs
