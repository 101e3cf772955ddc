// exchange.cu -- Adaptive Type Exchange in place (EGGS Sec. 3.2, Eqs. 3-5;
// App. D, Eqs. 17-19).  One thread per primitive; no buffer is reallocated,
// compacted or reordered.
#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

// Hamilton product a (x) b, quaternions as (w, x, y, z)
__device__ __forceinline__ float4 qmul(float4 a, float4 b) {
  return make_float4(a.x * b.x - a.y * b.y - a.z * b.z - a.w * b.w,
                     a.x * b.y + a.y * b.x + a.z * b.w - a.w * b.z,
                     a.x * b.z - a.y * b.w + a.z * b.x + a.w * b.y,
                     a.x * b.w + a.y * b.z - a.z * b.y + a.w * b.x);
}

// erank (Eq. 3) compared with theta.  Decided in binary32 when the margin is
// clear; otherwise in binary64 from the definition erank = exp(H).
__device__ __forceinline__ int erank_side(float l0, float l1, float l2, float theta) {
  const float m = fmaxf(l0, fmaxf(l1, l2));
  const float w0 = expf(2.f * (l0 - m)), w1 = expf(2.f * (l1 - m)), w2 = expf(2.f * (l2 - m));
  const float S = w0 + w1 + w2;
  float H = 0.f;
  const float ws[3] = {w0, w1, w2};
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float p = ws[k] / S;
    if (p > 0.f) H -= p * logf(p);
  }
  const float lt = logf(theta);
  if (fabsf(H - lt) > 1e-4f) return H < lt ? -1 : 1;
  const double q0 = exp(2.0 * (double)l0), q1 = exp(2.0 * (double)l1), q2 = exp(2.0 * (double)l2);
  const double s = q0 + q1 + q2;
  const double qs[3] = {q0, q1, q2};
  double Hd = 0.0;
  for (int k = 0; k < 3; ++k) {
    const double p = qs[k] / s;
    if (p > 0.0) Hd -= p * log(p);
  }
  const double er = exp(Hd);
  return er < (double)theta ? -1 : (er > (double)theta ? 1 : 0);
}

__global__ void __launch_bounds__(256) exchange_kernel(ExchangeArgs a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int flip = 0;
  if (i < a.n) {
    const int t = a.types[i] ? 1 : 0;
    float l0 = a.log_scales[3 * i], l1 = a.log_scales[3 * i + 1], l2 = a.log_scales[3 * i + 2];
    if (a.mode == HGS_EXCHANGE_MASK) {
      flip = a.mask[i] != 0;
    } else {
      const int side = erank_side(l0, l1, l2, a.theta);
      flip = t ? (side < 0) : (side > 0);
    }
    if (flip) {
      if (t == 1 && !(l2 <= l0 && l2 <= l1)) {
        // move the least significant scale to z: S* = P S P^T, R* = R P^T
        float4 q = reinterpret_cast<float4 *>(a.quats)[i];
        float4 p;
        float n0, n1, n2;
        if (l0 <= l1) {  // P_x
          p = make_float4(0.5f, 0.5f, 0.5f, 0.5f);
          n0 = l1; n1 = l2; n2 = l0;
        } else {         // P_y
          p = make_float4(0.5f, -0.5f, -0.5f, -0.5f);
          n0 = l2; n1 = l0; n2 = l1;
        }
        reinterpret_cast<float4 *>(a.quats)[i] = qmul(q, p);
        a.log_scales[3 * i] = n0;
        a.log_scales[3 * i + 1] = n1;
        a.log_scales[3 * i + 2] = n2;
      }
      a.types[i] = (uint8_t)(1 - t);
    }
  }
  const int cnt = __syncthreads_count(flip);
  if (threadIdx.x == 0 && cnt && a.n_flipped) atomicAdd(a.n_flipped, (unsigned long long)cnt);
}

int launch_exchange(const ExchangeArgs &a, cudaStream_t s) {
  if (a.n == 0) return 0;
  exchange_kernel<<<(unsigned)((a.n + 255) / 256), 256, 0, s>>>(a);
  return 0;
}

}  // namespace hgs
