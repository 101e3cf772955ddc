// train.cu -- the training loop around the rasterizer (EGGS App. A: the
// 3DGS setup, with Adaptive Type Exchange every 500 iterations and
// densification every 100 iterations from 500 to 15K):
//   * a fused Adam update over the parameter arrays (float4 streams);
//   * the per-primitive gradient statistic densification uses: the norm of
//     the loss gradient with respect to the projected centre (pixels), read
//     from the backward's record gradients, and a visibility count;
//   * densification in two launches: a plan (per-primitive action and output
//     count, exclusive scan, new count) and an apply (rows copied, cloned or
//     split into their new slots; new primitives get zero Adam moments);
//   * the opacity reset (alpha <- min(alpha, ceiling), moments zeroed).
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

// ---------------------------------------------------------------------------
// Adam (bias-corrected form): m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
// p -= (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
// ---------------------------------------------------------------------------
// step = lr / (1 - b1^t) and isb2 = 1 / sqrt(1 - b2^t) are the same for every
// element of a group, so each thread forms them once (one division per
// element remains).
struct AdamStep {
  float head, tail, isb2;
};
__device__ __forceinline__ AdamStep adam_step(const AdamArgs &a, const AdamGroup &g) {
  return AdamStep{g.lr / a.bc1, g.lr_tail / a.bc1, 1.0f / a.sqrt_bc2};
}
__device__ __forceinline__ float adam_one(float &p, float g, float &m, float &v, const AdamArgs &a, float step,
                                          float isb2) {
  m = fmaf(a.beta1, m, a.omb1 * g);
  v = fmaf(a.beta2, v, a.omb2 * g * g);
  p -= step * m / fmaf(sqrtf(v), isb2, a.eps);
  return p;
}

// Step size of the element whose position in its row of `period` is r
// (r < period + 3 is reduced once).
__device__ __forceinline__ float step_at(const AdamGroup &g, const AdamStep &st, uint32_t r) {
  if (g.period <= 0) return st.head;
  if (r >= (uint32_t)g.period) r -= (uint32_t)g.period;
  return r < (uint32_t)g.head ? st.head : st.tail;
}

// The row position advances by a fixed stride per grid step, so it is kept
// incrementally instead of divided per element.
__global__ void __launch_bounds__(256) adam_kernel(AdamArgs a, AdamGroup grp) {
  const int64_t n = grp.count;
  const bool vec = ((reinterpret_cast<uintptr_t>(grp.param) | reinterpret_cast<uintptr_t>(grp.grad) |
                     reinterpret_cast<uintptr_t>(grp.m) | reinterpret_cast<uintptr_t>(grp.v)) & 15u) == 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint64_t P = grp.period > 0 ? (uint64_t)grp.period : 1;
  const AdamStep st = adam_step(a, grp);
  int64_t done = 0;
  if (vec) {
    const int64_t n4 = n / 4;
    float4 *Pp = reinterpret_cast<float4 *>(grp.param), *M = reinterpret_cast<float4 *>(grp.m),
           *V = reinterpret_cast<float4 *>(grp.v);
    const float4 *G = reinterpret_cast<const float4 *>(grp.grad);
    uint32_t r = (uint32_t)((4 * (uint64_t)tid) % P);
    const uint32_t inc = (uint32_t)((4 * (uint64_t)stride) % P);
    for (int64_t k = tid; k < n4; k += stride) {
      float4 p = Pp[k], m = M[k], v = V[k];
      const float4 g = __ldg(G + k);
      adam_one(p.x, g.x, m.x, v.x, a, step_at(grp, st, r), st.isb2);
      adam_one(p.y, g.y, m.y, v.y, a, step_at(grp, st, r + 1), st.isb2);
      adam_one(p.z, g.z, m.z, v.z, a, step_at(grp, st, r + 2), st.isb2);
      adam_one(p.w, g.w, m.w, v.w, a, step_at(grp, st, r + 3), st.isb2);
      Pp[k] = p; M[k] = m; V[k] = v;
      r += inc;
      if (r >= (uint32_t)P) r -= (uint32_t)P;
    }
    done = n4 * 4;
  }
  for (int64_t k = done + tid; k < n; k += stride) {
    float p = grp.param[k], m = grp.m[k], v = grp.v[k];
    adam_one(p, grp.grad[k], m, v, a, step_at(grp, st, (uint32_t)((uint64_t)k % P)), st.isb2);
    grp.param[k] = p; grp.m[k] = m; grp.v[k] = v;
  }
}

int launch_adam(const AdamArgs &a, const AdamGroup &g, cudaStream_t s) {
  if (g.count <= 0) return 0;
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t want = (g.count / 4 + 255) / 256 + 1;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)sms * 8));
  adam_kernel<<<grid, 256, 0, s>>>(a, g);
  return 0;
}

// ---------------------------------------------------------------------------
// gradient statistic: |dL/d(projected centre)| from record slots 4, 5
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) grad_stats_kernel(int64_t n, const float *__restrict__ rec_grad,
                                                         const uint32_t *__restrict__ touched,
                                                         float *__restrict__ accum, float *__restrict__ count) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    if (__ldg(touched + i) == 0u) continue;
    const float2 g = __ldg(reinterpret_cast<const float2 *>(rec_grad + kGradW * i + 4));
    accum[i] += sqrtf(g.x * g.x + g.y * g.y);
    count[i] += 1.0f;
  }
}

int launch_grad_stats(int64_t n, const float *rec_grad, const uint32_t *touched, float *accum, float *count,
                      cudaStream_t s) {
  if (n <= 0) return 0;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  grad_stats_kernel<<<grid, 256, 0, s>>>(n, rec_grad, touched, accum, count);
  return 0;
}

// ---------------------------------------------------------------------------
// densification
// ---------------------------------------------------------------------------
// action: 0 remove, 1 keep, 2 keep + clone, 3 split into two; all decided
// in binary32.  Size = largest active scale (a surfel's two in-plane ones),
// compared as its log-scale against log(size threshold); opacity compared as
// its logit against logit(min opacity) -- monotonic maps, exact decisions.
__global__ void __launch_bounds__(256) densify_mark_kernel(DensifyPlanArgs a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const float cnt = a.vis_count[i];
    const float mg = cnt > 0.0f ? __fdiv_rn(a.grad_accum[i], cnt) : 0.0f;
    const float l0 = a.log_scales[3 * i], l1 = a.log_scales[3 * i + 1], l2 = a.log_scales[3 * i + 2];
    float lmax = fmaxf(l0, l1);
    if (a.types[i]) lmax = fmaxf(lmax, l2);
    const bool hot = mg >= a.grad_thresh, big = lmax > a.log_size_thresh;
    int act = hot ? (big ? 3 : 2) : 1;
    if (act == 1 && a.logits[i] < a.logit_min_opacity) act = 0;
    a.actions[i] = act;
    a.counts[i] = act == 0 ? 0 : (act == 1 ? 1 : 2);
  }
}

// exclusive scan of counts[0..n) into offsets[0..n], offsets[n] = total
__global__ void __launch_bounds__(1024) scan_block_sums(int64_t n, const int32_t *__restrict__ counts,
                                                        int64_t *__restrict__ partial, int per) {
  __shared__ int64_t ws[32];
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
  int64_t s = 0;
  for (int64_t i = b0 + threadIdx.x; i < b1; i += blockDim.x) s += counts[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += ws[w];
    partial[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(1024) scan_partials(int nb, int64_t *__restrict__ partial, int64_t *__restrict__ total,
                                                      int64_t *__restrict__ offsets_end) {
  __shared__ int64_t ws[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t v = tid < nb ? partial[tid] : 0;
  int64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) ws[warp] = incl;
  __syncthreads();
  int64_t base = 0;
  for (int w = 0; w < warp; ++w) base += ws[w];
  if (tid < nb) partial[tid] = base + incl - v;
  if (tid == blockDim.x - 1) {
    *total = base + incl;
    *offsets_end = base + incl;
  }
}

__global__ void __launch_bounds__(1024) scan_final(int64_t n, const int32_t *__restrict__ counts,
                                                   const int64_t *__restrict__ partial, int64_t *__restrict__ offsets,
                                                   int per) {
  __shared__ int64_t ws[32];
  __shared__ int64_t carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t b0 = (int64_t)blockIdx.x * per, b1 = min(n, b0 + per);
  if (tid == 0) carry = partial[blockIdx.x];
  __syncthreads();
  for (int64_t tb = b0; tb < b1; tb += blockDim.x) {
    const int64_t i = tb + tid;
    const int64_t c = i < b1 ? counts[i] : 0;
    int64_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) ws[warp] = incl;
    __syncthreads();
    int64_t wb = 0, all = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      if (w < warp) wb += ws[w];
      all += ws[w];
    }
    if (i < b1) offsets[i] = carry + wb + incl - c;
    __syncthreads();
    if (tid == 0) carry += all;
    __syncthreads();
  }
}

constexpr int kScanBlocks = 1024;

int launch_densify_plan(const DensifyPlanArgs &a, cudaStream_t s) {
  if (a.n <= 0) {
    cudaMemsetAsync(a.d_new_n, 0, sizeof(int64_t), s);
    cudaMemsetAsync(a.offsets, 0, sizeof(int64_t), s);
    return 0;
  }
  const int grid = (int)std::min<int64_t>((a.n + 255) / 256, 152 * 16);
  densify_mark_kernel<<<grid, 256, 0, s>>>(a);
  const int per = (int)((a.n + kScanBlocks - 1) / kScanBlocks);
  const int nb = (int)((a.n + per - 1) / per);
  scan_block_sums<<<nb, 1024, 0, s>>>(a.n, a.counts, a.partial, per);
  scan_partials<<<1, 1024, 0, s>>>(nb, a.partial, a.d_new_n, a.offsets + a.n);
  scan_final<<<nb, 1024, 0, s>>>(a.n, a.counts, a.partial, a.offsets, per);
  return 0;
}

__device__ __forceinline__ void copy_row(const float *src, float *dst, int64_t i, int64_t o, int w) {
  if (!src || !dst) return;
  for (int k = 0; k < w; ++k) dst[o * w + k] = src[i * w + k];
}
__device__ __forceinline__ void zero_row(float *dst, int64_t o, int w) {
  if (!dst) return;
  for (int k = 0; k < w; ++k) dst[o * w + k] = 0.0f;
}

// One thread per input primitive writes its 0, 1 or 2 output rows.
__global__ void __launch_bounds__(256) densify_apply_kernel(DensifyApplyArgs a) {
  const int nb3 = a.sh_floats;
  const int widths[5] = {3, 3, 4, 1, nb3};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < a.n; i += (int64_t)gridDim.x * blockDim.x) {
    const int act = a.actions[i];
    if (act == 0) continue;
    const int64_t o = a.offsets[i];
    const float *src[5] = {a.in.means, a.in.log_scales, a.in.quats, a.in.logits, a.in.sh};
    float *dst[5] = {a.out.means, a.out.log_scales, a.out.quats, a.out.logits, a.out.sh};
    if (act == 1 || act == 2) {
      for (int c = 0; c < (act == 2 ? 2 : 1); ++c) {
        for (int k = 0; k < 5; ++k) copy_row(src[k], dst[k], i, o + c, widths[k]);
        a.out.types[o + c] = a.in.types[i];
        for (int k = 0; k < 10; ++k) {
          if (c == 0) copy_row(a.in.moments[k], a.out.moments[k], i, o, widths[k % 5]);
          else zero_row(a.out.moments[k], o + c, widths[k % 5]);
        }
      }
      continue;
    }
    // split: two samples mu + R (s * z), scales / 1.6 (in-plane only for a surfel)
    const bool is3d = a.in.types[i] != 0;
    float q[4] = {a.in.quats[4 * i], a.in.quats[4 * i + 1], a.in.quats[4 * i + 2], a.in.quats[4 * i + 3]};
    const float qn = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
    const float w = q[0] * qn, x = q[1] * qn, y = q[2] * qn, z = q[3] * qn;
    const float R[9] = {1.f - 2.f * (y * y + z * z), 2.f * (x * y - w * z), 2.f * (x * z + w * y),
                        2.f * (x * y + w * z), 1.f - 2.f * (x * x + z * z), 2.f * (y * z - w * x),
                        2.f * (x * z - w * y), 2.f * (y * z + w * x), 1.f - 2.f * (x * x + y * y)};
    const float s[3] = {expf(a.in.log_scales[3 * i]), expf(a.in.log_scales[3 * i + 1]),
                        is3d ? expf(a.in.log_scales[3 * i + 2]) : 0.0f};
    const float shrink = logf(1.6f);
    for (int c = 0; c < 2; ++c) {
      const int64_t oc = o + c;
      const float *zz = a.normals_z + (6 * i + 3 * c);
      const float d[3] = {s[0] * zz[0], s[1] * zz[1], s[2] * zz[2]};
#pragma unroll
      for (int r = 0; r < 3; ++r)
        a.out.means[3 * oc + r] = a.in.means[3 * i + r] + (R[3 * r] * d[0] + R[3 * r + 1] * d[1] + R[3 * r + 2] * d[2]);
      a.out.log_scales[3 * oc] = a.in.log_scales[3 * i] - shrink;
      a.out.log_scales[3 * oc + 1] = a.in.log_scales[3 * i + 1] - shrink;
      a.out.log_scales[3 * oc + 2] = a.in.log_scales[3 * i + 2] - (is3d ? shrink : 0.0f);
      for (int k = 2; k < 5; ++k) copy_row(src[k], dst[k], i, oc, widths[k]);
      a.out.types[oc] = a.in.types[i];
      for (int k = 0; k < 10; ++k) zero_row(a.out.moments[k], oc, widths[k % 5]);
    }
  }
}

int launch_densify_apply(const DensifyApplyArgs &a, cudaStream_t s) {
  if (a.n <= 0) return 0;
  const int grid = (int)std::min<int64_t>((a.n + 255) / 256, 152 * 16);
  densify_apply_kernel<<<grid, 256, 0, s>>>(a);
  return 0;
}

// ---------------------------------------------------------------------------
// opacity reset: logit <- min(logit, cap); its Adam moments are zeroed
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) reset_opacity_kernel(int64_t n, float *logits, float cap, float *m, float *v) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    logits[i] = fminf(logits[i], cap);
    if (m) m[i] = 0.0f;
    if (v) v[i] = 0.0f;
  }
}

int launch_reset_opacity(int64_t n, float *logits, float cap, float *m, float *v, cudaStream_t s) {
  if (n <= 0) return 0;
  const int grid = (int)std::min<int64_t>((n + 255) / 256, 152 * 16);
  reset_opacity_kernel<<<grid, 256, 0, s>>>(n, logits, cap, m, v);
  return 0;
}

}  // namespace hgs
