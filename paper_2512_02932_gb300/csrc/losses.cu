// losses.cu -- the image losses of frequency-decoupled optimisation (EGGS
// §3.3, Eq. 8; App. E): the mean absolute error of the rendered image, and
// the squared errors of its level-1 Haar DWT bands, with the gradient image
// of each.
//
// Haar pair l = (1, 1)/sqrt2, h = (1, -1)/sqrt2.  On the 2x2 block
// (a b; c d) at rows 2i, 2i+1 and columns 2j, 2j+1 the four bands of
// App. E (I_LL = L I L^T, I_LH = H I L^T, I_HL = L I H^T, I_HH = H I H^T)
// are
//   LL = (a + b + c + d)/2    LH = (a + b - c - d)/2
//   HL = (a - b + c - d)/2    HH = (a - b - c + d)/2.
// The transform is linear, so the bands of (image - target) are the band
// differences.  L_low is the mean of dLL^2 over the C (H/2)(W/2) band
// elements, L_high the mean of dLH^2 + dHL^2 + dHH^2 over 3 C (H/2)(W/2); an
// odd last row or column lies outside every block and enters L1 only.  L1
// is the mean |image - target| over all C H W pixels (sign(0) = 0).
//
// A block takes whole block-rows (a channel's row pair), its threads the 2x2
// blocks along it, reading each block's two row pairs as float2 when the
// width is even.  Sums go from registers through a warp and block reduction
// to one double atomic per block and loss.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

__device__ __forceinline__ float sgnf(float x) { return x > 0.0f ? 1.0f : (x < 0.0f ? -1.0f : 0.0f); }

__device__ __forceinline__ void block_add3(float s1, float sl, float sh, double *out, double k1, double kl,
                                           double kh) {
  __shared__ float red[3][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    sl += __shfl_xor_sync(0xffffffffu, sl, o);
    sh += __shfl_xor_sync(0xffffffffu, sh, o);
  }
  if (lane == 0) { red[0][warp] = s1; red[1][warp] = sl; red[2][warp] = sh; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t1 = 0.0, tl = 0.0, th = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { t1 += red[0][w]; tl += red[1][w]; th += red[2][w]; }
    if (t1 != 0.0) atomicAdd(out + 0, t1 * k1);
    if (tl != 0.0) atomicAdd(out + 1, tl * kl);
    if (th != 0.0) atomicAdd(out + 2, th * kh);
  }
}

// The 2x2 block (bx) of block-row r (channel c, rows 2i, 2i+1): losses and
// gradient images.
__device__ __forceinline__ void haar_block(const LossArgs &a, size_t p0, bool vec, float g1, float gl, float gh,
                                           float &s1, float &sl, float &sh) {
  const size_t p1 = p0 + (size_t)a.W;
  float d00, d01, d10, d11;
  if (vec) {
    const float2 x0 = __ldg(reinterpret_cast<const float2 *>(a.img + p0));
    const float2 x1 = __ldg(reinterpret_cast<const float2 *>(a.img + p1));
    const float2 y0 = __ldg(reinterpret_cast<const float2 *>(a.tgt + p0));
    const float2 y1 = __ldg(reinterpret_cast<const float2 *>(a.tgt + p1));
    d00 = x0.x - y0.x; d01 = x0.y - y0.y; d10 = x1.x - y1.x; d11 = x1.y - y1.y;
  } else {
    d00 = a.img[p0] - a.tgt[p0]; d01 = a.img[p0 + 1] - a.tgt[p0 + 1];
    d10 = a.img[p1] - a.tgt[p1]; d11 = a.img[p1 + 1] - a.tgt[p1 + 1];
  }
  const float LL = 0.5f * (d00 + d01 + d10 + d11), LH = 0.5f * (d00 + d01 - d10 - d11);
  const float HL = 0.5f * (d00 - d01 + d10 - d11), HH = 0.5f * (d00 - d01 - d10 + d11);
  s1 += fabsf(d00) + fabsf(d01) + fabsf(d10) + fabsf(d11);
  sl += LL * LL;
  sh += LH * LH + HL * HL + HH * HH;
  // d/dx of mean(band^2): 2 band / n times the pixel's coefficient (+-1/2)
  if (a.g_l1) {
    const float2 u0 = make_float2(g1 * sgnf(d00), g1 * sgnf(d01)), u1 = make_float2(g1 * sgnf(d10), g1 * sgnf(d11));
    if (vec) { *reinterpret_cast<float2 *>(a.g_l1 + p0) = u0; *reinterpret_cast<float2 *>(a.g_l1 + p1) = u1; }
    else { a.g_l1[p0] = u0.x; a.g_l1[p0 + 1] = u0.y; a.g_l1[p1] = u1.x; a.g_l1[p1 + 1] = u1.y; }
  }
  if (a.g_low) {
    const float v = gl * LL;
    if (vec) {
      *reinterpret_cast<float2 *>(a.g_low + p0) = make_float2(v, v);
      *reinterpret_cast<float2 *>(a.g_low + p1) = make_float2(v, v);
    } else {
      a.g_low[p0] = v; a.g_low[p0 + 1] = v; a.g_low[p1] = v; a.g_low[p1 + 1] = v;
    }
  }
  if (a.g_high) {
    const float2 u0 = make_float2(gh * (LH + HL + HH), gh * (LH - HL - HH));
    const float2 u1 = make_float2(gh * (-LH + HL - HH), gh * (-LH - HL + HH));
    if (vec) { *reinterpret_cast<float2 *>(a.g_high + p0) = u0; *reinterpret_cast<float2 *>(a.g_high + p1) = u1; }
    else { a.g_high[p0] = u0.x; a.g_high[p0 + 1] = u0.y; a.g_high[p1] = u1.x; a.g_high[p1 + 1] = u1.y; }
  }
}

// Blocks stride over block-rows (channel, row pair); threads over the 2x2
// blocks of a row, so no index needs a division.
__global__ void __launch_bounds__(256) image_losses_kernel(LossArgs a) {
  const int H2 = a.H / 2, W2 = a.W / 2;
  const int rows = a.C * H2;
  const int64_t nblk = (int64_t)rows * W2;
  const double n_all = (double)a.C * a.H * a.W;
  const double n_low = (double)nblk, n_high = 3.0 * (double)nblk;
  const float g1 = (float)(a.w_l1 / n_all);
  const float gl = nblk ? (float)(a.w_low / n_low) : 0.0f;
  const float gh = nblk ? (float)(a.w_high / n_high) : 0.0f;
  const bool vec = (a.W % 2 == 0) &&
                   ((reinterpret_cast<uintptr_t>(a.img) | reinterpret_cast<uintptr_t>(a.tgt) |
                     reinterpret_cast<uintptr_t>(a.g_l1) | reinterpret_cast<uintptr_t>(a.g_low) |
                     reinterpret_cast<uintptr_t>(a.g_high)) & 7u) == 0;
  float s1 = 0.f, sl = 0.f, sh = 0.f;
  for (int r = blockIdx.x; r < rows; r += gridDim.x) {
    const int c = r / H2, i = r - c * H2;
    const size_t row0 = ((size_t)c * a.H + 2 * (size_t)i) * a.W;
    for (int j = threadIdx.x; j < W2; j += blockDim.x) haar_block(a, row0 + 2 * (size_t)j, vec, g1, gl, gh, s1, sl, sh);
  }
  // an odd last column (rows 0 .. 2 H2 - 1) and an odd last row (all columns)
  const int col_n = (a.W & 1) ? 2 * H2 : 0, row_n = (a.H & 1) ? a.W : 0;
  const int64_t tail = (int64_t)a.C * (col_n + row_n);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < tail; t += stride) {
    const int64_t c = t / (col_n + row_n), k = t - c * (col_n + row_n);
    const int64_t y = k < col_n ? k : a.H - 1, x = k < col_n ? a.W - 1 : k - col_n;
    const size_t p = (size_t)((c * a.H + y) * a.W + x);
    const float d = a.img[p] - a.tgt[p];
    s1 += fabsf(d);
    if (a.g_l1) a.g_l1[p] = g1 * sgnf(d);
    if (a.g_low) a.g_low[p] = 0.0f;
    if (a.g_high) a.g_high[p] = 0.0f;
  }
  block_add3(s1, sl, sh, a.loss, 1.0 / n_all, nblk ? 1.0 / n_low : 0.0, nblk ? 1.0 / n_high : 0.0);
}

int launch_image_losses(const LossArgs &a, cudaStream_t s) {
  // one block per block-row up to a few resident waves (each block ends in
  // three double atomics on the same three words, so not too many blocks)
  const int64_t rows = (int64_t)a.C * (a.H / 2);
  int sms = 152, dev = 0;
  if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(rows, (int64_t)sms * 4));
  image_losses_kernel<<<grid, 256, 0, s>>>(a);
  return 0;
}

}  // namespace hgs
