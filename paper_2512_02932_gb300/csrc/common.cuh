// common.cuh -- device-side definitions shared by the kernels of the hybrid
// 2D/3D Gaussian rasterizer (EGGS, Sec. 3.1-3.2, App. C-D) for sm_103a.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/hgs.h"

namespace hgs {

constexpr int kTile = 16;           // tile edge (pixels)
constexpr int kTilePix = kTile * kTile;
constexpr float kLog2e = 1.4426950408889634f;

// ---------------------------------------------------------------------------
// Render record: 5 x float4 (80 B) per primitive, written by preprocess and
// staged through shared memory by the render kernels.
//   r0 = (x_c, y_c, z_c, alpha_s)   projected centre (pixels), camera depth,
//        alpha_s = +alpha for a 3D Gaussian, -alpha for a 2D surfel
//   r1 = 3D: (W00, W01, W11, 0)  Cholesky factor of the conic (Eq. 1):
//        d = (W00 dx + W01 dy)^2 + (W11 dy)^2
//        2D: (Q00, Q01, Q10, Q11)
//   r2 = 3D: (0, 0, r, g)   2D: (Q20, Q21, r, g)
//   r3 = (b, nx, ny, nz)    colour blue, camera-space normal
//   r4 = (x_lo, y_lo, box_x, box_y)  low parts of the projected centre (the
//        centre is the double-float x_c + x_lo: binary32 alone cannot place
//        it to the 1e-4 px a sub-pixel splat needs) and the padded pixel box
//        outside which the pair never contributes, as two half2 (x0, x1) and
//        (y0, y1) rounded outwards; a warp skips a record whose box misses
//        its pixel block
// For a surfel, with (dx, dy) the pixel offset from the projected centre:
//   p = (Q00 dx + Q01 dy, Q10 dx + Q11 dy, Q20 dx + Q21 dy + 1),
//   (u, v) = (p0, p1) / p2, hit depth z = z_c / p2     (Eq. 14 re-centred)
// ---------------------------------------------------------------------------
struct Rec {
  float4 r0, r1, r2, r3, r4;
};
constexpr int kRecF4 = 5;

// Per-primitive gradient of the render record, accumulated by render_bwd
// (16 floats):
//   [0] d alpha  [1..3] d rgb  [4] d x_c  [5] d y_c  [6] d z_c
//   3D: [7] d h00  [8] d h01  [9] d h11: the footprint shape in its own
//       coordinates (u, v) = W (dx, dy), d = h00 u^2 + 2 h01 u v + h11 v^2
//       at H = I.  dL/d(conic) = W^T dL/dH W, but a needle's conic is
//       ill-conditioned and this form keeps the sums and the chain rule
//       free of cancellation.
//   2D: the homography's gradient in the splat's own coordinates (u, v):
//       [7..10] sum (du, dv) (u, v)^T row-major, [11..12] sum p2 dL/dp2 (u, v)
//   [13..15] d normal
constexpr int kGradW = 16;

// ---------------------------------------------------------------------------
// Binning-contract arithmetic: every operation is a correctly rounded binary32
// operation that the compiler may not fuse or reorder.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float cmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float cadd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float csub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float cdiv(float a, float b) { return __fdiv_rn(a, b); }
__device__ __forceinline__ float csqrt(float a) { return __fsqrt_rn(a); }

// Contract exp: x = k ln2 + r (Cody-Waite split of ln2), e^r by its degree-7
// Taylor polynomial in Horner form, times 2^k.
__device__ __forceinline__ float contract_exp(float x) {
  if (x != x) return x;
  if (x < -87.0f) return 0.0f;
  if (x > 88.0f) x = 88.0f;
  const float k = rintf(cmul(x, 0x1.715476p+0f));
  float r = csub(x, cmul(k, 0x1.62e4p-1f));
  r = csub(r, cmul(k, 0x1.7f7d1cp-20f));
  float p = 0x1.a01a02p-13f;           // 1/7!
  p = cadd(cmul(p, r), 0x1.6c16c2p-10f); // 1/6!
  p = cadd(cmul(p, r), 0x1.111112p-7f);  // 1/5!
  p = cadd(cmul(p, r), 0x1.555556p-5f);  // 1/4!
  p = cadd(cmul(p, r), 0x1.555556p-3f);  // 1/3!
  p = cadd(cmul(p, r), 0.5f);
  p = cadd(cmul(p, r), 1.0f);
  p = cadd(cmul(p, r), 1.0f);
  const int ki = (int)k;
  return cmul(p, __int_as_float((ki + 127) << 23));
}

// Contract log for normal x > 0: x = m 2^e, m in (sqrt(1/2), sqrt(2)],
// ln m = 2 atanh((m-1)/(m+1)) by the odd power series to t^13.
__device__ __forceinline__ float contract_log(float x) {
  if (!(x > 0.0f)) return -__int_as_float(0x7f800000);
  const uint32_t b = __float_as_uint(x);
  int e = (int)((b >> 23) & 0xffu) - 127;
  float m = __uint_as_float((b & 0x7fffffu) | 0x3f800000u);
  if (m > 0x1.6a09e6p+0f) {
    m = cmul(m, 0.5f);
    e = e + 1;
  }
  const float t = cdiv(csub(m, 1.0f), cadd(m, 1.0f));
  const float t2 = cmul(t, t);
  float s = 0x1.3b13b2p-4f;              // 1/13
  s = cadd(cmul(s, t2), 0x1.745d18p-4f); // 1/11
  s = cadd(cmul(s, t2), 0x1.c71c72p-4f); // 1/9
  s = cadd(cmul(s, t2), 0x1.24924ap-3f); // 1/7
  s = cadd(cmul(s, t2), 0x1.99999ap-3f); // 1/5
  s = cadd(cmul(s, t2), 0x1.555556p-2f); // 1/3
  s = cadd(cmul(s, t2), 1.0f);
  const float lnm = cmul(cmul(2.0f, t), s);
  const float fe = (float)e;
  return cadd(cmul(fe, 0x1.62e4p-1f), cadd(cmul(fe, 0x1.7f7d1cp-20f), lnm));
}

// ---------------------------------------------------------------------------
// fast hardware approximations for the per-pair loops
// ---------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// error-free transforms for the double-float projected centre
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float &p, float &e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}

__device__ __forceinline__ void set_error(int32_t *dev_err, int32_t code) {
  if (dev_err) atomicCAS(dev_err, 0, code);
}

// Kernel-argument views of the ABI structs.
struct CamK {
  float R[9], t[3];
  float fx, fy, cx, cy;
  float campos[3];  // camera centre in world space, -R^T t
  int W, H, TX, TY;
};

struct CfgK {
  float near_z, alpha_min, alpha_max, T_min, lambda_z, theta_z, T_z, dilation;
  float bg[3];
};

}  // namespace hgs
