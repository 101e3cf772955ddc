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

// Pixel boxes and tile sets of the contract.
__device__ __forceinline__ float pad_extent(float r) {
  return cadd(cmul(r, 1.0009765625f), 0.015625f);
}

// pixel-centre coverage of [lo, hi] along an axis of `extent` pixels ->
// inclusive tile range; false if no pixel centre is covered
__device__ __forceinline__ bool pixel_tiles(float lo, float hi, int extent, int *t0, int *t1) {
  float flo = csub(lo, 0.5f), fhi = csub(hi, 0.5f);
  if (!(flo <= fhi)) return false;
  flo = fmaxf(flo, -1.0f);
  fhi = fminf(fhi, (float)extent);
  int p0 = (int)ceilf(flo), p1 = (int)floorf(fhi);
  if (p0 < 0) p0 = 0;
  if (p1 > extent - 1) p1 = extent - 1;
  if (p0 > p1) return false;
  *t0 = p0 / kTile;
  *t1 = p1 / kTile;
  return true;
}

// Tile-set parameters of a binned primitive (three float4, written by the
// preprocess).  Ellipse mode: t0 = (centre x, centre y, chord slope k, padded
// half chord w), t1 = (1 / padded half height h, y of the leftmost point, y
// of the rightmost point, 0); the footprint's chord at height y is centred on
// x + k (y - centre y) with half length w sqrt(1 - ((y - centre y) / h)^2).
// Disc mode (a surfel reaching the near plane): the disc in
// pixel-homogeneous camera coordinates P = (fx X + cx Z, fy Y + cy Z, Z),
// t0 = (centre, dmax), t1 = (axis a, near), t2.xyz = axis b.  t2.w = flags
// (int bits): bits 0-1 the mode (0 ellipse, 1 the whole rectangle, 2 disc),
// bits 2-16 the tile-row offset of the primitive's image in a stacked grid,
// bits 17-31 the image width in pixels.
struct TileSet {
  float4 t0, t1, t2;
};
enum { kSetEllipse = 0, kSetRect = 1, kSetDisc = 2 };
__device__ __forceinline__ uint32_t tileset_flags(int mode, int row_off, int width) {
  return (uint32_t)mode | ((uint32_t)row_off << 2) | ((uint32_t)width << 17);
}

// The x-range of the pixels of (image-local) tile row lty whose rays hit a
// disc-mode surfel's disc in front of the near plane.  A pixel (x, y) sees
// P(u, v) = C + u a + v b (u^2 + v^2 <= dmax) at x = P0/P2, y = P1/P2, depth
// P2; over the row's band of pixel-centre heights [ya, yb] the points seen
// form the disc cut by three half-planes c + p u + q v >= 0 (P1 - ya P2,
// yb P2 - P1, P2 - near).  x is a ratio of affine functions, so its extremes
// over that convex set lie at points of the circle that a plane x P2 = P0
// touches, at the lines' crossings with the circle, or at the lines'
// crossings with each other; every candidate inside the set (relative
// tolerances 2^-12 on each half-plane, 2^-10 on the radius) is taken, and
// the range padded by 2^-9 |x| + 1/16 px.  false: no candidate.
static __device__ __noinline__ bool disc_span(const TileSet &s, int lty, float *xlo, float *xhi) {
  const float ya = cadd((float)(lty * kTile), 0.5f), yb = cadd(ya, (float)(kTile - 1));
  const float CX = s.t0.x, CY = s.t0.y, CZ = s.t0.z, r2 = s.t0.w;
  const float ax = s.t1.x, ay = s.t1.y, az = s.t1.z, nz = s.t1.w;
  const float bx = s.t2.x, by = s.t2.y, bz = s.t2.z;
  float c[3], p[3], q[3], tol[3];
  c[0] = csub(CY, cmul(ya, CZ)); p[0] = csub(ay, cmul(ya, az)); q[0] = csub(by, cmul(ya, bz));
  c[1] = csub(cmul(yb, CZ), CY); p[1] = csub(cmul(yb, az), ay); q[1] = csub(cmul(yb, bz), by);
  c[2] = csub(CZ, nz); p[2] = az; q[2] = bz;
  const float rho = csqrt(r2);
#pragma unroll
  for (int k = 0; k < 3; ++k)
    tol[k] = cmul(0x1p-12f, cadd(fabsf(c[k]), cmul(rho, cadd(fabsf(p[k]), fabsf(q[k])))));
  const float r2t = cmul(r2, 1.0009765625f);
  float lo = __int_as_float(0x7f800000), hi = -__int_as_float(0x7f800000);
  auto take = [&](float u, float v, bool on_circle) {
    if (!on_circle && !(cadd(cmul(u, u), cmul(v, v)) <= r2t)) return;
#pragma unroll
    for (int m = 0; m < 3; ++m)
      if (!(cadd(cadd(c[m], cmul(p[m], u)), cmul(q[m], v)) >= -tol[m])) return;
    const float D = cadd(cadd(CZ, cmul(az, u)), cmul(bz, v));
    if (!(D > 0.0f)) return;
    const float x = cdiv(cadd(cadd(CX, cmul(ax, u)), cmul(bx, v)), D);
    lo = fminf(lo, x);
    hi = fmaxf(hi, x);
  };
  // (a) tangency: (CX - x CZ)^2 = r2 ((ax - x az)^2 + (bx - x bz)^2)
  const float A = csub(cmul(CZ, CZ), cmul(r2, cadd(cmul(az, az), cmul(bz, bz))));
  const float B = csub(cmul(CX, CZ), cmul(r2, cadd(cmul(ax, az), cmul(bx, bz))));
  const float Cq = csub(cmul(CX, CX), cmul(r2, cadd(cmul(ax, ax), cmul(bx, bx))));
  const float dq = csub(cmul(B, B), cmul(A, Cq));
  if (dq >= 0.0f && A != 0.0f) {
    const float sq = csqrt(dq);
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const float xs = cdiv(k == 0 ? csub(B, sq) : cadd(B, sq), A);
      const float al = csub(CX, cmul(xs, CZ)), be0 = csub(ax, cmul(xs, az)), be1 = csub(bx, cmul(xs, bz));
      const float bb = cadd(cmul(be0, be0), cmul(be1, be1));
      if (!(bb > 0.0f)) continue;
      const float t = cdiv(-al, bb);
      take(cmul(t, be0), cmul(t, be1), true);
    }
  }
  // (b) each line's crossings with the circle
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const float pq = cadd(cmul(p[k], p[k]), cmul(q[k], q[k]));
    if (!(pq > 0.0f)) continue;
    const float t = cdiv(-c[k], pq);
    const float fu = cmul(t, p[k]), fv = cmul(t, q[k]);
    const float d2 = cdiv(cmul(c[k], c[k]), pq);
    if (!(d2 <= r2t)) continue;
    const float h = csqrt(cdiv(fmaxf(csub(r2, d2), 0.0f), pq));
    take(csub(fu, cmul(h, q[k])), cadd(fv, cmul(h, p[k])), true);
    take(cadd(fu, cmul(h, q[k])), csub(fv, cmul(h, p[k])), true);
  }
  // (c) the lines' crossings with each other
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i + 1; j < 3; ++j) {
      const float det = csub(cmul(p[i], q[j]), cmul(p[j], q[i]));
      if (det == 0.0f) continue;
      take(cdiv(csub(cmul(q[i], c[j]), cmul(q[j], c[i])), det), cdiv(csub(cmul(p[j], c[i]), cmul(p[i], c[j])), det),
           false);
    }
  if (!(lo <= hi)) return false;
  const float pad = cadd(cmul(0x1p-9f, fmaxf(fabsf(lo), fabsf(hi))), 0.0625f);
  *xlo = csub(lo, pad);
  *xhi = cadd(hi, pad);
  return true;
}

// Tile columns [c0, c1] of (stacked) tile row ty of a primitive's tile set,
// within its rectangle columns [tx0, tx1].  Ellipse mode: the pixel columns
// whose centres the padded ellipse reaches in the row's band of pixel-centre
// heights [16 ty + 0.5, 16 ty + 15.5]; over the band the chord's left end is
// least at the height nearest the leftmost point (the left end is convex in
// y) and the right end greatest nearest the rightmost point.  false: no tile.
__device__ __forceinline__ bool row_span(const TileSet &s, int ty, int tx0, int tx1, int *c0, int *c1) {
  const uint32_t fl = __float_as_uint(s.t2.w);
  const uint32_t mode = fl & 3u;
  if (mode == kSetRect) {
    *c0 = tx0;
    *c1 = tx1;
    return true;
  }
  const int lty = ty - (int)((fl >> 2) & 0x7fffu);
  const int width = (int)(fl >> 17);
  float xl, xr;
  if (mode == kSetDisc) {
    if (!disc_span(s, lty, &xl, &xr)) return false;
  } else {
    const float ya = cadd((float)(lty * kTile), 0.5f), yb = cadd(ya, (float)(kTile - 1));
    const float y1 = fminf(fmaxf(s.t1.y, ya), yb), y2 = fminf(fmaxf(s.t1.z, ya), yb);
    const float d1 = csub(y1, s.t0.y), d2 = csub(y2, s.t0.y);
    const float q1 = cmul(d1, s.t1.x), q2 = cmul(d2, s.t1.x);
    const float r1 = fmaxf(csub(1.0f, cmul(q1, q1)), 0.0f), r2 = fmaxf(csub(1.0f, cmul(q2, q2)), 0.0f);
    xl = csub(cadd(s.t0.x, cmul(s.t0.z, d1)), cmul(s.t0.w, csqrt(r1)));
    xr = cadd(cadd(s.t0.x, cmul(s.t0.z, d2)), cmul(s.t0.w, csqrt(r2)));
  }
  int a, b;
  if (!pixel_tiles(xl, xr, width, &a, &b)) return false;
  a = max(a, tx0);
  b = min(b, tx1);
  if (a > b) return false;
  *c0 = a;
  *c1 = b;
  return true;
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

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// pdl_launch may become resident while its predecessor in the stream is
// still finishing; grid_dep() at the top of such a kernel waits until the
// predecessor has completed and its writes are visible, before any global
// memory access, and then lets the successor's blocks be scheduled in turn
// (they wait the same way).  Launched normally, both instructions return at
// once.
__device__ __forceinline__ void grid_dep() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
static inline void pdl_launch(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...);
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
