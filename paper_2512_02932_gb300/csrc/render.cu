// render.cu -- per-tile blending of the hybrid rasterizer (EGGS Sec. 3.1,
// Eq. 1, Eq. 2) and its backward.
//
// Every tile (16x16 pixels) is split into four 8x8 quadrants; a lane owns two
// pixels of a quadrant, (x, y) and (x, y + 4), which share their column, so
// the per-pair evaluation after the x offset runs on both at once with the
// packed two-lane binary32 instructions (eval_pair2).
//
// Forward: a warp owns one quadrant and walks its tile's sorted list on its
// own, staging 32 records at a time into a private cp.async double buffer,
// skipping records that cannot reach its quadrant (block_may_hit), and
// leaving once every one of its pixels has terminated (T below T_min).  With
// a scheduling scratch the grid is persistent: warps take (tile, quadrant)
// items, tiles with the longest lists first.
//
// Backward (rgb cotangents, the image-loss case, one set or the three sets of
// frequency-decoupled optimisation): one warp per tile walks the list once
// from the latest contributor of any of its pixels back to the start,
// evaluates each record against the quadrants it can reach, and sums a
// record's gradient over all 256 pixels before one warp reduction and one
// set of atomics per (record, tile).  Tiles are handed out longest walk
// first.  The general backward (depth, normal or alpha cotangents) keeps one
// warp per quadrant.
//
// The per-pair evaluation is written with explicitly rounded operations, and
// the scalar and packed forms run the same operations in the same order, so
// every backward reproduces the forward's contribution decisions bit for bit.
#include <cuda_fp16.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

constexpr int kRW = 4;   // warps per CTA (one 16x16 tile, 8x8 pixels per warp)
constexpr int kCh = 32;  // records per staged chunk

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

struct PairEval {
  float dx, dy, z, q, g, araw, at, alpha, u, v, inv;
};

// Unified distance (Eq. 1) and contribution (Sec. 3.1) of one record at the
// pixel centre (px, py).  Returns true iff the pair contributes.
__device__ __forceinline__ bool eval_pair(const float4 &r0, const float4 &r1, const float4 &r2,
                                          const float4 &r4, float px, float py, const CfgK &f,
                                          PairEval &e) {
  // offset from the double-float projected centre (x_c + x_lo, y_c + y_lo)
  e.dx = __fsub_rn(__fsub_rn(px, r0.x), r4.x);
  e.dy = __fsub_rn(__fsub_rn(py, r0.y), r4.y);
  float q;
  if (r0.w > 0.0f) {
    // 3D: d = (x-mu')^T Sigma'^-1 (x-mu') of Eq. 1, evaluated as |W d|^2 with
    // W the Cholesky factor of the conic (u = W00 dx + W01 dy, v = W11 dy)
    e.u = __fmaf_rn(r1.x, e.dx, __fmul_rn(r1.y, e.dy));
    e.v = __fmul_rn(r1.z, e.dy);
    q = __fmaf_rn(e.u, e.u, __fmul_rn(e.v, e.v));
    e.alpha = r0.w;
    e.z = r0.z;
  } else {
    // 2D: ray-splat intersection (Eq. 14), re-centred on the projected centre
    const float p0 = __fmaf_rn(r1.x, e.dx, __fmul_rn(r1.y, e.dy));
    const float p1 = __fmaf_rn(r1.z, e.dx, __fmul_rn(r1.w, e.dy));
    const float p2 = __fmaf_rn(r2.x, e.dx, __fmaf_rn(r2.y, e.dy, 1.0f));
    if (!(p2 > 0.0f)) return false;
    e.inv = rcp_approx(p2);
    e.z = __fmul_rn(r0.z, e.inv);
    if (!(e.z > f.near_z)) return false;
    e.u = __fmul_rn(p0, e.inv);
    e.v = __fmul_rn(p1, e.inv);
    q = __fmaf_rn(e.u, e.u, __fmul_rn(e.v, e.v));
    e.alpha = -r0.w;
  }
  e.q = q;
  e.g = ex2_approx(__fmul_rn(q, -0.5f * kLog2e));
  e.araw = __fmul_rn(e.alpha, e.g);
  if (!(e.araw >= f.alpha_min)) return false;
  e.at = fminf(e.araw, f.alpha_max);
  return true;
}

// warp block origin (pixel coordinates of its top-left pixel) and the two
// pixels of this lane: (x, y) and (x, y + 4)
__device__ __forceinline__ void block_of(int local, int TX, int warp, int &bx, int &by) {
  bx = (local % TX) * kTile + (warp & 1) * 8;
  by = (local / TX) * kTile + (warp >> 1) * 8;
}

// ---------------------------------------------------------------------------
// staging helpers
// ---------------------------------------------------------------------------
// Copy the records of list entries [base, base + cnt) into this warp's buffer
// (lane l copies entry base + l) and, for the backward, their ids.
__device__ __forceinline__ void stage_chunk(const float4 *__restrict__ rec, const uint32_t *__restrict__ vals,
                                            uint32_t base, uint32_t end, float4 *buf, uint32_t *ids, int lane) {
  const uint32_t idx = base + lane;
  if (idx < end) {
    const uint32_t id = __ldg(vals + idx);
    if (ids) ids[lane] = id;
    const float4 *src = rec + kRecF4 * (size_t)id;
    float4 *dst = buf + lane * kRecF4;
#pragma unroll
    for (int k = 0; k < kRecF4; ++k) cp_async16(dst + k, src + k);
  }
  cp_async_commit();
}

__device__ __forceinline__ float2 unpack_box(float v) {
  const uint32_t u = __float_as_uint(v);
  return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}

// Squared distance from the origin to the segment P -> P + E (FP32; used
// only with a margin, see block_may_hit).
__device__ __forceinline__ float seg_dist2(float px, float py, float ex, float ey) {
  const float l2 = fmaf(ex, ex, ey * ey);
  const float t = fminf(fmaxf(-fmaf(px, ex, py * ey) * rcp_approx(l2), 0.0f), 1.0f);
  const float qx = fmaf(t, ex, px), qy = fmaf(t, ey, py);
  return fmaf(qx, qx, qy * qy);
}

// Can the record contribute to any pixel centre of the 8x8 block whose first
// centre is (bx + 0.5, by + 0.5)?  A pair contributes only if its distance d
// (Eq. 1) satisfies alpha * exp(-d/2) >= alpha_min, i.e. d <= 2 ln(alpha /
// alpha_min).  The test bounds d from below over the whole rectangle of the
// block's centres and keeps the record unless that bound exceeds the limit
// by a margin far above the FP32 error of either side, so it never drops a
// pair that eval_pair would accept and the rendered result is unchanged.
//  * 3D: d = u^2 + v^2 with u = W00 X + W01 Y, v = W11 Y (X, Y offsets from
//    the centre).  For fixed Y the minimum of u^2 over X in [x0, x1] is
//    max(a, -b, 0)^2 with a = W01 Y + W00 x0, b = W01 Y + W00 x1; the
//    resulting function of Y is convex, so its minimum over [y0, y1] is at
//    the clamp of whichever of its three piecewise minimisers (Y = 0 and the
//    two affine pieces' vertices) is global, and the least of the three
//    clamped values is exact.
//  * 2D: (u, v) = (p0, p1) / p2 with p = Q (X, Y, 1) (Eq. 14).  Where p2 > 0
//    over the rectangle the map is projective, so the rectangle goes to the
//    convex quadrilateral of its corners' images and the pixels' (u, v) lie
//    inside it; the block can be hit only if that quadrilateral meets the
//    disc u^2 + v^2 <= limit.  Corners behind the camera, or mapped too far
//    for FP32 to place the edges precisely, keep the record.
__device__ __forceinline__ bool block_may_hit(const float4 &r0, const float4 &r1, const float4 &r2,
                                              const float4 &r4, float bx, float by, const CfgK &f) {
  const float x0 = ((bx + 0.5f) - r0.x) - r4.x, y0 = ((by + 0.5f) - r0.y) - r4.y;
  const float x1 = x0 + 7.0f, y1 = y0 + 7.0f;
  const float ratio = __fdividef(fabsf(r0.w), f.alpha_min);
  if (!(ratio > 1.0f)) return false;  // alpha below alpha_min: never contributes
  const float lim = fmaf(2.0f * __logf(ratio), 1.001f, 0.05f);
  if (r0.w > 0.0f) {
    const float W00 = r1.x, W01 = r1.y, W11 = r1.z;
    const float C = fmaf(W01, W01, W11 * W11);
    const float k = -W01 * W00 * rcp_approx(C);
    const float c0 = fminf(fmaxf(0.0f, y0), y1);
    const float ca = fminf(fmaxf(k * x0, y0), y1);
    const float cb = fminf(fmaxf(k * x1, y0), y1);
    float dmin = 3.0e38f;
    const float ys[3] = {c0, ca, cb};
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const float Y = ys[i];
      const float a = fmaf(W01, Y, W00 * x0), b = fmaf(W01, Y, W00 * x1);
      const float m = fmaxf(fmaxf(a, -b), 0.0f);
      const float v = W11 * Y;
      dmin = fminf(dmin, fmaf(m, m, v * v));
    }
    return !(dmin > lim);
  }
  float u[4], v[4];
  const float xs[4] = {x0, x1, x1, x0}, yy[4] = {y0, y0, y1, y1};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float p0 = fmaf(r1.x, xs[i], r1.y * yy[i]);
    const float p1 = fmaf(r1.z, xs[i], r1.w * yy[i]);
    const float p2 = fmaf(r2.x, xs[i], fmaf(r2.y, yy[i], 1.0f));
    if (!(p2 > 0.0f)) return true;
    const float inv = rcp_approx(p2);
    u[i] = p0 * inv;
    v[i] = p1 * inv;
    if (!(fabsf(u[i]) < 1024.0f && fabsf(v[i]) < 1024.0f)) return true;
  }
  bool pos = true, neg = true;
  float dmin = 3.0e38f;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int j = (i + 1) & 3;
    const float ex = u[j] - u[i], ey = v[j] - v[i];
    const float c = fmaf(ey, u[i], -ex * v[i]);
    pos = pos && c >= 0.0f;
    neg = neg && c <= 0.0f;
    dmin = fminf(dmin, seg_dist2(u[i], v[i], ex, ey));
  }
  return pos || neg || !(dmin > lim);
}

// Bit l of the result is set iff staged record l (l < cnt) has a pixel box
// that meets this warp's 8x8 block of pixel centres [bx+0.5, bx+7.5] x
// [by+0.5, by+7.5] and passes block_may_hit.
__device__ __forceinline__ uint32_t chunk_mask(const float4 *buf, int cnt, int lane, float bx, float by,
                                               const CfgK &f) {
  bool hit = false;
  if (lane < cnt) {
    const float4 *r = buf + lane * kRecF4;
    const float4 b = r[4];
    const float2 x = unpack_box(b.z), y = unpack_box(b.w);
    hit = x.x <= bx + 7.5f && x.y >= bx + 0.5f && y.x <= by + 7.5f && y.y >= by + 0.5f;
    if (hit) hit = block_may_hit(r[0], r[1], r[2], b, bx, by, f);
  }
  return __ballot_sync(0xffffffffu, hit);
}

// ---------------------------------------------------------------------------
// Two pixels per lane with the packed two-lane binary32 instructions
// ---------------------------------------------------------------------------
// A lane owns the pixels (x, y) and (x, y + 4) of an 8x8 quadrant: they share
// the column, so the pair's x offset is one scalar and everything after it is
// evaluated for both pixels at once with the packed add / multiply / fused
// multiply-add (one instruction for two lanes of arithmetic).  Each packed
// operation rounds exactly like its scalar counterpart, and eval_pair2 runs
// the same operations in the same order as eval_pair, so both give the same
// contribution decisions bit for bit.
__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 sel2(bool k0, bool k1, float2 a, float2 b) {
  return make_float2(k0 ? a.x : b.x, k1 ? a.y : b.y);
}

struct Eval2 {
  float dx;
  float2 dy, u, v, q, g, araw, at, z, inv;
  bool c0, c1;
};

// eval_pair for the pixels (px, py.x) and (px, py.y).  For a pixel that does
// not contribute the fields are finite (a surfel's reciprocal is replaced by
// 0 where the ray misses the plane's front), so a caller may blend it in with
// weight 0.  eval_pair2_t is the same for a record known to be a 3D Gaussian
// (IS3D) or a surfel; eval_pair2 picks by the record's sign.
template <bool IS3D>
__device__ __forceinline__ void eval_pair2_t(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r4,
                                             float px, float2 py, const CfgK &f, Eval2 &e) {
  e.dx = __fsub_rn(__fsub_rn(px, r0.x), r4.x);
  e.dy = add2(add2(py, f2(-r0.y)), f2(-r4.y));
  float2 q;
  float alpha;
  if constexpr (IS3D) {
    e.u = fma2(f2(r1.x), f2(e.dx), mul2(f2(r1.y), e.dy));
    e.v = mul2(f2(r1.z), e.dy);
    q = fma2(e.u, e.u, mul2(e.v, e.v));
    alpha = r0.w;
    e.z = f2(r0.z);
    e.inv = f2(1.0f);
    e.c0 = e.c1 = true;
  } else {
    const float2 p0 = fma2(f2(r1.x), f2(e.dx), mul2(f2(r1.y), e.dy));
    const float2 p1 = fma2(f2(r1.z), f2(e.dx), mul2(f2(r1.w), e.dy));
    const float2 p2 = fma2(f2(r2.x), f2(e.dx), fma2(f2(r2.y), e.dy, f2(1.0f)));
    e.c0 = p2.x > 0.0f;
    e.c1 = p2.y > 0.0f;
    e.inv = make_float2(e.c0 ? rcp_approx(p2.x) : 0.0f, e.c1 ? rcp_approx(p2.y) : 0.0f);
    e.z = mul2(f2(r0.z), e.inv);
    e.c0 = e.c0 && e.z.x > f.near_z;
    e.c1 = e.c1 && e.z.y > f.near_z;
    e.u = mul2(p0, e.inv);
    e.v = mul2(p1, e.inv);
    q = fma2(e.u, e.u, mul2(e.v, e.v));
    alpha = -r0.w;
  }
  e.q = q;
  const float2 x = mul2(q, f2(-0.5f * kLog2e));
  e.g = make_float2(ex2_approx(x.x), ex2_approx(x.y));
  e.araw = mul2(f2(alpha), e.g);
  e.c0 = e.c0 && e.araw.x >= f.alpha_min;
  e.c1 = e.c1 && e.araw.y >= f.alpha_min;
  e.at = make_float2(fminf(e.araw.x, f.alpha_max), fminf(e.araw.y, f.alpha_max));
}
__device__ __forceinline__ void eval_pair2(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r4,
                                           float px, float2 py, const CfgK &f, Eval2 &e) {
  if (r0.w > 0.0f)
    eval_pair2_t<true>(r0, r1, r2, r4, px, py, f, e);
  else
    eval_pair2_t<false>(r0, r1, r2, r4, px, py, f, e);
}

// Block tests of one staged chunk against QW quadrants of a tile: bit l of
// m[k] is set iff staged record l (l < cnt) may hit quadrant q0 + k, tested
// only for the quadrants whose bit is set in `want` (the others get 0).
template <int QW>
__device__ __forceinline__ void chunk_masks(const float4 *buf, int cnt, int lane, float tx0, float ty0, int q0,
                                            uint32_t want, const CfgK &f, uint32_t (&m)[QW]) {
  float4 r0, r1, r2, b;
  const bool live = lane < cnt;
  float2 bxr, byr;
  if (live) {
    const float4 *r = buf + lane * kRecF4;
    r0 = r[0];
    r1 = r[1];
    r2 = r[2];
    b = r[4];
    bxr = unpack_box(b.z);
    byr = unpack_box(b.w);
  }
#pragma unroll
  for (int k = 0; k < QW; ++k) {
    const int q = q0 + k;
    const float bx = tx0 + 8.0f * (float)(q & 1), by = ty0 + 8.0f * (float)(q >> 1);
    bool hit = false;
    if (live && ((want >> k) & 1u)) {
      hit = bxr.x <= bx + 7.5f && bxr.y >= bx + 0.5f && byr.x <= by + 7.5f && byr.y >= by + 0.5f;
      if (hit) hit = block_may_hit(r0, r1, r2, b, bx, by, f);
    }
    m[k] = __ballot_sync(0xffffffffu, hit);
  }
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// Forward with packed pixel pairs: a warp owns QW quadrants of a tile (the
// CTA has 4 / QW warps), walks the tile's list once for all of them, and
// skips a quadrant once all its pixels have terminated.
// The forward's evaluation: eval_pair2's operations (so the same decisions),
// with the contribution decision as a 0/1 float m, so that the blend can
// mask by multiplication (packed) instead of selecting (one lane at a time).
// Every value is finite for a pixel that does not contribute: a surfel's
// reciprocal is 0 where the ray misses the plane's front, and where it hits,
// p2 = Q20 dx + Q21 dy + 1 is an exact product plus one binary32 rounded
// once, so a nonzero p2 is far above the range where 1/p2 overflows.
struct EvalF2 {
  float2 at, z, m;
};

__device__ __forceinline__ void eval_fwd2(const float4 &r0, const float4 &r1, const float4 &r2, const float4 &r4,
                                          float px, float2 py, const CfgK &f, EvalF2 &e) {
  const float dx = __fsub_rn(__fsub_rn(px, r0.x), r4.x);
  const float2 dy = add2(add2(py, f2(-r0.y)), f2(-r4.y));
  float2 q;
  float alpha;
  bool k0 = true, k1 = true;
  if (r0.w > 0.0f) {
    const float2 u = fma2(f2(r1.x), f2(dx), mul2(f2(r1.y), dy));
    const float2 v = mul2(f2(r1.z), dy);
    q = fma2(u, u, mul2(v, v));
    alpha = r0.w;
    e.z = f2(r0.z);
  } else {
    const float2 p0 = fma2(f2(r1.x), f2(dx), mul2(f2(r1.y), dy));
    const float2 p1 = fma2(f2(r1.z), f2(dx), mul2(f2(r1.w), dy));
    const float2 p2 = fma2(f2(r2.x), f2(dx), fma2(f2(r2.y), dy, f2(1.0f)));
    k0 = p2.x > 0.0f;
    k1 = p2.y > 0.0f;
    const float2 inv = make_float2(k0 ? rcp_approx(p2.x) : 0.0f, k1 ? rcp_approx(p2.y) : 0.0f);
    e.z = mul2(f2(r0.z), inv);
    k0 = k0 && e.z.x > f.near_z;
    k1 = k1 && e.z.y > f.near_z;
    const float2 u = mul2(p0, inv), v = mul2(p1, inv);
    q = fma2(u, u, mul2(v, v));
    alpha = -r0.w;
  }
  const float2 x = mul2(q, f2(-0.5f * kLog2e));
  const float2 araw = mul2(f2(alpha), make_float2(ex2_approx(x.x), ex2_approx(x.y)));
  e.m = make_float2(k0 && araw.x >= f.alpha_min ? 1.0f : 0.0f, k1 && araw.y >= f.alpha_min ? 1.0f : 0.0f);
  e.at = make_float2(fminf(araw.x, f.alpha_max), fminf(araw.y, f.alpha_max));
}

// Forward state of a lane's two pixels: live is 1 until the pixel
// terminates; last (the 1-based index of the last contributor) and nc (the
// contributors) are counted in binary32, exact below 2^24.
struct Fwd2 {
  float2 T, C0, C1, C2, D, N0, N1, N2, live, last, nc;
};

// Eq. 2 for the two pixels at once.  A pair counts where it contributes and
// the pixel is live (m); the pixel stops before it if T would fall below
// T_min; a pair that does not count has weight 0, and T * (1 - 0) leaves the
// transmittance as it was.
__device__ __forceinline__ void blend2(Fwd2 &s, const EvalF2 &e, const float4 &r2, const float4 &r3,
                                       const CfgK &cfg, float idx) {
  const float2 m = mul2(e.m, s.live);
  const float2 at = mul2(e.at, m);
  const float2 Tn = mul2(s.T, add2(f2(1.0f), neg2(at)));
  const float2 st = make_float2(Tn.x < cfg.T_min ? 1.0f : 0.0f, Tn.y < cfg.T_min ? 1.0f : 0.0f);
  s.live = fma2(neg2(st), s.live, s.live);
  const float2 keep = fma2(neg2(st), m, m);
  const float2 a2 = mul2(e.at, keep);
  const float2 w = mul2(a2, s.T);
  s.T = mul2(s.T, add2(f2(1.0f), neg2(a2)));
  // e.z is finite for every pair (see EvalF2), so a pair that does not count
  // adds w z = 0 to the depth, as it adds 0 to the colour
  const float2 z = e.z;
  s.C0 = fma2(w, f2(r2.z), s.C0);
  s.C1 = fma2(w, f2(r2.w), s.C1);
  s.C2 = fma2(w, f2(r3.x), s.C2);
  s.D = fma2(w, z, s.D);
  s.N0 = fma2(w, f2(r3.y), s.N0);
  s.N1 = fma2(w, f2(r3.z), s.N1);
  s.N2 = fma2(w, f2(r3.w), s.N2);
  s.last = fma2(keep, add2(f2(idx), neg2(s.last)), s.last);
  s.nc = add2(s.nc, keep);
}

__device__ __forceinline__ void write_pix1(const RenderArgs &a, int x, int y, float T, float C0, float C1, float C2,
                                           float D, float N0, float N1, float N2, uint32_t last, uint32_t nc) {
  if (x >= a.cam.W || y >= a.cam.H) return;
  const size_t HW = (size_t)a.cam.W * a.cam.H;
  const size_t p = (size_t)y * a.cam.W + x;
  a.rgb[p] = C0 + T * a.cfg.bg[0];
  a.rgb[p + HW] = C1 + T * a.cfg.bg[1];
  a.rgb[p + 2 * HW] = C2 + T * a.cfg.bg[2];
  a.depth[p] = D;
  a.normal[p] = N0;
  a.normal[p + HW] = N1;
  a.normal[p + 2 * HW] = N2;
  a.alpha[p] = 1.0f - T;
  a.T_final[p] = T;
  a.n_last[p] = last;
  if (a.n_contrib) a.n_contrib[p] = nc;
}

template <int QW>
__device__ __forceinline__ void render_tile_fwd2(const RenderArgs &a, int tile, int local, int q0,
                                                 float4 (*smw)[kCh * kRecF4]) {
  const int lane = threadIdx.x & 31;
  const int tx0 = (local % a.cam.TX) * kTile, ty0 = (local / a.cam.TX) * kTile;
  const int lx = lane & 7, ly = lane >> 3;
  Fwd2 s[QW];
  uint32_t live = 0;
#pragma unroll
  for (int k = 0; k < QW; ++k) {
    const int q = q0 + k;
    const int x = tx0 + 8 * (q & 1) + lx, y = ty0 + 8 * (q >> 1) + ly;
    s[k].T = f2(1.0f);
    s[k].C0 = s[k].C1 = s[k].C2 = s[k].D = s[k].N0 = s[k].N1 = s[k].N2 = f2(0.0f);
    s[k].last = s[k].nc = f2(0.0f);
    s[k].live = make_float2(x < a.cam.W && y < a.cam.H ? 1.0f : 0.0f, x < a.cam.W && y + 4 < a.cam.H ? 1.0f : 0.0f);
    if (__any_sync(0xffffffffu, s[k].live.x + s[k].live.y != 0.0f)) live |= 1u << k;
  }
  const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
  if (live && start < end) {
    const float4 *rec = reinterpret_cast<const float4 *>(a.rec);
    const float px = (float)(tx0 + lx) + 0.5f;  // + 8 for the right quadrants
    stage_chunk(rec, a.vals, start, end, &smw[0][0], nullptr, lane);
    int buf = 0;
    for (uint32_t base = start; base < end; base += kCh) {
      if (base + kCh < end) {
        stage_chunk(rec, a.vals, base + kCh, end, &smw[buf ^ 1][0], nullptr, lane);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const float4 *chunk = &smw[buf][0];
      uint32_t m[QW];
      chunk_masks<QW>(chunk, (int)min((uint32_t)kCh, end - base), lane, (float)tx0, (float)ty0, q0, live, a.cfg, m);
      uint32_t any = 0;
#pragma unroll
      for (int k = 0; k < QW; ++k) any |= m[k];
      while (any && live) {
        const int j = __ffs(any) - 1;
        any &= any - 1;
        const float4 *r = chunk + j * kRecF4;
        const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4];
        const float idx = (float)(base - start + (uint32_t)j + 1u);
#pragma unroll
        for (int k = 0; k < QW; ++k) {
          if (!((live >> k) & 1u) || !((m[k] >> j) & 1u)) continue;
          const int q = q0 + k;
          const float pyq = (float)(ty0 + 8 * (q >> 1) + ly) + 0.5f;
          EvalF2 e;
          eval_fwd2(r0, r1, r2, r4, px + 8.0f * (float)(q & 1), make_float2(pyq, pyq + 4.0f), a.cfg, e);
          blend2(s[k], e, r2, r3, a.cfg, idx);
          if (!__any_sync(0xffffffffu, s[k].live.x + s[k].live.y != 0.0f)) live &= ~(1u << k);
        }
      }
      if (!live) break;
      __syncwarp();
      buf ^= 1;
    }
    cp_async_wait<0>();
  }
#pragma unroll
  for (int k = 0; k < QW; ++k) {
    const int q = q0 + k;
    const int x = tx0 + 8 * (q & 1) + lx, y = ty0 + 8 * (q >> 1) + ly;
    write_pix1(a, x, y, s[k].T.x, s[k].C0.x, s[k].C1.x, s[k].C2.x, s[k].D.x, s[k].N0.x, s[k].N1.x, s[k].N2.x,
               (uint32_t)s[k].last.x, (uint32_t)s[k].nc.x);
    write_pix1(a, x, y + 4, s[k].T.y, s[k].C0.y, s[k].C1.y, s[k].C2.y, s[k].D.y, s[k].N0.y, s[k].N1.y, s[k].N2.y,
               (uint32_t)s[k].last.y, (uint32_t)s[k].nc.y);
  }
}

// Forward CTAs: four warps, one quadrant (8x8 pixels) each; six CTAs per SM
// (78 registers, no spills).
constexpr int kFwdWarps = 4;
constexpr int kFwdMinBlocks = 6;

__global__ void __launch_bounds__(kFwdWarps * 32, kFwdMinBlocks) render_fwd2_kernel(RenderArgs a) {
  __shared__ __align__(16) float4 sm[kFwdWarps][2][kCh * kRecF4];
  const int warp = threadIdx.x >> 5;
  render_tile_fwd2<1>(a, blockIdx.x, blockIdx.x, warp, sm[warp]);
}

// Persistent forward: every warp takes (tile, quadrant) items from `counter`
// in the order `order` lists the tiles (longest list first), four items per
// tile; warps never wait for each other.
__global__ void __launch_bounds__(kFwdWarps * 32, kFwdMinBlocks) render_fwd_sched_kernel(RenderArgs a,
                                                                                     const uint32_t *order,
                                                                  uint32_t *counter, int tiles) {
  grid_dep();
  __shared__ __align__(16) float4 sm[4][2][kCh * kRecF4];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  while (true) {
    uint32_t item = 0;
    if (lane == 0) item = atomicAdd(counter, 1u);
    item = __shfl_sync(0xffffffffu, item, 0);
    if (item >= 4u * (uint32_t)tiles) break;
    const int tile = (int)__ldg(order + (item >> 2));
    render_tile_fwd2<1>(a, tile, tile, (int)(item & 3u), sm[warp]);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(kFwdWarps * 32, kFwdMinBlocks) render_batch2_kernel(BatchRenderArgs b) {
  __shared__ __align__(16) float4 sm[kFwdWarps][2][kCh * kRecF4];
  const int gy = blockIdx.x / b.TXmax, tx = blockIdx.x % b.TXmax;
  int r = 0;
  while (r + 1 < b.nreq && gy >= b.row_off[r + 1]) ++r;
  const RenderArgs &a = b.req[r];
  if (tx >= a.cam.TX) return;
  const int warp = threadIdx.x >> 5;
  render_tile_fwd2<1>(a, blockIdx.x, (gy - b.row_off[r]) * a.cam.TX + tx, warp, sm[warp]);
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
// Sum 16 per-lane values over the warp by recursive halving: after five
// exchange steps lane l holds the total of component
// 8 b4 + 4 b3 + 2 b2 + b1 (b = bits of l); lanes l and l^1 hold the same one.
__device__ __forceinline__ float warp_sum16(float (&v)[16], int lane, int &comp) {
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 8];
    const float keep = hi ? v[i + 8] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 8;
    const float send = hi ? v[i] : v[i + 4];
    const float keep = hi ? v[i + 4] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 4;
    const float send = hi ? v[i] : v[i + 2];
    const float keep = hi ? v[i + 2] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  {
    const bool hi = lane & 2;
    const float send = hi ? v[0] : v[1];
    const float keep = hi ? v[1] : v[0];
    v[0] = keep + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  comp = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 + ((lane >> 1) & 1);
  return v[0];
}

struct BwdPix {
  float px, py, T;
  uint32_t last;
  float dC0, dC1, dC2, dD, dN0, dN1, dN2, dA;       // upstream gradient of the pixel
  // Everything behind the current pair, blended, only enters the gradient
  // through its dot product with the pixel's upstream gradient, so that dot
  // product is kept instead of the eight blended channels:
  // S = sum_k acc_k dC_k over rgb, depth, normal and alpha (acc_alpha
  // blends the constant 1), starting from the background colour.
  float S;
  bool inside;
};

__device__ __forceinline__ void load_bwd_pix(BwdPix &s, const RenderBwdArgs &a, int x, int y) {
  s.px = (float)x + 0.5f;
  s.py = (float)y + 0.5f;
  s.inside = x < a.cam.W && y < a.cam.H;
  s.T = 1.0f;
  s.last = 0;
  s.dC0 = s.dC1 = s.dC2 = s.dD = s.dN0 = s.dN1 = s.dN2 = s.dA = 0.f;
  s.S = 0.f;
  if (!s.inside) return;
  const size_t HW = (size_t)a.cam.W * a.cam.H;
  const size_t p = (size_t)y * a.cam.W + x;
  s.T = a.T_final[p];
  s.last = a.n_last[p];
  if (a.g_rgb) { s.dC0 = a.g_rgb[p]; s.dC1 = a.g_rgb[p + HW]; s.dC2 = a.g_rgb[p + 2 * HW]; }
  if (a.g_depth) s.dD = a.g_depth[p];
  if (a.g_normal) { s.dN0 = a.g_normal[p]; s.dN1 = a.g_normal[p + HW]; s.dN2 = a.g_normal[p + 2 * HW]; }
  if (a.g_alpha) s.dA = a.g_alpha[p];
  s.S = a.cfg.bg[0] * s.dC0 + a.cfg.bg[1] * s.dC1 + a.cfg.bg[2] * s.dC2;
}

// Add one contributing pair's gradient of the record (layout: common.cuh)
// into g, recovering the transmittance in front of it by division and
// updating the blended "behind" term (reverse replay of Eq. 2).  With
// cd = sum_k c_k dC_k over the record's channels, dL/dalpha is
// T_i (cd - S), and blending the pair in moves S by alpha (cd - S).
// FULL = false: only the rgb cotangent is nonzero (depth, normal and alpha
// gradients absent), so their terms and gradient slots (6, 13-15) vanish.
template <bool FULL>
__device__ __forceinline__ void pair_grad(float (&g)[16], BwdPix &s, const PairEval &e, const float4 &r0,
                                          const float4 &r1, const float4 &r2, const float4 &r3,
                                          const CfgK &cfg) {
  const float c0 = r2.z, c1 = r2.w, c2 = r3.x, n0 = r3.y, n1 = r3.z, n2 = r3.w;
  const float Ti = __fdividef(s.T, 1.0f - e.at);
  const float w = e.at * Ti;
  const float cd = FULL ? fmaf(c0, s.dC0, fmaf(c1, s.dC1, fmaf(c2, s.dC2, fmaf(e.z, s.dD,
                          fmaf(n0, s.dN0, fmaf(n1, s.dN1, fmaf(n2, s.dN2, s.dA)))))))
                        : fmaf(c0, s.dC0, fmaf(c1, s.dC1, c2 * s.dC2));
  const float fsum = cd - s.S;
  const float dat = Ti * fsum;
  s.S = fmaf(e.at, fsum, s.S);
  s.T = Ti;
  g[1] += w * s.dC0; g[2] += w * s.dC1; g[3] += w * s.dC2;
  if (FULL) { g[13] += w * s.dN0; g[14] += w * s.dN1; g[15] += w * s.dN2; }
  const float dzp = FULL ? w * s.dD : 0.0f;
  float dd = 0.f;
  if (e.araw <= cfg.alpha_max) {
    g[0] += dat * e.g;
    dd = dat * (-0.5f * e.at);
  }
  if (r0.w > 0.0f) {
    // shape gradient in the footprint's own coordinates (u, v) = W (dx, dy):
    // dL/dH for d = (u, v) H (u, v)^T at H = I (rounding-stable for needles)
    const float ddu = dd * e.u, ddv = dd * e.v;
    g[7] += ddu * e.u;
    g[8] += 2.0f * ddu * e.v;
    g[9] += ddv * e.v;
    g[4] -= dd * 2.0f * e.u * r1.x;
    g[5] -= dd * 2.0f * (e.u * r1.y + e.v * r1.z);
    if (FULL) g[6] += dzp;
  } else {
    // the homography's gradient in the splat's own coordinates:
    // (du, dv) (u, v)^T and p2 dL/dp2 (u, v) (the preprocess backward maps
    // them back to the parameters)
    const float du = 2.0f * e.u * dd, dv = 2.0f * e.v * dd;
    const float dp0 = du * e.inv, dp1 = dv * e.inv;
    const float dq2 = -(du * e.u + dv * e.v + dzp * e.z);
    const float dp2 = dq2 * e.inv;
    g[7] += du * e.u; g[8] += du * e.v;
    g[9] += dv * e.u; g[10] += dv * e.v;
    g[11] += dq2 * e.u; g[12] += dq2 * e.v;
    g[4] -= dp0 * r1.x + dp1 * r1.z + dp2 * r2.x;
    g[5] -= dp0 * r1.y + dp1 * r1.w + dp2 * r2.y;
    if (FULL) g[6] += dzp * e.inv;
  }
}

// Butterfly sums for the rgb-only backward, which reduces 9 (3D) or 12 (2D)
// of the 16 slots.  sum8: slots v[0..7] transposed over lanes 16, 8, 4 and
// finished over lanes 2, 1; lane l ends with slot ((l >> 2) & 7)'s total.
// sum4: slots v[0..3] over lanes 16, 8, finished over 4, 2, 1; lane l ends
// with slot ((l >> 3) & 3).  sum1: plain butterfly.
__device__ __forceinline__ float sum8(float (&v)[8], int lane) {
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 4];
    v[i] = (hi ? v[i + 4] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 8;
    const float send = hi ? v[i] : v[i + 2];
    v[i] = (hi ? v[i + 2] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  {
    const bool hi = lane & 4;
    const float send = hi ? v[0] : v[1];
    v[0] = (hi ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 2);
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 1);
  return v[0];
}
__device__ __forceinline__ float sum4(float (&v)[4], int lane) {
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const bool hi = lane & 16;
    const float send = hi ? v[i] : v[i + 2];
    v[i] = (hi ? v[i + 2] : v[i]) + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  {
    const bool hi = lane & 8;
    const float send = hi ? v[0] : v[1];
    v[0] = (hi ? v[1] : v[0]) + __shfl_xor_sync(0xffffffffu, send, 8);
  }
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xffffffffu, v[0], o);
  return v[0];
}
__device__ __forceinline__ float sum1(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Transpose sum of 32 values over the warp: after the five exchange steps
// lane l holds the warp total of value l.
__device__ __forceinline__ float sum32(float (&v)[32], int lane) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const bool hi = lane & o;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const float send = hi ? v[i] : v[i + o];
      v[i] = (hi ? v[i + o] : v[i]) + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// The three gradient sets of the frequency-decoupled backward in one
// transpose: 3D, 27 values (9 slots per set); surfels, 32 of the 36 values
// and a 4-value tail (set 2's slots 9..12).
__device__ __forceinline__ void reduce_record3(float (&g)[3][16], bool is3d, int lane, float *const (&rows)[3],
                                               uint32_t id) {
  // the reduced slots 0..5, 7.. (slot 6, the depth term, is absent without
  // a depth cotangent): the s-th is s + (s >= 6)
  auto slot = [](int s) { return s + (s >= 6 ? 1 : 0); };
  float v[32];
  const int per = is3d ? 9 : 12;
#pragma unroll
  for (int k = 0; k < 32; ++k) {
    // value k: set k / per, its (k % per)-th slot; zero past the 27 3D values
    const float a3 = k < 27 ? g[k / 9][slot(k % 9)] : 0.0f;
    const float a2 = g[k / 12][slot(k % 12)];
    v[k] = is3d ? a3 : a2;
  }
  float tail[4] = {g[2][slot(8)], g[2][slot(9)], g[2][slot(10)], g[2][slot(11)]};
  const float t = sum32(v, lane);
  if (lane < 3 * per) atomicAdd(rows[lane / per] + (size_t)id * kGradW + slot(lane % per), t);
  if (!is3d) {
    const float u = sum4(tail, lane);
    if ((lane & 7) == 0) atomicAdd(rows[2] + (size_t)id * kGradW + slot(8 + ((lane >> 3) & 3)), u);
  }
}

// Warp-reduce one record's gradient and add it to the record's row.
template <bool FULL>
__device__ __forceinline__ void reduce_record(float (&g)[16], bool is3d, int lane, float *row) {
  if (FULL) {
    int comp;
    const float v = warp_sum16(g, lane, comp);
    if ((lane & 1) == 0) atomicAdd(row + comp, v);
    return;
  }
  // slots 0-5, 7, 8 in one transpose; then 9 (3D) or 9-12 (2D).  One
  // atomic instruction adds all of them: lanes 4i hold the transpose's
  // slots, lane 1 (3D) or lanes 8i + 1 (2D) the others.
  float a[8] = {g[0], g[1], g[2], g[3], g[4], g[5], g[7], g[8]};
  const int s8 = (lane >> 2) & 7;
  const float v8 = sum8(a, lane);
  float vt;
  int st;
  bool tail;
  if (is3d) {
    vt = sum1(g[9]);
    st = 9;
    tail = lane == 1;
  } else {
    float b[4] = {g[9], g[10], g[11], g[12]};
    vt = sum4(b, lane);
    st = 9 + ((lane >> 3) & 3);
    tail = (lane & 7) == 1;
  }
  const bool head = (lane & 3) == 0;
  if (head || tail) atomicAdd(row + (head ? (s8 < 6 ? s8 : s8 + 1) : st), head ? v8 : vt);
}

// Reverse walk over a warp's part of one tile list (shared by both backward
// kernels): stage chunks of 32 records from the back with cp.async, test
// them against the warp's block, and call body(record, id, jrel) for each
// record that passes, newest first.
template <class Body>
__device__ __forceinline__ void bwd_walk(const RenderBwdArgs &a, int tile, int warp, int lane, int bx, int by,
                                         uint32_t wmax, float4 (*sm)[2][kCh * kRecF4],
                                         uint32_t (*sid)[2][kCh], Body &&body) {
  const uint32_t start = a.ranges[2 * tile];
  const float4 *rec = reinterpret_cast<const float4 *>(a.rec);
  const float fbx = (float)bx, fby = (float)by;
  uint32_t ce = start + wmax;
  uint32_t cs = ce - min((uint32_t)kCh, wmax);
  stage_chunk(rec, a.vals, cs, ce, &sm[warp][0][0], &sid[warp][0][0], lane);
  int buf = 0;
  while (true) {
    const bool has_next = cs > start;
    const uint32_t ncs = has_next ? cs - min((uint32_t)kCh, cs - start) : cs;
    if (has_next) {
      stage_chunk(rec, a.vals, ncs, cs, &sm[warp][buf ^ 1][0], &sid[warp][buf ^ 1][0], lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const float4 *chunk = &sm[warp][buf][0];
    uint32_t mask = chunk_mask(chunk, (int)(ce - cs), lane, fbx, fby, a.cfg);
    while (mask) {
      const int jj = 31 - __clz(mask);
      mask &= ~(1u << jj);
      body(chunk + jj * kRecF4, sid[warp][buf][jj], cs + (uint32_t)jj - start);
    }
    if (!has_next) break;
    __syncwarp();
    buf ^= 1;
    ce = cs;
    cs = ncs;
  }
  cp_async_wait<0>();
}

// Tile scheduling for the one-warp-per-tile backward.  A tile's work is its
// longest reverse walk (the largest n_last of its pixels); tiles are handed
// out longest first from an atomic counter, so that no long tile starts last
// and leaves the device idle behind it.
__global__ void k_tile_work(const uint32_t *__restrict__ n_last, int W, int H, int TX, int tiles,
                            uint32_t *__restrict__ work) {
  const int t = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (t >= tiles) return;
  const int tx0 = (t % TX) * kTile, ty0 = (t / TX) * kTile;
  uint32_t m = 0;
  for (int k = lane; k < kTilePix; k += 32) {
    const int x = tx0 + (k & 15), y = ty0 + (k >> 4);
    if (x < W && y < H) m = max(m, __ldg(n_last + (size_t)y * W + x));
  }
  m = __reduce_max_sync(0xffffffffu, m);
  if (lane == 0) work[t] = m;
}

// A tile's forward work estimate: its list length.
__global__ void k_tile_len(const uint32_t *__restrict__ ranges, int tiles, uint32_t *__restrict__ work) {
  grid_dep();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < tiles) work[t] = ranges[2 * t + 1] - ranges[2 * t];
}

// Half-octave buckets of the work, longest first; order[] lists the tiles by
// descending bucket.  One CTA; also clears the hand-out counter.
__device__ __forceinline__ int work_bucket(uint32_t w) {
  if (w == 0) return 0;
  const int e = 31 - __clz(w);
  return min(63, 2 * e + 1 + (e > 0 ? (int)((w >> (e - 1)) & 1u) : 0));
}

__global__ void __launch_bounds__(1024) k_tile_order(const uint32_t *__restrict__ work, int tiles,
                                                     uint32_t *__restrict__ order, uint32_t *__restrict__ counter) {
  grid_dep();
  __shared__ uint32_t cnt[64];
  if (threadIdx.x < 64) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) atomicAdd(&cnt[work_bucket(work[t])], 1u);
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int b = 63; b >= 0; --b) {
      const uint32_t c = cnt[b];
      cnt[b] = acc;
      acc += c;
    }
    *counter = 0;
  }
  __syncthreads();
  for (int t = threadIdx.x; t < tiles; t += blockDim.x) order[atomicAdd(&cnt[work_bucket(work[t])], 1u)] = (uint32_t)t;
}

// Per-pixel state of the one-warp-per-tile backward: transmittance and the
// blended dot product S stay in registers; the read-only cotangent and n_last
// of a lane's pixel pair sit in shared memory (lane-indexed, so the loads are
// conflict-free), which keeps the kernel's registers low enough for 20 warps
// per SM.
template <int NC>
struct Bwd4 {
  float2 T, S[NC];
};
template <int NC>
struct Bwd4Smem {
  float2 dC[4][3 * NC][32];  // [quadrant][set * 3 + channel][lane]: the lane's two pixels
  uint2 last[4][32];         // [quadrant][lane]
  uint32_t qmax[4];          // per quadrant: the latest contributor of any of its pixels
  uint32_t qb[kCh];          // per staged record: the quadrants it is evaluated against
};

// Quadrant bits of staged record `lane` (lane < cnt) of the one-warp-per-tile
// backward: bit k is set iff the record lies before quadrant k's latest
// contributor (the first lim[k] records of the chunk do) and may hit the
// quadrant (box overlap, then block_may_hit).  Kept in shared memory, so
// that no mask stays in registers across the record loop.
__device__ __forceinline__ uint32_t chunk_qbits(const float4 *buf, int cnt, int lane, float tx0, float ty0,
                                                const uint32_t (&lim)[4], const CfgK &f) {
  uint32_t bits = 0;
  if (lane < cnt) {
    const float4 *r = buf + lane * kRecF4;
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], b = r[4];
    const float2 bxr = unpack_box(b.z), byr = unpack_box(b.w);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      if ((uint32_t)lane >= lim[k]) continue;
      const float bx = tx0 + 8.0f * (float)(k & 1), by = ty0 + 8.0f * (float)(k >> 1);
      bool hit = bxr.x <= bx + 7.5f && bxr.y >= bx + 0.5f && byr.x <= by + 7.5f && byr.y >= by + 0.5f;
      if (hit) hit = block_may_hit(r0, r1, r2, b, bx, by, f);
      bits |= (hit ? 1u : 0u) << k;
    }
  }
  return bits;
}

// Reverse replay of one record for the two pixels of a lane and NC cotangent
// sets (sharing the evaluation and the transmittance step), accumulated into
// the per-record slots g[set] (pair_grad_rgb for both pixels).
template <int NC, bool IS3D>
__device__ __forceinline__ void pair_grad2s(float (&g)[NC][16], Bwd4<NC> &s, const Bwd4Smem<NC> &ps, int k,
                                            int lane, const Eval2 &e, bool c0, bool c1, const float4 &r0,
                                            const float4 &r1, const float4 &r2, const float4 &r3, const CfgK &cfg) {
  const float2 at = sel2(c0, c1, e.at, f2(0.0f));
  const float2 om = add2(f2(1.0f), neg2(at));
  const float2 Ti = mul2(s.T, make_float2(rcp_approx(om.x), rcp_approx(om.y)));
  s.T = Ti;  // T * rcp(1) = T where the pair does not reach the pixel (at = 0)
  const float2 w = mul2(at, Ti);
  const bool o0 = c0 && e.araw.x <= cfg.alpha_max, o1 = c1 && e.araw.y <= cfg.alpha_max;
  const float2 oTi = sel2(o0, o1, Ti, f2(0.0f));
  auto acc = [](float &gk, float2 a, float2 b) { gk = fmaf(a.x, b.x, fmaf(a.y, b.y, gk)); };
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float2 dC0 = ps.dC[k][3 * c][lane], dC1 = ps.dC[k][3 * c + 1][lane], dC2 = ps.dC[k][3 * c + 2][lane];
    const float2 cd = fma2(f2(r2.z), dC0, fma2(f2(r2.w), dC1, mul2(f2(r3.x), dC2)));
    const float2 fsum = add2(cd, neg2(s.S[c]));
    s.S[c] = fma2(at, fsum, s.S[c]);
    acc(g[c][1], w, dC0);
    acc(g[c][2], w, dC1);
    acc(g[c][3], w, dC2);
    const float2 dato = mul2(oTi, fsum);
    acc(g[c][0], dato, e.g);
    // the moments of pair_moments2 in scalar slots (moments_to_slots3 maps
    // them to the record-gradient slots once per record):
    //   [4] sum e p2^-1 u  [5] sum e p2^-1 v  [7] sum e u u  [8] sum e u v
    //   [9] sum e v v; surfels also [10] sum e p2^-1 q  [11] sum e q u
    //   [12] sum e q v      (e = dL/d(alpha) alpha, 3D: p2 = 1)
    const float2 ee = mul2(dato, at);
    const float2 eu = mul2(ee, e.u), ev = mul2(ee, e.v);
    acc(g[c][7], eu, e.u);
    acc(g[c][8], eu, e.v);
    acc(g[c][9], ev, e.v);
    if constexpr (IS3D) {
      g[c][4] += eu.x + eu.y;
      g[c][5] += ev.x + ev.y;
    } else {
      const float2 eq = mul2(ee, e.q), ei = mul2(ee, e.inv);
      acc(g[c][11], eq, e.u);
      acc(g[c][12], eq, e.v);
      acc(g[c][4], ei, e.u);
      acc(g[c][5], ei, e.v);
      acc(g[c][10], ei, e.q);
    }
  }
}

// The three-set moments of pair_grad2s mapped, per set, to the
// record-gradient slots (the same linear map as moments_to_slots).
template <int NC, bool IS3D>
__device__ __forceinline__ void moments_to_slots3(float (&g)[NC][16], const float4 &r1, const float4 &r2) {
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float m4 = g[c][4], m5 = g[c][5], m7 = g[c][7], m8 = g[c][8], m9 = g[c][9];
    if constexpr (IS3D) {
      g[c][4] = r1.x * m4;
      g[c][5] = fmaf(r1.y, m4, r1.z * m5);
      g[c][7] = -0.5f * m7;
      g[c][8] = -m8;
      g[c][9] = -0.5f * m9;
    } else {
      const float m10 = g[c][10];
      g[c][4] = fmaf(r1.x, m4, fmaf(r1.z, m5, -r2.x * m10));
      g[c][5] = fmaf(r1.y, m4, fmaf(r1.w, m5, -r2.y * m10));
      g[c][7] = -m7;
      g[c][8] = -m8;
      g[c][9] = -m8;
      g[c][10] = -m9;
      // [11], [12] are already the p2 dL/dp2 sums
    }
  }
}

// One cotangent set, with the per-record sums kept packed over the lane's
// two pixels (one packed FMA per term instead of two scalar ones) and in the
// form that needs the fewest products per pair: with e = dL/d(alpha) * alpha
// (= -2 dL/dd, zero where the pair does not contribute or alpha is clamped),
//   G[0] = sum dL/d(alpha) G      G[1..3] = sum w dL/dC
//   G[4..6] = sum e (u u, u v, v v)
//   G[7..8] = sum e p2^-1 (u, v)  (3D: p2 = 1)
//   2D only: G[9..10] = sum e q (u, v), G[11] = sum e p2^-1 q   (q = u^2 + v^2)
// moments_to_slots maps them, linearly, to the record-gradient slots.
template <bool IS3D>
__device__ __forceinline__ void pair_moments2(float2 (&G)[12], Bwd4<1> &s, const Bwd4Smem<1> &ps, int k, int lane,
                                              const Eval2 &e, bool c0, bool c1, const float4 &r2,
                                              const float4 &r3, const CfgK &cfg) {
  const float2 at = sel2(c0, c1, e.at, f2(0.0f));
  const float2 om = add2(f2(1.0f), neg2(at));
  // a pixel the pair does not reach has at = 0, and T * rcp(1) is T (the
  // approximate reciprocal of 1 is exactly 1 on sm_103a; no decision here
  // depends on T, so even a rounding-level change would only perturb the
  // gradient at the rounding level)
  const float2 Ti = mul2(s.T, make_float2(rcp_approx(om.x), rcp_approx(om.y)));
  s.T = Ti;
  const float2 w = mul2(at, Ti);
  const bool o0 = c0 && e.araw.x <= cfg.alpha_max, o1 = c1 && e.araw.y <= cfg.alpha_max;
  const float2 oTi = sel2(o0, o1, Ti, f2(0.0f));
  const float2 dC0 = ps.dC[k][0][lane], dC1 = ps.dC[k][1][lane], dC2 = ps.dC[k][2][lane];
  const float2 cd = fma2(f2(r2.z), dC0, fma2(f2(r2.w), dC1, mul2(f2(r3.x), dC2)));
  const float2 fsum = add2(cd, neg2(s.S[0]));
  s.S[0] = fma2(at, fsum, s.S[0]);
  G[1] = fma2(w, dC0, G[1]);
  G[2] = fma2(w, dC1, G[2]);
  G[3] = fma2(w, dC2, G[3]);
  const float2 dato = mul2(oTi, fsum);
  G[0] = fma2(dato, e.g, G[0]);
  const float2 ee = mul2(dato, at);
  const float2 eu = mul2(ee, e.u), ev = mul2(ee, e.v);
  G[4] = fma2(eu, e.u, G[4]);
  G[5] = fma2(eu, e.v, G[5]);
  G[6] = fma2(ev, e.v, G[6]);
  if constexpr (IS3D) {
    G[7] = add2(G[7], eu);
    G[8] = add2(G[8], ev);
  } else {
    const float2 eq = mul2(ee, e.q), ei = mul2(ee, e.inv);
    G[9] = fma2(eq, e.u, G[9]);
    G[10] = fma2(eq, e.v, G[10]);
    G[7] = fma2(ei, e.u, G[7]);
    G[8] = fma2(ei, e.v, G[8]);
    G[11] = fma2(ei, e.q, G[11]);
  }
}

// The record-gradient slots of one lane's moments (the map is linear, so the
// warp sum of the slots is the slots of the warp sum).
//  3D: dd = -e / 2, so d h00 = -G4 / 2, d h01 (as 2 u v) = -G5, d h11 = -G6 / 2,
//      and d x_c = -2 sum dd (W00 u) = W00 G7, d y_c = W01 G7 + W11 G8.
//  2D: du = -e u, dv = -e v and p2 dL/dp2 = e q give the four (du, dv) (u, v)
//      sums -G4, -G5, -G5, -G6 and (G9, G10); the centre gradient
//      -sum p2^-1 (du Q0k + dv Q1k + e q Q2k) is Q0k G7 + Q1k G8 - Q2k G11.
template <bool IS3D>
__device__ __forceinline__ void moments_to_slots(const float2 (&G)[12], const float4 &r1, const float4 &r2,
                                                 float (&g)[16]) {
  auto h = [](float2 a) { return a.x + a.y; };
#pragma unroll
  for (int i = 0; i < 4; ++i) g[i] = h(G[i]);
  const float m4 = h(G[4]), m5 = h(G[5]), m6 = h(G[6]), m7 = h(G[7]), m8 = h(G[8]);
  if constexpr (IS3D) {
    g[4] = r1.x * m7;
    g[5] = fmaf(r1.y, m7, r1.z * m8);
    g[7] = -0.5f * m4;
    g[8] = -m5;
    g[9] = -0.5f * m6;
  } else {
    const float m11 = h(G[11]);
    g[4] = fmaf(r1.x, m7, fmaf(r1.z, m8, -r2.x * m11));
    g[5] = fmaf(r1.y, m7, fmaf(r1.w, m8, -r2.y * m11));
    g[7] = -m4;
    g[8] = -m5;
    g[9] = -m5;
    g[10] = -m6;
    g[11] = h(G[9]);
    g[12] = h(G[10]);
  }
}

// One tile of the rgb-only backward by one warp (all four quadrants), NC
// cotangent sets.
template <int NC>
__device__ __forceinline__ void bwd4_tile(const RenderBwdArgs &a, int tile, int lane, float4 (*sm)[kCh * kRecF4],
                                          uint32_t (*sid)[kCh], Bwd4Smem<NC> &ps) {
  const int tx0 = (tile % a.cam.TX) * kTile, ty0 = (tile / a.cam.TX) * kTile;
  const int lx = lane & 7, ly = lane >> 3;
  const size_t HW = (size_t)a.cam.W * a.cam.H;
  Bwd4<NC> s[4];
  uint32_t wmax = 0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int x = tx0 + 8 * (k & 1) + lx, y = ty0 + 8 * (k >> 1) + ly;
    float Ts[2] = {1.0f, 1.0f};
    uint32_t l[2] = {0u, 0u};
    bool in[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int yy = y + 4 * h;
      in[h] = x < a.cam.W && yy < a.cam.H;
      if (in[h]) {
        const size_t p = (size_t)yy * a.cam.W + x;
        Ts[h] = a.T_final[p];
        l[h] = a.n_last[p];
      }
    }
    s[k].T = make_float2(Ts[0], Ts[1]);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const float *gc = a.g_rgbs[c];
      float2 d[3];
#pragma unroll
      for (int ch = 0; ch < 3; ++ch) {
        d[ch] = f2(0.0f);
        if (gc) {
          if (in[0]) d[ch].x = gc[(size_t)y * a.cam.W + x + ch * HW];
          if (in[1]) d[ch].y = gc[(size_t)(y + 4) * a.cam.W + x + ch * HW];
        }
        ps.dC[k][3 * c + ch][lane] = d[ch];
      }
      s[k].S[c] = fma2(f2(a.cfg.bg[0]), d[0], fma2(f2(a.cfg.bg[1]), d[1], mul2(f2(a.cfg.bg[2]), d[2])));
    }
    ps.last[k][lane] = make_uint2(l[0], l[1]);
    const uint32_t qm = __reduce_max_sync(0xffffffffu, max(l[0], l[1]));
    if (lane == 0) ps.qmax[k] = qm;
    wmax = max(wmax, qm);
  }
  __syncwarp();
  if (wmax == 0) return;
  const uint32_t start = a.ranges[2 * tile];
  const float4 *rec = reinterpret_cast<const float4 *>(a.rec);
  const float px = (float)(tx0 + lx) + 0.5f;
  uint32_t ce = start + wmax;
  uint32_t cs = ce - min((uint32_t)kCh, wmax);
  stage_chunk(rec, a.vals, cs, ce, &sm[0][0], &sid[0][0], lane);
  int buf = 0;
  while (true) {
    const bool has_next = cs > start;
    const uint32_t ncs = has_next ? cs - min((uint32_t)kCh, cs - start) : cs;
    if (has_next) {
      stage_chunk(rec, a.vals, ncs, cs, &sm[buf ^ 1][0], &sid[buf ^ 1][0], lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const float4 *chunk = &sm[buf][0];
    {
      uint32_t lim[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t q = ps.qmax[k];
        lim[k] = q > cs - start ? min((uint32_t)kCh, q - (cs - start)) : 0u;
      }
      ps.qb[lane] = chunk_qbits(chunk, (int)(ce - cs), lane, (float)tx0, (float)ty0, lim, a.cfg);
    }
    uint32_t any = __ballot_sync(0xffffffffu, ps.qb[lane] != 0u);
    __syncwarp();
    while (any) {
      const int jj = 31 - __clz(any);
      any &= ~(1u << jj);
      const float4 *r = chunk + jj * kRecF4;
      const uint32_t jrel = cs + (uint32_t)jj - start;
      const float4 r0 = r[0], r1 = r[1], r2 = r[2], r3 = r[3], r4 = r[4];
      const bool is3d = r0.w > 0.0f;
      const uint32_t qb = ps.qb[jj];
      if constexpr (NC == 1) {
        // the quadrant loop specialised for the record's kind
        auto record = [&](auto kind) {
          constexpr bool IS3D = decltype(kind)::value;
          float2 G[12];
#pragma unroll
          for (int i = 0; i < 12; ++i) G[i] = f2(0.0f);
          bool hit = false;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (!((qb >> k) & 1u)) continue;
            const float pyq = (float)(ty0 + 8 * (k >> 1) + ly) + 0.5f;
            Eval2 e;
            eval_pair2_t<IS3D>(r0, r1, r2, r4, px + 8.0f * (float)(k & 1), make_float2(pyq, pyq + 4.0f), a.cfg,
                               e);
            const uint2 l = ps.last[k][lane];
            const bool c0 = e.c0 && jrel < l.x, c1 = e.c1 && jrel < l.y;
            if (!__any_sync(0xffffffffu, c0 || c1)) continue;
            hit = true;
            pair_moments2<IS3D>(G, s[k], ps, k, lane, e, c0, c1, r2, r3, a.cfg);
          }
          if (!hit) return;
          float gs[16];
          moments_to_slots<IS3D>(G, r1, r2, gs);
          reduce_record<false>(gs, IS3D, lane, a.rec_grads[0] + (size_t)sid[buf][jj] * kGradW);
        };
        if (is3d)
          record(std::true_type{});
        else
          record(std::false_type{});
      } else {
        auto record = [&](auto kind) {
          constexpr bool IS3D = decltype(kind)::value;
          float gs[NC][16];
#pragma unroll
          for (int c = 0; c < NC; ++c)
#pragma unroll
            for (int i = 0; i < 16; ++i) gs[c][i] = 0.0f;
          bool hit = false;
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            if (!((qb >> k) & 1u)) continue;
            const float pyq = (float)(ty0 + 8 * (k >> 1) + ly) + 0.5f;
            Eval2 e;
            eval_pair2_t<IS3D>(r0, r1, r2, r4, px + 8.0f * (float)(k & 1), make_float2(pyq, pyq + 4.0f), a.cfg,
                               e);
            const uint2 l = ps.last[k][lane];
            const bool c0 = e.c0 && jrel < l.x, c1 = e.c1 && jrel < l.y;
            if (!__any_sync(0xffffffffu, c0 || c1)) continue;
            hit = true;
            pair_grad2s<NC, IS3D>(gs, s[k], ps, k, lane, e, c0, c1, r0, r1, r2, r3, a.cfg);
          }
          if (!hit) return;
          moments_to_slots3<NC, IS3D>(gs, r1, r2);
          reduce_record3(gs, IS3D, lane, a.rec_grads, sid[buf][jj]);
        };
        if (is3d)
          record(std::true_type{});
        else
          record(std::false_type{});
      }
    }
    if (!has_next) break;
    __syncwarp();
    buf ^= 1;
    ce = cs;
    cs = ncs;
  }
  cp_async_wait<0>();
}

// One warp per tile; with `order`, a persistent grid takes tiles longest
// first from `counter`, else CTA b takes tile b.  One cotangent set: 20
// one-warp CTAs per SM (96 registers, no spills); three sets: 16.
template <int NC>
__global__ void __launch_bounds__(32, NC == 1 ? 20 : 16) render_bwd_rgb4_kernel(RenderBwdArgs a, const uint32_t *order,
                                                                              uint32_t *counter, int tiles) {
  grid_dep();
  __shared__ __align__(16) float4 sm[2][kCh * kRecF4];
  __shared__ uint32_t sid[2][kCh];
  __shared__ Bwd4Smem<NC> ps;
  const int lane = threadIdx.x & 31;
  if (!order) {
    bwd4_tile<NC>(a, blockIdx.x, lane, sm, sid, ps);
    return;
  }
  while (true) {
    uint32_t t = 0;
    if (lane == 0) t = atomicAdd(counter, 1u);
    t = __shfl_sync(0xffffffffu, t, 0);
    if (t >= (uint32_t)tiles) break;
    bwd4_tile<NC>(a, (int)__ldg(order + t), lane, sm, sid, ps);
    __syncwarp();
  }
}

// general backward: any of the rgb, depth, normal and alpha cotangents
__global__ void __launch_bounds__(kRW * 32, 5) render_bwd_kernel(RenderBwdArgs a) {
  __shared__ __align__(16) float4 sm[kRW][2][kCh * kRecF4];
  __shared__ uint32_t sid[kRW][2][kCh];
  const int tile = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int bx, by;
  block_of(tile, a.cam.TX, warp, bx, by);
  BwdPix s[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) load_bwd_pix(s[k], a, bx + (lane & 7), by + (lane >> 3) + 4 * k);
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, max(s[0].last, s[1].last));
  if (wmax == 0) return;
  bwd_walk(a, tile, warp, lane, bx, by, wmax, sm, sid, [&](const float4 *r, uint32_t id, uint32_t jrel) {
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r4 = r[4];
    PairEval e0, e1;
    const bool c0 = s[0].inside && jrel < s[0].last && eval_pair(r0, r1, r2, r4, s[0].px, s[0].py, a.cfg, e0);
    const bool c1 = s[1].inside && jrel < s[1].last && eval_pair(r0, r1, r2, r4, s[1].px, s[1].py, a.cfg, e1);
    if (!__any_sync(0xffffffffu, c0 || c1)) return;
    float g[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) g[k] = 0.f;
    const float4 r3 = r[3];
    if (c0) pair_grad<true>(g, s[0], e0, r0, r1, r2, r3, a.cfg);
    if (c1) pair_grad<true>(g, s[1], e1, r0, r1, r2, r3, a.cfg);
    reduce_record<true>(g, r0.w > 0.0f, lane, a.rec_grad + (size_t)id * kGradW);
  });
}

// Prefer the largest shared-memory carve-out: the staging buffers decide how
// many tile CTAs fit on an SM.
static void prefer_shared(const void *fn) {
  cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
}

int launch_render_fwd(const RenderArgs &a, cudaStream_t s) {
  const int tiles = a.cam.TX * a.cam.TY;
  if (tiles <= 0) return 0;
  static bool once = (prefer_shared((const void *)render_fwd2_kernel), true);
  (void)once;
  if (!a.tile_sched) {
    render_fwd2_kernel<<<tiles, kFwdWarps * 32, 0, s>>>(a);
    return 0;
  }
  // longest lists first, every warp taking (tile, quadrant) items
  static int resident = [] {
    prefer_shared((const void *)render_fwd_sched_kernel);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, render_fwd_sched_kernel, 128, 0);
    return max(1, sms * max(per, 1));
  }();
  uint32_t *work = a.tile_sched, *order = a.tile_sched + tiles, *counter = a.tile_sched + 2 * (size_t)tiles;
  // programmatic dependent launches (grid_dep() at the top of each kernel)
  pdl_launch(k_tile_len, (tiles + 255) / 256, 256, 0, s, a.ranges, tiles, work);
  pdl_launch(k_tile_order, 1, 1024, 0, s, (const uint32_t *)work, tiles, order, counter);
  pdl_launch(render_fwd_sched_kernel, min(tiles, resident), 128, 0, s, a, (const uint32_t *)order, counter, tiles);
  return 0;
}

int launch_render_batch(const BatchRenderArgs &b, int rows, cudaStream_t s) {
  const int blocks = rows * b.TXmax;
  if (blocks <= 0) return 0;
  static bool once = (prefer_shared((const void *)render_batch2_kernel), true);
  (void)once;
  render_batch2_kernel<<<blocks, kFwdWarps * 32, 0, s>>>(b);
  return 0;
}

// The one-warp-per-tile rgb backward: with a scheduling scratch, the tiles'
// work and a longest-first order are computed on the device and a persistent
// grid (every resident CTA) takes the tiles in that order.
template <int NC>
static void launch_bwd4(const RenderBwdArgs &a, int tiles, cudaStream_t s) {
  static int resident = [] {
    prefer_shared((const void *)render_bwd_rgb4_kernel<NC>);
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, render_bwd_rgb4_kernel<NC>, 32, 0);
    return max(1, sms * max(per, 1));
  }();
  if (!a.tile_sched) {
    render_bwd_rgb4_kernel<NC><<<tiles, 32, 0, s>>>(a, nullptr, nullptr, tiles);
    return;
  }
  uint32_t *work = a.tile_sched, *order = a.tile_sched + tiles, *counter = a.tile_sched + 2 * (size_t)tiles;
  // (the first follows the record-gradient memset; the others are
  // programmatic dependent launches)
  k_tile_work<<<(tiles + 7) / 8, 256, 0, s>>>(a.n_last, a.cam.W, a.cam.H, a.cam.TX, tiles, work);
  pdl_launch(k_tile_order, 1, 1024, 0, s, (const uint32_t *)work, tiles, order, counter);
  pdl_launch(render_bwd_rgb4_kernel<NC>, min(tiles, resident), 32, 0, s, a, (const uint32_t *)order, counter, tiles);
}

int launch_render_bwd(const RenderBwdArgs &a, cudaStream_t s) {
  const int tiles = a.cam.TX * a.cam.TY;
  if (tiles <= 0) return 0;
  static bool once = (prefer_shared((const void *)render_bwd_kernel), true);
  (void)once;
  if (a.nc == 0 && (a.g_depth || a.g_normal || a.g_alpha)) {
    render_bwd_kernel<<<tiles, kRW * 32, 0, s>>>(a);
    return 0;
  }
  // rgb cotangents only: their depth/normal/alpha terms are identically 0
  RenderBwdArgs b = a;
  if (b.nc == 0) {
    b.nc = 1;
    b.g_rgbs[0] = a.g_rgb;
    b.rec_grads[0] = a.rec_grad;
  }
  if (b.nc == 3) {
    launch_bwd4<3>(b, tiles, s);
    return 0;
  }
  for (int c = 0; c < b.nc; ++c) {
    RenderBwdArgs one = b;
    one.g_rgbs[0] = b.g_rgbs[c];
    one.rec_grads[0] = b.rec_grads[c];
    launch_bwd4<1>(one, tiles, s);
  }
  return 0;
}

}  // namespace hgs
