// render.cu -- per-tile blending of the hybrid rasterizer (EGGS Sec. 3.1,
// Eq. 1, Eq. 2) and its backward.
//
// One CTA per 16x16 tile, 4 warps; each warp owns an 8x8 pixel block, two
// pixels per lane (rows y and y + 4), and walks the tile's sorted list on its
// own: it stages the list 32 records at a time into a private double buffer
// in shared memory with cp.async, skips records whose pixel box misses its
// block, and leaves as soon as a ballot says every one of its pixels has
// terminated (transmittance below T_min).  No CTA-wide barrier is ever
// taken, so warps of a tile never wait for each other.
//
// The per-pair evaluation (eval_pair) is written with explicitly rounded
// operations so the backward kernel reproduces the forward's contribution
// decisions bit for bit.
#include <cuda_fp16.h>

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
// forward
// ---------------------------------------------------------------------------
struct FwdPix {
  float px, py, T, C0, C1, C2, D, N0, N1, N2;
  uint32_t last, nc;
  bool inside, done;
};

// front-to-back blending of one contributor (Eq. 2), stopping before the
// first one that would take T below T_min
__device__ __forceinline__ void blend(FwdPix &s, const float4 *r, const float4 &r0, const float4 &r1,
                                      const float4 &r2, const float4 &r4, const CfgK &cfg, uint32_t idx) {
  if (s.done) return;
  PairEval e;
  if (!eval_pair(r0, r1, r2, r4, s.px, s.py, cfg, e)) return;
  const float Tn = s.T * (1.0f - e.at);
  if (Tn < cfg.T_min) {
    s.done = true;
    return;
  }
  const float w = e.at * s.T;
  const float4 r3 = r[3];
  s.C0 = fmaf(w, r2.z, s.C0);
  s.C1 = fmaf(w, r2.w, s.C1);
  s.C2 = fmaf(w, r3.x, s.C2);
  s.D = fmaf(w, e.z, s.D);
  s.N0 = fmaf(w, r3.y, s.N0);
  s.N1 = fmaf(w, r3.z, s.N1);
  s.N2 = fmaf(w, r3.w, s.N2);
  s.T = Tn;
  s.last = idx;
  s.nc += 1u;
}

__device__ __forceinline__ void write_pix(const RenderArgs &a, const FwdPix &s) {
  if (!s.inside) return;
  const size_t HW = (size_t)a.cam.W * a.cam.H;
  const size_t p = (size_t)(s.py - 0.5f) * a.cam.W + (size_t)(s.px - 0.5f);
  a.rgb[p] = s.C0 + s.T * a.cfg.bg[0];
  a.rgb[p + HW] = s.C1 + s.T * a.cfg.bg[1];
  a.rgb[p + 2 * HW] = s.C2 + s.T * a.cfg.bg[2];
  a.depth[p] = s.D;
  a.normal[p] = s.N0;
  a.normal[p + HW] = s.N1;
  a.normal[p + 2 * HW] = s.N2;
  a.alpha[p] = 1.0f - s.T;
  a.T_final[p] = s.T;
  a.n_last[p] = s.last;
  if (a.n_contrib) a.n_contrib[p] = s.nc;
}

// One 16x16 tile: `tile` indexes the ranges, `local` is the tile within the
// request's own grid (a.cam.TX columns).
__device__ __forceinline__ void render_tile_fwd(const RenderArgs &a, int tile, int local,
                                                float4 (*sm)[2][kCh * kRecF4]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int bx, by;
  block_of(local, a.cam.TX, warp, bx, by);
  FwdPix s[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const int x = bx + (lane & 7), y = by + (lane >> 3) + 4 * k;
    s[k].px = (float)x + 0.5f;
    s[k].py = (float)y + 0.5f;
    s[k].inside = x < a.cam.W && y < a.cam.H;
    s[k].done = !s[k].inside;
    s[k].T = 1.0f;
    s[k].C0 = s[k].C1 = s[k].C2 = s[k].D = s[k].N0 = s[k].N1 = s[k].N2 = 0.0f;
    s[k].last = s[k].nc = 0u;
  }
  if (__all_sync(0xffffffffu, s[0].done && s[1].done)) return;
  const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
  const float4 *rec = reinterpret_cast<const float4 *>(a.rec);
  const float fbx = (float)bx, fby = (float)by;

  if (start < end) stage_chunk(rec, a.vals, start, end, &sm[warp][0][0], nullptr, lane);
  int buf = 0;
  for (uint32_t base = start; base < end; base += kCh) {
    if (base + kCh < end) {
      stage_chunk(rec, a.vals, base + kCh, end, &sm[warp][buf ^ 1][0], nullptr, lane);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    const float4 *chunk = &sm[warp][buf][0];
    uint32_t mask = chunk_mask(chunk, (int)min((uint32_t)kCh, end - base), lane, fbx, fby, a.cfg);
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      if (s[0].done && s[1].done) continue;
      const float4 *r = chunk + j * kRecF4;
      const float4 r0 = r[0], r1 = r[1], r2 = r[2], r4 = r[4];
      const uint32_t idx = base - start + (uint32_t)j + 1u;
      blend(s[0], r, r0, r1, r2, r4, a.cfg, idx);
      blend(s[1], r, r0, r1, r2, r4, a.cfg, idx);
    }
    if (__all_sync(0xffffffffu, s[0].done && s[1].done)) break;
    __syncwarp();
    buf ^= 1;
  }
  cp_async_wait<0>();
  write_pix(a, s[0]);
  write_pix(a, s[1]);
}

__global__ void __launch_bounds__(kRW * 32) render_fwd_kernel(RenderArgs a) {
  __shared__ __align__(16) float4 sm[kRW][2][kCh * kRecF4];
  render_tile_fwd(a, blockIdx.x, blockIdx.x, sm);
}

__global__ void __launch_bounds__(kRW * 32) render_batch_kernel(BatchRenderArgs b) {
  __shared__ __align__(16) float4 sm[kRW][2][kCh * kRecF4];
  const int gy = blockIdx.x / b.TXmax, tx = blockIdx.x % b.TXmax;
  int r = 0;
  while (r + 1 < b.nreq && gy >= b.row_off[r + 1]) ++r;
  const RenderArgs &a = b.req[r];
  if (tx >= a.cam.TX) return;
  render_tile_fwd(a, blockIdx.x, (gy - b.row_off[r]) * a.cam.TX + tx, sm);
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
    // conic-space gradient: d = a dx^2 + 2 b dx dy + c dy^2
    const float ddx = dd * e.dx, ddy = dd * e.dy;
    g[7] += ddx * e.dx;
    g[8] += 2.0f * ddx * e.dy;
    g[9] += ddy * e.dy;
    g[4] -= dd * 2.0f * e.u * r1.x;
    g[5] -= dd * 2.0f * (e.u * r1.y + e.v * r1.z);
    if (FULL) g[6] += dzp;
  } else {
    const float du = 2.0f * e.u * dd, dv = 2.0f * e.v * dd;
    const float dp0 = du * e.inv, dp1 = dv * e.inv;
    const float dp2 = -(du * e.u + dv * e.v + dzp * e.z) * e.inv;
    g[7] += dp0 * e.dx; g[8] += dp0 * e.dy;
    g[9] += dp1 * e.dx; g[10] += dp1 * e.dy;
    g[11] += dp2 * e.dx; g[12] += dp2 * e.dy;
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
  // slots 0-5, 7, 8 in one transpose; then 9 (3D) or 9-12 (2D)
  float a[8] = {g[0], g[1], g[2], g[3], g[4], g[5], g[7], g[8]};
  const int s8 = (lane >> 2) & 7;
  const float v8 = sum8(a, lane);
  if ((lane & 3) == 0) atomicAdd(row + (s8 < 6 ? s8 : s8 + 1), v8);
  if (is3d) {
    const float v = sum1(g[9]);
    if (lane == 0) atomicAdd(row + 9, v);
  } else {
    float b[4] = {g[9], g[10], g[11], g[12]};
    const float v4 = sum4(b, lane);
    if ((lane & 7) == 0) atomicAdd(row + 9 + ((lane >> 3) & 3), v4);
  }
}

// Pixel state of the rgb-only backward with NC cotangent sets replayed at
// once: the transmittance is shared, each set keeps its cotangent and its
// blended dot product S (as in BwdPix).
template <int NC>
struct RgbPix {
  float px, py, T;
  uint32_t last;
  float dC[NC][3];
  float S[NC];
  bool inside;
};

template <int NC>
__device__ __forceinline__ void load_rgb_pix(RgbPix<NC> &s, const RenderBwdArgs &a, const float *const (&g)[3], int x,
                                             int y) {
  s.px = (float)x + 0.5f;
  s.py = (float)y + 0.5f;
  s.inside = x < a.cam.W && y < a.cam.H;
  s.T = 1.0f;
  s.last = 0;
#pragma unroll
  for (int c = 0; c < NC; ++c) { s.dC[c][0] = s.dC[c][1] = s.dC[c][2] = 0.f; s.S[c] = 0.f; }
  if (!s.inside) return;
  const size_t HW = (size_t)a.cam.W * a.cam.H;
  const size_t p = (size_t)y * a.cam.W + x;
  s.T = a.T_final[p];
  s.last = a.n_last[p];
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    if (g[c]) { s.dC[c][0] = g[c][p]; s.dC[c][1] = g[c][p + HW]; s.dC[c][2] = g[c][p + 2 * HW]; }
    s.S[c] = a.cfg.bg[0] * s.dC[c][0] + a.cfg.bg[1] * s.dC[c][1] + a.cfg.bg[2] * s.dC[c][2];
  }
}

// pair_grad<false> for NC cotangent sets sharing one evaluation and one
// transmittance step
template <int NC>
__device__ __forceinline__ void pair_grad_rgb(float (&g)[NC][16], RgbPix<NC> &s, const PairEval &e, const float4 &r0,
                                              const float4 &r1, const float4 &r2, const float4 &r3,
                                              const CfgK &cfg) {
  const float c0 = r2.z, c1 = r2.w, c2 = r3.x;
  const float Ti = __fdividef(s.T, 1.0f - e.at);
  const float w = e.at * Ti;
  s.T = Ti;
  const bool open = e.araw <= cfg.alpha_max;
#pragma unroll
  for (int c = 0; c < NC; ++c) {
    const float cd = fmaf(c0, s.dC[c][0], fmaf(c1, s.dC[c][1], c2 * s.dC[c][2]));
    const float fsum = cd - s.S[c];
    const float dat = Ti * fsum;
    s.S[c] = fmaf(e.at, fsum, s.S[c]);
    g[c][1] += w * s.dC[c][0]; g[c][2] += w * s.dC[c][1]; g[c][3] += w * s.dC[c][2];
    float dd = 0.f;
    if (open) {
      g[c][0] += dat * e.g;
      dd = dat * (-0.5f * e.at);
    }
    if (r0.w > 0.0f) {
      const float ddx = dd * e.dx, ddy = dd * e.dy;
      g[c][7] += ddx * e.dx;
      g[c][8] += 2.0f * ddx * e.dy;
      g[c][9] += ddy * e.dy;
      g[c][4] -= dd * 2.0f * e.u * r1.x;
      g[c][5] -= dd * 2.0f * (e.u * r1.y + e.v * r1.z);
    } else {
      const float du = 2.0f * e.u * dd, dv = 2.0f * e.v * dd;
      const float dp0 = du * e.inv, dp1 = dv * e.inv;
      const float dp2 = -(du * e.u + dv * e.v) * e.inv;
      g[c][7] += dp0 * e.dx; g[c][8] += dp0 * e.dy;
      g[c][9] += dp1 * e.dx; g[c][10] += dp1 * e.dy;
      g[c][11] += dp2 * e.dx; g[c][12] += dp2 * e.dy;
      g[c][4] -= dp0 * r1.x + dp1 * r1.z + dp2 * r2.x;
      g[c][5] -= dp0 * r1.y + dp1 * r1.w + dp2 * r2.y;
    }
  }
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

// rgb-only backward (image losses): NC cotangent sets replayed together
template <int NC>
__global__ void __launch_bounds__(kRW * 32, NC == 1 ? 5 : 4) render_bwd_rgb_kernel(RenderBwdArgs a) {
  __shared__ __align__(16) float4 sm[kRW][2][kCh * kRecF4];
  __shared__ uint32_t sid[kRW][2][kCh];
  const int tile = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int bx, by;
  block_of(tile, a.cam.TX, warp, bx, by);
  RgbPix<NC> s[2];
#pragma unroll
  for (int k = 0; k < 2; ++k) load_rgb_pix<NC>(s[k], a, a.g_rgbs, bx + (lane & 7), by + (lane >> 3) + 4 * k);
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, max(s[0].last, s[1].last));
  if (wmax == 0) return;
  bwd_walk(a, tile, warp, lane, bx, by, wmax, sm, sid, [&](const float4 *r, uint32_t id, uint32_t jrel) {
    const float4 r0 = r[0], r1 = r[1], r2 = r[2], r4 = r[4];
    PairEval e0, e1;
    const bool c0 = s[0].inside && jrel < s[0].last && eval_pair(r0, r1, r2, r4, s[0].px, s[0].py, a.cfg, e0);
    const bool c1 = s[1].inside && jrel < s[1].last && eval_pair(r0, r1, r2, r4, s[1].px, s[1].py, a.cfg, e1);
    if (!__any_sync(0xffffffffu, c0 || c1)) return;
    float g[NC][16];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int k = 0; k < 16; ++k) g[c][k] = 0.f;
    const float4 r3 = r[3];
    if (c0) pair_grad_rgb<NC>(g, s[0], e0, r0, r1, r2, r3, a.cfg);
    if (c1) pair_grad_rgb<NC>(g, s[1], e1, r0, r1, r2, r3, a.cfg);
    if constexpr (NC == 3) {
      reduce_record3(g, r0.w > 0.0f, lane, a.rec_grads, id);
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) reduce_record<false>(g[c], r0.w > 0.0f, lane, a.rec_grads[c] + (size_t)id * kGradW);
    }
  });
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
  static bool once = (prefer_shared((const void *)render_fwd_kernel), true);
  (void)once;
  render_fwd_kernel<<<tiles, kRW * 32, 0, s>>>(a);
  return 0;
}

int launch_render_batch(const BatchRenderArgs &b, int rows, cudaStream_t s) {
  const int blocks = rows * b.TXmax;
  if (blocks <= 0) return 0;
  static bool once = (prefer_shared((const void *)render_batch_kernel), true);
  (void)once;
  render_batch_kernel<<<blocks, kRW * 32, 0, s>>>(b);
  return 0;
}

int launch_render_bwd(const RenderBwdArgs &a, cudaStream_t s) {
  const int tiles = a.cam.TX * a.cam.TY;
  if (tiles <= 0) return 0;
  static bool once = (prefer_shared((const void *)render_bwd_kernel),
                      prefer_shared((const void *)render_bwd_rgb_kernel<1>),
                      prefer_shared((const void *)render_bwd_rgb_kernel<3>), true);
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
  if (b.nc == 3)
    render_bwd_rgb_kernel<3><<<tiles, kRW * 32, 0, s>>>(b);
  else
    for (int c = 0; c < b.nc; ++c) {
      RenderBwdArgs one = b;
      one.g_rgbs[0] = b.g_rgbs[c];
      one.rec_grads[0] = b.rec_grads[c];
      render_bwd_rgb_kernel<1><<<tiles, kRW * 32, 0, s>>>(one);
    }
  return 0;
}

}  // namespace hgs
