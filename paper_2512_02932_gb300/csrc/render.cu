// render.cu -- per-tile blending of the hybrid rasterizer (EGGS Sec. 3.1,
// Eq. 1, Eq. 2) and its backward.
//
// One CTA per 16x16 tile, 8 warps; each warp owns an 8x4 pixel block and
// walks the tile's sorted list on its own: it stages the list 32 records at a
// time into a private double buffer in shared memory with cp.async, and
// leaves as soon as a ballot says every one of its pixels has terminated
// (transmittance below T_min).  No CTA-wide barrier is ever taken, so warps
// of a tile never wait for each other.
//
// The per-pair evaluation (eval_pair) is written with explicitly rounded
// operations so the backward kernel reproduces the forward's contribution
// decisions bit for bit.
#include <cuda_fp16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

constexpr int kRW = 8;   // warps per CTA
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

__device__ __forceinline__ void pixel_of(int tile, int TX, int warp, int lane, int &px, int &py) {
  const int tx = tile % TX, ty = tile / TX;
  px = tx * kTile + (warp & 1) * 8 + (lane & 7);
  py = ty * kTile + (warp >> 1) * 4 + (lane >> 3);
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

// Bit l of the result is set iff staged record l (l < cnt) has a pixel box
// that meets this warp's 8x4 block of pixel centres [x0+0.5, x0+7.5] x
// [y0+0.5, y0+3.5].
__device__ __forceinline__ float2 unpack_box(float v) {
  const uint32_t u = __float_as_uint(v);
  return make_float2(__half2float(__ushort_as_half((unsigned short)(u & 0xffffu))),
                     __half2float(__ushort_as_half((unsigned short)(u >> 16))));
}

__device__ __forceinline__ uint32_t chunk_mask(const float4 *buf, int cnt, int lane, float bx0, float by0) {
  bool hit = false;
  if (lane < cnt) {
    const float4 b = buf[lane * kRecF4 + 4];
    const float2 bx = unpack_box(b.z), by = unpack_box(b.w);
    hit = bx.x <= bx0 + 7.5f && bx.y >= bx0 + 0.5f && by.x <= by0 + 3.5f && by.y >= by0 + 0.5f;
  }
  return __ballot_sync(0xffffffffu, hit);
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
// One 16x16 tile: `tile` indexes the ranges, `local` is the tile within the
// request's own grid (a.cam.TX columns).
__device__ __forceinline__ void render_tile_fwd(const RenderArgs &a, int tile, int local,
                                                float4 (*sm)[2][kCh * kRecF4]) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int pxi, pyi;
  pixel_of(local, a.cam.TX, warp, lane, pxi, pyi);
  const bool inside = pxi < a.cam.W && pyi < a.cam.H;
  const float px = (float)pxi + 0.5f, py = (float)pyi + 0.5f;
  const float wx0 = (float)((local % a.cam.TX) * kTile + (warp & 1) * 8);
  const float wy0 = (float)((local / a.cam.TX) * kTile + (warp >> 1) * 4);
  const uint32_t start = a.ranges[2 * tile], end = a.ranges[2 * tile + 1];
  const float4 *rec = reinterpret_cast<const float4 *>(a.rec);
  float T = 1.0f, C0 = 0.f, C1 = 0.f, C2 = 0.f, D = 0.f, N0 = 0.f, N1 = 0.f, N2 = 0.f;
  uint32_t last = 0, ncontrib = 0;
  bool done = !inside;
  if (__all_sync(0xffffffffu, done)) return;

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
    uint32_t mask = chunk_mask(chunk, (int)min((uint32_t)kCh, end - base), lane, wx0, wy0);
    while (mask) {
      const int j = __ffs(mask) - 1;
      mask &= mask - 1;
      if (done) continue;
      const float4 *r = chunk + j * kRecF4;
      const float4 r0 = r[0], r1 = r[1], r2 = r[2], r4 = r[4];
      PairEval e;
      if (!eval_pair(r0, r1, r2, r4, px, py, a.cfg, e)) continue;
      const float Tn = T * (1.0f - e.at);
      if (Tn < a.cfg.T_min) {
        done = true;
        continue;
      }
      const float w = e.at * T;
      const float4 r3 = r[3];
      C0 = fmaf(w, r2.z, C0);
      C1 = fmaf(w, r2.w, C1);
      C2 = fmaf(w, r3.x, C2);
      D = fmaf(w, e.z, D);
      N0 = fmaf(w, r3.y, N0);
      N1 = fmaf(w, r3.z, N1);
      N2 = fmaf(w, r3.w, N2);
      T = Tn;
      last = base - start + (uint32_t)j + 1u;
      ++ncontrib;
    }
    if (__all_sync(0xffffffffu, done)) break;
    __syncwarp();
    buf ^= 1;
  }
  cp_async_wait<0>();
  if (!inside) return;
  const size_t HW = (size_t)a.cam.W * a.cam.H;
  const size_t p = (size_t)pyi * a.cam.W + pxi;
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
  if (a.n_contrib) a.n_contrib[p] = ncontrib;
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

__global__ void __launch_bounds__(kRW * 32) render_bwd_kernel(RenderBwdArgs a) {
  __shared__ __align__(16) float4 sm[kRW][2][kCh * kRecF4];
  __shared__ uint32_t sid[kRW][2][kCh];
  const int tile = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int pxi, pyi;
  pixel_of(tile, a.cam.TX, warp, lane, pxi, pyi);
  const bool inside = pxi < a.cam.W && pyi < a.cam.H;
  const float px = (float)pxi + 0.5f, py = (float)pyi + 0.5f;
  const float wx0 = (float)((tile % a.cam.TX) * kTile + (warp & 1) * 8);
  const float wy0 = (float)((tile / a.cam.TX) * kTile + (warp >> 1) * 4);
  const uint32_t start = a.ranges[2 * tile];
  const size_t HW = (size_t)a.cam.W * a.cam.H;
  const size_t p = inside ? (size_t)pyi * a.cam.W + pxi : 0;
  float T = 1.0f;
  uint32_t last = 0;
  float dC0 = 0.f, dC1 = 0.f, dC2 = 0.f, dD = 0.f, dN0 = 0.f, dN1 = 0.f, dN2 = 0.f, dA = 0.f;
  if (inside) {
    T = a.T_final[p];
    last = a.n_last[p];
    if (a.g_rgb) { dC0 = a.g_rgb[p]; dC1 = a.g_rgb[p + HW]; dC2 = a.g_rgb[p + 2 * HW]; }
    if (a.g_depth) dD = a.g_depth[p];
    if (a.g_normal) { dN0 = a.g_normal[p]; dN1 = a.g_normal[p + HW]; dN2 = a.g_normal[p + 2 * HW]; }
    if (a.g_alpha) dA = a.g_alpha[p];
  }
  // accumulated colour / depth / normal / alpha of everything behind
  float ac0 = a.cfg.bg[0], ac1 = a.cfg.bg[1], ac2 = a.cfg.bg[2];
  float az = 0.f, an0 = 0.f, an1 = 0.f, an2 = 0.f, aa = 0.f;
  const uint32_t wmax = __reduce_max_sync(0xffffffffu, last);
  if (wmax == 0) return;
  const float4 *rec = reinterpret_cast<const float4 *>(a.rec);

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
    uint32_t mask = chunk_mask(chunk, (int)(ce - cs), lane, wx0, wy0);
    while (mask) {
      const int jj = 31 - __clz(mask);
      mask &= ~(1u << jj);
      const uint32_t j = cs + (uint32_t)jj;
      const float4 *r = chunk + jj * kRecF4;
      const float4 r0 = r[0], r1 = r[1], r2 = r[2], r4 = r[4];
      PairEval e;
      const bool contrib = inside && (j - start) < last && eval_pair(r0, r1, r2, r4, px, py, a.cfg, e);
      if (!__any_sync(0xffffffffu, contrib)) continue;
      float g[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) g[k] = 0.f;
      if (contrib) {
        const float4 r3 = r[3];
        const float c0 = r2.z, c1 = r2.w, c2 = r3.x, n0 = r3.y, n1 = r3.z, n2 = r3.w;
        const float om = 1.0f - e.at;
        const float Ti = __fdividef(T, om);
        const float w = e.at * Ti;
        const float fsum = (c0 - ac0) * dC0 + (c1 - ac1) * dC1 + (c2 - ac2) * dC2 + (e.z - az) * dD +
                           (n0 - an0) * dN0 + (n1 - an1) * dN1 + (n2 - an2) * dN2 + (1.0f - aa) * dA;
        const float dat = Ti * fsum;
        ac0 += e.at * (c0 - ac0); ac1 += e.at * (c1 - ac1); ac2 += e.at * (c2 - ac2);
        az += e.at * (e.z - az);
        an0 += e.at * (n0 - an0); an1 += e.at * (n1 - an1); an2 += e.at * (n2 - an2);
        aa += e.at * (1.0f - aa);
        T = Ti;
        g[1] = w * dC0; g[2] = w * dC1; g[3] = w * dC2;
        g[13] = w * dN0; g[14] = w * dN1; g[15] = w * dN2;
        const float dzp = w * dD;
        float dd = 0.f;
        if (e.araw <= a.cfg.alpha_max) {
          g[0] = dat * e.g;
          dd = dat * (-0.5f * e.at);
        }
        if (r0.w > 0.0f) {
          // conic-space gradient: d = a dx^2 + 2 b dx dy + c dy^2
          g[7] = dd * e.dx * e.dx;
          g[8] = dd * 2.0f * e.dx * e.dy;
          g[9] = dd * e.dy * e.dy;
          const float ddx = dd * 2.0f * e.u * r1.x;
          const float ddy = dd * 2.0f * (e.u * r1.y + e.v * r1.z);
          g[4] = -ddx; g[5] = -ddy; g[6] = dzp;
        } else {
          const float du = 2.0f * e.u * dd, dv = 2.0f * e.v * dd;
          const float dp0 = du * e.inv, dp1 = dv * e.inv;
          const float dp2 = -(du * e.u + dv * e.v + dzp * e.z) * e.inv;
          g[7] = dp0 * e.dx; g[8] = dp0 * e.dy;
          g[9] = dp1 * e.dx; g[10] = dp1 * e.dy;
          g[11] = dp2 * e.dx; g[12] = dp2 * e.dy;
          const float ddx = dp0 * r1.x + dp1 * r1.z + dp2 * r2.x;
          const float ddy = dp0 * r1.y + dp1 * r1.w + dp2 * r2.y;
          g[4] = -ddx; g[5] = -ddy; g[6] = dzp * e.inv;
        }
      }
      int comp;
      const float s = warp_sum16(g, lane, comp);
      if ((lane & 1) == 0) atomicAdd(a.rec_grad + (size_t)sid[warp][buf][jj] * kGradW + comp, s);
    }
    if (!has_next) break;
    __syncwarp();
    buf ^= 1;
    ce = cs;
    cs = ncs;
  }
  cp_async_wait<0>();
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
  static bool once = (prefer_shared((const void *)render_bwd_kernel), true);
  (void)once;
  render_bwd_kernel<<<tiles, kRW * 32, 0, s>>>(a);
  return 0;
}

}  // namespace hgs
