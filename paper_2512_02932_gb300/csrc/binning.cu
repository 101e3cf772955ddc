// binning.cu -- tile binning of the hybrid rasterizer: duplicate every binned
// primitive into the tiles of its rectangle and order the instances by the
// 64-bit key tile_id << 32 | depth_key (ties by primitive id).
//
// The key's low 32 bits depend only on the primitive, so the LSD radix sort
// is factored: its four depth digits are sorted once over the N binned
// primitives, the instances are emitted in that order, and only the tile
// digits are sorted over the K instances.  Every pass is stable, so the
// result is exactly the order of the 64-bit key with ties by id.
//
// Every kernel runs on a fixed grid (kSortBlocks) and reads the element count
// from device memory, so the whole pipeline needs no host synchronisation;
// capacity overflow is detected on the device and reported through the
// error word with nothing written out of bounds.
#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

constexpr int kTileElems = kSortThreads * kSortItems;  // 2048
constexpr uint32_t kNoDigit = 0xffffffffu;

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t bin_layout(void *base, int64_t n, int64_t capacity, BinWorkspace *ws) {
  size_t off = 0;
  char *b = static_cast<char *>(base);
  auto take = [&](size_t bytes) -> void * {
    void *p = b ? b + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t nn = (size_t)(n > 0 ? n : 1), cc = (size_t)(capacity > 0 ? capacity : 1);
  ws->hist = (uint32_t *)take(sizeof(uint32_t) * 256 * kSortBlocks + sizeof(uint32_t) * 256);
  ws->blk = (uint64_t *)take(sizeof(uint64_t) * kSortBlocks);
  ws->counters = (int64_t *)take(sizeof(int64_t) * 8);
  for (int k = 0; k < 2; ++k) {
    ws->dk[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
    ws->dv[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
  }
  ws->offs = (uint32_t *)take(sizeof(uint32_t) * nn);
  ws->tk[0] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tk[1] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tv = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->bytes = off;
  return off;
}

// Contiguous range of this block: whole 2048-element tiles, evenly shared.
__device__ __forceinline__ void block_range(int64_t n, int64_t &b0, int64_t &b1) {
  const int64_t tiles = (n + kTileElems - 1) / kTileElems;
  const int64_t per = (tiles + gridDim.x - 1) / gridDim.x;
  b0 = min(n, (int64_t)blockIdx.x * per * kTileElems);
  b1 = min(n, b0 + per * kTileElems);
}

__device__ __forceinline__ int64_t read_n(const int64_t *d_n, int64_t n_host) {
  return d_n ? *d_n : n_host;
}

__device__ __forceinline__ uint32_t lanemask_lt() {
  uint32_t m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// radix pass: per-block digit histograms
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
    k_hist(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ valid, const int64_t *d_n,
           int64_t n_host, const int64_t *d_abort, int shift, int bits, uint32_t *__restrict__ hist) {
  __shared__ uint32_t wh[kSortThreads / 32][256];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < (kSortThreads / 32) * 256; k += kSortThreads) (&wh[0][0])[k] = 0u;
  __syncthreads();
  const bool aborted = d_abort && *d_abort;
  const int64_t n = aborted ? 0 : read_n(d_n, n_host);
  int64_t b0, b1;
  block_range(n, b0, b1);
  const uint32_t mask = (1u << bits) - 1u;
  for (int64_t e = b0 + tid; e < b1; e += kSortThreads) {
    if (valid && __ldg(valid + e) == 0u) continue;
    const uint32_t d = (__ldg(keys + e) >> shift) & mask;
    atomicAdd(&wh[warp][d], 1u);
  }
  __syncthreads();
  uint32_t s = 0;
#pragma unroll
  for (int w = 0; w < kSortThreads / 32; ++w) s += wh[w][tid];
  hist[(size_t)tid * gridDim.x + blockIdx.x] = s;
}

// one block per digit: exclusive scan of that digit's per-block counts;
// digit totals go to dtot[256]
__global__ void __launch_bounds__(256) k_hist_scan(uint32_t *__restrict__ hist, int nblocks,
                                                   uint32_t *__restrict__ dtot) {
  __shared__ uint32_t wsum[8];
  const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint32_t *row = hist + (size_t)d * nblocks;
  const int per = (nblocks + 255) / 256;
  uint32_t loc[8];
  uint32_t sum = 0;
  for (int k = 0; k < per; ++k) {
    const int idx = tid * per + k;
    loc[k] = idx < nblocks ? row[idx] : 0u;
    sum += loc[k];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t wbase = 0;
  for (int w = 0; w < warp; ++w) wbase += wsum[w];
  uint32_t run = wbase + incl - sum;
  for (int k = 0; k < per; ++k) {
    const int idx = tid * per + k;
    if (idx < nblocks) row[idx] = run;
    run += loc[k];
  }
  if (tid == 255) dtot[d] = wbase + incl;
}

// stable scatter: ranks by warp-local match + per-warp digit counters.
// The next tile's keys and values are loaded while the current one is ranked
// (register double buffer); the per-digit bases are double-buffered so a tile
// takes two barriers.
struct TileRegs {
  uint32_t key[kSortItems], val[kSortItems], dig[kSortItems];
};

__device__ __forceinline__ void load_tile(TileRegs &t, const uint32_t *__restrict__ keys_in,
                                          const uint32_t *__restrict__ vals_in,
                                          const uint32_t *__restrict__ valid, int64_t tb, int64_t b1,
                                          int warp, int lane, int shift, uint32_t mask) {
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const int64_t e = tb + warp * (32 * kSortItems) + r * 32 + lane;
    t.dig[r] = kNoDigit;
    t.key[r] = 0u;
    t.val[r] = 0u;
    if (e < b1) {
      t.key[r] = __ldg(keys_in + e);
      t.val[r] = vals_in ? __ldg(vals_in + e) : (uint32_t)e;
      if (!valid || __ldg(valid + e) != 0u) t.dig[r] = (t.key[r] >> shift) & mask;
    }
  }
}

__global__ void __launch_bounds__(kSortThreads)
    k_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
              const uint32_t *__restrict__ valid, const int64_t *d_n, int64_t n_host,
              const int64_t *d_abort, int shift, int bits, const uint32_t *__restrict__ hist,
              const uint32_t *__restrict__ dtot, uint32_t *__restrict__ keys_out,
              uint32_t *__restrict__ vals_out, int64_t *count_out) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t base[2][256];
  __shared__ uint32_t wcnt[W][256];
  __shared__ uint32_t tdig[256];     // tile-local exclusive start of each digit
  __shared__ uint32_t scan_tmp[W];
  __shared__ uint32_t stage_k[kTileElems], stage_v[kTileElems];
  __shared__ uint32_t tile_count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool aborted = d_abort && *d_abort;
  const int64_t n = aborted ? 0 : read_n(d_n, n_host);
  // global base of each digit for this block
  {
    const uint32_t t = tid < (1 << bits) ? dtot[tid] : 0u;
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) scan_tmp[warp] = incl;
    __syncthreads();
    uint32_t wb = 0;
    for (int w = 0; w < warp; ++w) wb += scan_tmp[w];
    const uint32_t excl = wb + incl - t;
    base[0][tid] = excl + (tid < (1 << bits) ? hist[(size_t)tid * gridDim.x + blockIdx.x] : 0u);
    if (count_out && blockIdx.x == 0 && tid == 255) *count_out = aborted ? 0 : (int64_t)(wb + incl);
  }
  __syncthreads();
  int64_t b0, b1;
  block_range(n, b0, b1);
  const uint32_t mask = (1u << bits) - 1u;
  const uint32_t lt = lanemask_lt();
  TileRegs cur, nxt;
  if (b0 < b1) load_tile(cur, keys_in, vals_in, valid, b0, b1, warp, lane, shift, mask);
  int cb = 0;
  for (int64_t tb = b0; tb < b1; tb += kTileElems) {
    if (tb + kTileElems < b1)
      load_tile(nxt, keys_in, vals_in, valid, tb + kTileElems, b1, warp, lane, shift, mask);
    __syncwarp();
#pragma unroll
    for (int k = 0; k < 256 / 32; ++k) wcnt[warp][lane * 8 + k] = 0u;
    __syncwarp();
    // 1) warp-local stable ranks
    uint32_t loc[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t d = cur.dig[r];
      const uint32_t peers = __match_any_sync(0xffffffffu, d);
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (lane == leader && d != kNoDigit) {
        old = wcnt[warp][d];
        wcnt[warp][d] = old + __popc(peers);
      }
      old = __shfl_sync(0xffffffffu, old, leader);
      loc[r] = old + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    // 2) per digit: prefix over warps, then a tile-wide exclusive scan over
    //    digits (where each digit's run starts in the staged tile)
    uint32_t tot = 0;
    {
      uint32_t run = 0;
#pragma unroll
      for (int w = 0; w < W; ++w) {
        const uint32_t c = wcnt[w][tid];
        wcnt[w][tid] = run;
        run += c;
      }
      tot = run;
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) scan_tmp[warp] = incl;
    __syncthreads();
    {
      uint32_t wb = 0;
#pragma unroll
      for (int w = 0; w < W; ++w)
        if (w < warp) wb += scan_tmp[w];
      tdig[tid] = wb + incl - tot;
      base[cb ^ 1][tid] = base[cb][tid] + tot;
      if (tid == 255) tile_count = wb + incl;
    }
    __syncthreads();
    // 3) stage the tile in digit order
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t d = cur.dig[r];
      if (d != kNoDigit) {
        const uint32_t lpos = tdig[d] + wcnt[warp][d] + loc[r];
        stage_k[lpos] = cur.key[r];
        stage_v[lpos] = cur.val[r];
      }
    }
    __syncthreads();
    // 4) write the digit runs out: consecutive threads, consecutive addresses
    const uint32_t cnt = tile_count;
    for (uint32_t i = tid; i < cnt; i += kSortThreads) {
      const uint32_t key = stage_k[i];
      const uint32_t d = (key >> shift) & mask;
      const uint32_t pos = base[cb][d] + (i - tdig[d]);
      keys_out[pos] = key;
      vals_out[pos] = stage_v[i];
    }
    cb ^= 1;
    cur = nxt;
  }
}

// ---------------------------------------------------------------------------
// instance offsets: exclusive scan of touched[] in depth order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
    k_scan_partial(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ touched,
                   const int64_t *d_n, uint64_t *__restrict__ blk) {
  __shared__ uint64_t ws[kSortThreads / 32];
  const int tid = threadIdx.x;
  int64_t b0, b1;
  block_range(*d_n, b0, b1);
  uint64_t s = 0;
  for (int64_t j = b0 + tid; j < b1; j += kSortThreads) s += __ldg(touched + __ldg(ids + j));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((tid & 31) == 0) ws[tid >> 5] = s;
  __syncthreads();
  if (tid == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) t += ws[w];
    blk[blockIdx.x] = t;
  }
}

// single block: exclusive scan of the block partials, K, capacity check
__global__ void __launch_bounds__(1024)
    k_scan_top(uint64_t *__restrict__ blk, int nblocks, int64_t capacity, int64_t *counters,
               int64_t *d_count, int32_t *dev_err) {
  __shared__ uint64_t wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t v = tid < nblocks ? blk[tid] : 0ull;
  uint64_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint64_t wb = 0;
  for (int w = 0; w < warp; ++w) wb += wsum[w];
  if (tid < nblocks) blk[tid] = wb + incl - v;
  if (tid == 1023) {
    const uint64_t K = wb + incl;
    counters[1] = (int64_t)K;
    if (d_count) *d_count = (int64_t)K;
    const bool over = (int64_t)K > capacity || K > 0xffffffffull;
    counters[2] = over ? 1 : 0;
    if (over) set_error(dev_err, HGS_ERR_CAPACITY);
  }
}

__global__ void __launch_bounds__(kSortThreads)
    k_scan_final(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ touched,
                 const int64_t *counters, const uint64_t *__restrict__ blk,
                 uint32_t *__restrict__ offs) {
  __shared__ uint32_t wsum[kSortThreads / 32];
  __shared__ uint32_t carry;
  if (counters[2]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t b0, b1;
  block_range(counters[0], b0, b1);
  if (tid == 0) carry = (uint32_t)blk[blockIdx.x];
  __syncthreads();
  for (int64_t tb = b0; tb < b1; tb += kSortThreads) {
    const int64_t j = tb + tid;
    const uint32_t t = j < b1 ? __ldg(touched + __ldg(ids + j)) : 0u;
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wb = 0, all = 0;
#pragma unroll
    for (int w = 0; w < kSortThreads / 32; ++w) {
      if (w < warp) wb += wsum[w];
      all += wsum[w];
    }
    if (j < b1) offs[j] = carry + wb + incl - t;
    __syncthreads();
    if (tid == 0) carry += all;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// emit (tile id, primitive id) for every tile of each binned primitive,
// primitives in depth order.  A warp takes 32 consecutive primitives, whose
// instances form one contiguous output range; lanes write that range in
// order (coalesced), each output slot finding its owner lane by a binary
// search over the lanes' exclusive prefix.
// ---------------------------------------------------------------------------
constexpr uint32_t kBigRect = 256;  // tiles; larger rectangles go to k_emit_big

__global__ void __launch_bounds__(256)
    k_emit(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
           const uint16_t *__restrict__ rect, int64_t *counters, int TX,
           uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals, uint32_t *__restrict__ bigq) {
  if (counters[2]) return;
  const int64_t M = counters[0];
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t jb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); jb < M; jb += stride) {
    const int64_t j = jb + lane;
    uint32_t p = 0, off = 0, tx0 = 0, ty0 = 0, w = 1, cnt = 0;
    if (j < M) {
      p = __ldg(ids + j);
      off = __ldg(offs + j);
      const uint2 r = __ldg(reinterpret_cast<const uint2 *>(rect) + p);
      tx0 = r.x & 0xffffu;
      ty0 = r.y & 0xffffu;
      w = (r.x >> 16) - tx0 + 1;
      cnt = w * ((r.y >> 16) - ty0 + 1);
      if (cnt > kBigRect) {  // deferred: written by one block in k_emit_big
        const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(&counters[3]), 1ull);
        bigq[slot] = (uint32_t)j;
        cnt = 0;
      }
    }
    // exclusive prefix of the small counts within the warp
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t rel = j < M ? incl - cnt : 0xffffffffu;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
    const float inv_w = 1.0f / (float)w;
    for (uint32_t kb = 0; kb < total; kb += 32) {  // warp-uniform trip count
      const uint32_t k = kb + lane;
      // owner: the last lane with prefix <= k and a non-empty range
      int lo = 0;
#pragma unroll
      for (int step = 16; step > 0; step >>= 1) {
        const uint32_t pr = __shfl_sync(0xffffffffu, rel, lo + step);
        if (pr <= k) lo += step;
      }
      const uint32_t own_rel = __shfl_sync(0xffffffffu, rel, lo);
      const uint32_t own_off = __shfl_sync(0xffffffffu, off, lo);
      const uint32_t own_w = __shfl_sync(0xffffffffu, w, lo);
      const float own_iw = __shfl_sync(0xffffffffu, inv_w, lo);
      const uint32_t own_tx0 = __shfl_sync(0xffffffffu, tx0, lo);
      const uint32_t own_ty0 = __shfl_sync(0xffffffffu, ty0, lo);
      const uint32_t own_p = __shfl_sync(0xffffffffu, p, lo);
      const uint32_t l = k - own_rel;
      uint32_t dy = (uint32_t)((float)l * own_iw);
      uint32_t dx = l - dy * own_w;
      if ((int)dx < 0) { dy -= 1; dx += own_w; } else if (dx >= own_w) { dy += 1; dx -= own_w; }
      if (k < total) {
        tkeys[own_off + l] = (own_ty0 + dy) * TX + own_tx0 + dx;
        tvals[own_off + l] = own_p;
      }
    }
  }
}

// one block per deferred large rectangle
__global__ void __launch_bounds__(256)
    k_emit_big(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
               const uint16_t *__restrict__ rect, const int64_t *counters, int TX,
               const uint32_t *__restrict__ bigq, uint32_t *__restrict__ tkeys,
               uint32_t *__restrict__ tvals) {
  if (counters[2]) return;
  const int64_t nbig = counters[3];
  for (int64_t b = blockIdx.x; b < nbig; b += gridDim.x) {
    const uint32_t j = bigq[b];
    const uint32_t p = __ldg(ids + j), off = __ldg(offs + j);
    const uint2 r = __ldg(reinterpret_cast<const uint2 *>(rect) + p);
    const uint32_t tx0 = r.x & 0xffffu, ty0 = r.y & 0xffffu;
    const uint32_t w = (r.x >> 16) - tx0 + 1;
    const uint32_t cnt = w * ((r.y >> 16) - ty0 + 1);
    for (uint32_t k = threadIdx.x; k < cnt; k += blockDim.x) {
      const uint32_t dy = k / w, dx = k - dy * w;
      tkeys[off + k] = (ty0 + dy) * TX + tx0 + dx;
      tvals[off + k] = p;
    }
  }
}

__global__ void __launch_bounds__(256)
    k_ranges(const uint32_t *__restrict__ tkeys, const int64_t *counters, uint32_t *__restrict__ ranges) {
  if (counters[2]) return;
  const int64_t K = counters[1];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
       k += (int64_t)gridDim.x * blockDim.x) {
    const uint32_t t = tkeys[k];
    if (k == 0 || tkeys[k - 1] != t) ranges[2 * (size_t)t] = (uint32_t)k;
    if (k == K - 1 || tkeys[k + 1] != t) ranges[2 * (size_t)t + 1] = (uint32_t)(k + 1);
  }
}

__global__ void __launch_bounds__(256)
    k_keys64(const uint32_t *__restrict__ tkeys, const uint32_t *__restrict__ vals,
             const uint32_t *__restrict__ depth_key, const int64_t *counters, uint64_t *__restrict__ keys) {
  if (counters[2]) return;
  const int64_t K = counters[1];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
       k += (int64_t)gridDim.x * blockDim.x)
    keys[k] = ((uint64_t)tkeys[k] << 32) | __ldg(depth_key + vals[k]);
}

// ---------------------------------------------------------------------------
static void radix_pass(const uint32_t *kin, const uint32_t *vin, const uint32_t *valid,
                       const int64_t *d_n, int64_t n_host, const int64_t *d_abort, int shift,
                       int bits, const BinWorkspace &ws, uint32_t *kout, uint32_t *vout,
                       int64_t *count_out, cudaStream_t s) {
  uint32_t *dtot = ws.hist + 256 * kSortBlocks;
  k_hist<<<kSortBlocks, kSortThreads, 0, s>>>(kin, valid, d_n, n_host, d_abort, shift, bits, ws.hist);
  k_hist_scan<<<1 << bits, 256, 0, s>>>(ws.hist, kSortBlocks, dtot);
  if (bits < 8) cudaMemsetAsync(dtot + (1 << bits), 0, sizeof(uint32_t) * (256 - (1 << bits)), s);
  k_scatter<<<kSortBlocks, kSortThreads, 0, s>>>(kin, vin, valid, d_n, n_host, d_abort, shift, bits,
                                                 ws.hist, dtot, kout, vout, count_out);
}

int launch_bin_sort(const BinArgs &a, const BinWorkspace &ws, cudaStream_t s) {
  int64_t *ctr = ws.counters;
  cudaMemsetAsync(ctr, 0, sizeof(int64_t) * 8, s);
  cudaMemsetAsync(a.ranges, 0, sizeof(uint32_t) * 2 * (size_t)a.tiles, s);
  // 1) depth digits over the binned primitives (first pass compacts)
  radix_pass(a.depth_key, nullptr, a.touched, nullptr, a.n, nullptr, 0, 8, ws, ws.dk[0], ws.dv[0],
             &ctr[0], s);
  radix_pass(ws.dk[0], ws.dv[0], nullptr, &ctr[0], 0, nullptr, 8, 8, ws, ws.dk[1], ws.dv[1], nullptr, s);
  radix_pass(ws.dk[1], ws.dv[1], nullptr, &ctr[0], 0, nullptr, 16, 8, ws, ws.dk[0], ws.dv[0], nullptr, s);
  radix_pass(ws.dk[0], ws.dv[0], nullptr, &ctr[0], 0, nullptr, 24, 8, ws, ws.dk[1], ws.dv[1], nullptr, s);
  const uint32_t *ids = ws.dv[1];
  // 2) instance offsets and K (capacity check on the device)
  k_scan_partial<<<kSortBlocks, kSortThreads, 0, s>>>(ids, a.touched, &ctr[0], ws.blk);
  k_scan_top<<<1, 1024, 0, s>>>(ws.blk, kSortBlocks, a.capacity, ctr, a.d_count, a.dev_err);
  k_scan_final<<<kSortBlocks, kSortThreads, 0, s>>>(ids, a.touched, ctr, ws.blk, ws.offs);
  // 3) emit, then the tile digits
  const int passes = (a.tile_bits + 7) / 8;
  uint32_t *vbuf[2];
  vbuf[0] = (passes % 2 == 0) ? a.vals : ws.tv;
  vbuf[1] = (passes % 2 == 0) ? ws.tv : a.vals;
  // dk[0] is free once the depth sort is done: it holds the deferred queue
  k_emit<<<kSortBlocks, 256, 0, s>>>(ids, ws.offs, a.rect, ctr, a.TX, ws.tk[0], vbuf[0], ws.dk[0]);
  k_emit_big<<<kSortBlocks, 256, 0, s>>>(ids, ws.offs, a.rect, ctr, a.TX, ws.dk[0], ws.tk[0], vbuf[0]);
  // tile digits split evenly over the passes (13 bits -> 7 + 6): fewer
  // buckets per pass give longer runs in the scatter's coalesced write-out
  const int per_pass = (a.tile_bits + passes - 1) / passes;
  for (int p = 0; p < passes; ++p) {
    const int shift = per_pass * p;
    const int bits = min(per_pass, a.tile_bits - shift);
    radix_pass(ws.tk[p & 1], vbuf[p & 1], nullptr, &ctr[1], 0, &ctr[2], shift, bits, ws,
               ws.tk[(p + 1) & 1], vbuf[(p + 1) & 1], nullptr, s);
  }
  const uint32_t *tkeys = ws.tk[passes & 1];
  k_ranges<<<kSortBlocks, 256, 0, s>>>(tkeys, ctr, a.ranges);
  if (a.keys) k_keys64<<<kSortBlocks, 256, 0, s>>>(tkeys, a.vals, a.depth_key, ctr, a.keys);
  return 0;
}

}  // namespace hgs
