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

// stable scatter: ranks by warp-local match + per-warp digit counters
__global__ void __launch_bounds__(kSortThreads)
    k_scatter(const uint32_t *__restrict__ keys_in, const uint32_t *__restrict__ vals_in,
              const uint32_t *__restrict__ valid, const int64_t *d_n, int64_t n_host,
              const int64_t *d_abort, int shift, int bits, const uint32_t *__restrict__ hist,
              const uint32_t *__restrict__ dtot, uint32_t *__restrict__ keys_out,
              uint32_t *__restrict__ vals_out, int64_t *count_out) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t base[256];
  __shared__ uint32_t wcnt[W][256];
  __shared__ uint32_t scan_tmp[W];
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
    base[tid] = excl + (tid < (1 << bits) ? hist[(size_t)tid * gridDim.x + blockIdx.x] : 0u);
    if (count_out && blockIdx.x == 0 && tid == 255) *count_out = aborted ? 0 : (int64_t)(wb + incl);
  }
  __syncthreads();
  int64_t b0, b1;
  block_range(n, b0, b1);
  const uint32_t mask = (1u << bits) - 1u;
  const uint32_t lt = lanemask_lt();
  for (int64_t tb = b0; tb < b1; tb += kTileElems) {
    uint32_t key[kSortItems], val[kSortItems], dig[kSortItems], loc[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t e = tb + warp * (32 * kSortItems) + r * 32 + lane;
      dig[r] = kNoDigit;
      if (e < b1 && (!valid || __ldg(valid + e) != 0u)) {
        key[r] = __ldg(keys_in + e);
        val[r] = vals_in ? __ldg(vals_in + e) : (uint32_t)e;
        dig[r] = (key[r] >> shift) & mask;
      }
    }
#pragma unroll
    for (int k = 0; k < 256 / 32; ++k) wcnt[warp][lane * 8 + k] = 0u;
    __syncwarp();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t peers = __match_any_sync(0xffffffffu, dig[r]);
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (lane == leader && dig[r] != kNoDigit) {
        old = wcnt[warp][dig[r]];
        wcnt[warp][dig[r]] = old + __popc(peers);
      }
      old = __shfl_sync(0xffffffffu, old, leader);
      loc[r] = old + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
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
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      if (dig[r] != kNoDigit) {
        const uint32_t pos = base[dig[r]] + wcnt[warp][dig[r]] + loc[r];
        keys_out[pos] = key[r];
        vals_out[pos] = val[r];
      }
    }
    __syncthreads();
    base[tid] += tot;
    __syncthreads();
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
// primitives in depth order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    k_emit(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
           const uint16_t *__restrict__ rect, const int64_t *counters, int TX,
           uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals) {
  if (counters[2]) return;
  const int64_t M = counters[0];
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // grid-stride with whole warps alive so the cooperative path can shuffle
  for (int64_t jb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); jb < M; jb += stride) {
    const int64_t j = jb + lane;
    uint32_t p = 0, off = 0, tx0 = 0, tx1 = 0, ty0 = 0, ty1 = 0, cnt = 0;
    if (j < M) {
      p = __ldg(ids + j);
      off = __ldg(offs + j);
      const uint2 r = __ldg(reinterpret_cast<const uint2 *>(rect) + p);
      tx0 = r.x & 0xffffu; tx1 = r.x >> 16; ty0 = r.y & 0xffffu; ty1 = r.y >> 16;
      cnt = (tx1 - tx0 + 1) * (ty1 - ty0 + 1);
    }
    const bool big = cnt > 32;
    if (!big) {
      uint32_t k = off;
      for (uint32_t ty = ty0; ty <= ty1 && cnt; ++ty)
        for (uint32_t tx = tx0; tx <= tx1; ++tx, ++k) {
          tkeys[k] = ty * TX + tx;
          tvals[k] = p;
        }
    }
    uint32_t bigmask = __ballot_sync(0xffffffffu, big);
    while (bigmask) {
      const int src = __ffs(bigmask) - 1;
      bigmask &= bigmask - 1;
      const uint32_t bp = __shfl_sync(0xffffffffu, p, src);
      const uint32_t boff = __shfl_sync(0xffffffffu, off, src);
      const uint32_t btx0 = __shfl_sync(0xffffffffu, tx0, src);
      const uint32_t btx1 = __shfl_sync(0xffffffffu, tx1, src);
      const uint32_t bty0 = __shfl_sync(0xffffffffu, ty0, src);
      const uint32_t bcnt = __shfl_sync(0xffffffffu, cnt, src);
      const uint32_t w = btx1 - btx0 + 1;
      for (uint32_t k = lane; k < bcnt; k += 32) {
        const uint32_t ty = bty0 + k / w, tx = btx0 + k % w;
        tkeys[boff + k] = ty * TX + tx;
        tvals[boff + k] = bp;
      }
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
  k_emit<<<kSortBlocks, 256, 0, s>>>(ids, ws.offs, a.rect, ctr, a.TX, ws.tk[0], vbuf[0]);
  for (int p = 0; p < passes; ++p) {
    const int shift = 8 * p;
    const int bits = min(8, a.tile_bits - shift);
    radix_pass(ws.tk[p & 1], vbuf[p & 1], nullptr, &ctr[1], 0, &ctr[2], shift, bits, ws,
               ws.tk[(p + 1) & 1], vbuf[(p + 1) & 1], nullptr, s);
  }
  const uint32_t *tkeys = ws.tk[passes & 1];
  k_ranges<<<kSortBlocks, 256, 0, s>>>(tkeys, ctr, a.ranges);
  if (a.keys) k_keys64<<<kSortBlocks, 256, 0, s>>>(tkeys, a.vals, a.depth_key, ctr, a.keys);
  return 0;
}

}  // namespace hgs
