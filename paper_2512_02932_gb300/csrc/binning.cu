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
#include <algorithm>

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
  // the small head (counters, pass counters, histograms) is cleared with one memset
  ws->counters = (int64_t *)take(sizeof(int64_t) * 16 + sizeof(uint32_t) * 16 + sizeof(uint32_t) * 8 * 256);
  ws->tile_ctr = b ? reinterpret_cast<uint32_t *>(ws->counters + 16) : nullptr;
  ws->hist = b ? ws->tile_ctr + 16 : nullptr;
  ws->head_bytes = sizeof(int64_t) * 16 + sizeof(uint32_t) * 16 + sizeof(uint32_t) * 8 * 256;
  ws->blk = (uint64_t *)take(sizeof(uint64_t) * kSortBlocks);
  for (int k = 0; k < 2; ++k) {
    ws->dk[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
    ws->dv[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
  }
  ws->offs = (uint32_t *)take(sizeof(uint32_t) * nn);
  ws->tk[0] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tk[1] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tv = (uint32_t *)take(sizeof(uint32_t) * cc);
  // look-back status words: one per (2048-key tile, digit) of the larger sort
  const size_t tiles = (std::max(nn, cc) + kTileElems - 1) / kTileElems;
  for (int k = 0; k < 2; ++k) ws->status[k] = (uint64_t *)take(sizeof(uint64_t) * 256 * tiles);
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
// global digit histograms of up to four passes in one read of the keys
// ---------------------------------------------------------------------------
struct DigitSpec {
  int npass;
  int shift[4], bits[4];
};

struct HistArgs {
  const uint32_t *keys, *valid;  // valid: optional 0/1 filter
  const int64_t *d_n;            // element count on the device, or null: n_host
  int64_t n_host;
  const int64_t *d_abort;        // optional: nonzero -> no elements
  DigitSpec sp;
  uint32_t *hist;                // [npass][256], zero on entry
  uint64_t *status0;             // status words of the first pass, zeroed here
  int radix0;
  uint32_t *ranges;              // optional: set to (0xffffffff, 0) for `tiles`
  int tiles;
};

__device__ __forceinline__ int64_t hist_n(const HistArgs &a) {
  if (a.d_abort && *a.d_abort) return 0;
  return a.d_n ? *a.d_n : a.n_host;
}

// Counts runs of equal digits in a thread's four consecutive keys with one
// shared atomic per run.
__global__ void __launch_bounds__(256) k_digit_hist(HistArgs a) {
  __shared__ uint32_t h[4][256];
  const int tid = threadIdx.x;
  for (int k = tid; k < 4 * 256; k += 256) (&h[0][0])[k] = 0u;
  const int64_t n = hist_n(a);
  const int64_t gthreads = (int64_t)gridDim.x * blockDim.x, gid = (int64_t)blockIdx.x * blockDim.x + tid;
  {
    const int64_t zs = (n + kTileElems - 1) / kTileElems * a.radix0;
    for (int64_t k = gid; k < zs; k += gthreads) a.status0[k] = 0ull;
    if (a.ranges)
      for (int64_t k = gid; k < a.tiles; k += gthreads)
        reinterpret_cast<uint2 *>(a.ranges)[k] = make_uint2(0xffffffffu, 0u);
  }
  __syncthreads();
  const bool vec = ((reinterpret_cast<uintptr_t>(a.keys) | reinterpret_cast<uintptr_t>(a.valid)) & 15u) == 0;
  for (int64_t e = gid * 4; e < n; e += gthreads * 4) {
    uint32_t k[4], v[4];
    if (vec && e + 4 <= n) {
      const uint4 kk = __ldg(reinterpret_cast<const uint4 *>(a.keys + e));
      k[0] = kk.x; k[1] = kk.y; k[2] = kk.z; k[3] = kk.w;
      if (a.valid) {
        const uint4 vv = __ldg(reinterpret_cast<const uint4 *>(a.valid + e));
        v[0] = vv.x != 0u; v[1] = vv.y != 0u; v[2] = vv.z != 0u; v[3] = vv.w != 0u;
      } else {
        v[0] = v[1] = v[2] = v[3] = 1u;
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const bool in = e + i < n;
        k[i] = in ? __ldg(a.keys + e + i) : 0u;
        v[i] = in && (!a.valid || __ldg(a.valid + e + i) != 0u) ? 1u : 0u;
      }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      if (p >= a.sp.npass) break;
      const int sh = a.sp.shift[p];
      const uint32_t m = (1u << a.sp.bits[p]) - 1u;
      uint32_t dp = (k[0] >> sh) & m, c = v[0];
#pragma unroll
      for (int i = 1; i < 4; ++i) {
        const uint32_t d = (k[i] >> sh) & m;
        if (d != dp) {
          if (c) atomicAdd(&h[p][dp], c);
          dp = d;
          c = 0u;
        }
        c += v[i];
      }
      if (c) atomicAdd(&h[p][dp], c);
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < 4; ++p)
    if (p < a.sp.npass && tid < (1 << a.sp.bits[p]) && h[p][tid]) atomicAdd(&a.hist[p * 256 + tid], h[p][tid]);
}

// ---------------------------------------------------------------------------
// one stable radix pass with decoupled look-back (single sweep over the data)
// ---------------------------------------------------------------------------
// Tiles of 2048 keys are claimed in order through an atomic counter.  A tile
// ranks its keys (warp-local match + per-warp digit counters), publishes its
// per-digit counts, then walks back over earlier tiles' published words,
// adding counts until it meets a tile that already published its inclusive
// prefix; it then publishes its own.  Status word: flag in the top two bits
// (1 = this tile's count, 2 = inclusive prefix), value below.  A tile never
// waits for anything before publishing its count, and every earlier tile was
// claimed by a running block, so the walk always ends; it is nevertheless
// bounded, and a wait that runs out reports HGS_ERR_TIMEOUT and carries on
// with what it has (writes stay in bounds).
constexpr uint64_t kFlagCount = 1ull << 62, kFlagPrefix = 2ull << 62, kValueMask = (1ull << 62) - 1ull;
constexpr int kSpinLimit = 1 << 22;

__device__ __forceinline__ uint64_t ld_relaxed(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

struct SweepArgs {
  const uint32_t *keys_in, *vals_in;  // vals_in null: the value is the index
  const uint32_t *valid;              // optional 0/1 filter (compacting pass)
  const int64_t *d_n;                 // input count on the device, or null: n_host
  int64_t n_host;
  const int64_t *d_abort;
  int shift, bits;
  const uint32_t *ghist;              // this pass's global digit histogram [256]
  uint64_t *status;                   // [tiles << bits], zero on entry
  uint64_t *status_next;              // optional: zeroed for the next pass
  int next_radix;
  uint32_t *tile_ctr;                 // zero on entry
  uint32_t *keys_out, *vals_out;      // keys_out optional
  uint32_t *ranges;                   // optional (last tile pass): [start, end) per key
  int64_t *count_out;                 // optional: number of elements written
  int32_t *dev_err;
};

__global__ void __launch_bounds__(kSortThreads, 4) k_onesweep(SweepArgs a) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t wcnt[W][256];
  __shared__ uint32_t tdig[256];       // tile-local exclusive start of each digit
  __shared__ uint64_t gbase[256];      // global start of each digit in the output
  __shared__ uint64_t gpos[256];       // global start of this tile's run of each digit
  __shared__ uint32_t scan_tmp[W];
  __shared__ uint32_t stage_k[kTileElems], stage_v[kTileElems];
  __shared__ uint32_t s_tile, s_count;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool aborted = a.d_abort && *a.d_abort;
  const int64_t n = aborted ? 0 : (a.d_n ? *a.d_n : a.n_host);
  const int64_t ntiles = (n + kTileElems - 1) / kTileElems;
  const int R = 1 << a.bits;
  const uint32_t mask = (uint32_t)R - 1u;
  if (a.status_next) {
    const int64_t zs = ntiles * a.next_radix;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + tid; k < zs; k += (int64_t)gridDim.x * blockDim.x)
      a.status_next[k] = 0ull;
  }
  // exclusive scan of the global histogram: where each digit starts
  uint64_t n_out;
  {
    const uint32_t t = tid < R ? __ldg(a.ghist + tid) : 0u;
    uint32_t incl = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) scan_tmp[warp] = incl;
    __syncthreads();
    uint64_t wb = 0, all = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      if (w < warp) wb += scan_tmp[w];
      all += scan_tmp[w];
    }
    gbase[tid] = wb + incl - t;
    n_out = aborted ? 0 : all;
    if (a.count_out && blockIdx.x == 0 && tid == 0) *a.count_out = (int64_t)n_out;
  }
  const uint32_t lt = lanemask_lt();
  while (true) {
    if (tid == 0) s_tile = atomicAdd(a.tile_ctr, 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    if (tile >= ntiles) break;
    const int64_t tb = tile * kTileElems;
    uint32_t key[kSortItems], val[kSortItems], dig[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int64_t e = tb + warp * (32 * kSortItems) + r * 32 + lane;
      dig[r] = kNoDigit;
      key[r] = 0u;
      val[r] = 0u;
      if (e < n) {
        key[r] = __ldg(a.keys_in + e);
        val[r] = a.vals_in ? __ldg(a.vals_in + e) : (uint32_t)e;
        if (!a.valid || __ldg(a.valid + e) != 0u) dig[r] = (key[r] >> a.shift) & mask;
      }
    }
#pragma unroll
    for (int k = 0; k < 256 / 32; ++k) wcnt[warp][lane * 8 + k] = 0u;
    __syncwarp();
    // 1) warp-local stable ranks
    uint32_t loc[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t d = dig[r];
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
    // 2) per digit: prefix over warps and the tile's count; publish it
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c = wcnt[w][tid];
      wcnt[w][tid] = tot;
      tot += c;
    }
    if (tid < R) st_relaxed(a.status + (((size_t)tile) << a.bits) + tid, (tile == 0 ? kFlagPrefix : kFlagCount) | tot);
    //    tile-wide exclusive scan over digits (staging order)
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) scan_tmp[warp] = incl;
    // 3) look back for the exclusive prefix of each digit over earlier tiles
    if (tid < R) {
      uint64_t excl = 0;
      if (tile > 0) {
        int64_t j = tile - 1;
        int spins = 0;
        while (true) {
          const uint64_t w = ld_relaxed(a.status + (((size_t)j) << a.bits) + tid);
          const uint64_t f = w & ~kValueMask;
          if (f == 0ull) {
            if (++spins > kSpinLimit) {
              set_error(a.dev_err, HGS_ERR_TIMEOUT);
              break;
            }
            __nanosleep(64);
            continue;
          }
          excl += w & kValueMask;
          if (f == kFlagPrefix || j == 0) break;
          --j;
        }
        st_relaxed(a.status + (((size_t)tile) << a.bits) + tid, kFlagPrefix | (excl + tot));
      }
      gpos[tid] = gbase[tid] + excl;
    }
    __syncthreads();
    {
      uint32_t wb = 0;
#pragma unroll
      for (int w = 0; w < W; ++w)
        if (w < warp) wb += scan_tmp[w];
      tdig[tid] = wb + incl - tot;
      if (tid == 255) s_count = wb + incl;
    }
    __syncthreads();
    // 4) stage the tile in digit order
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t d = dig[r];
      if (d != kNoDigit) {
        const uint32_t lpos = tdig[d] + wcnt[warp][d] + loc[r];
        stage_k[lpos] = key[r];
        stage_v[lpos] = val[r];
      }
    }
    __syncthreads();
    // 5) write the digit runs out: consecutive threads, consecutive addresses.
    //    In the last pass of the tile sort equal keys are adjacent here, so
    //    each run's first and last element bound that tile's range.
    const uint32_t cnt = s_count;
    for (uint32_t i = tid; i < cnt; i += kSortThreads) {
      const uint32_t k = stage_k[i];
      const uint32_t d = (k >> a.shift) & mask;
      const uint64_t pos = gpos[d] + (i - tdig[d]);
      if (pos >= n_out) continue;
      if (a.keys_out) a.keys_out[pos] = k;
      a.vals_out[pos] = stage_v[i];
      if (a.ranges) {
        if (i == 0 || stage_k[i - 1] != k) atomicMin(a.ranges + 2 * (size_t)k, (uint32_t)pos);
        if (i + 1 == cnt || stage_k[i + 1] != k) atomicMax(a.ranges + 2 * (size_t)k + 1, (uint32_t)(pos + 1));
      }
    }
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

// tiles no instance reached keep their initial (0xffffffff, 0): make them [0, 0)
__global__ void __launch_bounds__(256) k_ranges_fix(uint32_t *__restrict__ ranges, int tiles) {
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
    uint2 *r = reinterpret_cast<uint2 *>(ranges) + t;
    if (r->x == 0xffffffffu) *r = make_uint2(0u, 0u);
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
// Blocks of the look-back passes: as many as fit on the device at once.
static int sweep_grid() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_onesweep, kSortThreads, 0);
    cached[dev] = std::max(1, sms) * std::max(1, per);
  }
  return cached[dev];
}

int launch_bin_sort(const BinArgs &a, const BinWorkspace &ws, cudaStream_t s) {
  int64_t *ctr = ws.counters;  // 0 = n_visible, 1 = K, 2 = overflow, 3 = deferred rects
  cudaMemsetAsync(ctr, 0, ws.head_bytes, s);
  const int G = sweep_grid();
  // 1) depth digits over the binned primitives (the first pass compacts)
  HistArgs h{};
  h.keys = a.depth_key;
  h.valid = a.touched;
  h.n_host = a.n;
  h.sp.npass = 4;
  for (int p = 0; p < 4; ++p) { h.sp.shift[p] = 8 * p; h.sp.bits[p] = 8; }
  h.hist = ws.hist;
  h.status0 = ws.status[0];
  h.radix0 = 256;
  k_digit_hist<<<G, 256, 0, s>>>(h);
  const uint32_t *dk_in = a.depth_key, *dv_in = nullptr;
  for (int p = 0; p < 4; ++p) {
    SweepArgs w{};
    w.keys_in = dk_in;
    w.vals_in = dv_in;
    w.valid = p == 0 ? a.touched : nullptr;
    w.d_n = p == 0 ? nullptr : &ctr[0];
    w.n_host = a.n;
    w.shift = 8 * p;
    w.bits = 8;
    w.ghist = ws.hist + 256 * p;
    w.status = ws.status[p & 1];
    w.status_next = p < 3 ? ws.status[(p + 1) & 1] : nullptr;
    w.next_radix = 256;
    w.tile_ctr = ws.tile_ctr + p;
    w.keys_out = ws.dk[p & 1];
    w.vals_out = ws.dv[p & 1];
    w.count_out = p == 0 ? &ctr[0] : nullptr;
    w.dev_err = a.dev_err;
    k_onesweep<<<G, kSortThreads, 0, s>>>(w);
    dk_in = ws.dk[p & 1];
    dv_in = ws.dv[p & 1];
  }
  const uint32_t *ids = ws.dv[1];
  // 2) instance offsets and K (capacity check on the device)
  k_scan_partial<<<kSortBlocks, kSortThreads, 0, s>>>(ids, a.touched, &ctr[0], ws.blk);
  k_scan_top<<<1, 1024, 0, s>>>(ws.blk, kSortBlocks, a.capacity, ctr, a.d_count, a.dev_err);
  k_scan_final<<<kSortBlocks, kSortThreads, 0, s>>>(ids, a.touched, ctr, ws.blk, ws.offs);
  // 3) emit, then the tile digits, split evenly over the passes (13 bits ->
  //    7 + 6): fewer buckets per pass give longer runs in the write-out
  const int passes = (a.tile_bits + 7) / 8;
  const int per_pass = (a.tile_bits + passes - 1) / passes;
  uint32_t *vbuf[2];
  vbuf[0] = (passes % 2 == 0) ? a.vals : ws.tv;
  vbuf[1] = (passes % 2 == 0) ? ws.tv : a.vals;
  // dk[0] is free once the depth sort is done: it holds the deferred queue
  k_emit<<<kSortBlocks, 256, 0, s>>>(ids, ws.offs, a.rect, ctr, a.TX, ws.tk[0], vbuf[0], ws.dk[0]);
  k_emit_big<<<kSortBlocks, 256, 0, s>>>(ids, ws.offs, a.rect, ctr, a.TX, ws.dk[0], ws.tk[0], vbuf[0]);
  HistArgs t{};
  t.keys = ws.tk[0];
  t.d_n = &ctr[1];
  t.d_abort = &ctr[2];
  t.sp.npass = passes;
  for (int p = 0; p < passes; ++p) {
    t.sp.shift[p] = per_pass * p;
    t.sp.bits[p] = std::min(per_pass, a.tile_bits - per_pass * p);
  }
  t.hist = ws.hist + 256 * 4;
  t.status0 = ws.status[0];
  t.radix0 = 1 << t.sp.bits[0];
  t.ranges = a.ranges;
  t.tiles = a.tiles;
  k_digit_hist<<<G, 256, 0, s>>>(t);
  for (int p = 0; p < passes; ++p) {
    const bool last = p + 1 == passes;
    SweepArgs w{};
    w.keys_in = ws.tk[p & 1];
    w.vals_in = vbuf[p & 1];
    w.d_n = &ctr[1];
    w.d_abort = &ctr[2];
    w.shift = t.sp.shift[p];
    w.bits = t.sp.bits[p];
    w.ghist = t.hist + 256 * p;
    w.status = ws.status[p & 1];
    w.status_next = last ? nullptr : ws.status[(p + 1) & 1];
    w.next_radix = last ? 0 : 1 << t.sp.bits[p + 1];
    w.tile_ctr = ws.tile_ctr + 4 + p;
    w.keys_out = (!last || a.keys) ? ws.tk[(p + 1) & 1] : nullptr;
    w.vals_out = vbuf[(p + 1) & 1];
    w.ranges = last ? a.ranges : nullptr;
    w.dev_err = a.dev_err;
    k_onesweep<<<G, kSortThreads, 0, s>>>(w);
  }
  k_ranges_fix<<<(a.tiles + 255) / 256, 256, 0, s>>>(a.ranges, a.tiles);
  if (a.keys) k_keys64<<<kSortBlocks, 256, 0, s>>>(ws.tk[passes & 1], a.vals, a.depth_key, ctr, a.keys);
  return 0;
}

}  // namespace hgs
