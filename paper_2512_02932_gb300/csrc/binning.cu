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
//
// When rectangles over kBigRect tiles carry most of the instances (heavy-
// tailed scenes), their instances skip the tile sort: they are listed from
// per-word coverage masks in depth order and merged with the sorted small
// instances (the wide path below).  The lists are the same either way.
#include <algorithm>

#include "common.cuh"
#include "kernels.cuh"

namespace hgs {

constexpr int kTileElems = kSortThreads * kSortItems;  // 2048
constexpr uint32_t kNoDigit = 0xffffffffu;
constexpr uint32_t kBigRect = 256;     // tiles: wider rectangles are deferred (k_emit_big) or take the wide path
constexpr int64_t kWideMax = 1 << 21;  // most wide primitives the mask path takes
constexpr size_t kMaskWordsMax = size_t(1) << 24;  // coverage-mask words (64 MiB)
constexpr int kWideRangesMax = 16;                 // word ranges per strip of the mask path

static size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

size_t bin_layout(void *base, int64_t n, int64_t capacity, int tiles, BinWorkspace *ws, bool wide) {
  size_t off = 0;
  char *b = static_cast<char *>(base);
  auto take = [&](size_t bytes) -> void * {
    void *p = b ? b + off : nullptr;
    off += align256(bytes);
    return p;
  };
  const size_t nn = (size_t)(n > 0 ? n : 1), cc = (size_t)(capacity > 0 ? capacity : 1);
  const size_t tt = (size_t)(tiles > 0 ? tiles : 1);
  // the small head (counters, pass counters, histograms) is cleared with one memset
  ws->counters = (int64_t *)take(sizeof(int64_t) * 16 + sizeof(uint32_t) * 16 + sizeof(uint32_t) * 8 * 256);
  ws->tile_ctr = b ? reinterpret_cast<uint32_t *>(ws->counters + 16) : nullptr;
  ws->hist = b ? ws->tile_ctr + 16 : nullptr;
  ws->head_bytes = sizeof(int64_t) * 16 + sizeof(uint32_t) * 16 + sizeof(uint32_t) * 8 * 256;
  ws->blk = (uint64_t *)take(sizeof(uint64_t) * 3 * kSortBlocks);
  for (int k = 0; k < 2; ++k) {
    ws->dk[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
    ws->dv[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
  }
  ws->offs = (uint32_t *)take(sizeof(uint32_t) * nn);
  ws->tk[0] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tk[1] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tv = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->chist = (uint32_t *)take(sizeof(uint32_t) * 256 * kSortBlocks);
  // wide path: the wide primitives' depth-order positions and ids, their
  // coverage masks (TX + TY words per 32 wide primitives, a budget that
  // scales with the tiles: TX + TY <= tiles + 1), the per-(range, tile)
  // counts, the list lengths, the small instances' ranges.  Without the
  // wide path (wide == false) none of it is reserved and every frame takes
  // the radix sort.
  if (!wide) {
    ws->wide_max = 0;
    ws->wide_j = ws->wide_id = ws->masks = ws->wide_cnt = ws->wide_len = ws->small_ranges = nullptr;
    ws->mask_words = 0;
    ws->count_tab = ws->count_tot = ws->count_bounds = nullptr;
    ws->count_chunks = 0;
    ws->bytes = off;
    return off;
  }
  // counting placement: a [chunks][tiles] table and the per-tile totals.  The
  // table's reservation does not depend on the tile count (chunks x tiles
  // never exceeds kCountMaxSMs x kCountSmem bytes), so that a workspace
  // sized for more tiles is large enough for fewer.
  {
    uint32_t *tab = (uint32_t *)take((size_t)kCountMaxSMs * kCountSmem);
    uint32_t *tot = (uint32_t *)take(sizeof(uint32_t) * tt);
    uint32_t *bounds = (uint32_t *)take(sizeof(uint32_t) * (kCountMaxChunks + 1));
    const bool use = tiles > 0 && tiles <= kCountTiles;
    ws->count_chunks = use ? kCountMaxSMs * count_warps(tiles) : 0;
    ws->count_tab = use ? tab : nullptr;
    ws->count_tot = use ? tot : nullptr;
    ws->count_bounds = use ? bounds : nullptr;
  }
  const int64_t wmax = std::min<int64_t>((int64_t)nn, kWideMax);
  ws->wide_max = wmax;
  ws->wide_j = (uint32_t *)take(sizeof(uint32_t) * (size_t)wmax);
  ws->wide_id = (uint32_t *)take(sizeof(uint32_t) * (size_t)wmax);
  ws->mask_words = std::min(std::min(kMaskWordsMax, tt << 10), (tt + 1) * (((size_t)wmax + 31) / 32));
  ws->masks = (uint32_t *)take(sizeof(uint32_t) * ws->mask_words);
  ws->wide_cnt = (uint32_t *)take(sizeof(uint32_t) * tt * kWideRangesMax);
  ws->wide_len = (uint32_t *)take(sizeof(uint32_t) * tt);
  ws->small_ranges = (uint32_t *)take(sizeof(uint32_t) * 2 * tt);
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
// histogram helpers
// ---------------------------------------------------------------------------
// Four consecutive keys (and 0/1 validity) starting at e; elements at or past
// `end` are invalid.  `vec`: keys and valid are 16-byte aligned.
__device__ __forceinline__ void load4(const uint32_t *__restrict__ keys, const uint32_t *__restrict__ valid,
                                      int64_t e, int64_t end, bool vec, uint32_t (&k)[4], uint32_t (&v)[4]) {
  if (vec && e + 4 <= end) {
    const uint4 kk = __ldg(reinterpret_cast<const uint4 *>(keys + e));
    k[0] = kk.x; k[1] = kk.y; k[2] = kk.z; k[3] = kk.w;
    if (valid) {
      const uint4 vv = __ldg(reinterpret_cast<const uint4 *>(valid + e));
      v[0] = vv.x != 0u; v[1] = vv.y != 0u; v[2] = vv.z != 0u; v[3] = vv.w != 0u;
    } else {
      v[0] = v[1] = v[2] = v[3] = 1u;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool in = e + i < end;
      k[i] = in ? __ldg(keys + e + i) : 0u;
      v[i] = in && (!valid || __ldg(valid + e + i) != 0u) ? 1u : 0u;
    }
  }
}

// Add four keys' digits to a shared histogram, one atomic per run of equal
// digits (runs are common: a primitive's instances share tile rows).
__device__ __forceinline__ void count_runs(uint32_t *h, const uint32_t (&k)[4], const uint32_t (&v)[4],
                                           int shift, uint32_t mask) {
  uint32_t dp = (k[0] >> shift) & mask, c = v[0];
#pragma unroll
  for (int i = 1; i < 4; ++i) {
    const uint32_t d = (k[i] >> shift) & mask;
    if (d != dp) {
      if (c) atomicAdd(&h[dp], c);
      dp = d;
      c = 0u;
    }
    c += v[i];
  }
  if (c) atomicAdd(&h[dp], c);
}

// ---------------------------------------------------------------------------
// one stable radix pass: chunk histograms, their scan, and the scatter
// ---------------------------------------------------------------------------
// The keys are cut into G contiguous chunks of whole 2048-key tiles, one per
// block of a grid that fits on the device at once.  k_chunk_hist counts each
// chunk's digits (and adds them to the pass's global histogram),
// k_chunk_scan turns the counts into each chunk's first output position per
// digit (digit base from the global histogram plus the counts of earlier
// chunks), and k_scatter walks its chunk tile by tile in order, so no block
// ever waits for another.
struct PassArgs {
  const uint32_t *keys_in, *vals_in;  // vals_in null: the value is the index
  const uint32_t *valid;              // optional 0/1 filter (compacting pass)
  const int64_t *d_n;                 // input count on the device, or null: n_host
  int64_t n_host;
  const int64_t *d_abort;
  int shift, bits;
  uint32_t *ghist;                    // [256] this pass's global digit histogram, zero on entry
  uint32_t *chist;                    // [256][kMaxChunks] chunk counts -> chunk offsets
  uint32_t *ranges_init;              // optional: set to (0xffffffff, 0) for `tiles` tiles
  int tiles;
  // tile passes: *wide != 0 on the wide path.  The first pass then also sets
  // wide_ranges_init like ranges_init and zeroes wide_zero[0, wide_zero_n);
  // the last one sends the values to vals_out_wide and the ranges to
  // ranges_wide and writes no keys.
  const int64_t *wide;
  uint32_t *wide_ranges_init, *wide_zero;
  int64_t wide_zero_n;
  uint32_t *vals_out_wide, *ranges_wide;
  uint32_t *keys_out, *vals_out;      // keys_out optional
  uint32_t *ranges;                   // optional (last tile pass): [start, end) per key
  int64_t *count_out;                 // optional: number of elements written
};
constexpr int kMaxChunks = kSortBlocks;

__device__ __forceinline__ int64_t pass_n(const PassArgs &a) {
  if (a.d_abort && *a.d_abort) return 0;
  return a.d_n ? *a.d_n : a.n_host;
}

// tiles [t0, t1) of this block's chunk
__device__ __forceinline__ void chunk_tiles(int64_t n, int64_t &t0, int64_t &t1) {
  const int64_t ntiles = (n + kTileElems - 1) / kTileElems;
  const int64_t per = (ntiles + gridDim.x - 1) / gridDim.x;
  t0 = min(ntiles, (int64_t)blockIdx.x * per);
  t1 = min(ntiles, t0 + per);
}

__global__ void __launch_bounds__(kSortThreads) k_chunk_hist(PassArgs a) {
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t h[W][256];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < W * 256; k += kSortThreads) (&h[0][0])[k] = 0u;
  __syncthreads();
  const int64_t n = pass_n(a);
  if (a.ranges_init)
    for (int t = blockIdx.x * blockDim.x + tid; t < a.tiles; t += gridDim.x * blockDim.x)
      reinterpret_cast<uint2 *>(a.ranges_init)[t] = make_uint2(0xffffffffu, 0u);
  if (a.wide_ranges_init && *a.wide) {
    for (int t = blockIdx.x * blockDim.x + tid; t < a.tiles; t += gridDim.x * blockDim.x)
      reinterpret_cast<uint2 *>(a.wide_ranges_init)[t] = make_uint2(0xffffffffu, 0u);
    for (int64_t t = blockIdx.x * blockDim.x + tid; t < a.wide_zero_n; t += gridDim.x * blockDim.x)
      a.wide_zero[t] = 0u;
  }
  int64_t t0, t1;
  chunk_tiles(n, t0, t1);
  const int64_t e0 = t0 * kTileElems, e1 = min(n, t1 * kTileElems);
  const uint32_t mask = (1u << a.bits) - 1u;
  const bool vec = ((reinterpret_cast<uintptr_t>(a.keys_in) | reinterpret_cast<uintptr_t>(a.valid)) & 15u) == 0;
  for (int64_t e = e0 + tid * 4; e < e1; e += kSortThreads * 16) {
    uint32_t k[4][4], v[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) load4(a.keys_in, a.valid, e + j * kSortThreads * 4, e1, vec, k[j], v[j]);
#pragma unroll
    for (int j = 0; j < 4; ++j) count_runs(h[warp], k[j], v[j], a.shift, mask);
  }
  __syncthreads();
  if (tid < (1 << a.bits)) {
    uint32_t c = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) c += h[w][tid];
    a.chist[(size_t)tid * kMaxChunks + blockIdx.x] = c;
    if (c) atomicAdd(a.ghist + tid, c);
  }
}

// one block per digit: chunk offsets = digit base + counts of earlier chunks
__global__ void __launch_bounds__(256) k_chunk_scan(PassArgs a, int nchunks) {
  __shared__ uint32_t wsum[8];
  __shared__ uint32_t s_base;
  const int d = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  {
    uint32_t v = tid < d ? __ldg(a.ghist + tid) : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) wsum[warp] = v;
    __syncthreads();
    if (tid == 0) {
      uint32_t t = 0;
      for (int w = 0; w < 8; ++w) t += wsum[w];
      s_base = t;
    }
    __syncthreads();
  }
  uint32_t *row = a.chist + (size_t)d * kMaxChunks;
  const int per = (nchunks + 255) / 256;
  uint32_t loc[kMaxChunks / 256];
  uint32_t sum = 0;
#pragma unroll
  for (int k = 0; k < kMaxChunks / 256; ++k) {
    const int idx = tid * per + k;
    loc[k] = (k < per && idx < nchunks) ? row[idx] : 0u;
    sum += loc[k];
  }
  uint32_t incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  __syncthreads();
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint32_t run = s_base;
  for (int w = 0; w < warp; ++w) run += wsum[w];
  run += incl - sum;
#pragma unroll
  for (int k = 0; k < kMaxChunks / 256; ++k) {
    const int idx = tid * per + k;
    if (k < per && idx < nchunks) row[idx] = run;
    run += loc[k];
  }
}

// Raw tiles are prefetched one ahead into shared memory with cp.async; the
// buffer of the tile being ranked is reused to stage it in digit order.
struct alignas(16) ScatterSmem {
  uint32_t raw_k[2][kTileElems], raw_v[2][kTileElems];
  uint32_t wcnt[kSortThreads / 32][256];
  uint32_t tdig[256];
  uint32_t base[2][256];
  uint32_t scan_tmp[kSortThreads / 32];
  uint32_t tile_count;
};

__device__ __forceinline__ void cp_async16g(void *smem, const void *gmem) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Copy tile `t` (elements [t*2048, min(n, t*2048+2048))) into buffer b.
__device__ __forceinline__ void fetch_tile(const PassArgs &a, ScatterSmem &sm, int b, int64_t t, int64_t n,
                                           bool vec, int tid) {
  const int64_t e0 = t * kTileElems;
  const int cnt = (int)min((int64_t)kTileElems, n - e0);
  if (vec && cnt == kTileElems) {
#pragma unroll
    for (int k = 0; k < kTileElems / 4 / kSortThreads; ++k) {
      const int q = (k * kSortThreads + tid) * 4;
      cp_async16g(&sm.raw_k[b][q], a.keys_in + e0 + q);
      if (a.vals_in) cp_async16g(&sm.raw_v[b][q], a.vals_in + e0 + q);
    }
  } else {
    for (int q = tid; q < cnt; q += kSortThreads) {
      sm.raw_k[b][q] = __ldg(a.keys_in + e0 + q);
      if (a.vals_in) sm.raw_v[b][q] = __ldg(a.vals_in + e0 + q);
    }
  }
  cp_commit();
}

template <int BITS>
__global__ void __launch_bounds__(kSortThreads) k_scatter(PassArgs a) {
  constexpr int W = kSortThreads / 32;
  if (a.vals_out_wide && *a.wide) {
    a.vals_out = a.vals_out_wide;
    a.ranges = a.ranges_wide;
    a.keys_out = nullptr;
  }
  extern __shared__ __align__(16) unsigned char smem_raw[];
  ScatterSmem &sm = *reinterpret_cast<ScatterSmem *>(smem_raw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = pass_n(a);
  int64_t t0, t1;
  chunk_tiles(n, t0, t1);
  constexpr int R = 1 << BITS;
  constexpr uint32_t mask = (uint32_t)R - 1u;
  if (a.count_out && blockIdx.x == 0 && tid == 0) {
    uint64_t all = 0;
    for (int d = 0; d < R; ++d) all += a.ghist[d];
    *a.count_out = (a.d_abort && *a.d_abort) ? 0 : (int64_t)all;
  }
  if (t0 >= t1) return;
  const bool vec = ((reinterpret_cast<uintptr_t>(a.keys_in) | reinterpret_cast<uintptr_t>(a.vals_in)) & 15u) == 0;
  sm.base[0][tid] = tid < R ? a.chist[(size_t)tid * kMaxChunks + blockIdx.x] : 0u;
  fetch_tile(a, sm, 0, t0, n, vec, tid);
  const uint32_t lt = lanemask_lt();
  int cb = 0;
  for (int64_t t = t0; t < t1; ++t) {
    const int b = (int)((t - t0) & 1);
    cp_wait_all();
    __syncthreads();
    if (t + 1 < t1) fetch_tile(a, sm, b ^ 1, t + 1, n, vec, tid);
    const int64_t e0 = t * kTileElems;
    uint32_t key[kSortItems], val[kSortItems], dig[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const int q = warp * (32 * kSortItems) + r * 32 + lane;
      const int64_t e = e0 + q;
      dig[r] = kNoDigit;
      key[r] = sm.raw_k[b][q];
      val[r] = a.vals_in ? sm.raw_v[b][q] : (uint32_t)e;
      if (e < n && (!a.valid || __ldg(a.valid + e) != 0u)) dig[r] = (key[r] >> a.shift) & mask;
    }
#pragma unroll
    for (int k = 0; k < 256 / 32; ++k) sm.wcnt[warp][lane * 8 + k] = 0u;
    __syncwarp();
    // 1) warp-local stable ranks; the lanes holding the same digit are found
    //    with one ballot per digit bit (plus one for validity)
    uint32_t loc[kSortItems];
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t d = dig[r];
      const bool ok = d != kNoDigit;
      uint32_t peers = __ballot_sync(0xffffffffu, ok);
      if (!ok) peers = ~peers;
#pragma unroll
      for (int bb = 0; bb < BITS; ++bb) {
        const bool bit = (d >> bb) & 1u;
        const uint32_t m = __ballot_sync(0xffffffffu, bit);
        peers &= bit ? m : ~m;
      }
      const int leader = __ffs(peers) - 1;
      uint32_t old = 0;
      if (lane == leader && ok) {
        old = sm.wcnt[warp][d];
        sm.wcnt[warp][d] = old + __popc(peers);
      }
      old = __shfl_sync(0xffffffffu, old, leader);
      loc[r] = old + __popc(peers & lt);
      __syncwarp();
    }
    __syncthreads();
    // 2) per digit: prefix over warps, the tile's count, and the tile-wide
    //    exclusive scan over digits (staging order)
    uint32_t tot = 0;
#pragma unroll
    for (int w = 0; w < W; ++w) {
      const uint32_t c = sm.wcnt[w][tid];
      sm.wcnt[w][tid] = tot;
      tot += c;
    }
    uint32_t incl = tot;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) sm.scan_tmp[warp] = incl;
    __syncthreads();
    {
      uint32_t wb = 0;
#pragma unroll
      for (int w = 0; w < W; ++w)
        if (w < warp) wb += sm.scan_tmp[w];
      sm.tdig[tid] = wb + incl - tot;
      sm.base[cb ^ 1][tid] = sm.base[cb][tid] + tot;
      if (tid == 255) sm.tile_count = wb + incl;
    }
    __syncthreads();
    // 3) stage the tile in digit order over its own raw buffer
#pragma unroll
    for (int r = 0; r < kSortItems; ++r) {
      const uint32_t d = dig[r];
      if (d != kNoDigit) {
        const uint32_t lpos = sm.tdig[d] + sm.wcnt[warp][d] + loc[r];
        sm.raw_k[b][lpos] = key[r];
        sm.raw_v[b][lpos] = val[r];
      }
    }
    __syncthreads();
    // 4) write the digit runs out: consecutive threads, consecutive addresses.
    //    In the last pass of the tile sort equal keys are adjacent here, so
    //    each run's first and last element bound that tile's range.
    const uint32_t cnt = sm.tile_count;
    for (uint32_t i = tid; i < cnt; i += kSortThreads) {
      const uint32_t k = sm.raw_k[b][i];
      const uint32_t d = (k >> a.shift) & mask;
      const uint32_t pos = sm.base[cb][d] + (i - sm.tdig[d]);
      if (a.keys_out) a.keys_out[pos] = k;
      a.vals_out[pos] = sm.raw_v[b][i];
      if (a.ranges) {
        if (i == 0 || sm.raw_k[b][i - 1] != k) atomicMin(a.ranges + 2 * (size_t)k, pos);
        if (i + 1 == cnt || sm.raw_k[b][i + 1] != k) atomicMax(a.ranges + 2 * (size_t)k + 1, pos + 1);
      }
    }
    cb ^= 1;
  }
  cp_wait_all();
}

// ---------------------------------------------------------------------------
// instance offsets: exclusive scans of touched[] in depth order
// ---------------------------------------------------------------------------
// Three sums per primitive of the depth order: all its instances, the
// instances of a rectangle of at most kBigRect tiles ("small"), and 1 for a
// wider rectangle.  When wide rectangles carry most of the instances (or the
// caller asks for it) they skip the radix sort: their per-tile lists are
// written by counting (k_wide_*) and merged with the sorted small instances.

__device__ __forceinline__ void split_counts(uint32_t t, uint64_t &all, uint64_t &small, uint64_t &wide) {
  all = t;
  small = t <= kBigRect ? t : 0u;
  wide = t > kBigRect ? 1u : 0u;
}

__global__ void __launch_bounds__(kSortThreads)
    k_scan_partial(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ touched,
                   const int64_t *d_n, uint64_t *__restrict__ blk) {
  __shared__ uint64_t ws[3][kSortThreads / 32];
  const int tid = threadIdx.x;
  int64_t b0, b1;
  block_range(*d_n, b0, b1);
  uint64_t s[3] = {0, 0, 0};
  for (int64_t j = b0 + tid; j < b1; j += kSortThreads) {
    uint64_t x, y, z;
    split_counts(__ldg(touched + __ldg(ids + j)), x, y, z);
    s[0] += x; s[1] += y; s[2] += z;
  }
#pragma unroll
  for (int k = 0; k < 3; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s[k] += __shfl_down_sync(0xffffffffu, s[k], o);
    if ((tid & 31) == 0) ws[k][tid >> 5] = s[k];
  }
  __syncthreads();
  if (tid < 3) {
    uint64_t t = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) t += ws[tid][w];
    blk[(size_t)tid * kSortBlocks + blockIdx.x] = t;
  }
}

// single block: exclusive scans of the block partials; K, the path, and the
// capacity check.  counters: 1 = K, 2 = overflow, 4 = wide path, 5 = small
// instances, 6 = wide primitives B, 7 = instances the radix sort takes,
// 9 = counting placement (instead of emit and the radix tile passes).
// The wide path is taken when it is allowed (B within wide_cap) and asked
// for (wide_cfg 1), or, under wide_cfg 0, when the wide instances outnumber
// both 8x the (32 tiles, 32 wide primitives) mask visits it costs and 5x
// the small instances it merges in (measured: with small instances at 13%
// of the wide ones the mask path took 82% of the radix path's time, at 6%
// under 40%).
__global__ void __launch_bounds__(1024)
    k_scan_top(uint64_t *__restrict__ blk, int nblocks, int64_t capacity, int wide_cfg, int64_t wide_cap,
               int tiles, int count_ok, int64_t *counters, int64_t *d_count, int32_t *dev_err) {
  __shared__ uint64_t wsum[3][32];
  __shared__ int s_wide;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  uint64_t v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = tid < nblocks ? blk[(size_t)k * kSortBlocks + tid] : 0ull;
  // the three totals decide the path
  {
    uint64_t r[3] = {v[0], v[1], v[2]};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
#pragma unroll
      for (int k = 0; k < 3; ++k) r[k] += __shfl_xor_sync(0xffffffffu, r[k], o);
    if (lane == 0)
#pragma unroll
      for (int k = 0; k < 3; ++k) wsum[k][warp] = r[k];
  }
  __syncthreads();
  if (tid == 0) {
    uint64_t K = 0, Ks = 0, B = 0;
    for (int w = 0; w < 32; ++w) {
      K += wsum[0][w];
      Ks += wsum[1][w];
      B += wsum[2][w];
    }
    const uint64_t Kw = K - Ks;
    counters[1] = (int64_t)K;
    if (d_count) *d_count = (int64_t)K;
    const bool over = (int64_t)K > capacity || K > 0xffffffffull;
    counters[2] = over ? 1 : 0;
    if (over) set_error(dev_err, HGS_ERR_CAPACITY);
    const uint64_t visits = (uint64_t)tiles * ((B + 31) / 32) / 32;
    const bool fits = B > 0 && (int64_t)B <= wide_cap;
    const bool wide = fits && (wide_cfg == 1 || (wide_cfg == 0 && Kw > 8 * visits && Kw > 5 * Ks));
    counters[4] = wide ? 1 : 0;
    // counting placement (small tile grids): the whole list, or on the wide
    // path the small instances
    counters[9] = (count_ok && !over) ? 1 : 0;
    counters[5] = (int64_t)Ks;
    counters[6] = (int64_t)B;
    counters[7] = wide ? (int64_t)Ks : (int64_t)K;
    s_wide = wide ? 1 : 0;
  }
  __syncthreads();
  // exclusive scans of the rows the path reads: all instances (radix path),
  // or the small instances and the wide primitives (wide path)
  const int k0 = s_wide ? 1 : 0, k1 = s_wide ? 3 : 1;
  for (int k = k0; k < k1; ++k) {
    uint64_t incl = k == 0 ? v[0] : (k == 1 ? v[1] : v[2]);
    const uint64_t own = incl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    __syncthreads();
    if (lane == 31) wsum[0][warp] = incl;
    __syncthreads();
    uint64_t wb = 0;
    for (int w = 0; w < warp; ++w) wb += wsum[0][w];
    if (tid < nblocks) blk[(size_t)k * kSortBlocks + tid] = wb + incl - own;
  }
}

// Offsets of each primitive's instances in the radix sort's input: all its
// instances, or on the wide path only those of small rectangles, where the
// wide primitives' depth-order positions are listed too (wide_j), and every
// position j gets (number of wide primitives ahead of it, primitive id) in
// the pair array kpos.
template <bool WIDE>
__device__ __forceinline__ void scan_final_body(const uint32_t *__restrict__ ids,
                                                const uint32_t *__restrict__ touched, const int64_t *counters,
                                                const uint64_t *__restrict__ blk, uint32_t *__restrict__ offs,
                                                uint32_t *__restrict__ wide_j, uint32_t *__restrict__ kpos) {
  constexpr int NS = WIDE ? 2 : 1;
  __shared__ uint32_t wsum[NS][kSortThreads / 32];
  __shared__ uint32_t carry[NS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  int64_t b0, b1;
  block_range(counters[0], b0, b1);
  if (tid == 0) {
    carry[0] = (uint32_t)blk[(size_t)(WIDE ? 1 : 0) * kSortBlocks + blockIdx.x];
    if (WIDE) carry[NS - 1] = (uint32_t)blk[(size_t)2 * kSortBlocks + blockIdx.x];
  }
  __syncthreads();
  for (int64_t tb = b0; tb < b1; tb += kSortThreads) {
    const int64_t j = tb + tid;
    const uint32_t pid = j < b1 ? __ldg(ids + j) : 0u;
    const uint32_t t = j < b1 ? __ldg(touched + pid) : 0u;
    uint32_t v[NS];
    v[0] = WIDE ? (t <= kBigRect ? t : 0u) : t;
    if (WIDE) v[NS - 1] = t > kBigRect ? 1u : 0u;
    uint32_t incl[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      incl[k] = v[k];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, incl[k], o);
        if (lane >= o) incl[k] += u;
      }
      if (lane == 31) wsum[k][warp] = incl[k];
    }
    __syncthreads();
    uint32_t wb[NS], all[NS];
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      wb[k] = 0;
      all[k] = 0;
#pragma unroll
      for (int w = 0; w < kSortThreads / 32; ++w) {
        if (w < warp) wb[k] += wsum[k][w];
        all[k] += wsum[k][w];
      }
    }
    if (j < b1) {
      offs[j] = carry[0] + wb[0] + incl[0] - v[0];
      if (WIDE) {
        const uint32_t before = carry[NS - 1] + wb[NS - 1] + incl[NS - 1] - v[NS - 1];
        // wide primitives ahead of j in depth order, and j's primitive id
        reinterpret_cast<uint2 *>(kpos)[j] = make_uint2(before, pid);
        if (v[NS - 1]) wide_j[before] = (uint32_t)j;
      }
    }
    __syncthreads();
    if (tid == 0) {
      carry[0] += all[0];
      if (WIDE) carry[NS - 1] += all[NS - 1];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kSortThreads, 8)
    k_scan_final(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ touched,
                 const int64_t *counters, const uint64_t *__restrict__ blk,
                 uint32_t *__restrict__ offs, uint32_t *__restrict__ wide_j, uint32_t *__restrict__ kpos) {
  if (counters[2]) return;
  if (counters[4]) scan_final_body<true>(ids, touched, counters, blk, offs, wide_j, kpos);
  else scan_final_body<false>(ids, touched, counters, blk, offs, wide_j, kpos);
}

// ---------------------------------------------------------------------------
// emit (tile id, primitive id) for every tile of each binned primitive,
// primitives in depth order.  A warp takes 32 consecutive primitives, whose
// instances form one contiguous output range; lanes write that range in
// order (coalesced), each output slot finding its owner lane by a binary
// search over the lanes' exclusive prefix.  Rectangles over kBigRect tiles
// are deferred to k_emit_big; on the wide path they are skipped (the mask
// path lists them) and the value is the depth-order position, which the
// merge compares.
// ---------------------------------------------------------------------------
template <bool WIDE>
__device__ __forceinline__ void emit_body(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
                                          const uint16_t *__restrict__ rect, int64_t *counters, int TX,
                                          uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals,
                                          uint32_t *__restrict__ bigq) {
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
      if (cnt > kBigRect) {
        if (!WIDE) {
          const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(&counters[3]), 1ull);
          bigq[slot] = (uint32_t)j;
        }
        cnt = 0;
      }
      if (WIDE) p = (uint32_t)j;
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

__global__ void __launch_bounds__(256)
    k_emit(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
           const uint16_t *__restrict__ rect, int64_t *counters, int TX,
           uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals, uint32_t *__restrict__ bigq) {
  if (counters[2]) return;
  if (counters[4]) emit_body<true>(ids, offs, rect, counters, TX, tkeys, tvals, bigq);
  else emit_body<false>(ids, offs, rect, counters, TX, tkeys, tvals, bigq);
}

// one block per deferred large rectangle
__global__ void __launch_bounds__(256)
    k_emit_big(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
               const uint16_t *__restrict__ rect, const int64_t *counters, int TX,
               const uint32_t *__restrict__ bigq, uint32_t *__restrict__ tkeys,
               uint32_t *__restrict__ tvals) {
  if (counters[2] || counters[4]) return;
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
  if (counters[2] || counters[4]) return;
  const int64_t K = counters[1];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
       k += (int64_t)gridDim.x * blockDim.x)
    keys[k] = ((uint64_t)tkeys[k] << 32) | __ldg(depth_key + vals[k]);
}

// ---------------------------------------------------------------------------
// wide path: the wide rectangles' tile lists from coverage masks
// ---------------------------------------------------------------------------
// The wide primitives (rectangles over kBigRect tiles) are numbered
// k = 0..B-1 in depth order and grouped in words of 32.  For every word
// there is one 32-bit mask per tile column, saying which of its rectangles
// span that column, and one per tile row; the word's primitives that cover
// tile (tx, ty) are the bits of colmask[tx] & rowmask[ty], in depth order.
// A warp takes a strip of 32 tiles of one row (a lane per tile) and a range
// of words; walking the words in order, each lane writes its tile's
// covering primitives to the tile's list, with the tile's small instances
// (as the radix sort ordered them) slotted in by kappa, the number of wide
// primitives ahead of them in depth order.  Each lane stores groups of four
// entries as one 16-byte store.  A counting pass (popcounts of the same masks,
// a strip and up to 64 words of one range per warp) gives every (range,
// tile) its output offset within the tile's list.
// Masks are stored word-major ([word][tx], then [word][ty]), so one warp's
// column masks are 32 consecutive words and its row mask one broadcast word.
constexpr int kWB = 8;              // words per prefetched batch
constexpr int kWideWarps = 2;

struct WideArgs {
  const uint32_t *ids;       // depth order -> primitive id
  const uint32_t *wide_j;    // [B] depth-order positions of the wide primitives, ascending
  uint32_t *wide_id;         // [B] their primitive ids
  const uint32_t *kpos;      // [M][2] per depth-order position: wide primitives ahead of it, primitive id
  const uint16_t *rect;
  int64_t *counters;         // 4 = wide path, 5 = small instances, 6 = B, 8 = next write item
  int TX, TY, tiles, strips, R;
  uint32_t *masks;           // [NW][TX] column masks, then [NW][TY] row masks
  uint32_t *cnt;             // [R][tiles] wide instances per (range, tile) -> exclusive over ranges (zeroed by the first tile pass)
  uint32_t *len;             // [tiles] list lengths
  uint32_t *small;           // small instances by tile: depth-order positions -> primitive ids
  uint32_t *kappa;           // [Ks] their kappa
  const uint32_t *small_ranges;  // [tiles][2], (0xffffffff, 0) when empty
  uint32_t *vals;            // [K] output: primitive ids
  uint64_t *keys;            // optional [K] output
  const uint32_t *depth_key;
  uint32_t *ranges;          // [tiles][2] output
};

__device__ __forceinline__ int wide_words(const int64_t *counters) { return (int)((counters[6] + 31) / 32); }
// words per range: a multiple of the batch
__device__ __forceinline__ int wide_wpr(int NW, int R) { return ((NW + R - 1) / R + kWB - 1) / kWB * kWB; }

// One block per 1024 wide primitives (32 words): ids and masks.
__global__ void __launch_bounds__(256) k_wide_build(WideArgs a) {
  __shared__ uint32_t xr[32 * 33], yr[32 * 33];  // packed (lo | hi << 16) spans, a padded row per word
  if (a.counters[2] || !a.counters[4]) return;
  const int64_t B = a.counters[6];
  const int NW = wide_words(a.counters);
  const int64_t groups = (B + 1023) / 1024;
  const int tid = threadIdx.x;
  uint32_t *colT = a.masks, *rowT = a.masks + (size_t)NW * a.TX;
  for (int64_t c = blockIdx.x; c < groups; c += gridDim.x) {
    for (int i = tid; i < 1024; i += 256) {
      const int64_t k = c * 1024 + i;
      uint32_t rx = 0x0000ffffu, ry = 0x0000ffffu;  // lo 0xffff > hi 0: spans nothing
      if (k < B) {
        const uint32_t p = __ldg(a.ids + __ldg(a.wide_j + k));
        a.wide_id[k] = p;
        const uint2 r = __ldg(reinterpret_cast<const uint2 *>(a.rect) + p);
        rx = r.x;
        ry = r.y;
      }
      xr[(i >> 5) * 33 + (i & 31)] = rx;
      yr[(i >> 5) * 33 + (i & 31)] = ry;
    }
    __syncthreads();
    const int nw = (int)(NW - c * 32 < 32 ? NW - c * 32 : 32);
    for (int wl = 0; wl < nw; ++wl) {
      const size_t w = (size_t)c * 32 + wl;
      const uint32_t *xs = xr + wl * 33, *ys = yr + wl * 33;
      for (int e = tid; e < a.TX + a.TY; e += 256) {
        const bool col = e < a.TX;
        const uint32_t v = col ? (uint32_t)e : (uint32_t)(e - a.TX);
        const uint32_t *sp = col ? xs : ys;
        uint32_t m = 0;
#pragma unroll 8
        for (int b = 0; b < 32; ++b) {
          const uint32_t q = sp[b];
          m |= (uint32_t)((q & 0xffffu) <= v && v <= (q >> 16)) << b;
        }
        if (col) colT[w * a.TX + v] = m;
        else rowT[w * a.TY + v] = m;
      }
    }
    __syncthreads();
  }
}

__device__ __forceinline__ void strip_of(const WideArgs &a, int item, int &r, int &ty, int &tx) {
  const int spr = (a.TX + 31) / 32;  // strips per row
  const int st = item / a.R;
  r = item - st * a.R;
  ty = st / spr;
  tx = (st - ty * spr) * 32 + (int)(threadIdx.x & 31);
}

// Counting pass: cnt[r][t] = covering wide primitives of range r's words.
// A warp takes a strip and a chunk of up to kCountWords words of one range
// and adds its lanes' popcounts (cnt is zeroed by the first tile pass).
constexpr int kCountWords = 64;
__global__ void __launch_bounds__(256) k_wide_count(WideArgs a) {
  if (a.counters[2] || !a.counters[4]) return;
  const int NW = wide_words(a.counters), wpr = wide_wpr(NW, a.R);
  const int subs = (wpr + kCountWords - 1) / kCountWords;  // chunks per range
  const uint32_t *colT = a.masks, *rowT = a.masks + (size_t)NW * a.TX;
  const int64_t items = (int64_t)a.strips * a.R * subs;
  const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t item = blockIdx.x * (int64_t)(blockDim.x >> 5) + (threadIdx.x >> 5); item < items; item += nwarps) {
    const int sub = (int)(item % subs);
    int r, ty, tx;
    strip_of(a, (int)(item / subs), r, ty, tx);
    const int w0 = r * wpr + sub * kCountWords;
    const int w1 = min(min(NW, r * wpr + wpr), w0 + kCountWords);
    if (w0 >= w1) continue;
    const bool ok = tx < a.TX;
    uint32_t c = 0;
    for (int w = w0; w < w1; w += kWB) {
      uint32_t cm[kWB], rm[kWB];
#pragma unroll
      for (int i = 0; i < kWB; ++i) {
        const bool in = ok && w + i < w1;
        cm[i] = in ? __ldg(colT + (size_t)(w + i) * a.TX + tx) : 0u;
        rm[i] = in ? __ldg(rowT + (size_t)(w + i) * a.TY + ty) : 0u;
      }
#pragma unroll
      for (int i = 0; i < kWB; ++i) c += __popc(cm[i] & rm[i]);
    }
    if (ok && c) atomicAdd(a.cnt + (size_t)r * a.tiles + (size_t)ty * a.TX + tx, c);
  }
}

// Per tile: the ranges' counts -> exclusive offsets, and the list length
// (wide + small).  Per small instance: its kappa, and the depth-order
// position replaced by the primitive id.
__global__ void __launch_bounds__(256) k_wide_tiles(WideArgs a) {
  if (a.counters[2] || !a.counters[4]) return;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < a.tiles; t += stride) {
    uint32_t run = 0;
    for (int r = 0; r < a.R; ++r) {
      uint32_t *p = a.cnt + (size_t)r * a.tiles + t;
      const uint32_t v = *p;
      *p = run;
      run += v;
    }
    const uint2 sr = reinterpret_cast<const uint2 *>(a.small_ranges)[t];
    a.len[t] = run + (sr.x == 0xffffffffu ? 0u : sr.y - sr.x);
  }
  const int64_t Ks = a.counters[5];
  uint32_t *__restrict__ small = a.small;
  uint32_t *__restrict__ kappa = a.kappa;
  // eight independent gathers in flight per thread: element q0 + i * stride
  for (int64_t q0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q0 < Ks; q0 += stride * 8) {
    uint32_t j[8];
    uint2 kp[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) j[i] = q0 + i * stride < Ks ? small[q0 + i * stride] : 0u;
#pragma unroll
    for (int i = 0; i < 8; ++i) kp[i] = __ldg(reinterpret_cast<const uint2 *>(a.kpos) + j[i]);
#pragma unroll
    for (int i = 0; i < 8; ++i)
      if (q0 + i * stride < Ks) {
        kappa[q0 + i * stride] = kp[i].x;
        small[q0 + i * stride] = kp[i].y;
      }
  }
}

// One block: exclusive scan of the list lengths over the tiles -> ranges.
__global__ void __launch_bounds__(1024) k_wide_prefix(WideArgs a) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  if (a.counters[2] || !a.counters[4]) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int base = 0; base < a.tiles; base += 4096) {
    uint32_t v[4], s = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = base + tid * 4 + i;
      v[i] = t < a.tiles ? a.len[t] : 0u;
      s += v[i];
    }
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wb = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) wb += wsum[w];
      all += wsum[w];
    }
    uint32_t run = carry + wb + incl - s;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int t = base + tid * 4 + i;
      if (t < a.tiles) reinterpret_cast<uint2 *>(a.ranges)[t] = v[i] ? make_uint2(run, run + v[i]) : make_uint2(0u, 0u);
      run += v[i];
    }
    __syncthreads();
    if (tid == 0) carry += all;
    __syncthreads();
  }
}

// Write pass, a warp per (strip, range), taken from a counter.  Each lane
// writes its tile's entries straight to the list: single words up to a
// 16-byte boundary, then groups of four as 16-byte stores.
__global__ void __launch_bounds__(kWideWarps * 32) k_wide_write(WideArgs a) {
  __shared__ uint32_t smask[kWideWarps][kWB * 32];  // the batch's colmask & rowmask, per lane
  __shared__ uint32_t sid[kWideWarps][kWB * 32];    // the batch's wide primitive ids
  if (a.counters[2] || !a.counters[4]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t *mk = smask[warp];
  uint32_t *wid = sid[warp];
  const int NW = wide_words(a.counters), wpr = wide_wpr(NW, a.R);
  const int64_t B = a.counters[6];
  const uint32_t *colT = a.masks, *rowT = a.masks + (size_t)NW * a.TX;
  const int items = a.strips * a.R;
  unsigned long long *next = reinterpret_cast<unsigned long long *>(a.counters + 8);
  const bool vec = (reinterpret_cast<uintptr_t>(a.vals) & 15u) == 0 && !a.keys;
  constexpr uint32_t kNone = 0xffffffffu;
  for (;;) {
    unsigned long long it = 0;
    if (lane == 0) it = atomicAdd(next, 1ull);
    const int item = (int)__shfl_sync(0xffffffffu, it, 0);
    if (item >= items) break;
    int r, ty, tx;
    strip_of(a, item, r, ty, tx);
    const int w0 = r * wpr, w1 = min(NW, w0 + wpr);
    const uint32_t K0 = (uint32_t)w0 * 32u;
    const uint32_t K1 = r + 1 < a.R ? (uint32_t)(w0 + wpr) * 32u : kNone;
    const int64_t t = (int64_t)ty * a.TX + tx;
    bool ok = tx < a.TX;
    uint32_t pos = 0, end = 0, sp = 0, se = 0;
    if (ok) {
      const uint2 rg = reinterpret_cast<const uint2 *>(a.ranges)[t];
      ok = rg.x != rg.y;
      if (ok) {
        const uint2 sr = reinterpret_cast<const uint2 *>(a.small_ranges)[t];
        uint32_t lo = 0, hi = 0;
        if (sr.x != 0xffffffffu) { lo = sr.x; hi = sr.y; }
        uint32_t l = lo, h = hi;
        while (l < h) {
          const uint32_t mid = (l + h) >> 1;
          if (__ldg(a.kappa + mid) < K0) l = mid + 1; else h = mid;
        }
        sp = l;
        h = hi;
        if (K1 != kNone)
          while (l < h) {
            const uint32_t mid = (l + h) >> 1;
            if (__ldg(a.kappa + mid) < K1) l = mid + 1; else h = mid;
          }
        se = h;
        pos = rg.x + a.cnt[(size_t)r * a.tiles + t] + (sp - lo);
        end = rg.y;
      }
    }
    const uint64_t tkey = (uint64_t)t << 32;
    uint32_t rk[4], ri[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const bool in = ok && sp + i < se;
      rk[i] = in ? __ldg(a.kappa + sp + i) : kNone;
      ri[i] = in ? __ldg(a.small + sp + i) : 0u;
    }
    uint32_t nleft = ok ? se - sp : 0u;
    // output staging: q0..q3 hold np entries for the 16-byte store at pos
    uint32_t q0 = 0, q1 = 0, q2 = 0, q3 = 0, np = 0;
    auto emit = [&](uint32_t v) {
      if (!vec || (pos & 3u) != 0u) {  // up to the boundary (or no vector stores): single words
        if (pos < end) {
          a.vals[pos] = v;
          if (a.keys) a.keys[pos] = tkey | __ldg(a.depth_key + v);
        }
        ++pos;
        return;
      }
      q0 = np == 0 ? v : q0;
      q1 = np == 1 ? v : q1;
      q2 = np == 2 ? v : q2;
      q3 = np == 3 ? v : q3;
      if (++np == 4) {
        if (pos < end && end - pos >= 4u) *reinterpret_cast<uint4 *>(a.vals + pos) = make_uint4(q0, q1, q2, q3);
        pos += 4;
        np = 0;
      }
    };
    auto pop_small = [&]() -> uint32_t {
      const uint32_t v = ri[0];
      rk[0] = rk[1]; ri[0] = ri[1];
      rk[1] = rk[2]; ri[1] = ri[2];
      rk[2] = rk[3]; ri[2] = ri[3];
      --nleft;
      if (nleft >= 4) {
        rk[3] = __ldg(a.kappa + se - nleft + 3);
        ri[3] = __ldg(a.small + se - nleft + 3);
      } else {
        rk[3] = kNone;
      }
      return v;
    };
    uint32_t cmn[kWB], rmn[kWB], idn[kWB];
    auto fetch = [&](int wb) {
#pragma unroll
      for (int i = 0; i < kWB; ++i) {
        const int w = wb + i;
        const bool in = w < w1;
        cmn[i] = in && ok ? __ldg(colT + (size_t)w * a.TX + tx) : 0u;
        rmn[i] = in && ok ? __ldg(rowT + (size_t)w * a.TY + ty) : 0u;
        idn[i] = in && (int64_t)w * 32 + lane < B ? __ldg(a.wide_id + (size_t)w * 32 + lane) : 0u;
      }
    };
    if (w0 < w1) fetch(w0);
    for (int wb = w0; wb < w1; wb += kWB) {
      __syncwarp();
#pragma unroll
      for (int i = 0; i < kWB; ++i) {
        mk[i * 32 + lane] = cmn[i] & rmn[i];
        wid[i * 32 + lane] = idn[i];
      }
      __syncwarp();
      if (wb + kWB < w1) fetch(wb + kWB);
      const int nb = min(kWB, w1 - wb);
#pragma unroll 1
      for (int i = 0; i < nb; ++i) {
        const uint32_t kb = (uint32_t)(wb + i) * 32u;
        uint32_t mw = mk[i * 32 + lane];
        const uint32_t *ids = wid + i * 32;
        // the word's wide bits in order, each small instance before the
        // first wide bit it does not follow
        for (;;) {
          const uint32_t b = mw ? (uint32_t)(__ffs(mw) - 1) : 31u;
          if (rk[0] <= kb + b) {
            emit(pop_small());
          } else if (mw) {
            emit(ids[b]);
            mw &= mw - 1u;
          } else {
            break;
          }
        }
      }
    }
    while (nleft) emit(pop_small());
    // the staged tail
    for (uint32_t k = 0; k < np; ++k) {
      const uint32_t v = k == 0 ? q0 : (k == 1 ? q1 : (k == 2 ? q2 : q3));
      if (pos < end && k < end - pos) a.vals[pos + k] = v;
    }
  }
}

// ---------------------------------------------------------------------------
// counting placement (tile grids up to kCountTiles)
// ---------------------------------------------------------------------------
// The binned primitives in depth order are cut into C contiguous chunks.
//  k_count        per chunk, the instances per tile: a 2D difference array of
//                 the chunk's rectangles in shared memory, summed in place
//  k_count_scan   per tile, the exclusive prefix of those counts over the
//                 chunks (in place) and the tile's total
//  k_count_starts one block: list starts (exclusive prefix of the totals over
//                 the tiles) and the ranges
//  k_place        one warp per chunk with a counter per tile in shared memory
//                 (list start + the chunk's offset): it takes its primitives
//                 one at a time in depth order, a lane per tile of the
//                 rectangle, and writes each instance at its tile's counter.
// Within a tile, the instances are in chunk order and, inside a chunk, in
// depth order: the order of the 64-bit key with ties by id, as the radix
// sort gives it.  On the wide path the same kernels list only the
// rectangles of at most kBigRect tiles, with the depth-order position as the
// value, into the small-instance buffer the mask path merges (what the radix
// tile passes give it on large grids); the first of them also clears the mask
// path's per-(range, tile) counts.
struct CountArgs {
  const uint32_t *ids;       // depth order -> primitive id (counters[0] of them)
  const uint16_t *rect;
  const uint32_t *depth_key;
  const int64_t *counters;   // 0 = binned primitives, 2 = overflow, 4 = wide path,
                             // 7 = instances listed here, 9 = counting path
  const uint32_t *offs;      // depth order -> first instance (exclusive prefix)
  uint32_t *bounds;          // [C + 1] chunk starts in depth order
  int TX, TY, tiles, C;
  uint32_t *tab;             // [C][tiles]
  uint32_t *tot;             // [tiles]
  uint32_t *vals;            // output (radix-free path): primitive ids
  uint64_t *keys;            // optional output
  uint32_t *ranges;          // output ranges
  uint32_t *small;           // wide path: small instances by tile (depth-order positions)
  uint32_t *small_ranges;    // wide path: their ranges, (0xffffffff, 0) when empty
  uint32_t *wide_cnt;        // wide path: [kWideRangesMax][tiles], cleared here
};

__device__ __forceinline__ void count_chunk(const CountArgs &a, int c, int64_t &j0, int64_t &j1) {
  j0 = a.bounds[c];
  j1 = a.bounds[c + 1];
}

// Chunk c starts at the first depth position j whose work prefix
// F(j) = offs[j] + kCountPrimCost j reaches c / C of the total, so chunks
// with large rectangles (the primitives nearest the camera) hold fewer
// primitives and every warp of k_place gets about the same work.
__global__ void __launch_bounds__(256) k_count_bounds(CountArgs a) {
  if (!a.counters[9]) return;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > a.C) return;
  const int64_t M = a.counters[0];
  const uint64_t total = (uint64_t)a.counters[7] + kCountPrimCost * (uint64_t)M;
  // total < 2^38 and c <= kCountMaxChunks < 2^12: the product fits 64 bits
  const uint64_t target = total * (uint64_t)c / (uint64_t)a.C;
  int64_t lo = 0, hi = M;  // first j in [0, M] with F(j) >= target (F(M) = total)
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    const uint64_t f = (uint64_t)__ldg(a.offs + mid) + kCountPrimCost * (uint64_t)mid;
    if (f >= target) hi = mid; else lo = mid + 1;
  }
  a.bounds[c] = (uint32_t)lo;
}

// the rectangle of depth-order position j: (x0, x1, y0, y1); false for a wide
// rectangle on the wide path (the mask path lists it)
__device__ __forceinline__ bool count_rect(const CountArgs &a, uint32_t id, bool wide, uint32_t &x0, uint32_t &x1,
                                           uint32_t &y0, uint32_t &y1) {
  const uint2 r = __ldg(reinterpret_cast<const uint2 *>(a.rect) + id);
  x0 = r.x & 0xffffu;
  x1 = r.x >> 16;
  y0 = r.y & 0xffffu;
  y1 = r.y >> 16;
  return !wide || (x1 - x0 + 1u) * (y1 - y0 + 1u) <= kBigRect;
}

__global__ void __launch_bounds__(256) k_count(CountArgs a) {
  extern __shared__ uint32_t diff[];  // [(TY + 1) * (TX + 1)]
  if (!a.counters[9]) return;
  const bool wide = a.counters[4] != 0;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int X = a.TX + 1, Y = a.TY + 1;
  for (int k = tid; k < X * Y; k += blockDim.x) diff[k] = 0u;
  __syncthreads();
  int64_t j0, j1;
  count_chunk(a, blockIdx.x, j0, j1);
  for (int64_t j = j0 + tid; j < j1; j += blockDim.x) {
    uint32_t x0, x1, y0, y1;
    if (!count_rect(a, __ldg(a.ids + j), wide, x0, x1, y0, y1)) continue;
    ++x1;
    ++y1;
    atomicAdd(&diff[y0 * X + x0], 1u);
    atomicAdd(&diff[y0 * X + x1], 0xffffffffu);
    atomicAdd(&diff[y1 * X + x0], 0xffffffffu);
    atomicAdd(&diff[y1 * X + x1], 1u);
  }
  __syncthreads();
  // prefix along each row (a warp per row), then down each column
  for (int y = warp; y < a.TY; y += blockDim.x / 32) {
    uint32_t carry = 0;
    for (int x0 = 0; x0 < a.TX; x0 += 32) {
      const int x = x0 + lane;
      uint32_t v = x < a.TX ? diff[y * X + x] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
      }
      if (x < a.TX) diff[y * X + x] = v + carry;
      carry += __shfl_sync(0xffffffffu, v, 31);
    }
  }
  __syncthreads();
  uint32_t *row = a.tab + (size_t)blockIdx.x * a.tiles;
  for (int x = tid; x < a.TX; x += blockDim.x) {
    uint32_t acc = 0;
    for (int y = 0; y < a.TY; ++y) {
      acc += diff[y * X + x];
      row[y * a.TX + x] = acc;
    }
  }
}

// 32 tiles per block; warp w scans the chunks [w * S, (w + 1) * S), eight
// loads in flight per lane
__global__ void __launch_bounds__(256) k_count_scan(CountArgs a) {
  __shared__ uint32_t seg[8][32];
  if (!a.counters[9]) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int t = blockIdx.x * 32 + lane;
  const bool in = t < a.tiles;
  if (a.counters[4] && in)
    for (int r = warp; r < kWideRangesMax; r += 8) a.wide_cnt[(size_t)r * a.tiles + t] = 0u;
  const int S = (a.C + 7) / 8;
  const int c0 = min(a.C, warp * S), c1 = min(a.C, c0 + S);
  const uint32_t *col = a.tab + t;
  uint32_t sum = 0;
  if (in) {
    int c = c0;
    for (; c + 8 <= c1; c += 8) {
      uint32_t v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = col[(size_t)(c + k) * a.tiles];
#pragma unroll
      for (int k = 0; k < 8; ++k) sum += v[k];
    }
    for (; c < c1; ++c) sum += col[(size_t)c * a.tiles];
  }
  seg[warp][lane] = sum;
  __syncthreads();
  if (warp == 0) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint32_t v = seg[w][lane];
      seg[w][lane] = run;
      run += v;
    }
    if (in) a.tot[t] = run;
  }
  __syncthreads();
  if (!in) return;
  uint32_t run = seg[warp][lane];
  uint32_t *wcol = a.tab + t;
  int c = c0;
  for (; c + 8 <= c1; c += 8) {
    uint32_t v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = wcol[(size_t)(c + k) * a.tiles];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      wcol[(size_t)(c + k) * a.tiles] = run;
      run += v[k];
    }
  }
  for (; c < c1; ++c) {
    const uint32_t v = wcol[(size_t)c * a.tiles];
    wcol[(size_t)c * a.tiles] = run;
    run += v;
  }
}

// One block: list starts and ranges ([0, 0) for an empty tile; on the wide
// path the small ranges, (0xffffffff, 0) when empty).  On overflow it only
// clears the ranges.
__global__ void __launch_bounds__(1024) k_count_starts(CountArgs a) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (a.counters[2]) {
    for (int t = tid; t < a.tiles; t += blockDim.x) reinterpret_cast<uint2 *>(a.ranges)[t] = make_uint2(0u, 0u);
    return;
  }
  if (!a.counters[9]) return;
  const bool wide = a.counters[4] != 0;
  uint2 *out = reinterpret_cast<uint2 *>(wide ? a.small_ranges : a.ranges);
  const uint2 empty = wide ? make_uint2(0xffffffffu, 0u) : make_uint2(0u, 0u);
  if (tid == 0) carry = 0;
  __syncthreads();
  for (int t0 = 0; t0 < a.tiles; t0 += 1024) {
    const int t = t0 + tid;
    const uint32_t v = t < a.tiles ? a.tot[t] : 0u;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += u;
    }
    if (lane == 31) wsum[warp] = incl;
    __syncthreads();
    uint32_t wb = 0, all = 0;
    for (int w = 0; w < 32; ++w) {
      if (w < warp) wb += wsum[w];
      all += wsum[w];
    }
    const uint32_t start = carry + wb + incl - v;
    if (t < a.tiles) {
      a.tot[t] = start;
      out[t] = v ? make_uint2(start, start + v) : empty;
    }
    __syncthreads();
    if (tid == 0) carry += all;
    __syncthreads();
  }
}

// k_place: each warp walks its chunk 32 primitives at a time: the lanes load
// the batch's ids, rectangles and depth keys together (one round of global
// latency per 32 primitives), then the warp places the batch's primitives one
// after another in depth order, a lane per tile of the rectangle.  Tiles of
// one rectangle are distinct, so each lane's counter update is private; the
// warp barrier between primitives orders updates of a tile two of them share.
__global__ void __launch_bounds__(512) k_place(CountArgs a) {
  extern __shared__ uint32_t smem_all[];  // [warps][tiles]
  if (!a.counters[9]) return;
  const bool wide = a.counters[4] != 0;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int c = blockIdx.x * (blockDim.x >> 5) + warp;
  if (c >= a.C) return;
  uint32_t *cnt = smem_all + (size_t)warp * a.tiles;
  const uint32_t *off = a.tab + (size_t)c * a.tiles;
  for (int t = lane; t < a.tiles; t += 32) cnt[t] = __ldg(a.tot + t) + __ldg(off + t);
  __syncwarp();
  uint32_t *dst = wide ? a.small : a.vals;
  uint64_t *keys = wide ? nullptr : a.keys;
  const uint32_t TX = (uint32_t)a.TX;
  int64_t j0, j1;
  count_chunk(a, c, j0, j1);
  for (int64_t jb = j0; jb < j1; jb += 32) {
    const int64_t j = jb + lane;
    uint32_t v = 0, x0 = 0, x1 = 0, y0 = 0, y1 = 0, w = 1, n = 0, dk = 0;
    if (j < j1) {
      const uint32_t id = __ldg(a.ids + j);
      if (count_rect(a, id, wide, x0, x1, y0, y1)) {
        w = x1 - x0 + 1u;
        n = w * (y1 - y0 + 1u);
      }
      v = wide ? (uint32_t)j : id;
      if (keys && n) dk = __ldg(a.depth_key + id);
    }
    const float iw = 1.0f / (float)w;
    uint32_t todo = __ballot_sync(0xffffffffu, n != 0u);
    while (todo) {
      const int o = __ffs(todo) - 1;
      todo &= todo - 1u;
      const uint32_t on = __shfl_sync(0xffffffffu, n, o), ow = __shfl_sync(0xffffffffu, w, o);
      const uint32_t ox0 = __shfl_sync(0xffffffffu, x0, o), oy0 = __shfl_sync(0xffffffffu, y0, o);
      const uint32_t ov = __shfl_sync(0xffffffffu, v, o), odk = __shfl_sync(0xffffffffu, dk, o);
      const float oiw = __shfl_sync(0xffffffffu, iw, o);
      for (uint32_t l = lane; l < on; l += 32) {
        // l = dy * w + dx; the binary32 quotient is off by at most one
        uint32_t dy = (uint32_t)((float)l * oiw);
        uint32_t dx = l - dy * ow;
        if ((int)dx < 0) { dy -= 1; dx += ow; } else if (dx >= ow) { dy += 1; dx -= ow; }
        const uint32_t t = (oy0 + dy) * TX + ox0 + dx;
        const uint32_t pos = cnt[t];
        cnt[t] = pos + 1u;
        dst[pos] = ov;
        if (keys) keys[pos] = ((uint64_t)t << 32) | odk;
      }
      __syncwarp();
    }
  }
}

// Chunks (blocks) of the radix passes: as many scatter blocks as fit on the
// device at once, so every chunk is in flight from the start.
static int pass_grid() {
  static int cached[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cached[dev] == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_scatter<8>, kSortThreads, sizeof(ScatterSmem));
    cached[dev] = std::min(kMaxChunks, std::max(1, sms) * std::max(1, per));
  }
  return cached[dev];
}

// grids of the wide path, per device: k_wide_build and its companions, and
// k_wide_write (every block resident); the SM count
static void wide_grids(int &build, int &write, int &sms_out) {
  static int cached[64][3] = {{0}};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) dev = 0;
  if (cached[dev][0] == 0) {
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_wide_write, kWideWarps * 32, 0);
    cached[dev][0] = std::max(1, sms) * 8;
    cached[dev][1] = std::max(1, sms) * std::max(1, per);
    cached[dev][2] = std::max(1, sms);
  }
  build = cached[dev][0];
  write = cached[dev][1];
  sms_out = cached[dev][2];
}

template <int B>
static void scatter_bits(const PassArgs &p, int G, cudaStream_t s) {
  if (p.bits == B)
    k_scatter<B><<<G, kSortThreads, sizeof(ScatterSmem), s>>>(p);
  else if constexpr (B > 1)
    scatter_bits<B - 1>(p, G, s);
}

static void radix_pass(const PassArgs &p, int G, cudaStream_t s) {
  k_chunk_hist<<<G, kSortThreads, 0, s>>>(p);
  k_chunk_scan<<<1 << p.bits, 256, 0, s>>>(p, G);
  scatter_bits<8>(p, G, s);
}

int launch_bin_sort(const BinArgs &a, const BinWorkspace &ws, cudaStream_t s) {
  int64_t *ctr = ws.counters;  // 0 = n_visible, 1 = K, 2 = overflow, 3 = deferred rects
  cudaMemsetAsync(ctr, 0, ws.head_bytes, s);
  const int G = pass_grid();
  // 1) depth digits over the binned primitives (the first pass compacts)
  const uint32_t *dk_in = a.depth_key, *dv_in = nullptr;
  for (int p = 0; p < 4; ++p) {
    PassArgs w{};
    w.keys_in = dk_in;
    w.vals_in = dv_in;
    w.valid = p == 0 ? a.touched : nullptr;
    w.d_n = p == 0 ? nullptr : &ctr[0];
    w.n_host = a.n;
    w.shift = 8 * p;
    w.bits = 8;
    w.ghist = ws.hist + 256 * p;
    w.chist = ws.chist;
    w.keys_out = ws.dk[p & 1];
    w.vals_out = ws.dv[p & 1];
    w.count_out = p == 0 ? &ctr[0] : nullptr;
    radix_pass(w, G, s);
    dk_in = ws.dk[p & 1];
    dv_in = ws.dv[p & 1];
  }
  const uint32_t *ids = ws.dv[1];
  // 2) instance offsets and K (capacity check on the device)
  k_scan_partial<<<kSortBlocks, kSortThreads, 0, s>>>(ids, a.touched, &ctr[0], ws.blk);
  // the wide path takes at most wide_cap primitives: its id arrays and the
  // mask budget (TX + TY words per 32 of them)
  const int TY = a.tiles / a.TX;
  const int64_t wide_cap =
      std::min<int64_t>(ws.wide_max, (int64_t)(ws.mask_words / (size_t)(a.TX + TY)) * 32);
  const bool counting = ws.count_tab != nullptr && a.tiles <= kCountTiles;
  k_scan_top<<<1, 1024, 0, s>>>(ws.blk, kSortBlocks, a.capacity, a.wide_cfg, wide_cap, a.tiles, counting ? 1 : 0,
                                ctr, a.d_count, a.dev_err);
  // dk[0] and dv[0] (contiguous) are free once the depth sort is done: dk[0]
  // holds the deferred queue, or, on the wide path, dk[0]..dv[0] the kpos pairs
  k_scan_final<<<kSortBlocks, kSortThreads, 0, s>>>(ids, a.touched, ctr, ws.blk, ws.offs, ws.wide_j, ws.dk[0]);
  const int passes = (a.tile_bits + 7) / 8;
  uint32_t *small = ws.tk[passes & 1], *kappa = ws.tk[(passes + 1) & 1];
  if (counting) {
    // 3) small tile grids: counting placement (each kernel returns at once
    //    unless counters[9], i.e. on overflow)
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int W = count_warps(a.tiles);
    small = ws.tk[0];
    kappa = ws.tk[1];
    CountArgs ca{};
    ca.ids = ids;
    ca.rect = a.rect;
    ca.depth_key = a.depth_key;
    ca.counters = ctr;
    ca.TX = a.TX;
    ca.TY = TY;
    ca.tiles = a.tiles;
    ca.C = std::min(ws.count_chunks, std::max(1, std::min(sms, kCountMaxSMs)) * W);
    ca.tab = ws.count_tab;
    ca.tot = ws.count_tot;
    ca.offs = ws.offs;
    ca.bounds = ws.count_bounds;
    ca.vals = a.vals;
    ca.keys = a.keys;
    ca.ranges = a.ranges;
    ca.small = small;
    ca.small_ranges = ws.small_ranges;
    ca.wide_cnt = ws.wide_cnt;
    const size_t dsm = sizeof(uint32_t) * (size_t)(a.TX + 1) * (TY + 1);
    const size_t psm = sizeof(uint32_t) * (size_t)W * a.tiles;
    static bool once = (cudaFuncSetAttribute(k_count, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024),
                        cudaFuncSetAttribute(k_place, cudaFuncAttributeMaxDynamicSharedMemorySize, kCountSmem),
                        true);
    (void)once;
    k_count_bounds<<<(ca.C + 256) / 256, 256, 0, s>>>(ca);
    k_count<<<ca.C, 256, dsm, s>>>(ca);
    k_count_scan<<<(a.tiles + 31) / 32, 256, 0, s>>>(ca);
    k_count_starts<<<1, 1024, 0, s>>>(ca);
    k_place<<<(ca.C + W - 1) / W, 32 * W, psm, s>>>(ca);
  } else {
    // 3) emit, then the tile digits, split evenly over the passes (13 bits ->
    //    7 + 6): fewer buckets per pass give longer runs in the write-out
    const int per_pass = (a.tile_bits + passes - 1) / passes;
    uint32_t *vbuf[2];
    vbuf[0] = (passes % 2 == 0) ? a.vals : ws.tv;
    vbuf[1] = (passes % 2 == 0) ? ws.tv : a.vals;
    k_emit<<<kSortBlocks, 256, 0, s>>>(ids, ws.offs, a.rect, ctr, a.TX, ws.tk[0], vbuf[0], ws.dk[0]);
    k_emit_big<<<kSortBlocks, 256, 0, s>>>(ids, ws.offs, a.rect, ctr, a.TX, ws.dk[0], ws.tk[0], vbuf[0]);
    int tshift[4], tbits[4];
    for (int p = 0; p < passes; ++p) {
      tshift[p] = per_pass * p;
      tbits[p] = std::min(per_pass, a.tile_bits - per_pass * p);
    }
    for (int p = 0; p < passes; ++p) {
      const bool last = p + 1 == passes;
      PassArgs w{};
      w.keys_in = ws.tk[p & 1];
      w.vals_in = vbuf[p & 1];
      w.d_n = &ctr[7];
      w.d_abort = &ctr[2];
      w.shift = tshift[p];
      w.bits = tbits[p];
      w.ghist = ws.hist + 256 * (4 + p);
      w.chist = ws.chist;
      w.ranges_init = p == 0 ? a.ranges : nullptr;
      w.tiles = a.tiles;
      w.keys_out = (!last || a.keys) ? ws.tk[(p + 1) & 1] : nullptr;
      w.vals_out = vbuf[(p + 1) & 1];
      w.ranges = last ? a.ranges : nullptr;
      w.wide = &ctr[4];
      if (p == 0) {
        w.wide_ranges_init = ws.small_ranges;
        w.wide_zero = ws.wide_cnt;
        w.wide_zero_n = (int64_t)kWideRangesMax * a.tiles;
      }
      if (last) {
        // wide path: the sorted small instances go to the key buffer this pass
        // would otherwise fill, their ranges to small_ranges
        w.vals_out_wide = ws.tk[(p + 1) & 1];
        w.ranges_wide = ws.small_ranges;
      }
      radix_pass(w, G, s);
    }
    k_ranges_fix<<<(a.tiles + 255) / 256, 256, 0, s>>>(a.ranges, a.tiles);
    if (a.keys) k_keys64<<<kSortBlocks, 256, 0, s>>>(ws.tk[passes & 1], a.vals, a.depth_key, ctr, a.keys);
  }
  // 4) wide path (every kernel returns at once when the frame does not take
  //    it).  The small instances, sorted by tile, are in `small` (from the
  //    counting placement or the radix tile passes); `kappa` is free and
  //    takes their kappa.
  {
    int gb = 1, gw = 1, sms = 1;
    wide_grids(gb, gw, sms);
    WideArgs wa{};
    wa.ids = ids;
    wa.wide_j = ws.wide_j;
    wa.wide_id = ws.wide_id;
    wa.kpos = ws.dk[0];
    wa.rect = a.rect;
    wa.counters = ctr;
    wa.TX = a.TX;
    wa.TY = TY;
    wa.tiles = a.tiles;
    wa.strips = TY * ((a.TX + 31) / 32);
    // about four (strip, range) items per resident warp of k_wide_write
    wa.R = std::max(1, std::min(kWideRangesMax, (gw * kWideWarps * 4 + wa.strips - 1) / wa.strips));
    wa.masks = ws.masks;
    wa.cnt = ws.wide_cnt;
    wa.len = ws.wide_len;
    wa.small = small;
    wa.kappa = kappa;
    wa.small_ranges = ws.small_ranges;
    wa.vals = a.vals;
    wa.keys = a.keys;
    wa.depth_key = a.depth_key;
    wa.ranges = a.ranges;
    k_wide_build<<<gb, 256, 0, s>>>(wa);
    k_wide_count<<<gb, 256, 0, s>>>(wa);
    k_wide_tiles<<<gb, 256, 0, s>>>(wa);
    k_wide_prefix<<<1, 1024, 0, s>>>(wa);
    k_wide_write<<<gw, kWideWarps * 32, 0, s>>>(wa);
  }
  return 0;
}

}  // namespace hgs
