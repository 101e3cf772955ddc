// binning.cu -- tile binning of the hybrid rasterizer: duplicate every binned
// primitive into the tiles of its tile set and order the instances by the
// 64-bit key tile_id << 32 | depth_key (ties by primitive id).
//
// A primitive's tile set is, row by row of its rectangle, the tile columns
// its footprint ellipse reaches (row_span, common.cuh): a needle lists the
// tiles along its length instead of its whole bounding rectangle.
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
// A warp emits primitives whose set spans at most kEmitRows tile rows and
// kBigSet tiles; larger ones are deferred to a block each (k_emit_big).
constexpr int kEmitRows = 8;
constexpr uint32_t kBigSet = 256;

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
  // the small head (counters, histograms) is cleared with one memset
  ws->head_bytes = sizeof(int64_t) * 16 + sizeof(uint32_t) * 8 * 256;
  ws->counters = (int64_t *)take(ws->head_bytes);
  ws->hist = b ? reinterpret_cast<uint32_t *>(ws->counters + 16) : nullptr;
  ws->blk = (uint64_t *)take(sizeof(uint64_t) * kSortBlocks);
  for (int k = 0; k < 2; ++k) {
    ws->dk[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
    ws->dv[k] = (uint32_t *)take(sizeof(uint32_t) * nn);
  }
  ws->offs = (uint32_t *)take(sizeof(uint32_t) * nn);
  ws->tk[0] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tk[1] = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->tv = (uint32_t *)take(sizeof(uint32_t) * cc);
  ws->chist = (uint32_t *)take(sizeof(uint32_t) * 256 * kSortBlocks);
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
  grid_dep();
  constexpr int W = kSortThreads / 32;
  __shared__ uint32_t h[W][256];
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int k = tid; k < W * 256; k += kSortThreads) (&h[0][0])[k] = 0u;
  __syncthreads();
  const int64_t n = pass_n(a);
  if (a.ranges_init)
    for (int t = blockIdx.x * blockDim.x + tid; t < a.tiles; t += gridDim.x * blockDim.x)
      reinterpret_cast<uint2 *>(a.ranges_init)[t] = make_uint2(0xffffffffu, 0u);
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
  grid_dep();
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
  grid_dep();
  constexpr int W = kSortThreads / 32;
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
// instance offsets: exclusive scan of touched[] in depth order
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kSortThreads)
    k_scan_partial(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ touched,
                   const int64_t *d_n, uint64_t *__restrict__ blk) {
  grid_dep();
  __shared__ uint64_t ws[kSortThreads / 32];
  const int tid = threadIdx.x;
  int64_t b0, b1;
  block_range(*d_n, b0, b1);
  uint64_t sum = 0;
  for (int64_t j = b0 + tid; j < b1; j += kSortThreads) sum += __ldg(touched + __ldg(ids + j));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) sum += __shfl_down_sync(0xffffffffu, sum, o);
  if ((tid & 31) == 0) ws[tid >> 5] = sum;
  __syncthreads();
  if (tid == 0) {
    uint64_t t = 0;
    for (int w = 0; w < kSortThreads / 32; ++w) t += ws[w];
    blk[blockIdx.x] = t;
  }
}

// single block: exclusive scan of the block partials, K and the capacity
// check.  counters: 1 = K, 2 = overflow.
__global__ void __launch_bounds__(1024)
    k_scan_top(uint64_t *__restrict__ blk, int nblocks, int64_t capacity, int64_t *counters, int64_t *d_count,
               int32_t *dev_err) {
  grid_dep();
  __shared__ uint64_t wsum[32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const uint64_t own = tid < nblocks ? blk[tid] : 0ull;
  uint64_t incl = own;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint64_t u = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += u;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  uint64_t wb = 0, K = 0;
  for (int w = 0; w < 32; ++w) {
    if (w < warp) wb += wsum[w];
    K += wsum[w];
  }
  if (tid < nblocks) blk[tid] = wb + incl - own;
  if (tid == 0) {
    counters[1] = (int64_t)K;
    if (d_count) *d_count = (int64_t)K;
    const bool over = (int64_t)K > capacity || K > 0xffffffffull;
    counters[2] = over ? 1 : 0;
    if (over) set_error(dev_err, HGS_ERR_CAPACITY);
  }
}

// offs[j]: the first instance of depth-order position j (K < 2^32 here)
__global__ void __launch_bounds__(kSortThreads, 8)
    k_scan_final(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ touched,
                 const int64_t *counters, const uint64_t *__restrict__ blk, uint32_t *__restrict__ offs) {
  grid_dep();
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
    const uint32_t v = j < b1 ? __ldg(touched + __ldg(ids + j)) : 0u;
    uint32_t incl = v;
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
    if (j < b1) offs[j] = carry + wb + incl - v;
    __syncthreads();
    if (tid == 0) carry += all;
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// emit (tile id, primitive id) for every tile of each binned primitive's set,
// primitives in depth order.  A warp takes 32 consecutive primitives, whose
// instances form one contiguous output range; lanes write that range in
// order (coalesced), each output slot finding its owner lane by a binary
// search over the lanes' exclusive prefix and its tile row in the owner's
// row table (first column and first instance of each row, in shared
// memory).  Sets over kBigSet tiles or kEmitRows rows are deferred to
// k_emit_big, a warp each.
// ---------------------------------------------------------------------------
__device__ __forceinline__ TileSet load_tileset(const float *tileset, uint32_t p) {
  const float4 *t = reinterpret_cast<const float4 *>(tileset) + 3 * (size_t)p;
  TileSet s;
  s.t0 = __ldg(t);
  s.t1 = __ldg(t + 1);
  s.t2 = __ldg(t + 2);
  return s;
}

__global__ void __launch_bounds__(256)
    k_emit(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs, const uint16_t *__restrict__ rect,
           const uint32_t *__restrict__ touched, const float *__restrict__ tileset, int64_t *counters, int TX,
           uint32_t *__restrict__ tkeys, uint32_t *__restrict__ tvals, uint32_t *__restrict__ bigq) {
  grid_dep();
  // per warp and lane: (first column | first instance << 16) of each row of
  // the lane's primitive, rows past its last 0xffffffff; the lanes' tile sets
  __shared__ uint32_t rows[256 / 32][32][kEmitRows];
  __shared__ TileSet sets[256 / 32][32];
  if (counters[2]) return;
  const int64_t M = counters[0];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t(&tab)[32][kEmitRows] = rows[warp];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t jb = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); jb < M; jb += stride) {
    const int64_t j = jb + lane;
    uint32_t p = 0, off = 0, ty0 = 0, cnt = 0;
    int tx0 = 0, tx1 = -1, nrows = 0;
    if (j < M) {
      p = __ldg(ids + j);
      off = __ldg(offs + j);
      cnt = __ldg(touched + p);
      const uint2 r = __ldg(reinterpret_cast<const uint2 *>(rect) + p);
      tx0 = (int)(r.x & 0xffffu);
      tx1 = (int)(r.x >> 16);
      ty0 = r.y & 0xffffu;
      nrows = (int)(r.y >> 16) - (int)ty0 + 1;
      if (cnt > kBigSet || nrows > kEmitRows) {
        const unsigned long long slot = atomicAdd(reinterpret_cast<unsigned long long *>(&counters[3]), 1ull);
        bigq[slot] = (uint32_t)j;
        cnt = 0;
        nrows = 0;
      } else {
        sets[warp][lane] = load_tileset(tileset, p);
      }
    }
#pragma unroll
    for (int q = 0; q < kEmitRows; ++q) tab[lane][q] = 0xffffffffu;
    // the row spans, the (lane, row) pairs spread over the lanes: the row
    // table first holds (first column | width << 16)
    {
      uint32_t incl = (uint32_t)nrows;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint32_t rrel = incl - (uint32_t)nrows;
      const uint32_t rtotal = __shfl_sync(0xffffffffu, incl, 31);
      __syncwarp();
      for (uint32_t kb = 0; kb < rtotal; kb += 32) {  // at most 8 rounds (8 rows per lane)
        const uint32_t k = kb + lane;
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t pr = __shfl_sync(0xffffffffu, rrel, lo + step);
          if (pr <= k) lo += step;
        }
        const uint32_t orel = __shfl_sync(0xffffffffu, rrel, lo);
        const int otx0 = __shfl_sync(0xffffffffu, tx0, lo), otx1 = __shfl_sync(0xffffffffu, tx1, lo);
        const uint32_t oty0 = __shfl_sync(0xffffffffu, ty0, lo);
        if (k < rtotal) {
          const uint32_t q = k - orel;
          int c0 = 0, c1 = -1;
          row_span(sets[warp][lo], (int)(oty0 + q), otx0, otx1, &c0, &c1);
          tab[lo][q] = (uint32_t)c0 | ((uint32_t)(c1 - c0 + 1) << 16);
        }
      }
      __syncwarp();
      // widths -> first instances, each lane over its own rows
      uint32_t first = 0;
#pragma unroll
      for (int q = 0; q < kEmitRows; ++q) {
        const uint32_t e = tab[lane][q];
        if (q < nrows) {
          tab[lane][q] = (e & 0xffffu) | (first << 16);
          first += e >> 16;
        }
      }
    }
    __syncwarp();
    // exclusive prefix of the counts within the warp
    uint32_t incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    const uint32_t rel = j < M ? incl - cnt : 0xffffffffu;
    const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
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
      const uint32_t own_ty0 = __shfl_sync(0xffffffffu, ty0, lo);
      const uint32_t own_p = __shfl_sync(0xffffffffu, p, lo);
      if (k < total) {
        const uint32_t l = k - own_rel;
        // the row holding instance l: the last row whose first instance is
        // <= l (an empty row shares its successor's first instance)
        uint32_t e = tab[lo][0];
        int rr = 0;
#pragma unroll
        for (int q = 1; q < kEmitRows; ++q) {
          const uint32_t f = tab[lo][q];
          if ((f >> 16) <= l) {
            e = f;
            rr = q;
          }
        }
        tkeys[own_off + l] = (own_ty0 + (uint32_t)rr) * (uint32_t)TX + (e & 0xffffu) + (l - (e >> 16));
        tvals[own_off + l] = own_p;
      }
    }
    __syncwarp();
  }
}

// One warp per deferred primitive: its tile rows 32 at a time (a lane per
// row: its span, then a warp scan of the widths), and each such chunk's
// instances written in order, a lane per instance finding its row by a
// binary search over the chunk's first instances.
__global__ void __launch_bounds__(256)
    k_emit_big(const uint32_t *__restrict__ ids, const uint32_t *__restrict__ offs,
               const uint16_t *__restrict__ rect, const float *__restrict__ tileset, int64_t *counters,
               int TX, const uint32_t *__restrict__ bigq, uint32_t *__restrict__ tkeys,
               uint32_t *__restrict__ tvals) {
  grid_dep();
  if (counters[2]) return;
  const int lane = threadIdx.x & 31;
  const int64_t nbig = counters[3];
  // Warps take the deferred primitives a batch at a time from a counter
  // (their sizes run from a few rows to the whole frame, so a fixed stride
  // left the busiest warp with 2.4 times the mean work); a batch is sized
  // for about four per warp, 1 to 8 primitives.  Within a batch, the next
  // primitive's queue entry and id are loaded, and its rectangle, set and
  // offset prefetched into L2, while the current one is written.
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int64_t kBigBatch = max((int64_t)1, min((int64_t)8, nbig / (4 * nw)));
  unsigned long long *next = reinterpret_cast<unsigned long long *>(&counters[4]);
  int64_t b = 0, bend = 0;
  uint32_t jn = 0, pn = 0;
  while (true) {
    if (b >= bend) {
      unsigned long long t = 0;
      if (lane == 0) t = atomicAdd(next, (unsigned long long)kBigBatch);
      t = __shfl_sync(0xffffffffu, t, 0);
      if ((int64_t)t >= nbig) break;
      b = (int64_t)t;
      bend = min(nbig, b + kBigBatch);
      jn = bigq[b];
      pn = __ldg(ids + jn);
    }
    const uint32_t j = jn, p = pn;
    const bool more = b + 1 < bend;
    if (more) {
      jn = bigq[b + 1];
      pn = __ldg(ids + jn);
    }
    ++b;
    uint32_t base = __ldg(offs + j);
    const uint2 r = __ldg(reinterpret_cast<const uint2 *>(rect) + p);
    const int tx0 = (int)(r.x & 0xffffu), tx1 = (int)(r.x >> 16);
    const int ty0 = (int)(r.y & 0xffffu);
    const int nrows = (int)(r.y >> 16) - ty0 + 1;
    const TileSet ts = load_tileset(tileset, p);
    if (more && lane < 3) {  // hints only
      const void *h = lane == 0   ? static_cast<const void *>(reinterpret_cast<const uint2 *>(rect) + pn)
                      : lane == 1 ? static_cast<const void *>(reinterpret_cast<const float4 *>(tileset) + 3 * (size_t)pn)
                                  : static_cast<const void *>(offs + jn);
      asm volatile("prefetch.global.L2 [%0];" ::"l"(h));
    }
    for (int r0 = 0; r0 < nrows; r0 += 32) {
      const int row = r0 + lane;
      uint32_t c0 = 0, w = 0;
      if (row < nrows) {
        int a, e;
        if (row_span(ts, ty0 + row, tx0, tx1, &a, &e)) {
          c0 = (uint32_t)a;
          w = (uint32_t)(e - a + 1);
        }
      }
      uint32_t incl = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const uint32_t first = incl - w;
      const uint32_t tot = __shfl_sync(0xffffffffu, incl, 31);
      for (uint32_t lb = 0; lb < tot; lb += 32) {  // warp-uniform trip count
        const uint32_t l = lb + lane;
        // the chunk row holding instance l: the last lane whose first
        // instance is <= l (an empty row shares its successor's first)
        int lo = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
          const uint32_t f = __shfl_sync(0xffffffffu, first, lo + step);
          if (f <= l) lo += step;
        }
        const uint32_t fk = __shfl_sync(0xffffffffu, first, lo), ck = __shfl_sync(0xffffffffu, c0, lo);
        if (l < tot) {
          tkeys[base + l] = (uint32_t)(ty0 + r0 + lo) * (uint32_t)TX + ck + (l - fk);
          tvals[base + l] = p;
        }
      }
      base += tot;
    }
  }
}

// tiles no instance reached keep their initial (0xffffffff, 0): make them [0, 0)
__global__ void __launch_bounds__(256) k_ranges_fix(uint32_t *__restrict__ ranges, int tiles) {
  grid_dep();
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < tiles; t += gridDim.x * blockDim.x) {
    uint2 *r = reinterpret_cast<uint2 *>(ranges) + t;
    if (r->x == 0xffffffffu) *r = make_uint2(0u, 0u);
  }
}

__global__ void __launch_bounds__(256)
    k_keys64(const uint32_t *__restrict__ tkeys, const uint32_t *__restrict__ vals,
             const uint32_t *__restrict__ depth_key, const int64_t *counters, uint64_t *__restrict__ keys) {
  grid_dep();
  if (counters[2]) return;
  const int64_t K = counters[1];
  for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < K;
       k += (int64_t)gridDim.x * blockDim.x)
    keys[k] = ((uint64_t)tkeys[k] << 32) | __ldg(depth_key + vals[k]);
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

template <int B>
static void scatter_bits(const PassArgs &p, int G, cudaStream_t s) {
  if (p.bits == B)
    pdl_launch(k_scatter<B>, G, kSortThreads, sizeof(ScatterSmem), s, p);
  else if constexpr (B > 1)
    scatter_bits<B - 1>(p, G, s);
}

// Every kernel of the sort after the first is launched with programmatic
// dependent launch (grid_dep() at its top): its blocks are already resident
// when its predecessor finishes.  The first follows a memset and is launched
// plainly.
static void radix_pass(const PassArgs &p, int G, cudaStream_t s, bool first = false) {
  if (first)
    k_chunk_hist<<<G, kSortThreads, 0, s>>>(p);
  else
    pdl_launch(k_chunk_hist, G, kSortThreads, 0, s, p);
  pdl_launch(k_chunk_scan, 1 << p.bits, 256, 0, s, p, G);
  scatter_bits<8>(p, G, s);
}

int launch_bin_sort(const BinArgs &a, const BinWorkspace &ws, cudaStream_t s) {
  int64_t *ctr = ws.counters;  // 0 = binned primitives, 1 = K, 2 = overflow, 3 = deferred primitives,
                               // 4 = deferred primitives handed out
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
    radix_pass(w, G, s, p == 0);
    dk_in = ws.dk[p & 1];
    dv_in = ws.dv[p & 1];
  }
  const uint32_t *ids = ws.dv[1];
  // 2) instance offsets and K (capacity check on the device)
  pdl_launch(k_scan_partial, kSortBlocks, kSortThreads, 0, s, ids, a.touched, &ctr[0], ws.blk);
  pdl_launch(k_scan_top, 1, 1024, 0, s, ws.blk, kSortBlocks, a.capacity, ctr, a.d_count, a.dev_err);
  pdl_launch(k_scan_final, kSortBlocks, kSortThreads, 0, s, ids, a.touched, ctr, ws.blk, ws.offs);
  // 3) emit (dk[0], free once the depth sort is done, holds the deferred
  //    queue), then the tile digits, split as evenly as the passes allow
  //    (13 bits -> 6 + 7): fewer buckets per pass give longer runs in the
  //    write-out
  const int passes = (a.tile_bits + 7) / 8;
  const int per_pass = (a.tile_bits + passes - 1) / passes;
  uint32_t *vbuf[2];
  vbuf[0] = (passes % 2 == 0) ? a.vals : ws.tv;
  vbuf[1] = (passes % 2 == 0) ? ws.tv : a.vals;
  pdl_launch(k_emit, kSortBlocks, 256, 0, s, ids, ws.offs, a.rect, a.touched, a.tileset, ctr, a.TX, ws.tk[0],
             vbuf[0], ws.dk[0]);
  pdl_launch(k_emit_big, kSortBlocks, 256, 0, s, ids, ws.offs, a.rect, a.tileset, ctr, a.TX, ws.dk[0], ws.tk[0],
             vbuf[0]);
  for (int p = 0; p < passes; ++p) {
    const bool last = p + 1 == passes;
    PassArgs w{};
    w.keys_in = ws.tk[p & 1];
    w.vals_in = vbuf[p & 1];
    w.d_n = &ctr[1];
    w.d_abort = &ctr[2];
    // the smaller digit first (13 bits: 6 + 7; 15 bits: 7 + 8): the second
    // pass then ranks the wider digit over keys already grouped by the
    // first, which measured faster at both sizes (stress binning 9.6 ->
    // 8.1 ms)
    const int first_bits = a.tile_bits - per_pass * (passes - 1);
    w.shift = p == 0 ? 0 : first_bits + per_pass * (p - 1);
    w.bits = p == 0 ? first_bits : per_pass;
    w.ghist = ws.hist + 256 * (4 + p);
    w.chist = ws.chist;
    w.ranges_init = p == 0 ? a.ranges : nullptr;
    w.tiles = a.tiles;
    w.keys_out = (!last || a.keys) ? ws.tk[(p + 1) & 1] : nullptr;
    w.vals_out = vbuf[(p + 1) & 1];
    w.ranges = last ? a.ranges : nullptr;
    radix_pass(w, G, s);
  }
  pdl_launch(k_ranges_fix, (a.tiles + 255) / 256, 256, 0, s, a.ranges, a.tiles);
  if (a.keys) pdl_launch(k_keys64, kSortBlocks, 256, 0, s, ws.tk[passes & 1], a.vals, a.depth_key, ctr, a.keys);
  return 0;
}

}  // namespace hgs
