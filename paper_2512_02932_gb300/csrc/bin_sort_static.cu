// bin_sort_static.cu -- hgs_bin_sort_static: the binning step with its
// scratch memory in a fixed, library-owned device array instead of a
// caller-supplied workspace.
//
// Who needs it: callers that cannot allocate device memory when they bin a
// frame -- for example a renderer embedded in a host application that owns
// the device allocator and forbids foreign cudaMalloc calls, or a real-time
// loop that must not call cudaMalloc/cudaFree because those calls can
// synchronise the whole device and stall other streams.  They still pass the
// per-primitive inputs and the output lists; only the sort's scratch comes
// from here.
//
// The array is a file-scope __device__ object, so every GPU that loads this
// library reserves kStaticScratchBytes for it until the process exits.  Host
// code never uses the array's name as an address: the first call on each
// device looks its device address up with cudaGetSymbolAddress (with that
// device current) and keeps it for later calls.  Every call shares the one
// array and it keeps whatever the previous call left in it; the binning
// kernels clear the parts that must start at zero themselves.  Two calls
// whose work overlaps on the GPU (for example on two streams) race on the
// array: serialise them.
#include <mutex>

#include "common.cuh"
#include "kernels.cuh"

namespace {

constexpr size_t kStaticScratchBytes = HGS_BIN_SORT_STATIC_BYTES;  // 64 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_bin_scratch[kStaticScratchBytes];

std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of g_bin_scratch on the current device (set-up once per
// device).  Returns nullptr if the lookup fails.
void *scratch_on_current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bin_scratch) != cudaSuccess || p == nullptr) return nullptr;
    g_scratch_ptr[dev] = p;
  }
  return g_scratch_ptr[dev];
}

}  // namespace

extern "C" int hgs_bin_sort_static(int64_t n, const hgs_projected *proj, const hgs_camera *cam,
                                   const hgs_config *cfg, int64_t capacity, hgs_binning *out,
                                   int32_t *dev_err, hgs_stream_t stream) {
  if (n < 0 || n >= (int64_t(1) << 31) || capacity < 0 || capacity > hgs::kMaxCapacity || !out || !out->ranges ||
      !out->d_count)
    return HGS_ERR_INVALID_ARG;
  if (capacity > 0 && !out->vals) return HGS_ERR_INVALID_ARG;
  if (!cam || !cfg || !proj) return HGS_ERR_INVALID_ARG;
  if (cfg->tile != hgs::kTile) return HGS_ERR_UNSUPPORTED;
  if (cam->width <= 0 || cam->height <= 0 || cam->width > 16384 || cam->height > 16384)
    return HGS_ERR_INVALID_ARG;
  if (n > 0 && (!proj->depth_key || !proj->touched || !proj->rect || !proj->tileset)) return HGS_ERR_INVALID_ARG;
  if (n > 0 && ((reinterpret_cast<uintptr_t>(proj->tileset) & 15u) || (reinterpret_cast<uintptr_t>(proj->rect) & 7u)))
    return HGS_ERR_INVALID_ARG;
  const int TX = (cam->width + hgs::kTile - 1) / hgs::kTile;
  const int TY = (cam->height + hgs::kTile - 1) / hgs::kTile;
  hgs::BinWorkspace probe;
  if (hgs::bin_layout(nullptr, n, capacity, &probe) > kStaticScratchBytes)
    return HGS_ERR_INVALID_ARG;
  void *scratch = scratch_on_current_device();
  if (!scratch) return HGS_ERR_CUDA;
  hgs::BinWorkspace w;
  hgs::bin_layout(scratch, n, capacity, &w);
  int tile_bits = 1;
  while ((1 << tile_bits) < TX * TY) ++tile_bits;
  hgs::BinArgs a;
  a.n = n;
  a.capacity = capacity;
  a.tiles = TX * TY;
  a.tile_bits = tile_bits;
  a.TX = TX;
  a.depth_key = proj->depth_key;
  a.touched = proj->touched;
  a.rect = proj->rect;
  a.tileset = proj->tileset;
  a.vals = out->vals;
  a.keys = out->keys;
  a.ranges = out->ranges;
  a.d_count = out->d_count;
  a.dev_err = dev_err;
  hgs::launch_bin_sort(a, w, reinterpret_cast<cudaStream_t>(stream));
  return cudaGetLastError() == cudaSuccess ? HGS_OK : HGS_ERR_CUDA;
}

