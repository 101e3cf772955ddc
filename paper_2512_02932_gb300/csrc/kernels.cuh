// kernels.cuh -- kernel argument blocks and launchers (internal to libhgs).
#pragma once
#include "common.cuh"

namespace hgs {

struct PrepArgs {
  const float *means, *log_scales, *quats, *logits, *sh;
  const uint8_t *types;
  int64_t n;
  CamK cam;
  CfgK cfg;
  // outputs (forward) / inputs (backward)
  float *rec;
  uint32_t *depth_key;
  uint16_t *rect;
  uint32_t *touched;
  float *tileset;  // [n][12]: TileSet of each binned primitive
};

struct PrepGradArgs {
  const float *rec_grad;  // [n,16]
  float *means, *log_scales, *quats, *logits, *sh;
};

int launch_preprocess_fwd(const PrepArgs &a, int deg, cudaStream_t s);

constexpr int kMaxBatch = 16;

struct BatchPrepArgs {
  int nreq;
  PrepArgs req[kMaxBatch];  // outputs already offset to the request's rows
  int deg[kMaxBatch];
  int row_off[kMaxBatch];   // first tile row of the request in the stacked grid
  int64_t base[kMaxBatch + 1];
};
int launch_preprocess_batch(const BatchPrepArgs &b, cudaStream_t s);
int launch_preprocess_bwd(const PrepArgs &a, const PrepGradArgs &g, int deg, cudaStream_t s);

// Frequency-decoupled optimisation (Algorithm 1): three record gradients in
// (appearance, low-frequency, high-frequency losses), one projected sum out.
struct PrepGradFdoArgs {
  const float *rec_color, *rec_low, *rec_high;  // [n,16] each
  float *means, *log_scales, *quats, *logits, *sh;
  unsigned long long *n_conflicts;              // optional counter
};
int launch_preprocess_bwd_fdo(const PrepArgs &a, const PrepGradFdoArgs &g, int deg, cudaStream_t s);

// ---------------------------------------------------------------------------
// binning
// ---------------------------------------------------------------------------
struct BinWorkspace {
  // carved from the caller's workspace by bin_layout()
  int64_t *counters;     // [16]: 0 = binned primitives, 1 = K, 2 = overflow flag, 3 = deferred primitives
  uint32_t *hist;        // [8][256] global digit histograms (4 depth + up to 4 tile passes)
  size_t head_bytes;     // counters and hist, cleared at the start of every sort
  uint64_t *blk;         // [kSortBlocks] scan partials
  uint32_t *dk[2], *dv[2];  // depth sort ping-pong, [n] each
  uint32_t *offs;        // [n] instance offsets in depth order
  uint32_t *tk[2];       // tile keys ping-pong, [capacity]
  uint32_t *tv;          // tile vals scratch, [capacity]
  uint32_t *chist;       // [256][kSortBlocks] per-chunk digit counts / offsets of a pass
  size_t bytes;
};

// Instance capacity limit: list offsets and ranges are 32-bit, so a frame
// lists at most 2^32 - 1 instances (a larger count is an overflow), and no
// buffer size computed from a capacity can wrap.
constexpr int64_t kMaxCapacity = HGS_MAX_CAPACITY;
constexpr int kSortBlocks = 1024;  // fixed grid of every sort/scan pass
constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;      // per thread per tile (tile = 2048 keys)

// wide = false reserves nothing for the wide-rectangle path (it is then never taken)
size_t bin_layout(void *base, int64_t n, int64_t capacity, BinWorkspace *ws);

struct BinArgs {
  int64_t n, capacity;
  int tiles, tile_bits, TX;
  const uint32_t *depth_key, *touched;
  const uint16_t *rect;
  const float *tileset;
  uint32_t *vals;
  uint64_t *keys;   // optional
  uint32_t *ranges;
  int64_t *d_count;
  int32_t *dev_err;
};

int launch_bin_sort(const BinArgs &a, const BinWorkspace &ws, cudaStream_t s);

// ---------------------------------------------------------------------------
// render
// ---------------------------------------------------------------------------
struct RenderArgs {
  const float *rec;
  const uint32_t *vals, *ranges;
  CamK cam;
  CfgK cfg;
  float *rgb, *depth, *normal, *alpha, *T_final;
  uint32_t *n_last;
  uint32_t *n_contrib;   // optional
  uint32_t *tile_sched;  // optional [2 * tiles + 1]: tile work, order, hand-out counter
};

struct RenderBwdArgs {
  const float *rec;
  const uint32_t *vals, *ranges;
  CamK cam;
  CfgK cfg;
  const float *T_final;
  const uint32_t *n_last;
  const float *g_rgb, *g_depth, *g_normal, *g_alpha;
  float *rec_grad;  // [n,16], zeroed before launch
  // rgb-only cotangents replayed together (frequency-decoupled optimisation):
  // nc sets, set k read from g_rgbs[k] and accumulated into rec_grads[k]
  // ([n,16] each, zeroed).  nc = 0: the single set g_rgb / rec_grad above.
  int nc;
  const float *g_rgbs[3];
  float *rec_grads[3];
  uint32_t *tile_sched;  // optional [2 * tiles + 1]: tile work, order, hand-out counter
};

int launch_render_fwd(const RenderArgs &a, cudaStream_t s);

// Batched render over a stacked tile grid: request r owns grid rows
// [row_off[r], row_off[r+1]) and columns [0, req[r].cam.TX); its ranges are
// indexed by the global tile id row * TXmax + column.
struct BatchRenderArgs {
  int nreq, TXmax;
  RenderArgs req[kMaxBatch];
  int row_off[kMaxBatch + 1];
};
int launch_render_batch(const BatchRenderArgs &b, int rows, cudaStream_t s);
int launch_render_bwd(const RenderBwdArgs &a, cudaStream_t s);

// ---------------------------------------------------------------------------
// image losses (frequency-decoupled optimisation)
// ---------------------------------------------------------------------------
struct LossArgs {
  const float *img, *tgt;        // [C,H,W]
  int C, H, W;
  double *loss;                  // [3]: L1, L_low, L_high, accumulated (zeroed by the caller)
  float *g_l1, *g_low, *g_high;  // optional gradient images [C,H,W]
  double w_l1, w_low, w_high;    // weights applied to the gradient images
};
int launch_image_losses(const LossArgs &a, cudaStream_t s);

// ---------------------------------------------------------------------------
// training loop
// ---------------------------------------------------------------------------
struct AdamArgs {
  float beta1, beta2, eps;
  float omb1, omb2;     // 1 - beta1, 1 - beta2 (formed in binary64, then rounded)
  float bc1, sqrt_bc2;  // 1 - beta1^t, sqrt(1 - beta2^t)
};
struct AdamGroup {
  float *param;
  const float *grad;
  float *m, *v;
  int64_t count;
  float lr;
  int period, head;  // period > 0: element k uses lr if k % period < head, else lr_tail
  float lr_tail;
};
int launch_adam(const AdamArgs &a, const AdamGroup &g, cudaStream_t s);
int launch_grad_stats(int64_t n, const float *rec_grad, const uint32_t *touched, float *accum, float *count,
                      cudaStream_t s);

struct DensifyPlanArgs {
  int64_t n;
  const float *grad_accum, *vis_count, *log_scales, *logits;
  const uint8_t *types;
  float grad_thresh, log_size_thresh, logit_min_opacity;
  int32_t *actions, *counts;  // [n]
  int64_t *offsets;           // [n+1]
  int64_t *partial;           // [1024] scan scratch
  int64_t *d_new_n;
};
int launch_densify_plan(const DensifyPlanArgs &a, cudaStream_t s);

struct TrainArraysK {
  float *means, *log_scales, *quats, *logits, *sh;
  uint8_t *types;
  float *moments[10];  // Adam m of the five arrays, then v of the five
};
struct DensifyApplyArgs {
  int64_t n;
  int sh_floats;       // (l+1)^2 * 3
  TrainArraysK in, out;
  const float *normals_z;  // [n,2,3]
  const int32_t *actions;
  const int64_t *offsets;
};
int launch_densify_apply(const DensifyApplyArgs &a, cudaStream_t s);
int launch_reset_opacity(int64_t n, float *logits, float cap, float *m, float *v, cudaStream_t s);

// ---------------------------------------------------------------------------
// exchange
// ---------------------------------------------------------------------------
struct ExchangeArgs {
  float *log_scales, *quats;
  uint8_t *types;
  int64_t n;
  int mode;
  float theta;
  const uint8_t *mask;
  unsigned long long *n_flipped;
};

int launch_exchange(const ExchangeArgs &a, cudaStream_t s);

// FP32 peak probe (roofline denominator of the render kernels)
int launch_alu_probe(int kind, int blocks, int iters, float *out, double *ops, cudaStream_t s);

}  // namespace hgs
