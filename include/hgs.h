/*
 * hgs.h -- C ABI of the hybrid 2D/3D Gaussian rasterizer for GB300 (sm_103a).
 *
 * The operation is the Hybrid Gaussian Rasterization of EGGS (Exchangeable
 * 2D/3D Gaussian Splatting, arXiv 2512.02932): each primitive carries a type
 * flag t (Sec. 3.1: t = 0 a 2D surfel, t = 1 a 3D Gaussian); 3D Gaussians are
 * projected affinely (App. C, Eq. 13), 2D surfels by ray-splat intersection
 * (App. C, Eqs. 14-15); both give a distance d (Eq. 1), a contribution
 * alpha * exp(-d/2) (Sec. 3.1) and are alpha-blended in one front-to-back
 * pass (Eq. 2).  Adaptive Type Exchange (Sec. 3.2, Eqs. 3-7) switches types
 * in place.
 *
 * Conventions (every entry point):
 *   - Every data pointer is a DEVICE pointer owned by the caller.  The library
 *     allocates nothing and frees nothing.  Structs themselves are read on the
 *     host during the call and may be discarded when it returns.
 *   - Calls are asynchronous on the given stream and do not synchronise,
 *     except hgs_check, which says so.
 *   - Return value: HGS_OK (0) or a negative hgs_status.  Host-side argument
 *     validation happens before anything is enqueued; on a non-zero return
 *     nothing was launched.
 *   - dev_err points to one device int32 the caller zeroes once; a kernel that
 *     detects a data-dependent error (capacity exceeded, a bounded wait that
 *     ran out) stores the first such status there.  hgs_check reads it.
 *   - No call prints, aborts or exits.
 *   - Float buffers are IEEE binary32, C-contiguous, 16-byte aligned where
 *     marked (A16).
 *
 * Camera: OpenCV convention (x right, y down, z forward), world-to-camera
 * x_c = R x_w + t, pinhole intrinsics fx, fy, cx, cy in pixels; pixel (i, j)
 * has its centre at (i + 0.5, j + 0.5).
 */
#ifndef HGS_H
#define HGS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* a cudaStream_t (same underlying type); NULL = the legacy default stream */
typedef struct CUstream_st *hgs_stream_t;

typedef enum {
  HGS_OK = 0,
  HGS_ERR_INVALID_ARG = -1, /* a pointer, size or setting is invalid */
  HGS_ERR_CAPACITY = -2,    /* instance buffer too small; required size written */
  HGS_ERR_CUDA = -3,        /* a CUDA launch or runtime call failed */
  HGS_ERR_TIMEOUT = -4,     /* a bounded device-side wait ran out */
  HGS_ERR_UNSUPPORTED = -5  /* a setting this build does not implement */
} hgs_status;

/* Scene parameters, one row per primitive (Sec. 3.1): centre mu, scale s
 * (stored as log s), rotation quaternion r (w, x, y, z; normalised on use),
 * opacity (stored as a logit; alpha = sigmoid), SH colour coefficients f of
 * degree l, and the type flag t.  SH layout: [n][(l+1)^2][3] (coefficient
 * major, RGB minor).  A 2D surfel's s_z is ignored by the rasterizer except
 * in the scale modulation of Eqs. 6-7. */
typedef struct {
  const float *means;          /* [n,3] */
  const float *log_scales;     /* [n,3] */
  const float *quats;          /* [n,4] */
  const float *opacity_logits; /* [n] */
  const float *sh;             /* [n,(l+1)^2,3] */
  const uint8_t *types;        /* [n] 0 = 2D surfel, 1 = 3D Gaussian */
  int64_t n;                   /* 0 <= n < 2^31 */
  int32_t sh_degree;           /* 0..3 */
} hgs_scene;

/* The same arrays, writable: the exchange remaps them in place. */
typedef struct {
  float *log_scales; /* [n,3] */
  float *quats;      /* [n,4] */
  uint8_t *types;    /* [n] */
  int64_t n;
} hgs_scene_mut;

typedef struct {
  float R[9]; /* world-to-camera rotation, row major */
  float t[3];
  float fx, fy, cx, cy;
  int32_t width, height; /* 1 .. 16384 */
} hgs_camera;

/* Render settings.  The paper fixes theta_z = 1.05 and T_z = 0.001 (App. A);
 * the rest are unstated and default to the 3DGS practice the paper builds on
 * (hgs_default_config). */
typedef struct {
  float near_z;    /* cull centres with z <= near_z; surfel hits need z > near_z */
  float alpha_min; /* a pair contributes iff alpha*exp(-d/2) >= alpha_min */
  float alpha_max; /* contribution clamp */
  float T_min;     /* stop before a contributor that takes T below T_min */
  float lambda_z;  /* scale modulation weight of Eq. 6 (not given in the paper) */
  float theta_z;   /* Eq. 7 threshold */
  float T_z;       /* Eq. 7 temperature */
  float dilation;  /* added to the diagonal of the projected 3D covariance */
  float bg[3];     /* background colour */
  int32_t tile;    /* tile edge in pixels; this build supports 16 only */
} hgs_config;

/* Per-primitive output of hgs_preprocess (caller-allocated, n rows each):
 *   rec        [n,20] float, A16: the render record (centre, depth, signed
 *              opacity, conic or surfel homography, colour, normal, pixel
 *              box); its content is private to the library and valid for one
 *              camera.
 *   depth_key  [n] uint32: bits of the binary32 camera-space centre depth.
 *   rect       [n,4] uint16: tile rectangle tx0, tx1, ty0, ty1 bounding the
 *              footprint (the region where alpha exp(-d/2) >= alpha_min).
 *   touched    [n] uint32: tiles in the primitive's tile set (0 = not binned).
 *   tileset    [n,12] float, A16: the tile set's parameters, private to the
 *              library: per tile row of the rectangle, the columns whose
 *              pixel centres the footprint can reach. */
typedef struct {
  float *rec;
  uint32_t *depth_key;
  uint16_t *rect;
  uint32_t *touched;
  float *tileset;
} hgs_projected;

/* Output of hgs_bin_sort.
 *   vals    [capacity] uint32: primitive ids of the tile instances, grouped by
 *           tile (row-major tile id), ordered inside a tile by (depth key, id).
 *   keys    [capacity] uint64, optional (may be NULL): tile_id << 32 | depth
 *           key of each instance -- the 64-bit sort key the list is ordered by.
 *   ranges  [tiles,2] uint32: [start, end) of each tile's instances in vals;
 *           an empty tile is [0, 0).
 *   d_count [1] int64: K, the number of instances, written even when K
 *           exceeds the capacity. */
typedef struct {
  uint32_t *vals;
  uint64_t *keys;
  uint32_t *ranges;
  int64_t *d_count;
} hgs_binning;

/* Planar per-pixel output of hgs_render_fwd (each [H,W] plane, row major). */
typedef struct {
  float *rgb;       /* [3,H,W] C + T_final * bg (Eq. 2) */
  float *depth;     /* [H,W] sum of w_i z_i: 3D centre depth, 2D hit depth */
  float *normal;    /* [3,H,W] sum of w_i n_i, camera space */
  float *alpha;     /* [H,W] 1 - T_final */
  float *T_final;   /* [H,W] final transmittance (needed by the backward) */
  uint32_t *n_last; /* [H,W] list entries consumed (needed by the backward) */
  uint32_t *n_contrib; /* [H,W] optional (may be NULL): contributing pairs */
  uint32_t *tile_sched; /* optional (may be NULL): [2 * tiles + 1] scratch in which the
                           rgb-only backward orders the tiles longest first (no
                           counterpart in the paper: scheduling only); NULL takes
                           them in grid order, with the same result */
} hgs_image;

/* Upstream gradients dL/d(outputs), same shapes as hgs_image; any may be NULL
 * (treated as zero). */
typedef struct {
  const float *rgb;
  const float *depth;
  const float *normal;
  const float *alpha;
} hgs_image_grad;

/* Gradients with respect to the raw parameters (overwritten, not added). */
typedef struct {
  float *means;          /* [n,3] */
  float *log_scales;     /* [n,3] */
  float *quats;          /* [n,4] */
  float *opacity_logits; /* [n] */
  float *sh;             /* [n,(l+1)^2,3] */
} hgs_scene_grad;

typedef enum { HGS_EXCHANGE_ERANK = 0, HGS_EXCHANGE_MASK = 1 } hgs_exchange_mode;

typedef struct {
  int32_t mode;          /* hgs_exchange_mode */
  float theta_e;         /* erank threshold (paper: 2.05) */
  const uint8_t *mask;   /* [n] device, MASK mode: flip where non-zero */
} hgs_exchange_cfg;

/* Fill *cfg with the defaults: near 0.2, alpha_min 1/255, alpha_max 0.99,
 * T_min 1e-4, lambda_z 1, theta_z 1.05, T_z 1e-3, dilation 0, bg 0, tile 16. */
void hgs_default_config(hgs_config *cfg);

/* Name of a status code (static string). */
const char *hgs_status_string(int status);

/* Synchronise `stream`, then copy the device error word to *host_err (may be
 * NULL) and return it (HGS_OK if none).  HGS_ERR_CUDA if the stream itself
 * reports an error. */
int hgs_check(const int32_t *dev_err, int32_t *host_err, hgs_stream_t stream);

/* hgs_preprocess -- per-primitive projection (Sec. 3.1, App. C).
 * For each primitive: activations (exp of log s, normalised r, sigmoid
 * opacity), camera-space centre, cull at z <= near_z, SH colour, and
 *   t = 1: projected 2D covariance Sigma' = J W Sigma W^T J^T (Eq. 13) and
 *          its inverse (the conic of Eq. 1);
 *   t = 0: the surfel's splat-to-screen homography (the WH of Eq. 15),
 *          inverted and re-centred so Eq. 14's (u, v) are affine functions
 *          of the pixel offset up to one perspective divide;
 * the scale-modulated opacity for t = 0 (Eqs. 6-7), the normal, and the
 * binning contract: depth key, tile rectangle and tile set from one fixed
 * sequence of binary32 operations (exact rounding, no fused multiply-add).
 * The tile set lists, per tile row, the tile columns that the footprint's
 * ellipse (Eq. 1 at alpha exp(-d/2) = alpha_min, Sec. 3.1) reaches over the
 * row's pixel-centre heights, padded for rounding; for a surfel whose disc
 * reaches the near plane, the columns of the pixels whose rays hit the disc
 * in front of the near plane.
 * Errors: HGS_ERR_INVALID_ARG for NULL pointers, n < 0, sh_degree outside
 * 0..3, a camera with non-positive size or focal, tile != 16 (UNSUPPORTED). */
int hgs_preprocess(const hgs_scene *scene, const hgs_camera *cam, const hgs_config *cfg,
                   hgs_projected *out, int32_t *dev_err, hgs_stream_t stream);

/* Bytes of device workspace hgs_bin_sort needs for n primitives, `capacity`
 * instances and `tiles` tiles.  Host only.  INVALID_ARG for capacity outside
 * 0 .. HGS_MAX_CAPACITY. */
#define HGS_MAX_CAPACITY 0xffffffffLL /* list offsets are 32-bit: at most 2^32 - 1 instances */
int hgs_bin_sort_workspace(int64_t n, int64_t capacity, int32_t tiles, size_t *bytes);

/* hgs_bin_sort -- duplicate each binned primitive into the tiles of its
 * tile set and order the instances by the 64-bit key tile << 32 | depth key,
 * ties by primitive id.  Implemented as an LSD radix sort whose low (depth)
 * digits are sorted once per primitive and whose high (tile) digits are
 * sorted per instance; the resulting order is that of the 64-bit key.
 * If K > capacity: writes K to out->d_count, stores HGS_ERR_CAPACITY in
 * *dev_err, zeroes the ranges, and writes no instance (no out-of-bounds
 * write).  The caller grows the buffers and calls again.
 * ws: device workspace of at least hgs_bin_sort_workspace() bytes, A16.
 * Errors: INVALID_ARG for NULL pointers, ws_bytes too small, capacity
 * outside 0 .. HGS_MAX_CAPACITY. */
int hgs_bin_sort(int64_t n, const hgs_projected *proj, const hgs_camera *cam,
                 const hgs_config *cfg, void *ws, size_t ws_bytes, int64_t capacity,
                 hgs_binning *out, int32_t *dev_err, hgs_stream_t stream);

/* hgs_fp32_probe -- a measurement, not part of the path: launches `blocks`
 * CTAs of 256 threads, each thread running 8 independent chains of `iters`
 * binary32 fused multiply-adds, so the caller can time the device's FP32
 * rate (the denominator of the render kernels' roofline).  d_out: device
 * float[blocks], written only by a branch that is never taken.  *flops
 * (host) receives the floating-point operations launched (2 per FMA).
 * Errors: INVALID_ARG for blocks < 1, iters < 1, NULL d_out or flops. */
int hgs_fp32_probe(int32_t blocks, int32_t iters, float *d_out, double *flops, hgs_stream_t stream);

/* hgs_alu_probe -- a measurement, not part of the path, with no counterpart
 * in the paper: like hgs_fp32_probe, `blocks` CTAs of 256 threads each run 8
 * independent chains of `iters` steps of one kind of operation, so that the
 * caller can time the peak rate of the unit the render kernels' per-pair loop
 * issues to:
 *   HGS_PROBE_FFMA   binary32 fused multiply-add, *ops = 2 flops per step
 *   HGS_PROBE_FFMA2  packed two-lane binary32 fused multiply-add (the form
 *                    the render kernels use for a lane's two pixels),
 *                    *ops = 4 flops per step
 *   HGS_PROBE_EX2    special-function base-2 exponential, *ops = 1 per step
 *   HGS_PROBE_RCP    special-function reciprocal (plus one add that keeps the
 *                    chain from being shortened), *ops = 1 per step
 * d_out: device float[blocks], written only by a branch never taken.
 * Errors: INVALID_ARG for an unknown kind, blocks < 1, iters < 1, NULL d_out
 * or ops. */
enum { HGS_PROBE_FFMA = 0, HGS_PROBE_FFMA2 = 1, HGS_PROBE_EX2 = 2, HGS_PROBE_RCP = 3 };
int hgs_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float *d_out, double *ops, hgs_stream_t stream);

/* hgs_bin_sort_static -- hgs_bin_sort without a caller-supplied workspace,
 * for callers that cannot allocate device memory while they render: a host
 * application that owns the GPU allocator and forbids other cudaMalloc calls,
 * or a real-time loop that must avoid cudaMalloc/cudaFree because they can
 * synchronise the device.  The paper has no counterpart; this is a deployment
 * convenience.  Inputs and outputs are exactly those of hgs_bin_sort (the
 * caller still owns proj and out); the sort's scratch is a library-owned
 * device array of HGS_BIN_SORT_STATIC_BYTES that every GPU loading the
 * library reserves until the process exits.
 * Limits: returns HGS_ERR_INVALID_ARG, launching nothing, for a capacity
 * outside 0 .. HGS_MAX_CAPACITY and when that scratch
 * (hgs_bin_sort_workspace(n, capacity, tiles)) exceeds
 * HGS_BIN_SORT_STATIC_BYTES (for example n = 1M with capacity 3.5M fits; the
 * 3M-primitive scene does not).  The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and it keeps the
 * previous call's contents (the kernels clear what must start at zero): calls
 * whose work can overlap on the GPU race, so serialise them.  Allocates
 * nothing; HGS_ERR_CUDA if the address lookup or a launch fails. */
#define HGS_BIN_SORT_STATIC_BYTES ((size_t)64 << 20)
int hgs_bin_sort_static(int64_t n, const hgs_projected *proj, const hgs_camera *cam,
                        const hgs_config *cfg, int64_t capacity, hgs_binning *out,
                        int32_t *dev_err, hgs_stream_t stream);

/* hgs_render_fwd -- per 16x16 tile, front-to-back blending over the tile's
 * sorted list (Eq. 2): per pair the unified distance of Eq. 1, contribution
 * a = min(alpha_max, alpha exp(-d/2)), skipped if a < alpha_min; stop before
 * the first contributor with T (1 - a) < T_min.  Writes every field of *out. */
int hgs_render_fwd(int64_t n, const hgs_projected *proj, const hgs_binning *bins,
                   const hgs_camera *cam, const hgs_config *cfg, hgs_image *out,
                   int32_t *dev_err, hgs_stream_t stream);

/* hgs_render_bwd -- gradients of a scalar loss with respect to the raw scene
 * parameters, given dL/d(outputs).  Replays each tile's list in reverse from
 * n_last, recovering the transmittance by division (T_i = T_{i+1}/(1 - a_i)),
 * accumulates per-primitive gradients of the render record (warp-reduced
 * atomics into grad_ws), then chains them through the projection, the SH
 * decode, the activations and the scale modulation.
 * grad_ws: [n,16] float device scratch, A16, zeroed by this call.
 * `fwd` must be the output of hgs_render_fwd for the same inputs. */
int hgs_render_bwd(const hgs_scene *scene, const hgs_projected *proj,
                   const hgs_binning *bins, const hgs_camera *cam, const hgs_config *cfg,
                   const hgs_image *fwd, const hgs_image_grad *dL, float *grad_ws,
                   hgs_scene_grad *out, int32_t *dev_err, hgs_stream_t stream);

/* One request of a batched render: a resident scene, a camera and the
 * request's own output planes (rgb, depth, normal, alpha, T_final, n_last as
 * in hgs_image, sized for this camera). */
typedef struct {
  hgs_scene scene;
  hgs_camera cam;
  hgs_image out;
} hgs_request;

#define HGS_MAX_BATCH 16

/* Bytes of device workspace hgs_render_batch needs for these requests and
 * `capacity` tile instances in total.  Host only.  INVALID_ARG for capacity
 * outside 0 .. HGS_MAX_CAPACITY (hgs_render_batch likewise). */
int hgs_render_batch_workspace(int nreq, const hgs_request *reqs, int64_t capacity, size_t *bytes);

/* hgs_render_batch -- the forward rasterizer (hgs_preprocess + hgs_bin_sort +
 * hgs_render_fwd) for up to HGS_MAX_BATCH requests of different scenes and
 * resolutions, each stage one launch for the whole batch (the serving form).
 * The requests' primitives are concatenated and their 16x16 tile grids are
 * stacked vertically into one grid (width = widest request), so one sort and
 * one render launch cover every request; each request's image is exactly the
 * one hgs_render_fwd would produce alone (a tile never mixes requests).
 * ws: device workspace of hgs_render_batch_workspace() bytes, A16; it holds
 * the combined records, the instance list and the sort scratch.
 * d_count (device int64) receives the batch's instance count K; if K >
 * capacity, HGS_ERR_CAPACITY is stored in *dev_err and the images hold only
 * the background (nothing out of bounds): grow and retry.
 * Errors: INVALID_ARG for nreq outside 1..HGS_MAX_BATCH, a bad scene, camera
 * or output pointer, a too small workspace; UNSUPPORTED for tile != 16 or a
 * stacked grid over 32767 tile rows. */
int hgs_render_batch(int nreq, const hgs_request *reqs, const hgs_config *cfg, void *ws, size_t ws_bytes,
                     int64_t capacity, int64_t *d_count, int32_t *dev_err, hgs_stream_t stream);

/* The two stages of hgs_render_bwd, for callers that want the per-primitive
 * gradient of the render record or time the stages separately:
 * hgs_render_bwd_records -- zero grad_ws, then replay every tile's list in
 *   reverse and accumulate dL/d(record) (centre, conic or surfel homography,
 *   opacity, colour, depth, normal: 16 floats per primitive) into grad_ws.
 * hgs_preprocess_bwd -- chain grad_ws through the projection, the SH decode,
 *   the activations and the scale modulation to the raw parameters.
 * Arguments and errors as in hgs_render_bwd. */
int hgs_render_bwd_records(const hgs_scene *scene, const hgs_projected *proj, const hgs_binning *bins,
                           const hgs_camera *cam, const hgs_config *cfg, const hgs_image *fwd,
                           const hgs_image_grad *dL, float *grad_ws, int32_t *dev_err, hgs_stream_t stream);
int hgs_preprocess_bwd(const hgs_scene *scene, const hgs_projected *proj, const hgs_camera *cam,
                       const hgs_config *cfg, const float *grad_ws, hgs_scene_grad *out, int32_t *dev_err,
                       hgs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Frequency-decoupled optimisation (Sec. 3.3, Eq. 8, Algorithm 1; App. E)
 * ------------------------------------------------------------------------- */

/* hgs_image_losses -- the image losses of Eq. 8 other than D-SSIM, with their
 * gradient images.  Level-1 Haar DWT (App. E) with l = (1,1)/sqrt2,
 * h = (1,-1)/sqrt2 on the 2x2 blocks (a b; c d) at rows 2i, 2i+1, columns
 * 2j, 2j+1: LL = (a+b+c+d)/2, LH = (a+b-c-d)/2, HL = (a-b+c-d)/2,
 * HH = (a-b-c+d)/2, applied to image - target.
 *   L1     = mean over C*H*W pixels of |image - target|
 *   L_low  = mean over the C*(H/2)*(W/2) LL coefficients of dLL^2
 *   L_high = mean over the 3*C*(H/2)*(W/2) LH, HL and HH coefficients of their squares
 * An odd last row or column lies outside every block and enters L1 only.
 * image, target: [C,H,W] float32 device arrays (caller-owned).
 * d_losses: device double[3] <- (L1, L_low, L_high); zeroed by this call.
 * g_l1, g_low, g_high: [C,H,W] float32 device outputs, each optional (NULL
 *   skips it): w_l1 dL1/dimage (sign(0) = 0), w_low dL_low/dimage,
 *   w_high dL_high/dimage.  Every pixel of a requested output is written.
 * Errors: INVALID_ARG for NULL image, target or d_losses, or C, H, W < 1. */
int hgs_image_losses(const float *image, const float *target, int32_t channels, int32_t height,
                     int32_t width, double w_l1, double w_low, double w_high, double *d_losses,
                     float *g_l1, float *g_low, float *g_high, hgs_stream_t stream);

/* hgs_render_bwd_fdo -- the backward of frequency-decoupled optimisation
 * (Algorithm 1).  g_color, g_low and g_high are the rgb cotangents ([3,H,W]
 * float32, device) of the appearance loss and of the (weighted) low- and
 * high-frequency losses.  Each is replayed through the rasterizer as in
 * hgs_render_bwd_records, giving per primitive three raw-parameter gradients
 * g^color, g^low, g^high (each the concatenation of the primitive's means,
 * log-scale, quaternion, opacity-logit and SH gradients).  Where
 * g^low . g^high < 0 a surfel (type 0) replaces g^high by g^high -
 * (g^high . g^low)/|g^low|^2 g^low (Eq. 9) and a 3D Gaussian replaces g^low
 * by g^low - (g^high . g^low)/|g^high|^2 g^high (Eq. 10).  *out receives
 * g^color + g^low + g^high.
 * grad_ws: [3,n,16] float device scratch, A16, zeroed by this call.
 * d_conflicts: device uint64 counter incremented once per conflicting
 *   primitive (may be NULL; not zeroed by this call).
 * Other arguments and errors as in hgs_render_bwd. */
int hgs_render_bwd_fdo(const hgs_scene *scene, const hgs_projected *proj, const hgs_binning *bins,
                       const hgs_camera *cam, const hgs_config *cfg, const hgs_image *fwd,
                       const float *g_color, const float *g_low, const float *g_high, float *grad_ws,
                       hgs_scene_grad *out, unsigned long long *d_conflicts, int32_t *dev_err,
                       hgs_stream_t stream);

/* ---------------------------------------------------------------------------
 * Training loop (App. A: the 3DGS schedule with Adaptive Type Exchange every
 * 500 iterations and densification every 100 iterations from 500 to 15K)
 * ------------------------------------------------------------------------- */

/* One parameter array and its Adam state: count float32 values each, device,
 * caller-owned (16-byte aligned arrays take the float4 path).  period > 0
 * splits the learning rate along rows: element k uses lr if k % period <
 * head and lr_tail otherwise (e.g. an SH row's DC and higher-order
 * coefficients); period = 0 uses lr throughout, otherwise period >= 4 and
 * head <= period. */
typedef struct {
  float *param;
  const float *grad;
  float *m, *v;
  int64_t count;
  float lr;
  int32_t period, head;
  float lr_tail;
} hgs_adam_group;

/* hgs_adam_step -- one Adam update (step t >= 1, bias-corrected):
 * m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2,
 * p -= (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps), per group.
 * The coefficients 1 - b1, 1 - b2 and the bias corrections are formed in
 * binary64 from the arguments and rounded once; the update is binary32.
 * Errors: INVALID_ARG for ngroups < 0, NULL groups or arrays, or t < 1. */
int hgs_adam_step(int32_t ngroups, const hgs_adam_group *groups, int32_t step, double beta1, double beta2,
                  double eps, hgs_stream_t stream);

/* hgs_grad_stats -- the statistic densification decides on: for every
 * primitive binned in the last hgs_bin_sort (touched > 0), accum += the norm
 * of its loss gradient with respect to the projected centre (pixels; record
 * gradient slots 4 and 5 left in grad_ws by hgs_render_bwd) and count += 1.
 * grad_ws: [n,16]; accum, count: [n] float32 device. */
int hgs_grad_stats(int64_t n, const float *grad_ws, const hgs_projected *proj, float *accum, float *count,
                   hgs_stream_t stream);

/* Densification thresholds, on the stored parameters: mean gradient
 * statistic (pixels), largest active log-scale, opacity logit. */
typedef struct {
  float grad_thresh;
  float log_size_thresh;
  float logit_min_opacity;
} hgs_densify_cfg;

/* Bytes of device workspace hgs_densify_plan needs for n primitives. */
int hgs_densify_workspace(int64_t n, size_t *bytes);

/* hgs_densify_plan -- the 3DGS densification decision per primitive, in
 * binary32: with g = accum / count (0 if never binned), size = the largest
 * active log-scale (a surfel's two in-plane axes):
 *   g >= grad_thresh and size <= log_size_thresh -> 2 (keep and clone)
 *   g >= grad_thresh and size >  log_size_thresh -> 3 (split into two)
 *   otherwise, logit < logit_min_opacity         -> 0 (remove), else 1 (keep).
 * actions: [n] int32; offsets: [n+1] int64, the first output row of each
 * primitive (exclusive scan of its 0/1/2 rows), offsets[n] = the new count,
 * also written to *d_new_n.  All device. */
int hgs_densify_plan(const hgs_scene *scene, const float *accum, const float *count, const hgs_densify_cfg *cfg,
                     int32_t *actions, int64_t *offsets, void *ws, size_t ws_bytes, int64_t *d_new_n,
                     hgs_stream_t stream);

/* Parameter arrays and Adam moments of a training scene (rows as in
 * hgs_scene; moments[k] and moments[5+k] are m and v of the k-th of means,
 * log-scales, quaternions, opacity logits, SH; any moment may be NULL). */
typedef struct {
  float *means, *log_scales, *quats, *opacity_logits, *sh;
  uint8_t *types;
  float *moments[10];
} hgs_train_arrays;

/* hgs_densify_apply -- write the densified scene into `out` (offsets[n]
 * rows): a kept primitive's row and moments are copied; a clone adds an
 * exact copy with zero moments; a split writes two rows centred at
 * mu + R (s * z) (z from normals_z [n,2,3], a surfel's third scale taken as
 * 0), with log-scales reduced by log 1.6 (a surfel's third kept), the other
 * parameters copied and zero moments.  in and out must not overlap. */
int hgs_densify_apply(int64_t n, int32_t sh_degree, const hgs_train_arrays *in, hgs_train_arrays *out,
                      const float *normals_z, const int32_t *actions, const int64_t *offsets,
                      hgs_stream_t stream);

/* hgs_reset_opacity -- alpha <- min(alpha, ceiling) on the logits; the
 * logits' Adam moments m, v (may be NULL) are zeroed. */
int hgs_reset_opacity(int64_t n, float *opacity_logits, float ceiling, float *m, float *v, hgs_stream_t stream);

/* hgs_exchange_types -- Adaptive Type Exchange (Sec. 3.2) in place.
 * ERANK mode: erank = exp(-sum p_i log p_i), p = q / |q|_1, q = (s_x^2,
 * s_y^2, s_z^2) (Eq. 3); a 3D Gaussian with erank < theta_e becomes 2D, a 2D
 * one with erank > theta_e becomes 3D (the comparison is decided in binary64
 * whenever binary32 cannot decide it).  MASK mode: flip where mask != 0.
 * 3D -> 2D reparameterises S* = P S P^T, R* = R P^T (Eqs. 4-5) with P = P_x
 * if s_x is the smallest scale, P_y if s_y is (ties: x), identity if s_z is
 * already the smallest; the quaternion becomes r (x) p with R(p) = P^T.
 * 2D -> 3D flips the flag only (Sec. 3.2).  No buffer is reallocated or
 * reordered.  *d_n_flipped (device int64, may be NULL) receives the count.
 * Errors: INVALID_ARG for NULL arrays or a NULL mask in MASK mode. */
int hgs_exchange_types(hgs_scene_mut *scene, const hgs_exchange_cfg *xcfg,
                       int64_t *d_n_flipped, int32_t *dev_err, hgs_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* HGS_H */
