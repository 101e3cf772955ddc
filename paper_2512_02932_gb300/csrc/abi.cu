// abi.cu -- extern "C" entry points of libhgs (declared in include/hgs.h).
// Host-side validation, conversion of the ABI structs to kernel argument
// blocks, and launches on the caller's stream.  Nothing here allocates,
// synchronises (except hgs_check) or prints.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"
#include "kernels.cuh"

using namespace hgs;

namespace {

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int cam_to_kernel(const hgs_camera *c, CamK *k) {
  if (!c) return HGS_ERR_INVALID_ARG;
  if (c->width <= 0 || c->height <= 0 || c->width > 16384 || c->height > 16384) return HGS_ERR_INVALID_ARG;
  if (!(c->fx > 0.f) || !(c->fy > 0.f) || !std::isfinite(c->cx) || !std::isfinite(c->cy))
    return HGS_ERR_INVALID_ARG;
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(c->R[i])) return HGS_ERR_INVALID_ARG;
  for (int i = 0; i < 3; ++i)
    if (!std::isfinite(c->t[i])) return HGS_ERR_INVALID_ARG;
  std::memcpy(k->R, c->R, sizeof(k->R));
  std::memcpy(k->t, c->t, sizeof(k->t));
  k->fx = c->fx; k->fy = c->fy; k->cx = c->cx; k->cy = c->cy;
  for (int i = 0; i < 3; ++i)
    k->campos[i] = -(c->R[i] * c->t[0] + c->R[3 + i] * c->t[1] + c->R[6 + i] * c->t[2]);
  k->W = c->width; k->H = c->height;
  k->TX = (c->width + kTile - 1) / kTile;
  k->TY = (c->height + kTile - 1) / kTile;
  return HGS_OK;
}

int cfg_to_kernel(const hgs_config *c, CfgK *k) {
  if (!c) return HGS_ERR_INVALID_ARG;
  if (c->tile != kTile) return HGS_ERR_UNSUPPORTED;
  if (!(c->alpha_min > 0.f) || !(c->alpha_max >= c->alpha_min) || !(c->alpha_max < 1.f) ||
      !(c->T_min > 0.f) || !(c->T_z > 0.f) || !(c->near_z > 0.f) || !(c->dilation >= 0.f) ||
      !std::isfinite(c->lambda_z) || !std::isfinite(c->theta_z))
    return HGS_ERR_INVALID_ARG;
  k->near_z = c->near_z; k->alpha_min = c->alpha_min; k->alpha_max = c->alpha_max;
  k->T_min = c->T_min; k->lambda_z = c->lambda_z; k->theta_z = c->theta_z; k->T_z = c->T_z;
  k->dilation = c->dilation;
  for (int i = 0; i < 3; ++i) k->bg[i] = c->bg[i];
  return HGS_OK;
}

int scene_ok(const hgs_scene *s) {
  if (!s || s->n < 0 || s->n >= (int64_t(1) << 31)) return HGS_ERR_INVALID_ARG;
  if (s->sh_degree < 0 || s->sh_degree > 3) return HGS_ERR_INVALID_ARG;
  if (s->n == 0) return HGS_OK;
  if (!s->means || !s->log_scales || !s->quats || !s->opacity_logits || !s->sh || !s->types)
    return HGS_ERR_INVALID_ARG;
  if (!aligned16(s->quats)) return HGS_ERR_INVALID_ARG;
  if ((s->sh_degree == 1 || s->sh_degree == 3) && !aligned16(s->sh)) return HGS_ERR_INVALID_ARG;
  return HGS_OK;
}

int proj_ok(const hgs_projected *p, int64_t n) {
  if (!p) return HGS_ERR_INVALID_ARG;
  if (n == 0) return HGS_OK;
  if (!p->rec || !p->depth_key || !p->rect || !p->touched || !p->tileset) return HGS_ERR_INVALID_ARG;
  if (!aligned16(p->rec) || !aligned16(p->tileset) || (reinterpret_cast<uintptr_t>(p->rect) & 7u))
    return HGS_ERR_INVALID_ARG;
  return HGS_OK;
}

int tile_bits_for(int tiles) {
  int b = 1;
  while ((1 << b) < tiles) ++b;
  return b;
}

int launched() { return cudaGetLastError() == cudaSuccess ? HGS_OK : HGS_ERR_CUDA; }

PrepArgs prep_args(const hgs_scene *s, const CamK &ck, const CfgK &fk, const hgs_projected *p) {
  PrepArgs a;
  a.means = s->means; a.log_scales = s->log_scales; a.quats = s->quats;
  a.logits = s->opacity_logits; a.sh = s->sh; a.types = s->types; a.n = s->n;
  a.cam = ck; a.cfg = fk;
  a.rec = p->rec; a.depth_key = p->depth_key; a.rect = p->rect; a.touched = p->touched;
  a.tileset = p->tileset;
  return a;
}

}  // namespace

extern "C" {

void hgs_default_config(hgs_config *c) {
  if (!c) return;
  c->near_z = 0.2f;
  c->alpha_min = 1.0f / 255.0f;
  c->alpha_max = 0.99f;
  c->T_min = 1e-4f;
  c->lambda_z = 1.0f;
  c->theta_z = 1.05f;
  c->T_z = 1e-3f;
  c->dilation = 0.0f;
  c->bg[0] = c->bg[1] = c->bg[2] = 0.0f;
  c->tile = kTile;
}

const char *hgs_status_string(int s) {
  switch (s) {
    case HGS_OK: return "HGS_OK";
    case HGS_ERR_INVALID_ARG: return "HGS_ERR_INVALID_ARG";
    case HGS_ERR_CAPACITY: return "HGS_ERR_CAPACITY";
    case HGS_ERR_CUDA: return "HGS_ERR_CUDA";
    case HGS_ERR_TIMEOUT: return "HGS_ERR_TIMEOUT";
    case HGS_ERR_UNSUPPORTED: return "HGS_ERR_UNSUPPORTED";
    default: return "HGS_ERR_UNKNOWN";
  }
}

int hgs_check(const int32_t *dev_err, int32_t *host_err, hgs_stream_t stream) {
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (cudaStreamSynchronize(s) != cudaSuccess) return HGS_ERR_CUDA;
  int32_t e = 0;
  if (dev_err && cudaMemcpy(&e, dev_err, sizeof(e), cudaMemcpyDeviceToHost) != cudaSuccess)
    return HGS_ERR_CUDA;
  if (host_err) *host_err = e;
  return e;
}

int hgs_preprocess(const hgs_scene *scene, const hgs_camera *cam, const hgs_config *cfg,
                   hgs_projected *out, int32_t *dev_err, hgs_stream_t stream) {
  (void)dev_err;
  int st;
  if ((st = scene_ok(scene)) != HGS_OK) return st;
  CamK ck;
  CfgK fk;
  if ((st = cam_to_kernel(cam, &ck)) != HGS_OK) return st;
  if ((st = cfg_to_kernel(cfg, &fk)) != HGS_OK) return st;
  if ((st = proj_ok(out, scene->n)) != HGS_OK) return st;
  if (scene->n == 0) return HGS_OK;
  launch_preprocess_fwd(prep_args(scene, ck, fk, out), scene->sh_degree,
                        reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

int hgs_bin_sort_workspace(int64_t n, int64_t capacity, int32_t tiles, size_t *bytes) {
  if (!bytes || n < 0 || capacity < 0 || capacity > kMaxCapacity || tiles <= 0) return HGS_ERR_INVALID_ARG;
  BinWorkspace ws;
  *bytes = bin_layout(nullptr, n, capacity, &ws);
  return HGS_OK;
}

int hgs_bin_sort(int64_t n, const hgs_projected *proj, const hgs_camera *cam, const hgs_config *cfg,
                 void *ws, size_t ws_bytes, int64_t capacity, hgs_binning *out, int32_t *dev_err,
                 hgs_stream_t stream) {
  int st;
  if (n < 0 || n >= (int64_t(1) << 31) || capacity < 0 || capacity > kMaxCapacity || !out || !out->ranges ||
      !out->d_count)
    return HGS_ERR_INVALID_ARG;
  if (capacity > 0 && !out->vals) return HGS_ERR_INVALID_ARG;
  CamK ck;
  CfgK fk;
  if ((st = cam_to_kernel(cam, &ck)) != HGS_OK) return st;
  if ((st = cfg_to_kernel(cfg, &fk)) != HGS_OK) return st;
  if ((st = proj_ok(proj, n)) != HGS_OK) return st;
  if (!ws || !aligned16(ws)) return HGS_ERR_INVALID_ARG;
  BinWorkspace w;
  const size_t need = bin_layout(ws, n, capacity, &w);
  if (ws_bytes < need) return HGS_ERR_INVALID_ARG;
  BinArgs a;
  a.n = n;
  a.capacity = capacity;
  a.tiles = ck.TX * ck.TY;
  a.tile_bits = tile_bits_for(a.tiles);
  a.TX = ck.TX;
  a.depth_key = proj->depth_key;
  a.touched = proj->touched;
  a.rect = proj->rect;
  a.tileset = proj->tileset;
  a.vals = out->vals;
  a.keys = out->keys;
  a.ranges = out->ranges;
  a.d_count = out->d_count;
  a.dev_err = dev_err;
  launch_bin_sort(a, w, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

int hgs_render_fwd(int64_t n, const hgs_projected *proj, const hgs_binning *bins, const hgs_camera *cam,
                   const hgs_config *cfg, hgs_image *out, int32_t *dev_err, hgs_stream_t stream) {
  (void)dev_err;
  int st;
  CamK ck;
  CfgK fk;
  if ((st = cam_to_kernel(cam, &ck)) != HGS_OK) return st;
  if ((st = cfg_to_kernel(cfg, &fk)) != HGS_OK) return st;
  if ((st = proj_ok(proj, n)) != HGS_OK) return st;
  if (!bins || !bins->ranges || (n > 0 && !bins->vals)) return HGS_ERR_INVALID_ARG;
  if (!out || !out->rgb || !out->depth || !out->normal || !out->alpha || !out->T_final || !out->n_last)
    return HGS_ERR_INVALID_ARG;
  RenderArgs a;
  a.rec = proj->rec;
  a.vals = bins->vals;
  a.ranges = bins->ranges;
  a.cam = ck;
  a.cfg = fk;
  a.rgb = out->rgb; a.depth = out->depth; a.normal = out->normal; a.alpha = out->alpha;
  a.T_final = out->T_final; a.n_last = out->n_last; a.n_contrib = out->n_contrib;
  a.tile_sched = out->tile_sched;
  launch_render_fwd(a, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

int hgs_render_bwd_records(const hgs_scene *scene, const hgs_projected *proj, const hgs_binning *bins,
                           const hgs_camera *cam, const hgs_config *cfg, const hgs_image *fwd,
                           const hgs_image_grad *dL, float *grad_ws, int32_t *dev_err, hgs_stream_t stream) {
  (void)dev_err;
  int st;
  if ((st = scene_ok(scene)) != HGS_OK) return st;
  CamK ck;
  CfgK fk;
  if ((st = cam_to_kernel(cam, &ck)) != HGS_OK) return st;
  if ((st = cfg_to_kernel(cfg, &fk)) != HGS_OK) return st;
  if ((st = proj_ok(proj, scene->n)) != HGS_OK) return st;
  if (!bins || !bins->ranges || (scene->n > 0 && !bins->vals)) return HGS_ERR_INVALID_ARG;
  if (!fwd || !fwd->T_final || !fwd->n_last || !dL) return HGS_ERR_INVALID_ARG;
  if (scene->n > 0 && (!grad_ws || !aligned16(grad_ws))) return HGS_ERR_INVALID_ARG;
  if (scene->n == 0) return HGS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaMemsetAsync(grad_ws, 0, sizeof(float) * kGradW * (size_t)scene->n, s);
  RenderBwdArgs r{};
  r.rec = proj->rec;
  r.vals = bins->vals;
  r.ranges = bins->ranges;
  r.cam = ck;
  r.cfg = fk;
  r.T_final = fwd->T_final;
  r.n_last = fwd->n_last;
  r.g_rgb = dL->rgb; r.g_depth = dL->depth; r.g_normal = dL->normal; r.g_alpha = dL->alpha;
  r.rec_grad = grad_ws;
  r.tile_sched = fwd->tile_sched;
  launch_render_bwd(r, s);
  return launched();
}

int hgs_preprocess_bwd(const hgs_scene *scene, const hgs_projected *proj, const hgs_camera *cam,
                       const hgs_config *cfg, const float *grad_ws, hgs_scene_grad *out, int32_t *dev_err,
                       hgs_stream_t stream) {
  (void)dev_err;
  int st;
  if ((st = scene_ok(scene)) != HGS_OK) return st;
  CamK ck;
  CfgK fk;
  if ((st = cam_to_kernel(cam, &ck)) != HGS_OK) return st;
  if ((st = cfg_to_kernel(cfg, &fk)) != HGS_OK) return st;
  if ((st = proj_ok(proj, scene->n)) != HGS_OK) return st;
  if (!out || (scene->n > 0 && (!out->means || !out->log_scales || !out->quats ||
                                !out->opacity_logits || !out->sh)))
    return HGS_ERR_INVALID_ARG;
  if (scene->n > 0 && (!grad_ws || !aligned16(grad_ws) || !aligned16(out->quats)))
    return HGS_ERR_INVALID_ARG;
  if ((scene->sh_degree == 1 || scene->sh_degree == 3) && scene->n > 0 && !aligned16(out->sh))
    return HGS_ERR_INVALID_ARG;
  if (scene->n == 0) return HGS_OK;
  PrepGradArgs g;
  g.rec_grad = grad_ws;
  g.means = out->means; g.log_scales = out->log_scales; g.quats = out->quats;
  g.logits = out->opacity_logits; g.sh = out->sh;
  hgs_projected pcopy = *proj;
  launch_preprocess_bwd(prep_args(scene, ck, fk, &pcopy), g, scene->sh_degree,
                        reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

int hgs_render_bwd(const hgs_scene *scene, const hgs_projected *proj, const hgs_binning *bins,
                   const hgs_camera *cam, const hgs_config *cfg, const hgs_image *fwd,
                   const hgs_image_grad *dL, float *grad_ws, hgs_scene_grad *out, int32_t *dev_err,
                   hgs_stream_t stream) {
  if (!out) return HGS_ERR_INVALID_ARG;
  int st = hgs_render_bwd_records(scene, proj, bins, cam, cfg, fwd, dL, grad_ws, dev_err, stream);
  if (st != HGS_OK) return st;
  return hgs_preprocess_bwd(scene, proj, cam, cfg, grad_ws, out, dev_err, stream);
}


int hgs_image_losses(const float *image, const float *target, int32_t channels, int32_t height,
                     int32_t width, double w_l1, double w_low, double w_high, double *d_losses,
                     float *g_l1, float *g_low, float *g_high, hgs_stream_t stream) {
  if (!image || !target || !d_losses || channels < 1 || height < 1 || width < 1) return HGS_ERR_INVALID_ARG;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  cudaMemsetAsync(d_losses, 0, 3 * sizeof(double), s);
  LossArgs a;
  a.img = image; a.tgt = target;
  a.C = channels; a.H = height; a.W = width;
  a.loss = d_losses;
  a.g_l1 = g_l1; a.g_low = g_low; a.g_high = g_high;
  a.w_l1 = w_l1; a.w_low = w_low; a.w_high = w_high;
  launch_image_losses(a, s);
  return launched();
}

int hgs_render_bwd_fdo(const hgs_scene *scene, const hgs_projected *proj, const hgs_binning *bins,
                       const hgs_camera *cam, const hgs_config *cfg, const hgs_image *fwd,
                       const float *g_color, const float *g_low, const float *g_high, float *grad_ws,
                       hgs_scene_grad *out, unsigned long long *d_conflicts, int32_t *dev_err,
                       hgs_stream_t stream) {
  (void)dev_err;
  int st;
  if (!g_color || !g_low || !g_high || !out) return HGS_ERR_INVALID_ARG;
  if ((st = scene_ok(scene)) != HGS_OK) return st;
  CamK ck;
  CfgK fk;
  if ((st = cam_to_kernel(cam, &ck)) != HGS_OK) return st;
  if ((st = cfg_to_kernel(cfg, &fk)) != HGS_OK) return st;
  if ((st = proj_ok(proj, scene->n)) != HGS_OK) return st;
  if (!bins || !bins->ranges || (scene->n > 0 && !bins->vals)) return HGS_ERR_INVALID_ARG;
  if (!fwd || !fwd->T_final || !fwd->n_last) return HGS_ERR_INVALID_ARG;
  if (scene->n > 0 && (!grad_ws || !aligned16(grad_ws))) return HGS_ERR_INVALID_ARG;
  if (scene->n > 0 && (!out->means || !out->log_scales || !out->quats || !out->opacity_logits || !out->sh ||
                       !aligned16(out->quats)))
    return HGS_ERR_INVALID_ARG;
  if ((scene->sh_degree == 1 || scene->sh_degree == 3) && scene->n > 0 && !aligned16(out->sh))
    return HGS_ERR_INVALID_ARG;
  if (scene->n == 0) return HGS_OK;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const size_t stride = (size_t)kGradW * (size_t)scene->n;
  // the three cotangents in one replay: one evaluation and transmittance step
  // per pair, three record-gradient sets
  cudaMemsetAsync(grad_ws, 0, 3 * sizeof(float) * stride, s);
  RenderBwdArgs r{};
  r.rec = proj->rec;
  r.vals = bins->vals;
  r.ranges = bins->ranges;
  r.cam = ck;
  r.cfg = fk;
  r.T_final = fwd->T_final;
  r.n_last = fwd->n_last;
  r.nc = 3;
  r.tile_sched = fwd->tile_sched;
  r.g_rgbs[0] = g_color; r.g_rgbs[1] = g_low; r.g_rgbs[2] = g_high;
  for (int k = 0; k < 3; ++k) r.rec_grads[k] = grad_ws + k * stride;
  launch_render_bwd(r, s);
  PrepGradFdoArgs g;
  g.rec_color = grad_ws; g.rec_low = grad_ws + stride; g.rec_high = grad_ws + 2 * stride;
  g.means = out->means; g.log_scales = out->log_scales; g.quats = out->quats;
  g.logits = out->opacity_logits; g.sh = out->sh;
  g.n_conflicts = d_conflicts;
  hgs_projected pcopy = *proj;
  launch_preprocess_bwd_fdo(prep_args(scene, ck, fk, &pcopy), g, scene->sh_degree, s);
  return launched();
}

int hgs_adam_step(int32_t ngroups, const hgs_adam_group *groups, int32_t step, double beta1, double beta2,
                  double eps, hgs_stream_t stream) {
  if (ngroups < 0 || (ngroups > 0 && !groups) || step < 1) return HGS_ERR_INVALID_ARG;
  for (int k = 0; k < ngroups; ++k)
    if (groups[k].count < 0 || groups[k].head < 0 || (groups[k].period != 0 && groups[k].period < 4) ||
        groups[k].head > std::max(groups[k].period, 0) ||
        (groups[k].count > 0 && (!groups[k].param || !groups[k].grad || !groups[k].m || !groups[k].v)))
      return HGS_ERR_INVALID_ARG;
  AdamArgs a;
  a.beta1 = (float)beta1; a.beta2 = (float)beta2; a.eps = (float)eps;
  a.omb1 = (float)(1.0 - beta1);
  a.omb2 = (float)(1.0 - beta2);
  a.bc1 = (float)(1.0 - std::pow(beta1, (double)step));
  a.sqrt_bc2 = (float)std::sqrt(1.0 - std::pow(beta2, (double)step));
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  for (int k = 0; k < ngroups; ++k) {
    AdamGroup g;
    g.param = groups[k].param; g.grad = groups[k].grad; g.m = groups[k].m; g.v = groups[k].v;
    g.count = groups[k].count; g.lr = groups[k].lr;
    g.period = groups[k].period; g.head = groups[k].head; g.lr_tail = groups[k].lr_tail;
    launch_adam(a, g, s);
  }
  return launched();
}

int hgs_grad_stats(int64_t n, const float *grad_ws, const hgs_projected *proj, float *accum, float *count,
                   hgs_stream_t stream) {
  if (n < 0 || (n > 0 && (!grad_ws || !proj || !proj->touched || !accum || !count))) return HGS_ERR_INVALID_ARG;
  launch_grad_stats(n, grad_ws, proj->touched, accum, count, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

int hgs_densify_workspace(int64_t n, size_t *bytes) {
  if (n < 0 || !bytes) return HGS_ERR_INVALID_ARG;
  *bytes = 256 + sizeof(int64_t) * 1024 + sizeof(int32_t) * (size_t)(n > 0 ? n : 1);
  return HGS_OK;
}

int hgs_densify_plan(const hgs_scene *scene, const float *accum, const float *count, const hgs_densify_cfg *cfg,
                     int32_t *actions, int64_t *offsets, void *ws, size_t ws_bytes, int64_t *d_new_n,
                     hgs_stream_t stream) {
  int st;
  if ((st = scene_ok(scene)) != HGS_OK) return st;
  if (!cfg || !offsets || !d_new_n) return HGS_ERR_INVALID_ARG;
  if (scene->n > 0 && (!accum || !count || !actions || !ws)) return HGS_ERR_INVALID_ARG;
  size_t need = 0;
  hgs_densify_workspace(scene->n, &need);
  if (scene->n > 0 && (ws_bytes < need || !aligned16(ws))) return HGS_ERR_INVALID_ARG;
  DensifyPlanArgs a;
  a.n = scene->n;
  a.grad_accum = accum; a.vis_count = count;
  a.log_scales = scene->log_scales; a.logits = scene->opacity_logits; a.types = scene->types;
  a.grad_thresh = cfg->grad_thresh; a.log_size_thresh = cfg->log_size_thresh;
  a.logit_min_opacity = cfg->logit_min_opacity;
  a.actions = actions;
  a.offsets = offsets;
  a.partial = reinterpret_cast<int64_t *>(static_cast<char *>(ws));
  a.counts = reinterpret_cast<int32_t *>(static_cast<char *>(ws) + 256 + sizeof(int64_t) * 1024);
  a.d_new_n = d_new_n;
  launch_densify_plan(a, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

static void train_arrays_k(const hgs_train_arrays *t, TrainArraysK *k) {
  k->means = t->means; k->log_scales = t->log_scales; k->quats = t->quats;
  k->logits = t->opacity_logits; k->sh = t->sh; k->types = t->types;
  for (int i = 0; i < 10; ++i) k->moments[i] = t->moments[i];
}

int hgs_densify_apply(int64_t n, int32_t sh_degree, const hgs_train_arrays *in, hgs_train_arrays *out,
                      const float *normals_z, const int32_t *actions, const int64_t *offsets,
                      hgs_stream_t stream) {
  if (n < 0 || sh_degree < 0 || sh_degree > 3 || !in || !out) return HGS_ERR_INVALID_ARG;
  if (n == 0) return HGS_OK;
  if (!normals_z || !actions || !offsets) return HGS_ERR_INVALID_ARG;
  const float *req_in[6] = {in->means, in->log_scales, in->quats, in->opacity_logits, in->sh,
                            reinterpret_cast<const float *>(in->types)};
  const float *req_out[6] = {out->means, out->log_scales, out->quats, out->opacity_logits, out->sh,
                             reinterpret_cast<const float *>(out->types)};
  for (int k = 0; k < 6; ++k)
    if (!req_in[k] || !req_out[k]) return HGS_ERR_INVALID_ARG;
  DensifyApplyArgs a;
  a.n = n;
  a.sh_floats = (sh_degree + 1) * (sh_degree + 1) * 3;
  train_arrays_k(in, &a.in);
  train_arrays_k(out, &a.out);
  a.normals_z = normals_z;
  a.actions = actions;
  a.offsets = offsets;
  launch_densify_apply(a, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

int hgs_reset_opacity(int64_t n, float *opacity_logits, float ceiling, float *m, float *v, hgs_stream_t stream) {
  if (n < 0 || (n > 0 && !opacity_logits) || !(ceiling > 0.0f && ceiling < 1.0f)) return HGS_ERR_INVALID_ARG;
  const float cap = (float)std::log((double)ceiling / (1.0 - (double)ceiling));
  launch_reset_opacity(n, opacity_logits, cap, m, v, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

}  // extern "C"

namespace {

struct BatchLayout {
  int64_t total_n;
  int TXmax, rows;
  size_t off_rec, off_key, off_rect, off_touched, off_tileset, off_vals, off_ranges, off_sort, bytes;
};

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

int batch_layout(int nreq, const hgs_request *reqs, int64_t capacity, BatchLayout *L) {
  if (nreq < 1 || nreq > HGS_MAX_BATCH || !reqs || capacity < 0 || capacity > kMaxCapacity)
    return HGS_ERR_INVALID_ARG;
  int64_t n = 0;
  int TXmax = 0, rows = 0;
  for (int r = 0; r < nreq; ++r) {
    const hgs_camera &c = reqs[r].cam;
    if (c.width <= 0 || c.height <= 0 || c.width > 16384 || c.height > 16384) return HGS_ERR_INVALID_ARG;
    if (reqs[r].scene.n < 0) return HGS_ERR_INVALID_ARG;
    n += reqs[r].scene.n;
    TXmax = std::max(TXmax, (c.width + kTile - 1) / kTile);
    rows += (c.height + kTile - 1) / kTile;
  }
  if (n >= (int64_t(1) << 31)) return HGS_ERR_INVALID_ARG;
  if (rows > 32767) return HGS_ERR_UNSUPPORTED;
  L->total_n = n;
  L->TXmax = TXmax;
  L->rows = rows;
  const size_t nn = (size_t)std::max<int64_t>(n, 1), cc = (size_t)std::max<int64_t>(capacity, 1);
  size_t off = 0;
  L->off_rec = off; off += al256(nn * kRecF4 * 16);
  L->off_key = off; off += al256(nn * 4);
  L->off_rect = off; off += al256(nn * 8);
  L->off_touched = off; off += al256(nn * 4);
  L->off_tileset = off; off += al256(nn * 48);
  L->off_vals = off; off += al256(cc * 4);
  L->off_ranges = off; off += al256((size_t)TXmax * rows * 8);
  L->off_sort = off;
  BinWorkspace w;
  off += al256(bin_layout(nullptr, n, capacity, &w));
  L->bytes = off;
  return HGS_OK;
}

}  // namespace

extern "C" {

int hgs_render_batch_workspace(int nreq, const hgs_request *reqs, int64_t capacity, size_t *bytes) {
  if (!bytes) return HGS_ERR_INVALID_ARG;
  BatchLayout L;
  const int st = batch_layout(nreq, reqs, capacity, &L);
  if (st != HGS_OK) return st;
  *bytes = L.bytes;
  return HGS_OK;
}

int hgs_render_batch(int nreq, const hgs_request *reqs, const hgs_config *cfg, void *ws, size_t ws_bytes,
                     int64_t capacity, int64_t *d_count, int32_t *dev_err, hgs_stream_t stream) {
  int st;
  BatchLayout L;
  if ((st = batch_layout(nreq, reqs, capacity, &L)) != HGS_OK) return st;
  CfgK fk;
  if ((st = cfg_to_kernel(cfg, &fk)) != HGS_OK) return st;
  if (!ws || !aligned16(ws) || ws_bytes < L.bytes || !d_count) return HGS_ERR_INVALID_ARG;
  char *base = static_cast<char *>(ws);
  float *rec = reinterpret_cast<float *>(base + L.off_rec);
  uint32_t *key = reinterpret_cast<uint32_t *>(base + L.off_key);
  uint16_t *rect = reinterpret_cast<uint16_t *>(base + L.off_rect);
  uint32_t *touched = reinterpret_cast<uint32_t *>(base + L.off_touched);
  float *tileset = reinterpret_cast<float *>(base + L.off_tileset);
  uint32_t *vals = reinterpret_cast<uint32_t *>(base + L.off_vals);
  uint32_t *ranges = reinterpret_cast<uint32_t *>(base + L.off_ranges);
  BatchPrepArgs bp;
  BatchRenderArgs br;
  bp.nreq = br.nreq = nreq;
  br.TXmax = L.TXmax;
  int64_t prim = 0;
  int row = 0;
  for (int r = 0; r < nreq; ++r) {
    const hgs_request &q = reqs[r];
    if ((st = scene_ok(&q.scene)) != HGS_OK) return st;
    CamK ck;
    if ((st = cam_to_kernel(&q.cam, &ck)) != HGS_OK) return st;
    const hgs_image &o = q.out;
    if (!o.rgb || !o.depth || !o.normal || !o.alpha || !o.T_final || !o.n_last) return HGS_ERR_INVALID_ARG;
    hgs_projected p;
    p.rec = rec + (size_t)prim * kRecF4 * 4;
    p.depth_key = key + prim;
    p.rect = rect + (size_t)prim * 4;
    p.touched = touched + prim;
    p.tileset = tileset + (size_t)prim * 12;
    bp.req[r] = prep_args(&q.scene, ck, fk, &p);
    bp.deg[r] = q.scene.sh_degree;
    bp.row_off[r] = row;
    bp.base[r] = prim;
    RenderArgs &a = br.req[r];
    a.rec = rec;  // records are addressed by their combined row
    a.vals = vals;
    a.ranges = ranges;
    a.cam = ck;
    a.cfg = fk;
    a.rgb = o.rgb; a.depth = o.depth; a.normal = o.normal; a.alpha = o.alpha;
    a.T_final = o.T_final; a.n_last = o.n_last; a.n_contrib = o.n_contrib;
    a.tile_sched = nullptr;
    br.row_off[r] = row;
    prim += q.scene.n;
    row += ck.TY;
  }
  bp.base[nreq] = prim;
  br.row_off[nreq] = row;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  launch_preprocess_batch(bp, s);
  BinWorkspace w;
  bin_layout(base + L.off_sort, L.total_n, capacity, &w);
  BinArgs b;
  b.n = L.total_n;
  b.capacity = capacity;
  b.tiles = L.TXmax * L.rows;
  b.tile_bits = tile_bits_for(b.tiles);
  b.TX = L.TXmax;
  b.depth_key = key;
  b.touched = touched;
  b.rect = rect;
  b.tileset = tileset;
  b.vals = vals;
  b.keys = nullptr;
  b.ranges = ranges;
  b.d_count = d_count;
  b.dev_err = dev_err;
  launch_bin_sort(b, w, s);
  launch_render_batch(br, L.rows, s);
  return launched();
}

int hgs_exchange_types(hgs_scene_mut *scene, const hgs_exchange_cfg *xcfg, int64_t *d_n_flipped,
                       int32_t *dev_err, hgs_stream_t stream) {
  (void)dev_err;
  if (!scene || !xcfg || scene->n < 0) return HGS_ERR_INVALID_ARG;
  if (xcfg->mode != HGS_EXCHANGE_ERANK && xcfg->mode != HGS_EXCHANGE_MASK) return HGS_ERR_INVALID_ARG;
  if (scene->n == 0) return HGS_OK;
  if (!scene->log_scales || !scene->quats || !scene->types || !aligned16(scene->quats))
    return HGS_ERR_INVALID_ARG;
  if (xcfg->mode == HGS_EXCHANGE_MASK && !xcfg->mask) return HGS_ERR_INVALID_ARG;
  if (xcfg->mode == HGS_EXCHANGE_ERANK && !(xcfg->theta_e > 0.f)) return HGS_ERR_INVALID_ARG;
  ExchangeArgs a;
  a.log_scales = scene->log_scales;
  a.quats = scene->quats;
  a.types = scene->types;
  a.n = scene->n;
  a.mode = xcfg->mode;
  a.theta = xcfg->theta_e;
  a.mask = xcfg->mask;
  a.n_flipped = reinterpret_cast<unsigned long long *>(d_n_flipped);
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  if (d_n_flipped) cudaMemsetAsync(d_n_flipped, 0, sizeof(int64_t), s);
  launch_exchange(a, s);
  return launched();
}

int hgs_fp32_probe(int32_t blocks, int32_t iters, float *d_out, double *flops, hgs_stream_t stream) {
  if (blocks < 1 || iters < 1 || !d_out || !flops) return HGS_ERR_INVALID_ARG;
  launch_alu_probe(HGS_PROBE_FFMA, blocks, iters, d_out, flops, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

int hgs_alu_probe(int32_t kind, int32_t blocks, int32_t iters, float *d_out, double *ops, hgs_stream_t stream) {
  if (kind < HGS_PROBE_FFMA || kind > HGS_PROBE_RCP) return HGS_ERR_INVALID_ARG;
  if (blocks < 1 || iters < 1 || !d_out || !ops) return HGS_ERR_INVALID_ARG;
  launch_alu_probe(kind, blocks, iters, d_out, ops, reinterpret_cast<cudaStream_t>(stream));
  return launched();
}

}  // extern "C"
