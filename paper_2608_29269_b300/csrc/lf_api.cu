// C ABI of the surfel ray tracer: context, scene/BVH management, environment
// tables and the render / adjoint entry points.  Every call validates its
// arguments before enqueuing anything and reports failures as lf_status.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "lf_ctx.h"
#include "lf_wavefront.h"

using namespace lf;

namespace {

lf_status fail(lf_ctx* c, lf_status s, const std::string& msg) {
  if (c) c->err = msg;
  return s;
}

lf_status cuda_fail(lf_ctx* c, cudaError_t e, const char* where) {
  return fail(c, LF_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define LF_CUDA(c, expr)                                         \
  do {                                                           \
    cudaError_t e__ = (expr);                                    \
    if (e__ != cudaSuccess) return cuda_fail((c), e__, #expr);   \
  } while (0)

template <class T>
cudaError_t dev_alloc(T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  return cudaMalloc(reinterpret_cast<void**>(p), sizeof(T) * count);
}

template <class T>
void dev_free(T*& p) {
  if (p) cudaFree(p);
  p = nullptr;
}

void free_scene_storage(lf_ctx* c) {
  dev_free(c->geo); dev_free(c->mat); dev_free(c->nodes); dev_free(c->leaf_parent); dev_free(c->node_parent);
  dev_free(c->flags); dev_free(c->keys); dev_free(c->vals); dev_free(c->keys_alt); dev_free(c->vals_alt);
  dev_free(c->counts); dev_free(c->node_range); dev_free(c->wnodes); dev_free(c->wsrc); dev_free(c->wqueue);
  c->cap_n = 0;
  c->wcap = 0;
}

// Camera basis in FP64: f = normalize(target - eye), r = normalize(f x up),
// u = r x f; th = tan(fovy / 2).
CamDev to_cam(const lf_camera& c) {
  double e[3] = {c.eye[0], c.eye[1], c.eye[2]};
  double f[3] = {(double)c.target[0] - e[0], (double)c.target[1] - e[1], (double)c.target[2] - e[2]};
  double fl = std::sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
  for (double& v : f) v = v / fl;
  double up[3] = {c.up[0], c.up[1], c.up[2]};
  double r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
  double rl = std::sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
  for (double& v : r) v = v / rl;
  double u[3] = {r[1] * f[2] - r[2] * f[1], r[2] * f[0] - r[0] * f[2], r[0] * f[1] - r[1] * f[0]};
  CamDev d;
  d.eye = make_float3(c.eye[0], c.eye[1], c.eye[2]);
  for (int k = 0; k < 3; ++k) { d.f[k] = f[k]; d.r[k] = r[k]; d.u[k] = u[k]; }
  d.th = std::tan(0.5 * (double)c.fovy_deg * 3.14159265358979323846 / 180.0);
  d.aspect = (double)c.width / (double)c.height;
  d.W = c.width;
  d.H = c.height;
  return d;
}

bool cam_ok(const lf_camera* c) {
  if (!c || c->width <= 0 || c->height <= 0) return false;
  if ((long long)c->width * c->height > (1LL << 30)) return false;
  if (!(c->fovy_deg > 0.0f && c->fovy_deg < 179.0f)) return false;
  double f[3] = {c->target[0] - c->eye[0], c->target[1] - c->eye[1], c->target[2] - c->eye[2]};
  double r[3] = {f[1] * c->up[2] - f[2] * c->up[1], f[2] * c->up[0] - f[0] * c->up[2],
                 f[0] * c->up[1] - f[1] * c->up[0]};
  return (f[0] * f[0] + f[1] * f[1] + f[2] * f[2]) > 0 && (r[0] * r[0] + r[1] * r[1] + r[2] * r[2]) > 0;
}

DevParams to_dev(const lf_params& p) {
  return DevParams{p.T_min, p.alpha_min, p.alpha_max, p.support_r2, p.eps_w, p.t_min, p.ray_offset, p.p_spec,
                   p.max_rounds, p.brdf_mode, p.sampling_mode, p.sampler};
}

}  // namespace

lf_status lf_ctx_fit(lf_ctx* c, int first_obj, int last_obj) {
  const int first_leaf = c->offsets[first_obj], last_leaf = c->offsets[last_obj + 1];
  const int n0 = c->node_off_h[first_obj], n1 = c->node_off_h[last_obj + 1];
  if (n1 > n0) LF_CUDA(c, cudaMemsetAsync(c->flags + n0, 0, sizeof(int) * (n1 - n0), c->stream));
  FitArgs a;
  a.first_leaf = first_leaf;
  a.n_leaves = last_leaf - first_leaf;
  a.n_obj = c->n_obj;
  a.leaf_off = c->offsets_dev;
  a.node_off = c->node_off_dev;
  a.sorted_ids = c->vals;
  a.geo = c->geo;
  a.mat = c->mat;
  a.nodes = c->nodes;
  a.flags = c->flags;
  a.leaf_parent = c->leaf_parent;
  a.node_parent = c->node_parent;
  a.insts = c->insts_dev;
  a.R = std::sqrt(c->params.support_r2);
  a.status = c->status_dev;
  LF_CUDA(c, launch_pack_fit(c->scene, a, c->stream));
  const int w0 = c->wnode_off_h[first_obj], w1 = c->wnode_off_h[last_obj + 1];
  if (w1 > w0) {
    WideArgs w = lf_ctx_wide_args(c);
    w.first_slot = WIDE * w0;
    LF_CUDA(c, launch_wide_boxes(w, WIDE * (w1 - w0), c->stream));
  }
  return LF_OK;
}

WideArgs lf_ctx_wide_args(lf_ctx* c) {
  WideArgs w;
  w.n_obj_total = c->n_obj;
  w.leaf_off = c->offsets_dev;
  w.node_off = c->node_off_dev;
  w.wnode_off = c->wnode_off_dev;
  w.node_range = c->node_range;
  w.nodes = c->nodes;
  w.wnodes = c->wnodes;
  w.wsrc = c->wsrc;
  w.wqueue = c->wqueue;
  w.status = c->status_dev;
  return w;
}

TraceArgs lf_ctx_trace_args(lf_ctx* c, int env_id) {
  TraceArgs a;
  a.insts = c->insts_dev;
  a.n_inst = c->n_obj;
  a.P = c->dp;
  const EnvSlot& e = c->env[env_id];
  a.env.rgb = e.rgb;
  a.env.pmf_row = e.tables;
  a.env.cdf_row = e.tables + e.H;
  a.env.pmf_col = e.tables + 2 * e.H;
  a.env.cdf_col = e.tables + 2 * e.H + (size_t)e.H * e.W;
  a.env.cdf_row_lo = e.tables + 2 * e.H + 2 * (size_t)e.H * e.W;
  a.env.cdf_col_lo = e.tables + 3 * e.H + 2 * (size_t)e.H * e.W;
  a.env.H = e.H;
  a.env.W = e.W;
  a.status = c->status_dev;
  a.counters = c->counters;
  return a;
}

CamDev lf_ctx_cam(const lf_camera& c) { return to_cam(c); }

// R must be a rotation (R R^T = I, det = +1, within FP32 tolerance) and t finite.
bool lf_is_rigid(const float R[9], const float t[3]) {
  double dmax = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int m = 0; m < 3; ++m) s += (double)R[3 * i + m] * R[3 * j + m];
      dmax = std::max(dmax, std::fabs(s - (i == j ? 1.0 : 0.0)));
    }
  double det = (double)R[0] * (R[4] * R[8] - R[5] * R[7]) - (double)R[1] * (R[3] * R[8] - R[5] * R[6]) +
               (double)R[2] * (R[3] * R[7] - R[4] * R[6]);
  return dmax < 1e-4 && std::fabs(det - 1.0) < 1e-4 && (!t || (std::isfinite(t[0]) && std::isfinite(t[1]) &&
                                                             std::isfinite(t[2])));
}

extern "C" {

lf_status lf_params_default(lf_params* p) {
  if (!p) return LF_ERR_INVALID;
  p->T_min = 1e-4f;
  p->alpha_min = 1.0f / 255.0f;
  p->alpha_max = 0.99f;
  p->support_r2 = 9.0f;
  p->eps_w = 1e-8f;
  p->t_min = 1e-4f;
  p->ray_offset = 1e-3f;
  p->p_spec = 0.5f;
  p->max_rounds = 64;
  p->brdf_mode = 0;
  p->sampling_mode = 0;
  p->sampler = 0;
  return LF_OK;
}

lf_status lf_create(const lf_params* params, void* stream, lf_ctx** out) {
  if (!out) return LF_ERR_INVALID;
  lf_params p;
  if (params) p = *params; else lf_params_default(&p);
  if (!(p.T_min >= 0.0f && p.alpha_min >= 0.0f && p.alpha_max > 0.0f && p.alpha_max < 1.0f &&
        p.support_r2 > 0.0f && p.eps_w >= 0.0f && p.t_min >= 0.0f && p.p_spec >= 0.0f && p.p_spec <= 1.0f &&
        p.max_rounds > 0 && (p.brdf_mode == 0 || p.brdf_mode == 1) && p.sampling_mode >= 0 &&
        p.sampling_mode <= 2 && (p.sampler == 0 || p.sampler == 1)))
    return LF_ERR_INVALID;
  lf_ctx* c = new lf_ctx();
  c->params = p;
  c->dp = to_dev(p);
  c->stream = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaGetDevice(&c->device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device);
  if (e == cudaSuccess) lf_static_scratch_forget(c->device);
  if (e == cudaSuccess) e = dev_alloc(&c->status_dev, 1);
  if (e == cudaSuccess) e = dev_alloc(&c->loss_dev, 1);
  if (e == cudaSuccess) e = cudaMemset(c->status_dev, 0, sizeof(int));
  if (e == cudaSuccess) e = dev_alloc(&c->offsets_dev, LF_MAX_OBJECTS + 1);
  if (e == cudaSuccess) e = dev_alloc(&c->node_off_dev, LF_MAX_OBJECTS + 1);
  if (e == cudaSuccess) e = dev_alloc(&c->wnode_off_dev, LF_MAX_OBJECTS + 1);
  if (e == cudaSuccess) e = dev_alloc(&c->bounds, 6 * LF_MAX_OBJECTS);
  if (e == cudaSuccess) e = dev_alloc(&c->insts_dev, LF_MAX_OBJECTS);
  if (e != cudaSuccess) {
    lf_destroy(c);
    return e == cudaErrorMemoryAllocation ? LF_ERR_OOM : LF_ERR_CUDA;
  }
  *out = c;
  return LF_OK;
}

lf_status lf_destroy(lf_ctx* c) {
  if (!c) return LF_ERR_INVALID;
  if (c->stream) cudaStreamSynchronize(c->stream); else cudaDeviceSynchronize();
  free_scene_storage(c);
  dev_free(c->status_dev); dev_free(c->loss_dev); dev_free(c->offsets_dev); dev_free(c->node_off_dev); dev_free(c->wnode_off_dev);
  dev_free(c->bounds);
  dev_free(c->insts_dev);
  for (EnvSlot& e : c->env) { dev_free(e.tables); dev_free(e.rowsum); dev_free(e.sin_row); }
  for (cudaEvent_t& e : c->prof_ev)
    if (e) cudaEventDestroy(e);
  delete c;
  return LF_OK;
}

lf_status lf_set_stream(lf_ctx* c, void* stream) {
  if (!c) return LF_ERR_INVALID;
  c->stream = static_cast<cudaStream_t>(stream);
  return LF_OK;
}

const char* lf_last_error(const lf_ctx* c) { return c ? c->err.c_str() : "null context"; }

lf_status lf_sync(lf_ctx* c) {
  if (!c) return LF_ERR_INVALID;
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  int st = 0;
  LF_CUDA(c, cudaMemcpy(&st, c->status_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (st != 0) {
    LF_CUDA(c, cudaMemset(c->status_dev, 0, sizeof(int)));
    return fail(c, (lf_status)st, st == LF_ERR_STACK ? "traversal stack overflow"
                                   : st == LF_ERR_ROUND_LIMIT ? "k-buffer round limit reached"
                                   : st == LF_ERR_BOUNDS      ? "device bounds check failed (see the printed index)"
                                                              : "device error");
  }
  return LF_OK;
}

lf_status lf_profile(lf_ctx* c, int enable) {
  if (!c) return LF_ERR_INVALID;
  if (enable && !c->prof_ev[0])
    for (cudaEvent_t& e : c->prof_ev) LF_CUDA(c, cudaEventCreate(&e));
  c->profile = enable != 0;
  return LF_OK;
}

lf_status lf_profile_read(lf_ctx* c, float* ms) {
  if (!c || !ms) return LF_ERR_INVALID;
  if (!c->prof_ev[0]) return fail(c, LF_ERR_NOT_BUILT, "profiling was never enabled");
  // primary, gen, NEE shadow, continuation, secondary shadow, count + combine;
  // shading adjoint, trace backward (0 until a profiled lf_trace_backward)
  const int a[8] = {0, 2, 3, 4, 5, 6, 8, 9}, b[8] = {1, 3, 4, 5, 6, 7, 9, 10};
  for (int i = 0; i < 8; ++i) {
    if (i >= 6 && !c->prof_bwd) {
      ms[i] = 0.0f;
      continue;
    }
    LF_CUDA(c, cudaEventSynchronize(c->prof_ev[b[i]]));
    LF_CUDA(c, cudaEventElapsedTime(ms + i, c->prof_ev[a[i]], c->prof_ev[b[i]]));
  }
  return LF_OK;
}

lf_status lf_set_counters(lf_ctx* c, unsigned long long* counters) {
  if (!c) return LF_ERR_INVALID;
  c->counters = counters;
  return LF_OK;
}

lf_status lf_bvh_build(lf_ctx* c, const lf_scene* s) {
  if (!c || !s) return LF_ERR_INVALID;
  if (s->n < 0 || s->n >= (1 << 24) || s->n_objects < 1 || s->n_objects > LF_MAX_OBJECTS || !s->object_offsets)
    return fail(c, LF_ERR_INVALID, "bad surfel or object count");
  if (s->n > 0 && (!s->mu_dev || !s->tu_dev || !s->tv_dev || !s->scale_dev || !s->opacity_dev || !s->albedo_dev ||
                   !s->metallic_dev || !s->roughness_dev))
    return fail(c, LF_ERR_INVALID, "null scene array");
  if (s->object_offsets[0] != 0 || s->object_offsets[s->n_objects] != s->n)
    return fail(c, LF_ERR_INVALID, "object offsets must run from 0 to n");
  int max_obj_n = 0;
  for (int k = 0; k < s->n_objects; ++k) {
    const int nk = s->object_offsets[k + 1] - s->object_offsets[k];
    if (nk < 0) return fail(c, LF_ERR_INVALID, "object offsets must be non-decreasing");
    max_obj_n = std::max(max_obj_n, nk);
  }
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  c->built = false;
  const int n = s->n, n_obj = s->n_objects;
  if ((size_t)n > c->cap_n) {
    free_scene_storage(c);
    const size_t cap = (size_t)n + (size_t)n / 8 + 64;
    const size_t tiles = (size_t)radix_tiles((int)cap) + 1;
    cudaError_t e = dev_alloc(&c->geo, (size_t)GEO * cap);
    if (e == cudaSuccess) e = dev_alloc(&c->mat, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->nodes, 4 * cap);
    if (e == cudaSuccess) e = dev_alloc(&c->leaf_parent, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->node_parent, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->flags, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->keys, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->vals, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->keys_alt, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->vals_alt, cap);
    if (e == cudaSuccess) e = dev_alloc(&c->counts, 256 * tiles);
    if (e == cudaSuccess) e = dev_alloc(&c->node_range, cap);
    // wide nodes: the sum over objects of wide_capacity(n_k) is at most wide_capacity(cap) + 2 LF_MAX_OBJECTS
    const size_t wcap = (size_t)wide_capacity((int)std::min<size_t>(cap, 1u << 30)) + 2 * LF_MAX_OBJECTS;
    if (e == cudaSuccess) e = dev_alloc(&c->wnodes, WNODE_Q * wcap);
    if (e == cudaSuccess) e = dev_alloc(&c->wsrc, WIDE * wcap);
    if (e == cudaSuccess) e = dev_alloc(&c->wqueue, wcap);
    c->wcap = wcap;
    if (e != cudaSuccess) {
      free_scene_storage(c);
      return fail(c, e == cudaErrorMemoryAllocation ? LF_ERR_OOM : LF_ERR_CUDA, "BVH storage allocation failed");
    }
    c->cap_n = cap;
  }
  c->scene = SceneDev{s->mu_dev, s->tu_dev, s->tv_dev, s->scale_dev, s->opacity_dev, s->albedo_dev,
                      s->metallic_dev, s->roughness_dev, n};
  c->n = n;
  c->n_obj = n_obj;
  c->offsets.assign(s->object_offsets, s->object_offsets + n_obj + 1);
  c->node_off_h.assign(n_obj + 1, 0);
  for (int k = 0; k < n_obj; ++k)
    c->node_off_h[k + 1] = c->node_off_h[k] + std::max(0, c->offsets[k + 1] - c->offsets[k] - 1);
  c->n_nodes = c->node_off_h[n_obj];
  c->wnode_off_h.assign(n_obj + 1, 0);
  for (int k = 0; k < n_obj; ++k)
    c->wnode_off_h[k + 1] = c->wnode_off_h[k] + wide_capacity(c->offsets[k + 1] - c->offsets[k]);
  LF_CUDA(c, cudaMemcpyAsync(c->offsets_dev, c->offsets.data(), sizeof(int) * (n_obj + 1), cudaMemcpyHostToDevice,
                             c->stream));
  LF_CUDA(c, cudaMemcpyAsync(c->node_off_dev, c->node_off_h.data(), sizeof(int) * (n_obj + 1),
                             cudaMemcpyHostToDevice, c->stream));
  LF_CUDA(c, cudaMemcpyAsync(c->wnode_off_dev, c->wnode_off_h.data(), sizeof(int) * (n_obj + 1),
                             cudaMemcpyHostToDevice, c->stream));
  // instance table (boxes are written by the fit)
  c->insts_h.assign(n_obj, Inst{});
  for (int k = 0; k < n_obj; ++k) {
    Inst& I = c->insts_h[k];
    const int nk = c->offsets[k + 1] - c->offsets[k];
    for (int a = 0; a < 3; ++a) { I.lo[a] = 1.0f; I.hi[a] = -1.0f; }
    I.root = nk >= 2 ? 0 : (nk == 1 ? ~0 : INT_MIN);
    I.n_leaves = nk;
    I.nodes = c->nodes + 4 * (size_t)c->node_off_h[k];
    I.geo = c->geo + (size_t)GEO * c->offsets[k];
    I.mat = c->mat + (size_t)c->offsets[k];
    I.id_base = c->offsets[k];
    I.n_wide = c->wnode_off_h[k + 1] - c->wnode_off_h[k];
    I.wnodes = c->wnodes + WNODE_Q * (size_t)c->wnode_off_h[k];
    I.wroot = nk > WLEAF ? 0 : (nk >= 1 ? ~0 : INT_MIN);
    I.wroot_count = nk > WLEAF ? 0 : nk;
  }
  LF_CUDA(c, cudaMemcpyAsync(c->insts_dev, c->insts_h.data(), sizeof(Inst) * n_obj, cudaMemcpyHostToDevice,
                             c->stream));
  if (n > 0) {
    LF_CUDA(c, launch_object_bounds(c->scene, c->offsets_dev, n_obj, max_obj_n, c->bounds, c->stream));
    LF_CUDA(c, launch_morton(c->scene, c->offsets_dev, n_obj, c->bounds, c->keys, c->vals, c->stream));
    LF_CUDA(c, launch_radix_sort(c->keys, c->vals, c->keys_alt, c->vals_alt, n, c->offsets_dev, n_obj, c->counts,
                                 c->stream));
    LF_CUDA(c, cudaMemsetAsync(c->leaf_parent, 0xff, sizeof(int) * (size_t)n, c->stream));
    LF_CUDA(c, cudaMemsetAsync(c->node_parent, 0xff, sizeof(int) * (size_t)n, c->stream));
    LF_CUDA(c, launch_hierarchy(c->keys, c->offsets_dev, c->node_off_dev, n_obj, c->n_nodes, c->nodes,
                                c->leaf_parent, c->node_parent, c->node_range, c->stream));
    const int n_wide = c->wnode_off_h[n_obj];
    if (n_wide > 0) LF_CUDA(c, cudaMemsetAsync(c->wsrc, 0xff, sizeof(int) * WIDE * (size_t)n_wide, c->stream));
    lf_status st = lf_ctx_fit(c, 0, n_obj - 1);  // binary boxes (no wide slots yet)
    if (st != LF_OK) return st;
    if (n_wide > 0) {  // collapse by box surface, then the wide boxes
      WideArgs w = lf_ctx_wide_args(c);
      w.first_obj = 0;
      w.n_objs = n_obj;
      LF_CUDA(c, launch_collapse(w, c->stream));
      w = lf_ctx_wide_args(c);
      LF_CUDA(c, launch_wide_boxes(w, WIDE * n_wide, c->stream));
    }
  }
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  c->built = true;
  const lf_status st = lf_sync(c);
  if (st != LF_OK) c->built = false;  // a malformed hierarchy is never traced
  return st;
}

lf_status lf_bvh_refit(lf_ctx* c, int k, const float R[9], const float t[3]) {
  if (!c || !R || !t) return LF_ERR_INVALID;
  if (!c->built) return fail(c, LF_ERR_NOT_BUILT, "no BVH");
  if (k < 0 || k >= c->n_obj) return fail(c, LF_ERR_INVALID, "bad object id");
  if (!lf_is_rigid(R, t)) return fail(c, LF_ERR_INVALID, "transform is not rigid");
  Mat34 T;
  std::memcpy(T.R, R, sizeof(T.R));
  std::memcpy(T.t, t, sizeof(T.t));
  LF_CUDA(c, launch_rigid(c->scene, c->offsets[k], c->offsets[k + 1], T, c->stream));
  return lf_ctx_fit(c, k, k);
}

lf_status lf_scene_sync(lf_ctx* c, int k) {
  if (!c) return LF_ERR_INVALID;
  if (!c->built) return fail(c, LF_ERR_NOT_BUILT, "no BVH");
  if (k < -1 || k >= c->n_obj) return fail(c, LF_ERR_INVALID, "bad object id");
  return k < 0 ? lf_ctx_fit(c, 0, c->n_obj - 1) : lf_ctx_fit(c, k, k);
}

lf_status lf_material_set(lf_ctx* c, int k, const float* rgb, float metallic, float roughness) {
  if (!c) return LF_ERR_INVALID;
  if (!c->built) return fail(c, LF_ERR_NOT_BUILT, "no BVH");
  if (k < 0 || k >= c->n_obj) return fail(c, LF_ERR_INVALID, "bad object id");
  if (metallic > 1.0f || roughness > 1.0f) return fail(c, LF_ERR_INVALID, "metallic/roughness above 1");
  float3 col = make_float3(0.f, 0.f, 0.f);
  if (rgb) col = make_float3(rgb[0], rgb[1], rgb[2]);
  LF_CUDA(c, launch_material(c->scene, c->offsets[k], c->offsets[k + 1], col, rgb ? 1 : 0, metallic, roughness,
                             c->stream));
  return lf_ctx_fit(c, k, k);
}

lf_status lf_env_set(lf_ctx* c, int id, const float* rgb, int H, int W) {
  if (!c) return LF_ERR_INVALID;
  if (id < 0 || id >= LF_MAX_ENVS || !rgb || H <= 0 || W <= 0 || (long long)H * W > (1LL << 26))
    return fail(c, LF_ERR_INVALID, "bad environment map");
  EnvSlot& e = c->env[id];
  const size_t need = 3 * (size_t)H + 3 * (size_t)H * W;  // + the CDFs' low parts
  if (need > e.cap || H > e.cap_h) {
    dev_free(e.tables); dev_free(e.rowsum); dev_free(e.sin_row);
    cudaError_t err = dev_alloc(&e.tables, need);
    if (err == cudaSuccess) err = dev_alloc(&e.rowsum, H);
    if (err == cudaSuccess) err = dev_alloc(&e.sin_row, H);
    if (err != cudaSuccess) {
      e.cap = 0; e.cap_h = 0; e.set = false;
      return fail(c, err == cudaErrorMemoryAllocation ? LF_ERR_OOM : LF_ERR_CUDA, "env table allocation failed");
    }
    e.cap = need;
    e.cap_h = H;
  }
  // sin(theta) at the row centres, computed on the host once per map.
  e.sin_host.resize(H);
  const double PI = 3.14159265358979323846;
  for (int r = 0; r < H; ++r) e.sin_host[r] = std::sin(PI * ((double)r + 0.5) / (double)H);
  LF_CUDA(c, cudaMemcpyAsync(e.sin_row, e.sin_host.data(), sizeof(double) * H, cudaMemcpyHostToDevice, c->stream));
  e.rgb = rgb;
  e.H = H;
  e.W = W;
  LF_CUDA(c, launch_env_tables(rgb, e.sin_row, H, W, e.rowsum, e.tables, e.tables + H, e.tables + 2 * H,
                               e.tables + 2 * H + (size_t)H * W, e.tables + 2 * H + 2 * (size_t)H * W,
                               e.tables + 3 * H + 2 * (size_t)H * W, c->stream));
  // the host sin table must outlive the asynchronous copy
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  e.set = true;
  return LF_OK;
}

lf_status lf_env_tables(lf_ctx* c, int id, float* pmf_row, float* cdf_row, float* pmf_col, float* cdf_col) {
  if (!c) return LF_ERR_INVALID;
  if (id < 0 || id >= LF_MAX_ENVS || !c->env[id].set) return fail(c, LF_ERR_NOT_BUILT, "environment not set");
  const EnvSlot& e = c->env[id];
  const size_t H = e.H, HW = (size_t)e.H * e.W;
  float* dst[4] = {pmf_row, cdf_row, pmf_col, cdf_col};
  const float* src[4] = {e.tables, e.tables + H, e.tables + 2 * H, e.tables + 2 * H + HW};
  const size_t cnt[4] = {H, H, HW, HW};
  for (int i = 0; i < 4; ++i)
    if (dst[i]) LF_CUDA(c, cudaMemcpyAsync(dst[i], src[i], sizeof(float) * cnt[i], cudaMemcpyDeviceToDevice, c->stream));
  return LF_OK;
}

static lf_status check_render(lf_ctx* c, const lf_camera* cam, int env_id) {
  if (!c) return LF_ERR_INVALID;
  if (!cam_ok(cam)) return fail(c, LF_ERR_INVALID, "bad camera");
  if (!c->built) return fail(c, LF_ERR_NOT_BUILT, "no BVH");
  if (env_id < 0 || env_id >= LF_MAX_ENVS || !c->env[env_id].set)
    return fail(c, LF_ERR_NOT_BUILT, "environment not set");
  return LF_OK;
}

lf_status lf_trace_primary(lf_ctx* c, const lf_camera* cam, int env_id, float* gbuf) {
  lf_status st = check_render(c, cam, env_id);
  if (st != LF_OK) return st;
  if (!gbuf) return fail(c, LF_ERR_INVALID, "null G-buffer");
  if (c->profile) LF_CUDA(c, cudaEventRecord(c->prof_ev[0], c->stream));
  LF_CUDA(c, launch_trace_primary(lf_ctx_trace_args(c, env_id), to_cam(*cam), gbuf, c->stream));
  if (c->profile) LF_CUDA(c, cudaEventRecord(c->prof_ev[1], c->stream));
  return LF_OK;
}

// One-job shading batch over the context's scene.
static ShadeBatch one_job(lf_ctx* c, const lf_camera* cam, const float* gbuf, int env_id, int spp, uint64_t seed,
                          float* rgb) {
  ShadeBatch B;
  B.n_jobs = 1;
  const int P = cam->width * cam->height;
  B.n_items = (long long)P * spp;
  B.n_pix_total = P;
  ShadeJob& J = B.jobs[0];
  const TraceArgs a = lf_ctx_trace_args(c, env_id);
  J.insts = a.insts;
  J.n_inst = a.n_inst;
  J.env = a.env;
  J.gbuf = gbuf;
  J.n_pix = P;
  J.rgb = rgb;
  J.spp = spp;
  J.k0 = (uint32_t)(seed & 0xffffffffu);
  J.k1 = (uint32_t)(seed >> 32);
  J.item0 = 0;
  J.pix0 = 0;
  return B;
}

size_t lf_shade_scratch_bytes(int width, int height, int spp) {
  if (width <= 0 || height <= 0 || spp <= 0) return 0;
  return sample_buf_bytes((long long)width * height * spp);
}

lf_status lf_shade_bounce(lf_ctx* c, const lf_camera* cam, const float* gbuf, int env_id, int spp, uint64_t seed,
                          float* rgb, unsigned long long* ray_count, void* samples, size_t samples_bytes) {
  lf_status st = check_render(c, cam, env_id);
  if (st != LF_OK) return st;
  if (!gbuf || !rgb || spp <= 0 || spp > (1 << 20)) return fail(c, LF_ERR_INVALID, "bad shading arguments");
  if ((long long)cam->width * cam->height * spp >= (1LL << 30)) return fail(c, LF_ERR_INVALID, "too many samples");
  if (!samples || samples_bytes < lf_shade_scratch_bytes(cam->width, cam->height, spp))
    return fail(c, LF_ERR_INVALID, "sample buffer too small");
  const ShadeBatch B = one_job(c, cam, gbuf, env_id, spp, seed, rgb);
  const SampleBuf S = sample_buf(samples, B.n_items);
  LF_CUDA(c, launch_shade_wavefront(B, c->dp, S, c->status_dev, ray_count, c->counters, c->sms, c->stream,
                                    c->profile ? c->prof_ev + 2 : nullptr));
  LF_CUDA(c, launch_shade_combine(B, c->dp, S, c->stream));
  if (c->profile) LF_CUDA(c, cudaEventRecord(c->prof_ev[7], c->stream));
  return LF_OK;
}

lf_status lf_shade_sample_terms(lf_ctx* c, const lf_camera* cam, const float* gbuf, int env_id, int spp,
                                const void* samples, size_t samples_bytes, float* terms) {
  lf_status st = check_render(c, cam, env_id);
  if (st != LF_OK) return st;
  if (!gbuf || !terms || spp <= 0 || spp > (1 << 20)) return fail(c, LF_ERR_INVALID, "bad arguments");
  if ((long long)cam->width * cam->height * spp >= (1LL << 30)) return fail(c, LF_ERR_INVALID, "too many samples");
  if (!samples || samples_bytes < lf_shade_scratch_bytes(cam->width, cam->height, spp))
    return fail(c, LF_ERR_INVALID, "sample buffer too small");
  const ShadeBatch B = one_job(c, cam, gbuf, env_id, spp, 0, nullptr);
  const SampleBuf S = sample_buf(const_cast<void*>(samples), B.n_items);
  LF_CUDA(c, launch_shade_terms(B, c->dp, S, terms, c->sms, c->stream));
  return LF_OK;
}

size_t lf_backward_scratch_bytes(int width, int height, int spp) {
  if (width <= 0 || height <= 0 || spp <= 0) return 0;
  return sizeof(float) * (size_t)SHADE_GRAD_CH * (size_t)width * (size_t)height + 256 +
         lf_shade_scratch_bytes(width, height, spp);
}

lf_status lf_trace_backward(lf_ctx* c, const lf_camera* cam, const float* gbuf, int env_id, int spp, uint64_t seed,
                            const float* dL_drgb, const float* dL_dgbuf, float* d_surfel, float* d_env,
                            const void* fwd_samples, void* scratch, size_t scratch_bytes) {
  lf_status st = check_render(c, cam, env_id);
  if (st != LF_OK) return st;
  if (!gbuf || !d_surfel) return fail(c, LF_ERR_INVALID, "null G-buffer or gradient");
  if (dL_drgb && (spp <= 0 || spp > (1 << 20))) return fail(c, LF_ERR_INVALID, "bad spp");
  const int n_pix = cam->width * cam->height;
  float* sg = nullptr;
  TraceArgs a = lf_ctx_trace_args(c, env_id);
  if (c->profile) LF_CUDA(c, cudaEventRecord(c->prof_ev[8], c->stream));
  if (dL_drgb) {
    const size_t sg_bytes = sizeof(float) * (size_t)SHADE_GRAD_CH * n_pix + 256;
    const size_t need = fwd_samples ? sg_bytes : lf_backward_scratch_bytes(cam->width, cam->height, spp);
    if (!scratch || scratch_bytes < need) return fail(c, LF_ERR_INVALID, "scratch too small");
    sg = static_cast<float*>(scratch);
    const ShadeBatch B = one_job(c, cam, gbuf, env_id, spp, seed, nullptr);
    SampleBuf S;
    if (fwd_samples) {
      S = sample_buf(const_cast<void*>(fwd_samples), B.n_items);
    } else {  // replay the forward's sample data with the same seed
      S = sample_buf(static_cast<char*>(scratch) + sg_bytes, B.n_items);
      LF_CUDA(c, launch_shade_wavefront(B, c->dp, S, c->status_dev, nullptr, nullptr, c->sms, c->stream));
    }
    LF_CUDA(c, launch_shade_combine_adjoint(B, c->dp, S, dL_drgb, sg, d_env, c->stream));
  }
  if (c->profile) LF_CUDA(c, cudaEventRecord(c->prof_ev[9], c->stream));
  LF_CUDA(c, launch_trace_backward(a, c->scene, to_cam(*cam), gbuf, sg, dL_dgbuf, d_surfel, d_env, c->stream));
  if (c->profile) {
    LF_CUDA(c, cudaEventRecord(c->prof_ev[10], c->stream));
    c->prof_bwd = true;
  }
  return LF_OK;
}

lf_status lf_philox(lf_ctx* c, const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out) {
  if (!c || n < 0 || (n > 0 && (!ctr || !out))) return LF_ERR_INVALID;
  LF_CUDA(c, launch_philox(ctr, n, k0, k1, out, c->stream));
  return LF_OK;
}

lf_status lf_bvh_info(lf_ctx* c, int k, int* n_internal, int* root_code) {
  if (!c) return LF_ERR_INVALID;
  if (!c->built) return fail(c, LF_ERR_NOT_BUILT, "no BVH");
  if (k < 0 || k >= c->n_obj) return fail(c, LF_ERR_INVALID, "bad object id");
  if (n_internal) *n_internal = c->node_off_h[k + 1] - c->node_off_h[k];
  if (root_code) *root_code = c->insts_h[k].root;
  return LF_OK;
}

lf_status lf_bvh_copy_nodes(lf_ctx* c, int k, float* host_out, size_t bytes) {
  if (!c || !host_out) return LF_ERR_INVALID;
  if (!c->built) return fail(c, LF_ERR_NOT_BUILT, "no BVH");
  if (k < 0 || k >= c->n_obj) return fail(c, LF_ERR_INVALID, "bad object id");
  const size_t nn = (size_t)(c->node_off_h[k + 1] - c->node_off_h[k]);
  if (bytes < nn * 64) return fail(c, LF_ERR_INVALID, "buffer too small");
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (nn) LF_CUDA(c, cudaMemcpy(host_out, c->nodes + 4 * (size_t)c->node_off_h[k], nn * 64, cudaMemcpyDeviceToHost));
  return LF_OK;
}

int lf_bvh_wide_node_bytes(void) { return (int)(WNODE_Q * sizeof(float4)); }

lf_status lf_bvh_copy_wide(lf_ctx* c, int k, float* host_out, size_t bytes, int* cap_nodes, int* root_code,
                           int* root_count, int* wide) {
  if (!c) return LF_ERR_INVALID;
  if (!c->built) return fail(c, LF_ERR_NOT_BUILT, "no BVH");
  if (k < 0 || k >= c->n_obj) return fail(c, LF_ERR_INVALID, "bad object id");
  const size_t nn = (size_t)(c->wnode_off_h[k + 1] - c->wnode_off_h[k]);
  if (cap_nodes) *cap_nodes = (int)nn;
  if (root_code) *root_code = c->insts_h[k].wroot;
  if (root_count) *root_count = c->insts_h[k].wroot_count;
  if (wide) *wide = WIDE;
  if (!host_out) return LF_OK;
  const size_t need = nn * 2 * WIDE * sizeof(float4);
  if (bytes < need) return fail(c, LF_ERR_INVALID, "buffer too small");
  LF_CUDA(c, cudaStreamSynchronize(c->stream));
  if (!nn) return LF_OK;
#if LF_WIDE_FP16
  // decode the compressed slots into the inspection layout; each corner is
  // centre + offset rounded outward, a box containing the one traversal tests
  std::vector<float4> raw(nn * WNODE_Q);
  LF_CUDA(c, cudaMemcpy(raw.data(), c->wnodes + WNODE_Q * (size_t)c->wnode_off_h[k], raw.size() * sizeof(float4),
                        cudaMemcpyDeviceToHost));
  auto half_at = [](unsigned word, int hi16) {
    return (double)__half2float(__ushort_as_half((unsigned short)(hi16 ? word >> 16 : word & 0xffffu)));
  };
  auto outward = [](double v, bool up) {
    float f = (float)v;
    if (up && (double)f < v) f = std::nextafter(f, INFINITY);
    if (!up && (double)f > v) f = std::nextafter(f, -INFINITY);
    return f;
  };
  float4* out = reinterpret_cast<float4*>(host_out);
  for (size_t w = 0; w < nn; ++w) {
    const float4 H = raw[WNODE_Q * w];
    for (int s = 0; s < WIDE; ++s) {
      const float4 q = raw[WNODE_Q * w + 1 + s];
      unsigned u[4];
      std::memcpy(u, &q, sizeof(u));
      int code = INT_MIN, count = 0;
      if (u[3] != WSLOT_EMPTY) {
        if ((int)u[3] >= 0) {
          code = (int)u[3];
        } else {
          count = (int)((u[3] >> 24) & 31u) + 1;
          code = ~(int)(u[3] & 0xffffffu);
        }
      }
      const double lo[3] = {H.x + half_at(u[0], 0), H.y + half_at(u[0], 1), H.z + half_at(u[1], 0)};
      const double hi[3] = {H.x + half_at(u[1], 1), H.y + half_at(u[2], 0), H.z + half_at(u[2], 1)};
      float4 L = make_float4(outward(lo[0], false), outward(lo[1], false), outward(lo[2], false), 0.0f);
      float4 U = make_float4(outward(hi[0], true), outward(hi[1], true), outward(hi[2], true), 0.0f);
      std::memcpy(&L.w, &code, sizeof(int));
      std::memcpy(&U.w, &count, sizeof(int));
      out[2 * WIDE * w + s] = L;
      out[2 * WIDE * w + WIDE + s] = U;
    }
  }
#else
  LF_CUDA(c, cudaMemcpy(host_out, c->wnodes + 2 * WIDE * (size_t)c->wnode_off_h[k], need, cudaMemcpyDeviceToHost));
#endif
  return LF_OK;
}

}  // extern "C"
