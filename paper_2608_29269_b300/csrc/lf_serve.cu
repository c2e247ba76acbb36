// Served edit-and-render loop (Sec. 3.4.2 edits on a device-resident scene).
//
// A request is one edit (rigid move of an object, material edit or
// environment swap) plus a camera.  Edits apply to the served scene in
// submission order; each creates a new VERSION of the edited object (copy on
// write: attributes, packed records, BVH nodes and instance entry), so an
// in-flight request keeps rendering exactly the scene state right after its
// own edit while later requests edit further.  Only the edited object's BLAS
// is refit (topology kept); the other objects share their current version.
//
// Continuous batching: a scheduler thread admits pending requests in FIFO
// order while a slot is free and their memory (frame, G-buffer, per-sample
// buffer, new version) fits the budget; requests admitted together (up to a
// work-item cap) form a group whose shading runs as one batched wavefront
// (work items of every request in the same launches).  Groups launch on a
// ladder of stream priorities: the oldest group in flight has precedence and
// younger ones fill the SMs its kernels leave idle, so groups overlap on the
// device without slowing the oldest; a group's finished frames are copied to
// pinned host memory.
// Completion is observed with events; memory of finished groups and of
// versions no request references any more is released stream-ordered.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lf_ctx.h"
#include "lf_wavefront.h"

using namespace lf;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// A launch group takes pending requests in FIFO order up to this many work
// items (pixels x samples); a larger request forms a group of its own.
// Small requests share launches; a large one does not hold small ones back.
constexpr long long GROUP_MAX_SAMPLES = 1ll << 22;

// Attribute layout of a version's raw copy (floats per surfel).
constexpr int RAW_FLOATS = 17;

struct Version {
  int obj = 0, n = 0;
  bool base = false;          // the context's own storage (never freed here)
  float* raw = nullptr;       // mu 3n | tu 3n | tv 3n | scale 2n | opacity n | albedo 3n | metallic n | roughness n
  float4* geo = nullptr;
  float4* mat = nullptr;
  float4* nodes = nullptr;
  float4* wnodes = nullptr;   // wide BVH (topology of the build, boxes of this version)
  int* flags = nullptr;
  Inst* inst = nullptr;       // device entry (box written by the fit)
  char* block = nullptr;      // single allocation holding everything above
  size_t bytes = 0;
  int refs = 0;               // requests in flight using it + 1 while current
  SceneDev view() const {
    SceneDev s;
    s.mu = raw;
    s.tu = raw + 3 * n;
    s.tv = raw + 6 * n;
    s.scale = raw + 9 * n;
    s.opacity = raw + 11 * n;
    s.albedo = raw + 12 * n;
    s.metallic = raw + 15 * n;
    s.roughness = raw + 16 * n;
    s.n = n;
    return s;
  }
};

struct Job {
  uint64_t ticket = 0;
  lf_request req{};
  double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
  int state = 0;  // 0 pending, 1 in flight, 2 done
  lf_status status = LF_OK;
  std::vector<Version*> snap;
  int env_id = 0;
  size_t bytes = 0;
  // device buffers (one block) and host frame
  char* block = nullptr;
  Inst* insts = nullptr;
  float* gbuf = nullptr;
  float* rgb = nullptr;
  float* host_frame = nullptr;
  unsigned long long rays = 0;
};

struct Group {
  std::vector<Job*> jobs;
  int level = 0;  // index into the server's streams (priority order)
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  char* samples = nullptr;
  unsigned long long* rays_dev = nullptr;
  unsigned long long* rays_host = nullptr;  // pinned slot
};

}  // namespace

struct lf_serve {
  lf_ctx* ctx = nullptr;
  size_t budget = 0, used = 0;
  int max_slots = 1, in_flight = 0;
  double window_s = 0.0;  // how long a lone request waits for company
  // streams[0] has the highest priority; a group launches on the stream one
  // below the youngest group in flight (the last stream serialises), so
  // older groups keep precedence and younger ones fill their tails.
  std::vector<cudaStream_t> streams;
  cudaStream_t edit_stream = nullptr;
  cudaEvent_t edit_event = nullptr;
  // Stream-ordered allocations come from this server's own pool, which keeps
  // up to the budget mapped between requests (the device's default pool
  // would return its memory at every synchronisation).
  cudaMemPool_t pool = nullptr;
  std::vector<Version*> current;               // current version per object
  std::vector<std::unique_ptr<Version>> versions;
  std::vector<float*> frame_pool;              // pinned host frames
  size_t frame_floats = 0;
  unsigned long long* ray_slots = nullptr;     // pinned per-group ray counters
  int next_slot = 0;
  int env_id = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> pending;
  std::map<uint64_t, std::unique_ptr<Job>> jobs;
  std::vector<Group*> groups;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread worker;
  std::string err;
};

namespace {

cudaError_t alloc_async(lf_serve* s, char** p, size_t bytes, cudaStream_t st) {
  return cudaMallocFromPoolAsync(reinterpret_cast<void**>(p), bytes ? bytes : 256, s->pool, st);
}

size_t frame_bytes_of(const lf_camera& c, int spp) {
  const size_t P = (size_t)c.width * c.height;
  return sizeof(float) * (LF_GBUF_CHANNELS + 3) * P + sizeof(Inst) * LF_MAX_OBJECTS + 1024 +
         sample_buf_bytes((long long)P * spp);
}

size_t version_bytes(int n) {
  return sizeof(float) * RAW_FLOATS * (size_t)n + sizeof(float4) * (GEO + 1 + 4) * (size_t)n +
         sizeof(float4) * WNODE_Q * (size_t)wide_capacity(n) + sizeof(int) * (size_t)n + sizeof(Inst) + 1280;
}

// New version of object k: copy the current one, apply the edit, repack and
// refit (all on the edit stream).
lf_status make_version(lf_serve* s, const lf_edit& e, Version** out) {
  lf_ctx* c = s->ctx;
  const int k = e.object_id;
  Version* cur = s->current[k];
  auto v = std::make_unique<Version>();
  v->obj = k;
  v->n = cur->n;
  const int n = v->n;
  v->bytes = version_bytes(n);
  if (alloc_async(s, &v->block, v->bytes, s->edit_stream) != cudaSuccess) return LF_ERR_OOM;
  char* p = v->block;
  auto take = [&](size_t b) { char* r = p; p += (b + 255) / 256 * 256; return r; };
  v->raw = reinterpret_cast<float*>(take(sizeof(float) * RAW_FLOATS * n));
  v->geo = reinterpret_cast<float4*>(take(sizeof(float4) * GEO * n));
  v->mat = reinterpret_cast<float4*>(take(sizeof(float4) * n));
  v->nodes = reinterpret_cast<float4*>(take(sizeof(float4) * 4 * std::max(1, n - 1)));
  const int nw = c->wnode_off_h[k + 1] - c->wnode_off_h[k];
  v->wnodes = reinterpret_cast<float4*>(take(sizeof(float4) * WNODE_Q * std::max(1, nw)));
  v->flags = reinterpret_cast<int*>(take(sizeof(int) * n));
  v->inst = reinterpret_cast<Inst*>(take(sizeof(Inst)));
  // copy attributes, nodes (child codes) and the instance entry
  const SceneDev dst = v->view();
  if (cur->base) {
    const SceneDev& src = c->scene;
    const size_t o = (size_t)c->offsets[k];
    const float* sp[8] = {src.mu + 3 * o, src.tu + 3 * o, src.tv + 3 * o, src.scale + 2 * o,
                          src.opacity + o, src.albedo + 3 * o, src.metallic + o, src.roughness + o};
    float* dp[8] = {dst.mu, dst.tu, dst.tv, dst.scale, dst.opacity, dst.albedo, dst.metallic, dst.roughness};
    const int w[8] = {3, 3, 3, 2, 1, 3, 1, 1};
    for (int f = 0; f < 8; ++f)
      if (cudaMemcpyAsync(dp[f], sp[f], sizeof(float) * w[f] * n, cudaMemcpyDeviceToDevice, s->edit_stream) !=
          cudaSuccess)
        return LF_ERR_CUDA;
  } else if (cudaMemcpyAsync(v->raw, cur->raw, sizeof(float) * RAW_FLOATS * n, cudaMemcpyDeviceToDevice,
                             s->edit_stream) != cudaSuccess) {
    return LF_ERR_CUDA;
  }
  if (n >= 2 && cudaMemcpyAsync(v->nodes, cur->nodes, sizeof(float4) * 4 * (n - 1), cudaMemcpyDeviceToDevice,
                                s->edit_stream) != cudaSuccess)
    return LF_ERR_CUDA;
  if (nw > 0 && cudaMemcpyAsync(v->wnodes, cur->wnodes, sizeof(float4) * WNODE_Q * nw, cudaMemcpyDeviceToDevice,
                                s->edit_stream) != cudaSuccess)
    return LF_ERR_CUDA;
  // the instance entry points at the version's arrays (its box is written by the fit)
  Inst hinst = c->insts_h[k];
  hinst.nodes = v->nodes;
  hinst.wnodes = v->wnodes;
  hinst.geo = v->geo;
  hinst.mat = v->mat;
  if (cudaMemcpyAsync(v->inst, &hinst, sizeof(Inst), cudaMemcpyHostToDevice, s->edit_stream) != cudaSuccess)
    return LF_ERR_CUDA;
  // the edit
  cudaError_t err = cudaSuccess;
  if (e.kind == LF_EDIT_MOVE) {
    Mat34 T;
    std::memcpy(T.R, e.R, sizeof(T.R));
    std::memcpy(T.t, e.t, sizeof(T.t));
    err = launch_rigid(dst, 0, n, T, s->edit_stream);
  } else {
    err = launch_material(dst, 0, n, make_float3(e.albedo[0], e.albedo[1], e.albedo[2]), e.set_albedo,
                          e.metallic, e.roughness, s->edit_stream);
  }
  if (err != cudaSuccess) return LF_ERR_CUDA;
  // repack + refit (topology of the build)
  const int nn = c->node_off_h[k + 1] - c->node_off_h[k];
  if (nn > 0 && cudaMemsetAsync(v->flags, 0, sizeof(int) * nn, s->edit_stream) != cudaSuccess) return LF_ERR_CUDA;
  FitArgs a;
  a.first_leaf = c->offsets[k];
  a.n_leaves = n;
  a.n_obj = c->n_obj;
  a.leaf_off = c->offsets_dev;
  a.node_off = c->node_off_dev;
  a.sorted_ids = c->vals;
  a.geo = v->geo;
  a.mat = v->mat;
  a.nodes = v->nodes;
  a.flags = v->flags;
  a.leaf_parent = c->leaf_parent;
  a.node_parent = c->node_parent;
  a.insts = v->inst;
  a.R = std::sqrt(c->params.support_r2);
  a.status = c->status_dev;
  a.leaf_base = c->offsets[k];
  a.node_base = c->node_off_h[k];
  a.id_base = c->offsets[k];
  a.inst_base = k;
  if (launch_pack_fit(dst, a, s->edit_stream) != cudaSuccess) return LF_ERR_CUDA;
  if (nw > 0) {  // wide boxes from the version's refit binary nodes
    WideArgs w = lf_ctx_wide_args(c);
    w.nodes = v->nodes;
    w.node_base = c->node_off_h[k];
    w.wnodes = v->wnodes;
    w.wnode_base = c->wnode_off_h[k];
    w.first_slot = WIDE * c->wnode_off_h[k];
    if (launch_wide_boxes(w, WIDE * nw, s->edit_stream) != cudaSuccess) return LF_ERR_CUDA;
  }
  *out = v.get();
  s->versions.push_back(std::move(v));
  return LF_OK;
}

void release_version(lf_serve* s, Version* v) {
  if (v->base || --v->refs > 0) return;
  cudaFreeAsync(v->block, s->edit_stream);
  for (auto it = s->versions.begin(); it != s->versions.end(); ++it)
    if (it->get() == v) {
      s->used -= v->bytes;
      s->versions.erase(it);
      break;
    }
}

// Admit one job: apply its edit, take its snapshot, allocate its buffers.
lf_status admit(lf_serve* s, Job* j) {
  lf_ctx* c = s->ctx;
  const lf_edit& e = j->req.edit;
  if (e.kind == LF_EDIT_ENV) s->env_id = e.env_id;
  if (e.kind == LF_EDIT_MOVE || e.kind == LF_EDIT_MATERIAL) {
    Version* v = nullptr;
    lf_status st = make_version(s, e, &v);
    if (st != LF_OK) return st;
    s->used += v->bytes;
    Version* old = s->current[e.object_id];
    s->current[e.object_id] = v;
    v->refs = 1;  // current
    release_version(s, old);
  }
  j->env_id = s->env_id;
  j->snap = s->current;
  for (Version* v : j->snap) ++v->refs;
  const lf_camera& cam = j->req.cam;
  const size_t P = (size_t)cam.width * cam.height;
  const size_t b_insts = (sizeof(Inst) * LF_MAX_OBJECTS + 255) / 256 * 256;
  const size_t b_gbuf = (sizeof(float) * LF_GBUF_CHANNELS * P + 255) / 256 * 256;
  const size_t b_rgb = (sizeof(float) * 3 * P + 255) / 256 * 256;
  if (alloc_async(s, &j->block, b_insts + b_gbuf + b_rgb, s->edit_stream) != cudaSuccess) return LF_ERR_OOM;
  j->insts = reinterpret_cast<Inst*>(j->block);
  j->gbuf = reinterpret_cast<float*>(j->block + b_insts);
  j->rgb = reinterpret_cast<float*>(j->block + b_insts + b_gbuf);
  InstPtrs ptrs;
  for (int k = 0; k < c->n_obj; ++k) ptrs.p[k] = j->snap[k]->inst;
  if (launch_gather_insts(ptrs, j->insts, c->n_obj, s->edit_stream) != cudaSuccess) return LF_ERR_CUDA;
  return LF_OK;
}

TraceArgs job_trace_args(lf_serve* s, Job* j) {
  TraceArgs a = lf_ctx_trace_args(s->ctx, j->env_id);
  a.insts = j->insts;
  a.counters = nullptr;
  return a;
}

lf_status launch_group(lf_serve* s, Group* g) {
  lf_ctx* c = s->ctx;
  g->level = s->groups.empty() ? 0 : std::min(s->groups.back()->level + 1, (int)s->streams.size() - 1);
  g->stream = s->streams[g->level];
  if (cudaEventRecord(s->edit_event, s->edit_stream) != cudaSuccess) return LF_ERR_CUDA;
  if (cudaStreamWaitEvent(g->stream, s->edit_event, 0) != cudaSuccess) return LF_ERR_CUDA;
  ShadeBatch B;
  B.n_jobs = (int)g->jobs.size();
  B.n_items = 0;
  B.n_pix_total = 0;
  // the primary rays of every request of the group in one launch
  PrimaryBatch PB;
  PB.n_jobs = (int)g->jobs.size();
  static_assert(MAX_PRIMARY_JOBS >= MAX_JOBS, "a launch group must fit one primary batch");
  for (size_t q = 0; q < g->jobs.size(); ++q) {
    Job* j = g->jobs[q];
    const TraceArgs a = job_trace_args(s, j);
    PrimaryJob& PJ = PB.jobs[q];
    PJ.insts = a.insts;
    PJ.n_inst = a.n_inst;
    PJ.env = a.env;
    PJ.cam = lf_ctx_cam(j->req.cam);
    PJ.gbuf = j->gbuf;
  }
  if (launch_trace_primary_batch(PB, c->dp, c->status_dev, g->stream) != cudaSuccess) return LF_ERR_CUDA;
  for (size_t q = 0; q < g->jobs.size(); ++q) {
    Job* j = g->jobs[q];
    const lf_camera& cam = j->req.cam;
    const TraceArgs a = job_trace_args(s, j);
    ShadeJob& J = B.jobs[q];
    J.insts = j->insts;
    J.n_inst = c->n_obj;
    J.env = a.env;
    J.gbuf = j->gbuf;
    J.n_pix = cam.width * cam.height;
    J.rgb = j->rgb;
    J.spp = j->req.spp;
    J.k0 = (uint32_t)(j->req.seed & 0xffffffffu);
    J.k1 = (uint32_t)(j->req.seed >> 32);
    J.item0 = B.n_items;
    J.pix0 = B.n_pix_total;
    B.n_items += (long long)J.n_pix * J.spp;
    B.n_pix_total += J.n_pix;
  }
  if (alloc_async(s, &g->samples, sample_buf_bytes(B.n_items) + 256, g->stream) != cudaSuccess) return LF_ERR_OOM;
  g->rays_dev = reinterpret_cast<unsigned long long*>(g->samples + sample_buf_bytes(B.n_items));
  if (cudaMemsetAsync(g->rays_dev, 0, sizeof(unsigned long long), g->stream) != cudaSuccess) return LF_ERR_CUDA;
  const SampleBuf S = sample_buf(g->samples, B.n_items);
  if (launch_shade_wavefront(B, c->dp, S, c->status_dev, g->rays_dev, nullptr, c->sms, g->stream) != cudaSuccess)
    return LF_ERR_CUDA;
  if (launch_shade_combine(B, c->dp, S, g->stream) != cudaSuccess) return LF_ERR_CUDA;
  for (Job* j : g->jobs) {
    const lf_camera& cam = j->req.cam;
    if (cudaMemcpyAsync(j->host_frame, j->rgb, sizeof(float) * 3 * cam.width * cam.height, cudaMemcpyDeviceToHost,
                        g->stream) != cudaSuccess)
      return LF_ERR_CUDA;
  }
  g->rays_host = s->ray_slots + (s->next_slot++ % 1024);
  if (cudaMemcpyAsync(g->rays_host, g->rays_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost, g->stream) !=
      cudaSuccess)
    return LF_ERR_CUDA;
  if (cudaEventCreateWithFlags(&g->done, cudaEventDisableTiming) != cudaSuccess) return LF_ERR_CUDA;
  if (cudaEventRecord(g->done, g->stream) != cudaSuccess) return LF_ERR_CUDA;
  return LF_OK;
}

void finish_group(lf_serve* s, Group* g, lf_status st) {
  const double t = now_s();
  const unsigned long long rays = (st == LF_OK && g->rays_host) ? *g->rays_host : 0ull;
  for (Job* j : g->jobs) {
    j->t_done = t;
    j->state = 2;
    j->status = st;
    j->rays = rays;  // shading rays of the whole launch group
    cudaFreeAsync(j->block, g->stream ? g->stream : s->edit_stream);
    s->used -= j->bytes;
    for (Version* v : j->snap) release_version(s, v);
    j->snap.clear();
    --s->in_flight;
  }
  if (g->samples) cudaFreeAsync(g->samples, g->stream);
  if (g->done) cudaEventDestroy(g->done);
  delete g;
}

void worker_main(lf_serve* s) {
  cudaSetDevice(s->ctx->device);
  std::unique_lock<std::mutex> lock(s->mu);
  while (true) {
    // retire finished groups
    for (size_t q = 0; q < s->groups.size();) {
      Group* g = s->groups[q];
      const cudaError_t e = cudaEventQuery(g->done);
      if (e == cudaErrorNotReady) { ++q; continue; }
      finish_group(s, g, e == cudaSuccess ? LF_OK : LF_ERR_CUDA);
      s->groups.erase(s->groups.begin() + q);
      s->cv_done.notify_all();
    }
    if (s->stop && s->pending.empty() && s->groups.empty()) break;
    // batching window: a request that arrived less than window_s ago waits
    // for more company while slots are free
    if (!s->pending.empty() && s->window_s > 0.0 && !s->stop &&
        (int)s->pending.size() < std::min(MAX_JOBS, s->max_slots - s->in_flight)) {
      const double age = now_s() - s->pending.front()->t_submit;
      if (age < s->window_s) {
        s->cv_work.wait_for(lock, std::chrono::duration<double>(std::min(s->window_s - age, 0.0005)));
        continue;
      }
    }
    // admit a group in FIFO order
    Group* g = nullptr;
    long long g_samples = 0;
    while (!s->pending.empty() && s->in_flight < s->max_slots && !s->frame_pool.empty() &&
           (!g || (int)g->jobs.size() < MAX_JOBS)) {
      Job* j = s->pending.front();
      const long long j_samples = (long long)j->req.cam.width * j->req.cam.height * j->req.spp;
      if (g && g_samples + j_samples > GROUP_MAX_SAMPLES) break;  // next group
      const size_t need = frame_bytes_of(j->req.cam, j->req.spp) +
                          ((j->req.edit.kind == LF_EDIT_MOVE || j->req.edit.kind == LF_EDIT_MATERIAL)
                               ? version_bytes(s->current[j->req.edit.object_id]->n) : 0);
      if (s->used + need > s->budget) {
        if (s->in_flight == 0 && (!g || g->jobs.empty())) {  // can never fit
          s->pending.pop_front();
          j->state = 2;
          j->status = LF_ERR_OOM;
          j->t_admit = j->t_done = now_s();
          s->cv_done.notify_all();
          continue;
        }
        break;
      }
      s->pending.pop_front();
      j->t_admit = now_s();
      j->host_frame = s->frame_pool.back();
      s->frame_pool.pop_back();
      const lf_status st = admit(s, j);  // accounts the new version's bytes itself
      j->bytes = frame_bytes_of(j->req.cam, j->req.spp);
      s->used += j->bytes;
      ++s->in_flight;
      if (st != LF_OK) {
        j->state = 2;
        j->status = st;
        j->t_done = now_s();
        s->used -= j->bytes;
        for (Version* v : j->snap) release_version(s, v);
        j->snap.clear();
        if (j->block) cudaFreeAsync(j->block, s->edit_stream);
        --s->in_flight;
        s->cv_done.notify_all();
        continue;
      }
      j->state = 1;
      if (!g) g = new Group();
      g->jobs.push_back(j);
      g_samples += j_samples;
    }
    if (g) {
      const double t = now_s();
      for (Job* j : g->jobs) j->t_start = t;
      const lf_status st = launch_group(s, g);
      if (st != LF_OK) {
        finish_group(s, g, st);
        s->cv_done.notify_all();
      } else {
        s->groups.push_back(g);
      }
      continue;
    }
    // nothing to launch: sleep until a request can be admitted (a submission,
    // or a frame handed back by lf_serve_poll), or poll in-flight work.  The
    // predicate must not hold while admission is blocked, or the loop would
    // spin with the lock held and starve lf_serve_poll.
    if (s->groups.empty())
      s->cv_work.wait(lock, [&] {
        return s->stop || (!s->pending.empty() && s->in_flight < s->max_slots && !s->frame_pool.empty());
      });
    else
      s->cv_work.wait_for(lock, std::chrono::microseconds(50));
  }
}

bool valid_request(const lf_serve* s, const lf_request* r) {
  const lf_camera& c = r->cam;
  if (c.width <= 0 || c.height <= 0 || (size_t)c.width * c.height * 3 > s->frame_floats) return false;
  if (!(c.fovy_deg > 0.0f && c.fovy_deg < 179.0f) || r->spp <= 0 || r->spp > 4096) return false;
  if ((long long)c.width * c.height * r->spp >= (1LL << 30)) return false;
  const lf_edit& e = r->edit;
  switch (e.kind) {
    case LF_EDIT_NONE: return true;
    case LF_EDIT_ENV: return e.env_id >= 0 && e.env_id < LF_MAX_ENVS && s->ctx->env[e.env_id].set;
    case LF_EDIT_MATERIAL:
      return e.object_id >= 0 && e.object_id < s->ctx->n_obj && e.metallic <= 1.0f && e.roughness <= 1.0f;
    case LF_EDIT_MOVE: {
      if (e.object_id < 0 || e.object_id >= s->ctx->n_obj) return false;
      double dmax = 0.0;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double d = 0.0;
          for (int m = 0; m < 3; ++m) d += (double)e.R[3 * i + m] * e.R[3 * j + m];
          dmax = std::max(dmax, std::fabs(d - (i == j ? 1.0 : 0.0)));
        }
      const double det = (double)e.R[0] * (e.R[4] * e.R[8] - e.R[5] * e.R[7]) -
                         (double)e.R[1] * (e.R[3] * e.R[8] - e.R[5] * e.R[6]) +
                         (double)e.R[2] * (e.R[3] * e.R[7] - e.R[4] * e.R[6]);
      return dmax < 1e-4 && std::fabs(det - 1.0) < 1e-4 && std::isfinite(e.t[0]) && std::isfinite(e.t[1]) &&
             std::isfinite(e.t[2]);
    }
    default: return false;
  }
}

}  // namespace

extern "C" {

lf_status lf_serve_create(lf_ctx* c, size_t budget, int max_slots, int n_streams, int batch_window_us,
                          lf_serve** out) {
  if (!c || !out || max_slots < 1 || n_streams < 1 || budget == 0 || batch_window_us < 0) return LF_ERR_INVALID;
  if (!c->built) return LF_ERR_NOT_BUILT;
  int env0 = -1;
  for (int i = 0; i < LF_MAX_ENVS; ++i)
    if (c->env[i].set) { env0 = i; break; }
  if (env0 < 0) return LF_ERR_NOT_BUILT;
  auto s = std::make_unique<lf_serve>();
  s->ctx = c;
  s->budget = budget;
  s->max_slots = max_slots;
  s->window_s = 1e-6 * batch_window_us;
  s->env_id = env0;
  cudaMemPoolProps props = {};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = c->device;
  if (cudaMemPoolCreate(&s->pool, &props) != cudaSuccess) return LF_ERR_CUDA;
  uint64_t keep = budget;
  if (cudaMemPoolSetAttribute(s->pool, cudaMemPoolAttrReleaseThreshold, &keep) != cudaSuccess) {
    cudaMemPoolDestroy(s->pool);
    return LF_ERR_CUDA;
  }
  if (cudaStreamCreateWithFlags(&s->edit_stream, cudaStreamNonBlocking) != cudaSuccess) return LF_ERR_CUDA;
  if (cudaEventCreateWithFlags(&s->edit_event, cudaEventDisableTiming) != cudaSuccess) return LF_ERR_CUDA;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return LF_ERR_CUDA;
  for (int i = 0; i < n_streams; ++i) {
    cudaStream_t st;
    const int prio = std::min(greatest + i, least);  // numerically lower = higher priority
    if (cudaStreamCreateWithPriority(&st, cudaStreamNonBlocking, prio) != cudaSuccess) return LF_ERR_CUDA;
    s->streams.push_back(st);
  }
  // base versions: the context's storage
  for (int k = 0; k < c->n_obj; ++k) {
    auto v = std::make_unique<Version>();
    v->obj = k;
    v->n = c->offsets[k + 1] - c->offsets[k];
    v->base = true;
    v->inst = c->insts_dev + k;
    v->nodes = c->nodes + 4 * (size_t)c->node_off_h[k];
    v->wnodes = c->wnodes + WNODE_Q * (size_t)c->wnode_off_h[k];
    v->refs = 1;
    s->current.push_back(v.get());
    s->versions.push_back(std::move(v));
  }
  // pinned frames (largest frame 1024 x 1024) and ray counters
  s->frame_floats = (size_t)1024 * 1024 * 3;
  if (cudaHostAlloc(reinterpret_cast<void**>(&s->ray_slots), sizeof(unsigned long long) * 1024,
                    cudaHostAllocDefault) != cudaSuccess)
    return LF_ERR_OOM;
  for (int i = 0; i < 2 * max_slots; ++i) {
    float* f = nullptr;
    if (cudaHostAlloc(reinterpret_cast<void**>(&f), sizeof(float) * s->frame_floats, cudaHostAllocDefault) !=
        cudaSuccess) {
      for (float* q : s->frame_pool) cudaFreeHost(q);
      return LF_ERR_OOM;
    }
    s->frame_pool.push_back(f);
  }
  lf_serve* raw = s.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return LF_OK;
}

lf_status lf_serve_submit(lf_serve* s, const lf_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return LF_ERR_INVALID;
  if (!valid_request(s, r)) return LF_ERR_INVALID;
  auto j = std::make_unique<Job>();
  j->req = *r;
  j->t_submit = now_s();
  std::lock_guard<std::mutex> lock(s->mu);
  if (s->stop) return LF_ERR_INVALID;
  j->ticket = s->next_ticket++;
  *ticket = j->ticket;
  s->pending.push_back(j.get());
  s->jobs[j->ticket] = std::move(j);
  s->cv_work.notify_one();
  return LF_OK;
}

lf_status lf_serve_poll(lf_serve* s, uint64_t ticket, int* done, float* frame, size_t frame_floats,
                        lf_timing* timing) {
  if (!s || !done) return LF_ERR_INVALID;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return LF_ERR_INVALID;
  Job* j = it->second.get();
  *done = j->state == 2 ? 1 : 0;
  if (!*done) return LF_OK;
  const lf_status st = j->status;
  if (timing) {
    timing->t_submit = j->t_submit;
    timing->t_admit = j->t_admit;
    timing->t_start = j->t_start;
    timing->t_done = j->t_done;
    timing->rays = j->rays;
  }
  if (frame && j->host_frame && st == LF_OK) {
    const size_t nf = (size_t)j->req.cam.width * j->req.cam.height * 3;
    if (frame_floats < nf) return LF_ERR_INVALID;
    std::memcpy(frame, j->host_frame, sizeof(float) * nf);
  }
  if (j->host_frame) s->frame_pool.push_back(j->host_frame);
  s->jobs.erase(it);
  s->cv_work.notify_one();
  return st;
}

lf_status lf_serve_cancel(lf_serve* s, uint64_t ticket) {
  if (!s) return LF_ERR_INVALID;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return LF_ERR_INVALID;
  Job* j = it->second.get();
  // a pending job is in the queue until the scheduler admits it, under this lock
  auto q = std::find(s->pending.begin(), s->pending.end(), j);
  if (j->state != 0 || q == s->pending.end()) return LF_ERR_BUSY;
  s->pending.erase(q);
  j->state = 2;
  j->status = LF_ERR_CANCELLED;
  j->t_admit = j->t_start = j->t_done = now_s();
  s->cv_done.notify_all();
  s->cv_work.notify_one();
  return LF_OK;
}

lf_status lf_serve_wait(lf_serve* s, uint64_t ticket, int timeout_ms) {
  if (!s) return LF_ERR_INVALID;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return LF_ERR_INVALID;
  Job* j = it->second.get();
  const bool ok = s->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), [&] { return j->state == 2; });
  return ok ? LF_OK : LF_ERR_TIMEOUT;
}

lf_status lf_serve_destroy(lf_serve* s) {
  if (!s) return LF_ERR_INVALID;
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
    s->cv_work.notify_all();
  }
  if (s->worker.joinable()) s->worker.join();
  for (auto& v : s->versions)
    if (!v->base && v->block) cudaFreeAsync(v->block, s->edit_stream);
  for (auto& kv : s->jobs)
    if (kv.second->host_frame) s->frame_pool.push_back(kv.second->host_frame);
  cudaStreamSynchronize(s->edit_stream);
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (float* f : s->frame_pool) cudaFreeHost(f);
  cudaFreeHost(s->ray_slots);
  cudaEventDestroy(s->edit_event);
  cudaStreamDestroy(s->edit_stream);
  if (s->pool) cudaMemPoolDestroy(s->pool);
  delete s;
  return LF_OK;
}

}  // extern "C"
