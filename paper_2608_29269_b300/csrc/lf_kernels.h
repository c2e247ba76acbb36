// Internal launcher interface between the C ABI (lf_api.cu) and the kernels.
#pragma once
#include <cuda_runtime.h>

#include "lf_common.cuh"

namespace lf {

struct SceneDev {
  float *mu, *tu, *tv, *scale, *opacity, *albedo, *metallic, *roughness;
  int n;
};

struct Mat34 {
  float R[9], t[3];
};

struct FitArgs {
  int first_leaf, n_leaves, n_obj;
  const int* leaf_off;  // device, n_obj + 1
  const int* node_off;  // device, n_obj + 1
  const unsigned* sorted_ids;
  float4* geo;
  float4* mat;
  float4* nodes;
  int* flags;
  const int* leaf_parent;
  const int* node_parent;
  Inst* insts;
  float R;  // support radius
  int* status;
  int leaf_base = 0, node_base = 0, id_base = 0, inst_base = 0;  // object-local storage (served versions)
};

// Wide BVH collapse (topology) and box copy.  Index bases are subtracted
// when addressing object-local storage (a served version); all bases are 0 for
// the context's own arrays.
struct WideArgs {
  int first_obj = 0, n_objs = 0;  // objects handled by the launch
  int n_obj_total = 0;            // objects in the offset tables
  const int* leaf_off = nullptr;  // device, n_obj_total + 1
  const int* node_off = nullptr;  // device, binary node offsets
  const int* wnode_off = nullptr; // device, wide node offsets
  const int2* node_range = nullptr;  // per binary node: first leaf, leaf count
  const float4* nodes = nullptr;  // binary nodes (index - node_base)
  float4* wnodes = nullptr;       // wide nodes (index - wnode_base)
  int* wsrc = nullptr;            // per wide slot: binary parent * 2 + side, -1 empty (slot - WIDE * wsrc_base)
  int* wqueue = nullptr;          // collapse queue (index - wnode_base)
  int node_base = 0, wnode_base = 0, wsrc_base = 0;
  int first_slot = 0;             // first global slot of a box copy
  int* status = nullptr;
};

// Wide nodes an object of n surfels can need.
inline int wide_capacity(int n) {
  if (n <= WLEAF) return 0;
  const long long nn = n;
  return (int)((nn * (WLEAF + 1) + (long long)(WIDE - 2) * nn) / ((long long)(WIDE - 1) * (WLEAF + 1)) + 2);
}

struct InstPtrs {
  const Inst* p[LF_MAX_OBJECTS];
};

// BVH build / refit (lf_bvh.cu)
cudaError_t launch_object_bounds(const SceneDev& s, const int* offsets_dev, int n_obj, int max_obj_n, int* bounds,
                                 cudaStream_t st);
cudaError_t launch_morton(const SceneDev& s, const int* offsets_dev, int n_obj, const int* bounds, unsigned* keys,
                          unsigned* vals, cudaStream_t st);
int radix_tiles(int n);
cudaError_t launch_radix_sort(unsigned* keys, unsigned* vals, unsigned* keys_alt, unsigned* vals_alt, int n,
                              const int* offsets_dev, int n_obj, unsigned* counts, cudaStream_t st);
cudaError_t launch_hierarchy(const unsigned* skeys, const int* leaf_off, const int* node_off, int n_obj,
                             int n_nodes_total, float4* nodes, int* leaf_parent, int* node_parent,
                             int2* node_range, cudaStream_t st);
cudaError_t launch_collapse(const WideArgs& a, cudaStream_t st);
cudaError_t launch_wide_boxes(const WideArgs& a, int n_slots, cudaStream_t st);
cudaError_t launch_pack_fit(const SceneDev& s, const FitArgs& a, cudaStream_t st);
cudaError_t launch_rigid(const SceneDev& s, int beg, int end, const Mat34& T, cudaStream_t st);
cudaError_t launch_material(const SceneDev& s, int beg, int end, float3 rgb, int set_rgb, float metal, float rough,
                            cudaStream_t st);
cudaError_t launch_env_tables(const float* rgb, const double* sin_row, int H, int W, double* rowsum, float* pmf_row,
                              float* cdf_row, float* pmf_col, float* cdf_col, float* cdf_row_lo, float* cdf_col_lo,
                              cudaStream_t st);
cudaError_t launch_gather_insts(const InstPtrs& src, Inst* dst, int n, cudaStream_t st);
cudaError_t launch_philox(const uint32_t* ctr, int n, uint32_t k0, uint32_t k1, uint32_t* out, cudaStream_t st);

// Rendering (lf_render.cu)
struct TraceArgs {
  const Inst* insts;
  int n_inst;
  DevParams P;
  EnvDev env;
  int* status;
  unsigned long long* counters;  // nullable: [nodes, tests, composited, rays]
};

cudaError_t launch_trace_primary(const TraceArgs& a, const CamDev& cam, float* gbuf, cudaStream_t st);

// Primary rays of up to MAX_PRIMARY_JOBS images in one launch, each with its
// own scene snapshot, environment, camera and G-buffer (the launcher fills
// tile0).
constexpr int MAX_PRIMARY_JOBS = 32;
struct PrimaryJob {
  const Inst* insts;
  int n_inst;
  EnvDev env;
  CamDev cam;
  float* gbuf;
  int tile0;
};
struct PrimaryBatch {
  int n_jobs;
  PrimaryJob jobs[MAX_PRIMARY_JOBS];
};
cudaError_t launch_trace_primary_batch(PrimaryBatch& B, const DevParams& P, int* status, cudaStream_t st);

// Adjoint (lf_backward.cu)
constexpr int SHADE_GRAD_CH = 9;  // per pixel: g_n (3), g_a (3), g_m, g_r, g_T
cudaError_t launch_trace_backward(const TraceArgs& a, const SceneDev& s, const CamDev& cam, const float* gbuf,
                                  const float* shade_grad, const float* dL_dgbuf, float* d_surfel, float* d_env,
                                  cudaStream_t st);

}  // namespace lf
