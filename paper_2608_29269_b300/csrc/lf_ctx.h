// Context object behind the opaque lf_ctx handle (shared by lf_api.cu and
// lf_serve.cu).
#pragma once
#include <climits>
#include <string>
#include <vector>

#include "lf_kernels.h"

struct EnvSlot {
  const float* rgb = nullptr;  // caller-owned texels
  int H = 0, W = 0;
  float* tables = nullptr;     // pmf_row (H) | cdf_row (H) | pmf_col (H*W) | cdf_col (H*W) |
                               // cdf_row low parts (H) | cdf_col low parts (H*W)
  double* rowsum = nullptr;
  double* sin_row = nullptr;
  std::vector<double> sin_host;
  size_t cap = 0;
  int cap_h = 0;
  bool set = false;
};

struct lf_ctx {
  lf_params params{};
  lf::DevParams dp{};
  cudaStream_t stream = nullptr;
  int device = 0;
  int sms = 148;
  int* status_dev = nullptr;
  double* loss_dev = nullptr;  // loss sum of the regulariser calls
  unsigned long long* counters = nullptr;
  bool profile = false;
  cudaEvent_t prof_ev[11] = {};  // primary | gen | NEE shadow | continuation | secondary shadow | combine;
                                 // 8..10: shading adjoint | trace backward
  bool prof_bwd = false;         // a profiled lf_trace_backward recorded events 8..10
  std::string err;
  // scene (caller-owned arrays) and its object layout
  lf::SceneDev scene{};
  bool built = false;
  int n = 0, n_obj = 0, n_nodes = 0;
  std::vector<int> offsets, node_off_h, wnode_off_h;
  int* offsets_dev = nullptr;
  int* node_off_dev = nullptr;
  int* wnode_off_dev = nullptr;
  int* bounds = nullptr;
  // library-owned BVH storage
  float4* geo = nullptr;
  float4* mat = nullptr;
  float4* nodes = nullptr;
  int2* node_range = nullptr;  // per binary node: first leaf, leaf count
  float4* wnodes = nullptr;    // wide BVH (WIDE slots of 2 float4 per node)
  int* wsrc = nullptr;         // per wide slot: binary parent * 2 + side, -1 empty
  int* wqueue = nullptr;       // collapse work queue
  size_t wcap = 0;             // wide nodes allocated
  int* leaf_parent = nullptr;
  int* node_parent = nullptr;
  int* flags = nullptr;
  unsigned* keys = nullptr;
  unsigned* vals = nullptr;  // leaf -> surfel id after the build
  unsigned* keys_alt = nullptr;
  unsigned* vals_alt = nullptr;
  unsigned* counts = nullptr;
  size_t cap_n = 0;
  lf::Inst* insts_dev = nullptr;
  std::vector<lf::Inst> insts_h;
  EnvSlot env[LF_MAX_ENVS];
};

// R (row-major 3x3) is a rotation within FP32 tolerance and t (nullable) is finite (lf_api.cu).
bool lf_is_rigid(const float R[9], const float t[3]);
// Repack + refit objects [first_obj, last_obj] (lf_api.cu).
lf_status lf_ctx_fit(lf_ctx* c, int first_obj, int last_obj);
lf::TraceArgs lf_ctx_trace_args(lf_ctx* c, int env_id);
// Wide-BVH arguments over the context's own storage (bases 0).
lf::WideArgs lf_ctx_wide_args(lf_ctx* c);
lf::CamDev lf_ctx_cam(const lf_camera& c);
// Drop the cached device address of the allocation-free entry point's
// scratch array for `device` (lf_static.cu); lf_create calls it.
void lf_static_scratch_forget(int device);
