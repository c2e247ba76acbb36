// Measurement helper: the L2 read bandwidth the trace kernels are compared
// with (their working set -- packed records and wide nodes -- stays in L2).
#include "lf_ctx.h"

namespace {

// Every thread streams float4 loads over the buffer `reps` times, caching at
// L2 only (ld.global.cg), so that after the first pass every load is served by
// L2.  The sum keeps the loads from being optimised away.
__global__ void k_l2_read(const float4* __restrict__ buf, long long n4, int reps, float* __restrict__ sink) {
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int r = 0; r < reps; ++r) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n4; i += stride) {
      const float4 v = __ldcg(buf + i);
      acc.x += v.x;
      acc.y += v.y;
      acc.z += v.z;
      acc.w += v.w;
    }
  }
  if (acc.x + acc.y + acc.z + acc.w == 1.0f) sink[0] = acc.x;  // never true for a zeroed buffer
}

}  // namespace

extern "C" {

lf_status lf_measure_l2_read(lf_ctx* c, size_t bytes, int reps, float* gbs) {
  if (!c || !gbs || bytes < (1u << 20) || reps < 1) return LF_ERR_INVALID;
  const long long n4 = (long long)(bytes / sizeof(float4));
  float4* buf = nullptr;
  float* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&buf, sizeof(float4) * (size_t)n4);
  if (e == cudaSuccess) e = cudaMalloc(&sink, sizeof(float));
  if (e == cudaSuccess) e = cudaMemsetAsync(buf, 0, sizeof(float4) * (size_t)n4, c->stream);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = c->sms * 8, block = 256;
  float ms = 0.0f;
  if (e == cudaSuccess) {
    k_l2_read<<<grid, block, 0, c->stream>>>(buf, n4, 2, sink);  // warm: bring the buffer into L2
    cudaEventRecord(e0, c->stream);
    k_l2_read<<<grid, block, 0, c->stream>>>(buf, n4, reps, sink);
    cudaEventRecord(e1, c->stream);
    e = cudaEventSynchronize(e1);
  }
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (buf) cudaFree(buf);
  if (sink) cudaFree(sink);
  if (e != cudaSuccess) {
    c->err = std::string("lf_measure_l2_read: ") + cudaGetErrorString(e);
    return LF_ERR_CUDA;
  }
  *gbs = (float)((double)sizeof(float4) * (double)n4 * reps / (ms * 1e-3) / 1e9);
  return LF_OK;
}

}  // extern "C"
