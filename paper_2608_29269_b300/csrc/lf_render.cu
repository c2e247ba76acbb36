// Primary-ray compositing (Eq. 6-7).
#include "lf_kernels.h"

namespace lf {

constexpr int TB = 128;  // threads per block
constexpr int STACK_SMEM = TB * STACK * (int)sizeof(int);

__device__ __forceinline__ void load_instances(Inst* dst, const Inst* src, int n) {
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < n * (int)(sizeof(Inst) / sizeof(float4)); i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// Slot 0 of the per-kernel counters: primary rays.
__device__ __forceinline__ void add_counters(unsigned long long* c, const Counters& k, unsigned comp, unsigned rays) {
  if (!c) return;
  atomicAdd(c + 0, (unsigned long long)k.nodes);
  atomicAdd(c + 1, (unsigned long long)k.tests);
  atomicAdd(c + 2, (unsigned long long)comp);
  atomicAdd(c + 3, (unsigned long long)rays);
}

// One thread per pixel, 16 x 8 pixel tiles.
__global__ void __launch_bounds__(TB) k_trace_primary(TraceArgs a, CamDev cam, float* __restrict__ gbuf) {
  __shared__ Inst s_inst[LF_MAX_OBJECTS];
  extern __shared__ int s_stack[];
  load_instances(s_inst, a.insts, a.n_inst);
  const int x = blockIdx.x * 16 + (threadIdx.x & 15), y = blockIdx.y * 8 + (threadIdx.x >> 4);
  if (x >= cam.W || y >= cam.H) return;
  const int p = y * cam.W + x;
  const size_t P = (size_t)cam.W * cam.H;
  const float3 d = camera_dir(cam, p);
  Counters cnt;
  unsigned comp = 0;
  Surface s;
  trace_composite(s_inst, a.n_inst, cam.eye, d, a.P, s_stack + threadIdx.x, TB, a.status, cnt, s, comp);
  const float3 rho = s.Sa + env_lookup(a.env, d) * s.T;
  float* g = gbuf + p;
  g[LF_CH_T * P] = s.T;
  g[LF_CH_W * P] = s.W;
  g[LF_CH_DEPTH * P] = s.depth;
  g[(LF_CH_X + 0) * P] = s.x.x; g[(LF_CH_X + 1) * P] = s.x.y; g[(LF_CH_X + 2) * P] = s.x.z;
  g[(LF_CH_N + 0) * P] = s.n.x; g[(LF_CH_N + 1) * P] = s.n.y; g[(LF_CH_N + 2) * P] = s.n.z;
  g[(LF_CH_A + 0) * P] = s.a.x; g[(LF_CH_A + 1) * P] = s.a.y; g[(LF_CH_A + 2) * P] = s.a.z;
  g[LF_CH_M * P] = s.m;
  g[LF_CH_R * P] = s.r;
  g[(LF_CH_RHO + 0) * P] = rho.x; g[(LF_CH_RHO + 1) * P] = rho.y; g[(LF_CH_RHO + 2) * P] = rho.z;
  g[LF_CH_NLEN * P] = s.nlen;
  g[LF_CH_HITS * P] = (float)s.hits;
  g[LF_CH_TSTOP * P] = key_t(s.stop_key);
  g[LF_CH_IDSTOP * P] = s.hits ? (float)(int)(s.stop_key & 0xffffffull) : -1.0f;
  g[(LF_CH_DIR + 0) * P] = d.x; g[(LF_CH_DIR + 1) * P] = d.y; g[(LF_CH_DIR + 2) * P] = d.z;
  g[LF_CH_STOPKEY_LO * P] = __uint_as_float((unsigned)(s.stop_key & 0xffffffffull));
  add_counters(a.counters, cnt, (unsigned)s.hits, 1u);
}

cudaError_t launch_trace_primary(const TraceArgs& a, const CamDev& cam, float* gbuf, cudaStream_t st) {
  dim3 grid((cam.W + 15) / 16, (cam.H + 7) / 8);
  k_trace_primary<<<grid, TB, STACK_SMEM, st>>>(a, cam, gbuf);
  return cudaGetLastError();
}

}  // namespace lf
