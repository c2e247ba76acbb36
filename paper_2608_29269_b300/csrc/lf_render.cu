// Primary-ray compositing (Eq. 6-7).
#include "lf_kernels.h"

namespace lf {

constexpr int TB = 128;  // threads per block
constexpr int STACK_SMEM = TB * STACK * (int)sizeof(int);

__device__ __forceinline__ void load_instances(Inst* dst, const Inst* src, int n) {
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < n * 4; i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

__device__ __forceinline__ void add_counters(unsigned long long* c, const Counters& k, unsigned comp, unsigned rays) {
  if (!c) return;
  atomicAdd(c + 0, (unsigned long long)k.nodes);
  atomicAdd(c + 1, (unsigned long long)k.tests);
  atomicAdd(c + 2, (unsigned long long)comp);
  atomicAdd(c + 3, (unsigned long long)rays);
}

// Persistent: lanes take pixels in 16 x 8 tile order (coherent primary rays)
// and fetch the next pixel when theirs is composited.
__global__ void __launch_bounds__(TB) k_trace_primary(TraceArgs a, CamDev cam, float* __restrict__ gbuf,
                                                      int* fetch) {
  __shared__ Inst s_inst[LF_MAX_OBJECTS];
  extern __shared__ int s_stack[];
  load_instances(s_inst, a.insts, a.n_inst);
  int* stack = s_stack + threadIdx.x;
  const int tiles_x = (cam.W + 15) / 16, tiles_y = (cam.H + 7) / 8;
  const int n = tiles_x * tiles_y * 128;
  const size_t P = (size_t)cam.W * cam.H;
  Counters cnt;
  unsigned comp = 0, rays = 0;
  bool live = false, exhausted = false;
  int p = 0;
  float3 d = f3(0.f, 0.f, 1.f);
  Ray ray;
  NearK kb;
  kb.P = a.P;
  Compositor cp;
  Trav tr;
  while (true) {
    const int k = warp_fetch(fetch, n, !live, exhausted);
    if (!live && k < n) {
      const int tile = k >> 7, w = k & 127;
      const int x = (tile % tiles_x) * 16 + (w & 15), y = (tile / tiles_x) * 8 + (w >> 4);
      if (x < cam.W && y < cam.H) {
        p = y * cam.W + x;
        d = camera_dir(cam, p);
        ray = make_ray(cam.eye, d);
        kb.o = cam.eye;
        kb.d = d;
        kb.reset(0ull);
        cp.init();
        tr.start(s_inst, a.n_inst, ray, kb.tlo(), kb.thi(), stack, TB);
        live = true;
      }
    }
    if (!__any_sync(0xffffffffu, live) && exhausted) break;
    if (!live) continue;
    const int leaf = tr.next_leaf(s_inst, ray, kb.tlo(), kb.thi(), stack, TB, cnt);
    if (leaf >= 0) {
      kb.leaf(leaf >> 25, leaf & 0xffffff, s_inst[leaf >> 25]);
      continue;
    }
    bool fin = tr.overflow;
    if (fin) report(a.status, LF_ERR_STACK);
    else fin = cp.round(kb, s_inst, cam.eye, d, a.P, a.status);
    if (!fin) {
      kb.reset(cp.last);
      tr.start(s_inst, a.n_inst, ray, kb.tlo(), kb.thi(), stack, TB);
      continue;
    }
    live = false;
    ++rays;
    comp += (unsigned)cp.hits;
    Surface s;
    cp.surface(d, a.P, s);
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
  }
  add_counters(a.counters, cnt, comp, rays);
}

cudaError_t launch_trace_primary(const TraceArgs& a, const CamDev& cam, float* gbuf, int* fetch, int sms,
                                 cudaStream_t st) {
  static int per_sm = 0;
  if (!per_sm && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_primary, TB, STACK_SMEM) !=
                      cudaSuccess || per_sm < 1))
    per_sm = 1;
  cudaError_t e = cudaMemsetAsync(fetch, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_trace_primary<<<per_sm * sms, TB, STACK_SMEM, st>>>(a, cam, gbuf, fetch);
  return cudaGetLastError();
}

}  // namespace lf
