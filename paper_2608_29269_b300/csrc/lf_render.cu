// Primary-ray compositing (Eq. 6-7) and one-bounce shading (Eq. 10-11).
#include "lf_kernels.h"

namespace lf {

constexpr int TB = 128;  // threads per block
constexpr int G = 8;     // sample lanes per pixel in the shading kernels
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

struct PixelRecord {
  float T;
  int hits;
  float3 x, n, a, d;
  float m, r;
};

__device__ __forceinline__ PixelRecord load_record(const float* __restrict__ gbuf, size_t P, int p) {
  PixelRecord q;
  const float* g = gbuf + p;
  q.T = __ldg(g + LF_CH_T * P);
  q.hits = (int)__ldg(g + LF_CH_HITS * P);
  q.x = f3(__ldg(g + (LF_CH_X + 0) * P), __ldg(g + (LF_CH_X + 1) * P), __ldg(g + (LF_CH_X + 2) * P));
  q.n = f3(__ldg(g + (LF_CH_N + 0) * P), __ldg(g + (LF_CH_N + 1) * P), __ldg(g + (LF_CH_N + 2) * P));
  q.a = f3(__ldg(g + (LF_CH_A + 0) * P), __ldg(g + (LF_CH_A + 1) * P), __ldg(g + (LF_CH_A + 2) * P));
  q.m = __ldg(g + LF_CH_M * P);
  q.r = __ldg(g + LF_CH_R * P);
  q.d = f3(__ldg(g + (LF_CH_DIR + 0) * P), __ldg(g + (LF_CH_DIR + 1) * P), __ldg(g + (LF_CH_DIR + 2) * P));
  return q;
}

// Eq. 11, one (pixel, sample): environment NEE at the primary record, a BSDF
// continuation from the cosine/GGX mixture to at most one secondary record
// with two environment NEE samples there; power-heuristic MIS between the
// primary NEE and the escaped part of the continuation.
__device__ __forceinline__ float3 shade_sample(const TraceArgs& a, const Inst* insts, const PixelRecord& q,
                                               uint32_t pixel, int s, uint32_t k0, uint32_t k1, int* stack,
                                               Counters& cnt, unsigned& rays, unsigned& comp) {
  const DevParams& P = a.P;
  const float3 wo = -q.d, n = q.n;
  const float3 xs = q.x + n * P.ray_offset;
  const float ps = P.brdf_mode == 1 ? 0.0f : P.p_spec;
  float u[9];
  sample_uniforms(pixel, (uint32_t)s, k0, k1, u);
  float3 c = f3(0.f, 0.f, 0.f);
  if (P.sampling_mode != 1) {
    float3 we;
    float pe;
    env_sample(a.env, u[0], u[1], we, pe);
    const float ce = dot3(n, we);
    if (ce > 0.0f && pe > 0.0f) {
      const float Ve = trace_shadow(insts, a.n_inst, xs, we, P, stack, TB, a.status, cnt);
      ++rays;
      const float pb = pdf_bsdf(n, wo, we, q.r, ps);
      const float wenv = P.sampling_mode == 2 ? 1.0f : pe * pe / (pe * pe + pb * pb);
      const float3 f = brdf_eval(n, wo, we, q.a, q.m, q.r, P.brdf_mode);
      c = mul3(f, env_lookup(a.env, we)) * (ce * Ve * wenv / pe);
    }
  }
  const float3 wi = (u[2] < ps) ? sample_ggx(n, wo, q.r, u[3], u[4]) : sample_cos(n, u[3], u[4]);
  const float ci = dot3(n, wi);
  const float pb = pdf_bsdf(n, wo, wi, q.r, ps);
  if (!(ci > 0.0f && pb > 0.0f)) return c;
  const float pei = env_pdf(a.env, wi);
  const float wb = P.sampling_mode == 1 ? 1.0f : pb * pb / (pb * pb + pei * pei);
  Surface s2;
  trace_composite(insts, a.n_inst, xs, wi, P, stack, TB, a.status, cnt, s2, comp);
  ++rays;
  float3 inc = P.sampling_mode == 2 ? f3(0.f, 0.f, 0.f) : env_lookup(a.env, wi) * (wb * s2.T);
  if (s2.hits > 0) {
    const float3 n2 = s2.n, wo2 = -wi;
    const float co2 = dot3(n2, wo2);
    const float3 xs2 = s2.x + n2 * P.ray_offset;
#pragma unroll 1
    for (int qq = 0; qq < 2; ++qq) {
      float3 wq;
      float pq;
      env_sample(a.env, u[5 + 2 * qq], u[6 + 2 * qq], wq, pq);
      const float cq = dot3(n2, wq);
      if (!(cq > 0.0f && co2 > 0.0f && pq > 0.0f)) continue;
      const float Vq = trace_shadow(insts, a.n_inst, xs2, wq, P, stack, TB, a.status, cnt);
      ++rays;
      const float3 f2 = brdf_eval(n2, wo2, wq, s2.a, s2.m, s2.r, P.brdf_mode);
      add3(inc, mul3(f2, env_lookup(a.env, wq)) * (cq * (1.0f - s2.T) * 0.5f * Vq / pq));
    }
  }
  const float3 f = brdf_eval(n, wo, wi, q.a, q.m, q.r, P.brdf_mode);
  add3(c, mul3(f * (ci / pb), inc));
  return c;
}

// G lanes per pixel; lane l takes samples l, l + G, ...; the lanes' partial
// sums are combined by a fixed xor tree (deterministic for a given spp).
__global__ void __launch_bounds__(TB) k_shade(TraceArgs a, const float* __restrict__ gbuf, int n_pix, int spp,
                                              uint32_t k0, uint32_t k1, float* __restrict__ rgb,
                                              unsigned long long* ray_count) {
  __shared__ Inst s_inst[LF_MAX_OBJECTS];
  extern __shared__ int s_stack[];
  load_instances(s_inst, a.insts, a.n_inst);
  const int p = blockIdx.x * (TB / G) + threadIdx.x / G, lane = threadIdx.x % G;
  const bool valid = p < n_pix;
  PixelRecord q;
  float3 sum = f3(0.f, 0.f, 0.f);
  unsigned rays = 0, comp = 0;
  Counters cnt;
  if (valid) {
    q = load_record(gbuf, (size_t)n_pix, p);
    if (q.hits > 0 && dot3(q.n, -q.d) > 0.0f) {
      for (int s = lane; s < spp; s += G)
        add3(sum, shade_sample(a, s_inst, q, (uint32_t)p, s, k0, k1, s_stack + threadIdx.x, cnt, rays, comp));
    }
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) {
    sum.x += __shfl_xor_sync(0xffffffffu, sum.x, off);
    sum.y += __shfl_xor_sync(0xffffffffu, sum.y, off);
    sum.z += __shfl_xor_sync(0xffffffffu, sum.z, off);
  }
  const unsigned wr = __reduce_add_sync(0xffffffffu, rays);
  if (ray_count && (threadIdx.x & 31) == 0 && wr) atomicAdd(ray_count, (unsigned long long)wr);
  if (a.counters) add_counters(a.counters, cnt, comp, rays);
  if (valid && lane == 0) {
    const float3 L = env_lookup(a.env, q.d) * q.T + sum * ((1.0f - q.T) / (float)spp);
    rgb[3 * p + 0] = L.x;
    rgb[3 * p + 1] = L.y;
    rgb[3 * p + 2] = L.z;
  }
}

cudaError_t launch_trace_primary(const TraceArgs& a, const CamDev& cam, float* gbuf, cudaStream_t st) {
  dim3 grid((cam.W + 15) / 16, (cam.H + 7) / 8);
  k_trace_primary<<<grid, TB, STACK_SMEM, st>>>(a, cam, gbuf);
  return cudaGetLastError();
}

cudaError_t launch_shade(const TraceArgs& a, const float* gbuf, int n_pix, int spp, uint32_t k0, uint32_t k1,
                         float* rgb, unsigned long long* ray_count, cudaStream_t st) {
  const int ppb = TB / G;
  k_shade<<<(n_pix + ppb - 1) / ppb, TB, STACK_SMEM, st>>>(a, gbuf, n_pix, spp, k0, k1, rgb, ray_count);
  return cudaGetLastError();
}

}  // namespace lf
