// Adjoint of the primary composite (Eq. 6-7).
//
// k_trace_backward re-traverses each primary ray back to front from the
// stored final transmittance and stop key (no per-ray hit lists), recovers
// T_j = T_{j+1} / (1 - alpha_j) and scatters the adjoint of Eq. 6-7 to the
// surfel parameters; its upstream gradients are those of the G-buffer
// channels plus the shading adjoint's record gradients (normal, base colour,
// metallic, roughness, final transmittance).
#include "lf_kernels.h"

namespace lf {

constexpr int TB = 128;
constexpr int STACK_SMEM = TB * STACK * (int)sizeof(int);

__device__ __forceinline__ void load_instances_b(Inst* dst, const Inst* src, int n) {
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < n * 4; i += blockDim.x) d[i] = s[i];
  __syncthreads();
}

// d_env += v at the four bilinear texels of direction w.
__device__ __forceinline__ void env_scatter_p(const EnvDev& e, float* __restrict__ d_env, float3 w, float3 v) {
  if (!d_env) return;
  const Bilin b = env_bilinear(e, w);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (b.w[k] == 0.0f) continue;
    float* t = d_env + 3 * b.idx[k];
    atomicAdd(t + 0, b.w[k] * v.x);
    atomicAdd(t + 1, b.w[k] * v.y);
    atomicAdd(t + 2, b.w[k] * v.z);
  }
}

// Adjoint of Eq. 6 for one hit, scattered to the raw surfel parameters.
__device__ __forceinline__ void surfel_adjoint(const SceneDev& sc, int id, float3 o, float3 d, const DevParams& P,
                                               float g_alpha, float3 g_x, float g_t_direct, float3 g_n, float3 g_a,
                                               float g_m, float g_r, float* __restrict__ d_surfel) {
  const float3 mu = f3(sc.mu[3 * id], sc.mu[3 * id + 1], sc.mu[3 * id + 2]);
  const float3 tu = f3(sc.tu[3 * id], sc.tu[3 * id + 1], sc.tu[3 * id + 2]);
  const float3 tv = f3(sc.tv[3 * id], sc.tv[3 * id + 1], sc.tv[3 * id + 2]);
  const float su = sc.scale[2 * id], sv = sc.scale[2 * id + 1], op = sc.opacity[id];
  const float3 c = cross3(tu, tv);
  const float cl = sqrtf(dot3(c, c));
  const float3 nh = c * (1.0f / cl);
  const float den = dot3(d, c);
  const float3 pm = mu - o;
  const float t = dot3(pm, c) / den;
  const float3 q = d * t - pm;  // x - mu
  const float u = dot3(q, tu) / su, v = dot3(q, tv) / sv;
  const float Gs = expf(-0.5f * (u * u + v * v));
  const float oG = op * Gs;
  const bool capped = oG > P.alpha_max;
  const float g_o = capped ? 0.0f : g_alpha * Gs;
  const float g_r2 = capped ? 0.0f : -0.5f * g_alpha * oG;
  const float g_u = 2.0f * u * g_r2, g_v = 2.0f * v * g_r2;
  const float3 g_q = tu * (g_u / su) + tv * (g_v / sv);
  float3 g_tu = q * (g_u / su), g_tv = q * (g_v / sv);
  const float g_su = -g_u * u / su, g_sv = -g_v * v / sv;
  const float g_t = g_t_direct + dot3(g_x, d) + dot3(g_q, d);
  const float3 g_mu = c * (g_t / den) - g_q;
  float3 g_c = q * (-g_t / den);
  const float3 g_nh = dot3(d, nh) < 0.0f ? g_n : -g_n;
  add3(g_c, (g_nh - nh * dot3(nh, g_nh)) * (1.0f / cl));
  add3(g_tu, cross3(tv, g_c));
  add3(g_tv, cross3(g_c, tu));
  float* o17 = d_surfel + (size_t)LF_G_STRIDE * id;
  atomicAdd(o17 + 0, g_mu.x); atomicAdd(o17 + 1, g_mu.y); atomicAdd(o17 + 2, g_mu.z);
  atomicAdd(o17 + 3, g_tu.x); atomicAdd(o17 + 4, g_tu.y); atomicAdd(o17 + 5, g_tu.z);
  atomicAdd(o17 + 6, g_tv.x); atomicAdd(o17 + 7, g_tv.y); atomicAdd(o17 + 8, g_tv.z);
  atomicAdd(o17 + 9, g_su); atomicAdd(o17 + 10, g_sv);
  atomicAdd(o17 + 11, g_o);
  atomicAdd(o17 + 12, g_a.x); atomicAdd(o17 + 13, g_a.y); atomicAdd(o17 + 14, g_a.z);
  atomicAdd(o17 + 15, g_m);
  atomicAdd(o17 + 16, g_r);
}

// Per-pixel adjoint state of the back-to-front pass.
struct BackState {
  float3 gSx, gSn, gSa;
  float gSt, gSm, gSr, gW;
  float S, Tn;  // suffix sum of Eq. 7's alpha adjoint; transmittance behind the current hit
  int remaining, rounds;
  unsigned long long bound;
  bool inclusive;
};

// Upstream gradients of one pixel's record -> adjoints of the Eq. 7 sums;
// false when the pixel has no composited hit.
__device__ __forceinline__ bool back_setup(const TraceArgs& a, const float* __restrict__ gbuf,
                                           const float* __restrict__ sg, const float* __restrict__ gg, size_t P,
                                           int p, float3& d, BackState& b, float* d_env) {
  const float* gb = gbuf + p;
  auto ch = [&](int c) { return __ldg(gb + (size_t)c * P); };
  auto up = [&](int c) { return gg ? __ldg(gg + (size_t)c * P + p) : 0.0f; };
  d = f3(ch(LF_CH_DIR), ch(LF_CH_DIR + 1), ch(LF_CH_DIR + 2));
  const float T = ch(LF_CH_T), W = ch(LF_CH_W), depth = ch(LF_CH_DEPTH), nlen = ch(LF_CH_NLEN);
  const float3 xb = f3(ch(LF_CH_X), ch(LF_CH_X + 1), ch(LF_CH_X + 2));
  const float3 nb = f3(ch(LF_CH_N), ch(LF_CH_N + 1), ch(LF_CH_N + 2));
  const float3 ab = f3(ch(LF_CH_A), ch(LF_CH_A + 1), ch(LF_CH_A + 2));
  const float mb = ch(LF_CH_M), rb = ch(LF_CH_R);
  const int hits = (int)ch(LF_CH_HITS);
  float3 g_n = f3(up(LF_CH_N), up(LF_CH_N + 1), up(LF_CH_N + 2));
  float3 g_a = f3(up(LF_CH_A), up(LF_CH_A + 1), up(LF_CH_A + 2));
  float g_m = up(LF_CH_M), g_r = up(LF_CH_R), g_T = up(LF_CH_T);
  const float g_W = up(LF_CH_W), g_depth = up(LF_CH_DEPTH);
  const float3 g_x = f3(up(LF_CH_X), up(LF_CH_X + 1), up(LF_CH_X + 2));
  const float3 g_rho = f3(up(LF_CH_RHO), up(LF_CH_RHO + 1), up(LF_CH_RHO + 2));
  if (sg) {
    g_n = g_n + f3(__ldg(sg + 0 * P + p), __ldg(sg + 1 * P + p), __ldg(sg + 2 * P + p));
    g_a = g_a + f3(__ldg(sg + 3 * P + p), __ldg(sg + 4 * P + p), __ldg(sg + 5 * P + p));
    g_m += __ldg(sg + 6 * P + p);
    g_r += __ldg(sg + 7 * P + p);
    g_T += __ldg(sg + 8 * P + p);
  }
  if (gg) {  // rho = sum w a + T E(d)
    const float3 Ed = env_lookup(a.env, d);
    g_T += dot3(g_rho, Ed);
    env_scatter_p(a.env, d_env, d, g_rho * T);
  }
  if (hits <= 0) return false;
  const float inv = 1.0f / (W + a.P.eps_w);
  b.gSx = g_x * inv;
  b.gSa = g_a * inv + g_rho;
  b.gSt = g_depth * inv;
  b.gSm = g_m * inv;
  b.gSr = g_r * inv;
  float3 gmv = f3(0.f, 0.f, 0.f), mv = f3(0.f, 0.f, 0.f);
  if (nlen >= 1e-12f) {
    gmv = (g_n - nb * dot3(nb, g_n)) * (1.0f / nlen);
    mv = nb * nlen;
  }
  b.gSn = gmv * inv;
  b.gW = g_W - inv * (dot3(g_x, xb) + g_depth * depth + dot3(g_a, ab) + g_m * mb + g_r * rb + dot3(gmv, mv));
  b.S = g_T * T;
  b.Tn = T;
  b.remaining = hits;
  b.rounds = 0;
  b.bound = ((unsigned long long)__float_as_uint(ch(LF_CH_TSTOP)) << 32) |
            (unsigned long long)__float_as_uint(ch(LF_CH_STOPKEY_LO));
  b.inclusive = true;
  return true;
}

// Persistent: lanes take pixels in 16 x 8 tile order; per pixel, rounds of
// "the K farthest hits at or below the bound" are processed back to front.
__global__ void __launch_bounds__(TB) k_trace_backward(TraceArgs a, SceneDev sc, CamDev cam,
                                                       const float* __restrict__ gbuf,
                                                       const float* __restrict__ sg,
                                                       const float* __restrict__ gg, float* __restrict__ d_surfel,
                                                       float* __restrict__ d_env, int* fetch) {
  __shared__ Inst s_inst[LF_MAX_OBJECTS];
  extern __shared__ int s_stack[];
  load_instances_b(s_inst, a.insts, a.n_inst);
  int* stack = s_stack + threadIdx.x;
  const int tiles_x = (cam.W + 15) / 16, tiles_y = (cam.H + 7) / 8;
  const int n = tiles_x * tiles_y * 128;
  const size_t P = (size_t)cam.W * cam.H;
  const DevParams& Pm = a.P;
  const float3 o = cam.eye;
  Counters cnt;
  bool live = false, exhausted = false;
  float3 d = f3(0.f, 0.f, 1.f);
  Ray ray;
  FarK kb;
  kb.P = Pm;
  BackState b;
  Trav tr;
  while (true) {
    const int k = warp_fetch(fetch, n, !live, exhausted);
    if (!live && k < n) {
      const int tile = k >> 7, w = k & 127;
      const int x = (tile % tiles_x) * 16 + (w & 15), y = (tile / tiles_x) * 8 + (w >> 4);
      if (x < cam.W && y < cam.H && back_setup(a, gbuf, sg, gg, P, y * cam.W + x, d, b, d_env)) {
        ray = make_ray(o, d);
        kb.o = o;
        kb.d = d;
        kb.reset(b.bound, b.inclusive);
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
    if (tr.overflow) {
      report(a.status, LF_ERR_STACK);
      live = false;
      continue;
    }
    const int nk = kb.cnt;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      if (j < nk && b.remaining > 0) {
        const int code = kb.bc[j];
        const Inst& I = s_inst[code >> 24];
        const int l = code & 0xffffff;
        const Rec rc = load_rec(I.geo, l);
        const float4 mt = __ldg(I.mat + l);
        float t, tl, alpha;
        hit_precise(rc, o, d, Pm, t, tl, alpha);
        const float3 nj = record_normal(rc, d);
        const float3 xj = o + d * t;
        const float Tj = b.Tn / (1.0f - alpha);
        const float wgt = Tj * alpha;
        const float gw = b.gW + dot3(b.gSx, xj) + b.gSt * t + dot3(b.gSn, nj) + b.gSa.x * mt.x +
                         b.gSa.y * mt.y + b.gSa.z * mt.z + b.gSm * mt.w + b.gSr * rc.g2.w;
        const float g_alpha = Tj * gw - b.S / (1.0f - alpha);
        b.S += gw * wgt;
        b.Tn = Tj;
        surfel_adjoint(sc, __float_as_int(rc.g1.w), o, d, Pm, g_alpha, b.gSx * wgt, b.gSt * wgt, b.gSn * wgt,
                       b.gSa * wgt, b.gSm * wgt, b.gSr * wgt, d_surfel);
        --b.remaining;
      }
    }
    if (b.remaining > 0 && nk == K && ++b.rounds < Pm.max_rounds) {
      b.bound = kb.bk[K - 1];
      b.inclusive = false;
      kb.reset(b.bound, false);
      tr.start(s_inst, a.n_inst, ray, kb.tlo(), kb.thi(), stack, TB);
      continue;
    }
    // finished; hits left over mean the re-traversal found fewer hits than
    // the forward composited
    if (b.remaining > 0) report(a.status, LF_ERR_ROUND_LIMIT);
    live = false;
  }
}

cudaError_t launch_trace_backward(const TraceArgs& a, const SceneDev& s, const CamDev& cam, const float* gbuf,
                                  const float* shade_grad, const float* dL_dgbuf, float* d_surfel, float* d_env,
                                  int* fetch, int sms, cudaStream_t st) {
  static int per_sm = 0;
  if (!per_sm && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_backward, TB, STACK_SMEM) !=
                      cudaSuccess || per_sm < 1))
    per_sm = 1;
  cudaError_t e = cudaMemsetAsync(fetch, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  k_trace_backward<<<per_sm * sms, TB, STACK_SMEM, st>>>(a, s, cam, gbuf, shade_grad, dL_dgbuf, d_surfel, d_env,
                                                         fetch);
  return cudaGetLastError();
}

}  // namespace lf
