// Adjoint of the primary composite (Eq. 6-7).
//
// k_trace_backward re-traverses each primary ray back to front from the
// stored final transmittance and stop key (no per-ray hit lists), recovers
// T_j = T_{j+1} / (1 - alpha_j) and scatters the adjoint of Eq. 6-7 to the
// surfel parameters; its upstream gradients are those of the G-buffer
// channels plus the shading adjoint's record gradients (normal, base colour,
// metallic, roughness, final transmittance).
#include "lf_coop.cuh"
#include "lf_kernels.h"

namespace lf {

constexpr int TB = 128;
#ifndef BACKWARD_MIN_BLOCKS
#define BACKWARD_MIN_BLOCKS 8  // resident blocks per SM asked of the compiler (10 and 12 measured slower)
#endif
#ifndef BACKWARD_RAY
#define BACKWARD_RAY RayR  // the ray in registers (RayS measured slower here)
#endif
constexpr int BGROUPS = TB / WIDE;  // pixels per block (one per lane group)
constexpr int BSTACK_SMEM = BGROUPS * CRAY_SMEM;
constexpr int BTILE_W = BGROUPS >= 4 ? 4 : BGROUPS;
constexpr int BTILE_H = BGROUPS / BTILE_W;

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

// WIDE lanes per pixel.  Each round collects the K hits just in front of the
// bound (cooperative far k-buffer, descending over the lanes), then processes
// them at once: with P_c = prod_{i <= c} (1 - alpha_i) over the lanes,
// T_c = T_in / P_c, and the running sum S of the later hits' gw w is an
// exclusive prefix sum; each lane scatters its own hit's adjoint.
template <class Cnt>
__global__ void __launch_bounds__(TB, BACKWARD_MIN_BLOCKS) k_trace_backward(TraceArgs a, SceneDev sc, CamDev cam,
                                                       const float* __restrict__ gbuf,
                                                       const float* __restrict__ sg,
                                                       const float* __restrict__ gg, float* __restrict__ d_surfel,
                                                       float* __restrict__ d_env) {
  extern __shared__ __align__(16) int s_cstack[];
  const Grp g = make_grp();
  const int gid = threadIdx.x / WIDE;
  const CStack st = ray_smem(reinterpret_cast<unsigned char*>(s_cstack), BGROUPS, gid);
  const int x = blockIdx.x * BTILE_W + gid % BTILE_W, y = blockIdx.y * BTILE_H + gid / BTILE_W;
  if (x >= cam.W || y >= cam.H) return;  // uniform over the group
  const int p = y * cam.W + x;
  const size_t P = (size_t)cam.W * cam.H;
  const DevParams& Pm = a.P;
  const float* gb = gbuf + p;
  auto ch = [&](int c) { return __ldg(gb + (size_t)c * P); };
  auto up = [&](int c) { return gg ? __ldg(gg + (size_t)c * P + p) : 0.0f; };
  const float3 o = cam.eye;
  const float3 d = f3(ch(LF_CH_DIR), ch(LF_CH_DIR + 1), ch(LF_CH_DIR + 2));
  const float T = ch(LF_CH_T), W = ch(LF_CH_W), depth = ch(LF_CH_DEPTH), nlen = ch(LF_CH_NLEN);
  const float3 xb = f3(ch(LF_CH_X), ch(LF_CH_X + 1), ch(LF_CH_X + 2));
  const float3 nb = f3(ch(LF_CH_N), ch(LF_CH_N + 1), ch(LF_CH_N + 2));
  const float3 ab = f3(ch(LF_CH_A), ch(LF_CH_A + 1), ch(LF_CH_A + 2));
  const float mb = ch(LF_CH_M), rb = ch(LF_CH_R);
  const int hits = (int)ch(LF_CH_HITS);
  // upstream gradients on the record
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
  // rho = sum w a + T E(d)
  if (gg) {
    const float3 Ed = env_lookup(a.env, d);
    g_T += dot3(g_rho, Ed);
    if (g.c == 0) env_scatter_p(a.env, d_env, d, g_rho * T);
  }
  if (hits <= 0) return;
  const float inv = 1.0f / (W + Pm.eps_w);
  const float3 gSx = g_x * inv, gSa = g_a * inv + g_rho;
  const float gSt = g_depth * inv, gSm = g_m * inv, gSr = g_r * inv;
  float3 gmv = f3(0.f, 0.f, 0.f), mv = f3(0.f, 0.f, 0.f);
  if (nlen >= 1e-12f) {
    gmv = (g_n - nb * dot3(nb, g_n)) * (1.0f / nlen);
    mv = nb * nlen;
  }
  const float3 gSn = gmv * inv;
  const float gW = g_W - inv * (dot3(g_x, xb) + g_depth * depth + dot3(g_a, ab) + g_m * mb + g_r * rb + dot3(gmv, mv));
  float S = g_T * T;
  float Tn = T;
  int remaining = hits;
  unsigned long long bound = ((unsigned long long)__float_as_uint(ch(LF_CH_TSTOP)) << 32) |
                             (unsigned long long)__float_as_uint(ch(LF_CH_STOPKEY_LO));
  bool inclusive = true;
  FarKCoop kb;
  kb.P = Pm;
  kb.mk = st.mk;
  kb.mc = st.mc;
  kb.insts = a.insts;
  kb.qc = st.qc;
  const auto ray = make_ray<BACKWARD_RAY>(st.ray, g.c, g.mask, o, d);
  Cnt cnt;
  unsigned adj = 0;  // hits whose gradient this ray scatters
  for (int round = 0; round < Pm.max_rounds && remaining > 0; ++round) {
    kb.reset(bound, inclusive);
    coop_traverse(g, a.insts, a.n_inst, ray, kb, st, a.status, cnt);
    const int n = kb.cnt;
    const int take = min(n, remaining);
    bool have = g.c < take;
    if (have) have = LF_IN_BOUNDS(kb.bc >> 24, a.n_inst, a.status, "hit instance") &&
                     LF_IN_BOUNDS(kb.bc & 0xffffff, a.insts[kb.bc >> 24].n_leaves, a.status, "hit surfel");
    float alpha = 0.0f, t = 0.0f, gw = 0.0f;
    Rec rc;
    float4 mt = make_float4(0.f, 0.f, 0.f, 0.f);
    float3 nj = f3(0.f, 0.f, 0.f);
    if (have) {
      const Inst& I = a.insts[kb.bc >> 24];
      const int l = kb.bc & 0xffffff;
      rc = load_rec(I.geo, I.n_leaves, l);
      mt = __ldg(I.mat + l);
      float tl;
      hit_precise(rc, o, f3(0.f, 0.f, 0.f), d, Pm, t, tl, alpha);
      nj = record_normal(rc, d);
      const float3 xj = o + d * t;
      gw = gW + dot3(gSx, xj) + gSt * t + dot3(gSn, nj) + gSa.x * mt.x + gSa.y * mt.y + gSa.z * mt.z +
           gSm * mt.w + gSr * rec_rough(rc);
    }
    // P_c = prod_{i <= c} (1 - alpha_i): T_c = Tn / P_c
    float q = have ? 1.0f - alpha : 1.0f;
#pragma unroll
    for (int off = 1; off < WIDE; off <<= 1) {
      const float v = __shfl_up_sync(g.mask, q, off, WIDE);
      if (g.c >= off) q *= v;
    }
    const float Tj = Tn / q;
    const float w = have ? Tj * alpha : 0.0f;
    // S before this hit: S_in + sum over the lanes in front (exclusive prefix sum of gw w)
    float e = have ? gw * w : 0.0f;
    float incl = e;
#pragma unroll
    for (int off = 1; off < WIDE; off <<= 1) {
      const float v = __shfl_up_sync(g.mask, incl, off, WIDE);
      if (g.c >= off) incl += v;
    }
    if (have) {
      const float Sj = S + (incl - e);
      const float g_alpha = Tj * gw - Sj / (1.0f - alpha);
      surfel_adjoint(sc, rec_id(rc), o, d, Pm, g_alpha, gSx * w, gSt * w, gSn * w, gSa * w, gSm * w,
                     gSr * w, d_surfel);
    }
    if (take > 0) {
      S += gshfl(g, incl, take - 1);
      Tn = gshfl(g, Tj, take - 1);
    }
    remaining -= take;
    adj += (unsigned)take;
    if (remaining > 0) {
      if (n < WIDE) {  // the forward composited more hits than the re-traversal finds
        if (g.c == 0) report(a.status, LF_ERR_ROUND_LIMIT);
        break;
      }
      bound = kb.kmin;
      inclusive = false;
    }
  }
  if (Cnt::on && a.counters && g.c == 0) {  // slot 4 of the per-kernel counters: adjoint rays
    atomicAdd(a.counters + 16, (unsigned long long)cnt.nodes);
    atomicAdd(a.counters + 17, (unsigned long long)cnt.tests);
    atomicAdd(a.counters + 18, (unsigned long long)adj);
    atomicAdd(a.counters + 19, 1ull);
  }
}

cudaError_t launch_trace_backward(const TraceArgs& a, const SceneDev& s, const CamDev& cam, const float* gbuf,
                                  const float* shade_grad, const float* dL_dgbuf, float* d_surfel, float* d_env,
                                  cudaStream_t st) {
  dim3 grid((cam.W + BTILE_W - 1) / BTILE_W, (cam.H + BTILE_H - 1) / BTILE_H);
  if (a.counters)
    k_trace_backward<Counters><<<grid, TB, BSTACK_SMEM, st>>>(a, s, cam, gbuf, shade_grad, dL_dgbuf, d_surfel, d_env);
  else
    k_trace_backward<NoCounters><<<grid, TB, BSTACK_SMEM, st>>>(a, s, cam, gbuf, shade_grad, dL_dgbuf, d_surfel,
                                                                d_env);
  return cudaGetLastError();
}

}  // namespace lf
