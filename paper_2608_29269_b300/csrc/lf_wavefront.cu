// One-bounce shading (Eq. 10-11) as a wavefront of small kernels, and its
// path-replay adjoint (Sec. 3.3).
//
// Work item = (job, pixel, sample).  Per batch:
//   k_wf_gen      per item: Philox uniforms; environment NEE direction and
//                 MIS factor; BSDF continuation direction from the
//                 cosine/GGX mixture; appends NEE shadow rays to queue A and
//                 continuation rays to queue B.
//   k_wf_shadow   queue A: visibility V_e of the NEE rays.
//   k_wf_continue queue B: k-buffer composite of the continuation ray to the
//                 secondary record.
//   k_wf_secondary queue B: two environment NEE samples at the secondary
//                 record (factor f2 cos / pdf, ray origin), appended to queue C.
//   k_wf_shadow   queue C: visibility V_q of the secondary NEE rays.
//   k_wf_combine  per pixel: sum of the per-sample terms in sample order,
//                 L = T E(d) + (1 - T) / S * sum.
// The per-sample buffer holds exactly the data path replay keeps fixed
// (directions, pdfs, MIS weights, visibilities, secondary factors), so the
// adjoint (k_wf_combine_adjoint) differentiates the combine without
// re-tracing when it is given the forward's buffer; without it the first
// four kernels are replayed with the same seed first.
#include <algorithm>

#include "lf_coop.cuh"
#include "lf_wavefront.h"

namespace lf {

constexpr int WB = 128;  // threads per block of the wavefront kernels
// Minimum resident blocks per SM asked of the compiler (caps registers) and
// where the traced ray is held (RayS: shared memory, RayR: registers).
// Measured on the 800x800x16 room step: shadow rays 16 blocks (full
// occupancy, 32 registers) with RayS, 4 % faster than RayR; continuation
// rays 8 blocks (64 registers) with RayS, 1 % faster than 10 blocks with
// either kind and 5 % faster than 8 blocks with RayR.
#ifndef WF_MIN_BLOCKS_SHADOW
#define WF_MIN_BLOCKS_SHADOW 16
#endif
#ifndef WF_MIN_BLOCKS_CONTINUE
#define WF_MIN_BLOCKS_CONTINUE 8
#endif
#ifndef WF_SHADOW_RAY
#define WF_SHADOW_RAY RayS
#endif
#ifndef WF_CONTINUE_RAY
#define WF_CONTINUE_RAY RayS
#endif
// Slots of SampleBuf::counts: queue lengths A, B, C (0-2); fetch cursors of
// the three trace kernels (4-6).
constexpr int CURSOR_A = 4, CURSOR_B = 5, CURSOR_C = 6, N_COUNTS = 8;

// A sample's pixel and index within its job from its offset in the job
// (under 2^30: the entry points refuse larger sample counts), by a 32-bit
// division instead of a 64-bit one.
__device__ __forceinline__ int pixel_of(long long loc, int spp) { return (int)((unsigned)loc / (unsigned)spp); }
__device__ __forceinline__ int sample_of(long long loc, int spp) { return (int)((unsigned)loc % (unsigned)spp); }

__device__ __forceinline__ int job_of_item(const ShadeBatch& B, long long item) {
  int lo = 0, hi = B.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.jobs[mid].item0 <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ int job_of_pixel(const ShadeBatch& B, int gp) {
  int lo = 0, hi = B.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.jobs[mid].pix0 <= gp) lo = mid; else hi = mid - 1;
  }
  return lo;
}

struct PixRec {
  float T;
  int hits;
  float3 x, n, a, d;
  float m, r;
  float3 n_lo;  // residuals of the normal and roughness (precise record)
  float r_lo;
};

__device__ __forceinline__ PixRec pix_record(const ShadeJob& J, int p) {
  const size_t P = (size_t)J.n_pix;
  const float* g = J.gbuf + p;
  PixRec q;
  q.T = __ldg(g + LF_CH_T * P);
  q.hits = (int)__ldg(g + LF_CH_HITS * P);
  q.x = f3(__ldg(g + LF_CH_X * P), __ldg(g + (LF_CH_X + 1) * P), __ldg(g + (LF_CH_X + 2) * P));
  q.n = f3(__ldg(g + LF_CH_N * P), __ldg(g + (LF_CH_N + 1) * P), __ldg(g + (LF_CH_N + 2) * P));
  q.a = f3(__ldg(g + LF_CH_A * P), __ldg(g + (LF_CH_A + 1) * P), __ldg(g + (LF_CH_A + 2) * P));
  q.m = __ldg(g + LF_CH_M * P);
  q.r = __ldg(g + LF_CH_R * P);
  q.d = f3(__ldg(g + LF_CH_DIR * P), __ldg(g + (LF_CH_DIR + 1) * P), __ldg(g + (LF_CH_DIR + 2) * P));
  q.n_lo = f3(__ldg(g + LF_CH_N_LO * P), __ldg(g + (LF_CH_N_LO + 1) * P), __ldg(g + (LF_CH_N_LO + 2) * P));
  q.r_lo = __ldg(g + LF_CH_R_LO * P);
  return q;
}

// (x + xlo) + n off as a double-float hi + lo: the sum of the two FP32
// values is exact as a pair (the product n off carries ~1e-11), so shading
// rays start at the record's position (with its residual xlo) plus the
// offset.
__device__ __forceinline__ float3 offset_origin(float3 x, float3 xlo, float3 n, float off, float3& lo) {
  float3 hi;
  two_sum(x.x, n.x * off, hi.x, lo.x);
  two_sum(x.y, n.y * off, hi.y, lo.y);
  two_sum(x.z, n.z * off, hi.z, lo.z);
  lo = lo + xlo;
  return hi;
}

__device__ __forceinline__ float3 pix_origin(const ShadeJob& J, int p, float off, float3& lo) {
  const size_t P = (size_t)J.n_pix;
  const float* g = J.gbuf + p;
  const float3 x = f3(__ldg(g + LF_CH_X * P), __ldg(g + (LF_CH_X + 1) * P), __ldg(g + (LF_CH_X + 2) * P));
  const float3 xlo = f3(__ldg(g + LF_CH_X_LO * P), __ldg(g + (LF_CH_X_LO + 1) * P), __ldg(g + (LF_CH_X_LO + 2) * P));
  const float3 n = f3(__ldg(g + LF_CH_N * P), __ldg(g + (LF_CH_N + 1) * P), __ldg(g + (LF_CH_N + 2) * P));
  return offset_origin(x, xlo, n, off, lo);
}

__device__ __forceinline__ float3 ld3(const float* const* pl, long long i) {
  return f3(pl[0][i], pl[1][i], pl[2][i]);
}
__device__ __forceinline__ void st3(float* const* pl, long long i, float3 v) {
  pl[0][i] = v.x;
  pl[1][i] = v.y;
  pl[2][i] = v.z;
}

// Warp-aggregated append of `value` to a queue when `pred` holds.  Called by
// all 32 lanes of the warp together.
__device__ __forceinline__ void queue_push(int* q, int* counter, int value, bool pred) {
  const unsigned m = __ballot_sync(0xffffffffu, pred);
  if (m == 0u) return;
  const int lane = threadIdx.x & 31;
  const int leader = __ffs(m) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (pred) q[base + __popc(m & ((1u << lane) - 1u))] = value;
}

__device__ __forceinline__ void load_insts(Inst* dst, const Inst* src, int n) {
  const float4* s = reinterpret_cast<const float4*>(src);
  float4* d = reinterpret_cast<float4*>(dst);
  for (int i = threadIdx.x; i < n * (int)(sizeof(Inst) / sizeof(float4)); i += blockDim.x) d[i] = s[i];
}

// ---------------------------------------------------------------- generation
__global__ void __launch_bounds__(WB) k_wf_gen(ShadeBatch B, DevParams P, SampleBuf S) {
  for (long long base = (long long)blockIdx.x * blockDim.x; base < B.n_items; base += (long long)gridDim.x * blockDim.x) {
    const long long i = base + threadIdx.x;
    bool e_ok = false, b_ok = false;
    if (i < B.n_items) {
    const ShadeJob& J = B.jobs[job_of_item(B, i)];
    const long long loc = i - J.item0;
    const int p = pixel_of(loc, J.spp), s = sample_of(loc, J.spp);
    const PixRec q = pix_record(J, p);
    const float3 wo = -q.d, n = q.n;
    const float ps = P.brdf_mode == 1 ? 0.0f : P.p_spec;
    float3 we = f3(0.f, 0.f, 1.f), wi = f3(0.f, 0.f, 1.f);
    float ek = 0.0f, bc = 0.0f, wb = 0.0f;
    if (q.hits > 0 && dot3(n, wo) > 0.0f) {
      float u[9];
      sample_uniforms((uint32_t)p, (uint32_t)s, J.k0, J.k1, P.sampler, u);
      if (P.sampling_mode != 1) {
        float pe;
        env_sample(J.env, u[0], u[1], we, pe);
        if (dot3(n, we) > 0.0f && pe > 0.0f) {
          const float pb = pdf_bsdf(n, wo, we, q.r, ps);
          ek = (P.sampling_mode == 2 ? 1.0f : pe * pe / (pe * pe + pb * pb)) / pe;
          e_ok = true;
        }
      }
      wi = sample_bsdf_dir(u[2] < ps, n, q.n_lo, wo, q.r, q.r_lo, u[3], u[4]);
      const float pb = pdf_bsdf(n, wo, wi, q.r, ps);
      if (dot3(n, wi) > 0.0f && pb > 0.0f) {
        const float pei = env_pdf(J.env, wi);
        wb = P.sampling_mode == 1 ? 1.0f : pb * pb / (pb * pb + pei * pei);
        bc = 1.0f / pb;
        b_ok = true;
      }
    }
    st3(S.we, i, we);
    S.ek[i] = ek;
    st3(S.wi, i, wi);
    S.bc[i] = bc;
    S.wb[i] = wb;
    S.T2[i] = 1.0f;
    st3(S.fk0, i, f3(0.f, 0.f, 0.f));
    st3(S.fk1, i, f3(0.f, 0.f, 0.f));
    }
    queue_push(S.qA, S.counts + 0, (int)i, e_ok);
    queue_push(S.qB, S.counts + 1, (int)i, b_ok);
  }
}

// ---------------------------------------------------------------- shadow rays
// which = 0: NEE rays of queue A (origin from the G-buffer, direction we)
// which = 1: secondary NEE rays of queue C (entry = item * 2 + q)
// WIDE lanes trace each ray through the wide BVH (lf_coop.cuh); a group takes
// the next queue entry as soon as its ray has ended.
constexpr int WGROUPS = WB / WIDE;  // rays per block in the cooperative kernels
constexpr int CSTACK_SMEM = WGROUPS * CRAY_SMEM;

__device__ __forceinline__ CStack group_stack(int* smem) {
  return ray_smem(reinterpret_cast<unsigned char*>(smem), WGROUPS, threadIdx.x / WIDE);
}

// Next queue entry for the group (one atomic per ray).
__device__ __forceinline__ int group_fetch(const Grp& g, int* cursor) {
  int k = 0;
  if (g.c == 0) k = atomicAdd(cursor, 1);
  return gshfl(g, k, 0);
}

template <class Cnt>
__global__ void __launch_bounds__(WB, WF_MIN_BLOCKS_SHADOW) k_wf_shadow(ShadeBatch B, DevParams P, SampleBuf S,
                                                                        int which, int* status,
                                                                        unsigned long long* counters) {
  extern __shared__ __align__(16) int s_cstack[];
  const Grp g = make_grp();
  const CStack st = group_stack(s_cstack);
  const int* q = which == 0 ? S.qA : S.qC;
  const int n = which == 0 ? S.counts[0] : S.counts[2];
  int* cursor = S.counts + (which == 0 ? CURSOR_A : CURSOR_C);
  Cnt cnt;
  for (int k = group_fetch(g, cursor); k < n; k = group_fetch(g, cursor)) {
    const int e = q[k];
    const long long item = which == 0 ? (long long)e : (long long)(e >> 1);
    if (!LF_IN_BOUNDS(item, B.n_items, status, "shadow ray item")) continue;
    const ShadeJob& J = B.jobs[job_of_item(B, item)];
    ShadowCoop v;
    v.P = P;
    v.insts = J.insts;
    v.qc = st.qc;
    v.qn = 0;
    float3 o, olo, d;
    if (which == 0) {
      const long long loc = item - J.item0;
      o = pix_origin(J, pixel_of(loc, J.spp), P.ray_offset, olo);
      d = ld3(S.we, item);
    } else {
      o = ld3(S.xs2, item);
      olo = ld3(S.xs2lo, item);
      d = (e & 1) ? ld3(S.wq1, item) : ld3(S.wq0, item);
    }
    v.V = 1.0f;
    v.stop = false;
    const auto ray = make_ray<WF_SHADOW_RAY>(st.ray, g.c, g.mask, o, d, olo);
    coop_traverse(g, J.insts, J.n_inst, ray, v, st, status, cnt);
    if (g.c == 0) {
      if (which == 0) S.Ve[item] = v.V;
      else if (e & 1) S.Vq1[item] = v.V;
      else S.Vq0[item] = v.V;
    }
  }
  if (Cnt::on && counters && g.c == 0) {  // slot 1: NEE shadow rays, slot 3: secondary shadow rays
    unsigned long long* c = counters + 4 * (which == 0 ? 1 : 3);
    atomicAdd(c + 0, (unsigned long long)cnt.nodes);
    atomicAdd(c + 1, (unsigned long long)cnt.tests);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(c + 3, (unsigned long long)n);
  }
}

// ---------------------------------------------------------------- continuation rays
// The secondary record between k_wf_continue and k_wf_secondary is held in
// planes that are written for good only afterwards: normal in wq0, base
// colour in fk0, metallic in Vq0, roughness in Vq1.
__device__ __forceinline__ float* const* rec_n2(const SampleBuf& S) { return S.wq0; }
__device__ __forceinline__ float* const* rec_a2(const SampleBuf& S) { return S.fk0; }
__device__ __forceinline__ float* rec_m2(const SampleBuf& S) { return S.Vq0; }
__device__ __forceinline__ float* rec_r2(const SampleBuf& S) { return S.Vq1; }

// One warp per ray: cooperative k-buffer composite of the continuation ray
// to the secondary record (lf_coop.cuh).  Lane 0 stores T2 and, when the ray
// found a surface (then T2 < 1), the record for k_wf_secondary: the NEE
// origin in xs2 and normal, base colour, metallic and roughness in planes
// that k_wf_secondary and the secondary shadow rays overwrite afterwards.
template <class Cnt>
__global__ void __launch_bounds__(WB, WF_MIN_BLOCKS_CONTINUE) k_wf_continue(ShadeBatch B, DevParams P, SampleBuf S,
                                                                            int* status,
                                                                            unsigned long long* counters) {
  extern __shared__ __align__(16) int s_cstack[];
  const Grp g = make_grp();
  const CStack st = group_stack(s_cstack);
  const int n = S.counts[1];
  Cnt cnt;
  unsigned comp = 0;
  for (int k = group_fetch(g, S.counts + CURSOR_B); k < n; k = group_fetch(g, S.counts + CURSOR_B)) {
    const long long item = S.qB[k];
    if (!LF_IN_BOUNDS(item, B.n_items, status, "continuation ray item")) continue;
    const ShadeJob& J = B.jobs[job_of_item(B, item)];
    const long long loc = item - J.item0;
    float3 xslo;
    const float3 xs = pix_origin(J, pixel_of(loc, J.spp), P.ray_offset, xslo);
    const float3 wi = ld3(S.wi, item);
    Surface s2;
    coop_composite<WF_CONTINUE_RAY>(g, J.insts, J.n_inst, xs, xslo, wi, P, st, status, cnt, s2, comp);
    if (g.c == 0) {
      S.T2[item] = s2.T;
      if (s2.hits > 0) {
        float3 lo;
        st3(S.xs2, item, offset_origin(s2.x, s2.x_lo, s2.n, P.ray_offset, lo));
        st3(S.xs2lo, item, lo);
        st3(rec_n2(S), item, s2.n);
        st3(rec_a2(S), item, s2.a);
        rec_m2(S)[item] = s2.m;
        rec_r2(S)[item] = s2.r;
      }
    }
  }
  if (Cnt::on && counters && g.c == 0) {  // slot 2: continuation rays
    atomicAdd(counters + 8, (unsigned long long)cnt.nodes);
    atomicAdd(counters + 9, (unsigned long long)cnt.tests);
    atomicAdd(counters + 10, (unsigned long long)comp);
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(counters + 11, (unsigned long long)n);
  }
}

// ---------------------------------------------------------------- secondary NEE sampling
// One thread per continuation ray that found a surface: the two environment
// NEE samples at the secondary record (factor f2 cos (1 - T2) / 2 / p_env),
// appended to queue C.  Kept out of the warp-per-ray continuation kernel,
// where two lanes would run the CDF searches while thirty wait.
__global__ void __launch_bounds__(WB) k_wf_secondary(ShadeBatch B, DevParams P, SampleBuf S) {
  const int n = S.counts[1];
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int k = base + threadIdx.x;
    long long item = 0;
    bool push0 = false, push1 = false;
    if (k < n) {
      item = S.qB[k];
      const float T2 = S.T2[item];
      if (T2 < 1.0f) {
        const ShadeJob& J = B.jobs[job_of_item(B, item)];
        const long long loc = item - J.item0;
        const int p = pixel_of(loc, J.spp), s = sample_of(loc, J.spp);
        const float3 n2 = ld3(rec_n2(S), item), a2 = ld3(rec_a2(S), item);
        const float m2 = rec_m2(S)[item], r2 = rec_r2(S)[item];
        const float3 wo2 = -ld3(S.wi, item);
        const float co2 = dot3(n2, wo2);
        float u[9];
        sample_uniforms((uint32_t)p, (uint32_t)s, J.k0, J.k1, P.sampler, u);
        const float uq[4] = {u[5], u[6], u[7], u[8]};
#pragma unroll
        for (int qq = 0; qq < 2; ++qq) {
          float3 wq;
          float pq;
          env_sample(J.env, uq[2 * qq], uq[2 * qq + 1], wq, pq);
          const float cq = dot3(n2, wq);
          const bool ok = cq > 0.0f && co2 > 0.0f && pq > 0.0f;
          float3 fk = f3(0.f, 0.f, 0.f);
          if (ok) fk = brdf_eval(n2, wo2, wq, a2, m2, r2, P.brdf_mode) * (cq * (1.0f - T2) * 0.5f / pq);
          if (qq == 0) { st3(S.wq0, item, wq); st3(S.fk0, item, fk); push0 = ok; }
          else { st3(S.wq1, item, wq); st3(S.fk1, item, fk); push1 = ok; }
        }
      }
    }
    queue_push(S.qC, S.counts + 2, (int)(item * 2), push0);
    queue_push(S.qC, S.counts + 2, (int)(item * 2 + 1), push1);
  }
}

// ---------------------------------------------------------------- combine
struct SampleTerms {
  float3 E_e, E_i, E_q0, E_q1;
};

// Value of one sample given the (live) primary record.
__device__ __forceinline__ float3 sample_value(const SampleBuf& S, long long i, const PixRec& q, const EnvDev& env,
                                               const DevParams& P, SampleTerms& Et) {
  const float3 wo = -q.d;
  float3 c = f3(0.f, 0.f, 0.f);
  const float ek = S.ek[i];
  if (ek > 0.0f) {
    const float3 we = ld3(S.we, i);
    Et.E_e = env_lookup(env, we);
    const float3 f = brdf_eval(q.n, wo, we, q.a, q.m, q.r, P.brdf_mode);
    c = mul3(f, Et.E_e) * (dot3(q.n, we) * S.Ve[i] * ek);
  }
  const float bc = S.bc[i];
  if (bc > 0.0f) {
    const float3 wi = ld3(S.wi, i);
    const float T2 = S.T2[i];
    float3 inc = f3(0.f, 0.f, 0.f);
    if (P.sampling_mode != 2) {
      Et.E_i = env_lookup(env, wi);
      inc = Et.E_i * (S.wb[i] * T2);
    }
    const float3 fk0 = ld3(S.fk0, i), fk1 = ld3(S.fk1, i);
    if (fk0.x != 0.f || fk0.y != 0.f || fk0.z != 0.f) {
      Et.E_q0 = env_lookup(env, ld3(S.wq0, i));
      add3(inc, mul3(fk0, Et.E_q0) * S.Vq0[i]);
    }
    if (fk1.x != 0.f || fk1.y != 0.f || fk1.z != 0.f) {
      Et.E_q1 = env_lookup(env, ld3(S.wq1, i));
      add3(inc, mul3(fk1, Et.E_q1) * S.Vq1[i]);
    }
    const float3 f = brdf_eval(q.n, wo, wi, q.a, q.m, q.r, P.brdf_mode);
    add3(c, mul3(f * (dot3(q.n, wi) * bc), inc));
  }
  return c;
}

// The combine and its adjoint run CG lanes per pixel: lane l of a pixel's
// group takes samples l, l + CG, ..., so each load of a per-sample plane
// reads CG consecutive floats (a full 32-byte sector) instead of one float
// per pixel at a stride of spp; the group then sums over shuffles in a fixed
// tree order.  Every lane of a warp reaches the shuffles (no early return).
constexpr int CG = 8;

template <class T>
__device__ __forceinline__ T group_sum(T v);
template <>
__device__ __forceinline__ float group_sum(float v) {
#pragma unroll
  for (int off = CG / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, CG);
  return v;
}
template <>
__device__ __forceinline__ float3 group_sum(float3 v) {
  return f3(group_sum(v.x), group_sum(v.y), group_sum(v.z));
}

__global__ void __launch_bounds__(WB) k_wf_combine(ShadeBatch B, DevParams P, SampleBuf S) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int gp = t / CG, l = t % CG;
  const bool live = gp < B.n_pix_total;
  const ShadeJob& J = B.jobs[live ? job_of_pixel(B, gp) : 0];
  const int p = gp - J.pix0;
  float3 sum = f3(0.f, 0.f, 0.f);
  PixRec q{};
  if (live) {
    q = pix_record(J, p);
    if (q.hits > 0 && dot3(q.n, -q.d) > 0.0f) {
      const long long i0 = J.item0 + (long long)p * J.spp;
      SampleTerms Et;
      for (int s = l; s < J.spp; s += CG) add3(sum, sample_value(S, i0 + s, q, J.env, P, Et));
    }
  }
  sum = group_sum(sum);
  if (!live || l != 0) return;
  const float3 L = env_lookup(J.env, q.d) * q.T + sum * ((1.0f - q.T) / (float)J.spp);
  J.rgb[3 * p + 0] = L.x;
  J.rgb[3 * p + 1] = L.y;
  J.rgb[3 * p + 2] = L.z;
}

// d_env += v at the four bilinear texels of direction w, warp-aggregated:
// the lanes that reach the same texel together (matched on its index) sum
// their contributions over shuffles and one of them adds the sum, so a
// texel that many lanes sample (the sun of an importance-sampled map) takes
// one atomic per warp instead of one per lane.
__device__ __forceinline__ void env_scatter(const EnvDev& e, float* __restrict__ d_env, float3 w, float3 v) {
  if (!d_env) return;
  const Bilin b = env_bilinear(e, w);
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int idx = b.w[k] != 0.0f ? b.idx[k] : -1;
    const unsigned peers = __match_any_sync(__activemask(), idx);
    if (idx < 0) continue;
    float3 c = v * b.w[k];
    if (peers != (1u << lane)) {
      float3 acc = f3(0.f, 0.f, 0.f);
      for (unsigned m = peers; m; m &= m - 1u) {  // the same order in every lane of the group
        const int src = __ffs(m) - 1;
        acc.x += __shfl_sync(peers, c.x, src);
        acc.y += __shfl_sync(peers, c.y, src);
        acc.z += __shfl_sync(peers, c.z, src);
      }
      c = acc;
    }
    if (lane == __ffs(peers) - 1) {
      float* t = d_env + 3 * idx;
      atomicAdd(t + 0, c.x);
      atomicAdd(t + 1, c.y);
      atomicAdd(t + 2, c.z);
    }
  }
}

// Adjoint of k_wf_combine with the sample data fixed: gradients of g . L with
// respect to the primary record (normal, base colour, metallic, roughness,
// T) into `sg` (9 planes) and to the environment texels into d_env.
__global__ void __launch_bounds__(WB) k_wf_combine_adjoint(ShadeBatch B, DevParams P, SampleBuf S,
                                                           const float* __restrict__ dL_drgb,
                                                           float* __restrict__ sg, float* __restrict__ d_env) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int gp = t / CG, l = t % CG;
  const bool live = gp < B.n_pix_total;
  const ShadeJob& J = B.jobs[live ? job_of_pixel(B, gp) : 0];
  const int p = gp - J.pix0;
  const size_t NP = (size_t)J.n_pix;
  PixRec q{};
  float3 g = f3(0.f, 0.f, 0.f);
  if (live) {
    q = pix_record(J, p);
    g = f3(__ldg(dL_drgb + 3 * p), __ldg(dL_drgb + 3 * p + 1), __ldg(dL_drgb + 3 * p + 2));
  }
  const float3 wo = -q.d;
  float3 sum = f3(0.f, 0.f, 0.f), gn = sum, ga = sum;
  float gm = 0.f, gr = 0.f;
  if (live && q.hits > 0 && dot3(q.n, wo) > 0.0f) {
    const float3 gc = g * ((1.0f - q.T) / (float)J.spp);
    const long long i0 = J.item0 + (long long)p * J.spp;
    for (int s = l; s < J.spp; s += CG) {
      const long long i = i0 + s;
      const float ek = S.ek[i];
      if (ek > 0.0f) {
        const float3 we = ld3(S.we, i);
        const float3 E = env_lookup(J.env, we);
        const float3 f = brdf_eval(q.n, wo, we, q.a, q.m, q.r, P.brdf_mode);
        const float ce = dot3(q.n, we), kk = S.Ve[i] * ek;
        add3(sum, mul3(f, E) * (ce * kk));
        brdf_adjoint(q.n, wo, we, q.a, q.m, q.r, P.brdf_mode, mul3(gc, E) * (ce * kk), gn, ga, gm, gr);
        add3(gn, we * (dot3(gc, mul3(f, E)) * kk));
        env_scatter(J.env, d_env, we, mul3(gc, f) * (ce * kk));
      }
      const float bc = S.bc[i];
      if (bc > 0.0f) {
        const float3 wi = ld3(S.wi, i);
        const float T2 = S.T2[i], wbT = S.wb[i] * T2;
        float3 inc = f3(0.f, 0.f, 0.f);
        if (P.sampling_mode != 2) inc = env_lookup(J.env, wi) * wbT;
        const float3 fk0 = ld3(S.fk0, i), fk1 = ld3(S.fk1, i);
        const bool q0 = fk0.x != 0.f || fk0.y != 0.f || fk0.z != 0.f;
        const bool q1 = fk1.x != 0.f || fk1.y != 0.f || fk1.z != 0.f;
        const float3 wq0 = ld3(S.wq0, i), wq1 = ld3(S.wq1, i);
        const float V0 = q0 ? S.Vq0[i] : 0.f, V1 = q1 ? S.Vq1[i] : 0.f;
        if (q0) add3(inc, mul3(fk0, env_lookup(J.env, wq0)) * V0);
        if (q1) add3(inc, mul3(fk1, env_lookup(J.env, wq1)) * V1);
        const float ci = dot3(q.n, wi);
        const float3 f = brdf_eval(q.n, wo, wi, q.a, q.m, q.r, P.brdf_mode);
        const float3 beta = f * (ci * bc);
        add3(sum, mul3(beta, inc));
        const float3 gbeta = mul3(gc, inc);
        brdf_adjoint(q.n, wo, wi, q.a, q.m, q.r, P.brdf_mode, gbeta * (ci * bc), gn, ga, gm, gr);
        add3(gn, wi * (dot3(gbeta, f) * bc));
        const float3 ginc = mul3(gc, beta);
        if (P.sampling_mode != 2) env_scatter(J.env, d_env, wi, ginc * wbT);
        if (q0) env_scatter(J.env, d_env, wq0, mul3(ginc, fk0) * V0);
        if (q1) env_scatter(J.env, d_env, wq1, mul3(ginc, fk1) * V1);
      }
    }
  }
  sum = group_sum(sum);
  gn = group_sum(gn);
  ga = group_sum(ga);
  gm = group_sum(gm);
  gr = group_sum(gr);
  if (!live || l != 0) return;
  const float3 Ed = env_lookup(J.env, q.d);
  const float inv = 1.0f / (float)J.spp;
  const float gT = g.x * (Ed.x - sum.x * inv) + g.y * (Ed.y - sum.y * inv) + g.z * (Ed.z - sum.z * inv);
  env_scatter(J.env, d_env, q.d, g * q.T);
  sg[0 * NP + p] = gn.x; sg[1 * NP + p] = gn.y; sg[2 * NP + p] = gn.z;
  sg[3 * NP + p] = ga.x; sg[4 * NP + p] = ga.y; sg[5 * NP + p] = ga.z;
  sg[6 * NP + p] = gm;
  sg[7 * NP + p] = gr;
  sg[8 * NP + p] = gT;
}

// Per-sample terms c_s of the combine (one thread per work item), for
// inspection: out[3 i + c] for item i; zero where the pixel has no surface
// facing the camera.
__global__ void __launch_bounds__(WB) k_wf_terms(ShadeBatch B, DevParams P, SampleBuf S, float* __restrict__ out) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < B.n_items;
       i += (long long)gridDim.x * blockDim.x) {
    const ShadeJob& J = B.jobs[job_of_item(B, i)];
    const int p = pixel_of(i - J.item0, J.spp);
    const PixRec q = pix_record(J, p);
    float3 c = f3(0.f, 0.f, 0.f);
    if (q.hits > 0 && dot3(q.n, -q.d) > 0.0f) {
      SampleTerms Et;
      c = sample_value(S, i, q, J.env, P, Et);
    }
    out[3 * i + 0] = c.x;
    out[3 * i + 1] = c.y;
    out[3 * i + 2] = c.z;
  }
}

__global__ void k_wf_count(const int* counts, unsigned long long* ray_count) {
  if (threadIdx.x == 0 && ray_count)
    atomicAdd(ray_count, (unsigned long long)counts[0] + (unsigned long long)counts[1] + (unsigned long long)counts[2]);
}

// ---------------------------------------------------------------- host side
size_t sample_buf_bytes(long long n_items) {
  const size_t ns = (size_t)n_items;
  return sizeof(float) * SAMPLE_PLANES * ns + sizeof(int) * 4 * ns + 256;
}

SampleBuf sample_buf(void* base, long long n_items) {
  SampleBuf S;
  float* f = static_cast<float*>(base);
  const size_t ns = (size_t)n_items;
  auto take = [&](int k) { float* r = f; f += (size_t)k * ns; return r; };
  float* p;
  p = take(3); S.we[0] = p; S.we[1] = p + ns; S.we[2] = p + 2 * ns;
  S.ek = take(1);
  S.Ve = take(1);
  p = take(3); S.wi[0] = p; S.wi[1] = p + ns; S.wi[2] = p + 2 * ns;
  S.bc = take(1);
  S.wb = take(1);
  S.T2 = take(1);
  p = take(3); S.xs2[0] = p; S.xs2[1] = p + ns; S.xs2[2] = p + 2 * ns;
  p = take(3); S.xs2lo[0] = p; S.xs2lo[1] = p + ns; S.xs2lo[2] = p + 2 * ns;
  p = take(3); S.wq0[0] = p; S.wq0[1] = p + ns; S.wq0[2] = p + 2 * ns;
  p = take(3); S.wq1[0] = p; S.wq1[1] = p + ns; S.wq1[2] = p + 2 * ns;
  p = take(3); S.fk0[0] = p; S.fk0[1] = p + ns; S.fk0[2] = p + 2 * ns;
  p = take(3); S.fk1[0] = p; S.fk1[1] = p + ns; S.fk1[2] = p + 2 * ns;
  S.Vq0 = take(1);
  S.Vq1 = take(1);
  int* q = reinterpret_cast<int*>(f);
  S.qA = q;
  S.qB = q + ns;
  S.qC = q + 2 * ns;
  S.counts = q + 4 * ns;
  return S;
}

static int wf_grid(long long n, int sms) {
  const long long blocks = (n + WB - 1) / WB;
  return (int)std::max<long long>(1, std::min<long long>(blocks, (long long)sms * 16));
}

// Persistent grid of a trace kernel: the blocks that fit on the GPU at once,
// no more than the work needs.
template <class K>
static int resident_grid(K kernel, long long n, int sms, int smem, int rays_per_block) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, WB, smem) != cudaSuccess || per_sm < 1)
    per_sm = 1;
  const long long blocks = (n + rays_per_block - 1) / rays_per_block;
  return (int)std::max<long long>(1, std::min<long long>(blocks, (long long)sms * per_sm));
}

cudaError_t launch_shade_wavefront(const ShadeBatch& B, const DevParams& P, const SampleBuf& S, int* status,
                                   unsigned long long* ray_count, unsigned long long* counters, int sms,
                                   cudaStream_t st, cudaEvent_t* ev) {
  if (B.n_items <= 0) return cudaSuccess;
  cudaError_t e = cudaMemsetAsync(S.counts, 0, N_COUNTS * sizeof(int), st);
  if (e != cudaSuccess) return e;
  // ev (nullable): 5 events bracketing gen | NEE shadow | continuation | secondary shadow
  auto mark = [&](int i) { if (ev) cudaEventRecord(ev[i], st); };
  mark(0);
  k_wf_gen<<<wf_grid(B.n_items, sms), WB, 0, st>>>(B, P, S);
  mark(1);
  // queue lengths are known only on the device: the trace kernels size
  // their loops from the counters (grids cover the worst case).
  // kernels compiled with counting only when the caller asked for counts
  auto shadow = counters ? k_wf_shadow<Counters> : k_wf_shadow<NoCounters>;
  auto cont = counters ? k_wf_continue<Counters> : k_wf_continue<NoCounters>;
  shadow<<<resident_grid(shadow, B.n_items, sms, CSTACK_SMEM, WGROUPS), WB, CSTACK_SMEM, st>>>(B, P, S, 0, status,
                                                                                              counters);
  mark(2);
  cont<<<resident_grid(cont, B.n_items, sms, CSTACK_SMEM, WGROUPS), WB, CSTACK_SMEM, st>>>(B, P, S, status, counters);
  k_wf_secondary<<<wf_grid(B.n_items, sms), WB, 0, st>>>(B, P, S);
  mark(3);
  shadow<<<resident_grid(shadow, 2 * B.n_items, sms, CSTACK_SMEM, WGROUPS), WB, CSTACK_SMEM, st>>>(B, P, S, 1,
                                                                                                  status, counters);
  mark(4);
  k_wf_count<<<1, 32, 0, st>>>(S.counts, ray_count);
  return cudaGetLastError();
}

cudaError_t launch_shade_combine(const ShadeBatch& B, const DevParams& P, const SampleBuf& S, cudaStream_t st) {
  const long long threads = (long long)B.n_pix_total * CG;
  if (B.n_pix_total > 0) k_wf_combine<<<(unsigned)((threads + WB - 1) / WB), WB, 0, st>>>(B, P, S);
  return cudaGetLastError();
}

cudaError_t launch_shade_terms(const ShadeBatch& B, const DevParams& P, const SampleBuf& S, float* out, int sms,
                               cudaStream_t st) {
  if (B.n_items > 0) k_wf_terms<<<wf_grid(B.n_items, sms), WB, 0, st>>>(B, P, S, out);
  return cudaGetLastError();
}

cudaError_t launch_shade_combine_adjoint(const ShadeBatch& B, const DevParams& P, const SampleBuf& S,
                                         const float* dL_drgb, float* sg, float* d_env, cudaStream_t st) {
  if (B.n_pix_total > 0)
    k_wf_combine_adjoint<<<(unsigned)(((long long)B.n_pix_total * CG + WB - 1) / WB), WB, 0, st>>>(B, P, S, dL_drgb,
                                                                                                     sg, d_env);
  return cudaGetLastError();
}

}  // namespace lf
