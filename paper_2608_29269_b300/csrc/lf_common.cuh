// Device-side building blocks of the surfel ray tracer (sm_103a).
//
// Record layouts (library-owned, in BVH leaf order per object, each quad in
// its own plane of n quads per object):
//   geo[0*n+l] = (mu.xyz, n^.x)        n^ = unit normal tu x tv, normalised in FP64
//   geo[1*n+l] = (n^.yz, a.xy)         then rounded, so that exactly coplanar
//   geo[2*n+l] = (a.z, b.xyz)          axis-aligned surfels get exactly equal t;
//   geo[3*n+l] = (opacity, id bits, roughness, 0)   a = tu/s_u, b = tv/s_v
//   mat[l]     = (albedo.rgb, metallic)
//   BVH2 node (64 B, child boxes stored in the parent):
//     n0 = (L.lo.xyz, L.hi.x)  n1 = (L.hi.yz, R.lo.xy)  n2 = (R.lo.z, R.hi.xyz)
//     n3 = (left code, right code, -, -) ; code >= 0 internal node, code < 0 leaf ~code
//   Wide node (WIDE child slots; lane c of a ray's warp reads slot c):
//     LF_WIDE_FP16 = 1: a header quad (centre.xyz of the node's box, 0), then
//       one quad per slot: (lo.xy, lo.z hi.x, hi.yz) as FP16 pairs relative to
//       the centre, rounded outward, and the slot word; slot word >= 0 wide
//       node, WSLOT_EMPTY empty, else a leaf: bit 31 | (count - 1) << 24 |
//       first surfel (24 bits)
//     LF_WIDE_FP16 = 0: WIDE quads (lo.xyz, code) then WIDE quads (hi.xyz,
//       count); code >= 0 wide node, code < 0 leaf of `count` consecutive
//       surfels from ~code, INT_MIN empty
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "lightfuse.h"

namespace lf {

// Children per wide BVH node = lanes per ray in the cooperative traversal =
// hits per k-buffer round.
constexpr int WIDE = LF_KBUF;
// Surfels at most in one leaf slot of the wide BVH.
#ifndef LF_WIDE_LEAF
#define LF_WIDE_LEAF LF_KBUF
#endif
constexpr int WLEAF = LF_WIDE_LEAF;
static_assert(WLEAF >= 1 && WLEAF <= WIDE, "a leaf is tested by at most WIDE lanes");
// Wide-node format: FP16 child boxes relative to the node centre (16 B per
// slot) or FP32 boxes (32 B per slot).
#ifndef LF_WIDE_FP16
#define LF_WIDE_FP16 0
#endif
#if LF_WIDE_FP16
constexpr int WNODE_Q = WIDE + 1;  // float4 quads per wide node
static_assert(WLEAF <= 32, "leaf counts take 5 bits of the slot word");
#else
constexpr int WNODE_Q = 2 * WIDE;
#endif
constexpr unsigned WSLOT_EMPTY = 0xffffffffu;
constexpr float PI_F = 3.14159265358979323846f;
constexpr float INV_PI_F = 0.318309886183790671538f;
constexpr float INV_2PI_F = 0.159154943091895335769f;
constexpr float BIG_F = 3.0e38f;

struct DevParams {
  float T_min, alpha_min, alpha_max, support_r2, eps_w, t_min, ray_offset, p_spec;
  int max_rounds, brdf_mode, sampling_mode, sampler;
};

// One TLAS entry: an object's BLAS in world space (Eq. 2 after its transform).
struct __align__(16) Inst {
  float lo[3];
  int root;  // child code of the binary BLAS root (>= 0 node, < 0 leaf ~code); INT_MIN: empty
  float hi[3];
  int n_leaves;
  const float4* nodes;   // binary BLAS
  const float4* geo;
  const float4* mat;
  int id_base;  // surfel id of the object's first surfel
  int n_wide;   // wide BLAS nodes of the object
  const float4* wnodes;  // wide BLAS (WIDE children per node)
  int wroot;             // wide root: >= 0 node, < 0 leaf ~first; INT_MIN: empty
  int wroot_count;       // surfels of a leaf root
};
static_assert(sizeof(Inst) == 80, "Inst is 80 bytes");

struct EnvDev {
  const float* rgb;  // H x W x 3
  const float* pmf_row;
  const float* cdf_row;
  const float* pmf_col;
  const float* cdf_col;
  const float* cdf_row_lo;  // FP64 CDF minus its FP32 rounding
  const float* cdf_col_lo;
  int H, W;
};

// Pinhole camera with its basis in FP64 (host-computed).  The ray direction
// of each pixel is evaluated in FP64 and rounded once to FP32, so every pixel
// traces a reproducible FP32 ray.
struct CamDev {
  float3 eye;
  double f[3], r[3], u[3];
  double th, aspect;  // tan(fovy/2), width/height
  int W, H;
};

// ------------------------------------------------------------------ status
__device__ __forceinline__ void report(int* status, int code) {
  if (status) atomicCAS(status, 0, code);
}

// Bounds checks of the LF_CHECKED build (off by default; then every check is
// the constant true and the kernels are the unchecked ones).  A failed check
// reports LF_ERR_BOUNDS through the status word, prints the index and its
// limit, and the caller skips the access -- no trap, so the context stays
// usable and lf_sync returns the error.
#ifndef LF_CHECKED
#define LF_CHECKED 0
#endif
#if LF_CHECKED
}  // namespace lf
#include <cstdio>
namespace lf {
static __device__ __noinline__ bool lf_bounds_fail(long long idx, long long lim, int* status, const char* what) {
  report(status, LF_ERR_BOUNDS);
  printf("lightfuse bounds check failed: %s index %lld outside [0, %lld)\n", what, idx, lim);
  return false;
}
#define LF_IN_BOUNDS(idx, lim, status, what)                                                     \
  ((long long)(idx) >= 0 && (long long)(idx) < (long long)(lim)                                \
       ? true                                                                                    \
       : ::lf::lf_bounds_fail((long long)(idx), (long long)(lim), (status), (what)))
#else
#define LF_IN_BOUNDS(idx, lim, status, what) true
#endif

// ------------------------------------------------------------------ vectors
__device__ __forceinline__ float3 f3(float x, float y, float z) { return make_float3(x, y, z); }
__device__ __forceinline__ float3 operator+(float3 a, float3 b) { return f3(a.x + b.x, a.y + b.y, a.z + b.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return f3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 operator-(float3 a) { return f3(-a.x, -a.y, -a.z); }
__device__ __forceinline__ float3 operator*(float3 a, float s) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 operator*(float s, float3 a) { return f3(a.x * s, a.y * s, a.z * s); }
__device__ __forceinline__ float3 mul3(float3 a, float3 b) { return f3(a.x * b.x, a.y * b.y, a.z * b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
  return f3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float3 normalize3(float3 a) { return a * (1.0f / sqrtf(dot3(a, a))); }
__device__ __forceinline__ void add3(float3& a, float3 b) { a.x += b.x; a.y += b.y; a.z += b.z; }

// Correctly rounded, contraction-free forms used by the intersection so that
// every kernel (forward, shading, adjoint) computes bit-identical hits.
__device__ __forceinline__ float dot_rn(float3 a, float3 b) {
  return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ float3 cross_rn(float3 a, float3 b) {
  return f3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
            __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}

// ------------------------------------------------------------------ Philox4x32-10
// Salmon, Moraes, Dror, Shaw (SC'11): ten rounds, two 32x32->64 products per
// round, Weyl key schedule.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int i = 0; i < 10; ++i) {
    uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
    uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return c;
}

// The nine uniforms of (pixel, sample): NEE (0,1), lobe 2, BSDF (3,4),
// secondary NEE #1 (5,6), #2 (7,8).  Counter (pixel, sample, group, 0).
// Sobol points in 9 dimensions (Joe and Kuo 2008 direction numbers: the
// first dimension is van der Corput, the next eight use the primitive
// polynomials of degree s with coefficients a and initial numbers m), as
// 32-bit fractions: point i is the XOR of the direction numbers of the set
// bits of i.  Tabulated at compile time from the recurrence
//   v_k = v_{k-s} ^ (v_{k-s} >> s) ^ XOR_{j=1..s-1} a_j v_{k-j},  v_k = m_k 2^(31-k) for k < s.
struct SobolDirs {
  uint32_t v[9][32];
};
constexpr SobolDirs make_sobol_dirs() {
  SobolDirs t{};
  const int S[9] = {0, 1, 2, 3, 3, 4, 4, 5, 5};
  const int A[9] = {0, 0, 1, 1, 2, 1, 4, 2, 4};
  const uint32_t M[9][5] = {{1, 0, 0, 0, 0}, {1, 0, 0, 0, 0}, {1, 3, 0, 0, 0}, {1, 3, 1, 0, 0}, {1, 1, 1, 0, 0},
                            {1, 1, 3, 3, 0}, {1, 3, 5, 13, 0}, {1, 1, 5, 5, 17}, {1, 1, 5, 5, 5}};
  for (int k = 0; k < 32; ++k) t.v[0][k] = 1u << (31 - k);
  for (int d = 1; d < 9; ++d) {
    const int s = S[d];
    for (int k = 0; k < 32; ++k) {
      if (k < s) {
        t.v[d][k] = M[d][k] << (31 - k);
      } else {
        uint32_t x = t.v[d][k - s] ^ (t.v[d][k - s] >> s);
        for (int j = 1; j < s; ++j)
          if ((A[d] >> (s - 1 - j)) & 1) x ^= t.v[d][k - j];
        t.v[d][k] = x;
      }
    }
  }
  return t;
}
__constant__ const SobolDirs kSobol = make_sobol_dirs();

__device__ __forceinline__ uint32_t sobol32(uint32_t index, int dim) {
  uint32_t x = 0u;
  for (int k = 0; index != 0u; ++k, index >>= 1)
    if (index & 1u) x ^= kSobol.v[dim][k];
  return x;
}

// The nine uniforms of one (pixel, sample): NEE (0,1), lobe 2, BSDF (3,4),
// secondary NEE #1 (5,6), secondary NEE #2 (7,8).
//  sampler 0: Philox4x32-10 of counter (pixel, sample, group, 0), groups 0-2.
//  sampler 1: Sobol point `sample` rotated per pixel (Cranley-Patterson):
//             u_d = ((sobol_d >> 8) + (r_d >> 8)) mod 2^24, r = Philox of
//             counter (pixel, 0xffffffff, group, 1), groups 0-2.
// Both in 24-bit fixed point, so the values are exact.
__device__ __forceinline__ void sample_uniforms(uint32_t pixel, uint32_t s, uint32_t k0, uint32_t k1, int sampler,
                                                float u[9]) {
  uint32_t w[12];
  const uint32_t ctr1 = sampler == 1 ? 0xffffffffu : s, ctr3 = sampler == 1 ? 1u : 0u;
#pragma unroll
  for (uint32_t g = 0; g < 3; ++g) {
    const uint4 r = philox4x32_10(make_uint4(pixel, ctr1, g, ctr3), k0, k1);
    w[4 * g] = r.x; w[4 * g + 1] = r.y; w[4 * g + 2] = r.z; w[4 * g + 3] = r.w;
  }
#pragma unroll
  for (int d = 0; d < 9; ++d) {
    uint32_t x = w[d] >> 8;
    if (sampler == 1) x = ((sobol32(s, d) >> 8) + x) & 0xffffffu;
    u[d] = (float)x * (1.0f / 16777216.0f);
  }
}

// ------------------------------------------------------------------ Eq. 6
constexpr int GEO = 4;  // float4 per packed surfel record

// Packed record: the first three quads are what the quick plane test reads
// (centre, normal, both scaled axes); the fourth (opacity, id, roughness) is
// read only for candidates that pass it.
struct Rec {
  float4 g0, g1, g2, g3;
};
__device__ __forceinline__ float3 rec_mu(const Rec& r) { return f3(r.g0.x, r.g0.y, r.g0.z); }
__device__ __forceinline__ float3 rec_n(const Rec& r) { return f3(r.g0.w, r.g1.x, r.g1.y); }
__device__ __forceinline__ float3 rec_a(const Rec& r) { return f3(r.g1.z, r.g1.w, r.g2.x); }
__device__ __forceinline__ float3 rec_b(const Rec& r) { return f3(r.g2.y, r.g2.z, r.g2.w); }
__device__ __forceinline__ float rec_opacity(const Rec& r) { return r.g3.x; }
__device__ __forceinline__ int rec_id(const Rec& r) { return __float_as_int(r.g3.y); }
__device__ __forceinline__ float rec_rough(const Rec& r) { return r.g3.z; }
// An object's records are stored as GEO planes of n quads (quad k of record l
// at geo[k * n + l]), so the lanes of a warp reading consecutive records
// read consecutive 16-byte quads.
__device__ __forceinline__ void load_rec3(const float4* geo, int n, int l, Rec& r) {
  r.g0 = __ldg(geo + l);
  r.g1 = __ldg(geo + n + l);
  r.g2 = __ldg(geo + 2 * n + l);
}
__device__ __forceinline__ void load_rec_tail(const float4* geo, int n, int l, Rec& r) {
  r.g3 = __ldg(geo + 3 * n + l);
}
__device__ __forceinline__ Rec load_rec(const float4* geo, int n, int l) {
  Rec r;
  load_rec3(geo, n, l, r);
  load_rec_tail(geo, n, l, r);
  return r;
}

// Error-free transformations: TwoSum (Knuth) and TwoProd via FMA.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
// Double-float values hi + lo (|lo| <= ulp(hi) / 2) and the operations the
// precise composite needs, after Dekker (1971): a sum by TwoSum, a product by
// TwoProd, a quotient and a square root by one correction step of the FP32
// result with its exactly formed residual; relative error ~1e-14.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_renorm(float s, float e) {  // |s| >= |e|
  DF r;
  r.hi = __fadd_rn(s, e);
  r.lo = __fsub_rn(e, __fsub_rn(r.hi, s));
  return r;
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  float s, e;
  two_sum(a.hi, b.hi, s, e);
  return df_renorm(s, __fadd_rn(e, __fadd_rn(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  float p, e;
  two_prod(a.hi, b.hi, p, e);
  return df_renorm(p, __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e)));
}
__device__ __forceinline__ DF df_div(DF a, DF b) {
  const float q = __fdiv_rn(a.hi, b.hi);
  float p, e;
  two_prod(q, b.hi, p, e);  // q b.hi exactly
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), __fsub_rn(a.lo, __fmul_rn(q, b.lo)));
  return df_renorm(q, __fdiv_rn(r, b.hi));
}
__device__ __forceinline__ DF df_sqrt(DF a) {  // a > 0
  const float s = __fsqrt_rn(a.hi);
  float p, e;
  two_prod(s, s, p, e);
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
  return df_renorm(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}

// (ah + al) . b as a renormalised double-float (compensated dot product,
// Ogita, Rump and Oishi 2005).
__device__ __forceinline__ void dot2(float3 ah, float3 al, float3 b, float& hi, float& lo) {
  float s, c, p, e, s2, e2;
  two_prod(ah.x, b.x, s, c);
  two_prod(ah.y, b.y, p, e);
  two_sum(s, p, s2, e2);
  s = s2;
  c = __fadd_rn(c, __fadd_rn(e, e2));
  two_prod(ah.z, b.z, p, e);
  two_sum(s, p, s2, e2);
  s = s2;
  c = __fadd_rn(c, __fadd_rn(e, e2));
  c = __fmaf_rn(al.x, b.x, c);
  c = __fmaf_rn(al.y, b.y, c);
  c = __fmaf_rn(al.z, b.z, c);
  hi = __fadd_rn(s, c);
  lo = __fsub_rn(c, __fsub_rn(hi, s));
}

// Plane hit of a packed surfel record (Eq. 6), in two stages.
//
// hit_quick: FP32 depth and u^2 + v^2; rejects candidates behind the origin
// or clearly outside the support (conservative margins).
//
// hit_precise: the ray depth as a double-float t + tl (error ~1e-14
// relative for the FP32 inputs: TwoSum / TwoProd error-free transforms and a
// compensated dot product), the offset q = o + t d - mu to ~1e-9 absolute,
// then u, v, the support and opacity tests and alpha~.  The depth order of
// near-coincident surfels and the support decision therefore do not depend
// on FP32 rounding.
__device__ __forceinline__ bool hit_quick(const Rec& r, const float3 o, const float3 d, const DevParams& P,
                                          float& t32) {
  const float3 a = rec_a(r), b = rec_b(r), nh = rec_n(r);
  const float3 p = f3(r.g0.x - o.x, r.g0.y - o.y, r.g0.z - o.z);
  t32 = __fdividef(dot3(p, nh), dot3(d, nh));
  if (!(t32 > 0.5f * P.t_min) || !(t32 < BIG_F)) return false;
  const float3 q = f3(fmaf(t32, d.x, -p.x), fmaf(t32, d.y, -p.y), fmaf(t32, d.z, -p.z));
  const float u = dot3(q, a), v = dot3(q, b);
  return fmaf(u, u, v * v) <= 1.001f * P.support_r2;
}

__device__ __forceinline__ bool hit_precise(const Rec& r, const float3 o, const float3 olo, const float3 d,
                                            const DevParams& P, float& t, float& tl, float& alpha) {
  const float3 a = rec_a(r), b = rec_b(r), nh = rec_n(r);
  float3 ph, pl;
  two_sum(r.g0.x, -o.x, ph.x, pl.x);
  two_sum(r.g0.y, -o.y, ph.y, pl.y);
  two_sum(r.g0.z, -o.z, ph.z, pl.z);
  pl = f3(__fsub_rn(pl.x, olo.x), __fsub_rn(pl.y, olo.y), __fsub_rn(pl.z, olo.z));
  float nhi, nlo, dhi, dlo;
  dot2(ph, pl, nh, nhi, nlo);
  dot2(d, f3(0.f, 0.f, 0.f), nh, dhi, dlo);
  // t0 need not be correctly rounded: the residual below is formed exactly
  // (FMA) from whatever t0 is, and t1 = res / d is a correction ~2^-23 t,
  // whose own relative error of 2 ulp is far below the double-float's.
  const float t0 = __fdividef(nhi, dhi);
  const float res = __fadd_rn(__fmaf_rn(-t0, dhi, nhi), __fmaf_rn(-t0, dlo, nlo));
  const float t1 = __fdividef(res, dhi);
  t = __fadd_rn(t0, t1);
  tl = __fsub_rn(t1, __fsub_rn(t, t0));
  if (!(t > P.t_min) || !(t < BIG_F)) return false;
  const float3 q = f3(__fadd_rn(__fmaf_rn(t, d.x, -ph.x), __fmaf_rn(tl, d.x, -pl.x)),
                      __fadd_rn(__fmaf_rn(t, d.y, -ph.y), __fmaf_rn(tl, d.y, -pl.y)),
                      __fadd_rn(__fmaf_rn(t, d.z, -ph.z), __fmaf_rn(tl, d.z, -pl.z)));
  const float u = dot_rn(q, a), v = dot_rn(q, b);
  const float r2 = __fmaf_rn(u, u, __fmul_rn(v, v));
  if (!(r2 <= P.support_r2)) return false;
  alpha = fminf(P.alpha_max, __fmul_rn(rec_opacity(r), expf(__fmul_rn(-0.5f, r2))));
  return alpha >= P.alpha_min;
}

// Full test of record l: the quick test on its first three quads, then the
// fourth quad and the precise test for a candidate that passes.
__device__ __forceinline__ bool hit_surfel(const float4* geo, int n, int l, const float3 o, const float3 olo,
                                           const float3 d, const DevParams& P, Rec& r, float& t32, float& t,
                                           float& tl, float& alpha) {
  load_rec3(geo, n, l, r);
  if (!hit_quick(r, o, d, P, t32)) return false;
  load_rec_tail(geo, n, l, r);
  return hit_precise(r, o, olo, d, P, t, tl, alpha);
}

// 64-bit sort key of a hit: FP32 depth bits | low depth part quantised to
// 1/256 of an ulp | 24-bit surfel id.  Integer order = (depth, id) order;
// depths closer than 1/256 ulp (~2e-10 relative) fall back to the id.
__device__ __forceinline__ unsigned long long hit_key(float t, float tl, int id) {
  const unsigned tb = __float_as_uint(t);
  const float ulp = __uint_as_float(tb & 0x7f800000u) * 1.1920928955078125e-7f;
  const int q = min(255, max(0, __float2int_rn(tl / ulp * 256.0f) + 128));
  return ((unsigned long long)tb << 32) | ((unsigned long long)q << 24) | (unsigned long long)(id & 0xffffff);
}
__device__ __forceinline__ float key_t(unsigned long long k) { return __uint_as_float((unsigned)(k >> 32)); }
// The low part of the depth that hit_key kept (to 1/256 of an ulp of key_t).
__device__ __forceinline__ float key_tl(unsigned long long k) {
  const unsigned tb = (unsigned)(k >> 32);
  const float ulp = __uint_as_float(tb & 0x7f800000u) * 1.1920928955078125e-7f;
  return (float)((int)((k >> 24) & 0xffu) - 128) * (ulp * (1.0f / 256.0f));
}

// Normal of a packed record facing the ray (two-sided surfels).
__device__ __forceinline__ float3 record_normal(const Rec& r, const float3 d) {
  const float3 n = rec_n(r);
  return dot3(d, n) < 0.0f ? n : -n;
}

// ------------------------------------------------------------------ environment
struct Bilin {
  int idx[4];
  float w[4];
};

__device__ __forceinline__ void dir_angles(float3 w, float& th, float& ph) {
  th = acosf(fminf(1.0f, fmaxf(-1.0f, w.y)));
  ph = atan2f(w.x, -w.z) + PI_F;
}

__device__ __forceinline__ Bilin env_bilinear(const EnvDev& e, float3 w) {
  float th, ph;
  dir_angles(w, th, ph);
  float u = ph * INV_2PI_F * (float)e.W - 0.5f, v = th * INV_PI_F * (float)e.H - 0.5f;
  float x0f = floorf(u), y0f = floorf(v);
  float fx = u - x0f, fy = v - y0f;
  int x0 = (int)x0f, y0 = (int)y0f;
  int x0m = ((x0 % e.W) + e.W) % e.W, x1m = (((x0 + 1) % e.W) + e.W) % e.W;
  int y0c = min(e.H - 1, max(0, y0)), y1c = min(e.H - 1, max(0, y0 + 1));
  Bilin b;
  b.idx[0] = y0c * e.W + x0m; b.w[0] = (1.0f - fx) * (1.0f - fy);
  b.idx[1] = y0c * e.W + x1m; b.w[1] = fx * (1.0f - fy);
  b.idx[2] = y1c * e.W + x0m; b.w[2] = (1.0f - fx) * fy;
  b.idx[3] = y1c * e.W + x1m; b.w[3] = fx * fy;
  return b;
}

__device__ __forceinline__ float3 env_lookup(const EnvDev& e, float3 w) {
  Bilin b = env_bilinear(e, w);
  float3 s = f3(0.f, 0.f, 0.f);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float* t = e.rgb + 3 * b.idx[k];
    s.x += b.w[k] * __ldg(t);
    s.y += b.w[k] * __ldg(t + 1);
    s.z += b.w[k] * __ldg(t + 2);
  }
  return s;
}

// First index i in [0, n) with f[i] > u (f non-decreasing, f[n-1] == 1 > u).
__device__ __forceinline__ int first_greater(const float* __restrict__ f, int n, float u) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (__ldg(f + mid) > u) hi = mid; else lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ float env_pdf(const EnvDev& e, float3 w) {
  float th, ph;
  dir_angles(w, th, ph);
  int r = min(e.H - 1, max(0, (int)floorf(th * INV_PI_F * (float)e.H)));
  int c = min(e.W - 1, max(0, (int)floorf(ph * INV_2PI_F * (float)e.W)));
  float st = fmaxf(sinf(th), 1e-12f);
  return __ldg(e.pmf_row + r) * __ldg(e.pmf_col + r * e.W + c) * ((float)e.H * (float)e.W) /
         (2.0f * PI_F * PI_F * st);
}

// Position of uniform u inside the texel [lo, hi) of a CDF given as
// double-float pairs (h, l): u - lo and hi - lo are formed from the pairs,
// so fr carries the FP64 table's accuracy, not its FP32 rounding (which is a
// sizeable fraction of a narrow texel).
__device__ __forceinline__ float in_texel(float u, float loh, float lol, float hih, float hil) {
  const float num = __fsub_rn(__fsub_rn(u, loh), lol);
  const float den = __fadd_rn(__fsub_rn(hih, loh), __fsub_rn(hil, lol));
  return fminf(fmaxf(num / den, 0.0f), 1.0f);
}

__device__ __forceinline__ void env_sample(const EnvDev& e, float u1, float u2, float3& w, float& pdf) {
  int r = first_greater(e.cdf_row, e.H, u1);
  float lo = r > 0 ? __ldg(e.cdf_row + r - 1) : 0.0f, hi = __ldg(e.cdf_row + r);
  float lol = r > 0 ? __ldg(e.cdf_row_lo + r - 1) : 0.0f, hil = __ldg(e.cdf_row_lo + r);
  float fr = in_texel(u1, lo, lol, hi, hil);
  const float* row = e.cdf_col + r * e.W;
  const float* rowl = e.cdf_col_lo + r * e.W;
  int c = first_greater(row, e.W, u2);
  float clo = c > 0 ? __ldg(row + c - 1) : 0.0f, chi = __ldg(row + c);
  float clol = c > 0 ? __ldg(rowl + c - 1) : 0.0f, chil = __ldg(rowl + c);
  float fc = in_texel(u2, clo, clol, chi, chil);
  // theta = pi (r + fr) / H, phi - pi = pi (2 (c + fc) / W - 1): sincospif
  // takes the angles in units of pi, so no FP32 multiple of pi is formed
  float st, ct, sp, cp;
  sincospif(((float)r + fr) / (float)e.H, &st, &ct);
  sincospif(2.0f * ((float)c + fc) / (float)e.W - 1.0f, &sp, &cp);
  w = f3(st * sp, ct, -st * cp);
  pdf = __ldg(e.pmf_row + r) * __ldg(e.pmf_col + r * e.W + c) * ((float)e.H * (float)e.W) /
        (2.0f * PI_F * PI_F * fmaxf(st, 1e-12f));
}

// ------------------------------------------------------------------ BRDF
// Metallic-roughness: k_d/pi + F D G / (4 cos_i cos_o); GGX D (Walter et al.
// 2007), separable Smith G, Schlick F; k_d = a (1-m), F0 = 0.04 (1-m) + a m,
// alpha_g = r^2.  brdf_mode 1: a / pi.
//
// GGX denominator (n.h)^2 (alpha_g^2 - 1) + 1 = |n x h|^2 + alpha_g^2 (n.h)^2
// for unit n and h: the right-hand form has no cancellation when h is close
// to n (a glossy lobe), where 1 - (n.h)^2 computed from n.h loses most of its
// digits in FP32.
__device__ __forceinline__ float ggx_den(float3 n, float3 h, float nh, float a2) {
  const float3 c = f3(n.y * h.z - n.z * h.y, n.z * h.x - n.x * h.z, n.x * h.y - n.y * h.x);
  return fmaf(a2 * nh, nh, dot3(c, c));
}
__device__ __forceinline__ float3 brdf_eval(float3 n, float3 wo, float3 wi, float3 a, float m, float r, int mode) {
  float ci = dot3(n, wi), co = dot3(n, wo);
  if (!(ci > 0.0f) || !(co > 0.0f)) return f3(0.f, 0.f, 0.f);
  if (mode == 1) return a * INV_PI_F;
  float one_m = 1.0f - m;
  float3 F0 = f3(0.04f * one_m + a.x * m, 0.04f * one_m + a.y * m, 0.04f * one_m + a.z * m);
  float ag = r * r, a2 = ag * ag;
  float3 h = normalize3(wi + wo);
  float nh = dot3(n, h), oh = dot3(wo, h);
  float den = ggx_den(n, h, nh, a2);
  float D = a2 / (PI_F * den * den);
  float Qi = 2.0f / (ci + sqrtf(a2 + (1.0f - a2) * ci * ci));
  float Qo = 2.0f / (co + sqrtf(a2 + (1.0f - a2) * co * co));
  float spec = 0.25f * D * Qi * Qo;
  float x = 1.0f - oh, x2 = x * x, fw = x2 * x2 * x;
  return f3(a.x * one_m * INV_PI_F + (F0.x + (1.0f - F0.x) * fw) * spec,
            a.y * one_m * INV_PI_F + (F0.y + (1.0f - F0.y) * fw) * spec,
            a.z * one_m * INV_PI_F + (F0.z + (1.0f - F0.z) * fw) * spec);
}

// Adjoint of brdf_eval for fixed directions: adds d(gf . f) to gn, ga, gm, gr.
__device__ __forceinline__ void brdf_adjoint(float3 n, float3 wo, float3 wi, float3 a, float m, float r, int mode,
                                             float3 gf, float3& gn, float3& ga, float& gm, float& gr) {
  float ci = dot3(n, wi), co = dot3(n, wo);
  if (!(ci > 0.0f) || !(co > 0.0f)) return;
  if (mode == 1) { add3(ga, gf * INV_PI_F); return; }
  float one_m = 1.0f - m;
  float3 F0 = f3(0.04f * one_m + a.x * m, 0.04f * one_m + a.y * m, 0.04f * one_m + a.z * m);
  float ag = r * r, a2 = ag * ag;
  float3 h = normalize3(wi + wo);
  float nh = dot3(n, h), oh = dot3(wo, h);
  float den = ggx_den(n, h, nh, a2);
  float D = a2 / (PI_F * den * den);
  float si = sqrtf(a2 + (1.0f - a2) * ci * ci), so = sqrtf(a2 + (1.0f - a2) * co * co);
  float Qi = 2.0f / (ci + si), Qo = 2.0f / (co + so);
  float spec = 0.25f * D * Qi * Qo;
  float x = 1.0f - oh, x2 = x * x, fw = x2 * x2 * x;
  float3 F = f3(F0.x + (1.0f - F0.x) * fw, F0.y + (1.0f - F0.y) * fw, F0.z + (1.0f - F0.z) * fw);
  // diffuse k_d / pi with k_d = a (1 - m)
  float3 gkd = gf * INV_PI_F;
  add3(ga, gkd * one_m);
  gm -= dot3(gkd, a);
  // F = F0 (1 - fw) + fw ; F0 = 0.04 (1 - m) + a m
  float3 gF0 = gf * (spec * (1.0f - fw));
  add3(ga, gF0 * m);
  gm += gF0.x * (a.x - 0.04f) + gF0.y * (a.y - 0.04f) + gF0.z * (a.z - 0.04f);
  float gspec = dot3(gf, F);
  // spec = D Qi Qo / 4
  float gD = gspec * 0.25f * Qi * Qo, gQi = gspec * 0.25f * D * Qo, gQo = gspec * 0.25f * D * Qi;
  // Q(c) = 2 / (c + s(c)), s = sqrt(a2 + (1 - a2) c^2)
  float dQi_dc = -0.5f * Qi * Qi * (1.0f + (1.0f - a2) * ci / si);
  float dQo_dc = -0.5f * Qo * Qo * (1.0f + (1.0f - a2) * co / so);
  float dQi_da2 = -0.5f * Qi * Qi * (1.0f - ci * ci) / (2.0f * si);
  float dQo_da2 = -0.5f * Qo * Qo * (1.0f - co * co) / (2.0f * so);
  // D = a2 / (pi den^2), den = nh^2 (a2 - 1) + 1
  float dD_dnh = -4.0f * a2 * nh * (a2 - 1.0f) / (PI_F * den * den * den);
  float dD_da2 = (den - 2.0f * a2 * nh * nh) / (PI_F * den * den * den);
  float ga2 = gD * dD_da2 + gQi * dQi_da2 + gQo * dQo_da2;
  gr += ga2 * 4.0f * r * ag;  // d(r^4)/dr
  add3(gn, wi * (gQi * dQi_dc) + wo * (gQo * dQo_dc) + h * (gD * dD_dnh));
}

// ------------------------------------------------------------------ sampling
// BSDF sample direction: the cosine lobe (Malley's method) or, when `spec`,
// the mirrored GGX half vector with density D(h)(n.h) (Walter et al. 2007).
// The local direction, the frame (b1, b2, n) after Duff et al. 2017 of the
// record's normal with its residual (n + nlo) and the reflection are
// assembled in double-float arithmetic (the DF operations above, ~1e-14)
// from the FP32 inputs (roughness r + rlo) and rounded once, so the FP32
// rounding of the result (~5e-8 rad) is about its only error; in FP32 the
// frame and the reflection 2 (wo.h) h - wo (which doubles the rounding
// errors of h and of the roughness) gave up to 6e-7 rad at roughness 0.7,
// enough to flip a support decision of a glossy metal's continuation ray.
// Double-float rather than FP64 because FP64 runs at a small fraction of
// the FP32 rate on this part: sample generation 1.70 -> 0.68 ms at the same
// accuracy.  The azimuth is sincospif's (one ulp, ~6e-8).  One code path for
// both lobes, so a warp whose samples pick both pays for the assembly once.
//
// GGX: cos^2 theta_h = (1 - u1) / (1 + (a2 - 1) u1), evaluated as
// (1 - u1) / ((1 - u1) + a2 u1) and sin^2 as a2 u1 / (same), which keeps the
// digits of both for a glossy lobe (small a2) at either end of u1 (1 - u1 is
// exact for the 24-bit uniforms).
__device__ __forceinline__ DF dff(float x) { return DF{x, 0.0f}; }
__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sqrt0(DF a) { return a.hi > 0.0f ? df_sqrt(a) : DF{0.0f, 0.0f}; }
__device__ __forceinline__ DF df_fma(DF a, DF b, DF c) { return df_add(df_mul(a, b), c); }
__device__ __forceinline__ float3 sample_bsdf_dir(bool spec, float3 n, float3 nlo, float3 wo, float r, float rlo,
                                                  float u1, float u2) {
  DF st, ct;
  const float om = 1.0f - u1;  // exact for the 24-bit uniforms
  if (spec) {
    const DF rd{r, rlo};
    const DF ag = df_mul(rd, rd), a2 = df_mul(ag, ag), a2u = df_mul(a2, dff(u1));
    const DF inv = df_div(dff(1.0f), df_add(a2u, dff(om)));
    ct = df_sqrt0(df_mul(dff(om), inv));
    st = df_sqrt0(df_mul(a2u, inv));
  } else {
    st = df_sqrt0(dff(u1));
    ct = df_sqrt0(dff(om));
  }
  float spf, cpf;
  sincospif(2.0f * u2, &spf, &cpf);  // angle 2 pi u2 without rounding 2 pi u2
  const DF sp = df_mul(dff(spf), st), cp = df_mul(dff(cpf), st);
  const DF nx{n.x, nlo.x}, ny{n.y, nlo.y}, nz{n.z, nlo.z};
  const bool pos = nz.hi > 0.0f || (nz.hi == 0.0f && !signbit(nz.lo != 0.0f ? nz.lo : nz.hi));
  const float sgn = pos ? 1.0f : -1.0f;
  const DF a = df_div(dff(-1.0f), df_add(dff(sgn), nz));
  const DF b = df_mul(df_mul(nx, ny), a), nx2a = df_mul(df_mul(nx, nx), a);
  const DF b1x = df_add(dff(1.0f), pos ? nx2a : df_neg(nx2a)), b1y = pos ? b : df_neg(b), b1z = pos ? df_neg(nx) : nx;
  const DF b2x = b, b2y = df_add(dff(sgn), df_mul(df_mul(ny, ny), a)), b2z = df_neg(ny);
  DF vx = df_fma(b1x, cp, df_fma(b2x, sp, df_mul(nx, ct)));
  DF vy = df_fma(b1y, cp, df_fma(b2y, sp, df_mul(ny, ct)));
  DF vz = df_fma(b1z, cp, df_fma(b2z, sp, df_mul(nz, ct)));
  if (spec) {
    const DF oh = df_fma(dff(wo.x), vx, df_fma(dff(wo.y), vy, df_mul(dff(wo.z), vz)));
    const DF oh2{2.0f * oh.hi, 2.0f * oh.lo};
    vx = df_fma(vx, oh2, dff(-wo.x));
    vy = df_fma(vy, oh2, dff(-wo.y));
    vz = df_fma(vz, oh2, dff(-wo.z));
  }
  return f3(vx.hi, vy.hi, vz.hi);
}

__device__ __forceinline__ float pdf_bsdf(float3 n, float3 wo, float3 wi, float r, float p_spec) {
  float pc = fmaxf(0.0f, dot3(n, wi)) * INV_PI_F;
  float pg = 0.0f;
  if (p_spec > 0.0f) {
    float3 hs = wi + wo;
    float hl = sqrtf(dot3(hs, hs));
    if (hl > 0.0f) {
      float3 h = hs * (1.0f / hl);
      float nh = dot3(n, h), oh = dot3(wo, h);
      if (nh > 0.0f && oh > 0.0f) {
        float ag = r * r, a2 = ag * ag, den = ggx_den(n, h, nh, a2);
        pg = a2 / (PI_F * den * den) * nh / (4.0f * oh);
      }
    }
  }
  return p_spec * pg + (1.0f - p_spec) * pc;
}

// ------------------------------------------------------------------ camera
__device__ __forceinline__ float3 camera_dir(const CamDev& c, int p) {
  const int x = p % c.W, y = p / c.W;
  const double sx = __dmul_rn(__dmul_rn(__dsub_rn(__dmul_rn(__ddiv_rn(__dadd_rn((double)x, 0.5), (double)c.W), 2.0), 1.0),
                                        c.th), c.aspect);
  const double sy = __dmul_rn(__dsub_rn(1.0, __dmul_rn(__ddiv_rn(__dadd_rn((double)y, 0.5), (double)c.H), 2.0)), c.th);
  double v[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) v[k] = __dadd_rn(__dadd_rn(c.f[k], __dmul_rn(c.r[k], sx)), __dmul_rn(c.u[k], sy));
  const double l = __dsqrt_rn(__dadd_rn(__dadd_rn(__dmul_rn(v[0], v[0]), __dmul_rn(v[1], v[1])), __dmul_rn(v[2], v[2])));
  return f3((float)__ddiv_rn(v[0], l), (float)__ddiv_rn(v[1], l), (float)__ddiv_rn(v[2], l));
}

// ------------------------------------------------------------------ traversal
// The origin is o + olo: shading rays start at a G-buffer position plus an
// offset along the normal, whose sum a double-float keeps exactly (the
// precise hit test subtracts olo; the culling tests use o alone).
//
// The lanes that trace a ray together all need the same 15 values (o, d,
// 1/d, o/d, olo).  RayR keeps them in registers, in every lane; RayS keeps
// them once per ray in shared memory (five 16-byte quads written by
// make_ray) and each test reads the quads it needs when it runs (a
// broadcast load), which frees those registers in every lane for the
// traversal and hit-test state.  Each kernel takes the kind that measured
// faster for it: RayS where the register cap forces spills (the shadow
// rays at 32 registers), RayR elsewhere.
constexpr int RAY_QUADS = 5;  // shared-memory quads per ray: o, d, inv, oinv, olo

__device__ __forceinline__ float3 lds3(unsigned a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a));
  return f3(v.x, v.y, v.z);
}
__device__ __forceinline__ void sts3(unsigned a, float3 v) {
  asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(a), "f"(v.x), "f"(v.y), "f"(v.z), "f"(0.0f)
               : "memory");
}

struct RayS {
  unsigned s;  // shared-memory address of the ray's quads
  __device__ __forceinline__ float3 o() const { return lds3(s); }
  __device__ __forceinline__ float3 d() const { return lds3(s + 16); }
  __device__ __forceinline__ float3 inv() const { return lds3(s + 32); }
  __device__ __forceinline__ float3 oinv() const { return lds3(s + 48); }
  __device__ __forceinline__ float3 olo() const { return lds3(s + 64); }
};
struct RayR {
  float3 o_, d_, inv_, oinv_, olo_;
  __device__ __forceinline__ float3 o() const { return o_; }
  __device__ __forceinline__ float3 d() const { return d_; }
  __device__ __forceinline__ float3 inv() const { return inv_; }
  __device__ __forceinline__ float3 oinv() const { return oinv_; }
  __device__ __forceinline__ float3 olo() const { return olo_; }
};

// The ray from o + olo along d.  `slot` is the ray's RAY_QUADS quads of
// shared memory (used by RayS); `lane` and `mask` are the calling lane's
// index within the lanes of the ray and their warp mask (all of them call).
template <class R>
__device__ __forceinline__ R make_ray(float4* slot, int lane, unsigned mask, float3 o, float3 d,
                                      float3 olo = f3(0.f, 0.f, 0.f)) {
  const float ix = 1.0f / (fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x));
  const float iy = 1.0f / (fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y));
  const float iz = 1.0f / (fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z));
  const float3 inv = f3(ix, iy, iz), oinv = f3(o.x * ix, o.y * iy, o.z * iz);
  R r;
  if constexpr (sizeof(R) == sizeof(RayS)) {
    r.s = (unsigned)__cvta_generic_to_shared(slot);
    __syncwarp(mask);  // the previous ray's readers are done with the slot
    if (lane < RAY_QUADS)
      sts3(r.s + 16 * lane, lane == 0 ? o : lane == 1 ? d : lane == 2 ? inv : lane == 3 ? oinv : olo);
    __syncwarp(mask);
  } else {
    r.o_ = o;
    r.d_ = d;
    r.inv_ = inv;
    r.oinv_ = oinv;
    r.olo_ = olo;
  }
  return r;
}

// Slab test of [lo, hi] against the ray clipped to [tlo, thi].
template <class Ray>
__device__ __forceinline__ bool slab(float lx, float ly, float lz, float hx, float hy, float hz, const Ray& r,
                                     float tlo, float thi, float& tnear) {
  const float3 inv = r.inv(), oinv = r.oinv();
  float tx0 = fmaf(lx, inv.x, -oinv.x), tx1 = fmaf(hx, inv.x, -oinv.x);
  float ty0 = fmaf(ly, inv.y, -oinv.y), ty1 = fmaf(hy, inv.y, -oinv.y);
  float tz0 = fmaf(lz, inv.z, -oinv.z), tz1 = fmaf(hz, inv.z, -oinv.z);
  tnear = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tlo));
  float tfar = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), thi));
  return tnear <= tfar;
}

// Slab test of a compressed wide slot: FP16 box corners relative to the node
// centre H (rounded outward when packed).  The plane distances are
// (H + rel - o) / d = rel * inv + (H * inv - o * inv): one FMA per plane after
// the node's three centre terms.
__device__ __forceinline__ float2 h2_bits(unsigned u) {  // low half -> .x
  return __half22float2(__halves2half2(__ushort_as_half((unsigned short)(u & 0xffffu)),
                                       __ushort_as_half((unsigned short)(u >> 16))));
}
template <class Ray>
__device__ __forceinline__ bool slab_rel(const uint4& S, const float4& H, const Ray& r, float tlo, float thi,
                                         float& tnear) {
  const float3 inv = r.inv(), oinv = r.oinv();
  const float cx = fmaf(H.x, inv.x, -oinv.x), cy = fmaf(H.y, inv.y, -oinv.y), cz = fmaf(H.z, inv.z, -oinv.z);
  const float2 lxy = h2_bits(S.x), lzhx = h2_bits(S.y), hyz = h2_bits(S.z);
  const float tx0 = fmaf(lxy.x, inv.x, cx), tx1 = fmaf(lzhx.y, inv.x, cx);
  const float ty0 = fmaf(lxy.y, inv.y, cy), ty1 = fmaf(hyz.x, inv.y, cy);
  const float tz0 = fmaf(lzhx.x, inv.z, cz), tz1 = fmaf(hyz.y, inv.z, cz);
  tnear = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), tlo));
  const float tfar = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), thi));
  return tnear <= tfar;
}

// Traversal counters of one thread (for the roofline accounting): the trace
// kernels are compiled with Counters when the caller asked for counts and
// with NoCounters, which costs nothing, otherwise.
struct Counters {
  static constexpr bool on = true;
  unsigned nodes = 0, tests = 0;
  __device__ __forceinline__ void node() { ++nodes; }
  __device__ __forceinline__ void test(int n) { tests += (unsigned)n; }
};
struct NoCounters {
  static constexpr bool on = false;
  unsigned nodes = 0, tests = 0;
  __device__ __forceinline__ void node() {}
  __device__ __forceinline__ void test(int) {}
};

// Stack entries name (instance, node or leaf): instance << 25 | leaf flag
// (bit 24) | index.
constexpr int LEAF_BIT = 1 << 24;

// Composited surface record of one ray (Eq. 7).
struct Surface {
  float T, W, depth, m, r, nlen;
  float3 x, n, a;
  float3 x_lo, n_lo;  // residuals of x and n below their FP32 values (precise composite; else 0)
  float r_lo;
  float3 Sa;  // sum w a (un-normalised)
  int hits;
  unsigned long long stop_key;  // key of the last composited hit (0: none)
};

}  // namespace lf
