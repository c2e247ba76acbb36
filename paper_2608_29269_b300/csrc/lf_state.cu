// Cross-state supervision (Sec. 3.2): one shared canonical scene, assembled
// per observed state by Eq. 2 -- the background B as it is, object o placed by
// the rigid transform T_{k,o} = (R_{k,o}, t_{k,o}) acting on the centres and
// tangent axes of its surfels -- and the adjoint that carries a state's
// per-surfel gradient back to the canonical parameters, so that the residuals
// of every state update the same surfels.
//
// Both kernels evaluate each component in FP64 as ((R0 x0 + R1 x1) + R2 x2)
// (+ t): every product of two FP32 values is exact in FP64 and the sums are
// explicit round-to-nearest adds, so the result rounded once to FP32 does not
// depend on FMA contraction (the same arithmetic as lf_bvh_refit).
#include "lf_ctx.h"

namespace lf {
namespace {

constexpr int SB = 256;

struct StateXf {
  Mat34 T[LF_MAX_OBJECTS];  // T[0] (the background) is not read
};

// Object of surfel i: the last k with off[k] <= i (empty objects skipped).
__device__ __forceinline__ int object_of(const int* __restrict__ off, int n_obj, int i) {
  int lo = 0, hi = n_obj - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= i) lo = mid; else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ double rot_row(const float* R, int r, float x0, float x1, float x2) {
  return __dadd_rn(__dadd_rn(__dmul_rn(R[3 * r], x0), __dmul_rn(R[3 * r + 1], x1)), __dmul_rn(R[3 * r + 2], x2));
}
// Row j of R^T g: column j of R.
__device__ __forceinline__ float rot_col(const float* R, int j, float g0, float g1, float g2) {
  return __double2float_rn(__dadd_rn(__dadd_rn(__dmul_rn(R[j], g0), __dmul_rn(R[3 + j], g1)), __dmul_rn(R[6 + j], g2)));
}

// One thread per surfel: the state's mu, tu, tv from the canonical ones, and
// copies of the shared attributes whose arrays differ (copy_mask bit per
// field: scale, opacity, albedo, metallic, roughness).
__global__ void __launch_bounds__(SB) k_assemble(SceneDev w, SceneDev cs, const int* __restrict__ off, int n_obj,
                                                 StateXf X, unsigned copy_mask) {
  const int i = blockIdx.x * SB + threadIdx.x;
  if (i >= w.n) return;
  const int o = object_of(off, n_obj, i);
  const float* src[3] = {cs.mu + 3 * i, cs.tu + 3 * i, cs.tv + 3 * i};
  float* dst[3] = {w.mu + 3 * i, w.tu + 3 * i, w.tv + 3 * i};
#pragma unroll
  for (int f = 0; f < 3; ++f) {
    const float x0 = src[f][0], x1 = src[f][1], x2 = src[f][2];
    if (o == 0) {
      dst[f][0] = x0; dst[f][1] = x1; dst[f][2] = x2;
    } else {
      const float* R = X.T[o].R;
#pragma unroll
      for (int r = 0; r < 3; ++r) {
        const double y = rot_row(R, r, x0, x1, x2);
        dst[f][r] = __double2float_rn(f == 0 ? __dadd_rn(y, (double)X.T[o].t[r]) : y);
      }
    }
  }
  if (copy_mask & 1u) { w.scale[2 * i] = cs.scale[2 * i]; w.scale[2 * i + 1] = cs.scale[2 * i + 1]; }
  if (copy_mask & 2u) w.opacity[i] = cs.opacity[i];
  if (copy_mask & 4u)
    for (int c = 0; c < 3; ++c) w.albedo[3 * i + c] = cs.albedo[3 * i + c];
  if (copy_mask & 8u) w.metallic[i] = cs.metallic[i];
  if (copy_mask & 16u) w.roughness[i] = cs.roughness[i];
}

// One thread per gradient entry (coalesced over the N x 17 rows): mu, tu and
// tv entries of a moved object become rows of R^T g, every other entry passes.
__global__ void __launch_bounds__(SB) k_state_pullback(const float* __restrict__ gw, float* __restrict__ gc, int n,
                                                       const int* __restrict__ off, int n_obj, StateXf X) {
  const long long e = (long long)blockIdx.x * SB + threadIdx.x;
  if (e >= (long long)n * LF_G_STRIDE) return;
  const int i = (int)(e / LF_G_STRIDE), k = (int)(e - (long long)i * LF_G_STRIDE);
  float v = gw[e];
  if (k < LF_G_S) {
    const int o = object_of(off, n_obj, i);
    if (o != 0) {
      const float* g = gw + (long long)i * LF_G_STRIDE + (k / 3) * 3;
      v = rot_col(X.T[o].R, k % 3, g[0], g[1], g[2]);
    }
  }
  gc[e] += v;
}

bool fill_xf(const float* R, const float* t, int n_obj, StateXf& X) {
  for (int o = 1; o < n_obj; ++o) {
    const float* Ro = R + 9 * (o - 1);
    const float* to = t ? t + 3 * (o - 1) : nullptr;
    if (!lf_is_rigid(Ro, to)) return false;
    for (int q = 0; q < 9; ++q) X.T[o].R[q] = Ro[q];
    for (int q = 0; q < 3; ++q) X.T[o].t[q] = to ? to[q] : 0.0f;
  }
  return true;
}

lf_status state_fail(lf_ctx* c, lf_status s, const char* msg) {
  c->err = msg;
  return s;
}

}  // namespace
}  // namespace lf

using namespace lf;

extern "C" {

lf_status lf_state_assemble(lf_ctx* c, const lf_scene* canonical, const float* R, const float* t) {
  if (!c) return LF_ERR_INVALID;
  if (!c->built) return state_fail(c, LF_ERR_NOT_BUILT, "lf_state_assemble: no BVH");
  if (!canonical || (c->n_obj > 1 && (!R || !t)))
    return state_fail(c, LF_ERR_INVALID, "lf_state_assemble: missing canonical scene or transforms");
  if (canonical->n != c->n || canonical->n_objects != c->n_obj || !canonical->object_offsets)
    return state_fail(c, LF_ERR_INVALID, "lf_state_assemble: canonical scene does not match the built scene");
  for (int k = 0; k <= c->n_obj; ++k)
    if (canonical->object_offsets[k] != c->offsets[k])
      return state_fail(c, LF_ERR_INVALID, "lf_state_assemble: object offsets differ from the built scene");
  const SceneDev& w = c->scene;
  SceneDev cs{canonical->mu_dev, canonical->tu_dev, canonical->tv_dev, canonical->scale_dev,
              canonical->opacity_dev, canonical->albedo_dev, canonical->metallic_dev, canonical->roughness_dev,
              canonical->n};
  if (!cs.mu || !cs.tu || !cs.tv || !cs.scale || !cs.opacity || !cs.albedo || !cs.metallic || !cs.roughness)
    return state_fail(c, LF_ERR_INVALID, "lf_state_assemble: null canonical array");
  if (cs.mu == w.mu || cs.tu == w.tu || cs.tv == w.tv)
    return state_fail(c, LF_ERR_INVALID, "lf_state_assemble: canonical centres/axes alias the built scene's");
  StateXf X{};
  if (!fill_xf(R, t, c->n_obj, X)) return state_fail(c, LF_ERR_INVALID, "lf_state_assemble: transform is not rigid");
  const unsigned mask = (cs.scale != w.scale ? 1u : 0u) | (cs.opacity != w.opacity ? 2u : 0u) |
                        (cs.albedo != w.albedo ? 4u : 0u) | (cs.metallic != w.metallic ? 8u : 0u) |
                        (cs.roughness != w.roughness ? 16u : 0u);
  if (c->n > 0) {
    k_assemble<<<(c->n + SB - 1) / SB, SB, 0, c->stream>>>(w, cs, c->offsets_dev, c->n_obj, X, mask);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      c->err = std::string("lf_state_assemble: ") + cudaGetErrorString(e);
      return LF_ERR_CUDA;
    }
  }
  return lf_ctx_fit(c, 0, c->n_obj - 1);
}

lf_status lf_state_pullback(lf_ctx* c, const float* R, const float* d_world, float* d_canonical) {
  if (!c) return LF_ERR_INVALID;
  if (!c->built) return state_fail(c, LF_ERR_NOT_BUILT, "lf_state_pullback: no BVH");
  if (!d_world || !d_canonical || (c->n_obj > 1 && !R))
    return state_fail(c, LF_ERR_INVALID, "lf_state_pullback: null argument");
  const size_t bytes = sizeof(float) * LF_G_STRIDE * (size_t)c->n;
  const char *a = reinterpret_cast<const char*>(d_world), *b = reinterpret_cast<const char*>(d_canonical);
  if (a < b + bytes && b < a + bytes) return state_fail(c, LF_ERR_INVALID, "lf_state_pullback: buffers overlap");
  StateXf X{};
  if (!fill_xf(R, nullptr, c->n_obj, X)) return state_fail(c, LF_ERR_INVALID, "lf_state_pullback: R is not a rotation");
  const long long total = (long long)c->n * LF_G_STRIDE;
  if (total > 0) {
    k_state_pullback<<<(unsigned)((total + SB - 1) / SB), SB, 0, c->stream>>>(d_world, d_canonical, c->n,
                                                                               c->offsets_dev, c->n_obj, X);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      c->err = std::string("lf_state_pullback: ") + cudaGetErrorString(e);
      return LF_ERR_CUDA;
    }
  }
  return LF_OK;
}

}  // extern "C"
