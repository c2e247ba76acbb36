// Geometry-refinement losses of one view on the traced G-buffer (Eq. 8-9)
// and their gradient with respect to the G-buffer's depth and normal planes,
// which lf_trace_backward then carries to the surfels.
//
//   L_D  = || C (D - D*) ||_1 / (|| C D* ||_1 + eps)
//   L_N  = 1 - <N, N*>_F / (H W)
//   L_DN = 1 - <N^D, N*>_F / (H W)
//
// N^D, the depth-derived normal, is normalize(P_x x P_y) with P(q) =
// eye + D(q) d(q) the back-projected position along the pixel's ray,
// P_x = P(x+1, y) - P(x-1, y) and P_y = P(x, y-1) - P(x, y+1) (central
// differences; image right and up, so it faces the camera on a visible
// surface); it is 0 on the image border and where the pixel or one of its
// four neighbours has no composited hit.
//
// Two passes over the pixels: k_geo_terms forms the four image sums (FP64,
// block reduction + one atomic per block) and, for each pixel with a
// depth-derived normal, the gradients of its P_x and P_y for the normal-term
// weight g = -N* / (H W); k_geo_grad gathers them from the four neighbours
// into the depth gradient (P(q) enters the differences of the pixels beside
// it) and adds the depth and normal gradients to the caller's G-buffer
// gradient.
#include "lf_ctx.h"

namespace lf {
namespace {

constexpr int GB = 256;

struct GeoArgs {
  const float* gbuf;
  int W, H;
  size_t P;
  const float* dref;   // W*H
  const float* conf;   // W*H
  const float* nref;   // 3 planes of W*H
  double* sums;        // [4]: sum C|D - D*|, sum C|D*|, sum <N, N*>, sum <N^D, N*>
  float* dpx;          // 3 planes: d(loss term)/d P_x per pixel
  float* dpy;          // 3 planes: d(loss term)/d P_y per pixel
};

__device__ __forceinline__ float3 plane3(const float* base, size_t P, int p) {
  return f3(base[p], base[P + p], base[2 * P + p]);
}
__device__ __forceinline__ bool hit_at(const GeoArgs& a, int p) { return a.gbuf[LF_CH_HITS * a.P + p] > 0.0f; }
// D(q) d(q) in FP64: position differences are taken without the eye (it
// cancels) and without rounding the products, so the central differences
// keep their digits.
__device__ __forceinline__ double3 offset_at(const GeoArgs& a, int p) {
  const double D = a.gbuf[LF_CH_DEPTH * a.P + p];
  const float3 d = plane3(a.gbuf + LF_CH_DIR * a.P, a.P, p);
  return make_double3(D * d.x, D * d.y, D * d.z);
}
__device__ __forceinline__ double3 dsub(double3 u, double3 v) { return make_double3(u.x - v.x, u.y - v.y, u.z - v.z); }

__device__ __forceinline__ double block_sum(double v, double* s_warp) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) s_warp[warp] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < GB / 32; ++w) t += s_warp[w];
  return t;  // valid in thread 0
}

__global__ void __launch_bounds__(GB) k_geo_terms(GeoArgs a) {
  __shared__ double s_warp[GB / 32];
  const int p = blockIdx.x * GB + threadIdx.x;
  double t0 = 0.0, t1 = 0.0, t2 = 0.0, t3 = 0.0;
  if (p < (int)a.P) {
    const int x = p % a.W, y = p / a.W;
    const float D = a.gbuf[LF_CH_DEPTH * a.P + p], Ds = a.dref[p], C = a.conf[p];
    t0 = (double)C * fabs((double)D - (double)Ds);
    t1 = fabs((double)C * (double)Ds);
    const float3 N = plane3(a.gbuf + LF_CH_N * a.P, a.P, p), Ns = plane3(a.nref, a.P, p);
    t2 = (double)N.x * Ns.x + (double)N.y * Ns.y + (double)N.z * Ns.z;
    float3 gx = f3(0.f, 0.f, 0.f), gy = gx;
    if (x > 0 && x < a.W - 1 && y > 0 && y < a.H - 1 && hit_at(a, p) && hit_at(a, p - 1) && hit_at(a, p + 1) &&
        hit_at(a, p - a.W) && hit_at(a, p + a.W)) {
      const double3 pxd = dsub(offset_at(a, p + 1), offset_at(a, p - 1));
      const double3 pyd = dsub(offset_at(a, p - a.W), offset_at(a, p + a.W));
      const double3 cd = make_double3(pxd.y * pyd.z - pxd.z * pyd.y, pxd.z * pyd.x - pxd.x * pyd.z,
                                      pxd.x * pyd.y - pxd.y * pyd.x);
      const double lend = sqrt(cd.x * cd.x + cd.y * cd.y + cd.z * cd.z);
      if (lend > 0.0) {
        const float3 ND = f3((float)(cd.x / lend), (float)(cd.y / lend), (float)(cd.z / lend));
        const float3 px = f3((float)pxd.x, (float)pxd.y, (float)pxd.z), py = f3((float)pyd.x, (float)pyd.y, (float)pyd.z);
        const float len = (float)lend;
        t3 = (double)ND.x * Ns.x + (double)ND.y * Ns.y + (double)ND.z * Ns.z;
        const float3 g = Ns * (-1.0f / (float)a.P);          // d(-<N^D, N*>/HW)/d N^D
        const float3 dc = (g - ND * dot3(ND, g)) * (1.0f / len);  // through the normalisation
        gx = cross3(py, dc);  // d/d P_x of (P_x x P_y) . dc
        gy = cross3(dc, px);
      }
    }
    a.dpx[p] = gx.x; a.dpx[a.P + p] = gx.y; a.dpx[2 * a.P + p] = gx.z;
    a.dpy[p] = gy.x; a.dpy[a.P + p] = gy.y; a.dpy[2 * a.P + p] = gy.z;
  }
  const double s0 = block_sum(t0, s_warp), s1 = block_sum(t1, s_warp), s2 = block_sum(t2, s_warp),
               s3 = block_sum(t3, s_warp);
  if (threadIdx.x == 0) {
    atomicAdd(a.sums + 0, s0);
    atomicAdd(a.sums + 1, s1);
    atomicAdd(a.sums + 2, s2);
    atomicAdd(a.sums + 3, s3);
  }
}

__global__ void __launch_bounds__(GB) k_geo_grad(GeoArgs a, float eps, float wD, float wN, float wDN,
                                                 float* __restrict__ dgb) {
  const int p = blockIdx.x * GB + threadIdx.x;
  if (p >= (int)a.P) return;
  const int x = p % a.W, y = p / a.W;
  const float D = a.gbuf[LF_CH_DEPTH * a.P + p], Ds = a.dref[p], C = a.conf[p];
  const float sgn = D > Ds ? 1.0f : (D < Ds ? -1.0f : 0.0f);
  float gD = (float)((double)wD * C * sgn / (a.sums[1] + eps));
  // P(q) enters P_x of its left and right neighbours and P_y of those above and below
  float3 dP = f3(0.f, 0.f, 0.f);
  if (x > 0) add3(dP, plane3(a.dpx, a.P, p - 1));
  if (x < a.W - 1) dP = dP - plane3(a.dpx, a.P, p + 1);
  if (y < a.H - 1) add3(dP, plane3(a.dpy, a.P, p + a.W));
  if (y > 0) dP = dP - plane3(a.dpy, a.P, p - a.W);
  gD += wDN * dot3(dP, plane3(a.gbuf + LF_CH_DIR * a.P, a.P, p));
  dgb[LF_CH_DEPTH * a.P + p] += gD;
  const float3 Ns = plane3(a.nref, a.P, p);
  const float s = -wN / (float)a.P;
  dgb[(LF_CH_N + 0) * a.P + p] += s * Ns.x;
  dgb[(LF_CH_N + 1) * a.P + p] += s * Ns.y;
  dgb[(LF_CH_N + 2) * a.P + p] += s * Ns.z;
}

size_t geo_scratch(int w, int h) { return 256 + sizeof(float) * 6 * (size_t)w * h; }

}  // namespace
}  // namespace lf

using namespace lf;

extern "C" {

size_t lf_geometry_loss_scratch_bytes(int width, int height) {
  if (width <= 0 || height <= 0) return 0;
  return geo_scratch(width, height);
}

lf_status lf_geometry_loss(lf_ctx* c, const lf_camera* cam, const float* gbuf, const float* depth_ref,
                           const float* depth_conf, const float* normal_ref, float eps, const float* weights,
                           float* dL_dgbuf, void* scratch, size_t scratch_bytes, double* losses) {
  if (!c) return LF_ERR_INVALID;
  if (!cam || cam->width <= 0 || cam->height <= 0 || !gbuf || !depth_ref || !depth_conf || !normal_ref ||
      !scratch || !(eps >= 0.0f)) {
    c->err = "lf_geometry_loss: bad arguments";
    return LF_ERR_INVALID;
  }
  if (scratch_bytes < geo_scratch(cam->width, cam->height)) {
    c->err = "lf_geometry_loss: scratch too small";
    return LF_ERR_INVALID;
  }
  GeoArgs a;
  a.gbuf = gbuf;
  a.W = cam->width;
  a.H = cam->height;
  a.P = (size_t)a.W * a.H;
  a.dref = depth_ref;
  a.conf = depth_conf;
  a.nref = normal_ref;
  a.sums = static_cast<double*>(scratch);
  a.dpx = reinterpret_cast<float*>(static_cast<char*>(scratch) + 256);
  a.dpy = a.dpx + 3 * a.P;
  const int blocks = (int)((a.P + GB - 1) / GB);
  cudaError_t e = cudaMemsetAsync(a.sums, 0, 4 * sizeof(double), c->stream);
  if (e == cudaSuccess) {
    k_geo_terms<<<blocks, GB, 0, c->stream>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && dL_dgbuf) {
    const float w[3] = {weights ? weights[0] : 1.0f, weights ? weights[1] : 1.0f, weights ? weights[2] : 1.0f};
    k_geo_grad<<<blocks, GB, 0, c->stream>>>(a, eps, w[0], w[1], w[2], dL_dgbuf);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && losses) {
    double s[4];
    e = cudaMemcpyAsync(s, a.sums, sizeof(s), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) {
      losses[0] = s[0] / (s[1] + (double)eps);
      losses[1] = 1.0 - s[2] / (double)a.P;
      losses[2] = 1.0 - s[3] / (double)a.P;
    }
  }
  if (e != cudaSuccess) {
    c->err = std::string("lf_geometry_loss: ") + cudaGetErrorString(e);
    return LF_ERR_CUDA;
  }
  return LF_OK;
}

}  // extern "C"
