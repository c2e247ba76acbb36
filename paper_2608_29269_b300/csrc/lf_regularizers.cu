// Regularisers of the training objectives and their gradients:
//   L_alpha = || A - 1 ||_1 / (H W)                      (Eq. 4)  A = traced weight sum W of each pixel
//   L_s     = (1/N) sum_i max(0, ||s_i||_inf / s_max - 1)^2  (Eq. 5)  a tie splits the gradient evenly
//   L_TV(E) = (1 / (3 H W)) sum |E(r, c+1) - E(r, c)| + |E(r+1, c) - E(r, c)|   (Eq. 14)
//             anisotropic L1, wrapping in azimuth (columns), not across the poles (rows)
// Each is one elementwise pass that adds weight * gradient to the caller's
// buffer and block-sums its terms in FP64 into the context's loss slot.
#include "lf_ctx.h"

namespace lf {
namespace {

constexpr int RB = 256;

__device__ __forceinline__ void block_add(double v, double* out) {
  __shared__ double s_w[RB / 32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < RB / 32; ++w) t += s_w[w];
    atomicAdd(out, t);
  }
}

__device__ __forceinline__ float sgnf(float v) { return v > 0.0f ? 1.0f : (v < 0.0f ? -1.0f : 0.0f); }

__global__ void __launch_bounds__(RB) k_opacity_loss(const float* __restrict__ gbuf, size_t P, float weight,
                                                     float* __restrict__ dgb, double* sum) {
  const size_t p = (size_t)blockIdx.x * RB + threadIdx.x;
  double term = 0.0;
  if (p < P) {
    const float W = gbuf[LF_CH_W * P + p];
    term = fabs((double)W - 1.0);
    if (dgb) dgb[LF_CH_W * P + p] += weight * sgnf(W - 1.0f) / (float)P;
  }
  block_add(term, sum);
}

__global__ void __launch_bounds__(RB) k_scale_loss(const float* __restrict__ scale, int n, float s_max, float weight,
                                                   float* __restrict__ d_surfel, double* sum) {
  const int i = blockIdx.x * RB + threadIdx.x;
  double term = 0.0;
  if (i < n) {
    const float su = scale[2 * i], sv = scale[2 * i + 1];
    const double r = (double)fmaxf(su, sv) / (double)s_max - 1.0;  // FP64: r is a small difference near s_max
    if (r > 0.0) {
      term = r * r;
      if (d_surfel) {
        const float g = (float)((double)weight * 2.0 * r / ((double)s_max * (double)n));
        float* o = d_surfel + (size_t)LF_G_STRIDE * i + 9;  // scale columns
        if (su == sv) {
          o[0] += 0.5f * g;
          o[1] += 0.5f * g;
        } else if (su > sv) {
          o[0] += g;
        } else {
          o[1] += g;
        }
      }
    }
  }
  block_add(term, sum);
}

__global__ void __launch_bounds__(RB) k_env_tv(const float* __restrict__ E, int H, int W, float weight,
                                               float* __restrict__ d_env, double* sum) {
  const long long k = (long long)blockIdx.x * RB + threadIdx.x;  // texel * 3 + channel
  const long long total = 3ll * H * W;
  double term = 0.0;
  if (k < total) {
    const int ch = (int)(k % 3);
    const long long t = k / 3;
    const int r = (int)(t / W), c = (int)(t % W);
    auto at = [&](int rr, int cc) { return E[3 * ((long long)rr * W + cc) + ch]; };
    const float e = at(r, c);
    const float du = at(r, (c + 1) % W) - e;              // this texel's azimuthal difference
    const float du_l = e - at(r, (c + W - 1) % W);        // the left neighbour's
    term = fabs((double)du);
    float g = -sgnf(du) + sgnf(du_l);
    if (r < H - 1) {
      const float dv = at(r + 1, c) - e;
      term += fabs((double)dv);
      g -= sgnf(dv);
    }
    if (r > 0) g += sgnf(e - at(r - 1, c));
    if (d_env) d_env[k] += weight * g / (float)total;
  }
  block_add(term, sum);
}

lf_status finish(lf_ctx* c, double scale, double* loss, const char* what) {
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss) {
    double s = 0.0;
    e = cudaMemcpyAsync(&s, c->loss_dev, sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) *loss = s * scale;
  }
  if (e != cudaSuccess) {
    c->err = std::string(what) + ": " + cudaGetErrorString(e);
    return LF_ERR_CUDA;
  }
  return LF_OK;
}

}  // namespace
}  // namespace lf

using namespace lf;

extern "C" {

lf_status lf_opacity_loss(lf_ctx* c, const lf_camera* cam, const float* gbuf, float weight, float* dL_dgbuf,
                          double* loss) {
  if (!c) return LF_ERR_INVALID;
  if (!cam || cam->width <= 0 || cam->height <= 0 || !gbuf) {
    c->err = "lf_opacity_loss: bad arguments";
    return LF_ERR_INVALID;
  }
  const size_t P = (size_t)cam->width * cam->height;
  if (cudaMemsetAsync(c->loss_dev, 0, sizeof(double), c->stream) != cudaSuccess) return LF_ERR_CUDA;
  k_opacity_loss<<<(unsigned)((P + RB - 1) / RB), RB, 0, c->stream>>>(gbuf, P, weight, dL_dgbuf, c->loss_dev);
  return finish(c, 1.0 / (double)P, loss, "lf_opacity_loss");
}

lf_status lf_scale_loss(lf_ctx* c, const float* scale, int n, float s_max, float weight, float* d_surfel,
                        double* loss) {
  if (!c) return LF_ERR_INVALID;
  if (!scale || n <= 0 || !(s_max > 0.0f)) {
    c->err = "lf_scale_loss: bad arguments";
    return LF_ERR_INVALID;
  }
  if (cudaMemsetAsync(c->loss_dev, 0, sizeof(double), c->stream) != cudaSuccess) return LF_ERR_CUDA;
  k_scale_loss<<<(n + RB - 1) / RB, RB, 0, c->stream>>>(scale, n, s_max, weight, d_surfel, c->loss_dev);
  return finish(c, 1.0 / (double)n, loss, "lf_scale_loss");
}

lf_status lf_env_tv_loss(lf_ctx* c, const float* rgb, int H, int W, float weight, float* d_env, double* loss) {
  if (!c) return LF_ERR_INVALID;
  if (!rgb || H <= 0 || W <= 0) {
    c->err = "lf_env_tv_loss: bad arguments";
    return LF_ERR_INVALID;
  }
  const long long total = 3ll * H * W;
  if (cudaMemsetAsync(c->loss_dev, 0, sizeof(double), c->stream) != cudaSuccess) return LF_ERR_CUDA;
  k_env_tv<<<(unsigned)((total + RB - 1) / RB), RB, 0, c->stream>>>(rgb, H, W, weight, d_env, c->loss_dev);
  return finish(c, 1.0 / (double)total, loss, "lf_env_tv_loss");
}

}  // extern "C"
