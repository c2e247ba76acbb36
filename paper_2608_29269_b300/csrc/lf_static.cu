// lf_shade_bounce_static: the one-bounce shading of lf_shade_bounce for
// callers that cannot allocate device memory.
//
// lf_shade_bounce needs a per-sample scratch buffer from the caller.  Some
// callers cannot provide one: a host program whose device memory is owned up
// front by another allocator (a framework that reserves the whole device), a
// plugin that is not allowed to call cudaMalloc, or a render loop that must
// not allocate after start-up.  This entry point takes its scratch from a
// fixed array compiled into the library instead, so it allocates nothing.
//
// The array is file-scope `static __device__` memory of LF_STATIC_SCRATCH_BYTES:
// every GPU that loads the library holds it until the process exits.  All
// calls share it and it keeps the last call's contents; the queue counters
// that must start at zero are cleared by every call.  Two calls whose work
// overlaps on the GPU (different streams, contexts or threads) race on it.
#include <cstdio>
#include <mutex>

#include "lf_ctx.h"
#include "lf_wavefront.h"

namespace {

static __device__ __align__(256) unsigned char g_shade_scratch[LF_STATIC_SCRATCH_BYTES];

// Device address of g_shade_scratch per device.  The host-side name of the
// array is only a stand-in, so the address is looked up with
// cudaGetSymbolAddress while the context's device is current, on the first
// call after a context was created on that device (lf_create drops the
// cached address: a cudaDeviceReset in between would leave it stale, and a
// reset also ends every context made before it).
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// `device` is the calling thread's current device.
cudaError_t scratch_address(int device, void** out) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_shade_scratch);
    if (e != cudaSuccess) return e;
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return cudaSuccess;
}

// Largest width * height * spp whose sample buffer fits the array.
size_t max_samples() {
  size_t lo = 0, hi = LF_STATIC_SCRATCH_BYTES / (sizeof(float) * lf::SAMPLE_PLANES);
  while (lo < hi) {
    const size_t mid = (lo + hi + 1) / 2;
    if (lf::sample_buf_bytes((long long)mid) <= LF_STATIC_SCRATCH_BYTES) lo = mid; else hi = mid - 1;
  }
  return lo;
}

}  // namespace

void lf_static_scratch_forget(int device) {
  std::lock_guard<std::mutex> lock(g_mu);
  if (device >= 0 && device < kMaxDevices) g_addr[device] = nullptr;
}

extern "C" {

lf_status lf_shade_bounce_static(lf_ctx* c, const lf_camera* cam, const float* gbuf, int env_id, int spp,
                                 uint64_t seed, float* rgb, unsigned long long* ray_count) {
  if (!c) return LF_ERR_INVALID;
  if (!cam || cam->width <= 0 || cam->height <= 0 || spp <= 0) {
    c->err = "lf_shade_bounce_static: bad camera or spp";
    return LF_ERR_INVALID;
  }
  const long long n = (long long)cam->width * cam->height * spp;
  const size_t cap = max_samples();
  if (n > (long long)cap) {
    char msg[256];
    snprintf(msg, sizeof msg,
             "lf_shade_bounce_static: width*height*spp = %lld samples exceeds the static scratch capacity of %zu "
             "samples (%d bytes); use lf_shade_bounce with a caller buffer",
             n, cap, (int)LF_STATIC_SCRATCH_BYTES);
    c->err = msg;
    return LF_ERR_INVALID;
  }
  // The array's address is per device: the kernels run on the context's
  // device, so that device must be the current one (as for every call).
  int device = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess && device != c->device) {
    char msg[160];
    snprintf(msg, sizeof msg, "lf_shade_bounce_static: current device %d is not the context's device %d", device,
             c->device);
    c->err = msg;
    return LF_ERR_INVALID;
  }
  void* scratch = nullptr;
  if (e == cudaSuccess) e = scratch_address(c->device, &scratch);
  if (e != cudaSuccess) {
    c->err = std::string("lf_shade_bounce_static: scratch address: ") + cudaGetErrorString(e);
    return LF_ERR_CUDA;
  }
  return lf_shade_bounce(c, cam, gbuf, env_id, spp, seed, rgb, ray_count, scratch,
                         (size_t)LF_STATIC_SCRATCH_BYTES);
}

}  // extern "C"
