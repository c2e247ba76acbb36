// Primary-ray compositing (Eq. 6-7).
#include "lf_coop.cuh"
#include "lf_kernels.h"

namespace lf {

constexpr int TB = 128;                      // threads per block
constexpr int RGROUPS = TB / WIDE;           // pixels per block (one per lane group)
constexpr int RSTACK_SMEM = RGROUPS * CRAY_SMEM;
constexpr int TILE_W = RGROUPS >= 4 ? 4 : RGROUPS;  // a block's pixels form a TILE_W x TILE_H tile
constexpr int TILE_H = RGROUPS / TILE_W;

// WIDE lanes per pixel: cooperative k-buffer composite of the primary ray
// (lf_coop.cuh); lane 0 writes the G-buffer.
template <class Cnt>
__global__ void __launch_bounds__(TB, 8) k_trace_primary(TraceArgs a, CamDev cam, float* __restrict__ gbuf) {
  extern __shared__ __align__(16) int s_cstack[];
  const Grp g = make_grp();
  const int gid = threadIdx.x / WIDE;
  const CStack st = ray_smem(reinterpret_cast<unsigned char*>(s_cstack), RGROUPS, gid);
  const int x = blockIdx.x * TILE_W + gid % TILE_W, y = blockIdx.y * TILE_H + gid / TILE_W;
  if (x >= cam.W || y >= cam.H) return;  // uniform over the group
  const int p = y * cam.W + x;
  const size_t P = (size_t)cam.W * cam.H;
  float3 d = f3(0.f, 0.f, 0.f);
  if (g.c == 0) d = camera_dir(cam, p);  // FP64 once per pixel
  d = f3(gshfl(g, d.x, 0), gshfl(g, d.y, 0), gshfl(g, d.z, 0));
  Cnt cnt;
  unsigned comp = 0;
  Surface s;
  coop_composite(g, a.insts, a.n_inst, cam.eye, d, a.P, st, a.status, cnt, s, comp);
  if (g.c != 0) return;
  const float3 rho = s.Sa + env_lookup(a.env, d) * s.T;
  float* gp = gbuf + p;
  gp[LF_CH_T * P] = s.T;
  gp[LF_CH_W * P] = s.W;
  gp[LF_CH_DEPTH * P] = s.depth;
  gp[(LF_CH_X + 0) * P] = s.x.x; gp[(LF_CH_X + 1) * P] = s.x.y; gp[(LF_CH_X + 2) * P] = s.x.z;
  gp[(LF_CH_N + 0) * P] = s.n.x; gp[(LF_CH_N + 1) * P] = s.n.y; gp[(LF_CH_N + 2) * P] = s.n.z;
  gp[(LF_CH_A + 0) * P] = s.a.x; gp[(LF_CH_A + 1) * P] = s.a.y; gp[(LF_CH_A + 2) * P] = s.a.z;
  gp[LF_CH_M * P] = s.m;
  gp[LF_CH_R * P] = s.r;
  gp[(LF_CH_RHO + 0) * P] = rho.x; gp[(LF_CH_RHO + 1) * P] = rho.y; gp[(LF_CH_RHO + 2) * P] = rho.z;
  gp[LF_CH_NLEN * P] = s.nlen;
  gp[LF_CH_HITS * P] = (float)s.hits;
  gp[LF_CH_TSTOP * P] = key_t(s.stop_key);
  gp[LF_CH_IDSTOP * P] = s.hits ? (float)(int)(s.stop_key & 0xffffffull) : -1.0f;
  gp[(LF_CH_DIR + 0) * P] = d.x; gp[(LF_CH_DIR + 1) * P] = d.y; gp[(LF_CH_DIR + 2) * P] = d.z;
  gp[LF_CH_STOPKEY_LO * P] = __uint_as_float((unsigned)(s.stop_key & 0xffffffffull));
  if (Cnt::on && a.counters) {  // slot 0 of the per-kernel counters: primary rays
    atomicAdd(a.counters + 0, (unsigned long long)cnt.nodes);
    atomicAdd(a.counters + 1, (unsigned long long)cnt.tests);
    atomicAdd(a.counters + 2, (unsigned long long)comp);
    atomicAdd(a.counters + 3, 1ull);
  }
}

cudaError_t launch_trace_primary(const TraceArgs& a, const CamDev& cam, float* gbuf, cudaStream_t st) {
  dim3 grid((cam.W + TILE_W - 1) / TILE_W, (cam.H + TILE_H - 1) / TILE_H);
  if (a.counters) k_trace_primary<Counters><<<grid, TB, RSTACK_SMEM, st>>>(a, cam, gbuf);
  else k_trace_primary<NoCounters><<<grid, TB, RSTACK_SMEM, st>>>(a, cam, gbuf);
  return cudaGetLastError();
}

}  // namespace lf
