// Primary-ray compositing (Eq. 6-7).
#include "lf_coop.cuh"
#include "lf_kernels.h"

namespace lf {

constexpr int TB = 128;                      // threads per block
#ifndef PRIMARY_MIN_BLOCKS
#define PRIMARY_MIN_BLOCKS 12  // resident blocks per SM asked of the compiler (4 % faster than 8, measured)
#endif
#ifndef PRIMARY_RAY
#define PRIMARY_RAY RayR  // the primary ray in registers (RayS measured slower here)
#endif
constexpr int RGROUPS = TB / WIDE;           // lane groups per block (one ray each at a time)
// Each group traces a strip of PSTRIP pixels one after another, and its
// first PSTRIP lanes compute the strip's camera rays together beforehand:
// the direction is FP64 (rounded once, as the oracle's), whose instructions
// cost the same for one active lane as for all, so one pass serves the
// strip (one ray at a time on lane 0 cost 0.75 ms of a 4.3 ms launch).
constexpr int PSTRIP = 8;
static_assert(PSTRIP <= WIDE, "a lane per pixel of the strip");
constexpr int SW = 4, SH = PSTRIP / SW;           // a strip is SW x SH pixels
constexpr int GX = 2, GY = RGROUPS / GX;          // the block's groups, GX x GY strips
constexpr int TILE_W = GX * SW, TILE_H = GY * SH;  // a block's pixels form a TILE_W x TILE_H tile
constexpr int RDIR_SMEM = RGROUPS * PSTRIP * (int)sizeof(float4);  // the strips' directions
constexpr int RSTACK_SMEM = RGROUPS * CRAY_SMEM + RDIR_SMEM;

// WIDE lanes per pixel: cooperative k-buffer composite of the primary ray
// through pixel (x, y) (lf_coop.cuh); lane 0 writes the G-buffer.
template <class Cnt>
__device__ __forceinline__ void trace_pixel(const Grp& g, const CStack& st, const Inst* insts, int n_inst,
                                            const DevParams& P, const EnvDev& env, int* status,
                                            unsigned long long* counters, const CamDev& cam, float* __restrict__ gbuf,
                                            int x, int y, float3 d) {
  const int p = y * cam.W + x;
  const size_t NP = (size_t)cam.W * cam.H;
  Cnt cnt;
  unsigned comp = 0;
  Surface s;
  coop_composite<PRIMARY_RAY, true>(g, insts, n_inst, cam.eye, f3(0.f, 0.f, 0.f), d, P, st, status, cnt, s, comp);
  if (g.c != 0) return;
  const float3 rho = s.Sa + env_lookup(env, d) * s.T;
  float* gp = gbuf + p;
  gp[LF_CH_T * NP] = s.T;
  gp[LF_CH_W * NP] = s.W;
  gp[LF_CH_DEPTH * NP] = s.depth;
  gp[(LF_CH_X + 0) * NP] = s.x.x; gp[(LF_CH_X + 1) * NP] = s.x.y; gp[(LF_CH_X + 2) * NP] = s.x.z;
  gp[(LF_CH_N + 0) * NP] = s.n.x; gp[(LF_CH_N + 1) * NP] = s.n.y; gp[(LF_CH_N + 2) * NP] = s.n.z;
  gp[(LF_CH_A + 0) * NP] = s.a.x; gp[(LF_CH_A + 1) * NP] = s.a.y; gp[(LF_CH_A + 2) * NP] = s.a.z;
  gp[LF_CH_M * NP] = s.m;
  gp[LF_CH_R * NP] = s.r;
  gp[(LF_CH_RHO + 0) * NP] = rho.x; gp[(LF_CH_RHO + 1) * NP] = rho.y; gp[(LF_CH_RHO + 2) * NP] = rho.z;
  gp[LF_CH_NLEN * NP] = s.nlen;
  gp[LF_CH_HITS * NP] = (float)s.hits;
  gp[LF_CH_TSTOP * NP] = key_t(s.stop_key);
  gp[LF_CH_IDSTOP * NP] = s.hits ? (float)(int)(s.stop_key & 0xffffffull) : -1.0f;
  gp[(LF_CH_DIR + 0) * NP] = d.x; gp[(LF_CH_DIR + 1) * NP] = d.y; gp[(LF_CH_DIR + 2) * NP] = d.z;
  gp[LF_CH_STOPKEY_LO * NP] = __uint_as_float((unsigned)(s.stop_key & 0xffffffffull));
  gp[(LF_CH_X_LO + 0) * NP] = s.x_lo.x; gp[(LF_CH_X_LO + 1) * NP] = s.x_lo.y; gp[(LF_CH_X_LO + 2) * NP] = s.x_lo.z;
  gp[(LF_CH_N_LO + 0) * NP] = s.n_lo.x; gp[(LF_CH_N_LO + 1) * NP] = s.n_lo.y; gp[(LF_CH_N_LO + 2) * NP] = s.n_lo.z;
  gp[LF_CH_R_LO * NP] = s.r_lo;
  if (Cnt::on && counters) {  // slot 0 of the per-kernel counters: primary rays
    atomicAdd(counters + 0, (unsigned long long)cnt.nodes);
    atomicAdd(counters + 1, (unsigned long long)cnt.tests);
    atomicAdd(counters + 2, (unsigned long long)comp);
    atomicAdd(counters + 3, 1ull);
  }
}

// The strip of group gid in the tile at (tx, ty) pixels: its camera rays
// (lanes c < PSTRIP, pixel c), then its pixels one after another.
template <class Cnt>
__device__ __forceinline__ void trace_strip(const Grp& g, int gid, const CStack& st, float4* dirs, const Inst* insts,
                                            int n_inst, const DevParams& P, const EnvDev& env, int* status,
                                            unsigned long long* counters, const CamDev& cam,
                                            float* __restrict__ gbuf, int tx, int ty) {
  const int x0 = tx + (gid % GX) * SW, y0 = ty + (gid / GX) * SH;
  if (g.c < PSTRIP) {
    const int x = x0 + g.c % SW, y = y0 + g.c / SW;
    float3 d = f3(0.f, 0.f, 0.f);
    if (x < cam.W && y < cam.H) d = camera_dir(cam, y * cam.W + x);
    dirs[g.c] = make_float4(d.x, d.y, d.z, 0.0f);
  }
  __syncwarp(g.mask);
  for (int j = 0; j < PSTRIP; ++j) {
    const int x = x0 + j % SW, y = y0 + j / SW;
    if (x >= cam.W || y >= cam.H) continue;  // uniform over the group
    const float4 d = dirs[j];
    trace_pixel<Cnt>(g, st, insts, n_inst, P, env, status, counters, cam, gbuf, x, y, f3(d.x, d.y, d.z));
  }
}

__device__ __forceinline__ float4* strip_dirs(int* smem, int gid) {
  return reinterpret_cast<float4*>(reinterpret_cast<unsigned char*>(smem) + RGROUPS * CRAY_SMEM) + gid * PSTRIP;
}

template <class Cnt>
__global__ void __launch_bounds__(TB, PRIMARY_MIN_BLOCKS) k_trace_primary(TraceArgs a, CamDev cam, float* __restrict__ gbuf) {
  extern __shared__ __align__(16) int s_cstack[];
  const Grp g = make_grp();
  const int gid = threadIdx.x / WIDE;
  const CStack st = ray_smem(reinterpret_cast<unsigned char*>(s_cstack), RGROUPS, gid);
  trace_strip<Cnt>(g, gid, st, strip_dirs(s_cstack, gid), a.insts, a.n_inst, a.P, a.env, a.status, a.counters, cam,
                   gbuf, blockIdx.x * TILE_W, blockIdx.y * TILE_H);
}

// Primary rays of several images in one launch (the served loop's launch
// group): block b belongs to the job whose tile range holds it.
__global__ void __launch_bounds__(TB, PRIMARY_MIN_BLOCKS) k_trace_primary_batch(PrimaryBatch B, DevParams P, int* status) {
  extern __shared__ __align__(16) int s_cstack[];
  const Grp g = make_grp();
  const int gid = threadIdx.x / WIDE;
  const CStack st = ray_smem(reinterpret_cast<unsigned char*>(s_cstack), RGROUPS, gid);
  int lo = 0, hi = B.n_jobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (B.jobs[mid].tile0 <= (int)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const PrimaryJob& J = B.jobs[lo];
  const int tile = (int)blockIdx.x - J.tile0;
  const int tiles_x = (J.cam.W + TILE_W - 1) / TILE_W;
  trace_strip<NoCounters>(g, gid, st, strip_dirs(s_cstack, gid), J.insts, J.n_inst, P, J.env, status, nullptr,
                          J.cam, J.gbuf, (tile % tiles_x) * TILE_W, (tile / tiles_x) * TILE_H);
}

int primary_tiles(int W, int H) { return ((W + TILE_W - 1) / TILE_W) * ((H + TILE_H - 1) / TILE_H); }

cudaError_t launch_trace_primary_batch(PrimaryBatch& B, const DevParams& P, int* status, cudaStream_t st) {
  int tiles = 0;
  for (int q = 0; q < B.n_jobs; ++q) {
    B.jobs[q].tile0 = tiles;
    tiles += primary_tiles(B.jobs[q].cam.W, B.jobs[q].cam.H);
  }
  if (tiles > 0) k_trace_primary_batch<<<tiles, TB, RSTACK_SMEM, st>>>(B, P, status);
  return cudaGetLastError();
}

cudaError_t launch_trace_primary(const TraceArgs& a, const CamDev& cam, float* gbuf, cudaStream_t st) {
  dim3 grid((cam.W + TILE_W - 1) / TILE_W, (cam.H + TILE_H - 1) / TILE_H);
  if (a.counters) k_trace_primary<Counters><<<grid, TB, RSTACK_SMEM, st>>>(a, cam, gbuf);
  else k_trace_primary<NoCounters><<<grid, TB, RSTACK_SMEM, st>>>(a, cam, gbuf);
  return cudaGetLastError();
}

}  // namespace lf
