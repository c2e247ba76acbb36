// Wavefront shading: batch description and per-sample buffer layout.
#pragma once
#include "lf_kernels.h"

namespace lf {

constexpr int MAX_JOBS = 32;
constexpr int SAMPLE_PLANES = 31;

// One image of a shading batch: its scene snapshot (instances), environment,
// G-buffer (planes of n_pix floats), output and sampling parameters.  Its
// items are [item0, item0 + n_pix * spp) and its pixels [pix0, pix0 + n_pix)
// in the batch-wide numbering.
struct ShadeJob {
  const Inst* insts;
  int n_inst;
  EnvDev env;
  const float* gbuf;
  int n_pix;
  float* rgb;
  int spp;
  uint32_t k0, k1;
  long long item0;
  int pix0;
};

struct ShadeBatch {
  int n_jobs;
  long long n_items;
  int n_pix_total;
  ShadeJob jobs[MAX_JOBS];
};

// Per-sample planes (n_items floats each) and ray queues.
struct SampleBuf {
  float* we[3];
  float* ek;   // MIS weight / pdf of the NEE sample; 0: no NEE ray
  float* Ve;
  float* wi[3];
  float* bc;   // 1 / pdf of the continuation; 0: no continuation ray
  float* wb;   // MIS weight of the escaped continuation
  float* T2;
  float* xs2[3];    // origin of the secondary NEE rays, high part
  float* xs2lo[3];  // and its low part (double-float)
  float* wq0[3];
  float* wq1[3];
  float* fk0[3];  // f2 cos / pdf * (1 - T2) / 2 of secondary NEE #1; 0: none
  float* fk1[3];
  float* Vq0;
  float* Vq1;
  int* qA;
  int* qB;
  int* qC;
  int* counts;  // queue lengths A, B, C
};

size_t sample_buf_bytes(long long n_items);
SampleBuf sample_buf(void* base, long long n_items);
cudaError_t launch_shade_wavefront(const ShadeBatch& B, const DevParams& P, const SampleBuf& S, int* status,
                                   unsigned long long* ray_count, unsigned long long* counters, int sms,
                                   cudaStream_t st, cudaEvent_t* ev = nullptr);
cudaError_t launch_shade_combine(const ShadeBatch& B, const DevParams& P, const SampleBuf& S, cudaStream_t st);
cudaError_t launch_shade_terms(const ShadeBatch& B, const DevParams& P, const SampleBuf& S, float* out, int sms,
                               cudaStream_t st);
cudaError_t launch_shade_combine_adjoint(const ShadeBatch& B, const DevParams& P, const SampleBuf& S,
                                         const float* dL_drgb, float* sg, float* d_env, cudaStream_t st);

}  // namespace lf
