/*
 * lightfuse.h - C ABI of the B300 (sm_103a) surfel ray tracer.
 *
 * Differentiable ray tracing of 2D Gaussian surfels (Eq. 1) with one-bounce
 * physically based shading under an environment map (Eq. 10-11), for scenes
 * assembled from a shared background plus rigidly movable objects (Eq. 2).
 *
 * Conventions shared by every call
 *   - Pointers named *_dev are CUDA device pointers owned by the caller; they
 *     must stay valid for as long as the context uses them (the scene arrays
 *     until the next lf_bvh_build or lf_destroy, an environment map until it
 *     is replaced).  Other pointers are host pointers, read during the call.
 *   - All work is enqueued asynchronously on the context's CUDA stream; no
 *     call synchronises except lf_sync, lf_bvh_build (it reads object
 *     offsets and sizes) and the serving calls that say so.
 *   - Render calls allocate nothing.  lf_bvh_build and lf_env_set allocate
 *     library-owned device storage (BVH nodes, packed records, sampling
 *     tables) when the scene or map grows.
 *   - Errors are returned as lf_status; the library never aborts, traps or
 *     exits.  Kernels report device-side conditions (traversal stack
 *     overflow, round limit; in a build compiled with LF_CHECKED=1 also a
 *     failed bounds check, LF_ERR_BOUNDS) through a device status word that
 *     lf_sync returns.  lf_last_error gives a human-readable message.
 *   - Floating point data are FP32.  Gradients are ACCUMULATED (+=) into the
 *     caller's buffers; the caller zeroes them.
 *   - Limits: at most LF_MAX_OBJECTS objects (background included), at most
 *     2^24 surfels per object and 2^24 surfels in total (surfel ids and hit
 *     counts are stored exactly in FP32 G-buffer channels).
 */
#ifndef LIGHTFUSE_H
#define LIGHTFUSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LF_MAX_OBJECTS 64
#define LF_MAX_ENVS 16     /* environment map slots                              */
#define LF_KBUF 32         /* hits per k-buffer round = children per wide BVH node = lanes per ray */
#define LF_STACK_DEPTH 128 /* traversal stack entries per ray (shared memory)                    */

typedef enum {
  LF_OK = 0,
  LF_ERR_INVALID = 1,     /* bad argument; nothing was enqueued              */
  LF_ERR_OOM = 2,         /* device allocation failed / over memory budget   */
  LF_ERR_CUDA = 3,        /* a CUDA runtime call failed                      */
  LF_ERR_STACK = 4,       /* a traversal stack overflowed (device status)    */
  LF_ERR_ROUND_LIMIT = 5, /* a ray needed more than max_rounds k-buffer rounds */
  LF_ERR_TIMEOUT = 6,     /* a wait ran out of time                          */
  LF_ERR_BUSY = 7,        /* no free slot (serving)                          */
  LF_ERR_NOT_BUILT = 8,   /* render before lf_bvh_build / lf_env_set         */
  LF_ERR_BOUNDS = 9,      /* a device bounds check failed (LF_CHECKED builds) */
  LF_ERR_CANCELLED = 10   /* a served request was cancelled before admission */
} lf_status;

/*
 * Method constants.  The paper fixes only the 0.99 opacity cap (Sec. 3.2,
 * Eq. 6); the others are readings of what it leaves open.
 */
typedef struct {
  float T_min;       /* compositing stops after the hit whose T falls below  */
  float alpha_min;   /* Eq. 6: hits with alpha~ below this are discarded     */
  float alpha_max;   /* Eq. 6: alpha~ = min(alpha_max, o exp(-|xi|^2/2))     */
  float support_r2;  /* Eq. 6: finite support u^2 + v^2 <= support_r2        */
  float eps_w;       /* Eq. 7: z = sum w z / (sum w + eps_w)                 */
  float t_min;       /* hits need t > t_min                                  */
  float ray_offset;  /* secondary rays start at x + ray_offset * n           */
  float p_spec;      /* Eq. 11: probability of the GGX lobe in the mixture   */
  int max_rounds;    /* k-buffer rounds per ray before LF_ERR_ROUND_LIMIT    */
  int brdf_mode;     /* 0 Lambert + GGX metallic-roughness, 1 Lambert a/pi   */
  int sampling_mode; /* 0 MIS (NEE + BSDF), 1 BSDF only, 2 NEE only          */
  int sampler;       /* 0 Philox4x32-10 uniforms; 1 Sobol points (Joe-Kuo     */
                     /* direction numbers) with a per-pixel Philox rotation   */
} lf_params;

/* Scene: caller-owned FP32 device arrays, surfel i at index i.  Object k
 * owns the contiguous surfels [object_offsets[k], object_offsets[k+1]);
 * object 0 is the background.  Eq. 1: centre mu, tangent axes tu, tv (the
 * surfel normal is tu x tv), in-plane scales (s_u, s_v), opacity o, base
 * colour a, metallic m, roughness r. */
typedef struct {
  float* mu_dev;        /* N x 3 */
  float* tu_dev;        /* N x 3 */
  float* tv_dev;        /* N x 3 */
  float* scale_dev;     /* N x 2 */
  float* opacity_dev;   /* N     */
  float* albedo_dev;    /* N x 3 */
  float* metallic_dev;  /* N     */
  float* roughness_dev; /* N     */
  int n;
  const int* object_offsets; /* host, n_objects + 1 entries, offsets[0] = 0, offsets[n_objects] = n */
  int n_objects;
} lf_scene;

/* Pinhole camera: pixel (x, y) looks through its centre; fovy is vertical. */
typedef struct {
  float eye[3], target[3], up[3];
  float fovy_deg;
  int width, height;
} lf_camera;

/* G-buffer written by lf_trace_primary: LF_GBUF_CHANNELS planes of P = W*H
 * floats, channel c of pixel p at gbuf[c * P + p] (p = y * width + x). */
enum {
  LF_CH_T = 0,       /* final transmittance T                         */
  LF_CH_W = 1,       /* sum of weights (= 1 - T)                      */
  LF_CH_DEPTH = 2,   /* composited ray distance                       */
  LF_CH_X = 3,       /* composited position (3)                       */
  LF_CH_N = 6,       /* composited, renormalised normal (3)           */
  LF_CH_A = 9,       /* composited base colour (3)                    */
  LF_CH_M = 12,      /* composited metallic                           */
  LF_CH_R = 13,      /* composited roughness                          */
  LF_CH_RHO = 14,    /* unlit radiance sum w a + T E(d) (3)           */
  LF_CH_NLEN = 17,   /* length of the normal before renormalising     */
  LF_CH_HITS = 18,   /* number of composited hits                     */
  LF_CH_TSTOP = 19,  /* ray distance of the last composited hit       */
                     /* (with LF_CH_STOPKEY_LO: its 64-bit sort key)  */
  LF_CH_IDSTOP = 20, /* surfel id of the last composited hit (-1: none) */
  LF_CH_DIR = 21,    /* primary ray direction (3)                     */
  LF_CH_STOPKEY_LO = 24, /* raw bits: low word of the stop hit's sort key */
  LF_CH_X_LO = 25,   /* residual of the position below its FP32 value (3) */
  LF_CH_N_LO = 28,   /* residual of the normal (3)                    */
  LF_CH_R_LO = 31,   /* residual of the roughness                     */
                     /* (x + x_lo etc.: the composite to ~1e-14; shading */
                     /* rays start from and sample around these pairs) */
  LF_GBUF_CHANNELS = 32,
  LF_GBUF_DIFF = 17  /* channels 0..16 accept an upstream gradient    */
};

/* Per-surfel gradient layout: 17 floats per surfel. */
enum { LF_G_MU = 0, LF_G_TU = 3, LF_G_TV = 6, LF_G_S = 9, LF_G_O = 11, LF_G_A = 12, LF_G_M = 15, LF_G_R = 16,
       LF_G_STRIDE = 17 };

typedef struct lf_ctx lf_ctx;

/* Defaults: T_min 1e-4, alpha_min 1/255, alpha_max 0.99, support_r2 9,
 * eps_w 1e-8, t_min 1e-4, ray_offset 1e-3, p_spec 0.5, max_rounds 64, sampler 0. */
lf_status lf_params_default(lf_params* out);

/* Create a context bound to the current CUDA device and `stream` (a
 * cudaStream_t; NULL = legacy default stream).  Allocates the device status
 * word.  *out is set only on LF_OK. */
lf_status lf_create(const lf_params* params, void* stream, lf_ctx** out);
lf_status lf_destroy(lf_ctx* ctx);
lf_status lf_set_stream(lf_ctx* ctx, void* stream);
const char* lf_last_error(const lf_ctx* ctx);

/* Wait for the context's stream, then read and clear the device status word. */
lf_status lf_sync(lf_ctx* ctx);

/*
 * Build the two-level acceleration structure (Eq. 2 assembly: one BLAS per
 * object, background included, under a flat TLAS of object boxes).  Per
 * object: surfel AABBs at the support radius, 30-bit Morton codes of their
 * centres in the object's bounds, an LSD radix sort, Karras hierarchy
 * (duplicate codes ordered by index), bottom-up box fit.  Packs the surfel
 * records the traversal reads.  Keeps the scene pointers.  Synchronises.
 */
lf_status lf_bvh_build(lf_ctx* ctx, const lf_scene* scene);

/*
 * Rigid object rearrangement (Eq. 2: T = (R, t) acts on centres and
 * orientations only).  Applies mu <- R mu + t, tu <- R tu, tv <- R tv IN
 * PLACE to object `object_id`'s surfels in the caller's arrays, repacks
 * them, refits that object's BLAS (topology kept) and updates the TLAS.
 * R is row-major 3x3 (host), t is 3 floats (host).
 */
lf_status lf_bvh_refit(lf_ctx* ctx, int object_id, const float R[9], const float t[3]);

/* After the caller changed any surfel attribute of object `object_id`
 * (-1: all objects) in place: repack its records and refit its BLAS. */
lf_status lf_scene_sync(lf_ctx* ctx, int object_id);

/* Material edit (Sec. 3.4.2): overwrite object `object_id`'s base colour
 * (rgb != NULL), metallic (>= 0) and/or roughness (>= 0) in the caller's
 * arrays and repack. */
lf_status lf_material_set(lf_ctx* ctx, int object_id, const float* rgb, float metallic, float roughness);

/*
 * Cross-state supervision (Sec. 3.2, "Cross-state supervision"; Eq. 2).  A
 * single canonical scene holds the shared parameters; observed state k is
 * S_k = B u T_{k,1}(O_1) u ... u T_{k,M}(O_M): the background (object 0) as
 * it is and object o = 1..M moved by the rigid transform
 * T_{k,o} = (R_{k,o}, t_{k,o}), which acts only on the surfel centres and
 * tangent axes (mu = R mu^c + t, tu = R tu^c, tv = R tv^c).
 *
 * lf_state_assemble writes state k's mu, tu, tv into the scene the context
 * was built on (each component in FP64 with exact products, one rounding, as
 * lf_bvh_refit), copies scale, opacity and materials from `canonical` where
 * its arrays are not the built scene's own (they may be shared), and refits
 * every BLAS and the TLAS on the build's topology.  `canonical` is a
 * caller-owned device scene with the built scene's n and object_offsets; its
 * mu, tu, tv must not be the built scene's arrays.  R: host, (n_objects - 1)
 * row-major 3x3 rotations for objects 1..M; t: host, (n_objects - 1) x 3.
 * Errors: LF_ERR_NOT_BUILT before lf_bvh_build; LF_ERR_INVALID for a
 * mismatched scene, aliased geometry arrays or a transform that is not
 * rigid (nothing is enqueued then).
 *
 * lf_state_pullback is its adjoint, so that the residuals of every state
 * update the same canonical surfels: d_canonical += J^T d_world over the
 * LF_G_* layout (N x 17 FP32, device, caller-owned, must not overlap).  For
 * a surfel of object o >= 1 the mu, tu and tv triples g add R^T g (FP64,
 * one rounding, then an FP32 add); every other entry, and all of the
 * background's, adds unchanged.  R as above (t does not enter).
 */
lf_status lf_state_assemble(lf_ctx* ctx, const lf_scene* canonical, const float* R, const float* t);
lf_status lf_state_pullback(lf_ctx* ctx, const float* R, const float* d_world, float* d_canonical);

/*
 * Register environment map `env_id` (0 <= env_id < LF_MAX_ENVS): H x W x 3 FP32
 * texels, row 0 looking up (+y), column 0 at phi = 0 of the y-up
 * equirectangular mapping theta = acos(w_y), phi = atan2(w_x, -w_z) + pi.
 * Builds the importance-sampling tables (texel weight = (Rec.709 luminance
 * + 1e-6) * sin(theta at the row centre), FP64 sums, FP32 tables plus the
 * FP32 residuals of the FP64 CDF values, so a sample's position inside its
 * texel carries the FP64 table's accuracy).  The texels are read in place
 * at render time.
 */
lf_status lf_env_set(lf_ctx* ctx, int env_id, const float* rgb_dev, int H, int W);

/*
 * Primary rays (Eq. 6-7): per pixel, rounds of "collect the LF_KBUF nearest
 * accepted hits with key (t, id) beyond the last round's key", composited
 * front to back until T < T_min.  Writes the G-buffer (see LF_CH_*); the
 * radiance channel uses environment `env_id` for T E(d).
 * gbuf_dev: LF_GBUF_CHANNELS * width * height floats.
 */
lf_status lf_trace_primary(lf_ctx* ctx, const lf_camera* cam, int env_id, float* gbuf_dev);

/*
 * One-bounce shading (Eq. 11, Sec. 4.2 path budget): per pixel and sample,
 * Philox4x32-10 uniforms keyed by `seed` with counter (pixel, sample, group,
 * 0); one environment NEE sample with a shadow ray, one BSDF continuation
 * from the cosine/GGX mixture traced to a secondary record, two environment
 * NEE samples with shadow rays there; power-heuristic MIS.
 * rgb_dev[p*3 + c] = T E(d) + (1 - T) / spp * sum_s (NEE + BSDF terms),
 * the sum taken in sample order.
 * samples_dev: caller scratch of at least lf_shade_scratch_bytes(width,
 * height, spp) bytes; on return it holds the per-sample data path replay
 * keeps fixed (directions, pdfs, MIS weights, visibilities, secondary
 * factors), which lf_trace_backward can reuse.
 * ray_count_dev (nullable): a device uint64 the call ADDS the number of
 * shading rays it traced to.
 */
size_t lf_shade_scratch_bytes(int width, int height, int spp);
lf_status lf_shade_bounce(lf_ctx* ctx, const lf_camera* cam, const float* gbuf_dev, int env_id, int spp,
                          uint64_t seed, float* rgb_dev, unsigned long long* ray_count_dev, void* samples_dev,
                          size_t samples_bytes);

/*
 * Allocation-free variant of lf_shade_bounce.  The paper has no counterpart:
 * this is a convenience of the library.  It is for callers that cannot
 * allocate device memory (a host whose device memory is owned by another
 * allocator, a plugin that may not call cudaMalloc, a loop that must not
 * allocate after start-up): instead of a caller buffer, the per-sample
 * scratch is a fixed array of LF_STATIC_SCRATCH_BYTES inside the library,
 * which every GPU that loads the library holds until the process exits.
 * Same arguments and results as lf_shade_bounce without the sample buffer.
 *   - width * height * spp must be at most (LF_STATIC_SCRATCH_BYTES - 256) /
 *     140 = 479,347 samples (lf_shade_scratch_bytes gives the bytes a count
 *     needs); larger requests return LF_ERR_INVALID with a message and
 *     enqueue nothing.
 *   - The calling thread's current device must be the context's device
 *     (LF_ERR_INVALID otherwise).  The first call after a context was
 *     created on a device looks up the array's device address there (with
 *     that device current); make that first call before any stream capture.
 *     A cudaDeviceReset ends the contexts made before it; the next lf_create
 *     on the device makes the following call look the address up again.
 *   - All calls share the array, which keeps the last call's contents; each
 *     call clears the counters that must start at zero.  Calls whose work
 *     overlaps on the GPU (other streams, contexts or threads) race on it.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine.
 */
#define LF_STATIC_SCRATCH_BYTES (64u << 20)
lf_status lf_shade_bounce_static(lf_ctx* ctx, const lf_camera* cam, const float* gbuf_dev, int env_id, int spp,
                                 uint64_t seed, float* rgb_dev, unsigned long long* ray_count_dev);

/*
 * The per-sample terms of Eq. 11 behind an lf_shade_bounce result (an
 * inspection call): terms_dev[(p * spp + s) * 3 + c] = c_s, the NEE plus BSDF
 * term of sample s of pixel p evaluated from the G-buffer and the sample
 * buffer `samples_dev` of the lf_shade_bounce call with the same camera,
 * G-buffer, environment and spp, so that
 * rgb = T E(d) + (1 - T) / spp * sum_s c_s up to the order of the sum.
 * Zero for pixels without a surface facing the camera.  terms_dev: device,
 * width * height * spp * 3 floats.
 */
lf_status lf_shade_sample_terms(lf_ctx* ctx, const lf_camera* cam, const float* gbuf_dev, int env_id, int spp,
                                const void* samples_dev, size_t samples_bytes, float* terms_dev);

/* Scratch bytes lf_trace_backward needs for a width x height image at spp
 * samples when it has to replay the shading (fwd_samples == NULL); with the
 * forward's sample buffer it needs 9 * width * height floats (+256 B). */
size_t lf_backward_scratch_bytes(int width, int height, int spp);

/*
 * Adjoint of lf_trace_primary + lf_shade_bounce under path replay (Sec. 3.3):
 * the sampled directions, pdfs, MIS weights, visibilities and secondary
 * records stay fixed; gradients flow through the primary record and every
 * environment lookup.  The primary pass re-traverses each ray back to front
 * from the stored final transmittance and stop key (no per-ray hit lists),
 * recovering T_j = T_{j+1} / (1 - alpha_j), and scatters the Eq. 6-7
 * adjoint to the surfels.
 *   gbuf_dev:     the G-buffer of the forward pass (unchanged scene).
 *   dL_drgb_dev:  P x 3 (nullable: no shading term).
 *   dL_dgbuf_dev: LF_GBUF_CHANNELS planes (nullable); channels
 *                 0..LF_GBUF_DIFF-1 are used.
 *   d_surfel_dev: N x 17 (LF_G_* layout), accumulated.
 *   d_env_dev:    H x W x 3 of `env_id`, accumulated (nullable).
 *   fwd_samples_dev: the sample buffer of the lf_shade_bounce call with the
 *                 same camera, environment, spp, seed and scene (nullable:
 *                 the shading samples are then replayed into scratch).
 *   scratch_dev:  lf_backward_scratch_bytes(...) bytes (see above).
 */
lf_status lf_trace_backward(lf_ctx* ctx, const lf_camera* cam, const float* gbuf_dev, int env_id, int spp,
                            uint64_t seed, const float* dL_drgb_dev, const float* dL_dgbuf_dev,
                            float* d_surfel_dev, float* d_env_dev, const void* fwd_samples_dev, void* scratch_dev,
                            size_t scratch_bytes);

/*
 * Traversal counters for roofline accounting: when counters_dev (20 x uint64
 * on the device) is non-NULL, the trace kernels ADD, per kernel slot k
 * (0 primary rays, 1 NEE shadow rays, 2 continuation rays, 3 secondary
 * shadow rays, 4 adjoint re-traversal), [node visits, surfel tests,
 * composited hits (slot 4: hits whose gradient is scattered), rays (slot 4:
 * pixels with a hit)] to counters_dev[4k .. 4k+3].  NULL turns counting off.
 */
lf_status lf_set_counters(lf_ctx* ctx, unsigned long long* counters_dev);

/*
 * Per-kernel timing with CUDA events on the context's stream: while enabled,
 * lf_trace_primary and lf_shade_bounce record events around their kernels;
 * lf_profile_read waits for them and returns the milliseconds of the last
 * calls' kernels: [primary, sample generation, NEE shadow rays, continuation
 * rays, secondary shadow rays, combine, shading adjoint (with the replayed
 * wavefront when no forward sample buffer is given), adjoint re-traversal];
 * the last two are 0 until a profiled lf_trace_backward has run.
 */
lf_status lf_profile(lf_ctx* ctx, int enable);
lf_status lf_profile_read(lf_ctx* ctx, float* ms8);

/*
 * Geometry-refinement losses of one view on a traced G-buffer (Eq. 8-9):
 *   L_D  = ||C (D - D*)||_1 / (||C D*||_1 + eps)   depth, confidence-weighted
 *   L_N  = 1 - <N, N*>_F / (W H)                    rendered normals
 *   L_DN = 1 - <N^D, N*>_F / (W H)                  depth-derived normals
 * D and N are the G-buffer's depth (ray distance) and renormalised normal
 * planes; N^D(x, y) = normalize(P_x x P_y) from central differences of the
 * back-projected positions P = eye + D d along the G-buffer's ray directions,
 * P_x = P(x+1, y) - P(x-1, y), P_y = P(x, y-1) - P(x, y+1); it is 0 on the
 * image border and where the pixel or a 4-neighbour has no composited hit.
 * depth_ref, depth_conf: W*H device floats; normal_ref: 3 planes of W*H.
 * weights (host, 3, NULL = ones) weight the terms in the gradient, which is
 * ADDED to the depth and normal planes of dL_dgbuf (device, the G-buffer
 * layout; NULL: losses only) and can then be passed to lf_trace_backward.
 * scratch: device, 256-byte aligned, lf_geometry_loss_scratch_bytes().
 * losses (host, 3: L_D, L_N, L_DN, unweighted) may be NULL; when given, the
 * call synchronises the context's stream.
 */
size_t lf_geometry_loss_scratch_bytes(int width, int height);
lf_status lf_geometry_loss(lf_ctx* ctx, const lf_camera* cam, const float* gbuf_dev, const float* depth_ref_dev,
                           const float* depth_conf_dev, const float* normal_ref_dev, float eps,
                           const float* weights_host, float* dL_dgbuf_dev, void* scratch_dev, size_t scratch_bytes,
                           double* losses_host);

/*
 * Regularisers of the training objectives.  Each ADDS weight * gradient to
 * the caller's device buffer (NULL: loss only) and, when `loss` (host) is
 * given, returns the unweighted value after synchronising the stream.
 *  lf_opacity_loss  L_alpha = ||A - 1||_1 / (W H) (Eq. 4) with A the traced
 *                   weight sum (G-buffer plane LF_CH_W); gradient into that
 *                   plane of dL_dgbuf (the G-buffer layout).
 *  lf_scale_loss    L_s = (1/N) sum_i max(0, max(s_u, s_v)_i / s_max - 1)^2
 *                   (Eq. 5) over `scale` (device, N x 2); gradient into the
 *                   scale columns of d_surfel (N x LF_G_STRIDE); a tie of the
 *                   two scales splits it evenly.
 *  lf_env_tv_loss   L_TV(E) = (1 / (3 H W)) sum |E(r,c+1) - E(r,c)| +
 *                   |E(r+1,c) - E(r,c)| (Eq. 14, anisotropic L1; wraps in
 *                   azimuth, not across the poles) of `rgb` (device H x W x 3);
 *                   gradient into d_env (H x W x 3).
 */
lf_status lf_opacity_loss(lf_ctx* ctx, const lf_camera* cam, const float* gbuf_dev, float weight,
                          float* dL_dgbuf_dev, double* loss_host);
lf_status lf_scale_loss(lf_ctx* ctx, const float* scale_dev, int n, float s_max, float weight, float* d_surfel_dev,
                        double* loss_host);
lf_status lf_env_tv_loss(lf_ctx* ctx, const float* rgb_dev, int H, int W, float weight, float* d_env_dev,
                         double* loss_host);

/*
 * Measurement helper (no counterpart in the paper): read bandwidth of the L2
 * cache in GB/s, from `reps` passes of float4 loads cached at L2 only over a
 * device buffer of `bytes` (at least 1 MiB; keep it well below the L2 size),
 * after one warm-up pass.  Allocates and frees its own buffer; synchronises
 * the context's stream.
 */
lf_status lf_measure_l2_read(lf_ctx* ctx, size_t bytes, int reps, float* gbs);

/* Philox4x32-10 of n counters (device n x 4 words) with key (k0, k1). */
lf_status lf_philox(lf_ctx* ctx, const uint32_t* ctr_dev, int n, uint32_t k0, uint32_t k1, uint32_t* out_dev);

/* Copy the sampling tables of `env_id` (device FP32: H, H, H*W, H*W). */
lf_status lf_env_tables(lf_ctx* ctx, int env_id, float* pmf_row_dev, float* cdf_row_dev, float* pmf_col_dev,
                        float* cdf_col_dev);

/* BVH inspection: number of internal nodes of object k, and a host copy of
 * its nodes (16 floats each: child boxes and child codes, see the build). */
lf_status lf_bvh_info(lf_ctx* ctx, int object_id, int* n_internal, int* root_code);
lf_status lf_bvh_copy_nodes(lf_ctx* ctx, int object_id, float* host_out, size_t bytes);
/* Wide BVH inspection: host copy of object k's wide nodes, decoded
 * (capacity *cap_nodes nodes; a node is *wide quads (lo.xyz, child code as
 * int bits) followed by *wide quads (hi.xyz, leaf surfel count as int bits),
 * one pair per child slot; compressed boxes are decoded rounding outward, so
 * each contains the box the traversal tests), and its root (code >= 0 wide node, < 0 leaf of
 * *root_count surfels from leaf ~code, INT_MIN empty).  host_out may be NULL
 * to query the sizes only. */
lf_status lf_bvh_copy_wide(lf_ctx* ctx, int object_id, float* host_out, size_t bytes, int* cap_nodes, int* root_code,
                           int* root_count, int* wide);
/* Bytes one wide node occupies on the device (the traversal reads all of them
 * per node visit): a 16-byte header plus 16 bytes per child slot (FP16 boxes
 * relative to the node centre), or 32 bytes per slot in the FP32 build. */
int lf_bvh_wide_node_bytes(void);

/* ---------------------------------------------------------------- serving
 *
 * The editing and relighting stage of the method (Sec. 3.4.2) served as a
 * request loop.  The paper's edits are a target rigid transform of an
 * object (Eq. 2: T = (R, t) on its surfel centres and orientations), a
 * change of base colour, metallic or roughness, and a recovered or
 * user-provided environment map; each edited state is then re-traced and
 * shaded (Eq. 6-7, Eq. 11).  The loop itself (admission, batching, latency)
 * has no counterpart in the paper.
 *
 * A request is one edit plus one camera.  Edits are applied to the served
 * scene in submission order, each creating a new version of the edited
 * object (copy on write), so a request renders exactly the scene state
 * after its own edit, even while later requests are already editing.
 * Admission: a request is admitted when a slot is free and its frame and
 * object version fit under the memory budget; admitted requests are
 * batched into shared kernel launches (one primary-ray launch and one
 * shading wavefront carry the work of every request of a launch group) on
 * a pool of streams, so their work overlaps on the device.
 */
typedef enum { LF_EDIT_NONE = 0, LF_EDIT_MOVE = 1, LF_EDIT_MATERIAL = 2, LF_EDIT_ENV = 3 } lf_edit_kind;

/* One edit of Sec. 3.4.2.  MOVE is Eq. 2's rigid transform (as
 * lf_bvh_refit), MATERIAL the base-colour / metallic / roughness edit (as
 * lf_material_set), ENV the switch to another registered environment map
 * (the recovered or user-provided lighting of the relit state). */
typedef struct {
  int kind;          /* lf_edit_kind */
  int object_id;     /* MOVE / MATERIAL */
  float R[9], t[3];  /* MOVE: x -> R x + t applied to the object's current pose */
  float albedo[3];   /* MATERIAL: new base colour (if set_albedo) */
  float metallic, roughness; /* MATERIAL: new values when >= 0 */
  int set_albedo;
  int env_id;        /* ENV: environment used from this request on */
} lf_edit;

typedef struct {
  lf_edit edit;
  lf_camera cam;
  int spp;
  uint64_t seed;
} lf_request;

typedef struct {
  double t_submit, t_admit, t_start, t_done; /* seconds, steady clock */
  unsigned long long rays;
} lf_timing;

typedef struct lf_serve lf_serve;

/* Create a server over the context's built scene and environments (the
 * context's scene must not be modified while the server runs).
 * mem_budget_bytes bounds the device memory of in-flight requests (frame,
 * G-buffer, per-sample buffer) and of live object versions; max_slots bounds
 * the requests in flight; n_streams is the stream pool the launch groups
 * rotate over; batch_window_us is how long the oldest pending request may
 * wait for others to join its launch group while slots are free (0: admit
 * at once).  Frames are at most 1024 x 1024.
 * Each finished request keeps its pinned host frame until lf_serve_poll
 * returns it; the server owns 2 * max_slots frames, so a client must poll
 * finished requests for admission to go on (waiting on a later ticket while
 * 2 * max_slots finished ones stay unpolled ends in LF_ERR_TIMEOUT). */
lf_status lf_serve_create(lf_ctx* ctx, size_t mem_budget_bytes, int max_slots, int n_streams, int batch_window_us,
                          lf_serve** out);
/* Enqueue a request (host copy); returns its ticket.  Never blocks.  The
 * frame is the one-bounce render (Eq. 6-7, Eq. 11) of the scene state after
 * the request's own edit: LF_ERR_INVALID (nothing enqueued) for an unknown
 * object or environment, a MOVE that is not rigid, or a camera beyond
 * 1024 x 1024. */
lf_status lf_serve_submit(lf_serve* srv, const lf_request* req, uint64_t* ticket);
/* done = 1 when finished; then frame_host (width*height*3 floats, may be
 * NULL) receives the image and timing (may be NULL) the timestamps. */
lf_status lf_serve_poll(lf_serve* srv, uint64_t ticket, int* done, float* frame_host, size_t frame_floats,
                        lf_timing* timing);
/* Block until the ticket is done or timeout_ms passes (LF_ERR_TIMEOUT). */
lf_status lf_serve_wait(lf_serve* srv, uint64_t ticket, int timeout_ms);
/* Withdraw a request that has not been admitted yet: LF_OK, and the ticket
 * is done with status LF_ERR_CANCELLED (lf_serve_poll returns it and frees
 * the ticket; no frame).  A request already admitted runs to the end and
 * LF_ERR_BUSY is returned (poll it as usual); an unknown ticket gives
 * LF_ERR_INVALID.  Nothing on the GPU is interrupted. */
lf_status lf_serve_cancel(lf_serve* srv, uint64_t ticket);
lf_status lf_serve_destroy(lf_serve* srv);

#ifdef __cplusplus
}
#endif
#endif /* LIGHTFUSE_H */
