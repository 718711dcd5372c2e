/*
 * usrt.h -- C ABI of the GB300 (sm_103a) differentiable Monte Carlo ultrasound ray tracer.
 *
 * The library implements the hot path of "Fully Differentiable Ultrasound Simulation Utilizing
 * Ray-Tracing" (arXiv 2604.15017): full-path Monte Carlo acoustic transport through a triangle
 * scene with point scatterers (Sec. 2.3.1-2.3.3), the pulse splat into per-element channel data
 * (Sec. 2.3.4, Eq. axial_sig), delay-and-sum beamforming (Eq. das), envelope detection and log
 * compression (Sec. 2.3.4), the l1/l2 image loss (Eq. weighted_l1_l2_loss) and the
 * fixed-sample vector-Jacobian product back to the continuous parameters (Sec. 3.2, Eq.
 * chain_rule; Eq. das_adjoint).  Every arithmetic step runs in the library's own CUDA kernels,
 * in FP32.
 *
 * Conventions shared by every call
 *   - Units: SI (m, s, Hz, kg/m^3).  Attenuation alpha in dB/cm/MHz.
 *   - Parameter vector theta (HOST, float[3*M+2]):
 *       [c_0, rho_0, alpha_0, c_1, rho_1, alpha_1, ..., c_{M-1}, rho_{M-1}, alpha_{M-1}, A_s, f0]
 *     M media (medium 0 holds the probe), scatterer amplitude scale A_s, centre frequency f0.
 *     A scene uploaded with rough != 0 takes M more entries, a GGX roughness per medium
 *     (float[4*M+2]); dL/dtheta then has the same length.
 *   - Probe: elements e = 0..n_elem-1 at x_e = (e - (n_elem-1)/2) * pitch, z = 0, normal +z,
 *     element face pitch x h_el.  Transmit tx uses plane-wave steering angle angles[tx].
 *   - Channel data rf: DEVICE float[n_tx][n_elem][n_samples], sample n at t = n / fs.
 *   - Images: DEVICE float[n_lines][n_depth] (depth contiguous); line l at
 *     x0 + l (x1-x0)/(n_lines-1), depth d at z0 + d (z1-z0)/(n_depth-1).
 *   - "*_dev" pointers are device memory owned by the caller; they must be 16-byte aligned.
 *     Host pointers are read during the call only.  The library owns scenes, path records and
 *     workspaces, all charged against the context's memory budget.
 *   - Calls enqueue work on the caller's CUDA stream (passed as void*, a cudaStream_t) and
 *     return without synchronising unless stated.  Scratch buffers grow on first use; make the
 *     first call of each shape outside CUDA-graph capture.
 *   - Every call returns a us_status (0 = success, < 0 = error).  No exception or abort
 *     crosses the ABI; us_last_error() describes the most recent failure of the context.
 *     Device-side faults are reported by status words, never by traps.
 */
#ifndef USRT_H
#define USRT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  US_OK = 0,
  US_ERR_ARG = -1,      /* invalid argument, size or alignment */
  US_ERR_OOM = -2,      /* allocation failed, or the memory budget refuses the request */
  US_ERR_CUDA = -3,     /* a CUDA runtime call failed */
  US_ERR_TIMEOUT = -4,  /* a bounded device wait gave up (reported through a status word) */
  US_ERR_OVERFLOW = -5, /* a fixed-capacity device list overflowed (secondary-ray crossings) */
  US_ERR_STATE = -6     /* call order: e.g. adjoint in record mode without a kept record */
} us_status;

typedef struct us_ctx us_ctx;

/* Scene: triangles with the media on their two sides, plus point scatterers. */
typedef struct {
  int32_t n_tris;
  const float* tris;     /* HOST, n_tris * 9: v0, v1, v2 (x, y, z) in metres */
  const int32_t* media;  /* HOST, n_tris * 2: (m_front, m_back); front = side the normal
                            (v1 - v0) x (v2 - v0) points to */
  int32_t n_media;       /* M, number of media referenced by theta (<= 32) */
  int32_t n_scat;
  const float* scat_pos; /* HOST, n_scat * 3 */
  const float* scat_amp; /* HOST, n_scat: per-scatterer amplitude s_j */
  float r_s;             /* scatterer radius: a primary ray interacts at its closest approach
                            when that lies within r_s of the centre */
  int32_t rough;         /* != 0: rough interfaces (Sec. 2.3.2, Eq. GGX_PDF).  theta then
                            carries, after A_s and f0, a GGX roughness alpha in [0, 1] per medium
                            (4M + 2 parameters, and dL/dtheta as many): a triangle's interface
                            takes the roughness of its back-side medium (the region it bounds);
                            alpha = 0 is the smooth interface */
} us_scene_desc;

/* Acquisition: probe, transmits, sampling and transport limits (Sec. 2.3.1-2.3.4). */
typedef struct {
  int32_t n_elem;        /* <= 256 */
  float pitch;           /* element pitch = element width (kerf 0) */
  float h_el;            /* element height (elevation) */
  int32_t n_tx;          /* <= 64 transmits */
  const float* angles;   /* HOST, n_tx steering angles [rad] */
  float fs;              /* sampling rate [Hz] */
  int32_t n_samples;     /* multiple of 4, <= 4096 */
  int32_t k_max;         /* maximum interactions per path (<= 15) */
  int32_t n_rays;        /* rays per emitting element and transmit */
  float bw;              /* -6 dB fractional bandwidth of the pulse */
  float alpha_m;         /* receive directivity main-lobe angle [rad] (Eq. cutoff) */
  float alpha_c;         /* receive directivity cutoff angle [rad] */
  float c_bf;            /* beamforming / steering-delay sound speed */
  int32_t split_mode;    /* 0: P_reflect = R^2 (Sec. 2.3.2); 1: fixed P_reflect = split_q */
  float split_q;
  uint32_t stream_id;    /* third Philox counter word (independent scenes / requests) */
  int32_t tx_elem;       /* -1: every element emits; else only this element (single-element
                            transmit), or the sub-aperture below */
  int32_t n_tx_elem;     /* with tx_elem >= 0: elements tx_elem .. tx_elem + n_tx_elem - 1 emit
                            (0 or 1: tx_elem alone); tx_elem + n_tx_elem <= n_elem.  A ray keeps
                            its index (element x n_rays + ray) whatever the sub-aperture, so
                            disjoint sub-apertures with one seed partition the full aperture's
                            realisation exactly (micro-batches over elements) */
  int32_t rough_nee;     /* != 0: secondary rays also at rough interface events (Sec. 2.3.3), the
                            microfacet BSDF evaluated toward the element; they and the primary's
                            own direct hits after such an event are combined by the balance
                            heuristic of multiple importance sampling (scenes with rough != 0) */
} us_acq_desc;

/* Image grid, dynamic range and loss weights. */
typedef struct {
  int32_t n_lines;
  int32_t n_depth;       /* power of two, 16..4096 (FFT envelope) */
  float x0, x1, z0, z1;
  float dr_db;           /* dynamic range: B = max(20 log10(E / E_max), -dr_db) */
  float lambda1, lambda2;/* loss weights (Eq. weighted_l1_l2_loss) */
  float f_number;        /* DAS element weights w_e(x, z) of Eq. das: <= 0 a Hann window over the
                            array; > 0 a dynamic receive aperture, the Hann window
                            cos^2(pi xi / 2), |xi| < 1, of xi = (x_e - x) / a with half-width
                            a = max(z / (2 f_number), pitch) */
} us_img_desc;

/* Transport statistics of the most recent us_forward / us_trace on a context. */
#define US_MAX_ROUNDS 17 /* segments per path: k_max <= 15, plus the last round's arrivals */
typedef struct {
  int64_t n_paths;
  int64_t segments;      /* primary closest-hit queries (one per path segment) */
  int64_t nee_queries;   /* secondary-ray all-crossings queries */
  int64_t arrivals;      /* arrivals splatted (transducer hits + secondary rays) */
  int64_t dropped;       /* arrivals dropped: crossing-list overflow */
  int32_t status;        /* device status word: 0, or a us_status raised on the device */
  int32_t pad;
  int64_t live[US_MAX_ROUNDS];  /* paths entering segment k (rounds past k_max + 1 hold 0) */
} us_stats;

/* ---------------------------------------------------------------------------------------- */
/* Context and scenes                                                                        */
/* ---------------------------------------------------------------------------------------- */

/* Create a context on CUDA device `device`.  mem_budget_bytes caps the library's own device
 * allocations (scenes, records, workspaces); 0 = no cap.  *out receives the context. */
int us_create(us_ctx** out, int device, size_t mem_budget_bytes);

/* Destroy a context: synchronises the device, frees every scene and workspace. */
void us_destroy(us_ctx* ctx);

/* Text of the most recent error on this context ("" if none).  Owned by the context. */
const char* us_last_error(us_ctx* ctx);

/* Upload a scene and build its BVH (binned SAH over triangles and scatterer spheres) on the
 * host; the BVH and primitive data stay resident on the device until released.
 * Synchronous.  *scene_id receives a handle (> 0). */
int us_scene_upload(us_ctx* ctx, const us_scene_desc* desc, uint64_t* scene_id);

/* Release a scene's device memory (synchronises the device first). */
int us_scene_release(us_ctx* ctx, uint64_t scene_id);

/* Bytes currently allocated by the context, and its budget. */
int us_memory(us_ctx* ctx, size_t* used, size_t* budget);

/* Context options. */
enum {
  /* DAS kernel: 0 (default) reads channel data through the read-only cache; 1 stages each
   * (element, transmit) window in shared memory with TMA bulk copies (cp.async.bulk +
   * mbarrier).  Both give the same image; which is faster depends on the shape. */
  US_OPT_DAS_TMA = 0,
  /* lanes (concurrent request pipelines, each with its own stream and workspaces) used by
   * us_forward_batch; default 4, at most 16 */
  US_OPT_LANES = 1,
  /* secondary rays on a second stream: 0 runs each round's secondary-ray kernel after that
   * round's primary rays on the call's stream; p in 1..100 (default 100) runs it on a second
   * stream of the lane (forked and joined with events, so the call stays one stream-ordered
   * unit), overlapping the next rounds' primary rays, with p % of its resident grid. */
  US_OPT_NEE_STREAM = 2,
  /* fault injection for tests of the timeout report (default 0): 1 makes the fused envelope
   * kernel's grid barrier wait for one arrival more than there are blocks, with a 1 ms limit,
   * so that the wait runs out: the image is written as NaN and us_get_status returns
   * US_ERR_TIMEOUT.  The fault is injected from the host (a kernel argument); nothing faults. */
  US_OPT_FAULT_BARRIER = 3,
  US_N_OPTS
};
int us_set_option(us_ctx* ctx, int option, int value);

/* Status of the context's kernels outside the transport (TMA-staged DAS waits, the fused
 * envelope kernel's grid barrier): synchronises the device, then *device_status = US_OK, or
 * US_ERR_TIMEOUT / US_ERR_OVERFLOW if any of them gave up since the last clear (their bounded
 * waits return instead of hanging).  clear != 0 resets the word.  The transport's own status
 * is reported by us_get_stats.  Returns US_ERR_ARG for a null argument, US_ERR_CUDA if the
 * synchronisation fails. */
int us_get_status(us_ctx* ctx, int clear, int* device_status);

/* Envelope + log compression kernels, process-wide: enable != 0 (the default) uses the
 * cooperative fused kernel whenever the image's lines fit co-resident blocks; 0 always takes
 * the two-kernel path (envelope, then log compression; the path images too large for the fused
 * kernel take).  Both give the same image.  Applies to every call that forms a B-mode image
 * (us_forward, us_bmode, us_envlog, us_envlog_noalloc); meant for tests of the second path. */
void us_set_envlog_fused(int enable);

/* Transposed DAS kernels, process-wide: enable != 0 (the default) uses the tiled kernel
 * (per-tile sample windows in shared memory, one global atomic per window entry) whenever
 * n_tx <= 32; 0 always takes the untiled kernel (one global atomic per tap).  Both give the
 * same bits (the same fixed-point contributions).  Applies to us_das_adjoint, us_bmode_vjp and
 * us_adjoint; meant for tests of the second path. */
void us_set_das_adj_tiled(int enable);

/* ---------------------------------------------------------------------------------------- */
/* Tracing: per-stage device time and kernel launch counts                                   */
/* ---------------------------------------------------------------------------------------- */

/* Stages timed by us_profile (CUDA events recorded on the launching stream around each
 * stage's kernels). */
enum {
  US_STAGE_GENERATE = 0, US_STAGE_TRAVERSE, US_STAGE_INTERACT, US_STAGE_NEE, US_STAGE_SPLAT_SORT,
  US_STAGE_SPLAT_ROWS, US_STAGE_DAS, US_STAGE_ENVLOG, US_STAGE_LOSS, US_STAGE_ENVLOG_VJP, US_STAGE_DAS_ADJ,
  US_STAGE_NEE_ADJ, US_STAGE_PATH_ADJ, US_STAGE_OTHER, US_STAGE_DAS_ACQ,
  US_STAGE_RAY_SORT,  /* each round's coherence sort of the path queue */
  US_STAGE_JOB_SORT,  /* each round's sort of the secondary-ray jobs (on the lane's second stream
                         when US_OPT_NEE_STREAM is on: its span then overlaps other stages) */
  US_N_STAGES
};

/* enable != 0 starts recording stage events (and clears what was accumulated); 0 stops. */
int us_profile(us_ctx* ctx, int enable);

/* Synchronise on the recorded events and return, per stage, the summed device time [ms] and
 * the number of kernels launched since the last us_profile(ctx, 1).  Arrays hold n entries
 * (at most US_N_STAGES are written). */
int us_profile_read(us_ctx* ctx, double* ms, int64_t* launches, int n);

/* Total number of kernels this context has launched since it was created. */
int us_launch_count(us_ctx* ctx, int64_t* n);

/* ---------------------------------------------------------------------------------------- */
/* S1: sample streams                                                                        */
/* ---------------------------------------------------------------------------------------- */

/* Philox4x32-10 (Salmon et al., SC'11): out_dev[4 i + j] = word j of block
 * philox(ctr = (c0_base + i, c1, c2, c3), key = (k0, k1)), i < n.  The transport draws block
 * (ray_id, tx, stream_id, event) with key (seed_lo, seed_hi) and uses u = (x >> 8) * 2^-24. */
int us_philox_fill(us_ctx* ctx, uint32_t c0_base, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                   uint32_t k1, int64_t n, uint32_t* out_dev, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Forward hot path                                                                          */
/* ---------------------------------------------------------------------------------------- */

/* Full forward pass (Sec. 2.3; Eq. das): emission, wavefront transport (closest hits,
 * Fresnel/Snell interfaces, attenuation, receiver-guided secondary rays at scatterers and, with
 * acq->rough_nee, at rough interface events), sort-
 * based pulse splat -> rf_dev, DAS -> envelope -> log compression -> bmode_dev (dB, in
 * [-dr_db, 0]).  bmode_dev may be NULL (channel data only); img may then be NULL.
 * keep_record != 0 keeps the per-path event record on the context for us_adjoint in record
 * mode and for us_get_record.  seed fixes every sample (common random numbers, Sec. 3.2). */
int us_forward(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq,
               const us_img_desc* img, uint64_t seed, int keep_record, float* rf_dev, float* bmode_dev,
               void* stream);

/* Statistics of the most recent forward pass (synchronises the stream of that pass). */
int us_get_stats(us_ctx* ctx, us_stats* out);

/* Copy the kept record of paths [path_lo, path_lo + n) to out_dev (uint32 per event,
 * n * (k_max + 1) entries).  Event word: bits 0-19 primitive id (element for the transducer),
 * bits 20-21 class (0 none/escape, 1 transducer, 2 triangle, 3 scatterer), bits 22-23 interface
 * choice (0 none, 1 reflect, 2 transmit, 3 total internal reflection), bits 24-31 secondary-ray
 * element.  Path p = tx * rays_per_tx + local ray. */
int us_get_record(us_ctx* ctx, int64_t path_lo, int64_t n, uint32_t* out_dev, void* stream);

/* Copy arrivals [lo, lo + n) of the most recent forward pass on this context (us_get_stats:
 * `arrivals` of them, in the order the transport appended them, which varies between runs) to
 * out_dev (DEVICE uint32[n][4], caller-owned).  Arrival word 0: row = tx * n_elem + element;
 * word 1: time as fixed point, t = (word1 * 2^-18 - 64) / fs; word 2: the amplitude's float
 * bits; word 3: the path p = tx * rays_per_tx + local ray whose transducer hit or secondary ray
 * (Sec. 2.3.3) made it.  Errors: US_ERR_ARG (range outside the list, null out_dev with n > 0),
 * US_ERR_STATE (no forward pass yet).  Synchronises the stream of that pass. */
int us_get_arrivals(us_ctx* ctx, int64_t lo, int64_t n, uint32_t* out_dev, void* stream);

/* S6 alone: splat an explicit arrival list into rf_dev (zeroed first).  Arrival i lands on
 * row tx_dev[i] * n_elem + e_dev[i] at time tau_dev[i] [s] with amplitude a_dev[i] (Eq.
 * axial_sig, pulse centre frequency f0). */
int us_splat(us_ctx* ctx, const us_acq_desc* acq, float f0, int64_t n, const int32_t* tx_dev,
             const int32_t* e_dev, const float* tau_dev, const float* a_dev, float* rf_dev, void* stream);

/* S7 alone: DAS (Eq. das), rf_dev -> irf_dev [n_lines][n_depth], transmits summed coherently,
 * Hann apodisation, linear interpolation, samples outside the record count as zero. */
int us_das(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev, float* irf_dev,
           void* stream);

/* S8 alone: fused envelope (|analytic signal| along depth) and log compression with the
 * dynamic-range clip, irf_dev -> bmode_dev. */
int us_envlog(us_ctx* ctx, const us_img_desc* img, const float* irf_dev, float* bmode_dev, void* stream);

/* Allocation-free S8: the same fused envelope + log compression as us_envlog, for callers that
 * cannot allocate device memory at call time (work issued inside another framework's memory
 * pool or under a hard memory cap, work enqueued while a stream is being captured, or serving
 * loops that cannot afford a first-call allocation and the synchronisation it implies).  The
 * paper has no counterpart; this is a deployment variant.
 *   - Needs no context and calls no allocator: its scratch (the envelope image and the packed
 *     maximum) lives in a fixed device array of the library, sized for at most
 *     US_ENVLOG_NOALLOC_MAX_PIXELS = n_lines * n_depth pixels (1 MiB of floats), that every GPU
 *     which loads the library holds until the process exits.
 *   - Runs on the current CUDA device.  The first call on each device resolves that array's
 *     address and the launch shape, and so does the first call after the device's context
 *     changed (a device reset, a new primary context); make such a call before any stream
 *     capture.
 *   - Reports only its own launches' status: an error pending from unrelated earlier work is
 *     neither returned nor cleared.  The fused kernel's bounded barrier, should it ever expire,
 *     writes NaN (this entry point keeps no status word).
 *   - All calls share the one array and each call overwrites it (the maximum is cleared at the
 *     start of every call), so calls whose work overlaps on the GPU (other streams, other host
 *     threads) race and must be serialised by the caller.
 *   - Returns US_ERR_ARG for a NULL pointer, an invalid image shape or more pixels than the
 *     limit; US_ERR_CUDA if the set-up or the launch fails.  There is no us_last_error text. */
#define US_ENVLOG_NOALLOC_MAX_PIXELS (256 * 1024)
int us_envlog_noalloc(const us_img_desc* img, const float* irf_dev, float* bmode_dev, void* stream);

/* RF -> B-mode (S7 + S8). */
int us_bmode(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev,
             float* bmode_dev, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Loss and adjoint                                                                          */
/* ---------------------------------------------------------------------------------------- */

/* S9a: l1/l2 loss (Eq. weighted_l1_l2_loss, normalised by the pixel count) and its exact
 * gradient: loss_dev[0] = L, dL_dB_dev = dL/dB (may be NULL). */
int us_loss(us_ctx* ctx, const us_img_desc* img, const float* bmode_dev, const float* bref_dev, float* loss_dev,
            float* dL_dB_dev, void* stream);

/* S9b alone: VJP of the fused envelope/log stage: dL/dI_rf from dL/dB. */
int us_envlog_vjp(us_ctx* ctx, const us_img_desc* img, const float* irf_dev, const float* dL_dB_dev,
                  float* dL_dirf_dev, void* stream);

/* S10 alone: transposed DAS (Eq. das_adjoint), a scatter of dL/dI_rf back to the two
 * interpolation samples of every tap; dL_drf_dev is overwritten.  Deterministic: the scatter
 * accumulates in 64-bit fixed point (scale 2^k, the largest power of two with
 * max|dL/dI_rf| x 2^k < 2^40 and pixels x max|dL/dI_rf| x 2^k < 2^62; a tap splits its
 * pixel's integer weight exactly between its two samples), so repeated calls give the same bits
 * whatever the order of the device's atomics.  A non-finite dL/dI_rf makes every entry NaN. */
int us_das_adjoint(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* dL_dirf_dev,
                   float* dL_drf_dev, void* stream);

/* dL/dRF from dL/dB through log, envelope and DAS (S7 recomputed, S9b, S10); deterministic
 * like us_das_adjoint. */
int us_bmode_vjp(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev,
                 const float* dL_dB_dev, float* dL_drf_dev, void* stream);

/* S11 alone: splat adjoint per arrival: ga = sum_n g[n] s(t_n - tau),
 * gt = -a sum_n g[n] s'(t_n - tau), gf = a sum_n g[n] ds(t_n - tau)/df0 (the pulse width
 * follows f0 at fixed fractional bandwidth). */
int us_splat_adjoint(us_ctx* ctx, const us_acq_desc* acq, float f0, int64_t n, const int32_t* tx_dev,
                     const int32_t* e_dev, const float* tau_dev, const float* a_dev, const float* dL_drf_dev,
                     float* ga_dev, float* gt_dev, float* gf_dev, void* stream);

/* S11 + S12: fixed-sample transport VJP (Sec. 3.2, Eq. chain_rule): dL/dtheta from dL/dRF for
 * the realisation fixed by seed.  mode 0 = record (uses the record kept by the last
 * us_forward with keep_record on this scene, theta, acq and seed), mode 1 = recompute (re-runs
 * the transport in chunks of paths to regenerate the decisions).  dL_dtheta_dev: DEVICE
 * float[3M+2] (4M+2 in a rough scene), overwritten. */
int us_transport_vjp(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, uint64_t seed,
                     int mode, const float* dL_drf_dev, float* dL_dtheta_dev, void* stream);

/* Full adjoint: dL/dB -> dL/dRF (us_bmode_vjp) -> dL/dtheta (us_transport_vjp).
 * dL_drf_dev is an optional output (NULL: a library workspace is used).  In mode 0 rf_dev must
 * hold the RF of that same forward pass, unchanged: when it is the buffer the forward pass
 * wrote (and B-mode was formed there), the beamformed image the forward pass made from it is
 * reused instead of beamforming the RF again. */
int us_adjoint(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, const us_img_desc* img,
               uint64_t seed, int mode, const float* rf_dev, const float* dL_dB_dev, float* dL_dtheta_dev,
               float* dL_drf_dev, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Acquisition-parameter gradients: beamforming sound speed c_bf, element pitch, steer angles */
/* ---------------------------------------------------------------------------------------- */
/* These parameters enter the forward model through the emission (Sec. 2.3.1: ray origins on
 * the element faces, x = p (e - (N_e - 1)/2 + u - 1/2), and the time stamp tau_tx = (x_e sin th +
 * W/2 |sin th|) / c_bf with W = (N_e - 1) p), through the secondary rays' targets (Sec. 2.3.3:
 * the element centres x_e = p (e - (N_e - 1)/2)), and through the plane-wave DAS delays of
 * Eq. das.  The gradient is that of the fixed realisation (Sec. 3.2): which element a ray
 * reaches, and whether it reaches the array at all, are decisions held fixed, so the pitch's
 * effect on the element binning is not part of it.  d|sin th|/dth is taken as
 * sgn(sin th) cos th with sgn(0) = 0, the mean of the two one-sided derivatives at th = 0.
 * Gradient layout (dL_dacq_dev, DEVICE float[2 + n_tx], caller-owned, overwritten):
 *   [0] = dL/dc_bf (per m/s), [1] = dL/dpitch (per m),
 *   [2 + t] = dL/d(steering angle of transmit t) (per radian). */

/* DAS part alone: sum_p dL/dI_rf(p) dI_rf(p)/d(c_bf, pitch, th_t) with the RF held fixed.  The slope
 * of each tap is that of the linear-interpolation interval holding its delay.  rf_dev: DEVICE
 * float[n_tx][n_elem][n_samples]; dL_dirf_dev: DEVICE float[n_lines][n_depth].  Errors:
 * US_ERR_ARG (a null buffer, an invalid descriptor), US_ERR_OOM (workspace), US_ERR_CUDA. */
int us_das_acq_vjp(us_ctx* ctx, const us_acq_desc* acq, const us_img_desc* img, const float* rf_dev,
                   const float* dL_dirf_dev, float* dL_dacq_dev, void* stream);

/* Transport part alone: us_transport_vjp (same arguments, modes and record-mode requirements)
 * that also carries each path's time and origin adjoints at emission, and each secondary ray's
 * sensitivity to its target element's position, into dL_dacq_dev.  Errors: those of
 * us_transport_vjp (US_ERR_STATE in record mode without the matching forward pass), and
 * US_ERR_ARG for a null dL_dacq_dev. */
int us_transport_vjp_acq(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, uint64_t seed,
                         int mode, const float* dL_drf_dev, float* dL_dtheta_dev, float* dL_dacq_dev,
                         void* stream);

/* Full adjoint with the acquisition gradient: us_adjoint (same arguments and requirements) plus
 * dL_dacq_dev = DAS part + transport part.  Errors: those of us_adjoint, and US_ERR_ARG for a
 * null dL_dacq_dev. */
int us_adjoint_acq(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, const us_img_desc* img,
                   uint64_t seed, int mode, const float* rf_dev, const float* dL_dB_dev, float* dL_dtheta_dev,
                   float* dL_dacq_dev, float* dL_drf_dev, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Shape gradients: dL/d(triangle vertices)                                                   */
/* ---------------------------------------------------------------------------------------- */
/* The gradient of the fixed realisation (Sec. 3.2) with respect to the scene's triangle
 * vertices: every path keeps the triangles it hits and the secondary rays keep the triangles
 * they cross, while the planes and normals of those triangles move with their vertices (hit
 * distances, specular and Snell directions, Fresnel coefficients, secondary-ray crossing
 * distances and transmission coefficients).  Whether a ray hits a triangle at all is a
 * decision held fixed, so silhouette terms are not part of it.  dL_dtris_dev: DEVICE
 * float[n_tris][9] (v0, v1, v2 of each triangle in the order of the scene's tris), caller-
 * owned, overwritten; accumulated with float atomics, so the last bits vary between runs. */

/* Transport part: us_transport_vjp (same arguments, modes and record-mode requirements) plus
 * dL/d(triangle vertices).  Errors: those of us_transport_vjp, and US_ERR_ARG for a null
 * dL_dtris_dev. */
int us_transport_vjp_shape(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, uint64_t seed,
                           int mode, const float* dL_drf_dev, float* dL_dtheta_dev, float* dL_dtris_dev,
                           void* stream);

/* Full adjoint: us_adjoint (same arguments and requirements) plus dL/d(triangle vertices).
 * Errors: those of us_adjoint, and US_ERR_ARG for a null dL_dtris_dev. */
int us_adjoint_shape(us_ctx* ctx, uint64_t scene, const float* theta, const us_acq_desc* acq, const us_img_desc* img,
                     uint64_t seed, int mode, const float* rf_dev, const float* dL_dB_dev, float* dL_dtheta_dev,
                     float* dL_dtris_dev, float* dL_drf_dev, void* stream);

/* Chain rule to shape parameters q_j (a radius, a thickness, ...):
 * dL_dq_dev[j] = sum_i dL_dtris_dev[i] * dtris_dq_dev[j * 9 n_tris + i] for j < n_param, with
 * dtris_dq_dev the parameters' vertex tangents (DEVICE float[n_param][n_tris][9]) and dL_dq_dev
 * DEVICE float[n_param], caller-owned, overwritten.  1 <= n_param <= 65535; fixed summation
 * order (the same result bit for bit on every call).  Errors: US_ERR_ARG (a null buffer,
 * n_tris < 0, n_param outside its range), US_ERR_CUDA. */
int us_shape_param_grad(us_ctx* ctx, int64_t n_tris, const float* dL_dtris_dev, int n_param, const float* dtris_dq_dev,
                        float* dL_dq_dev, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Inverse problem: parameterisation and optimiser step (Sec. 3.4, Sec. 3.7, Alg. 1)         */
/* ---------------------------------------------------------------------------------------- */

/* Physical parameters from the optimiser's unconstrained variables (Sec. 3.4, Eq. clip01 and
 * Eq. scale_phys): theta[j] = lo[j] + clip(theta_u[j], 0, 1) (hi[j] - lo[j]).  All arrays are
 * DEVICE float[n], caller-owned; 1 <= n <= 1024.  Stream-ordered. */
int us_param_map(us_ctx* ctx, int n, const float* theta_u_dev, const float* lo_dev, const float* hi_dev,
                 float* theta_dev, void* stream);

/* One Adam step on theta_u (Sec. 3.7, Eq. adam) from the gradient with respect to the PHYSICAL
 * parameters (dL/dtheta, e.g. from us_adjoint): the gradient is carried back through the scale
 * and the clip (Eq. clip_grad: zero where theta_u lies outside (0, 1)), scaled down to global
 * L2 norm clip_norm when it is longer (clip_norm <= 0: no clipping), then
 *   m = beta1 m + (1 - beta1) g,  v = beta2 v + (1 - beta2) g^2,
 *   theta_u -= lr[j] (m / (1 - beta1^step)) / (sqrt(v / (1 - beta2^step)) + eps).
 * lr_dev holds one learning rate per parameter (parameter groups).  step counts from 1.
 * theta_u_dev, m_dev, v_dev are updated in place (m, v start at zero).  All arrays DEVICE
 * float[n], caller-owned; 1 <= n <= 1024. */
int us_adam_step(us_ctx* ctx, int n, float* theta_u_dev, const float* dL_dtheta_dev, const float* lo_dev,
                 const float* hi_dev, const float* lr_dev, float beta1, float beta2, float eps, float clip_norm,
                 int step, float* m_dev, float* v_dev, void* stream);

/* ---------------------------------------------------------------------------------------- */
/* Batching (many scenes / probe poses of uneven size)                                       */
/* ---------------------------------------------------------------------------------------- */

/* One request of a batch.  bref_dev == NULL: forward only (rf_dev, bmode_dev as in
 * us_forward).  bref_dev != NULL: forward + l1/l2 loss against bref_dev + adjoint in record
 * mode, writing loss_dev[0] and dL_dtheta_dev (float[3M+2]).  Host pointers must stay valid
 * for the duration of the call; device buffers until the batch has run. */
typedef struct {
  uint64_t scene;
  const float* theta;
  const us_acq_desc* acq;
  const us_img_desc* img;
  uint64_t seed;
  float* rf_dev;
  float* bmode_dev;
  const float* bref_dev;
  float* loss_dev;
  float* dL_dtheta_dev;
} us_request;

/* Run n requests as one stream-ordered unit on `stream`: they are spread round-robin over
 * US_OPT_LANES lanes (own stream and workspaces each; forked from and joined back to
 * `stream`), so small requests overlap on the device.  After one call outside capture has sized
 * the lanes' workspaces, the call can be captured in a CUDA graph and replayed.  Each
 * request's results are those of the corresponding single calls. */
int us_forward_batch(us_ctx* ctx, int n, const us_request* reqs, void* stream);

/* Autotuner: times the batch for lane counts {1, 2, 4, 8} and traversal grids of {1, 2, 4} x
 * the resident blocks per SM, keeps the fastest on the context and reports it.  Synchronous. */
int us_autotune_batch(us_ctx* ctx, int n, const us_request* reqs, void* stream, int* best_lanes,
                      int* best_trav_per_sm);

/* Serving: run one request on lane `lane` (1..16; lane 0 belongs to the single-request calls)
 * on the caller's `stream`.  Requests on different lanes may run concurrently on different
 * streams; requests on one lane must be stream-ordered.  */
int us_run_request(us_ctx* ctx, int lane, const us_request* req, void* stream);

/* Device memory [bytes] a request's workspaces need on a lane (admission control). */
int us_request_bytes(us_ctx* ctx, const us_request* req, size_t* bytes);

#ifdef __cplusplus
}
#endif

#endif /* USRT_H */
