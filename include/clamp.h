/*
 * clamp.h -- C ABI of the GB300 (sm_103a) CLAMP hot path.
 *
 * CLAMP (Allen, Rabb, Buzzard, Bouman, "CLAMP: Majorized Plug-and-Play for
 * Coherent 3D Lidar Imaging", IEEE TCI 11, 2025) reconstructs a real
 * reflectance r from L looks y_l = A g_l + eta_l, A = D(a) F (Eq. (A)), by a
 * MACE iteration (Alg. 2) over L majorized forward agents and one prior agent.
 *
 * Conventions for every entry point
 *  - Volumes are [nz][ny][nx], x fastest.  Complex arrays are interleaved
 *    (re, im) float32 pairs.  Frequency-domain arrays (y, pupil, window) are in
 *    unshifted FFT order, DC at index 0.  Per-look arrays are [L][n] with
 *    n = nx*ny*nz, look-major.
 *  - Axis lengths must be 8, 16, 32, 64, 96, 128, 192 or 256 (radix 2/4/8/16 and 3 passes);
 *    nx must be a multiple of 16.
 *  - Unless a function says "host", every array pointer is caller-owned DEVICE
 *    memory on the current CUDA device; the library never frees it.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    stream-ordered and asynchronous unless documented otherwise.
 *  - Scratch: `ws` / `ws_bytes` is a caller-owned device buffer, 256-byte
 *    aligned, of at least the size the matching *_workspace_size query
 *    returns; the library keeps nothing in it between calls unless stated.
 *  - Errors: every call returns a clamp_status and never aborts; on failure
 *    clamp_last_error() gives a message (thread-local).  Invalid arguments are
 *    rejected before any launch.
 */
#ifndef CLAMP_H
#define CLAMP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum clamp_status {
  CLAMP_OK = 0,
  CLAMP_EINVAL = 1,      /* invalid argument (shape, pointer, parameter) */
  CLAMP_ENOMEM = 2,      /* workspace too small or device allocation failed */
  CLAMP_ECUDA = 3,       /* CUDA runtime error */
  CLAMP_ENOTCONV = 4,    /* iteration did not reach the tolerance */
  CLAMP_ETIMEOUT = 5,    /* a bounded device wait gave up */
  CLAMP_ENONFINITE = 6,  /* a non-finite value appeared in the state */
  CLAMP_EUNSUPPORTED = 7 /* size or option not supported by this build */
} clamp_status;

/* Flags for clamp_params.flags. */
#define CLAMP_FLAG_MU_INIT_NO_ALPHA 0x1 /* mu_l = A^H y_l (Alg. 2) instead of A^H y_l / alpha (Sec. IV-A) */
/* Reflectance update by the exact prox of the EM surrogate: per voxel the positive root of
 * r^3 - v r^2 + sigma^2 r - sigma^2 K = 0 with the smallest objective (Sec. III-B, the
 * "closed form by solving for a root of a cubic"), instead of App. A's quadratic step. */
#define CLAMP_FLAG_EXACT_PROX 0x2
/* No-aperture ablation (Sec. IV-A): a = 1 everywhere (pupil and window are ignored,
 * alpha = 1) and the mu update is the closed-form minimiser of h,
 * mu = F^H y / (1 + sigma_w^2 / (r' + sigma_w^2)); no FFT runs per iteration. */
#define CLAMP_FLAG_NO_APERTURE 0x4
/* Prior-agent schedule.  Within an iteration the prior agent and the forward agents both
 * read the previous w and write disjoint state, so the prior may run on a second stream
 * beside the forward agents (forked from and joined back to the caller's stream, so stream
 * order and graph capture are kept; see clamp_prior_concurrent).  By default it does for
 * problems of at most 2^25 voxel-looks (n L), where the prior's few waves of tensor-core
 * CTAs leave SMs that the FFT passes fill, and not above that, where both saturate the
 * GPU and only contend.  These flags force either schedule (at most one may be set). */
#define CLAMP_FLAG_PRIOR_CONCURRENT 0x8
#define CLAMP_FLAG_PRIOR_SERIAL 0x10
/* Forward-agent schedule.  The gradient d = F^H[a (y - a F mu)] / sigma_w^2 - D mu
 * (Eq. h-gradient) and ||A d|| need the y and z transforms only where the pupil is
 * nonzero, so by default the forward agents transform whole x rows once and everything
 * else on the pupil's support (the band-limited schedule); F mu is formed once per call and
 * then advanced by gamma F d.  The full-spectrum schedule transforms every axis of F mu,
 * F(D mu) and F^H(F d) over the whole volume (five passes).  Both compute the same
 * quantities up to FP32 rounding.  The band-limited schedule is used when its arrays fit
 * the agent scratch (clamp_workspace_size), which holds whenever the pupil covers at most
 * about half of the (ky, kx) plane; these flags force either (at most one may be set;
 * CLAMP_FLAG_BAND_SPECTRUM falls back to the full spectrum when the arrays do not fit). */
#define CLAMP_FLAG_FULL_SPECTRUM 0x20
#define CLAMP_FLAG_BAND_SPECTRUM 0x40

/* Problem and iteration parameters (Sec. II-B, Sec. III, Sec. IV-A). */
typedef struct clamp_params {
  int32_t nx, ny, nz;   /* volume shape */
  int32_t looks;        /* L >= 1 forward agents */
  float noise_var;      /* sigma_w^2 > 0: data-noise variance (Eqs. forward-model, mu-objective) */
  float prox_var;       /* sigma^2 > 0: forward-agent proximal parameter (Eq. prox) */
  float rho;            /* Mann parameter in (0, 1) (Eq. mann); the paper uses 0.5 */
  float prior_weight;   /* upsilon_{L+1} in (0, 1); each look gets (1 - prior_weight)/L (Sec. III-A) */
  int32_t max_iters;    /* iterations run by clamp_reconstruct */
  int32_t k0;           /* iterations already done (resume); beta uses k = k0 + 1, k0 + 2, ... */
  int32_t flags;        /* CLAMP_FLAG_* */
  int32_t check_every;  /* clamp_reconstruct reads the residual back every this many iterations (tol > 0) */
  double tol;           /* stop when the convergence error <= tol (0 = run max_iters) */
  int32_t init_mu_steps; /* with a given r_init: this many mu updates of the forward agents
                            (Alg. 2 steps 5-8 with r' = r_init held fixed) before the first
                            iteration, so mu starts consistent with r_init; 0..1000 */
  int32_t reserved;     /* set to 0 */
} clamp_params;

/* Per-run report of clamp_reconstruct (host memory). */
typedef struct clamp_report {
  int32_t iters;        /* iterations run */
  int32_t converged;    /* 1 if the convergence error reached tol */
  double ce_residual;   /* last convergence error (Eq. mace-convergence-error) */
  double mu_residual;   /* last mu-residual, floored form (Eq. residual) */
  double* ce_hist;      /* optional host array [max_iters], filled when non-NULL */
  double* mu_hist;      /* optional host array [max_iters], filled when non-NULL */
} clamp_report;

/* Opaque prior-agent handle (owns its device weights). */
typedef struct clamp_denoiser clamp_denoiser;

#define CLAMP_DENOISER_FP32 0
#define CLAMP_DENOISER_BF16 1

const char* clamp_last_error(void);
const char* clamp_version(void);

/* 1 if `n` is a supported axis length. */
int32_t clamp_supported_length(int32_t n);

/* Validates a parameter block; CLAMP_OK or CLAMP_EINVAL / CLAMP_EUNSUPPORTED. */
clamp_status clamp_check_params(const clamp_params* p);

/* Scratch bytes needed by clamp_init, clamp_forward_prox and clamp_mace_step for `p`
 * (about 24 bytes per voxel-look plus reduction partials).  0 if `p` is invalid. */
size_t clamp_workspace_size(const clamp_params* p);

/* Scratch bytes clamp_reconstruct needs: state (mu, r, w), the forward-agent
 * scratch and the denoiser's scratch.  0 if invalid. */
size_t clamp_reconstruct_workspace_size(const clamp_params* p, const clamp_denoiser* den);

/* Orthonormal 3D DFT F (or F^H when inverse != 0) of `batch` volumes (Eq. (A):
 * F is the orthonormal DFT, scale 1/sqrt(n) each way).  in, out: complex
 * [batch][n]; in == out is allowed.  Uses out as its only scratch. */
clamp_status clamp_fft3(int32_t nx, int32_t ny, int32_t nz, int32_t batch,
                        const float* in, float* out, int32_t inverse, void* stream);

/* Data simulation (Eqs. forward-model, g-given-r): y_l = a .* F(sqrt(r) .* z_l) + sqrt(sigma_w^2) eta_l
 * with a = window[kz] * pupil[ky][kx].  r: float [n]; speckle z, noise eta: complex [L][n]
 * (CN(0,1) draws supplied by the caller); y: complex [L][n] out.  sigma_w^2 = p->noise_var. */
clamp_status clamp_simulate(const clamp_params* p, const float* r, const float* speckle,
                            const float* noise, const float* pupil, const float* window,
                            float* y, void* stream);

/* Initialisation of Alg. 2 as in Sec. IV-A: r0 = (1/L) sum_l |A^H y_l|^2 floored at
 * 1e-12 max(r0) (or r_init when non-NULL), r_j = w_j = r0 for j = 1..L+1, and
 * mu_l = A^H y_l / alpha with alpha = mean(a^2).
 * y: complex [L][n]; pupil [ny][nx]; window [nz]; r_init: float [n] or NULL;
 * mu: complex [L][n] out; r, w: float [L+1][n] out (row L is the prior agent's). */
clamp_status clamp_init(const clamp_params* p, const float* y, const float* pupil,
                        const float* window, const float* r_init, float* mu, float* r, float* w,
                        void* ws, size_t ws_bytes, void* stream);

/* All L majorized forward agents for CLAMP iteration k >= 1 (Alg. 2, steps 5-9):
 * c_l = sigma_w^2 r_l / (alpha r_l + sigma_w^2); d = -grad h(mu_l) (Eq. h-gradient);
 * exact line search gamma (Eq. mu-update); mu_l += gamma d; r_l <- the App. A
 * quadratic-surrogate prox of w_l with beta = 1 + 2/ln(k+1), anchored at the old r_l.
 * mu: complex [L][n] in/out; r: float [>= L][n] in/out (rows 0..L-1 used);
 * w: float [>= L][n] in.  mu_residual: optional DEVICE double out, the look-averaged
 * floored mu-residual (Eq. residual) at the incoming mu. */
clamp_status clamp_forward_prox(const clamp_params* p, int32_t k, const float* y,
                                const float* pupil, const float* window, float* mu, float* r,
                                const float* w, double* mu_residual, void* ws, size_t ws_bytes,
                                void* stream);

/* Prior agent r_prior = H(w_prior) (Alg. 2, step 11).  Both float [n]. */
clamp_status clamp_denoise(const clamp_denoiser* den, const float* w_prior, float* r_prior,
                           int32_t nx, int32_t ny, int32_t nz, void* ws, size_t ws_bytes,
                           void* stream);

/* MACE step (Alg. 2, steps 12-14; Eq. mann): wbar_old = sum_j ups_j w_j,
 * x = 2r - w, w <- w + 2 rho (G(x) - r), wbar = sum_j ups_j w_j (new w).
 * r: float [L+1][n] agent outputs; w: float [L+1][n] in/out; wbar: float [n] out;
 * ce_residual: optional DEVICE double out, the convergence error
 * ||r - G(w)|| / ||G(w)|| (Eq. mace-convergence-error) of the incoming w. */
clamp_status clamp_mace_step(const clamp_params* p, const float* r, float* w, float* wbar,
                             double* ce_residual, void* ws, size_t ws_bytes, void* stream);

/* The MACE step of clamp_mace_step without any device allocation, for callers that
 * cannot allocate device memory themselves (an application allocator that owns the
 * GPU's memory, or a loop that must not allocate once running).  No counterpart in
 * the paper: same arguments and results as clamp_mace_step, minus the workspace.
 * Its only scratch (the convergence-error partial sums) lives in a 32 KiB static
 * device array that every GPU loading this library keeps until exit; the first call
 * on a device looks up that array's address (so make it before any stream capture).
 * Calls no cudaMalloc/cudaFree.  All calls share the array: calls that overlap on
 * the GPU (other streams, other threads) race and must be serialised by the caller.
 * Returns CLAMP_ENOMEM if the partial sums would not fit the array (never for the
 * volumes clamp_check_params accepts: at most 1216 reduction blocks x 16 bytes).
 * The array's address is cached per device ordinal: after cudaDeviceReset, call
 * clamp_release_cache() before the next call so that it is looked up again. */
clamp_status clamp_mace_step_noalloc(const clamp_params* p, const float* r, float* w, float* wbar,
                                     double* ce_residual, void* stream);

/* Prior agents. */
clamp_status clamp_denoiser_create_gauss(float sigma, clamp_denoiser** out);
/* The l2,1 prior agent of the paper's comparison method (Sec. IV: "l2-regularization in
 * cross-range and l1-regularization in range"): the proximal map of lam * sum_z ||r_z||_2,
 * r_z the (y, x) plane of range bin z, i.e. each plane shrunk in l2 norm by lam:
 * H(w)_z = max(0, 1 - lam / ||w_z||) w_z.  The plane norms are FP64 sums.  lam >= 0
 * (lam = 0 is the identity).  Workspace: clamp_denoise_workspace_size bytes (one FP64
 * partial sum per CTA and plane); in == out is allowed. */
clamp_status clamp_denoiser_create_l21(float lam, clamp_denoiser** out);
/* Residual CNN H(x) = x + CNN(x), 3x3x3 convs, zero padding; layer i maps
 * c_in -> c_out (1 -> C -> ... -> C -> 1), ReLU after every layer but the last.
 * weights_host: all layers' [c_out][c_in][3][3][3] float32 concatenated;
 * biases_host: all layers' [c_out] concatenated.  dtype: CLAMP_DENOISER_FP32 or _BF16.
 * BF16: weights and every layer's input are rounded to bfloat16, products accumulate in
 * FP32 on the tensor cores; needs channels in {16, 32, 48, 64} and volumes with
 * nx % 128 == 0, ny % 2 == 0, nz % 2 == 0 (else CLAMP_EUNSUPPORTED at use).
 * FP32: on the tensor cores through a TF32x3 split when channels are in {16, 32, 48} and
 * nx % 128 == 0, ny % 2 == 0, nz % 2 == 0; otherwise on FP32 CUDA cores. */
clamp_status clamp_denoiser_create_cnn(int32_t layers, int32_t channels, int32_t dtype,
                                       const float* weights_host, const float* biases_host,
                                       clamp_denoiser** out);
void clamp_denoiser_destroy(clamp_denoiser* den);

/* Self-check of the bounded waits the tensor-core kernels use so that a missing MMA
 * completion makes them report CLAMP_ETIMEOUT instead of hanging: one mbarrier receives
 * its arrival (the wait must succeed), nothing arrives on another (the wait must give up
 * after `limit` polls, 1 <= limit <= 2^20).  result: host int32[2] = {first wait
 * succeeded, second wait succeeded}; a sound build gives {1, 0}.  Synchronous.  The paper
 * has no counterpart. */
clamp_status clamp_selftest_bounded_wait(int32_t limit, int32_t* result);

/* Bounds-checking build query.  The test variant of the library (built with
 * CLAMP_BOUNDS_CHECK defined) tests every global-memory index of the hot-path kernels (the
 * forward agents' band passes, pass C, the CNN prior's tensor-core convolutions and tap
 * gather) against the extent of the buffer it addresses, skips an access that falls
 * outside and records the first offending site code (101-199 band passes, 201-299 pass C,
 * 301-399 CNN prior).  Writes that code, or 0 if none was recorded, to *site (host
 * pointer) and clears the record if `reset` is non-zero.  Returns 1 for the checked
 * build, 0 for the product build (*site is then always 0), or a negative clamp_status
 * if reading the record failed.  Synchronous (reads device memory).  The paper has no
 * counterpart. */
int32_t clamp_bounds_check(int32_t reset, uint32_t* site);

/* Tensor-core building block check: D[128][n] = A[128][k] B[n][k]^T with A, B BF16
 * (row-major, k contiguous) and D FP32, on one CTA through tcgen05 MMAs with TMEM
 * accumulators -- the same descriptor conventions the BF16 CNN prior uses.
 * 16 <= n, k <= 256, multiples of 16.  Device pointers. */
clamp_status clamp_tc_gemm_bf16(int32_t n, int32_t k, const void* a, const void* b, float* d, void* stream);

/* Same with FP32 A, B through the TF32x3 split the FP32 CNN prior uses
 * (hi*hi + hi*lo + lo*hi on kind::tf32).  16 <= n <= 256 (multiple of 16), 8 <= k <= 192
 * (multiple of 8); CLAMP_EINVAL if the operands exceed shared memory. */
clamp_status clamp_tc_gemm_tf32x3(int32_t n, int32_t k, const float* a, const float* b, float* d, void* stream);
size_t clamp_denoise_workspace_size(const clamp_denoiser* den, int32_t nx, int32_t ny, int32_t nz);

/* Scratch bytes clamp_iterate needs (forward-agent scratch plus the denoiser's). */
size_t clamp_iterate_workspace_size(const clamp_params* p, const clamp_denoiser* den);

/* 1 if iterations with these parameters run the prior agent concurrently with the forward
 * agents (CLAMP_FLAG_PRIOR_* and the default size rule above), else 0; -1 for invalid
 * parameters.  Host-only.  A call made while `stream` is being captured, before the
 * library created its side stream on this host thread and device, runs serially. */
int32_t clamp_prior_concurrent(const clamp_params* p);

/* Runs `iters` CLAMP iterations k = k_first, ..., k_first + iters - 1 (the loop body of
 * Alg. 2: all forward agents, the prior agent on w_{L+1}, the MACE step) on a
 * caller-held state, so a run can be resumed from {mu, r, w, k}.
 * mu: complex [L][n], r, w: float [L+1][n] (in/out); wbar: float [n] out (sum_j ups_j w_j
 * after the last step, the Alg. 2 output).  ce_out, mu_out: optional DEVICE double
 * arrays [iters] receiving the convergence error and mu-residual of each iteration.
 * events: optional array of 4 * iters cudaEvent_t handles recorded per iteration: before
 * the forward agents (and the fork of the prior), after their line search, after the
 * prior agent, after the MACE pass (for timing).  All are recorded on `stream` except the
 * third under the concurrent schedule, which is recorded on the side stream the prior
 * runs on.  Stream-ordered, no host synchronisation after argument checks. */
clamp_status clamp_iterate(const clamp_params* p, int32_t k_first, int32_t iters, const float* y,
                           const float* pupil, const float* window, const clamp_denoiser* den,
                           float* mu, float* r, float* w, float* wbar, double* ce_out,
                           double* mu_out, void* ws, size_t ws_bytes, void* const* events,
                           void* stream);

/* Full CLAMP reconstruction (Alg. 2) on device buffers: init, then up to
 * p->max_iters iterations of forward agents + prior agent + MACE step, stopping
 * early when tol > 0 and the convergence error <= tol (checked every
 * p->check_every iterations).  r_out: float [n] <- r* = wbar (Alg. 2 output).
 * ws may be NULL (the call then allocates and frees its scratch).  Synchronises
 * the stream when report != NULL or tol > 0. */
clamp_status clamp_reconstruct(const clamp_params* p, const float* y, const float* pupil,
                               const float* window, const clamp_denoiser* den,
                               const float* r_init, float* r_out, clamp_report* report,
                               void* ws, size_t ws_bytes, void* stream);

/* Same on HOST buffers (pageable or pinned): copies y, pupil, window and r_init to
 * the device, reconstructs, copies r_out back and synchronises.  Device scratch is
 * kept in a per-device cache between calls (clamp_release_cache frees it;
 * clamp_release_cache also forgets the device addresses clamp_mace_step_noalloc caches). */
clamp_status clamp_reconstruct_host(const clamp_params* p, const float* y_host,
                                    const float* pupil_host, const float* window_host,
                                    const clamp_denoiser* den, const float* r_init_host,
                                    float* r_out_host, clamp_report* report, void* stream);
void clamp_release_cache(void);

/* Host staging memory for clamp_reconstruct_host: `bytes` of zeroed host memory backed by
 * transparent huge pages where the kernel offers them (an anonymous mapping started on a
 * huge-page boundary, madvise(MADV_HUGEPAGE), touched before use) and page-locked for the
 * current CUDA device (cudaHostRegister).  Host-to-device copies from it need few I/O
 * translations; on GB300 hosts a 2 GB upload from it took 10.2 ms every time, where the
 * same upload from base-page pinned memory sometimes took 50-100 ms.  *out receives the
 * host pointer (huge-page aligned, 2 MiB at least), or NULL on failure; free it with
 * clamp_host_free.  CLAMP_EINVAL for bytes == 0 or out == NULL, CLAMP_ENOMEM if the
 * mapping fails, CLAMP_ECUDA if the registration fails (nothing is kept then).
 * Synchronous; not part of the paper's method. */
clamp_status clamp_host_alloc(size_t bytes, void** out);
/* Unregisters and unmaps memory from clamp_host_alloc; NULL is ignored, and so is a
 * pointer the allocator did not return. */
void clamp_host_free(void* p);

/* ---- Autotuner.  Each forward-agent FFT pass (x, y, fused z, inverse y, inverse x) has
 * launch variants: 0 = default radix plan and tile, 1 = alternative radix plan,
 * 2 = other tile schedule (half the rows per CTA in x passes, 32 columns per CTA in
 * y / z passes).  The tuner times every valid variant of each pass on `ws` (a
 * clamp_workspace_size buffer; its contents are overwritten) and caches the fastest per
 * (device, nx, ny, nz, looks); every later call on that geometry uses the cached choice.
 * variants_out: optional host int32[5].  Synchronises. */
clamp_status clamp_autotune(const clamp_params* p, const float* y, const float* pupil, const float* window,
                            void* ws, size_t ws_bytes, void* stream, int32_t* variants_out);
/* Sets the cached choice for a geometry by hand (host int32[5]). */
clamp_status clamp_autotune_set(const clamp_params* p, const int32_t* variants);
/* Sets the band-limited schedule's row-pass variant for a geometry (0: the default tile of
 * rows per CTA; 1: tiles of half as many rows, three CTAs per SM; 2: the default tile with
 * mu and r' prefetched to L2 and read after the inverse transform, three CTAs per SM),
 * keeping the other cached choices.  clamp_autotune times all three and keeps the fastest. */
clamp_status clamp_autotune_set_band(const clamp_params* p, int32_t row_variant);
/* Which forward-agent schedule iterations with these parameters and this aperture run
 * (CLAMP_FLAG_*_SPECTRUM, the autotuner's cached choice, else the band-limited one when its
 * arrays fit the scratch).  pupil [ny][nx], window [nz]: device.  info (host int32[5]):
 * schedule (1 band-limited, 0 full spectrum), the support's column count |{(ky, kx):
 * pupil != 0}|, the band's column count |{kx: some pupil(ky, kx) != 0}|, 1 if the
 * band-limited arrays fit, and the band-limited row-pass variant (clamp_autotune_set_band).
 * Reads the pupil back (synchronises `stream`). */
clamp_status clamp_agent_schedule(const clamp_params* p, const float* pupil, const float* window, void* stream,
                                  int32_t* info);

/* ---- Batched reconstruction: many scenes of uneven size and look count in one launch. */

/* One scene of a batch: its parameters (shape, looks, variances, iterations) and DEVICE
 * buffers laid out as for clamp_reconstruct. */
typedef struct clamp_scene {
  clamp_params p;
  const float* y;       /* complex [L][n] */
  const float* pupil;   /* [ny][nx] */
  const float* window;  /* [nz] */
  float* r_out;         /* [n] <- r* */
} clamp_scene;

typedef struct clamp_batch clamp_batch;  /* opaque plan: captured CUDA graph + per-scene state */

/* Scratch bytes for a batch (the sum of the scenes' reconstruction workspaces). */
size_t clamp_batch_workspace_size(const clamp_scene* scenes, int32_t count, const clamp_denoiser* den);

/* Builds a batch plan: checks every scene, partitions `ws` among them, autotunes the
 * forward-agent passes of every distinct scene geometry (clamp_autotune) and captures
 * into ONE CUDA graph, for every scene as an independent branch, the Alg. 2
 * initialisation followed by p.max_iters iterations (forward agents, prior agent,
 * MACE step), with a timing event at the start and at the end of each branch.
 * Scenes, denoiser and ws must stay valid while the plan is used.  Synchronises. */
clamp_status clamp_batch_create(const clamp_scene* scenes, int32_t count, const clamp_denoiser* den, void* ws,
                                size_t ws_bytes, clamp_batch** out);
/* Launches the whole batch with one cudaGraphLaunch on `stream` (asynchronous). */
clamp_status clamp_batch_launch(clamp_batch* b, void* stream);
/* After the launch completed (synchronises `stream`): per-scene latency from the launch
 * start to the end of that scene's branch, milliseconds, host array [count]. */
clamp_status clamp_batch_latencies(clamp_batch* b, void* stream, float* latency_ms);
/* Per-scene final convergence error (host array [count]); synchronises. */
clamp_status clamp_batch_residuals(clamp_batch* b, void* stream, double* ce);
void clamp_batch_destroy(clamp_batch* b);


/* The initial image of Alg. 2 alone: r0 = (1/L) sum_l |A^H y_l|^2 (the speckle average;
 * Sec. IV-A), floored at 1e-12 of its maximum as the initialisation floors it.
 * r0: device float [n].  ws: at least clamp_workspace_size(p) bytes. */
clamp_status clamp_speckle_average(const clamp_params* p, const float* y, const float* pupil, const float* window,
                                   float* r0, void* ws, size_t ws_bytes, void* stream);

/* ---- Point-cloud metrics of a reconstruction (Sec. IV-B, Eqs. pc-distance, nrmse).
 * P = voxels of r_hat above `threshold` (the paper's noise floor sigma_w^2 / alpha), Q =
 * voxels of r_true above 0, with voxel-grid coordinates.  Each p in P is matched to its
 * nearest q in Q (Euclidean, in voxels; ties to the smallest linear index); points with
 * no q within max_dist (the paper: 3 x the Rayleigh resolution) are removed.
 * out (host double[6]): mean distance of the kept points, false-positive rate (removed /
 * |P|), NRMSE(beta* r_hat, r) over the kept points, kept count, removed count, beta* =
 * sum r_hat r_q / sum r_hat^2.  r_hat, r_true: device float [nz][ny][nx]; max_dist in
 * [0, 64]; ws: clamp_point_cloud_workspace_size() bytes.  Synchronises `stream`. */
size_t clamp_point_cloud_workspace_size(void);
clamp_status clamp_point_cloud_metrics(const float* r_hat, const float* r_true, int32_t nx, int32_t ny, int32_t nz,
                                       float threshold, float max_dist, double* out, void* ws, size_t ws_bytes,
                                       void* stream);

/* ---- Learned warm start: a 3-level 3D U-Net mapping the speckle-averaged image to an
 * initial reflectance, trained on the GPU with these kernels.
 *
 * Architecture (encoder-decoder with concatenated skips, the pattern of the prior in
 * Sec. III-C; channels c1/c2/c3 per level, 3x3x3 convs with zero padding):
 *   e1 = relu(conv(x))  s1 = relu(conv(e1))       [c1, full size]
 *   p1 = maxpool2(s1);  e2 = relu(conv(p1))  s2 = relu(conv(e2))   [c2, half]
 *   p2 = maxpool2(s2);  b1 = relu(conv(p2))  b2 = relu(conv(b1))   [c3, quarter]
 *   u2 = tconv2(b2);    d2 = relu(conv(relu(conv([u2, s2]))))      [c2, half]
 *   u1 = tconv2(d2);    d1 = relu(conv(relu(conv([u1, s1]))))      [c1, full]
 *   out = conv1x1(d1)                                              [1]
 * maxpool2: 2x2x2 max-pooling; tconv2: transposed conv with a 2x2x2 kernel and stride 2.
 * Parameters, in this order, each layer's weights then its c_out biases (float32):
 *   3x3x3 conv: W[c_out][c_in][3][3][3] (cross-correlation, tap (dz,dy,dx) reads the
 *   input at offset (dz-1, dy-1, dx-1));  tconv2: W[c_in][c_out][2][2][2] with
 *   out[2v + d] = b + sum_ci W[ci][co][d] in[v];  1x1: W[1][c1].
 * Layers: conv 1->c1, c1->c1, c1->c2, c2->c2, c2->c3, c3->c3, tconv c3->c2,
 *   conv 2c2->c2, c2->c2, tconv c2->c1, conv 2c1->c1, c1->c1, 1x1 c1->1.
 * Tensors are float32 [batch][channels][nz][ny][nx] on the device; nx, ny, nz must be
 * multiples of 4.  dtype CLAMP_DENOISER_BF16: every conv rounds its weights and inputs
 * (forward) or its two operands (gradients) to bfloat16 and accumulates in FP32 (the 3x3x3
 * convs on the tensor cores where clamp_unet_set_tensor_cores allows);
 * CLAMP_DENOISER_FP32: all FP32.  Master weights, gradients and Adam moments are FP32. */
typedef struct clamp_unet clamp_unet;

/* params_host: parameter_count floats, or NULL for zeros. */
clamp_status clamp_unet_create(int32_t c1, int32_t c2, int32_t c3, int32_t dtype, const float* params_host,
                               clamp_unet** out);
void clamp_unet_destroy(clamp_unet* u);
int64_t clamp_unet_param_count(const clamp_unet* u);
/* Host copies of the state: which = 0 parameters, 1 gradients (of the last backward),
 * 2 Adam first moments, 3 Adam second moments.  Synchronous. */
clamp_status clamp_unet_get(const clamp_unet* u, int32_t which, float* host);
clamp_status clamp_unet_set(clamp_unet* u, int32_t which, const float* host);
/* Scratch bytes for a batch at (nx, ny, nz); training != 0 adds the gradient buffers. */
size_t clamp_unet_workspace_size(const clamp_unet* u, int32_t batch, int32_t nx, int32_t ny, int32_t nz,
                                 int32_t training);
/* y[batch][n] = U-Net(x[batch][n]) (device pointers). */
clamp_status clamp_unet_forward(clamp_unet* u, const float* x, float* y, int32_t batch, int32_t nx, int32_t ny,
                                int32_t nz, void* ws, size_t ws_bytes, void* stream);
/* Forward pass, loss = mean((U-Net(x) - target)^2) over all batch * n outputs, and the
 * gradient of the loss with respect to every parameter (overwrites the gradient buffer).
 * loss: optional DEVICE double. */
clamp_status clamp_unet_backward(clamp_unet* u, const float* x, const float* target, int32_t batch, int32_t nx,
                                 int32_t ny, int32_t nz, double* loss, void* ws, size_t ws_bytes, void* stream);
/* Forward pass and loss = mean((U-Net(x) - target)^2) only (device double); ws as for
 * clamp_unet_backward (training != 0). */
clamp_status clamp_unet_loss(clamp_unet* u, const float* x, const float* target, int32_t batch, int32_t nx,
                             int32_t ny, int32_t nz, double* loss, void* ws, size_t ws_bytes, void* stream);
/* Per-sample normalisation of training pairs: m_b = sum(x_b) / norm_count (FP64),
 * x_out_b = x_b / m_b and, when t is non-NULL, t_out_b = t_b / m_b; a sample with m_b <= 0
 * is copied unscaled.  The warm start uses norm_count = nx * ny (energy per (x, y) column,
 * which does not change with the range extent nz).  x, t: device float [batch][n]; the
 * outputs may alias the inputs. */
clamp_status clamp_unet_normalize(int32_t batch, int64_t n, int64_t norm_count, const float* x, const float* t,
                                  float* x_out, float* t_out, void* stream);
/* The warm start: m = sum(r0) / (nx ny), r_init = m * max(U-Net(r0 / m), floor_rel).  r0 is
 * the speckle average (clamp_speckle_average); r_init goes to clamp_reconstruct.  ws: at
 * least clamp_unet_workspace_size(u, 1, nx, ny, nz, 0) bytes. */
clamp_status clamp_unet_warm_start(clamp_unet* u, int32_t nx, int32_t ny, int32_t nz, const float* r0,
                                   float floor_rel, float* r_init, void* ws, size_t ws_bytes, void* stream);
/* The 3D U-Net prior agent (Sec. III-C): a denoiser H(w) = m max(U(w / m), floor_rel),
 * m = sum(w) / (nx ny), U a clamp_unet trained as a denoiser.  The denoiser borrows `net`:
 * the caller keeps it alive, unchanged, while the denoiser is in use, and destroys it
 * after clamp_denoiser_destroy.  Volumes need nx, ny, nz multiples of 4 (else
 * CLAMP_EUNSUPPORTED at use); workspace: clamp_unet_workspace_size(net, 1, nx, ny, nz, 0). */
clamp_status clamp_denoiser_create_unet(clamp_unet* net, float floor_rel, clamp_denoiser** out);
/* BF16 networks: on = 1 (the default) runs every 3x3x3 conv with 16k input channels and 16,
 * 32 or 64 output channels, forward and data gradient, on the tensor cores (tcgen05, BF16
 * operands, FP32 accumulation) wherever the level's shape allows it (nx = 16 with ny a
 * multiple of 8, or nx a multiple of 32 with ny a multiple of 4); on = 0 keeps them on the CUDA
 * cores.  Both round the same operands to bfloat16; only the order of the FP32 sums
 * differs.  The first conv (one input channel), the transposed convs, the 1x1 conv and the
 * weight gradients stay on the CUDA cores.  FP32 networks ignore the setting. */
clamp_status clamp_unet_set_tensor_cores(clamp_unet* u, int32_t on);
/* Synchronous check of the network's tensor-core waits since the last check: CLAMP_ETIMEOUT
 * (and the flag cleared) if a bounded wait gave up, else CLAMP_OK. */
clamp_status clamp_unet_check(clamp_unet* u);
/* One Adam step (Kingma and Ba, 2015, with bias correction; t >= 1 is the step number)
 * on the parameters from the current gradients. */
clamp_status clamp_unet_adam(clamp_unet* u, float lr, float beta1, float beta2, float eps, int32_t t,
                             void* stream);

#ifdef __cplusplus
}
#endif
#endif /* CLAMP_H */
