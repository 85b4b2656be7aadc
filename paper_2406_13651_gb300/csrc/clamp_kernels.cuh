// clamp_kernels.cuh -- launch interface of the CLAMP device passes (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace clamp {

// ---- bounds-checking build
// Compiled with -DCLAMP_BOUNDS_CHECK (a build of its own, libclamp_checked.so), the hot
// kernels test each global index they compute against the extent of its buffer before the
// access; an index outside skips the access and records its site code (the first one wins)
// in a device word of the translation unit.  The default build compiles the tests away.
#if defined(CLAMP_BOUNDS_CHECK)
static __device__ unsigned int s_bounds_site;
__device__ __forceinline__ bool clamp_in_bounds(long long i, long long n, unsigned int site) {
  if (i >= 0 && i < n) return true;
  atomicCAS(&s_bounds_site, 0u, site);
  return false;
}
#define CLAMP_IN_BOUNDS(i, n, site) ::clamp::clamp_in_bounds((long long)(i), (long long)(n), (site))
// Reads (and with reset clears) this translation unit's recorded site.
static inline cudaError_t bounds_site_local(unsigned int* site, bool reset) {
  cudaError_t e = cudaMemcpyFromSymbol(site, s_bounds_site, sizeof(unsigned int));
  if (e == cudaSuccess && reset) {
    const unsigned int zero = 0;
    e = cudaMemcpyToSymbol(s_bounds_site, &zero, sizeof(unsigned int));
  }
  return e;
}
#else
#define CLAMP_IN_BOUNDS(i, n, site) true
static inline cudaError_t bounds_site_local(unsigned int* site, bool) {
  *site = 0;
  return cudaSuccess;
}
#endif
// Per translation unit (band passes, set-up and prox/Mann passes, tensor-core convs).
cudaError_t bounds_site_band(unsigned int* site, bool reset);
cudaError_t bounds_site_kernels(unsigned int* site, bool reset);
cudaError_t bounds_site_tc(unsigned int* site, bool reset);

constexpr int NT = 256;   // threads per CTA in every FFT pass
constexpr int LC = 16;    // adjacent x-columns per CTA in the y / z passes

// Rows (x-lines) per CTA in the x passes.
__host__ __device__ constexpr int rows_per_cta(int N) { return N <= 32 ? 64 : (N <= 128 ? 32 : 16); }  // 96 -> 32, 192 -> 16

// Launch variants of the forward-agent FFT passes, chosen per pass by the autotuner:
// 0 = default radix plan and tile, 1 = alternative radix plan (PlanB), 2 = other tile
// schedule (half the rows per CTA in x passes, 32 columns per CTA in y / z passes),
// 3 = persistent CTAs with a two-stage cp.async pipeline (half the rows per tile in x
// passes, pipe_cols(N) columns in y / z passes).
constexpr int kVariants = 4;
__host__ __device__ constexpr int variant_rows(int N, int V) {
  return (V == 2 || V == 3) ? (rows_per_cta(N) / 2 < 8 ? 8 : rows_per_cta(N) / 2) : rows_per_cta(N);
}
__host__ __device__ constexpr int variant_cols(int V) { return V == 2 ? 32 : LC; }
// Columns per tile of the pipelined y / z passes (length-N transforms): two tile buffers
// must fit shared memory at least once per SM.
__host__ __device__ constexpr int pipe_cols(int N) { return N > 128 ? 8 : 16; }
// Passes of the forward agent: A_x, A_y, fused z, B_y, B_x.
struct AgentVariants {
  int v[5] = {0, 0, 0, 0, 0};
  int schedule = -1;   // forward-agent schedule: -1 not timed (band-limited when it fits), 0 full spectrum, 1 band-limited
  int band_x = 0;      // band-limited row pass: 0 rows_per_cta rows per CTA, 1 half as many, 2 mu / r' read late
};
// True if variant V of pass `pass` can run on the geometry.
bool variant_valid(int pass, int V, int nx, int ny, int nz);

struct Geom {
  int nx, ny, nz, L;
  long long n;  // nx * ny * nz
};

// Scalars shared by the passes of one forward-agent evaluation.
struct AgentScalars {
  float nv;        // sigma_w^2
  float alpha;     // mean(a^2)
  float floor;     // sigma_w^2 / alpha (noise floor of h)
  float sc_x, sc_y, sc_z;  // 1/sqrt(nx), 1/sqrt(ny), 1/sqrt(nz) (exact, from double)
};

// Reduction partial layout in the workspace (doubles).
struct Partials {
  double* s1;   // [L][pz]  ||Fd||^2        (z pass)
  double* s2;   // [L][pz]  ||a Fd||^2      (z pass)
  double* s4;   // [L][pz]  ||a y||^2       (z pass)
  double* s3;   // [L][px]  sum |d|^2 D     (x pass)
  int pz, px;
};

// Twiddle tables (host-computed, uploaded once per device).
cudaError_t upload_twiddles();
// Device address of the length-N twiddle table (N a supported axis length).
const float2* twiddle_table(int N);

// ---- band-limited forward agent (band_agent.cu): the gradient's transforms on the
// aperture's support only.  Support S = {(ky, kx): pupil != 0} (row by row), band
// B = {kx: any pupil(ky, kx) != 0}; counts padded to multiples of 16.
struct BandShape {
  int nS, nSp, nbx, nbxp;
};
struct BandTables {
  int nS, nSp, nbx, nbxp;
  int* sidx;      // [ny][nbxp] support index of (ky, band column b), or -1
  int* s_kykx;    // [nSp] ky * nx + kx of support column s (padding: 0)
  float* s_pup;   // [nSp] pupil value of support column s (padding: 0)
  int* bx;        // [nbxp] kx of band column b (padding: -1)
  int* bpos;      // [nx] band column of kx, or -1
};
struct BandArgs {
  BandTables t;
  int nx, ny, nz, L;          // L: looks (the launchers set it)
  long long n, plane;         // nx ny nz, nx ny
  const float2* y;            // [L][n] data (full spectrum layout)
  const float* window;        // [nz]
  const float2* mu;           // [L][n]
  const float* rprev;         // [L][n] r'
  float2* d;                  // [L][n] gradient direction out
  float2* Ms;                 // [L][nz][nSp] F mu on the support (kept across iterations)
  float2* Fd;                 // [L][nz][nSp] Gz, then F d on the support
  float2* band;               // [L][nz][ny][nbxp] band rows
  const float* gamma_prev;    // [L] step of the previous evaluation (spectrum update), or null
  float inv_nv, floor, sc_x, sc_y, sc_z;
  double *s1, *s2, *s3, *s4;  // partials: s1, s3 [L][px]; s2, s4 [L][pS]
  int px;
};
BandShape band_shape(const float* pupil_host, int nx, int ny);
size_t band_table_bytes(const BandShape& b, int nx, int ny);
BandTables band_tables_at(const BandShape& b, int nx, int ny, void* base);
int band_pS(const BandShape& b);
// S1 / S3 partial sums per look of the row pass (x_variant 0, 2: rows_per_cta rows per CTA; 1: half as many).
int band_px(int nx, int ny, int nz, int x_variant);
// Builds the device tables from the device pupil (one CTA).
cudaError_t launch_band_tables(const float* pupil, int nx, int ny, const BandTables& t, cudaStream_t st);
// Ms <- F mu on the support (first axis x over whole rows, then y and z on band / support).
cudaError_t launch_band_spectrum(const BandArgs& a, int L, cudaStream_t st);
// P1-P5 and the line search: d, F d on the support, gamma_l and the floored mu-residual per look.
// x_variant: 0 the row pass with rows_per_cta rows per CTA, 1 with half as many (three CTAs per SM), 2 the
// first with mu and r' prefetched to L2 and read after the inverse transform (three CTAs per SM).
cudaError_t launch_band_agent(const BandArgs& a, int L, float nv, float* gamma, double* mures, int x_variant,
                              cudaStream_t st);

// ---- forward agent (Alg. 2 steps 6-8): pass A (x, y), fused z pass, pass B (y, x)
// p.pz / p.px receive the partial counts per look the chosen variants produce.
cudaError_t launch_agent_fft(const Geom& g, const AgentScalars& s, const float2* mu, const float* rprev,
                             const float2* y, const float* pupil, const float* window, float4* T,
                             float2* U, Partials& p, const AgentVariants& var, cudaStream_t st);
// Variant 3 of pass `pass` (persistent, cp.async-pipelined); tw: the length-N twiddle
// table of that pass's axis.
cudaError_t launch_pipe_pass(int pass, const Geom& g, const AgentScalars& s, const float2* mu, const float* rprev,
                             const float2* y, const float* pupil, const float* window, float4* T, float2* U,
                             Partials& p, const float2* tw, cudaStream_t st);
// One forward-agent pass alone (for timing variants): pass in 0..4.
cudaError_t launch_agent_pass(int pass, int V, const Geom& g, const AgentScalars& s, const float2* mu,
                              const float* rprev, const float2* y, const float* pupil, const float* window,
                              float4* T, float2* U, Partials& p, cudaStream_t st);
// Largest partial counts per look over all variants (workspace sizing).
int max_pz(int nx, int ny);
int max_px(int nx, int ny, int nz);
// gamma_l = S1 / (S2 / sigma_w^2 + S3) and the floored mu-residual per look.
cudaError_t launch_gamma(const Geom& g, float nv, const Partials& p, float* gamma, double* mures,
                         cudaStream_t st);
// mean of mures[0..L) -> *out (device double)
cudaError_t launch_mean(const double* v, int L, double* out, cudaStream_t st);

// ---- pass C variants
struct PassC {
  const float2* d;
  float2* mu;
  float* r;          // [L+1][n]
  float* w;          // [L+1][n]
  float* wbar;       // [n] (MACE variants)
  const float* gamma;
  float nv, alpha, prox_var, beta;
  float inv_prox_var, inv_beta;   // 1 / prox_var, 1 / beta (host, rounded once)
  float ups_look, ups_prior, rho;
  double* part_num;  // CE partials (MACE variants)
  double* part_den;
  int* err;          // device error word (non-finite)
  int exact_prox;    // 1: exact cubic-root prox instead of the quadratic-surrogate step
  int closed_mu;     // 1: mu = d / (1 + sigma_w^2 / (r' + sigma_w^2)) with d holding F^H y (no aperture)
};
int passc_blocks(long long n);
// CTAs (and CE partial sums) of launch_pass_c_fused; at most passc_blocks(n).
int passc_fused_blocks(long long n, int L);
// mu <- mu + gamma_l d for all looks (the mu half of pass C: Eq. mu-update).
cudaError_t launch_mu_update(const Geom& g, float2* mu, const float2* d, const float* gamma, cudaStream_t st);
cudaError_t launch_pass_c_fused(const Geom& g, const PassC& c, cudaStream_t st);
cudaError_t launch_prox_only(const Geom& g, const PassC& c, cudaStream_t st);
cudaError_t launch_mace_only(const Geom& g, const PassC& c, cudaStream_t st);
// CE = sqrt(sum num / sum den) over nblk partials -> *ce (and ring[idx] if ring)
cudaError_t launch_ce_final(const double* num, const double* den, int nblk, double* ce, cudaStream_t st);

// ---- plain transforms and data set-up
cudaError_t launch_fft3(const Geom& g, const float2* in, float2* out, bool inverse, float sc_x, float sc_y,
                        float sc_z, cudaStream_t st);
cudaError_t launch_simulate(const Geom& g, const float* r, const float2* z, const float2* eta,
                            const float* pupil, const float* window, float sig_w, float2* y, float sc_x,
                            float sc_y, float sc_z, cudaStream_t st);
// mu = A^H y * mu_scale (inverse transform of a .* y); with pupil == nullptr, a = 1 (F^H y).
cudaError_t launch_adjoint(const Geom& g, const float2* y, const float* pupil, const float* window,
                           float mu_scale, float2* mu, float sc_x, float sc_y, float sc_z, cudaStream_t st);
// r0 = (1/L) sum |mu|^2 / mu_scale^2 (or r_init), floored at 1e-12 max, broadcast to r, w rows 0..L
cudaError_t launch_init_state(const Geom& g, const float2* mu, float mu_scale, const float* r_init, float* r,
                              float* w, float* max_part, int* nblk_out, cudaStream_t st);

// ---- prior agents
cudaError_t launch_gauss3(int nx, int ny, int nz, const float* in, float* out, float g0, float g1, cudaStream_t st);

// device error word helpers
cudaError_t launch_nonfinite_check(const float* x, long long count, int* err, cudaStream_t st);

}  // namespace clamp
