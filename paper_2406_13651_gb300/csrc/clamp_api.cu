// clamp_api.cu -- the C ABI (include/clamp.h): argument checks, workspace
// layout, per-device set-up and the CLAMP iteration driver (Alg. 2).
#include "../../include/clamp.h"
#include "clamp_internal.cuh"
#include "clamp_kernels.cuh"
#include "denoise.cuh"

#include <math.h>
#include <sys/mman.h>
#include <unistd.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <nvtx3/nvToolsExt.h>

#include <map>
#include <mutex>
#include <set>
#include <tuple>
#include <string>
#include <vector>

using namespace clamp;

// ---------------------------------------------------------------- errors

static thread_local std::string g_err;

clamp_status api_fail(clamp_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

static clamp_status cuda_fail(cudaError_t e, const char* where) {
  return api_fail(CLAMP_ECUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define API_CUDA(x, where)                             \
  do {                                                 \
    cudaError_t _e = (x);                              \
    if (_e != cudaSuccess) return cuda_fail(_e, where); \
  } while (0)

extern "C" const char* clamp_last_error(void) { return g_err.c_str(); }
extern "C" const char* clamp_version(void) { return "clamp-gb300 0.1 (sm_103a)"; }

extern "C" int32_t clamp_bounds_check(int32_t reset, uint32_t* site) {
  if (!site) return -(int32_t)api_fail(CLAMP_EINVAL, "clamp_bounds_check: null site");
  // each translation unit keeps its own record: report the first non-zero one
  unsigned int s[3] = {0u, 0u, 0u};
  cudaError_t e = bounds_site_band(&s[0], reset != 0);
  if (e == cudaSuccess) e = bounds_site_kernels(&s[1], reset != 0);
  if (e == cudaSuccess) e = bounds_site_tc(&s[2], reset != 0);
  if (e != cudaSuccess) return -(int32_t)cuda_fail(e, "clamp_bounds_check");
  *site = s[0] ? s[0] : (s[1] ? s[1] : s[2]);
#if defined(CLAMP_BOUNDS_CHECK)
  return 1;
#else
  return 0;
#endif
}

// ---------------------------------------------------------------- per-device set-up

static std::mutex g_dev_mu;
static std::set<int> g_dev_ready;

clamp_status api_ensure_device() {
  int dev = -1;
  API_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_dev_mu);
  if (g_dev_ready.count(dev)) return CLAMP_OK;
  API_CUDA(upload_twiddles(), "twiddle upload");
  g_dev_ready.insert(dev);
  return CLAMP_OK;
}

// ---------------------------------------------------------------- validation

extern "C" int32_t clamp_supported_length(int32_t n) {
  return (n == 8 || n == 16 || n == 32 || n == 64 || n == 96 || n == 128 || n == 192 || n == 256) ? 1 : 0;
}

static clamp_status check_shape(int nx, int ny, int nz) {
  if (!clamp_supported_length(nx) || !clamp_supported_length(ny) || !clamp_supported_length(nz))
    return api_fail(CLAMP_EUNSUPPORTED, "volume %dx%dx%d (nx,ny,nz): axis lengths must be 8, 16, 32, 64, 96, 128, 192 or 256",
                nx, ny, nz);
  if (nx % LC) return api_fail(CLAMP_EUNSUPPORTED, "nx=%d must be a multiple of %d", nx, LC);
  return CLAMP_OK;
}

extern "C" clamp_status clamp_check_params(const clamp_params* p) {
  if (!p) return api_fail(CLAMP_EINVAL, "params is NULL");
  clamp_status s = check_shape(p->nx, p->ny, p->nz);
  if (s != CLAMP_OK) return s;
  if (p->looks < 1 || p->looks > 4096) return api_fail(CLAMP_EINVAL, "looks=%d must be in [1, 4096]", p->looks);
  if (!(p->noise_var > 0.f) || !isfinite(p->noise_var)) return api_fail(CLAMP_EINVAL, "noise_var must be > 0");
  if (!(p->prox_var > 0.f) || !isfinite(p->prox_var)) return api_fail(CLAMP_EINVAL, "prox_var must be > 0");
  if (!(p->rho > 0.f && p->rho < 1.f)) return api_fail(CLAMP_EINVAL, "rho=%g must be in (0, 1)", p->rho);
  if (!(p->prior_weight > 0.f && p->prior_weight < 1.f))
    return api_fail(CLAMP_EINVAL, "prior_weight=%g must be in (0, 1)", p->prior_weight);
  if (p->max_iters < 0) return api_fail(CLAMP_EINVAL, "max_iters must be >= 0");
  if (p->k0 < 0) return api_fail(CLAMP_EINVAL, "k0 must be >= 0");
  if (!(p->tol >= 0.0)) return api_fail(CLAMP_EINVAL, "tol must be >= 0");
  if (p->init_mu_steps < 0 || p->init_mu_steps > 1000) return api_fail(CLAMP_EINVAL, "init_mu_steps must be in [0, 1000]");
  if ((p->flags & CLAMP_FLAG_PRIOR_CONCURRENT) && (p->flags & CLAMP_FLAG_PRIOR_SERIAL))
    return api_fail(CLAMP_EINVAL, "CLAMP_FLAG_PRIOR_CONCURRENT and CLAMP_FLAG_PRIOR_SERIAL are exclusive");
  if ((p->flags & CLAMP_FLAG_FULL_SPECTRUM) && (p->flags & CLAMP_FLAG_BAND_SPECTRUM))
    return api_fail(CLAMP_EINVAL, "CLAMP_FLAG_FULL_SPECTRUM and CLAMP_FLAG_BAND_SPECTRUM are exclusive");
  return CLAMP_OK;
}

// The prior agent's schedule (the size rule and flags documented with CLAMP_FLAG_PRIOR_*).
static bool prior_concurrent(const clamp_params* p) {
  if (p->flags & CLAMP_FLAG_PRIOR_CONCURRENT) return true;
  if (p->flags & CLAMP_FLAG_PRIOR_SERIAL) return false;
  return (long long)p->nx * p->ny * p->nz * p->looks <= (1LL << 25);
}

extern "C" int32_t clamp_prior_concurrent(const clamp_params* p) {
  if (clamp_check_params(p) != CLAMP_OK) return -1;
  return prior_concurrent(p) ? 1 : 0;
}

// ---------------------------------------------------------------- workspace layout

namespace {
struct Arena {
  size_t off = 0;
  template <class T>
  size_t take(long long count) {
    const size_t o = off;
    off += ((size_t)count * sizeof(T) + 255) & ~(size_t)255;
    return o;
  }
};

struct AgentLayout {
  size_t T, U, s1, s2, s4, s3, gamma, mures, num, den, maxp, scal, err;
  int pz, px, nbc;
  size_t bytes;
};

AgentLayout agent_layout(const clamp_params* p) {
  AgentLayout a{};
  const long long n = (long long)p->nx * p->ny * p->nz, L = p->looks;
  a.pz = max_pz(p->nx, p->ny);              // largest partial counts over all launch variants
  a.px = max_px(p->nx, p->ny, p->nz);
  a.nbc = passc_blocks(n);
  Arena ar;
  a.T = ar.take<float4>(L * n);
  a.U = ar.take<float2>(L * n);
  a.s1 = ar.take<double>(L * a.pz);
  a.s2 = ar.take<double>(L * a.pz);
  a.s4 = ar.take<double>(L * a.pz);
  a.s3 = ar.take<double>(L * a.px);
  a.gamma = ar.take<float>(L);
  a.mures = ar.take<double>(L);
  a.num = ar.take<double>(a.nbc);
  a.den = ar.take<double>(a.nbc);
  a.maxp = ar.take<float>(a.nbc);
  a.scal = ar.take<double>(8);
  a.err = ar.take<int>(8);
  a.bytes = ar.off;
  return a;
}

// The band-limited schedule's arrays inside the agent scratch's T region (16 bytes per
// voxel-look): tables, F mu and F d on the support, band rows.
struct BandLayout {
  size_t tables, Ms, Fd, band, bytes;
};

BandLayout band_layout(const clamp_params* p, const BandShape& b) {
  BandLayout bl{};
  const long long L = p->looks;
  Arena ar;
  bl.tables = ar.off;
  ar.off += band_table_bytes(b, p->nx, p->ny);
  bl.Ms = ar.take<float2>(L * p->nz * (long long)b.nSp);
  bl.Fd = ar.take<float2>(L * p->nz * (long long)b.nSp);
  bl.band = ar.take<float2>(L * p->nz * (long long)p->ny * b.nbxp);
  bl.bytes = ar.off;
  return bl;
}

bool band_fits(const clamp_params* p, const BandShape& b) {
  const long long n = (long long)p->nx * p->ny * p->nz;
  return band_layout(p, b).bytes <= (size_t)(16 * n * p->looks);
}

struct ReconLayout {
  size_t mu, r, w, ce_ring, mu_ring, agent, den;
  size_t bytes;
};

ReconLayout recon_layout(const clamp_params* p, const clamp_denoiser* den) {
  ReconLayout r{};
  const long long n = (long long)p->nx * p->ny * p->nz, L = p->looks;
  Arena ar;
  r.mu = ar.take<float2>(L * n);
  r.r = ar.take<float>((L + 1) * n);
  r.w = ar.take<float>((L + 1) * n);
  const int ring = p->max_iters > 0 ? p->max_iters : 1;
  r.ce_ring = ar.take<double>(ring);
  r.mu_ring = ar.take<double>(ring);
  r.agent = ar.off;
  r.den = ar.off + agent_layout(p).bytes;  // the denoiser scratch follows the agent scratch
  ar.off += agent_layout(p).bytes + ((denoise_ws_bytes(den, p->nx, p->ny, p->nz) + 255) & ~(size_t)255);
  r.bytes = ar.off;
  return r;
}

template <class T>
T* at(void* base, size_t off) {
  return reinterpret_cast<T*>(static_cast<char*>(base) + off);
}

}  // namespace

using Derived = ReconPlan;

// alpha = mean(a^2) for the separable aperture a = window[kz] * pupil[ky][kx] (host, double).
clamp_status recon_prepare(const clamp_params* p, const float* pupil, const float* window, cudaStream_t st,
                           ReconPlan* d) {
  d->g.nx = p->nx;
  d->g.ny = p->ny;
  d->g.nz = p->nz;
  d->g.L = p->looks;
  d->g.n = (long long)p->nx * p->ny * p->nz;
  d->band = BandShape{};
  d->band_fits = false;
  if (p->flags & CLAMP_FLAG_NO_APERTURE) {  // a = 1: alpha = 1, nothing to read back
    d->alpha = 1.0;
    d->s.nv = p->noise_var;
    d->s.alpha = 1.0f;
    d->s.floor = p->noise_var;
    d->s.sc_x = (float)(1.0 / sqrt((double)p->nx));
    d->s.sc_y = (float)(1.0 / sqrt((double)p->ny));
    d->s.sc_z = (float)(1.0 / sqrt((double)p->nz));
    return CLAMP_OK;
  }
  std::vector<float> hp((size_t)p->nx * p->ny), hw(p->nz);
  API_CUDA(cudaMemcpyAsync(hp.data(), pupil, hp.size() * sizeof(float), cudaMemcpyDeviceToHost, st), "pupil read");
  API_CUDA(cudaMemcpyAsync(hw.data(), window, hw.size() * sizeof(float), cudaMemcpyDeviceToHost, st), "window read");
  API_CUDA(cudaStreamSynchronize(st), "pupil read");
  return recon_prepare_host(p, hp.data(), hw.data(), d);
}

// The same from host copies of the pupil and window (no device access, no synchronisation).
clamp_status recon_prepare_host(const clamp_params* p, const float* hp, const float* hw, ReconPlan* d) {
  d->g.nx = p->nx;
  d->g.ny = p->ny;
  d->g.nz = p->nz;
  d->g.L = p->looks;
  d->g.n = (long long)p->nx * p->ny * p->nz;
  d->band = BandShape{};
  d->band_fits = false;
  const size_t np = (size_t)p->nx * p->ny;
  double sp = 0, sw = 0;
  for (size_t i = 0; i < np; ++i) {
    if (!isfinite(hp[i])) return api_fail(CLAMP_EINVAL, "pupil has a non-finite value");
    sp += (double)hp[i] * hp[i];
  }
  for (int i = 0; i < p->nz; ++i) {
    if (!isfinite(hw[i])) return api_fail(CLAMP_EINVAL, "window has a non-finite value");
    sw += (double)hw[i] * hw[i];
  }
  const double alpha = (sp / np) * (sw / p->nz);
  if (!(alpha > 0)) return api_fail(CLAMP_EINVAL, "aperture is identically zero (alpha = 0)");
  d->alpha = alpha;
  d->band = band_shape(hp, p->nx, p->ny);
  d->band_fits = band_fits(p, d->band);
  d->s.nv = p->noise_var;
  d->s.alpha = (float)alpha;
  d->s.floor = (float)((double)p->noise_var / alpha);
  d->s.sc_x = (float)(1.0 / sqrt((double)p->nx));
  d->s.sc_y = (float)(1.0 / sqrt((double)p->ny));
  d->s.sc_z = (float)(1.0 / sqrt((double)p->nz));
  return CLAMP_OK;
}

namespace {
Partials partials(const AgentLayout& a, void* ws) {
  Partials p{};
  p.s1 = at<double>(ws, a.s1);
  p.s2 = at<double>(ws, a.s2);
  p.s4 = at<double>(ws, a.s4);
  p.s3 = at<double>(ws, a.s3);
  p.pz = a.pz;
  p.px = a.px;
  return p;
}

clamp_status need_ptrs(std::initializer_list<const void*> ptrs, const char* what) {
  for (const void* q : ptrs)
    if (!q) return api_fail(CLAMP_EINVAL, "%s: NULL array argument", what);
  return CLAMP_OK;
}

clamp_status check_ws(void* ws, size_t have, size_t need, const char* what) {
  if (!ws) return api_fail(CLAMP_EINVAL, "%s: workspace is NULL", what);
  if (((uintptr_t)ws) & 255) return api_fail(CLAMP_EINVAL, "%s: workspace must be 256-byte aligned", what);
  if (have < need) return api_fail(CLAMP_ENOMEM, "%s: workspace %zu bytes < %zu needed", what, have, need);
  return CLAMP_OK;
}
}  // namespace

#define API_TRY(x)                       \
  do {                                   \
    clamp_status _s = (x);               \
    if (_s != CLAMP_OK) return _s;       \
  } while (0)

extern "C" size_t clamp_workspace_size(const clamp_params* p) {
  if (clamp_check_params(p) != CLAMP_OK) return 0;
  return agent_layout(p).bytes;
}

extern "C" size_t clamp_reconstruct_workspace_size(const clamp_params* p, const clamp_denoiser* den) {
  if (clamp_check_params(p) != CLAMP_OK) return 0;
  return recon_layout(p, den).bytes;
}

// ---------------------------------------------------------------- entry points

extern "C" clamp_status clamp_fft3(int32_t nx, int32_t ny, int32_t nz, int32_t batch, const float* in, float* out,
                                   int32_t inverse, void* stream) {
  API_TRY(check_shape(nx, ny, nz));
  if (batch < 1) return api_fail(CLAMP_EINVAL, "batch=%d must be >= 1", batch);
  API_TRY(need_ptrs({in, out}, "clamp_fft3"));
  API_TRY(api_ensure_device());
  Geom g{nx, ny, nz, batch, (long long)nx * ny * nz};
  API_CUDA(launch_fft3(g, reinterpret_cast<const float2*>(in), reinterpret_cast<float2*>(out), inverse != 0,
                       (float)(1.0 / sqrt((double)nx)), (float)(1.0 / sqrt((double)ny)),
                       (float)(1.0 / sqrt((double)nz)), (cudaStream_t)stream),
           "clamp_fft3 launch");
  return CLAMP_OK;
}

extern "C" clamp_status clamp_simulate(const clamp_params* p, const float* r, const float* speckle, const float* noise,
                                       const float* pupil, const float* window, float* y, void* stream) {
  API_TRY(clamp_check_params(p));
  API_TRY(need_ptrs({r, speckle, noise, pupil, window, y}, "clamp_simulate"));
  API_TRY(api_ensure_device());
  Geom g{p->nx, p->ny, p->nz, p->looks, (long long)p->nx * p->ny * p->nz};
  API_CUDA(launch_simulate(g, r, reinterpret_cast<const float2*>(speckle), reinterpret_cast<const float2*>(noise),
                           pupil, window, (float)sqrt((double)p->noise_var), reinterpret_cast<float2*>(y),
                           (float)(1.0 / sqrt((double)p->nx)), (float)(1.0 / sqrt((double)p->ny)),
                           (float)(1.0 / sqrt((double)p->nz)), (cudaStream_t)stream),
           "clamp_simulate launch");
  return CLAMP_OK;
}

static clamp_status do_init(const clamp_params* p, const Derived& d, const float* y, const float* pupil,
                            const float* window, const float* r_init, float2* mu, float* r, float* w,
                            const AgentLayout& al, void* ws, cudaStream_t st) {
  const double mu_scale = (p->flags & CLAMP_FLAG_MU_INIT_NO_ALPHA) ? 1.0 : 1.0 / d.alpha;
  const bool noap = (p->flags & CLAMP_FLAG_NO_APERTURE) != 0;
  API_CUDA(launch_adjoint(d.g, reinterpret_cast<const float2*>(y), noap ? nullptr : pupil, window, (float)mu_scale,
                          mu, d.s.sc_x, d.s.sc_y, d.s.sc_z, st),
           "adjoint launch");
  API_CUDA(launch_init_state(d.g, mu, (float)mu_scale, r_init, r, w, at<float>(ws, al.maxp), nullptr, st),
           "init launch");
  return CLAMP_OK;
}

static clamp_status do_init_warm(const clamp_params* p, const Derived& d, const float* y, const float* pupil,
                                 const float* window, const float* r_init, float2* mu, float* r, float* w,
                                 const AgentLayout& al, void* ws, cudaStream_t st);

extern "C" clamp_status clamp_init(const clamp_params* p, const float* y, const float* pupil, const float* window,
                                   const float* r_init, float* mu, float* r, float* w, void* ws, size_t ws_bytes,
                                   void* stream) {
  API_TRY(clamp_check_params(p));
  API_TRY(need_ptrs({y, pupil, window, mu, r, w}, "clamp_init"));
  const AgentLayout al = agent_layout(p);
  API_TRY(check_ws(ws, ws_bytes, al.bytes, "clamp_init"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  Derived d;
  API_TRY(recon_prepare(p, pupil, window, st, &d));
  return do_init_warm(p, d, y, pupil, window, r_init, reinterpret_cast<float2*>(mu), r, w, al, ws, st);
}

// The initial image of Alg. 2 on its own: r0 = (1/L) sum_l |A^H y_l / alpha|^2 (the
// speckle average), floored as the initialisation floors it.  mu goes to the workspace's
// U region and the broadcast state rows to its T region; row L of r is r0.
extern "C" clamp_status clamp_speckle_average(const clamp_params* p, const float* y, const float* pupil,
                                              const float* window, float* r0, void* ws, size_t ws_bytes,
                                              void* stream) {
  API_TRY(clamp_check_params(p));
  API_TRY(need_ptrs({y, pupil, window, r0}, "clamp_speckle_average"));
  const AgentLayout al = agent_layout(p);
  API_TRY(check_ws(ws, ws_bytes, al.bytes, "clamp_speckle_average"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  Derived d;
  API_TRY(recon_prepare(p, pupil, window, st, &d));
  const long long n = d.g.n, L = d.g.L;
  float* rs = at<float>(ws, al.T);          // [L+1][n]
  float* wsr = rs + (L + 1) * n;            // [L+1][n]  (4 L n floats >= 2 (L+1) n)
  API_TRY(do_init(p, d, y, pupil, window, nullptr, at<float2>(ws, al.U), rs, wsr, al, ws, st));
  API_CUDA(cudaMemcpyAsync(r0, rs + L * n, sizeof(float) * n, cudaMemcpyDeviceToDevice, st), "r0 copy");
  return CLAMP_OK;
}

static float beta_of(int k) { return (float)(1.0 + 2.0 / log((double)k + 1.0)); }

// ---------------------------------------------------------------- autotuner cache

namespace {
struct TuneKey {
  int dev, nx, ny, nz, L;
  bool operator<(const TuneKey& o) const {
    return std::tie(dev, nx, ny, nz, L) < std::tie(o.dev, o.nx, o.ny, o.nz, o.L);
  }
};
std::mutex g_tune_mu;
std::map<TuneKey, AgentVariants> g_tune;

TuneKey tune_key(const Geom& g) {
  int dev = 0;
  cudaGetDevice(&dev);
  return TuneKey{dev, g.nx, g.ny, g.nz, g.L};
}

AgentVariants tuned_variants(const Geom& g) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  auto it = g_tune.find(tune_key(g));
  return it == g_tune.end() ? AgentVariants{} : it->second;
}
}  // namespace

// Whether the forward agents run the band-limited schedule (CLAMP_FLAG_*_SPECTRUM, the
// autotuner's cached choice, else whenever its arrays fit the scratch).
static bool use_band(const clamp_params* p, const Derived& d) {
  if (!d.band_fits || (p->flags & CLAMP_FLAG_NO_APERTURE) || (p->flags & CLAMP_FLAG_FULL_SPECTRUM)) return false;
  if (p->flags & CLAMP_FLAG_BAND_SPECTRUM) return true;
  return tuned_variants(d.g).schedule != 0;
}

static BandArgs band_args(const clamp_params* p, const Derived& d, const float* y, const float* window,
                          const float2* mu, const float* r, const AgentLayout& al, void* ws) {
  const BandLayout bl = band_layout(p, d.band);
  void* T = at<char>(ws, al.T);
  BandArgs a{};
  a.t = band_tables_at(d.band, p->nx, p->ny, at<char>(T, bl.tables));
  a.nx = p->nx;
  a.ny = p->ny;
  a.nz = p->nz;
  a.n = d.g.n;
  a.plane = (long long)p->nx * p->ny;
  a.y = reinterpret_cast<const float2*>(y);
  a.window = window;
  a.mu = mu;
  a.rprev = r;
  a.d = at<float2>(ws, al.U);
  a.Ms = at<float2>(T, bl.Ms);
  a.Fd = at<float2>(T, bl.Fd);
  a.band = at<float2>(T, bl.band);
  a.inv_nv = 1.0f / p->noise_var;
  a.floor = d.s.floor;
  a.sc_x = d.s.sc_x;
  a.sc_y = d.s.sc_y;
  a.sc_z = d.s.sc_z;
  a.s1 = at<double>(ws, al.s1);
  a.s2 = at<double>(ws, al.s2);
  a.s3 = at<double>(ws, al.s3);
  a.s4 = at<double>(ws, al.s4);
  a.L = p->looks;
  a.px = band_px(p->nx, p->ny, p->nz, 0);
  return a;
}

// Forward-agent gradient, line search and mu-residual of every look into the agent scratch
// (d in U, gamma, mures).  Band-limited schedule: `fresh` builds the support tables and
// F mu first; otherwise F mu is the previous call's, advanced here by the previous gamma F d.
static clamp_status agent_ffts(const clamp_params* p, const Derived& d, const float* y, const float* pupil,
                               const float* window, const float2* mu, const float* r, const AgentLayout& al,
                               void* ws, bool fresh, cudaStream_t st) {
  if (use_band(p, d)) {
    BandArgs a = band_args(p, d, y, window, mu, r, al, ws);
    if (fresh) {
      API_CUDA(launch_band_tables(pupil, p->nx, p->ny, a.t, st), "support tables");
      API_CUDA(launch_band_spectrum(a, p->looks, st), "F mu on the support");
    }
    a.gamma_prev = fresh ? nullptr : at<float>(ws, al.gamma);
    API_CUDA(launch_band_agent(a, p->looks, p->noise_var, at<float>(ws, al.gamma), at<double>(ws, al.mures),
                               tuned_variants(d.g).band_x, st),
             "band-limited forward-agent passes");
    return CLAMP_OK;
  }
  Partials pt = partials(al, ws);
  API_CUDA(launch_agent_fft(d.g, d.s, mu, r, reinterpret_cast<const float2*>(y), pupil, window,
                            at<float4>(ws, al.T), at<float2>(ws, al.U), pt, tuned_variants(d.g), st),
           "forward-agent FFT passes");
  API_CUDA(launch_gamma(d.g, d.s.nv, pt, at<float>(ws, al.gamma), at<double>(ws, al.mures), st), "line search");
  return CLAMP_OK;
}

// Initialisation (do_init) and, when the caller gives r_init (a warm start), p->init_mu_steps
// mu updates of every forward agent with r' = r_init fixed (Alg. 2 steps 5-8 without the
// prox): the back-projected mu of the initialisation is far from the posterior mean that
// r_init implies, and the first iterations would otherwise spend themselves repairing it.
static clamp_status do_init_warm(const clamp_params* p, const Derived& d, const float* y, const float* pupil,
                                 const float* window, const float* r_init, float2* mu, float* r, float* w,
                                 const AgentLayout& al, void* ws, cudaStream_t st) {
  API_TRY(do_init(p, d, y, pupil, window, r_init, mu, r, w, al, ws, st));
  if (!r_init || p->init_mu_steps <= 0 || (p->flags & CLAMP_FLAG_NO_APERTURE)) return CLAMP_OK;
  for (int s = 0; s < p->init_mu_steps; ++s) {
    API_TRY(agent_ffts(p, d, y, pupil, window, mu, r, al, ws, s == 0, st));
    API_CUDA(launch_mu_update(d.g, mu, at<float2>(ws, al.U), at<float>(ws, al.gamma), st), "mu update");
  }
  return CLAMP_OK;
}

// Times every valid launch variant of each forward-agent pass on the agent scratch `ws`
// (contents irrelevant: the passes have no data-dependent control flow) and stores the
// fastest per pass for this geometry.  Synchronises `st`.
clamp_status autotune_agent(const clamp_params* p, const ReconPlan& d, const float* y, const float* pupil,
                            const float* window, void* ws, cudaStream_t st, AgentVariants* out) {
  const AgentLayout al = agent_layout(p);
  float4* T = at<float4>(ws, al.T);
  float2* U = at<float2>(ws, al.U);
  const float2* mu = U;                                  // timing only: any buffers of the right size
  const float* rp = reinterpret_cast<const float*>(U);
  cudaEvent_t e0, e1;
  API_CUDA(cudaEventCreate(&e0), "event");
  API_CUDA(cudaEventCreate(&e1), "event");
  AgentVariants best;
  float full_ms = 0.f;
  for (int pass = 0; pass < 5; ++pass) {
    float best_ms = 1e30f;
    for (int V = 0; V < kVariants; ++V) {
      if (!variant_valid(pass, V, p->nx, p->ny, p->nz)) continue;
      Partials pt = partials(al, ws);
      cudaError_t e = launch_agent_pass(pass, V, d.g, d.s, mu, rp, reinterpret_cast<const float2*>(y), pupil, window,
                                        T, U, pt, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
        e = launch_agent_pass(pass, V, d.g, d.s, mu, rp, reinterpret_cast<const float2*>(y), pupil, window, T, U, pt,
                              st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return cuda_fail(e, "autotune");
      }
      if (ms < best_ms) {
        best_ms = ms;
        best.v[pass] = V;
      }
    }
    full_ms += best_ms;
  }
  // the band-limited schedule as a whole, with each row-pass variant (tables from the real
  // pupil: its indices come from them)
  best.schedule = 0;
  if (d.band_fits && !(p->flags & CLAMP_FLAG_NO_APERTURE)) {
    BandArgs a = band_args(p, d, y, window, mu, rp, al, ws);
    a.gamma_prev = at<float>(ws, al.gamma);
    float band_ms = 1e30f;
    cudaError_t e = launch_band_tables(pupil, p->nx, p->ny, a.t, st);
    for (int xv = 0; xv < 3 && e == cudaSuccess; ++xv) {
      e = launch_band_agent(a, p->looks, p->noise_var, at<float>(ws, al.gamma), at<double>(ws, al.mures), xv, st);
      if (e == cudaSuccess) e = cudaEventRecord(e0, st);
      for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep)
        e = launch_band_agent(a, p->looks, p->noise_var, at<float>(ws, al.gamma), at<double>(ws, al.mures), xv,
                              st);
      if (e == cudaSuccess) e = cudaEventRecord(e1, st);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && ms < band_ms) {
        band_ms = ms;
        best.band_x = xv;
      }
    }
    if (e != cudaSuccess) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return cuda_fail(e, "autotune (band-limited schedule)");
    }
    best.schedule = band_ms <= full_ms ? 1 : 0;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[tune_key(d.g)] = best;
  }
  if (out) *out = best;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_autotune(const clamp_params* p, const float* y, const float* pupil, const float* window,
                                       void* ws, size_t ws_bytes, void* stream, int32_t* variants_out) {
  API_TRY(clamp_check_params(p));
  API_TRY(need_ptrs({y, pupil, window}, "clamp_autotune"));
  API_TRY(check_ws(ws, ws_bytes, agent_layout(p).bytes, "clamp_autotune"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  Derived d;
  API_TRY(recon_prepare(p, pupil, window, st, &d));
  AgentVariants v;
  API_TRY(autotune_agent(p, d, y, pupil, window, ws, st, &v));
  if (variants_out)
    for (int i = 0; i < 5; ++i) variants_out[i] = v.v[i];
  return CLAMP_OK;
}

extern "C" clamp_status clamp_agent_schedule(const clamp_params* p, const float* pupil, const float* window,
                                             void* stream, int32_t* info) {
  API_TRY(clamp_check_params(p));
  API_TRY(need_ptrs({pupil, window, info}, "clamp_agent_schedule"));
  API_TRY(api_ensure_device());
  Derived d;
  API_TRY(recon_prepare(p, pupil, window, (cudaStream_t)stream, &d));
  info[0] = use_band(p, d) ? 1 : 0;
  info[1] = d.band.nS;
  info[2] = d.band.nbx;
  info[3] = d.band_fits ? 1 : 0;
  info[4] = tuned_variants(d.g).band_x;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_autotune_set_band(const clamp_params* p, int32_t row_variant) {
  API_TRY(clamp_check_params(p));
  if (row_variant < 0 || row_variant > 2)
    return api_fail(CLAMP_EINVAL, "clamp_autotune_set_band: row_variant=%d must be 0, 1 or 2", row_variant);
  Geom g{p->nx, p->ny, p->nz, p->looks, (long long)p->nx * p->ny * p->nz};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(g)].band_x = row_variant;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_autotune_set(const clamp_params* p, const int32_t* variants) {
  API_TRY(clamp_check_params(p));
  if (!variants) return api_fail(CLAMP_EINVAL, "clamp_autotune_set: variants is NULL");
  AgentVariants v;
  for (int i = 0; i < 5; ++i) {
    if (!variant_valid(i, variants[i], p->nx, p->ny, p->nz))
      return api_fail(CLAMP_EINVAL, "clamp_autotune_set: variant %d not valid for pass %d", variants[i], i);
    v.v[i] = variants[i];
  }
  Geom g{p->nx, p->ny, p->nz, p->looks, (long long)p->nx * p->ny * p->nz};
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[tune_key(g)] = v;
  return CLAMP_OK;
}

static PassC passc_args(const clamp_params* p, const Derived& d, const AgentLayout& al, void* ws, float2* mu,
                        float* r, float* w, float* wbar, int k) {
  PassC c{};
  c.d = at<float2>(ws, al.U);
  c.mu = mu;
  c.r = r;
  c.w = w;
  c.wbar = wbar;
  c.gamma = at<float>(ws, al.gamma);
  c.nv = p->noise_var;
  c.alpha = d.s.alpha;
  c.prox_var = p->prox_var;
  c.beta = k > 0 ? beta_of(k) : 1.0f;
  c.inv_prox_var = (float)(1.0 / (double)p->prox_var);
  c.inv_beta = (float)(1.0 / (double)c.beta);
  c.ups_look = (float)((1.0 - (double)p->prior_weight) / p->looks);
  c.ups_prior = p->prior_weight;
  c.rho = p->rho;
  c.part_num = at<double>(ws, al.num);
  c.part_den = at<double>(ws, al.den);
  c.err = at<int>(ws, al.err);
  c.exact_prox = (p->flags & CLAMP_FLAG_EXACT_PROX) ? 1 : 0;
  c.closed_mu = (p->flags & CLAMP_FLAG_NO_APERTURE) ? 1 : 0;
  return c;
}

// No-aperture ablation: U <- F^H y for all looks (the closed-form mu update reads it).
static clamp_status ablation_prepare(const Derived& d, const float* y, const AgentLayout& al, void* ws,
                                     cudaStream_t st) {
  API_CUDA(launch_adjoint(d.g, reinterpret_cast<const float2*>(y), nullptr, nullptr, 1.0f, at<float2>(ws, al.U),
                          d.s.sc_x, d.s.sc_y, d.s.sc_z, st),
           "F^H y");
  return CLAMP_OK;
}

extern "C" clamp_status clamp_forward_prox(const clamp_params* p, int32_t k, const float* y, const float* pupil,
                                           const float* window, float* mu, float* r, const float* w,
                                           double* mu_residual, void* ws, size_t ws_bytes, void* stream) {
  API_TRY(clamp_check_params(p));
  if (k < 1) return api_fail(CLAMP_EINVAL, "iteration index k=%d must be >= 1", k);
  API_TRY(need_ptrs({y, pupil, window, mu, r, w}, "clamp_forward_prox"));
  const AgentLayout al = agent_layout(p);
  API_TRY(check_ws(ws, ws_bytes, al.bytes, "clamp_forward_prox"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  Derived d;
  API_TRY(recon_prepare(p, pupil, window, st, &d));
  if (p->flags & CLAMP_FLAG_NO_APERTURE) {
    API_TRY(ablation_prepare(d, y, al, ws, st));
    if (mu_residual) API_CUDA(cudaMemsetAsync(mu_residual, 0, sizeof(double), st), "mu residual");
  } else {
    API_TRY(agent_ffts(p, d, y, pupil, window, reinterpret_cast<float2*>(mu), r, al, ws, true, st));
    if (mu_residual) API_CUDA(launch_mean(at<double>(ws, al.mures), p->looks, mu_residual, st), "mu residual");
  }
  PassC c = passc_args(p, d, al, ws, reinterpret_cast<float2*>(mu), r, const_cast<float*>(w), nullptr, k);
  c.err = nullptr;
  API_CUDA(launch_prox_only(d.g, c, st), "prox pass");
  return CLAMP_OK;
}

extern "C" clamp_status clamp_mace_step(const clamp_params* p, const float* r, float* w, float* wbar,
                                        double* ce_residual, void* ws, size_t ws_bytes, void* stream) {
  API_TRY(clamp_check_params(p));
  API_TRY(need_ptrs({r, w, wbar}, "clamp_mace_step"));
  const AgentLayout al = agent_layout(p);
  API_TRY(check_ws(ws, ws_bytes, al.bytes, "clamp_mace_step"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  Derived d{};
  d.g = Geom{p->nx, p->ny, p->nz, p->looks, (long long)p->nx * p->ny * p->nz};
  PassC c = passc_args(p, d, al, ws, nullptr, const_cast<float*>(r), w, wbar, 0);
  c.err = nullptr;
  API_CUDA(launch_mace_only(d.g, c, st), "MACE pass");
  if (ce_residual) API_CUDA(launch_ce_final(c.part_num, c.part_den, al.nbc, ce_residual, st), "CE residual");
  return CLAMP_OK;
}

extern "C" clamp_status clamp_denoise(const clamp_denoiser* den, const float* w_prior, float* r_prior, int32_t nx,
                                      int32_t ny, int32_t nz, void* ws, size_t ws_bytes, void* stream) {
  if (!den) return api_fail(CLAMP_EINVAL, "denoiser is NULL");
  if (nx < 1 || ny < 1 || nz < 1 || nx > 4096 || ny > 4096 || nz > 4096)
    return api_fail(CLAMP_EINVAL, "denoiser volume %dx%dx%d out of range", nx, ny, nz);
  API_TRY(need_ptrs({w_prior, r_prior}, "clamp_denoise"));
  if (!denoise_supports(den, nx, ny, nz))
    return api_fail(CLAMP_EUNSUPPORTED, "BF16 CNN prior needs nx %% 128 == 0, ny %% 4 == 0, nz %% 2 == 0 (got %dx%dx%d)",
                nx, ny, nz);
  const size_t need = denoise_ws_bytes(den, nx, ny, nz);
  if (need) API_TRY(check_ws(ws, ws_bytes, need, "clamp_denoise"));
  API_TRY(api_ensure_device());
  API_CUDA(denoise_apply(den, w_prior, r_prior, nx, ny, nz, ws, nullptr, (cudaStream_t)stream), "denoiser");
  return CLAMP_OK;
}

extern "C" size_t clamp_denoise_workspace_size(const clamp_denoiser* den, int32_t nx, int32_t ny, int32_t nz) {
  return den ? denoise_ws_bytes(den, nx, ny, nz) : 0;
}

// ---------------------------------------------------------------- driver (Alg. 2)

static size_t iterate_ws_bytes(const clamp_params* p, const clamp_denoiser* den) {
  return agent_layout(p).bytes + ((denoise_ws_bytes(den, p->nx, p->ny, p->nz) + 255) & ~(size_t)255);
}

extern "C" size_t clamp_iterate_workspace_size(const clamp_params* p, const clamp_denoiser* den) {
  if (clamp_check_params(p) != CLAMP_OK) return 0;
  return iterate_ws_bytes(p, den);
}

// The prior agent's side stream and its fork/join events: one set per host thread and
// device, created on first use outside stream capture (so no two callers, and no capture
// on another thread, share them) and kept for the thread's lifetime (three handles; no
// destructor, which could run after the CUDA runtime has unloaded at process exit);
// nullptr means run serially.
struct SideStream {
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
};
static SideStream* side_stream(cudaStream_t st) {
  thread_local SideStream tab[32];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 32) return nullptr;
  SideStream& ss = tab[dev];
  if (!ss.s) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return nullptr;
    SideStream fresh;
    if (cudaStreamCreateWithFlags(&fresh.s, cudaStreamNonBlocking) == cudaSuccess &&
        cudaEventCreateWithFlags(&fresh.fork, cudaEventDisableTiming) == cudaSuccess &&
        cudaEventCreateWithFlags(&fresh.join, cudaEventDisableTiming) == cudaSuccess) {
      ss = fresh;
    } else {   // all or nothing
      if (fresh.join) cudaEventDestroy(fresh.join);
      if (fresh.fork) cudaEventDestroy(fresh.fork);
      if (fresh.s) cudaStreamDestroy(fresh.s);
      cudaGetLastError();
      return nullptr;
    }
  }
  return &ss;
}

// Named NVTX range around the host-side enqueue of a phase (shows each iteration's forward
// agents, prior agent and MACE step on a profiler's timeline; no cost without a tool).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

// One to many loop bodies of Alg. 2 on the state (mu, r, w); ws = agent scratch then denoiser scratch.
// `spectrum_ready`: the agent scratch already holds the band-limited schedule's F mu for this
// mu, one pending step behind (a previous call of the same run); otherwise it is rebuilt.
static clamp_status iterate_impl(const clamp_params* p, const Derived& d, int k_first, int iters, const float* y,
                                 const float* pupil, const float* window, const clamp_denoiser* den, float2* mu,
                                 float* r, float* w, float* wbar, double* ce_out, double* mu_out, void* ws,
                                 void* const* events, bool spectrum_ready, cudaStream_t st) {
  const AgentLayout al = agent_layout(p);
  void* dws = static_cast<char*>(ws) + al.bytes;
  const long long n = d.g.n;
  const bool noap = (p->flags & CLAMP_FLAG_NO_APERTURE) != 0;
  if (noap && iters > 0) API_TRY(ablation_prepare(d, y, al, ws, st));
  // concurrent schedule: the prior agent forks off `st` after the previous MACE pass and
  // the MACE pass joins it; within the iteration it shares no state with the forward agents
  SideStream* ss = prior_concurrent(p) ? side_stream(st) : nullptr;
  for (int it = 0; it < iters; ++it) {
    const int k = k_first + it;
    NvtxRange r_it("clamp iteration");
    if (events) API_CUDA(cudaEventRecord((cudaEvent_t)events[4 * it + 0], st), "event");
    if (ss) {
      NvtxRange r_prior("prior agent (side stream)");
      API_CUDA(cudaEventRecord(ss->fork, st), "event");
      API_CUDA(cudaStreamWaitEvent(ss->s, ss->fork, 0), "event");
      API_CUDA(denoise_apply(den, w + (long long)p->looks * n, r + (long long)p->looks * n, p->nx, p->ny, p->nz,
                             dws, at<int>(ws, al.err), ss->s),
               "denoiser");
      if (events) API_CUDA(cudaEventRecord((cudaEvent_t)events[4 * it + 2], ss->s), "event");
      API_CUDA(cudaEventRecord(ss->join, ss->s), "event");
    }
    if (noap) {
      if (mu_out) API_CUDA(cudaMemsetAsync(mu_out + it, 0, sizeof(double), st), "mu residual");
    } else {
      NvtxRange r_agents("forward agents");
      API_TRY(agent_ffts(p, d, y, pupil, window, mu, r, al, ws, it == 0 && !spectrum_ready, st));
      if (mu_out) API_CUDA(launch_mean(at<double>(ws, al.mures), p->looks, mu_out + it, st), "mu residual");
    }
    if (events) API_CUDA(cudaEventRecord((cudaEvent_t)events[4 * it + 1], st), "event");
    if (ss) {
      API_CUDA(cudaStreamWaitEvent(st, ss->join, 0), "event");
    } else {
      NvtxRange r_prior("prior agent");
      API_CUDA(denoise_apply(den, w + (long long)p->looks * n, r + (long long)p->looks * n, p->nx, p->ny, p->nz,
                             dws, at<int>(ws, al.err), st),
               "denoiser");
      if (events) API_CUDA(cudaEventRecord((cudaEvent_t)events[4 * it + 2], st), "event");
    }
    NvtxRange r_mace("prox + MACE step");
    PassC c = passc_args(p, d, al, ws, mu, r, w, wbar, k);
    API_CUDA(launch_pass_c_fused(d.g, c, st), "fused prox + MACE pass");
    if (ce_out)
      API_CUDA(launch_ce_final(c.part_num, c.part_den, passc_fused_blocks(n, p->looks), ce_out + it, st),
               "CE residual");
    if (events) API_CUDA(cudaEventRecord((cudaEvent_t)events[4 * it + 3], st), "event");
  }
  return CLAMP_OK;
}

// Initialisation and p->max_iters iterations with no host synchronisation (capturable).
clamp_status recon_enqueue(const clamp_params* p, const ReconPlan& d, const float* y, const float* pupil,
                           const float* window, const clamp_denoiser* den, const float* r_init, float* r_out, void* ws,
                           cudaStream_t st) {
  const ReconLayout rl = recon_layout(p, den);
  const AgentLayout al = agent_layout(p);
  void* aws = static_cast<char*>(ws) + rl.agent;
  float2* mu = at<float2>(ws, rl.mu);
  float* r = at<float>(ws, rl.r);
  float* w = at<float>(ws, rl.w);
  const long long n = (long long)p->nx * p->ny * p->nz;
  API_CUDA(cudaMemsetAsync(at<int>(aws, al.err), 0, sizeof(int), st), "memset");
  API_TRY(do_init_warm(p, d, y, pupil, window, r_init, mu, r, w, al, aws, st));
  if (p->max_iters == 0)
    API_CUDA(cudaMemcpyAsync(r_out, r + (long long)p->looks * n, n * sizeof(float), cudaMemcpyDeviceToDevice, st),
             "copy");
  for (int it = 0; it < p->max_iters; ++it)
    API_TRY(iterate_impl(p, d, p->k0 + it + 1, 1, y, pupil, window, den, mu, r, w, r_out,
                         at<double>(ws, rl.ce_ring) + it, at<double>(ws, rl.mu_ring) + it, aws, nullptr, it > 0, st));
  return CLAMP_OK;
}

size_t recon_agent_offset(const clamp_params* p, const clamp_denoiser* den) { return recon_layout(p, den).agent; }

const double* recon_ce_ring(const clamp_params* p, const clamp_denoiser* den, const void* ws) {
  return reinterpret_cast<const double*>(static_cast<const char*>(ws) + recon_layout(p, den).ce_ring);
}

extern "C" clamp_status clamp_iterate(const clamp_params* p, int32_t k_first, int32_t iters, const float* y,
                                      const float* pupil, const float* window, const clamp_denoiser* den, float* mu,
                                      float* r, float* w, float* wbar, double* ce_out, double* mu_out, void* ws,
                                      size_t ws_bytes, void* const* events, void* stream) {
  API_TRY(clamp_check_params(p));
  if (!den) return api_fail(CLAMP_EINVAL, "clamp_iterate: denoiser is NULL");
  if (!denoise_supports(den, p->nx, p->ny, p->nz))
    return api_fail(CLAMP_EUNSUPPORTED, "clamp_iterate: the prior agent does not support this volume");
  if (k_first < 1 || iters < 0) return api_fail(CLAMP_EINVAL, "clamp_iterate: k_first=%d must be >= 1, iters >= 0",
                                            k_first);
  API_TRY(need_ptrs({y, pupil, window, mu, r, w, wbar}, "clamp_iterate"));
  API_TRY(check_ws(ws, ws_bytes, iterate_ws_bytes(p, den), "clamp_iterate"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  Derived d;
  API_TRY(recon_prepare(p, pupil, window, st, &d));
  API_CUDA(cudaMemsetAsync(at<int>(ws, agent_layout(p).err), 0, sizeof(int), st), "memset");
  return iterate_impl(p, d, k_first, iters, y, pupil, window, den, reinterpret_cast<float2*>(mu), r, w, wbar, ce_out,
                      mu_out, ws, events, false, st);
}

// `plan`: the aperture statistics when the caller already has them (host inputs), else NULL
// (read from the device pupil and window, one synchronisation).
static clamp_status reconstruct_impl(const clamp_params* p, const float* y, const float* pupil, const float* window,
                                     const clamp_denoiser* den, const float* r_init, float* r_out,
                                     clamp_report* report, void* ws, cudaStream_t st,
                                     const ReconPlan* plan = nullptr) {
  const ReconLayout rl = recon_layout(p, den);
  const AgentLayout al = agent_layout(p);
  void* aws = static_cast<char*>(ws) + rl.agent;
  float2* mu = at<float2>(ws, rl.mu);
  float* r = at<float>(ws, rl.r);
  float* w = at<float>(ws, rl.w);
  double* ce_ring = at<double>(ws, rl.ce_ring);
  double* mu_ring = at<double>(ws, rl.mu_ring);
  const long long n = (long long)p->nx * p->ny * p->nz;
  Derived d;
  if (plan) d = *plan;
  else API_TRY(recon_prepare(p, pupil, window, st, &d));
  API_CUDA(cudaMemsetAsync(at<int>(aws, al.err), 0, sizeof(int), st), "memset");
  API_TRY(do_init_warm(p, d, y, pupil, window, r_init, mu, r, w, al, aws, st));
  if (p->max_iters == 0) {
    // r* = wbar of the initial state = r0
    API_CUDA(cudaMemcpyAsync(r_out, r + (long long)p->looks * n, n * sizeof(float), cudaMemcpyDeviceToDevice, st),
             "copy");
  }
  const int check = p->check_every > 0 ? p->check_every : 10;
  int done = 0;
  bool converged = false;
  std::vector<double> ce_h(p->max_iters > 0 ? p->max_iters : 1), mu_h(ce_h.size());
  int synced_upto = 0;
  for (int it = 0; it < p->max_iters; ++it) {
    const int k = p->k0 + it + 1;
    API_TRY(iterate_impl(p, d, k, 1, y, pupil, window, den, mu, r, w, r_out, ce_ring + it, mu_ring + it, aws,
                         nullptr, it > 0, st));
    done = it + 1;
    const bool last = (it + 1 == p->max_iters);
    if ((p->tol > 0 && ((it + 1) % check == 0 || last)) || (last && report)) {
      int herr = 0;
      API_CUDA(cudaMemcpyAsync(ce_h.data() + synced_upto, ce_ring + synced_upto, (done - synced_upto) * sizeof(double),
                               cudaMemcpyDeviceToHost, st),
               "residual readback");
      API_CUDA(cudaMemcpyAsync(&herr, at<int>(aws, al.err), sizeof(int), cudaMemcpyDeviceToHost, st), "readback");
      API_CUDA(cudaStreamSynchronize(st), "residual readback");
      if (herr & 2) return api_fail(CLAMP_ETIMEOUT, "a bounded tensor-core wait gave up at or before iteration %d", k);
      if (herr) return api_fail(CLAMP_ENONFINITE, "non-finite value in the state at or before iteration %d", k);
      for (int i = synced_upto; i < done; ++i) {
        if (p->tol > 0 && ce_h[i] <= p->tol) {
          converged = true;
        }
      }
      synced_upto = done;
      if (converged) break;
    }
  }
  if (report) {
    report->iters = done;
    report->converged = converged ? 1 : 0;
    if (done > 0) {
      API_CUDA(cudaMemcpyAsync(ce_h.data(), ce_ring, done * sizeof(double), cudaMemcpyDeviceToHost, st), "report");
      API_CUDA(cudaMemcpyAsync(mu_h.data(), mu_ring, done * sizeof(double), cudaMemcpyDeviceToHost, st), "report");
      API_CUDA(cudaStreamSynchronize(st), "report");
      report->ce_residual = ce_h[done - 1];
      report->mu_residual = mu_h[done - 1];
      if (report->ce_hist) memcpy(report->ce_hist, ce_h.data(), done * sizeof(double));
      if (report->mu_hist) memcpy(report->mu_hist, mu_h.data(), done * sizeof(double));
    } else {
      report->ce_residual = report->mu_residual = 0.0;
    }
  }
  return CLAMP_OK;
}

extern "C" clamp_status clamp_reconstruct(const clamp_params* p, const float* y, const float* pupil,
                                          const float* window, const clamp_denoiser* den, const float* r_init,
                                          float* r_out, clamp_report* report, void* ws, size_t ws_bytes,
                                          void* stream) {
  API_TRY(clamp_check_params(p));
  if (!den) return api_fail(CLAMP_EINVAL, "clamp_reconstruct: denoiser is NULL");
  if (!denoise_supports(den, p->nx, p->ny, p->nz))
    return api_fail(CLAMP_EUNSUPPORTED, "clamp_reconstruct: the prior agent does not support this volume");
  API_TRY(need_ptrs({y, pupil, window, r_out}, "clamp_reconstruct"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  const size_t need = recon_layout(p, den).bytes;
  void* own = nullptr;
  if (!ws) {
    API_CUDA(cudaMalloc(&own, need), "workspace allocation");
    ws = own;
    ws_bytes = need;
  }
  clamp_status s = check_ws(ws, ws_bytes, need, "clamp_reconstruct");
  if (s == CLAMP_OK) s = reconstruct_impl(p, y, pupil, window, den, r_init, r_out, report, ws, st);
  if (own) {
    cudaStreamSynchronize(st);
    cudaFree(own);
  }
  return s;
}

// ---------------------------------------------------------------- host-buffer variant with a device cache

namespace {
struct HostCache {
  int dev = -1;
  void* buf = nullptr;
  size_t bytes = 0;
};
std::mutex g_cache_mu;
std::vector<HostCache> g_cache;
}  // namespace

extern "C" void clamp_release_cache(void) {
  std::lock_guard<std::mutex> lk(g_cache_mu);
  int cur = -1;
  cudaGetDevice(&cur);
  for (auto& c : g_cache) {
    if (c.buf) {
      cudaSetDevice(c.dev);
      cudaFree(c.buf);
    }
  }
  g_cache.clear();
  if (cur >= 0) cudaSetDevice(cur);
  noalloc_forget();
}

extern "C" clamp_status clamp_reconstruct_host(const clamp_params* p, const float* y_host, const float* pupil_host,
                                               const float* window_host, const clamp_denoiser* den,
                                               const float* r_init_host, float* r_out_host, clamp_report* report,
                                               void* stream) {
  API_TRY(clamp_check_params(p));
  if (!den) return api_fail(CLAMP_EINVAL, "clamp_reconstruct_host: denoiser is NULL");
  if (!denoise_supports(den, p->nx, p->ny, p->nz))
    return api_fail(CLAMP_EUNSUPPORTED, "clamp_reconstruct_host: the prior agent does not support this volume");
  API_TRY(need_ptrs({y_host, pupil_host, window_host, r_out_host}, "clamp_reconstruct_host"));
  API_TRY(api_ensure_device());
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = (long long)p->nx * p->ny * p->nz, L = p->looks;
  Arena ar;
  const size_t o_y = ar.take<float2>(L * n), o_p = ar.take<float>((long long)p->nx * p->ny),
               o_w = ar.take<float>(p->nz), o_ri = ar.take<float>(n), o_ro = ar.take<float>(n);
  const size_t o_ws = ar.off;
  const size_t need = o_ws + recon_layout(p, den).bytes;
  int dev = 0;
  API_CUDA(cudaGetDevice(&dev), "cudaGetDevice");
  std::lock_guard<std::mutex> lk(g_cache_mu);
  HostCache* hc = nullptr;
  for (auto& c : g_cache)
    if (c.dev == dev) hc = &c;
  if (!hc) {
    g_cache.push_back(HostCache{dev, nullptr, 0});
    hc = &g_cache.back();
  }
  if (hc->bytes < need) {
    if (hc->buf) {
      API_CUDA(cudaDeviceSynchronize(), "sync");
      cudaFree(hc->buf);
      hc->buf = nullptr;
      hc->bytes = 0;
    }
    API_CUDA(cudaMalloc(&hc->buf, need), "device cache allocation");
    hc->bytes = need;
  }
  // the aperture statistics come from the host copies: the call synchronises only at its end
  ReconPlan plan;
  if (p->flags & CLAMP_FLAG_NO_APERTURE) API_TRY(recon_prepare(p, nullptr, nullptr, st, &plan));
  else API_TRY(recon_prepare_host(p, pupil_host, window_host, &plan));
  char* b = static_cast<char*>(hc->buf);
  API_CUDA(cudaMemcpyAsync(b + o_y, y_host, L * n * sizeof(float2), cudaMemcpyHostToDevice, st), "y upload");
  API_CUDA(cudaMemcpyAsync(b + o_p, pupil_host, (size_t)p->nx * p->ny * sizeof(float), cudaMemcpyHostToDevice, st),
           "pupil upload");
  API_CUDA(cudaMemcpyAsync(b + o_w, window_host, p->nz * sizeof(float), cudaMemcpyHostToDevice, st), "window upload");
  if (r_init_host)
    API_CUDA(cudaMemcpyAsync(b + o_ri, r_init_host, n * sizeof(float), cudaMemcpyHostToDevice, st), "r_init upload");
  clamp_status s = reconstruct_impl(p, reinterpret_cast<float*>(b + o_y), reinterpret_cast<float*>(b + o_p),
                                    reinterpret_cast<float*>(b + o_w), den,
                                    r_init_host ? reinterpret_cast<float*>(b + o_ri) : nullptr,
                                    reinterpret_cast<float*>(b + o_ro), report, b + o_ws, st, &plan);
  if (s != CLAMP_OK) return s;
  API_CUDA(cudaMemcpyAsync(r_out_host, b + o_ro, n * sizeof(float), cudaMemcpyDeviceToHost, st), "r_out download");
  API_CUDA(cudaStreamSynchronize(st), "sync");
  return CLAMP_OK;
}

// ---------------------------------------------------------------- huge-page host staging memory

namespace {
std::mutex g_host_mu;
std::map<void*, std::pair<void*, size_t>> g_host_allocs;   // user pointer -> (mapping, mapping length)

size_t huge_page_bytes() {
  size_t hp = 2u << 20;   // the usual PMD size with 4 KB base pages
  if (FILE* f = fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r")) {
    unsigned long long v = 0;
    if (fscanf(f, "%llu", &v) == 1 && v >= 4096 && (v & (v - 1)) == 0) hp = (size_t)v;
    fclose(f);
  }
  return hp;
}
}  // namespace

extern "C" clamp_status clamp_host_alloc(size_t bytes, void** out) {
  if (out) *out = nullptr;
  if (!out || bytes == 0) return api_fail(CLAMP_EINVAL, "clamp_host_alloc: bytes must be > 0 and out non-NULL");
  const size_t page = (size_t)sysconf(_SC_PAGESIZE);
  const size_t hp = huge_page_bytes();
  const size_t len = (bytes + page - 1) / page * page;
  const size_t map_len = len + hp;   // slack to start the block on a huge-page boundary
  void* raw = mmap(nullptr, map_len, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (raw == MAP_FAILED) return api_fail(CLAMP_ENOMEM, "clamp_host_alloc: mmap of %zu bytes failed", map_len);
  char* p = reinterpret_cast<char*>(((uintptr_t)raw + hp - 1) / hp * hp);
  madvise(p, len, MADV_HUGEPAGE);   // advisory: base pages remain if the kernel declines
  for (size_t o = 0; o < len; o += 4096) p[o] = 0;   // populate before registering
  const cudaError_t e = cudaHostRegister(p, len, cudaHostRegisterDefault);
  if (e != cudaSuccess) {
    munmap(raw, map_len);
    return cuda_fail(e, "clamp_host_alloc: cudaHostRegister");
  }
  std::lock_guard<std::mutex> lk(g_host_mu);
  g_host_allocs[p] = {raw, map_len};
  *out = p;
  return CLAMP_OK;
}

extern "C" void clamp_host_free(void* p) {
  if (!p) return;
  std::pair<void*, size_t> m;
  {
    std::lock_guard<std::mutex> lk(g_host_mu);
    auto it = g_host_allocs.find(p);
    if (it == g_host_allocs.end()) return;
    m = it->second;
    g_host_allocs.erase(it);
  }
  cudaHostUnregister(p);
  munmap(m.first, m.second);
}
