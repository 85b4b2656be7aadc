// clamp_noalloc.cu -- the MACE step without any device allocation.
//
// Some callers cannot allocate device memory themselves: code embedded in a
// host application whose own allocator owns every byte of the GPU (a raw
// cudaMalloc there would bypass its accounting, or fail because the pool
// already holds the memory), and long-running real-time loops that must not
// allocate once they have started, since an allocation can stall or fail in
// the middle of a run.  clamp_mace_step needs a small scratch buffer (the
// per-block partial sums of the convergence-error reduction) that such a
// caller could not provide.  clamp_mace_step_noalloc takes that scratch from
// the fixed array below instead.
//
// The array is a file-scope __device__ object: every GPU that loads this
// library reserves its 32 KiB until the process exits.  In host code its name
// only stands for the device object; the device address is obtained once per
// device with cudaGetSymbolAddress (with that device current) and passed to
// the kernels.  That lookup can load the library's device code, which a
// stream being captured must not see: make the first call on each device
// before any stream capture.  The address is cached per device ordinal; after
// cudaDeviceReset the module is loaded again (possibly elsewhere), so a caller
// that resets a device calls clamp_release_cache(), which forgets the cached
// addresses, before the next call.
#include "../../include/clamp.h"
#include "clamp_internal.cuh"
#include "clamp_kernels.cuh"

#include <math.h>

#include <map>
#include <mutex>

namespace {

// Scratch for the reduction partials: 2 doubles per reduction block.
constexpr int kNoAllocDoubles = 4096;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocDoubles];

std::mutex g_noalloc_mu;
std::map<int, double*> g_noalloc_ptr;  // device ordinal -> device address of the array

// Device address of the array on the current device, looked up on the first call per device.
cudaError_t noalloc_scratch(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  auto it = g_noalloc_ptr.find(dev);
  if (it != g_noalloc_ptr.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  double* ptr = nullptr;
  e = cudaGetSymbolAddress((void**)&ptr, g_noalloc_scratch);
  if (e != cudaSuccess) return e;
  g_noalloc_ptr[dev] = ptr;
  *out = ptr;
  return cudaSuccess;
}

}  // namespace

// Forgets the cached device addresses (clamp_release_cache).
void noalloc_forget() {
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  g_noalloc_ptr.clear();
}

extern "C" clamp_status clamp_mace_step_noalloc(const clamp_params* p, const float* r, float* w, float* wbar,
                                                double* ce_residual, void* stream) {
  clamp_status s = clamp_check_params(p);
  if (s != CLAMP_OK) return s;
  if (!r || !w || !wbar) return api_fail(CLAMP_EINVAL, "clamp_mace_step_noalloc: NULL array argument");
  const long long n = (long long)p->nx * p->ny * p->nz;
  const int nblk = clamp::passc_blocks(n);
  if (2 * nblk > kNoAllocDoubles)   // the partials would not fit the static array
    return api_fail(CLAMP_ENOMEM, "clamp_mace_step_noalloc: %d reduction blocks exceed the %d-double static scratch",
                    nblk, kNoAllocDoubles);
  double* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess)
    return api_fail(CLAMP_ECUDA, "clamp_mace_step_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  cudaStream_t st = (cudaStream_t)stream;
  clamp::Geom g{p->nx, p->ny, p->nz, p->looks, n};
  clamp::PassC c{};
  c.r = const_cast<float*>(r);
  c.w = w;
  c.wbar = wbar;
  c.ups_look = (float)((1.0 - (double)p->prior_weight) / p->looks);
  c.ups_prior = p->prior_weight;
  c.rho = p->rho;
  // Every block writes its own partial slot before k_ce_final reads them, so no
  // part of the array has to start at zero and stale contents are never read.
  c.part_num = scratch;
  c.part_den = scratch + nblk;
  c.err = nullptr;
  e = clamp::launch_mace_only(g, c, st);
  if (e == cudaSuccess && ce_residual) e = clamp::launch_ce_final(c.part_num, c.part_den, nblk, ce_residual, st);
  if (e != cudaSuccess) return api_fail(CLAMP_ECUDA, "clamp_mace_step_noalloc: launch: %s", cudaGetErrorString(e));
  return CLAMP_OK;
}
