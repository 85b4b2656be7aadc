// clamp_internal.cuh -- pieces of the C ABI implementation shared between translation units.
#pragma once
#include "../../include/clamp.h"
#include "clamp_kernels.cuh"

// Records an error message for clamp_last_error() and returns `s`.
clamp_status api_fail(clamp_status s, const char* fmt, ...);
// Per-device set-up (twiddle tables); idempotent.
clamp_status api_ensure_device();
// Forgets the per-device addresses of clamp_mace_step_noalloc's static scratch.
void noalloc_forget();

// Per-problem constants: geometry, alpha = mean(a^2), noise floor, FFT scales.
struct ReconPlan {
  clamp::Geom g;
  clamp::AgentScalars s;
  double alpha;
  clamp::BandShape band;   // the aperture's support and band (counted from the pupil)
  bool band_fits;          // the band-limited schedule's arrays fit the agent scratch
};

// Reads the aperture back to compute alpha (synchronises `st`): call before any capture.
clamp_status recon_prepare(const clamp_params* p, const float* pupil, const float* window, cudaStream_t st,
                           ReconPlan* out);
clamp_status recon_prepare_host(const clamp_params* p, const float* pupil_host, const float* window_host,
                                ReconPlan* d);
// Enqueues the Alg. 2 initialisation and p->max_iters iterations on `st` without any host
// synchronisation; ws is laid out as for clamp_reconstruct.
clamp_status recon_enqueue(const clamp_params* p, const ReconPlan& plan, const float* y, const float* pupil,
                           const float* window, const clamp_denoiser* den, const float* r_init, float* r_out,
                           void* ws, cudaStream_t st);
// Device ring of per-iteration convergence errors inside a clamp_reconstruct workspace.
const double* recon_ce_ring(const clamp_params* p, const clamp_denoiser* den, const void* ws);
// Times the launch variants of the forward-agent passes on agent scratch `ws` and caches the
// fastest per geometry (synchronises `st`).
clamp_status autotune_agent(const clamp_params* p, const ReconPlan& plan, const float* y, const float* pupil,
                            const float* window, void* ws, cudaStream_t st, clamp::AgentVariants* out);
// Byte offset of the forward-agent scratch inside a clamp_reconstruct workspace.
size_t recon_agent_offset(const clamp_params* p, const clamp_denoiser* den);

// The U-Net's 3x3x3 conv on the tensor cores (BF16 operands, FP32 accumulation), FP32
// channel-planar tensors in and out; W is FP32 [co][ci][27] (packed to BF16 into wpk,
// unet_conv3_tc_wpk_bytes(ci, co) bytes, on the stream).  err: device word, bit 2 set when a
// bounded wait gave up.
namespace clamp {
bool unet_conv3_tc_supported(int ci, int co, int nx, int ny);
size_t unet_conv3_tc_wpk_bytes(int ci, int co);
cudaError_t unet_conv3_tc(const float* in, long long in_bs, int ci, float* out, long long out_bs, int co,
                          const float* W, const float* bias, bool relu, int B, int nx, int ny, int nz, uint4* wpk,
                          int* err, cudaStream_t st);
}  // namespace clamp
