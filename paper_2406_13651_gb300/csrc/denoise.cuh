// denoise.cuh -- prior agents H (internal interface).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <stdint.h>

#include <vector>

struct clamp_unet;

struct clamp_denoiser {
  int kind = 0;              // 0 = Gaussian smoother, 1 = residual CNN, 2 = U-Net prior (borrowed net), 3 = l2,1 prox
  float g0 = 0.f, g1 = 1.f;  // Gaussian taps [g0, g1, g0]
  int layers = 0, channels = 0, dtype = 0;
  int dev = -1;
  std::vector<int> cin, cout;
  std::vector<float*> w;      // per layer, device, [cout][cin][27]
  std::vector<float*> b;      // per layer, device, [cout]
  std::vector<void*> w16;     // per layer, device, tensor-core packed weights (layers >= 1)
  void* w_last = nullptr;     // BF16 prior: last layer's weights for the tap-sum GEMM (device)
  clamp_unet* unet = nullptr; // kind 2: the caller's network (not owned)
  float floor_rel = 1e-3f;    // kind 2: output floor in units of the input's column energy
  float lam = 0.f;            // kind 3: l2,1 weight
};

size_t denoise_ws_bytes(const clamp_denoiser* d, int nx, int ny, int nz);
// True if the denoiser can run on an nx x ny x nz volume (the BF16 CNN runs only on the
// tensor cores: nx % 128 == 0, ny % 4 == 0, nz % 2 == 0, 16..64 channels in steps of 16).
bool denoise_supports(const clamp_denoiser* d, int nx, int ny, int nz);
// err: optional device error word (bit 2: a bounded tensor-core wait gave up).
cudaError_t denoise_apply(const clamp_denoiser* d, const float* in, float* out, int nx, int ny, int nz, void* ws,
                          int* err, cudaStream_t st);

namespace clamp {
// Tensor-core CNN prior (BF16, or FP32 through the TF32x3 split), implemented in tc_conv.cu.
bool tc_denoiser_supports(const clamp_denoiser* d, int nx, int ny, int nz);
size_t tc_denoise_ws_bytes(const clamp_denoiser* d, int nx, int ny, int nz);
cudaError_t tc_denoise_apply(const clamp_denoiser* d, const float* in, float* out, int nx, int ny, int nz, void* ws,
                             int* err, cudaStream_t st);
std::vector<uint8_t> pack_tc_weights(const float* W, int cin, int cout, int npad, bool bf16);
// First BF16 layer (1 -> C) on tensor cores: W [C][27] as BF16 B[co][k], k = tap < 27, zero to 32.
std::vector<uint8_t> pack_first_tc_weights(const float* W, int cout);
// Last BF16 layer (C -> 1): W [1][C][27] as BF16 B[tap][c] in [C/8][32][8] (taps padded to 32).
std::vector<uint8_t> pack_last_tc_weights(const float* W, int cin);
float bf16_round_value(float f);
}  // namespace clamp
