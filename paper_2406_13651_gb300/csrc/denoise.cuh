// denoise.cuh -- prior agents H (internal interface).
#pragma once
#include <cuda_runtime.h>
#include <stddef.h>

#include <vector>

struct clamp_denoiser {
  int kind = 0;              // 0 = Gaussian smoother, 1 = residual CNN
  float g0 = 0.f, g1 = 1.f;  // Gaussian taps [g0, g1, g0]
  int layers = 0, channels = 0, dtype = 0;
  int dev = -1;
  std::vector<int> cin, cout;
  std::vector<float*> w;      // per layer, device, [cout][cin][27]
  std::vector<float*> b;      // per layer, device, [cout]
  std::vector<void*> w16;     // per layer, device, bf16 packed weights (dtype BF16)
};

size_t denoise_ws_bytes(const clamp_denoiser* d, int nx, int ny, int nz);
cudaError_t denoise_apply(const clamp_denoiser* d, const float* in, float* out, int nx, int ny, int nz, void* ws,
                          cudaStream_t st);
