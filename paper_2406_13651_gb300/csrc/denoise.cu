// denoise.cu -- prior agents: 3x3x3 Gaussian smoother and the residual 3D CNN
// H(x) = x + CNN(x) (3x3x3 convs, zero padding, ReLU on hidden layers).
//
// FP32 convolution: direct 3x3x3 conv as a shared-memory tiled kernel.  A CTA
// computes a 32(x) x TY(y) x 1(z) voxel tile for CO*CG output channels; each
// thread keeps 4 consecutive x voxels x CO channels in registers.  Input
// channels are staged CINC at a time: the (TY+2) x 34 x 3 halo of each and the
// matching 27 x CO*CG weights.
#include "../../include/clamp.h"
#include "clamp_kernels.cuh"
#include "denoise.cuh"

#include <math.h>
#include <stdio.h>

#include <string>

namespace clamp {

constexpr int CV_TX = 32;  // output x per CTA
constexpr int CV_VX = 4;   // output x per thread

template <int CO, int CG, int CINC>
struct ConvCfg {
  static constexpr int TY = NT / ((CV_TX / CV_VX) * CG);  // output rows per CTA
  static constexpr int IX = CV_TX + 2, IY = TY + 2;
  static constexpr int IN_FLOATS = CINC * 3 * IY * IX;
  static constexpr int W_FLOATS = CINC * 27 * CO * CG;
  static constexpr size_t SMEM = sizeof(float) * (IN_FLOATS + W_FLOATS);
};

// out[co][v] = bias[co] + sum_ci sum_taps W[co][ci][tap] in[ci][v + tap]  (+ resid[v]) (ReLU)
template <int CO, int CG, int CINC, bool RELU>
__global__ void __launch_bounds__(NT) k_conv3_f32(const float* __restrict__ in, int cin, float* __restrict__ out,
                                                  int cout, const float* __restrict__ W,
                                                  const float* __restrict__ bias, const float* __restrict__ resid,
                                                  int nx, int ny, int nz) {
  using C = ConvCfg<CO, CG, CINC>;
  constexpr int TY = C::TY, IX = C::IX, IY = C::IY, COT = CO * CG;
  extern __shared__ float4 smem4[];
  float* s_in = reinterpret_cast<float*>(smem4);
  float* s_w = s_in + C::IN_FLOATS;
  const int tx = threadIdx.x % (CV_TX / CV_VX);
  const int ty = (threadIdx.x / (CV_TX / CV_VX)) % TY;
  const int cg = threadIdx.x / ((CV_TX / CV_VX) * TY);
  const int x0 = blockIdx.x * CV_TX, y0 = blockIdx.y * TY;
  const int ncb = (cout + COT - 1) / COT;
  const int z = blockIdx.z / ncb, cb = blockIdx.z % ncb;
  const long long plane = (long long)nx * ny, n = plane * nz;
  float acc[CV_VX][CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    const int co = cb * COT + cg * CO + o;
    const float bv = co < cout ? __ldg(&bias[co]) : 0.f;
#pragma unroll
    for (int v = 0; v < CV_VX; ++v) acc[v][o] = bv;
  }
  for (int c0 = 0; c0 < cin; c0 += CINC) {
    __syncthreads();
    for (int e = threadIdx.x; e < C::IN_FLOATS; e += NT) {
      const int xi = e % IX;
      const int yi = (e / IX) % IY;
      const int zi = (e / (IX * IY)) % 3;
      const int ci = e / (IX * IY * 3);
      const int gx = x0 + xi - 1, gy = y0 + yi - 1, gz = z + zi - 1;
      float v = 0.f;
      if (c0 + ci < cin && gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
        v = __ldg(&in[(long long)(c0 + ci) * n + (long long)gz * plane + (long long)gy * nx + gx]);
      s_in[e] = v;
    }
    for (int e = threadIdx.x; e < C::W_FLOATS; e += NT) {
      const int o = e % COT;
      const int tap = (e / COT) % 27;
      const int ci = e / (COT * 27);
      const int co = cb * COT + o;
      s_w[e] = (co < cout && c0 + ci < cin) ? __ldg(&W[((long long)co * cin + c0 + ci) * 27 + tap]) : 0.f;
    }
    __syncthreads();
#pragma unroll 1
    for (int ci = 0; ci < CINC; ++ci) {
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const float* row = s_in + ((ci * 3 + dz) * IY + ty + dy) * IX + tx * CV_VX;
          float xin[CV_VX + 2];
#pragma unroll
          for (int q = 0; q < CV_VX + 2; ++q) xin[q] = row[q];
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const float* wp = s_w + (ci * 27 + dz * 9 + dy * 3 + dx) * COT + cg * CO;
            float wv[CO];
#pragma unroll
            for (int o = 0; o < CO; ++o) wv[o] = wp[o];
#pragma unroll
            for (int v = 0; v < CV_VX; ++v)
#pragma unroll
              for (int o = 0; o < CO; ++o) acc[v][o] = fmaf(xin[v + dx], wv[o], acc[v][o]);
          }
        }
      }
    }
  }
  const int gy = y0 + ty;
  if (gy >= ny) return;
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    const int co = cb * COT + cg * CO + o;
    if (co >= cout) continue;
#pragma unroll
    for (int v = 0; v < CV_VX; ++v) {
      const int gx = x0 + tx * CV_VX + v;
      if (gx >= nx) continue;
      const long long vox = (long long)z * plane + (long long)gy * nx + gx;
      float r = acc[v][o];
      if (RELU) r = fmaxf(r, 0.f);
      if (resid) r += resid[vox];
      out[(long long)co * n + vox] = r;
    }
  }
}

template <int CO, int CG, int CINC, bool RELU>
static cudaError_t run_conv(const float* in, int cin, float* out, int cout, const float* W, const float* b,
                            const float* resid, int nx, int ny, int nz, cudaStream_t st) {
  using C = ConvCfg<CO, CG, CINC>;
  auto kern = k_conv3_f32<CO, CG, CINC, RELU>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
  if (e != cudaSuccess) return e;
  const int ncb = (cout + CO * CG - 1) / (CO * CG);
  dim3 grid((nx + CV_TX - 1) / CV_TX, (ny + C::TY - 1) / C::TY, nz * ncb);
  kern<<<grid, NT, C::SMEM, st>>>(in, cin, out, cout, W, b, resid, nx, ny, nz);
  return cudaGetLastError();
}

// Single-output-channel layer (the CNN's last layer, SIMT fallback): out[v] = b + sum_ci sum_taps
// W[ci][tap] in[ci][v+tap] (+ resid[v]).  A thread computes a 2(x) x 2(y) block at one z, so each
// input value it loads from shared memory feeds up to 4 accumulators per tap plane.
constexpr int C1_TX = 32, C1_TY = 32, C1_CINC = 4;
constexpr int C1_IX = C1_TX + 2, C1_IY = C1_TY + 2;
constexpr size_t C1_SMEM = sizeof(float) * (C1_CINC * 3 * C1_IY * C1_IX + C1_CINC * 27);

__global__ void __launch_bounds__(NT) k_conv3_c1(const float* __restrict__ in, int cin, float* __restrict__ out,
                                                 const float* __restrict__ W, const float* __restrict__ bias,
                                                 const float* __restrict__ resid, int nx, int ny, int nz) {
  extern __shared__ float4 smem4[];
  float* s_in = reinterpret_cast<float*>(smem4);
  float* s_w = s_in + C1_CINC * 3 * C1_IY * C1_IX;
  const int tx = threadIdx.x % (C1_TX / 2), ty = threadIdx.x / (C1_TX / 2);  // 16 x 16 threads
  const int x0 = blockIdx.x * C1_TX, y0 = blockIdx.y * C1_TY, z = blockIdx.z;
  const long long plane = (long long)nx * ny, n = plane * nz;
  float acc[2][2];
  const float b0 = __ldg(&bias[0]);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int c = 0; c < 2; ++c) acc[a][c] = b0;
  for (int c0 = 0; c0 < cin; c0 += C1_CINC) {
    __syncthreads();
    for (int e = threadIdx.x; e < C1_CINC * 3 * C1_IY * C1_IX; e += NT) {
      const int xi = e % C1_IX;
      const int yi = (e / C1_IX) % C1_IY;
      const int zi = (e / (C1_IX * C1_IY)) % 3;
      const int ci = e / (C1_IX * C1_IY * 3);
      const int gx = x0 + xi - 1, gy = y0 + yi - 1, gz = z + zi - 1;
      float v = 0.f;
      if (c0 + ci < cin && gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
        v = __ldg(&in[(long long)(c0 + ci) * n + (long long)gz * plane + (long long)gy * nx + gx]);
      s_in[e] = v;
    }
    for (int e = threadIdx.x; e < C1_CINC * 27; e += NT)
      s_w[e] = (c0 + e / 27 < cin) ? __ldg(&W[(long long)c0 * 27 + e]) : 0.f;
    __syncthreads();
#pragma unroll 1
    for (int ci = 0; ci < C1_CINC; ++ci) {
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
        float xin[4][4];
        const float* base = s_in + ((ci * 3 + dz) * C1_IY + ty * 2) * C1_IX + tx * 2;
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 4; ++c) xin[a][c] = base[a * C1_IX + c];
#pragma unroll
        for (int dy = 0; dy < 3; ++dy)
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const float wv = s_w[ci * 27 + dz * 9 + dy * 3 + dx];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
              for (int c = 0; c < 2; ++c) acc[a][c] = fmaf(xin[a + dy][c + dx], wv, acc[a][c]);
          }
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 2; ++a) {
    const int gy = y0 + ty * 2 + a;
    if (gy >= ny) continue;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      const int gx = x0 + tx * 2 + c;
      if (gx >= nx) continue;
      const long long vox = (long long)z * plane + (long long)gy * nx + gx;
      out[vox] = acc[a][c] + (resid ? resid[vox] : 0.f);
    }
  }
}

static cudaError_t run_conv_c1(const float* in, int cin, float* out, const float* W, const float* b,
                               const float* resid, int nx, int ny, int nz, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_conv3_c1, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C1_SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid((nx + C1_TX - 1) / C1_TX, (ny + C1_TY - 1) / C1_TY, nz);
  k_conv3_c1<<<grid, NT, C1_SMEM, st>>>(in, cin, out, W, b, resid, nx, ny, nz);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- l2,1 prior agent

// Prox of lam * sum_z ||r_z||_2 over the (y, x) planes r_z of the range bins (the l2,1
// comparison prior of Sec. IV): r_z = max(0, 1 - lam / ||x_z||) x_z.  Pass 1 writes one
// FP64 sum of squares per (CTA, plane); pass 2 has every CTA of a plane add its plane's
// partials in the same fixed order, so all CTAs apply the same factor.  Both passes read
// the plane as float4 (nx is a multiple of 16, so a plane is a whole number of float4).
constexpr int L21_PER = 4;   // float4 per thread per CTA

__global__ void __launch_bounds__(NT) k_l21_norm(const float4* __restrict__ x, long long plane4,
                                                 double* __restrict__ part) {
  const int z = blockIdx.y;
  const float4* xz = x + (long long)z * plane4;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < L21_PER; ++k) {
    const long long i = ((long long)blockIdx.x * L21_PER + k) * NT + threadIdx.x;
    if (i < plane4) {
      const float4 v = xz[i];
      acc = fmaf(v.x, v.x, fmaf(v.y, v.y, fmaf(v.z, v.z, fmaf(v.w, v.w, acc))));
    }
  }
  __shared__ double red[NT / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = (double)acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += red[w];
    part[(long long)z * gridDim.x + blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(NT) k_l21_shrink(const float4* __restrict__ x, long long plane4,
                                                   const double* __restrict__ part, double lam,
                                                   float4* __restrict__ out) {
  const int z = blockIdx.y;
  __shared__ float s_fac;
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) s += part[(long long)z * gridDim.x + b];
    const double nrm = sqrt(s);
    s_fac = nrm > lam ? (float)(1.0 - lam / nrm) : 0.0f;
  }
  __syncthreads();
  const float f = s_fac;
  const float4* xz = x + (long long)z * plane4;
  float4* oz = out + (long long)z * plane4;
#pragma unroll
  for (int k = 0; k < L21_PER; ++k) {
    const long long i = ((long long)blockIdx.x * L21_PER + k) * NT + threadIdx.x;
    if (i < plane4) {
      const float4 v = xz[i];
      oz[i] = make_float4(f * v.x, f * v.y, f * v.z, f * v.w);
    }
  }
}

static int l21_blocks_per_plane(int nx, int ny) {
  const long long plane4 = (long long)nx * ny / 4;
  return (int)((plane4 + (long long)NT * L21_PER - 1) / ((long long)NT * L21_PER));
}

static cudaError_t run_l21(const float* in, float* out, double lam, int nx, int ny, int nz, void* ws,
                           cudaStream_t st) {
  const long long plane4 = (long long)nx * ny / 4;
  const dim3 grid(l21_blocks_per_plane(nx, ny), nz);
  double* part = static_cast<double*>(ws);
  k_l21_norm<<<grid, NT, 0, st>>>(reinterpret_cast<const float4*>(in), plane4, part);
  k_l21_shrink<<<grid, NT, 0, st>>>(reinterpret_cast<const float4*>(in), plane4, part, lam,
                                    reinterpret_cast<float4*>(out));
  return cudaGetLastError();
}

}  // namespace clamp

using namespace clamp;

size_t denoise_ws_bytes(const clamp_denoiser* d, int nx, int ny, int nz) {
  if (d && d->kind == 2) return clamp_unet_workspace_size(d->unet, 1, nx, ny, nz, 0);
  if (d && d->kind == 3) return (((size_t)l21_blocks_per_plane(nx, ny) * nz * sizeof(double)) + 255) & ~(size_t)255;
  if (!d || d->kind != 1) return 0;
  if (d->dtype == CLAMP_DENOISER_BF16) return tc_denoise_ws_bytes(d, nx, ny, nz);
  const size_t n = (size_t)nx * ny * nz;
  return 2 * (((size_t)d->channels * n * sizeof(float) + 255) & ~(size_t)255);
}

bool denoise_supports(const clamp_denoiser* d, int nx, int ny, int nz) {
  if (d->kind == 2) return nx % 4 == 0 && ny % 4 == 0 && nz % 4 == 0;
  if (d->kind == 1 && d->dtype == CLAMP_DENOISER_BF16) return tc_denoiser_supports(d, nx, ny, nz);
  return true;
}

cudaError_t denoise_apply(const clamp_denoiser* d, const float* in, float* out, int nx, int ny, int nz, void* ws,
                          int* err, cudaStream_t st) {
  if (d->kind == 0) {
    return launch_gauss3(nx, ny, nz, in, out, d->g0, d->g1, st);
  }
  if (d->kind == 2) {  // U-Net prior: the warm-start map m max(U(w / m), floor) on w
    const clamp_status s = clamp_unet_warm_start(d->unet, nx, ny, nz, in, d->floor_rel, out, ws,
                                                 denoise_ws_bytes(d, nx, ny, nz), st);
    return s == CLAMP_OK ? cudaSuccess : cudaErrorInvalidValue;
  }
  if (d->kind == 3) return run_l21(in, out, (double)d->lam, nx, ny, nz, ws, st);
  // tensor-core path (BF16, or FP32 through TF32x3) when the volume fits its tiling
  if (tc_denoiser_supports(d, nx, ny, nz)) return tc_denoise_apply(d, in, out, nx, ny, nz, ws, err, st);
  if (d->dtype == CLAMP_DENOISER_BF16) return cudaErrorInvalidValue;
  const size_t n = (size_t)nx * ny * nz;
  float* A = static_cast<float*>(ws);
  float* B = A + ((((size_t)d->channels * n * sizeof(float) + 255) & ~(size_t)255) / sizeof(float));
  const float* cur = in;
  for (int i = 0; i < d->layers; ++i) {
    const bool last = i == d->layers - 1;
    float* dst = last ? out : (cur == A ? B : A);
    cudaError_t e;
    if (last) {
      e = run_conv_c1(cur, d->cin[i], dst, d->w[i], d->b[i], in, nx, ny, nz, st);
    } else if (d->cin[i] == 1) {
      e = run_conv<8, 4, 1, true>(cur, 1, dst, d->cout[i], d->w[i], d->b[i], nullptr, nx, ny, nz, st);
    } else {
      e = run_conv<8, 4, 8, true>(cur, d->cin[i], dst, d->cout[i], d->w[i], d->b[i], nullptr, nx, ny, nz, st);
    }
    if (e != cudaSuccess) return e;
    cur = dst;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------- C ABI

static thread_local std::string g_den_err;

extern "C" clamp_status clamp_denoiser_create_gauss(float sigma, clamp_denoiser** out) {
  if (!out) return CLAMP_EINVAL;
  if (!(sigma > 0.f) || !isfinite(sigma)) return CLAMP_EINVAL;
  clamp_denoiser* d = new clamp_denoiser();
  d->kind = 0;
  const double e = exp(-1.0 / (2.0 * (double)sigma * sigma));
  d->g0 = (float)(e / (1.0 + 2.0 * e));
  d->g1 = (float)(1.0 / (1.0 + 2.0 * e));
  cudaGetDevice(&d->dev);
  *out = d;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_denoiser_create_l21(float lam, clamp_denoiser** out) {
  if (!out) return CLAMP_EINVAL;
  if (!(lam >= 0.f) || !isfinite(lam)) return CLAMP_EINVAL;
  clamp_denoiser* d = new clamp_denoiser();
  d->kind = 3;
  d->lam = lam;
  cudaGetDevice(&d->dev);
  *out = d;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_denoiser_create_unet(clamp_unet* net, float floor_rel, clamp_denoiser** out) {
  if (!out || !net || !(floor_rel >= 0.f) || !isfinite(floor_rel)) return CLAMP_EINVAL;
  clamp_denoiser* d = new clamp_denoiser();
  d->kind = 2;
  d->unet = net;
  d->floor_rel = floor_rel;
  cudaGetDevice(&d->dev);
  *out = d;
  return CLAMP_OK;
}

extern "C" void clamp_denoiser_destroy(clamp_denoiser* d) {
  if (!d) return;
  for (float* p : d->w)
    if (p) cudaFree(p);
  for (float* p : d->b)
    if (p) cudaFree(p);
  for (void* p : d->w16)
    if (p) cudaFree(p);
  if (d->w_last) cudaFree(d->w_last);
  delete d;
}

extern "C" clamp_status clamp_denoiser_create_cnn(int32_t layers, int32_t channels, int32_t dtype,
                                                  const float* weights_host, const float* biases_host,
                                                  clamp_denoiser** out) {
  if (!out || !weights_host || !biases_host) return CLAMP_EINVAL;
  if (layers < 2 || layers > 64 || channels < 1 || channels > 256) return CLAMP_EINVAL;
  if (dtype != CLAMP_DENOISER_FP32 && dtype != CLAMP_DENOISER_BF16) return CLAMP_EINVAL;
  if (dtype == CLAMP_DENOISER_BF16 && (channels % 16 || channels > 64)) return CLAMP_EUNSUPPORTED;
  clamp_denoiser* d = new clamp_denoiser();
  d->kind = 1;
  d->layers = layers;
  d->channels = channels;
  d->dtype = dtype;
  cudaGetDevice(&d->dev);
  const float* wp = weights_host;
  const float* bp = biases_host;
  auto upload = [](void** dst, const void* src, size_t bytes) {
    return cudaMalloc(dst, bytes) == cudaSuccess && cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice) == cudaSuccess;
  };
  for (int i = 0; i < layers; ++i) {
    const int ci = i == 0 ? 1 : channels;
    const int co = i == layers - 1 ? 1 : channels;
    d->cin.push_back(ci);
    d->cout.push_back(co);
    const size_t wn = (size_t)co * ci * 27;
    void *wd = nullptr, *bd = nullptr, *w16 = nullptr;
    bool ok = upload(&bd, bp, co * sizeof(float));
    const bool bf = dtype == CLAMP_DENOISER_BF16;
    const bool last = i == layers - 1;
    if (!bf || i == 0) {
      // float weights: every FP32 layer (CUDA-core paths, including the tensor path's last
      // layer) and the first BF16 layer (BF16-rounded values)
      std::vector<float> wf(wp, wp + wn);
      if (bf)
        for (auto& v : wf) v = clamp::bf16_round_value(v);
      ok = ok && upload(&wd, wf.data(), wn * sizeof(float));
    }
    const int chunk = bf ? 16 : 8;
    if (i > 0 && (!last || bf) && ci % chunk == 0) {   // layers on the tensor cores
      const std::vector<uint8_t> pk = clamp::pack_tc_weights(wp, ci, co, co == 1 ? 16 : co, bf);
      ok = ok && upload(&w16, pk.data(), pk.size());
    } else if (i == 0 && bf && co % 16 == 0 && co <= 64) {   // first BF16 layer: im2col on the tensor cores
      const std::vector<uint8_t> pk = clamp::pack_first_tc_weights(wp, co);
      ok = ok && upload(&w16, pk.data(), pk.size());
    }
    if (last && bf && ci % 16 == 0 && ci <= 64) {   // last BF16 layer: tap sums on the tensor cores
      const std::vector<uint8_t> pk = clamp::pack_last_tc_weights(wp, ci);
      ok = ok && upload(&d->w_last, pk.data(), pk.size());
    }
    d->w.push_back(static_cast<float*>(wd));
    d->b.push_back(static_cast<float*>(bd));
    d->w16.push_back(w16);
    if (!ok) {
      clamp_denoiser_destroy(d);
      return CLAMP_ECUDA;
    }
    wp += wn;
    bp += co;
  }
  *out = d;
  return CLAMP_OK;
}
