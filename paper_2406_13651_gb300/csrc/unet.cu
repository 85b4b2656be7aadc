// unet.cu -- the learned warm start: a 3-level 3D U-Net (encoder: two 3x3x3 conv + ReLU
// per level and 2^3 max-pooling; decoder: 2^3 stride-2 transposed conv, concatenation
// with the encoder skip, two 3x3x3 conv + ReLU; a final 1x1x1 conv), trained on the
// GPU with these forward and backward kernels and Adam (FP32).
//
// Tensors are channel-planar per sample: [B][C][nz][ny][nx].  A concatenation buffer
// holds the decoder's upsampled channels first and the encoder skip after them, so the
// skip's conv writes straight into it (no copy).
#include "../../include/clamp.h"
#include "clamp_internal.cuh"
#include "clamp_kernels.cuh"

#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace clamp {
namespace unet {

constexpr int UT = 256;

// BF16 mode: an operand rounded to bfloat16 (round to nearest even) and widened back.
template <bool BF>
__device__ __forceinline__ float opnd(float x) {
  if constexpr (BF) return __bfloat162float(__float2bfloat16_rn(x));
  else return x;
}
__device__ __forceinline__ float opr(float x, int bf) {
  return bf ? __bfloat162float(__float2bfloat16_rn(x)) : x;
}

enum LayerKind { CONV3 = 0, TCONV = 1, CONV1 = 2 };
struct Layer {
  int kind, ci, co;
  size_t w, b;  // offsets (floats) into the parameter buffer
  size_t nw;    // weight count
};

// ---------------------------------------------------------------- 3x3x3 conv (forward and dgrad)

constexpr int CX = 32, CVX = 4;  // output x per CTA, per thread

// out[b][co][v] = bias[co] + sum_ci sum_tap W[co][ci][tap] in[b][ci][v + tap] (zero padding), optional ReLU.
// in / out address sample b at in + b * in_bs, channel c at + c * n.
template <int CO, int CG, int CINC, bool BF>
__global__ void __launch_bounds__(UT) k_conv3(const float* __restrict__ in, long long in_bs, int ci_n,
                                              float* __restrict__ out, long long out_bs, int co_n,
                                              const float* __restrict__ W, const float* __restrict__ bias, int relu,
                                              int nx, int ny, int nz) {
  constexpr int TY = UT / ((CX / CVX) * CG), IX = CX + 2, IY = TY + 2, COT = CO * CG;
  __shared__ float s_in[CINC * 3 * IY * IX];
  __shared__ float s_w[CINC * 27 * COT];
  const int tx = threadIdx.x % (CX / CVX);
  const int ty = (threadIdx.x / (CX / CVX)) % TY;
  const int cg = threadIdx.x / ((CX / CVX) * TY);
  const int x0 = blockIdx.x * CX, y0 = blockIdx.y * TY;
  const int ncb = (co_n + COT - 1) / COT;
  const int zz = blockIdx.z / ncb, cb = blockIdx.z % ncb;
  const int b = zz / nz, z = zz % nz;
  const long long plane = (long long)nx * ny, n = plane * nz;
  const float* inb = in + (long long)b * in_bs;
  float acc[CVX][CO];
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    const int co = cb * COT + cg * CO + o;
    const float bv = (bias && co < co_n) ? __ldg(&bias[co]) : 0.f;
#pragma unroll
    for (int v = 0; v < CVX; ++v) acc[v][o] = bv;
  }
  for (int c0 = 0; c0 < ci_n; c0 += CINC) {
    __syncthreads();
    for (int e = threadIdx.x; e < CINC * 3 * IY * IX; e += UT) {
      const int xi = e % IX, yi = (e / IX) % IY, zi = (e / (IX * IY)) % 3, ci = e / (IX * IY * 3);
      const int gx = x0 + xi - 1, gy = y0 + yi - 1, gz = z + zi - 1;
      float v = 0.f;
      if (c0 + ci < ci_n && gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
        v = __ldg(&inb[(long long)(c0 + ci) * n + (long long)gz * plane + (long long)gy * nx + gx]);
      s_in[e] = opnd<BF>(v);
    }
    for (int e = threadIdx.x; e < CINC * 27 * COT; e += UT) {
      const int o = e % COT, tap = (e / COT) % 27, ci = e / (COT * 27);
      const int co = cb * COT + o;
      s_w[e] = (co < co_n && c0 + ci < ci_n) ? opnd<BF>(__ldg(&W[((long long)co * ci_n + c0 + ci) * 27 + tap])) : 0.f;
    }
    __syncthreads();
#pragma unroll 1
    for (int ci = 0; ci < CINC; ++ci) {
#pragma unroll
      for (int dz = 0; dz < 3; ++dz) {
#pragma unroll
        for (int dy = 0; dy < 3; ++dy) {
          const float* row = s_in + ((ci * 3 + dz) * IY + ty + dy) * IX + tx * CVX;
          float xin[CVX + 2];
#pragma unroll
          for (int q = 0; q < CVX + 2; ++q) xin[q] = row[q];
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const float* wp = s_w + (ci * 27 + dz * 9 + dy * 3 + dx) * COT + cg * CO;
#pragma unroll
            for (int o = 0; o < CO; ++o) {
              const float wv = wp[o];
#pragma unroll
              for (int v = 0; v < CVX; ++v) acc[v][o] = fmaf(xin[v + dx], wv, acc[v][o]);
            }
          }
        }
      }
    }
  }
  const int gy = y0 + ty;
  if (gy >= ny) return;
  float* outb = out + (long long)b * out_bs;
#pragma unroll
  for (int o = 0; o < CO; ++o) {
    const int co = cb * COT + cg * CO + o;
    if (co >= co_n) continue;
#pragma unroll
    for (int v = 0; v < CVX; ++v) {
      const int gx = x0 + tx * CVX + v;
      if (gx >= nx) continue;
      float r = acc[v][o];
      if (relu) r = fmaxf(r, 0.f);
      outb[(long long)co * n + (long long)z * plane + (long long)gy * nx + gx] = r;
    }
  }
}

template <bool BF>
static void conv3_launch(const float* in, long long in_bs, int ci, float* out, long long out_bs, int co,
                         const float* W, const float* bias, bool relu, int B, int nx, int ny, int nz, cudaStream_t st) {
  constexpr int CO = 8;
  if (co <= 16) {
    constexpr int CG = 2, TY = UT / ((CX / CVX) * CG);
    dim3 grid((nx + CX - 1) / CX, (ny + TY - 1) / TY, B * nz * ((co + CO * CG - 1) / (CO * CG)));
    if (ci == 1)
      k_conv3<CO, CG, 1, BF><<<grid, UT, 0, st>>>(in, in_bs, ci, out, out_bs, co, W, bias, relu, nx, ny, nz);
    else
      k_conv3<CO, CG, 4, BF><<<grid, UT, 0, st>>>(in, in_bs, ci, out, out_bs, co, W, bias, relu, nx, ny, nz);
  } else {
    constexpr int CG = 4, TY = UT / ((CX / CVX) * CG);
    dim3 grid((nx + CX - 1) / CX, (ny + TY - 1) / TY, B * nz * ((co + CO * CG - 1) / (CO * CG)));
    if (ci == 1)
      k_conv3<CO, CG, 1, BF><<<grid, UT, 0, st>>>(in, in_bs, ci, out, out_bs, co, W, bias, relu, nx, ny, nz);
    else
      k_conv3<CO, CG, 4, BF><<<grid, UT, 0, st>>>(in, in_bs, ci, out, out_bs, co, W, bias, relu, nx, ny, nz);
  }
}
// Tensor-core path of a network (BF16 only): packed-weight scratch, error word, switch.
struct TcCtx {
  uint4* wpk;
  int* err;
  bool on;
};

static cudaError_t conv3(bool bf, const float* in, long long in_bs, int ci, float* out, long long out_bs, int co,
                         const float* W, const float* bias, bool relu, int B, int nx, int ny, int nz, cudaStream_t st,
                         const TcCtx& tc) {
  if (bf && tc.on && unet_conv3_tc_supported(ci, co, nx, ny))
    return unet_conv3_tc(in, in_bs, ci, out, out_bs, co, W, bias, relu, B, nx, ny, nz, tc.wpk, tc.err, st);
  // grid.z = samples * nz * channel blocks must stay <= 65535: launch sample chunks
  const int per = std::max(1, 65535 / (nz * ((co + 15) / 16)));
  for (int b0 = 0; b0 < B; b0 += per) {
    const int bc = std::min(per, B - b0);
    const float* i0 = in + (long long)b0 * in_bs;
    float* o0 = out + (long long)b0 * out_bs;
    if (bf) conv3_launch<true>(i0, in_bs, ci, o0, out_bs, co, W, bias, relu, bc, nx, ny, nz, st);
    else conv3_launch<false>(i0, in_bs, ci, o0, out_bs, co, W, bias, relu, bc, nx, ny, nz, st);
  }
  return cudaGetLastError();
}

// W'[ci][co][26 - tap] = W[co][ci][tap]: the dgrad of a 3x3x3 conv is the conv of the output
// gradient with these weights.
__global__ void k_flip(const float* __restrict__ W, float* __restrict__ Wf, int ci_n, int co_n) {
  const int total = ci_n * co_n * 27;
  for (int e = blockIdx.x * UT + threadIdx.x; e < total; e += gridDim.x * UT) {
    const int tap = e % 27, ci = (e / 27) % ci_n, co = e / (27 * ci_n);
    Wf[((long long)ci * co_n + co) * 27 + (26 - tap)] = W[e];
  }
}

// dW[co][ci][tap] += sum_{b, v} G[b][co][v] in[b][ci][v + tap], for one input channel ci and 16
// output channels per CTA; CTAs stride over (sample, plane, 4-row) chunks; atomics combine them.
constexpr int WG_CO = 16, WG_ROWS = 4;
__global__ void __launch_bounds__(WG_CO * 27) k_wgrad3(const float* __restrict__ in, long long in_bs, int ci_n,
                                                       const float* __restrict__ G, long long g_bs, int co_n,
                                                       float* __restrict__ dW, int B, int nx, int ny, int nz, int bf) {
  extern __shared__ float sm[];
  const int IXH = nx + 2, halo = 3 * (WG_ROWS + 2) * IXH, vox = WG_ROWS * nx;
  float* s_x = sm;              // [3][ROWS+2][nx+2]
  float* s_g = sm + halo;       // [WG_CO][ROWS][nx]
  const int ci = blockIdx.y, cob = blockIdx.z * WG_CO;
  const int t = threadIdx.x, col = t / 27, tap = t % 27;
  const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
  const long long plane = (long long)nx * ny, n = plane * nz;
  const int row_blocks = (ny + WG_ROWS - 1) / WG_ROWS;
  const long long chunks = (long long)B * nz * row_blocks;
  float acc = 0.f;
  for (long long ch = blockIdx.x; ch < chunks; ch += gridDim.x) {
    const int rb = (int)(ch % row_blocks), z = (int)((ch / row_blocks) % nz), b = (int)(ch / ((long long)row_blocks * nz));
    const int y0 = rb * WG_ROWS;
    __syncthreads();
    for (int e = t; e < halo; e += blockDim.x) {
      const int xi = e % IXH, yi = (e / IXH) % (WG_ROWS + 2), zi = e / (IXH * (WG_ROWS + 2));
      const int gx = xi - 1, gy = y0 + yi - 1, gz = z + zi - 1;
      float v = 0.f;
      if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz)
        v = in[(long long)b * in_bs + (long long)ci * n + (long long)gz * plane + (long long)gy * nx + gx];
      s_x[e] = opr(v, bf);
    }
    for (int e = t; e < WG_CO * vox; e += blockDim.x) {
      const int o = e / vox, r = (e % vox) / nx, x = e % nx;
      const int co = cob + o, gy = y0 + r;
      s_g[e] = (co < co_n && gy < ny) ? opr(G[(long long)b * g_bs + (long long)co * n + (long long)z * plane + (long long)gy * nx + x], bf) : 0.f;
    }
    __syncthreads();
    if (col < WG_CO) {
      const float* g = s_g + col * vox;
      for (int r = 0; r < WG_ROWS; ++r) {
        const float* xr = s_x + (dz * (WG_ROWS + 2) + r + dy) * IXH + dx;
        const float* gr = g + r * nx;
        for (int x = 0; x < nx; ++x) acc = fmaf(gr[x], xr[x], acc);
      }
    }
  }
  if (col < WG_CO && cob + col < co_n) atomicAdd(&dW[((long long)(cob + col) * ci_n + ci) * 27 + tap], acc);
}

// db[c] += sum_{b, v} G[b][c][v]
__global__ void __launch_bounds__(UT) k_bias_grad(const float* __restrict__ G, long long g_bs, int c_n, int B,
                                                  long long n, float* __restrict__ db) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (long long i = threadIdx.x; i < (long long)B * n; i += UT) {
    const long long b = i / n, v = i % n;
    acc += G[b * g_bs + (long long)c * n + v];
  }
  __shared__ float red[UT];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = UT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) db[c] += red[0];
}

// ---------------------------------------------------------------- pooling, transposed conv, 1x1 conv

// 2^3 max-pool: out[b][c][v] over the 8 children of v; arg[] keeps which child won.
__global__ void k_pool_fwd(const float* __restrict__ in, long long in_bs, float* __restrict__ out,
                           unsigned char* __restrict__ arg, int C, int B, int nx, int ny, int nz) {
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2;
  const long long on = (long long)ox * oy * oz, n = (long long)nx * ny * nz, total = (long long)B * C * on;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < total; i += (long long)gridDim.x * UT) {
    const long long v = i % on, bc = i / on;
    const int c = (int)(bc % C), b = (int)(bc / C);
    const int x = (int)(v % ox), y = (int)((v / ox) % oy), z = (int)(v / ((long long)ox * oy));
    const float* src = in + (long long)b * in_bs + (long long)c * n;
    float best = -INFINITY;
    int bi = 0;
    for (int d = 0; d < 8; ++d) {
      const float val = src[(long long)(2 * z + (d >> 2)) * nx * ny + (long long)(2 * y + ((d >> 1) & 1)) * nx + 2 * x + (d & 1)];
      if (val > best) {
        best = val;
        bi = d;
      }
    }
    out[i] = best;
    arg[i] = (unsigned char)bi;
  }
}

// din[child] += dout for the winning child of every pooled voxel (children are disjoint).
__global__ void k_pool_bwd(const float* __restrict__ dout, const unsigned char* __restrict__ arg,
                           float* __restrict__ din, long long din_bs, int C, int B, int nx, int ny, int nz) {
  const int ox = nx / 2, oy = ny / 2, oz = nz / 2;
  const long long on = (long long)ox * oy * oz, n = (long long)nx * ny * nz, total = (long long)B * C * on;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < total; i += (long long)gridDim.x * UT) {
    const long long v = i % on, bc = i / on;
    const int c = (int)(bc % C), b = (int)(bc / C);
    const int x = (int)(v % ox), y = (int)((v / ox) % oy), z = (int)(v / ((long long)ox * oy));
    const int d = arg[i];
    din[(long long)b * din_bs + (long long)c * n + (long long)(2 * z + (d >> 2)) * nx * ny +
        (long long)(2 * y + ((d >> 1) & 1)) * nx + 2 * x + (d & 1)] += dout[i];
  }
}

// Transposed conv, kernel 2^3, stride 2: out[b][co][2v + d] = bias[co] + sum_ci W[ci][co][d] in[b][ci][v].
// (nx, ny, nz) are the OUTPUT dimensions.
__global__ void k_tconv_fwd(const float* __restrict__ in, int ci_n, float* __restrict__ out, long long out_bs,
                            int co_n, const float* __restrict__ W, const float* __restrict__ bias, int B, int nx,
                            int ny, int nz, int bf) {
  const long long n = (long long)nx * ny * nz, total = (long long)B * co_n * n;
  const int ix = nx / 2, iy = ny / 2;
  const long long in_n = n / 8;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < total; i += (long long)gridDim.x * UT) {
    const long long v = i % n, bc = i / n;
    const int co = (int)(bc % co_n), b = (int)(bc / co_n);
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / ((long long)nx * ny));
    const int d = ((z & 1) << 2) | ((y & 1) << 1) | (x & 1);
    const long long iv = (long long)(z >> 1) * ix * iy + (long long)(y >> 1) * ix + (x >> 1);
    float acc = bias[co];
    for (int ci = 0; ci < ci_n; ++ci)
      acc = fmaf(opr(__ldg(&W[((long long)ci * co_n + co) * 8 + d]), bf), opr(in[((long long)b * ci_n + ci) * in_n + iv], bf), acc);
    out[(long long)b * out_bs + (long long)co * n + v] = acc;
  }
}

// din[b][ci][v] = sum_co sum_d W[ci][co][d] dout[b][co][2v + d]  ((nx, ny, nz) = output dims)
__global__ void k_tconv_dgrad(const float* __restrict__ dout, long long dout_bs, int co_n, float* __restrict__ din,
                              int ci_n, const float* __restrict__ W, int B, int nx, int ny, int nz, int bf) {
  const long long n = (long long)nx * ny * nz, in_n = n / 8, total = (long long)B * ci_n * in_n;
  const int ix = nx / 2, iy = ny / 2;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < total; i += (long long)gridDim.x * UT) {
    const long long v = i % in_n, bc = i / in_n;
    const int ci = (int)(bc % ci_n), b = (int)(bc / ci_n);
    const int x = (int)(v % ix), y = (int)((v / ix) % iy), z = (int)(v / ((long long)ix * iy));
    float acc = 0.f;
    for (int co = 0; co < co_n; ++co) {
      const float* g = dout + (long long)b * dout_bs + (long long)co * n;
      for (int d = 0; d < 8; ++d)
        acc = fmaf(opr(__ldg(&W[((long long)ci * co_n + co) * 8 + d]), bf),
                   opr(g[(long long)(2 * z + (d >> 2)) * nx * ny + (long long)(2 * y + ((d >> 1) & 1)) * nx + 2 * x + (d & 1)], bf),
                   acc);
    }
    din[i] = acc;
  }
}

// dW[ci][co][d] += sum_{b, v} in[b][ci][v] dout[b][co][2v + d]: one CTA per (ci, co).
__global__ void __launch_bounds__(UT) k_tconv_wgrad(const float* __restrict__ in, int ci_n,
                                                    const float* __restrict__ dout, long long dout_bs, int co_n,
                                                    float* __restrict__ dW, int B, int nx, int ny, int nz, int bf) {
  const int ci = blockIdx.x, co = blockIdx.y;
  const long long n = (long long)nx * ny * nz, in_n = n / 8;
  const int ix = nx / 2, iy = ny / 2;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (long long i = threadIdx.x; i < (long long)B * in_n; i += UT) {
    const long long b = i / in_n, v = i % in_n;
    const int x = (int)(v % ix), y = (int)((v / ix) % iy), z = (int)(v / ((long long)ix * iy));
    const float xv = opr(in[(b * ci_n + ci) * in_n + v], bf);
    const float* g = dout + b * dout_bs + (long long)co * n;
#pragma unroll
    for (int d = 0; d < 8; ++d)
      acc[d] = fmaf(xv, opr(g[(long long)(2 * z + (d >> 2)) * nx * ny + (long long)(2 * y + ((d >> 1) & 1)) * nx + 2 * x + (d & 1)], bf),
                    acc[d]);
  }
  __shared__ float red[8][UT];
#pragma unroll
  for (int d = 0; d < 8; ++d) red[d][threadIdx.x] = acc[d];
  __syncthreads();
  for (int o = UT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int d = 0; d < 8; ++d) red[d][threadIdx.x] += red[d][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x < 8) dW[((long long)ci * co_n + co) * 8 + threadIdx.x] += red[threadIdx.x][0];
}

// 1x1x1 conv to one channel: out[b][v] = bias + sum_c W[c] in[b][c][v]
__global__ void k_conv1_fwd(const float* __restrict__ in, int c_n, const float* __restrict__ W,
                            const float* __restrict__ bias, float* __restrict__ out, int B, long long n, int bf) {
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < (long long)B * n; i += (long long)gridDim.x * UT) {
    const long long b = i / n, v = i % n;
    float acc = bias[0];
    for (int c = 0; c < c_n; ++c) acc = fmaf(opr(W[c], bf), opr(in[(b * c_n + c) * n + v], bf), acc);
    out[i] = acc;
  }
}
// din[b][c][v] = W[c] dout[b][v]
__global__ void k_conv1_dgrad(const float* __restrict__ dout, int c_n, const float* __restrict__ W,
                              float* __restrict__ din, int B, long long n, int bf) {
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < (long long)B * c_n * n; i += (long long)gridDim.x * UT) {
    const long long v = i % n, bc = i / n;
    const int c = (int)(bc % c_n);
    const long long b = bc / c_n;
    din[i] = opr(W[c], bf) * opr(dout[b * n + v], bf);
  }
}
// dW[c] += sum in[b][c][v] dout[b][v] (one CTA per channel; c == c_n: the bias)
__global__ void __launch_bounds__(UT) k_conv1_wgrad(const float* __restrict__ in, int c_n,
                                                    const float* __restrict__ dout, float* __restrict__ dW,
                                                    float* __restrict__ db, int B, long long n, int bf) {
  const int c = blockIdx.x;
  float acc = 0.f;
  for (long long i = threadIdx.x; i < (long long)B * n; i += UT) {
    const long long b = i / n, v = i % n;
    acc += (c < c_n ? opr(in[(b * c_n + c) * n + v], bf) * opr(dout[i], bf) : dout[i]);
  }
  __shared__ float red[UT];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = UT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (c < c_n) dW[c] += red[0];
    else db[0] += red[0];
  }
}

// g <- g * (y > 0) for a ReLU output y (sample strides allow concat views)
__global__ void k_relu_bwd(float* __restrict__ g, long long g_bs, const float* __restrict__ y, long long y_bs,
                           int C, int B, long long n) {
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < (long long)B * C * n; i += (long long)gridDim.x * UT) {
    const long long b = i / ((long long)C * n), r = i % ((long long)C * n);
    if (!(y[b * y_bs + r] > 0.f)) g[b * g_bs + r] = 0.f;
  }
}

// MSE: loss = mean (p - t)^2, g = 2 (p - t) / N; loss accumulated in FP64 partials.
__global__ void __launch_bounds__(UT) k_mse(const float* __restrict__ p, const float* __restrict__ t,
                                            float* __restrict__ g, long long N, double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < N; i += (long long)gridDim.x * UT) {
    const float d = p[i] - t[i];
    g[i] = 2.0f * d / (float)N;
    acc += (double)d * d;
  }
  __shared__ double red[UT];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = UT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}
__global__ void k_mse_final(const double* part, int nb, long long N, double* loss) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < nb; ++i) a += part[i];
    *loss = a / (double)N;
  }
}

// Adam (Kingma and Ba, 2015): m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2; p -= lr_t m / (sqrt(v) + eps_t)
__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long count, float lr_t, float b1, float b2, float eps_t) {
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < count; i += (long long)gridDim.x * UT) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr_t * mi / (sqrtf(vi) + eps_t);
  }
}

// Per-sample normalisation (one CTA per sample): m = sum(x_b) / norm_count in FP64,
// xo = x / m, to = t / m (m <= 0 leaves the sample unscaled).
constexpr int NORM_T = 1024;
__global__ void __launch_bounds__(NORM_T) k_sample_norm(const float* __restrict__ x, const float* __restrict__ t,
                                                        float* __restrict__ xo, float* __restrict__ to, long long n,
                                                        double norm_count) {
  const long long base = (long long)blockIdx.x * n;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < n; i += NORM_T) acc += (double)x[base + i];
  __shared__ double red[NORM_T];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = NORM_T / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double m = red[0] / norm_count;
  const float inv = m > 0.0 ? (float)(1.0 / m) : 1.0f;
  for (long long i = threadIdx.x; i < n; i += NORM_T) {
    xo[base + i] = x[base + i] * inv;
    if (t) to[base + i] = t[base + i] * inv;
  }
}

// FP64 partial sums of x over a grid-stride split (one partial per CTA).
__global__ void __launch_bounds__(UT) k_sum_part(const float* __restrict__ x, long long n, double* __restrict__ part) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < n; i += (long long)gridDim.x * UT) acc += x[i];
  __shared__ double red[UT];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = UT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__device__ double mean_of_parts(const double* part, int np, double norm_count) {
  __shared__ double m_s;
  if (threadIdx.x == 0) {
    double a = 0.0;
    for (int i = 0; i < np; ++i) a += part[i];
    m_s = a / norm_count;
  }
  __syncthreads();
  return m_s;
}

// xo = x / m, m = sum(x) / norm_count from the partials (m <= 0 leaves x unscaled)
__global__ void __launch_bounds__(UT) k_scale_by_mean(const float* __restrict__ x, long long n,
                                                     const double* __restrict__ part, int np, double norm_count,
                                                     float* __restrict__ xo) {
  const double m = mean_of_parts(part, np, norm_count);
  const float inv = m > 0.0 ? (float)(1.0 / m) : 1.0f;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < n; i += (long long)gridDim.x * UT) xo[i] = x[i] * inv;
}

// r_init = m * max(out, floor): the network's output back in the input's units, kept positive.
__global__ void __launch_bounds__(UT) k_warm_map(const float* __restrict__ out, long long n,
                                                 const double* __restrict__ part, int np, double norm_count,
                                                 float floor_rel, float* __restrict__ r) {
  const double m = mean_of_parts(part, np, norm_count);
  const float sc = m > 0.0 ? (float)m : 1.0f;
  for (long long i = (long long)blockIdx.x * UT + threadIdx.x; i < n; i += (long long)gridDim.x * UT)
    r[i] = sc * fmaxf(out[i], floor_rel);
}

static unsigned grid_for(long long work) {
  long long b = (work + UT - 1) / UT;
  return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

}  // namespace unet
}  // namespace clamp

using namespace clamp::unet;

struct clamp_unet {
  int c1, c2, c3, dev, bf;
  std::vector<Layer> layers;
  size_t count = 0;
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr, *flip = nullptr;
  size_t flip_count = 0;
  uint4* wpk = nullptr;   // BF16 packed weights of the conv on the tensor cores
  int* err = nullptr;     // device word: bit 2 = a tensor-core wait gave up
  int tc = 1;             // BF16 convs on the tensor cores where supported
  TcCtx ctx() const { return TcCtx{wpk, err, bf != 0 && tc != 0}; }
};

// Workspace: activations and their gradients for batch B at (nx, ny, nz).
namespace {
struct Acts {
  float *e1a, *cat1, *p1, *e2a, *cat2, *p2, *bta, *btb, *d2a, *d2b, *d1a, *d1b, *out, *xin;
  float *ge1a, *gcat1, *gp1, *ge2a, *gcat2, *gp2, *gbta, *gbtb, *gd2a, *gd2b, *gd1a, *gd1b, *gout;
  unsigned char *arg1, *arg2;
  double* part;
  size_t bytes;
};

Acts acts_layout(const clamp_unet* u, int B, int nx, int ny, int nz, void* base, bool with_grads) {
  const long long n1 = (long long)nx * ny * nz, n2 = n1 / 8, n3 = n1 / 64;
  size_t off = 0;
  char* b = static_cast<char*>(base);
  auto take = [&](long long floats) -> float* {
    float* r = b ? reinterpret_cast<float*>(b + off) : nullptr;
    off += ((size_t)floats * sizeof(float) + 255) & ~(size_t)255;
    return r;
  };
  Acts a{};
  const int c1 = u->c1, c2 = u->c2, c3 = u->c3;
  float** fw[] = {&a.e1a, &a.cat1, &a.p1, &a.e2a, &a.cat2, &a.p2, &a.bta, &a.btb, &a.d2a, &a.d2b, &a.d1a, &a.d1b, &a.out};
  const long long sz[] = {c1 * n1, 2LL * c1 * n1, c1 * n2, c2 * n2, 2LL * c2 * n2, c2 * n3, c3 * n3, c3 * n3,
                          c2 * n2, c2 * n2, c1 * n1, c1 * n1, n1};
  for (int i = 0; i < 13; ++i) *fw[i] = take(B * sz[i]);
  a.xin = take(B * n1);
  if (with_grads) {
    float** gw[] = {&a.ge1a, &a.gcat1, &a.gp1, &a.ge2a, &a.gcat2, &a.gp2, &a.gbta, &a.gbtb, &a.gd2a, &a.gd2b, &a.gd1a, &a.gd1b, &a.gout};
    for (int i = 0; i < 13; ++i) *gw[i] = take(B * sz[i]);
  }
  a.arg1 = reinterpret_cast<unsigned char*>(take((B * c1 * n2 + 3) / 4));
  a.arg2 = reinterpret_cast<unsigned char*>(take((B * c2 * n3 + 3) / 4));
  a.part = reinterpret_cast<double*>(take(2 * 152 * 16));
  a.bytes = off;
  return a;
}

bool unet_shape_ok(int B, int nx, int ny, int nz) {
  return B >= 1 && nx >= 4 && ny >= 4 && nz >= 4 && nx % 4 == 0 && ny % 4 == 0 && nz % 4 == 0;
}
}  // namespace

extern "C" clamp_status clamp_unet_create(int32_t c1, int32_t c2, int32_t c3, int32_t dtype, const float* params_host,
                                          clamp_unet** out) {
  if (!out || c1 < 1 || c2 < 1 || c3 < 1 || c1 > 256 || c2 > 256 || c3 > 256)
    return api_fail(CLAMP_EINVAL, "clamp_unet_create: channel counts must be in [1, 256]");
  if (dtype != CLAMP_DENOISER_FP32 && dtype != CLAMP_DENOISER_BF16)
    return api_fail(CLAMP_EINVAL, "clamp_unet_create: dtype must be CLAMP_DENOISER_FP32 or CLAMP_DENOISER_BF16");
  clamp_unet* u = new clamp_unet();
  u->bf = dtype == CLAMP_DENOISER_BF16;
  u->c1 = c1;
  u->c2 = c2;
  u->c3 = c3;
  cudaGetDevice(&u->dev);
  const int spec[13][3] = {{CONV3, 1, c1},      {CONV3, c1, c1}, {CONV3, c1, c2}, {CONV3, c2, c2}, {CONV3, c2, c3},
                           {CONV3, c3, c3},     {TCONV, c3, c2}, {CONV3, 2 * c2, c2}, {CONV3, c2, c2},
                           {TCONV, c2, c1},     {CONV3, 2 * c1, c1}, {CONV3, c1, c1}, {CONV1, c1, 1}};
  size_t off = 0;
  for (auto& s : spec) {
    Layer L{s[0], s[1], s[2], 0, 0, 0};
    L.nw = (size_t)s[1] * s[2] * (s[0] == CONV3 ? 27 : s[0] == TCONV ? 8 : 1);
    L.w = off;
    off += L.nw;
    L.b = off;
    off += s[2];
    if (s[0] == CONV3) u->flip_count = std::max(u->flip_count, L.nw);
    u->layers.push_back(L);
  }
  u->count = off;
  const size_t bytes = off * sizeof(float);
  size_t wpk_bytes = 16;
  for (const Layer& L : u->layers)
    if (L.kind == CONV3 && L.ci >= 16)   // forward (ci -> co) and data gradient (co -> ci)
      wpk_bytes = std::max({wpk_bytes, clamp::unet_conv3_tc_wpk_bytes(L.ci, L.co),
                            clamp::unet_conv3_tc_wpk_bytes(L.co, L.ci)});
  if (cudaMalloc(&u->p, bytes) != cudaSuccess || cudaMalloc(&u->g, bytes) != cudaSuccess ||
      cudaMalloc(&u->m, bytes) != cudaSuccess || cudaMalloc(&u->v, bytes) != cudaSuccess ||
      cudaMalloc(&u->flip, u->flip_count * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&u->wpk, wpk_bytes) != cudaSuccess || cudaMalloc(&u->err, sizeof(int)) != cudaSuccess) {
    clamp_unet_destroy(u);
    return api_fail(CLAMP_ENOMEM, "clamp_unet_create: device allocation failed");
  }
  cudaError_t e = cudaSuccess;
  for (float* q : {u->g, u->m, u->v})
    if (e == cudaSuccess) e = cudaMemset(q, 0, bytes);
  if (e == cudaSuccess) e = cudaMemset(u->err, 0, sizeof(int));
  if (e == cudaSuccess)
    e = params_host ? cudaMemcpy(u->p, params_host, bytes, cudaMemcpyHostToDevice) : cudaMemset(u->p, 0, bytes);
  if (e != cudaSuccess) {
    clamp_unet_destroy(u);
    return api_fail(CLAMP_ECUDA, "clamp_unet_create: %s", cudaGetErrorString(e));
  }
  *out = u;
  return CLAMP_OK;
}

extern "C" void clamp_unet_destroy(clamp_unet* u) {
  if (!u) return;
  for (float* q : {u->p, u->g, u->m, u->v, u->flip})
    if (q) cudaFree(q);
  if (u->wpk) cudaFree(u->wpk);
  if (u->err) cudaFree(u->err);
  delete u;
}

extern "C" int64_t clamp_unet_param_count(const clamp_unet* u) { return u ? (int64_t)u->count : 0; }

static float* unet_state(const clamp_unet* u, int which) {
  switch (which) {
    case 0: return u->p;
    case 1: return u->g;
    case 2: return u->m;
    case 3: return u->v;
    default: return nullptr;
  }
}

extern "C" clamp_status clamp_unet_get(const clamp_unet* u, int32_t which, float* host) {
  if (!u || !host || !unet_state(u, which)) return api_fail(CLAMP_EINVAL, "clamp_unet_get: bad arguments");
  const cudaError_t e = cudaMemcpy(host, unet_state(u, which), u->count * sizeof(float), cudaMemcpyDeviceToHost);
  return e == cudaSuccess ? CLAMP_OK : api_fail(CLAMP_ECUDA, "clamp_unet_get: %s", cudaGetErrorString(e));
}

extern "C" clamp_status clamp_unet_set(clamp_unet* u, int32_t which, const float* host) {
  if (!u || !host || !unet_state(u, which)) return api_fail(CLAMP_EINVAL, "clamp_unet_set: bad arguments");
  const cudaError_t e = cudaMemcpy(unet_state(u, which), host, u->count * sizeof(float), cudaMemcpyHostToDevice);
  return e == cudaSuccess ? CLAMP_OK : api_fail(CLAMP_ECUDA, "clamp_unet_set: %s", cudaGetErrorString(e));
}

extern "C" size_t clamp_unet_workspace_size(const clamp_unet* u, int32_t batch, int32_t nx, int32_t ny, int32_t nz,
                                            int32_t training) {
  if (!u || !unet_shape_ok(batch, nx, ny, nz)) return 0;
  return acts_layout(u, batch, nx, ny, nz, nullptr, training != 0).bytes;
}

// The network's buffers live on the device it was created on.
static bool on_unet_device(const clamp_unet* u, const char* where) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != u->dev) {
    api_fail(CLAMP_EINVAL, "%s: the network was created on device %d, current device is %d", where, u->dev, dev);
    return false;
  }
  return true;
}

#define U_TRY(x)                                                                       \
  do {                                                                                 \
    cudaError_t _e = (x);                                                              \
    if (_e != cudaSuccess) return api_fail(CLAMP_ECUDA, "unet: %s", cudaGetErrorString(_e)); \
  } while (0)

static clamp_status unet_forward(clamp_unet* u, const float* x, int B, int nx, int ny, int nz, const Acts& a,
                                 cudaStream_t st) {
  const bool bf = u->bf != 0;
  const int c1 = u->c1, c2 = u->c2, c3 = u->c3;
  const long long n1 = (long long)nx * ny * nz, n2 = n1 / 8, n3 = n1 / 64;
  const int hx = nx / 2, hy = ny / 2, hz = nz / 2, qx = nx / 4, qy = ny / 4, qz = nz / 4;
  auto W = [&](int i) { return u->p + u->layers[i].w; };
  auto Bi = [&](int i) { return u->p + u->layers[i].b; };
  U_TRY(conv3(bf, x, n1, 1, a.e1a, c1 * n1, c1, W(0), Bi(0), true, B, nx, ny, nz, st, u->ctx()));
  U_TRY(conv3(bf, a.e1a, c1 * n1, c1, a.cat1 + c1 * n1, 2 * c1 * n1, c1, W(1), Bi(1), true, B, nx, ny, nz, st, u->ctx()));  // s1
  k_pool_fwd<<<grid_for(B * c1 * n2), UT, 0, st>>>(a.cat1 + c1 * n1, 2 * c1 * n1, a.p1, a.arg1, c1, B, nx, ny, nz);
  U_TRY(cudaGetLastError());
  U_TRY(conv3(bf, a.p1, c1 * n2, c1, a.e2a, c2 * n2, c2, W(2), Bi(2), true, B, hx, hy, hz, st, u->ctx()));
  U_TRY(conv3(bf, a.e2a, c2 * n2, c2, a.cat2 + c2 * n2, 2 * c2 * n2, c2, W(3), Bi(3), true, B, hx, hy, hz, st, u->ctx()));  // s2
  k_pool_fwd<<<grid_for(B * c2 * n3), UT, 0, st>>>(a.cat2 + c2 * n2, 2 * c2 * n2, a.p2, a.arg2, c2, B, hx, hy, hz);
  U_TRY(cudaGetLastError());
  U_TRY(conv3(bf, a.p2, c2 * n3, c2, a.bta, c3 * n3, c3, W(4), Bi(4), true, B, qx, qy, qz, st, u->ctx()));
  U_TRY(conv3(bf, a.bta, c3 * n3, c3, a.btb, c3 * n3, c3, W(5), Bi(5), true, B, qx, qy, qz, st, u->ctx()));
  k_tconv_fwd<<<grid_for(B * c2 * n2), UT, 0, st>>>(a.btb, c3, a.cat2, 2 * c2 * n2, c2, W(6), Bi(6), B, hx, hy, hz, bf);
  U_TRY(cudaGetLastError());
  U_TRY(conv3(bf, a.cat2, 2 * c2 * n2, 2 * c2, a.d2a, c2 * n2, c2, W(7), Bi(7), true, B, hx, hy, hz, st, u->ctx()));
  U_TRY(conv3(bf, a.d2a, c2 * n2, c2, a.d2b, c2 * n2, c2, W(8), Bi(8), true, B, hx, hy, hz, st, u->ctx()));
  k_tconv_fwd<<<grid_for(B * c1 * n1), UT, 0, st>>>(a.d2b, c2, a.cat1, 2 * c1 * n1, c1, W(9), Bi(9), B, nx, ny, nz, bf);
  U_TRY(cudaGetLastError());
  U_TRY(conv3(bf, a.cat1, 2 * c1 * n1, 2 * c1, a.d1a, c1 * n1, c1, W(10), Bi(10), true, B, nx, ny, nz, st, u->ctx()));
  U_TRY(conv3(bf, a.d1a, c1 * n1, c1, a.d1b, c1 * n1, c1, W(11), Bi(11), true, B, nx, ny, nz, st, u->ctx()));
  k_conv1_fwd<<<grid_for(B * n1), UT, 0, st>>>(a.d1b, c1, W(12), Bi(12), a.out, B, n1, bf);
  U_TRY(cudaGetLastError());
  return CLAMP_OK;
}

extern "C" clamp_status clamp_unet_forward(clamp_unet* u, const float* x, float* y, int32_t batch, int32_t nx,
                                           int32_t ny, int32_t nz, void* ws, size_t ws_bytes, void* stream) {
  if (!u || !x || !y) return api_fail(CLAMP_EINVAL, "clamp_unet_forward: NULL argument");
  if (!on_unet_device(u, "clamp_unet_forward")) return CLAMP_EINVAL;
  if (!unet_shape_ok(batch, nx, ny, nz))
    return api_fail(CLAMP_EINVAL, "clamp_unet_forward: nx, ny, nz must be multiples of 4");
  const Acts a = acts_layout(u, batch, nx, ny, nz, ws, false);
  if (!ws || ws_bytes < a.bytes) return api_fail(CLAMP_ENOMEM, "clamp_unet_forward: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  clamp_status s = unet_forward(u, x, batch, nx, ny, nz, a, st);
  if (s != CLAMP_OK) return s;
  const long long n1 = (long long)nx * ny * nz;
  U_TRY(cudaMemcpyAsync(y, a.out, sizeof(float) * batch * n1, cudaMemcpyDeviceToDevice, st));
  return CLAMP_OK;
}

// conv3 backward for layer li: input `in` (ci channels, sample stride in_bs), output gradient
// `g` (co channels, stride g_bs); writes din (if non-NULL) and accumulates dW, db.
static clamp_status conv3_bwd(clamp_unet* u, int li, const float* in, long long in_bs, const float* g, long long g_bs,
                              float* din, long long din_bs, int B, int nx, int ny, int nz, cudaStream_t st) {
  const Layer& L = u->layers[li];
  const bool bf = u->bf != 0;
  const long long n = (long long)nx * ny * nz;
  if (din) {
    k_flip<<<grid_for((long long)L.nw), UT, 0, st>>>(u->p + L.w, u->flip, L.ci, L.co);
    U_TRY(cudaGetLastError());
    U_TRY(conv3(bf, g, g_bs, L.co, din, din_bs, L.ci, u->flip, nullptr, false, B, nx, ny, nz, st, u->ctx()));
  }
  const size_t smem = sizeof(float) * (3 * (WG_ROWS + 2) * (nx + 2) + WG_CO * WG_ROWS * nx);
  U_TRY(cudaFuncSetAttribute(k_wgrad3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const long long chunks = (long long)B * nz * ((ny + WG_ROWS - 1) / WG_ROWS);
  const long long rest = (long long)L.ci * ((L.co + WG_CO - 1) / WG_CO);
  const long long want = std::max(1LL, std::min(chunks, (4LL * 152 + rest - 1) / rest));
  dim3 grid((unsigned)want, L.ci, (L.co + WG_CO - 1) / WG_CO);
  k_wgrad3<<<grid, WG_CO * 27, smem, st>>>(in, in_bs, L.ci, g, g_bs, L.co, u->g + L.w, B, nx, ny, nz, u->bf);
  U_TRY(cudaGetLastError());
  k_bias_grad<<<L.co, UT, 0, st>>>(g, g_bs, L.co, B, n, u->g + L.b);
  U_TRY(cudaGetLastError());
  return CLAMP_OK;
}

extern "C" clamp_status clamp_unet_backward(clamp_unet* u, const float* x, const float* target, int32_t batch,
                                            int32_t nx, int32_t ny, int32_t nz, double* loss, void* ws,
                                            size_t ws_bytes, void* stream) {
  if (!u || !x || !target) return api_fail(CLAMP_EINVAL, "clamp_unet_backward: NULL argument");
  if (!on_unet_device(u, "clamp_unet_backward")) return CLAMP_EINVAL;
  if (!unet_shape_ok(batch, nx, ny, nz))
    return api_fail(CLAMP_EINVAL, "clamp_unet_backward: nx, ny, nz must be multiples of 4");
  const Acts a = acts_layout(u, batch, nx, ny, nz, ws, true);
  if (!ws || ws_bytes < a.bytes) return api_fail(CLAMP_ENOMEM, "clamp_unet_backward: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const int bf = u->bf;
  const int B = batch, c1 = u->c1, c2 = u->c2, c3 = u->c3;
  const long long n1 = (long long)nx * ny * nz, n2 = n1 / 8, n3 = n1 / 64;
  const int hx = nx / 2, hy = ny / 2, hz = nz / 2, qx = nx / 4, qy = ny / 4, qz = nz / 4;
  clamp_status s = unet_forward(u, x, B, nx, ny, nz, a, st);
  if (s != CLAMP_OK) return s;
  U_TRY(cudaMemsetAsync(u->g, 0, u->count * sizeof(float), st));
  // loss and its gradient
  const unsigned nb = grid_for(B * n1);
  k_mse<<<nb, UT, 0, st>>>(a.out, target, a.gout, B * n1, a.part);
  U_TRY(cudaGetLastError());
  if (loss) {
    k_mse_final<<<1, 32, 0, st>>>(a.part, (int)nb, B * n1, loss);
    U_TRY(cudaGetLastError());
  }
  auto W = [&](int i) { return u->p + u->layers[i].w; };
  // output 1x1 conv
  k_conv1_dgrad<<<grid_for(B * c1 * n1), UT, 0, st>>>(a.gout, c1, W(12), a.gd1b, B, n1, bf);
  k_conv1_wgrad<<<c1 + 1, UT, 0, st>>>(a.d1b, c1, a.gout, u->g + u->layers[12].w, u->g + u->layers[12].b, B, n1, bf);
  U_TRY(cudaGetLastError());
  // decoder level 1
  k_relu_bwd<<<grid_for(B * c1 * n1), UT, 0, st>>>(a.gd1b, c1 * n1, a.d1b, c1 * n1, c1, B, n1);
  s = conv3_bwd(u, 11, a.d1a, c1 * n1, a.gd1b, c1 * n1, a.gd1a, c1 * n1, B, nx, ny, nz, st);
  if (s != CLAMP_OK) return s;
  k_relu_bwd<<<grid_for(B * c1 * n1), UT, 0, st>>>(a.gd1a, c1 * n1, a.d1a, c1 * n1, c1, B, n1);
  s = conv3_bwd(u, 10, a.cat1, 2 * c1 * n1, a.gd1a, c1 * n1, a.gcat1, 2 * c1 * n1, B, nx, ny, nz, st);
  if (s != CLAMP_OK) return s;
  // transposed conv up1: u1 = cat1[:, :c1] from d2b
  k_tconv_dgrad<<<grid_for(B * c2 * n2), UT, 0, st>>>(a.gcat1, 2 * c1 * n1, c1, a.gd2b, c2, W(9), B, nx, ny, nz, bf);
  k_tconv_wgrad<<<dim3(c2, c1), UT, 0, st>>>(a.d2b, c2, a.gcat1, 2 * c1 * n1, c1, u->g + u->layers[9].w, B, nx, ny, nz, bf);
  k_bias_grad<<<c1, UT, 0, st>>>(a.gcat1, 2 * c1 * n1, c1, B, n1, u->g + u->layers[9].b);
  U_TRY(cudaGetLastError());
  // decoder level 2
  k_relu_bwd<<<grid_for(B * c2 * n2), UT, 0, st>>>(a.gd2b, c2 * n2, a.d2b, c2 * n2, c2, B, n2);
  s = conv3_bwd(u, 8, a.d2a, c2 * n2, a.gd2b, c2 * n2, a.gd2a, c2 * n2, B, hx, hy, hz, st);
  if (s != CLAMP_OK) return s;
  k_relu_bwd<<<grid_for(B * c2 * n2), UT, 0, st>>>(a.gd2a, c2 * n2, a.d2a, c2 * n2, c2, B, n2);
  s = conv3_bwd(u, 7, a.cat2, 2 * c2 * n2, a.gd2a, c2 * n2, a.gcat2, 2 * c2 * n2, B, hx, hy, hz, st);
  if (s != CLAMP_OK) return s;
  // transposed conv up2: u2 = cat2[:, :c2] from btb
  k_tconv_dgrad<<<grid_for(B * c3 * n3), UT, 0, st>>>(a.gcat2, 2 * c2 * n2, c2, a.gbtb, c3, W(6), B, hx, hy, hz, bf);
  k_tconv_wgrad<<<dim3(c3, c2), UT, 0, st>>>(a.btb, c3, a.gcat2, 2 * c2 * n2, c2, u->g + u->layers[6].w, B, hx, hy, hz, bf);
  k_bias_grad<<<c2, UT, 0, st>>>(a.gcat2, 2 * c2 * n2, c2, B, n2, u->g + u->layers[6].b);
  U_TRY(cudaGetLastError());
  // bottleneck
  k_relu_bwd<<<grid_for(B * c3 * n3), UT, 0, st>>>(a.gbtb, c3 * n3, a.btb, c3 * n3, c3, B, n3);
  s = conv3_bwd(u, 5, a.bta, c3 * n3, a.gbtb, c3 * n3, a.gbta, c3 * n3, B, qx, qy, qz, st);
  if (s != CLAMP_OK) return s;
  k_relu_bwd<<<grid_for(B * c3 * n3), UT, 0, st>>>(a.gbta, c3 * n3, a.bta, c3 * n3, c3, B, n3);
  s = conv3_bwd(u, 4, a.p2, c2 * n3, a.gbta, c3 * n3, a.gp2, c2 * n3, B, qx, qy, qz, st);
  if (s != CLAMP_OK) return s;
  // pool 2 into the skip s2 = cat2[:, c2:] (its gradient already holds the concat path)
  k_pool_bwd<<<grid_for(B * c2 * n3), UT, 0, st>>>(a.gp2, a.arg2, a.gcat2 + c2 * n2, 2 * c2 * n2, c2, B, hx, hy, hz);
  U_TRY(cudaGetLastError());
  // encoder level 2
  k_relu_bwd<<<grid_for(B * c2 * n2), UT, 0, st>>>(a.gcat2 + c2 * n2, 2 * c2 * n2, a.cat2 + c2 * n2, 2 * c2 * n2, c2, B, n2);
  s = conv3_bwd(u, 3, a.e2a, c2 * n2, a.gcat2 + c2 * n2, 2 * c2 * n2, a.ge2a, c2 * n2, B, hx, hy, hz, st);
  if (s != CLAMP_OK) return s;
  k_relu_bwd<<<grid_for(B * c2 * n2), UT, 0, st>>>(a.ge2a, c2 * n2, a.e2a, c2 * n2, c2, B, n2);
  s = conv3_bwd(u, 2, a.p1, c1 * n2, a.ge2a, c2 * n2, a.gp1, c1 * n2, B, hx, hy, hz, st);
  if (s != CLAMP_OK) return s;
  // pool 1 into the skip s1 = cat1[:, c1:]
  k_pool_bwd<<<grid_for(B * c1 * n2), UT, 0, st>>>(a.gp1, a.arg1, a.gcat1 + c1 * n1, 2 * c1 * n1, c1, B, nx, ny, nz);
  U_TRY(cudaGetLastError());
  // encoder level 1
  k_relu_bwd<<<grid_for(B * c1 * n1), UT, 0, st>>>(a.gcat1 + c1 * n1, 2 * c1 * n1, a.cat1 + c1 * n1, 2 * c1 * n1, c1, B, n1);
  s = conv3_bwd(u, 1, a.e1a, c1 * n1, a.gcat1 + c1 * n1, 2 * c1 * n1, a.ge1a, c1 * n1, B, nx, ny, nz, st);
  if (s != CLAMP_OK) return s;
  k_relu_bwd<<<grid_for(B * c1 * n1), UT, 0, st>>>(a.ge1a, c1 * n1, a.e1a, c1 * n1, c1, B, n1);
  s = conv3_bwd(u, 0, x, n1, a.ge1a, c1 * n1, nullptr, 0, B, nx, ny, nz, st);
  if (s != CLAMP_OK) return s;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_unet_adam(clamp_unet* u, float lr, float beta1, float beta2, float eps, int32_t t,
                                        void* stream) {
  if (!u || t < 1) return api_fail(CLAMP_EINVAL, "clamp_unet_adam: bad arguments");
  if (!on_unet_device(u, "clamp_unet_adam")) return CLAMP_EINVAL;
  const double bc1 = 1.0 - pow((double)beta1, t), bc2 = 1.0 - pow((double)beta2, t);
  const float lr_t = (float)(lr * sqrt(bc2) / bc1), eps_t = (float)(eps * sqrt(bc2));
  k_adam<<<grid_for((long long)u->count), UT, 0, (cudaStream_t)stream>>>(u->p, u->g, u->m, u->v, (long long)u->count,
                                                                          lr_t, beta1, beta2, eps_t);
  U_TRY(cudaGetLastError());
  return CLAMP_OK;
}

extern "C" clamp_status clamp_unet_set_tensor_cores(clamp_unet* u, int32_t on) {
  if (!u || (on != 0 && on != 1)) return api_fail(CLAMP_EINVAL, "clamp_unet_set_tensor_cores: bad arguments");
  u->tc = on;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_unet_check(clamp_unet* u) {
  if (!u) return api_fail(CLAMP_EINVAL, "clamp_unet_check: NULL network");
  if (!on_unet_device(u, "clamp_unet_check")) return CLAMP_EINVAL;
  int h = 0;
  U_TRY(cudaMemcpy(&h, u->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (!h) return CLAMP_OK;
  U_TRY(cudaMemset(u->err, 0, sizeof(int)));
  return api_fail(CLAMP_ETIMEOUT, "clamp_unet_check: a bounded tensor-core wait gave up");
}

extern "C" clamp_status clamp_unet_normalize(int32_t batch, int64_t n, int64_t norm_count, const float* x,
                                             const float* t, float* x_out, float* t_out, void* stream) {
  if (batch < 1 || n < 1 || norm_count < 1 || !x || !x_out || (t && !t_out))
    return api_fail(CLAMP_EINVAL, "clamp_unet_normalize: bad arguments");
  k_sample_norm<<<batch, NORM_T, 0, (cudaStream_t)stream>>>(x, t, x_out, t_out, (long long)n, (double)norm_count);
  U_TRY(cudaGetLastError());
  return CLAMP_OK;
}

extern "C" clamp_status clamp_unet_warm_start(clamp_unet* u, int32_t nx, int32_t ny, int32_t nz, const float* r0,
                                              float floor_rel, float* r_init, void* ws, size_t ws_bytes,
                                              void* stream) {
  if (!u || !r0 || !r_init) return api_fail(CLAMP_EINVAL, "clamp_unet_warm_start: NULL argument");
  if (!on_unet_device(u, "clamp_unet_warm_start")) return CLAMP_EINVAL;
  if (!unet_shape_ok(1, nx, ny, nz))
    return api_fail(CLAMP_EINVAL, "clamp_unet_warm_start: nx, ny, nz must be multiples of 4");
  const Acts a = acts_layout(u, 1, nx, ny, nz, ws, false);
  if (!ws || ws_bytes < a.bytes) return api_fail(CLAMP_ENOMEM, "clamp_unet_warm_start: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = (long long)nx * ny * nz;
  const unsigned np = grid_for(n);
  k_sum_part<<<np, UT, 0, st>>>(r0, n, a.part);
  const double cols = (double)nx * ny;   // m = sum(r0) / (nx ny): energy per (x, y) column
  k_scale_by_mean<<<grid_for(n), UT, 0, st>>>(r0, n, a.part, (int)np, cols, a.xin);
  U_TRY(cudaGetLastError());
  clamp_status s = unet_forward(u, a.xin, 1, nx, ny, nz, a, st);
  if (s != CLAMP_OK) return s;
  k_warm_map<<<grid_for(n), UT, 0, st>>>(a.out, n, a.part, (int)np, cols, floor_rel, r_init);
  U_TRY(cudaGetLastError());
  return CLAMP_OK;
}

extern "C" clamp_status clamp_unet_loss(clamp_unet* u, const float* x, const float* target, int32_t batch,
                                        int32_t nx, int32_t ny, int32_t nz, double* loss, void* ws, size_t ws_bytes,
                                        void* stream) {
  if (!u || !x || !target || !loss) return api_fail(CLAMP_EINVAL, "clamp_unet_loss: NULL argument");
  if (!on_unet_device(u, "clamp_unet_loss")) return CLAMP_EINVAL;
  if (!unet_shape_ok(batch, nx, ny, nz))
    return api_fail(CLAMP_EINVAL, "clamp_unet_loss: nx, ny, nz must be multiples of 4");
  const Acts a = acts_layout(u, batch, nx, ny, nz, ws, true);   // the loss gradient goes to gout
  if (!ws || ws_bytes < a.bytes) return api_fail(CLAMP_ENOMEM, "clamp_unet_loss: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  clamp_status s = unet_forward(u, x, batch, nx, ny, nz, a, st);
  if (s != CLAMP_OK) return s;
  const long long N = (long long)batch * nx * ny * nz;
  const unsigned nb = grid_for(N);
  k_mse<<<nb, UT, 0, st>>>(a.out, target, a.gout, N, a.part);
  k_mse_final<<<1, 32, 0, st>>>(a.part, (int)nb, N, loss);
  U_TRY(cudaGetLastError());
  return CLAMP_OK;
}
