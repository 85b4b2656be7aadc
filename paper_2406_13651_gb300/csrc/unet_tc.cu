// unet_tc.cu -- the U-Net's 3x3x3 convolutions on the 5th-generation tensor cores (tcgen05),
// BF16 operands and FP32 accumulation: the forward conv and, with flipped weights, the data
// gradient of the backward pass (Sec. III-C's U-Net prior and the learned warm start).
//
// The U-Net keeps FP32 channel-planar tensors [batch][C][nz][ny][nx] (pooling, transposed
// convs, skips and the weight gradient read them), so this kernel converts on the fly: it
// loads FP32 halo voxels, rounds them to BF16 (round to nearest even, as the CUDA-core BF16
// path does) and writes them in the no-swizzle K-major layout, and its epilogue writes FP32
// planar outputs with bias and optional ReLU.
//
// Implicit GEMM per CTA: M = 128 output voxels (TW = min(nx, 32) consecutive x voxels in
// R = 128 / TW rows of one z plane), N = C_out, K = 27 taps x C_in in chunks of 16 input
// channels.  The x taps are three shifted copies of the halo (copy dx holds, at x, the
// voxel x + dx - 1, zero outside the volume), so each tap (dz, dy, dx) is one MMA whose A
// operand starts at copy dx, plane dz, row dy: the 128 rows of the tile are contiguous
// there whatever TW is.  One thread issues the 27 MMAs of a chunk into an FP32 TMEM
// accumulator and commits them to an mbarrier; the wait is bounded and sets an error bit
// instead of hanging.
#include "../../include/clamp.h"
#include "clamp_internal.cuh"
#include "clamp_kernels.cuh"
#include "tc_core.cuh"

#include <cuda_bf16.h>

#include <algorithm>

namespace clamp {
namespace unet_tc {

constexpr int UNT = 256;   // threads per CTA
constexpr uint32_t kWaitLimit = 1u << 22;

// Tile: TW = 32 x voxels in R = 4 rows (16 x 8 at nx = 16).  Narrow tiles keep the three
// shifted halo copies small, 3 (R + 2) TW voxels per plane against 3 (128 + 2) x 3 for a
// 128-voxel row, so two or three CTAs share an SM and one stages while another's MMAs run.
__host__ __device__ constexpr int tile_w(int nx) { return nx < 32 ? nx : 32; }
__host__ __device__ constexpr int tmem_cols(int c) { return c <= 32 ? 32 : c <= 64 ? 64 : 128; }

// Shared memory of one CTA: three shifted halo copies [dx][cg][plane][row][TW] of 16-byte
// channel groups, the chunk's weights [tap][cg][C_out][8 channels] and the mbarrier.
__host__ __device__ inline size_t copy_bytes(int tw) { return (size_t)2 * 3 * (128 / tw + 2) * tw * 16; }
__host__ __device__ inline size_t smem_bytes(int tw, int cout) {
  return 1024 + 3 * copy_bytes(tw) + (size_t)27 * 2 * cout * 16 + 64;
}

__device__ __forceinline__ uint32_t bf16x2(float a, float b) {
  return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(a)) |
         ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(b)) << 16);
}

__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(tc::smem_addr(smem_dst)), "l"(gsrc) : "memory");
}

// wpk[((c * 27 + tap) * 2 + cg) * C_out + co] = BF16 W[co][16 c + 8 cg + k][tap], k = 0..7.
__global__ void k_pack_weights(const float* __restrict__ W, int ci_n, int co_n, uint4* __restrict__ wpk) {
  const int total = (ci_n / 16) * 27 * 2 * co_n;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int co = e % co_n, cg = (e / co_n) % 2, tap = (e / (2 * co_n)) % 27, c = e / (54 * co_n);
    const int ci0 = 16 * c + 8 * cg;
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = W[((long long)co * ci_n + ci0 + k) * 27 + tap];
    wpk[e] = make_uint4(bf16x2(v[0], v[1]), bf16x2(v[2], v[3]), bf16x2(v[4], v[5]), bf16x2(v[6], v[7]));
  }
}

template <int COUT>
__global__ void __launch_bounds__(UNT, 2)
    k_conv3_unet_tc(const float* __restrict__ in, long long in_bs, int ci_n, float* __restrict__ out,
                    long long out_bs, const uint4* __restrict__ wpk, const float* __restrict__ bias, int relu,
                    int nx, int ny, int nz, int* err) {
  static_assert(COUT % 16 == 0 && COUT <= 64, "output channels");
  constexpr uint32_t TCOLS = tmem_cols(COUT);
  const int tw = tile_w(nx), R = 128 / tw, HR = R + 2;
  extern __shared__ unsigned char ut_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)ut_smem_raw + 1023) & ~(uintptr_t)1023);
  const size_t cpy = copy_bytes(tw);
  uint4* s_a = reinterpret_cast<uint4*>(base);                          // [3 dx][2 cg][3 planes][HR][tw]
  uint4* s_w = reinterpret_cast<uint4*>(base + 3 * cpy);                // [27][2][COUT]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(s_w + 27 * 2 * COUT);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * tw, y0 = blockIdx.y * R;
  const int b = blockIdx.z / nz, z = blockIdx.z % nz;
  const long long plane = (long long)nx * ny, n = plane * nz;
  const float* inb = in + (long long)b * in_bs;

  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    *abort_flag = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, TCOLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t a_s = tc::smem_addr(s_a), w_s = tc::smem_addr(s_w);
  const uint32_t plane_b = (uint32_t)(HR * tw * 16), cg_b = 3 * plane_b, dx_b = 2 * cg_b;
  const int nchunks = ci_n / 16;
  const int src_w = tw + 2, nsrc = 3 * HR * src_w;
  bool aborted = false;
  uint32_t fail_parity = 0;

  for (int c = 0; c < nchunks; ++c) {
    // weights of the chunk (already BF16, 16-byte groups)
    const uint4* wsrc = wpk + (long long)c * 27 * 2 * COUT;
    for (int e = tid; e < 27 * 2 * COUT; e += UNT) cp_async16(&s_w[e], &wsrc[e]);
    // halo: source voxel (plane p, row h, xs) with 16 channels -> copies dx at x = xs - dx
    for (int e = tid; e < nsrc; e += UNT) {
      const int xs = e % src_w, h = (e / src_w) % HR, p = e / (src_w * HR);
      const int gx = x0 + xs - 1, gy = y0 + h - 1, gz = z + p - 1;
      const bool inb_ = gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz;
      // (outside the volume the pointer stays at a valid element and nothing is used)
      const float* src = inb + (long long)(16 * c) * n +
                         (inb_ ? (long long)gz * plane + (long long)gy * nx + gx : 0LL);
      float v[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) v[k] = inb_ ? __ldg(src + (long long)k * n) : 0.f;
      const uint4 g0 = make_uint4(bf16x2(v[0], v[1]), bf16x2(v[2], v[3]), bf16x2(v[4], v[5]), bf16x2(v[6], v[7]));
      const uint4 g1 =
          make_uint4(bf16x2(v[8], v[9]), bf16x2(v[10], v[11]), bf16x2(v[12], v[13]), bf16x2(v[14], v[15]));
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int x = xs - dx;
        if (x < 0 || x >= tw) continue;
        uint4* d = s_a + (size_t)dx * (dx_b / 16) + ((size_t)p * HR + h) * tw + x;
        d[0] = g0;
        d[cg_b / 16] = g1;
      }
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint32_t idesc = tc::idesc_bf16_f32(128, COUT);
#pragma unroll 1
      for (int tap = 0; tap < 27; ++tap) {
        const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
        const uint64_t ad = tc::make_desc(a_s + dx * dx_b + dz * plane_b + dy * tw * 16, cg_b, 128);
        const uint64_t bd = tc::make_desc(w_s + tap * 2 * COUT * 16, COUT * 16, 128);
        tc::mma_bf16(tbase, ad, bd, idesc, (c > 0 || tap > 0) ? 1u : 0u);
      }
      tc::mma_commit(mbar);
    }
    // the chunk's MMAs read the buffers the next chunk overwrites: one thread waits
    if (tid == 0 && !tc::mbar_wait_bounded(mbar, (uint32_t)(c & 1), kWaitLimit)) *abort_flag = 1;
    __syncthreads();
    if (*abort_flag) {
      aborted = true;
      fail_parity = (uint32_t)(c & 1);
      break;
    }
  }
  tc::fence_after_sync();
  if (!aborted) {
    // warp w reads TMEM lanes 32 (w % 4) .. + 31 (voxels) and half the output channels
    const int q = warp & 3, hh = warp >> 2;
    const int i = 32 * q + lane;
    const long long vox = (long long)z * plane + (long long)(y0 + i / tw) * nx + x0 + i % tw;
    float* outb = out + (long long)b * out_bs + vox;
    const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16);
    constexpr int HALF = COUT / 2;
#pragma unroll
    for (int j = 0; j < HALF / 8; ++j) {
      const int col = hh * HALF + 8 * j;
      float v[8];
      tc::tmem_ld_x8(trow + (uint32_t)col, v);
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        float r = v[k] + (bias ? __ldg(&bias[col + k]) : 0.f);
        if (relu) r = fmaxf(r, 0.f);
        outb[(long long)(col + k) * n] = r;
      }
    }
  } else if (tid == 0) {
    if (err) atomicOr(err, 2);
    tc::mbar_wait_bounded(mbar, fail_parity, kWaitLimit);   // bounded wait for MMAs in flight before TMEM is freed
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, TCOLS);
}

}  // namespace unet_tc

using namespace unet_tc;

bool unet_conv3_tc_supported(int ci, int co, int nx, int ny) {
  if (ci < 16 || ci % 16 != 0 || (co != 16 && co != 32 && co != 64)) return false;
  const int tw = tile_w(nx);
  return (nx == 16 || nx % 32 == 0) && ny % (128 / tw) == 0;
}

size_t unet_conv3_tc_wpk_bytes(int ci, int co) { return (size_t)(ci / 16) * 27 * 2 * co * 16; }

template <int COUT>
static cudaError_t launch_cout(const float* in, long long in_bs, int ci, float* out, long long out_bs,
                               const uint4* wpk, const float* bias, bool relu, int B, int nx, int ny, int nz, int* err,
                               cudaStream_t st) {
  const int tw = tile_w(nx);
  const size_t smem = smem_bytes(tw, COUT);
  cudaError_t e = cudaFuncSetAttribute(k_conv3_unet_tc<COUT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  // grid.z = samples x planes stays <= 65535: launch sample chunks
  const int per = std::max(1, 65535 / nz);
  for (int b0 = 0; b0 < B; b0 += per) {
    const int bc = std::min(per, B - b0);
    const dim3 grid(nx / tw, ny / (128 / tw), bc * nz);
    k_conv3_unet_tc<COUT><<<grid, UNT, smem, st>>>(in + (long long)b0 * in_bs, in_bs, ci, out + (long long)b0 * out_bs,
                                                  out_bs, wpk, bias, relu ? 1 : 0, nx, ny, nz, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t unet_conv3_tc(const float* in, long long in_bs, int ci, float* out, long long out_bs, int co,
                          const float* W, const float* bias, bool relu, int B, int nx, int ny, int nz, uint4* wpk,
                          int* err, cudaStream_t st) {
  if (!unet_conv3_tc_supported(ci, co, nx, ny)) return cudaErrorInvalidValue;
  const int total = (ci / 16) * 27 * 2 * co;
  k_pack_weights<<<(total + 255) / 256, 256, 0, st>>>(W, ci, co, wpk);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch (co) {
    case 16: return launch_cout<16>(in, in_bs, ci, out, out_bs, wpk, bias, relu, B, nx, ny, nz, err, st);
    case 32: return launch_cout<32>(in, in_bs, ci, out, out_bs, wpk, bias, relu, B, nx, ny, nz, err, st);
    default: return launch_cout<64>(in, in_bs, ci, out, out_bs, wpk, bias, relu, B, nx, ny, nz, err, st);
  }
}

}  // namespace clamp
