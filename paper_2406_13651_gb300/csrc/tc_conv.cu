// tc_conv.cu -- 3x3x3 convolutions of the CNN prior on the 5th-generation tensor cores (tcgen05).
//
// Implicit GEMM: for one output tile of 128 consecutive x voxels (M = 128) and all
// output channels (N), K runs over 27 taps x input channels.  A CTA computes TY x TZ
// such tiles.  For each chunk of input channels it stages the zero-padded input halo
// (130 x (TY+2) x (TZ+2) voxels, channels-last in 16-byte channel groups) and the
// chunk's weights in shared memory in the no-swizzle K-major core-matrix layout; a tap
// is then only an offset of the A descriptor's start address.
//
// Tiles of one z-row that read the same shifted halo window (tile ty with tap dy reads
// halo row ty + dy) share one MMA: the weights are packed per (dz, dx) as three
// consecutive dy blocks in the order dy = 2, 1, 0, so the taps of tiles ty_lo..ty_hi for
// halo row hy (dy = hy - ty) form one contiguous N range, and those tiles' accumulators
// are adjacent TMEM columns.  One MMA with N = (tiles) x C_out replaces one per tile,
// which halves the A-operand reads for the inner rows.  At the first chunk every
// accumulator is cleared by one MMA against a zero weight block, so every later MMA
// accumulates.  One thread issues the chunk's MMAs into FP32 accumulators in TMEM and
// commits them to an mbarrier (a warp-wide elected issue measured slower here); the
// epilogue reads TMEM (tcgen05.ld), adds the bias, applies ReLU and writes the next
// layer's activations, or (last layer) FP32 plus the residual input.
//
// Two operand kinds:
//  * BF16: kind::f16 with BF16 operands, 16 channels per chunk (the BF16 prior).
//  * TF32x3: kind::tf32 with every FP32 operand split as hi + lo, both rounded to nearest
//    TF32 (hi = RN(x), lo = RN(x - hi)); hi*hi + hi*lo + lo*hi keeps each product to
//    about 2^-21 relative with zero-mean residuals, so the FP32 prior keeps FP32 accuracy.
//    (Truncating hi instead biases lo to the sign of x, and the dropped lo*lo terms then
//    add up across the 27 x Cin products of an output.)
//
// Activation layouts: BF16 [C/8][nz][ny][nx][8], FP32 [C/4][nz][ny][nx][4]: 16 bytes per
// voxel per channel group.
#include "../../include/clamp.h"
#include "clamp_kernels.cuh"
#include "denoise.cuh"
#include "tc_core.cuh"

#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

namespace clamp {

constexpr int TCX = 128, TC_HX = TCX + 2, TC_NT = 256;
constexpr uint32_t kWaitLimit = 1u << 22;

__host__ __device__ constexpr int pow2_cols(int c) {
  return c <= 32 ? 32 : c <= 64 ? 64 : c <= 128 ? 128 : c <= 256 ? 256 : 512;
}

enum TcKindId { TC_BF16 = 0, TC_TF32X3 = 1 };

template <int KIND>
struct TcKind;
template <>
struct TcKind<TC_BF16> {
  static constexpr int EPV = 8;      // channels per 16-byte group
  static constexpr int SPLIT = 1;    // operand copies (hi only)
  // 2 x 2 rows per CTA: about 107 KB of shared memory and at most 256 TMEM columns at
  // 48 channels, so two CTAs share an SM and one stages its next chunk while the
  // other's MMAs run.
  static constexpr int TY = 2, TZ = 2;
  static constexpr int MIN_CTAS = 2;
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
  }
};
template <>
struct TcKind<TC_TF32X3> {
  static constexpr int EPV = 4;
  static constexpr int SPLIT = 2;    // hi and lo copies
  static constexpr int TY = 2, TZ = 2;
  static constexpr int MIN_CTAS = 1;
  __host__ __device__ static constexpr uint32_t idesc(int M, int N) {
    return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
  }
};

__device__ __forceinline__ void mma_kind(int kind, uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  if (kind == TC_BF16) {
    tc::mma_bf16(d, a, b, idesc, acc);
  } else {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
  }
}

// TF32x3 at <= 32 channels runs k_conv3_tc_plane (tiles of 4 rows x 1 plane).
__host__ __device__ constexpr bool tc_tall(int kind, int cin) { return kind == TC_TF32X3 && cin <= 32; }

template <int KIND, int CIN, int NPAD>
struct TcCfg {
  using K = TcKind<KIND>;
  static constexpr int TY = K::TY, TZ = K::TZ, MT = TY * TZ, HY = TY + 2, HZ = TZ + 2;
  static constexpr int CH = 2 * K::EPV;               // input channels per chunk (one MMA K step)
  static constexpr int CHUNKS = CIN / CH;
  static constexpr int HALO_VEC = 2 * HZ * HY * TC_HX;  // 16-byte vectors per chunk, per split
  static constexpr int W_VEC = 27 * 2 * NPAD;          // [dz][dx][2][dy = 2, 1, 0][NPAD]
  static constexpr int ZB_VEC = 2 * NPAD;              // zero weight block (accumulator clear)
  // BF16 2 x 2 tiles with 5 C_out <= 256: a halo row in the middle of both z-rows feeds the
  // four tiles with one MMA (N = 5 C_out: the tiles' accumulators at TMEM columns
  // (3 tz + ty) C_out, a spare block between the z-rows takes the fifth product), the
  // weights held as [dx][cg][dz = 2, 1, 0][dy = 2, 1, 0] so the four taps (and the spare's)
  // are consecutive blocks.
  static constexpr bool MERGE = KIND == TC_BF16 && TY == 2 && TZ == 2 && 5 * NPAD <= 256;
  static constexpr int CS = MERGE ? 3 : TY;             // accumulator blocks per z-row
  static constexpr int TMEM_COLS = pow2_cols(MERGE ? 5 * NPAD : MT * NPAD);
  static constexpr size_t SMEM = 1024 + 16 * ((size_t)K::SPLIT * (HALO_VEC + W_VEC) + ZB_VEC) + 64;
  static_assert(CIN % CH == 0 && NPAD % 16 == 0 && MT * NPAD <= 512 && TY * NPAD <= 256, "tile");
  static_assert(SMEM <= 227 * 1024, "shared memory");
};

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  const __nv_bfloat16 lo = __float2bfloat16_rn(a), hi = __float2bfloat16_rn(b);
  return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}
// Round to the nearest TF32 value (10 explicit mantissa bits), ties to even.
__device__ __forceinline__ float tf32_rn(float x) {
  uint32_t u = __float_as_uint(x);
  u += 0xFFFu + ((u >> 13) & 1u);
  return __uint_as_float(u & 0xFFFFE000u);
}

// 16-byte asynchronous global -> shared copy; with valid == false nothing is read and the
// destination is zero-filled.
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(tc::smem_addr(smem_dst)), "l"(gsrc),
               "r"(valid ? 16 : 0)
               : "memory");
}
// 4-byte variant (cp.async.ca): for rows whose start is not 16-byte aligned.
__device__ __forceinline__ void cp_async4(void* smem_dst, const void* gsrc, bool valid) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(tc::smem_addr(smem_dst)), "l"(gsrc),
               "r"(valid ? 4 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

// Persistent: a CTA walks the tiles blockIdx.x, blockIdx.x + gridDim.x, ... (tile t = x
// tile fastest, then y pairs, then z pairs).  TMEM, the mbarrier and the zero block are set
// up once; the first chunk of the next tile is staged while the current tile's epilogue
// drains TMEM.
//
// TAPS (BF16, the network's last hidden layer): the layer's activations (bias, ReLU,
// BF16) go to shared memory instead of HBM and feed at once the last layer's per-voxel tap
// sums, P_tap[v] = sum_c W_last[tap][c] h[v][c], as a second GEMM (M = 128 voxels, K = C,
// N = 27 taps padded to 32) into the tile's TMEM columns; the kernel writes P (FP32
// [27][n]) and the last layer is left with its gather.  This saves writing and reading
// the 2 C bytes per voxel of the last hidden activations.
template <int KIND, int CIN, int NPAD, bool LAST, bool TAPS = false>
__global__ void __launch_bounds__(TC_NT, TcKind<KIND>::MIN_CTAS)
    k_conv3_tc(const uint4* __restrict__ in, const uint4* __restrict__ wpk, const float* __restrict__ bias,
               uint4* __restrict__ out_act, float* __restrict__ out_f32, const float* __restrict__ resid, int nx,
               int ny, int nz, int* err, const uint4* __restrict__ wtaps = nullptr, float* __restrict__ P = nullptr) {
  static_assert(!TAPS || (KIND == TC_BF16 && !LAST && NPAD >= 32 && NPAD % 16 == 0), "tap-sum fusion");
  using Cfg = TcCfg<KIND, CIN, NPAD>;
  using Kd = TcKind<KIND>;
  constexpr int TY = Cfg::TY, HY = Cfg::HY, HZ = Cfg::HZ, MT = Cfg::MT;
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint4* s_halo = reinterpret_cast<uint4*>(base);              // [SPLIT][2][HZ][HY][HX]
  uint4* s_w = s_halo + Kd::SPLIT * Cfg::HALO_VEC;             // [SPLIT][3 dz][3 dx][2][3 dy][NPAD]
  uint4* s_zero = s_w + Kd::SPLIT * Cfg::W_VEC;                 // [2][NPAD] zeros
  uint64_t* mbar = reinterpret_cast<uint64_t*>(s_zero + Cfg::ZB_VEC);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long plane = (long long)nx * ny, n = plane * nz;
  const int tiles_x = nx / TCX, tiles_y = ny / TY, ntiles = tiles_x * tiles_y * (nz / Cfg::TZ);
  // extents of the global buffers (16-byte vectors) that the bounds-checking build tests
  [[maybe_unused]] const long long in_ext = (long long)(CIN / Kd::EPV) * n,
                                   out_ext = (long long)(NPAD / Kd::EPV) * n,
                                   w_ext = (long long)Kd::SPLIT * Cfg::CHUNKS * Cfg::W_VEC;

  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    *abort_flag = 0;
  }
  for (int e = tid; e < Cfg::ZB_VEC; e += TC_NT) s_zero[e] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tc::tmem_alloc(tslot, Cfg::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t halo_s = tc::smem_addr(s_halo), w_s = tc::smem_addr(s_w), z_s = tc::smem_addr(s_zero);
  constexpr uint32_t LBO_A = HZ * HY * TC_HX * 16;  // channel group 0 -> 1
  // channel group 0 -> 1: within a (dz, dx) block, or (merged layout) within a dx block
  constexpr uint32_t LBO_B = (Cfg::MERGE ? 9 : 3) * NPAD * 16;
  constexpr uint32_t SPLIT_A = 16u * Cfg::HALO_VEC, SPLIT_B = 16u * Cfg::W_VEC;  // hi -> lo copies
  // TMEM column of tile mt's accumulator (tile = ty + TY tz)
  auto acc_col = [](int mt) { return (uint32_t)(((mt / TY) * Cfg::CS + mt % TY) * NPAD); };
  bool aborted = false;
  uint32_t phase = 0;   // MMA commits completed so far (the mbarrier's phase parity)

  // Chunk staging: cp.async 16-byte copies (zero-fill outside the volume), all in flight
  // at once, in one commit group per halo plane: group p holds halo plane p and the
  // weights of dz = p, the first taps that reach it.  Each warp takes whole halo rows
  // (channel group, y: row-uniform bounds and base address) with its lanes along x, so a
  // copy costs a few instructions to issue.  BF16 waits for the groups one plane at a time
  // and issues the MMAs that read a plane as soon as it has landed, while the later planes
  // are still in flight; TF32x3 lands the raw FP32 halo in the lo copy, waits for all of it
  // and splits it in place.
  uint4* s_raw = s_halo + (Kd::SPLIT - 1) * Cfg::HALO_VEC;
  constexpr int WDZ = Cfg::W_VEC / 3;   // weights of one dz
  const uint64_t a0 = tc::make_desc(halo_s, LBO_A, 128);
  const uint64_t b0 = tc::make_desc(w_s, LBO_B, 128);
  auto stage = [&](int c, int x0, int y0, int z0) {
#pragma unroll
    for (int hz = 0; hz < HZ; ++hz) {
      if (hz < 3) {
        for (int sp = 0; sp < Kd::SPLIT; ++sp) {
          const uint4* wsrc = wpk + ((long long)sp * Cfg::CHUNKS + c) * Cfg::W_VEC + hz * WDZ;
          if constexpr (Cfg::MERGE) {   // packed [dx][cg][dy blk][n] of this dz -> [dx][cg][dz blk][dy blk][n]
            for (int e = tid; e < WDZ; e += TC_NT) {
              const int nn = e % NPAD, t = e / NPAD, dyb = t % 3, dxc = t / 3;   // dxc = 2 dx + cg
              cp_async16(&s_w[(dxc * 9 + (2 - hz) * 3 + dyb) * NPAD + nn], &wsrc[e],
                         CLAMP_IN_BOUNDS(wsrc + e - wpk, w_ext, 301) &&
                             CLAMP_IN_BOUNDS((dxc * 9 + (2 - hz) * 3 + dyb) * NPAD + nn, Cfg::W_VEC, 302));
            }
          } else {
            uint4* wdst = s_w + sp * Cfg::W_VEC + hz * WDZ;
            for (int e = tid; e < WDZ; e += TC_NT)
              cp_async16(&wdst[e], &wsrc[e], CLAMP_IN_BOUNDS(wsrc + e - wpk, w_ext, 301));
          }
        }
      }
      const int gz = z0 + hz - 1;
      for (int r = warp; r < 2 * HY; r += TC_NT / 32) {
        const int cg = r / HY, yr = r % HY;
        const int gy = y0 + yr - 1;
        const bool rin = gy >= 0 && gy < ny && gz >= 0 && gz < nz;
        const long long rbase = (long long)(2 * c + cg) * n + (long long)gz * plane + (long long)gy * nx;
        uint4* drow = s_raw + ((cg * HZ + hz) * HY + yr) * TC_HX;
        for (int xr = lane; xr < TC_HX; xr += 32) {
          const int gx = x0 + xr - 1;
          const bool inb = rin && gx >= 0 && gx < nx;
          cp_async16(&drow[xr], inb ? &in[rbase + gx] : in, inb && CLAMP_IN_BOUNDS(rbase + gx, in_ext, 303));
        }
      }
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
  };
  // MMAs of one chunk that read halo plane hz: tiles tz with tap dz = hz - tz.  Descriptors
  // differ only in the start-address field (bits 0-13, 16-byte units), so each MMA adds a
  // compile-time offset to a base descriptor.
  auto issue_plane = [&](int hz) {
    if constexpr (Cfg::MERGE) {
      if (hz == 1 || hz == 2) {   // middle rows of a middle plane: all four tiles, one MMA per dx
#pragma unroll
        for (int hy = 1; hy <= 2; ++hy) {
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const uint64_t aoff = (uint64_t)((hz * HY + hy) * TC_HX + dx);
            // blocks (dz, dy) = (hz, hy), (hz, hy - 1), spare, (hz - 1, hy), (hz - 1, hy - 1)
            const uint64_t boff = (uint64_t)((dx * 18 + (2 - hz) * 3 + (2 - hy)) * NPAD);
            mma_kind(KIND, tbase, a0 + aoff, b0 + boff, Kd::idesc(128, 5 * NPAD), 1u);
          }
        }
      }
    }
#pragma unroll
    for (int tz = 0; tz < Cfg::TZ; ++tz) {
      const int dz = hz - tz;
      if (dz < 0 || dz > 2) continue;
#pragma unroll
      for (int hy = 0; hy < HY; ++hy) {
        if (Cfg::MERGE && (hz == 1 || hz == 2) && (hy == 1 || hy == 2)) continue;   // merged above
        // tiles ty_lo..ty_hi of z-row tz read halo row hy with taps dy = hy - ty
        const int ty_lo = hy - 2 > 0 ? hy - 2 : 0, ty_hi = hy < TY - 1 ? hy : TY - 1;
        const int ntile = ty_hi - ty_lo + 1;
        const uint32_t idesc = Kd::idesc(128, ntile * NPAD);
        const uint32_t dcol = tbase + acc_col(tz * TY + ty_lo);
        const int dyp = 2 - (hy - ty_lo);   // block index of the first tile's tap (dy = hy - ty_lo)
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const uint64_t aoff = (uint64_t)((hz * HY + hy) * TC_HX + dx);
          const uint64_t boff = Cfg::MERGE ? (uint64_t)((dx * 18 + (2 - dz) * 3 + dyp) * NPAD)
                                           : (uint64_t)((dz * 3 + dx) * 6 * NPAD + dyp * NPAD);
#pragma unroll
          for (int sp = 0; sp < (KIND == TC_BF16 ? 1 : 3); ++sp) {
            // TF32x3 terms: (a_lo, b_hi), (a_hi, b_lo), (a_hi, b_hi)
            const uint64_t a_sp = (KIND == TC_BF16 || sp > 0) ? 0 : (uint64_t)(SPLIT_A >> 4);
            const uint64_t b_sp = (KIND != TC_BF16 && sp == 1) ? (uint64_t)(SPLIT_B >> 4) : 0;
            mma_kind(KIND, dcol, a0 + a_sp + aoff, b0 + b_sp + boff, idesc, 1u);
          }
        }
      }
    }
  };
  auto clear_acc = [&]() {   // D = A x 0 for every accumulator (first chunk of a tile)
    const uint64_t bz = tc::make_desc(z_s, NPAD * 16, 128);
#pragma unroll
    for (int mt = 0; mt < MT; ++mt) mma_kind(KIND, tbase + acc_col(mt), a0, bz, Kd::idesc(128, NPAD), 0u);
  };
  static_assert(HZ == 4, "one commit group per halo plane: the waits below name groups 3..0");

  int tile = blockIdx.x;
  auto origin = [&](int t, int& x0, int& y0, int& z0) {
    x0 = (t % tiles_x) * TCX;
    t /= tiles_x;
    y0 = (t % tiles_y) * TY;
    z0 = (t / tiles_y) * Cfg::TZ;
  };
  if (tile < ntiles) {
    int x0, y0, z0;
    origin(tile, x0, y0, z0);
    stage(0, x0, y0, z0);
  }
  while (tile < ntiles && !aborted) {
    int x0, y0, z0;
    origin(tile, x0, y0, z0);
    for (int c = 0; c < Cfg::CHUNKS; ++c) {
      if (c > 0) stage(c, x0, y0, z0);   // the buffers are free: the previous chunk's MMAs completed
      if constexpr (KIND == TC_BF16) {
#pragma unroll
        for (int hz = 0; hz < HZ; ++hz) {
          if (hz == 0) asm volatile("cp.async.wait_group 3;" ::: "memory");
          else if (hz == 1) asm volatile("cp.async.wait_group 2;" ::: "memory");
          else if (hz == 2) asm volatile("cp.async.wait_group 1;" ::: "memory");
          else asm volatile("cp.async.wait_group 0;" ::: "memory");
          tc::fence_proxy_async();
          __syncthreads();
          if (tid == 0) {
            tc::fence_after_sync();
            if (c == 0 && hz == 0) clear_acc();
            issue_plane(hz);
            if (hz == HZ - 1) tc::mma_commit(mbar);
          }
        }
      } else {
        asm volatile("cp.async.wait_group 0;" ::: "memory");
        __syncthreads();
        float4* hi = reinterpret_cast<float4*>(s_halo);
        float4* lo = reinterpret_cast<float4*>(s_raw);
        for (int e = tid; e < Cfg::HALO_VEC; e += TC_NT) {
          const float4 f = lo[e];
          const float4 h = make_float4(tf32_rn(f.x), tf32_rn(f.y), tf32_rn(f.z), tf32_rn(f.w));
          hi[e] = h;
          lo[e] = make_float4(tf32_rn(f.x - h.x), tf32_rn(f.y - h.y), tf32_rn(f.z - h.z), tf32_rn(f.w - h.w));
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
          tc::fence_after_sync();
          if (c == 0) clear_acc();
#pragma unroll
          for (int hz = 0; hz < HZ; ++hz) issue_plane(hz);
          tc::mma_commit(mbar);
        }
      }
      // the chunk's MMAs read the buffers the next chunk overwrites: one thread waits for
      // their commit, the others at the barrier (which takes no issue slots from the CTA
      // staging beside this one)
      if (tid == 0 && !tc::mbar_wait_bounded(mbar, phase & 1u, kWaitLimit)) *abort_flag = 1;
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      ++phase;
    }
    if (aborted) break;
    const int next = tile + (int)gridDim.x;
    if constexpr (TAPS) {
      constexpr int G = NPAD / 8;   // channel groups of the activations (K of the tap GEMM)
      // tap weights [G][32 taps][8 channels] into the weight buffer (free: the MMAs are done)
      for (int e = tid; e < G * 32; e += TC_NT) cp_async16(&s_w[e], &wtaps[e], true);
      asm volatile("cp.async.commit_group;" ::: "memory");
      tc::fence_after_sync();
      // the hidden layer's activations, as the tap GEMM's A: [MT][G][128 voxels] x 16 B in
      // the halo buffer (free as well)
      const int q = warp & 3, h = warp >> 2;
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + acc_col(mt);
        constexpr int HALF = NPAD / 2;
#pragma unroll
        for (int j = 0; j < HALF / 8; ++j) {
          const int col = h * HALF + 8 * j;
          float v[8];
          tc::tmem_ld_x8(trow + (uint32_t)col, v);
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = fmaxf(v[i] + __ldg(&bias[col + i]), 0.f);
          s_halo[(mt * G + col / 8) * 128 + 32 * q + lane] =
              make_uint4(pack_bf16x2(v[0], v[1]), pack_bf16x2(v[2], v[3]), pack_bf16x2(v[4], v[5]),
                         pack_bf16x2(v[6], v[7]));
        }
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      tc::fence_proxy_async();
      tc::fence_before_sync();
      __syncthreads();
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
#pragma unroll
          for (int ks = 0; ks < G / 2; ++ks)
            tc::mma_bf16(tbase + acc_col(mt),
                         tc::make_desc(halo_s + (uint32_t)((mt * G + 2 * ks) * 128 * 16), 128 * 16, 128),
                         tc::make_desc(w_s + (uint32_t)(2 * ks * 32 * 16), 32 * 16, 128), Kd::idesc(128, 32),
                         ks ? 1u : 0u);
        tc::mma_commit(mbar);
      }
      if (tid == 0 && !tc::mbar_wait_bounded(mbar, phase & 1u, kWaitLimit)) *abort_flag = 1;
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      ++phase;
      // the tap GEMM has read both shared buffers: the next tile's first chunk lands while
      // the tap sums drain
      if (next < ntiles) {
        int nx0, ny0, nz0;
        origin(next, nx0, ny0, nz0);
        stage(0, nx0, ny0, nz0);
      }
      tc::fence_after_sync();
#pragma unroll 1
      for (int mt = 0; mt < MT; ++mt) {
        const int gy = y0 + mt % TY, gz = z0 + mt / TY, gx = x0 + 32 * q + lane;
        const long long vox = (long long)gz * plane + (long long)gy * nx + gx;
        const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + acc_col(mt);
#pragma unroll
        for (int j = 0; j < 2; ++j) {
          const int col = h * 16 + 8 * j;
          float t[8];
          tc::tmem_ld_x8(trow + (uint32_t)col, t);
#pragma unroll
          for (int i = 0; i < 8; ++i)
            if (col + i < 27 && CLAMP_IN_BOUNDS((long long)(col + i) * n + vox, 27 * n, 304))
              P[(long long)(col + i) * n + vox] = t[i];
        }
      }
      // TMEM reads complete before the next tile's first MMA overwrites them
      tc::fence_before_sync();
      __syncthreads();
      tile = next;
      continue;
    }
    if (next < ntiles) {   // the next tile's first chunk lands while this tile's epilogue runs
      int nx0, ny0, nz0;
      origin(next, nx0, ny0, nz0);
      stage(0, nx0, ny0, nz0);
    }
    tc::fence_after_sync();
    const int q = warp & 3, h = warp >> 2;
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      const int gy = y0 + mt % TY, gz = z0 + mt / TY, gx = x0 + 32 * q + lane;
      const long long vox = (long long)gz * plane + (long long)gy * nx + gx;
      const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + acc_col(mt);
      if constexpr (LAST) {   // one output channel (column 0): FP32 plus the residual input
        if (h == 0 && CLAMP_IN_BOUNDS(vox, n, 305)) {
          float v[8];
          tc::tmem_ld_x8(trow, v);
          out_f32[vox] = v[0] + __ldg(&bias[0]) + resid[vox];
        }
        continue;
      }
      constexpr int HALF = NPAD / 2;
#pragma unroll
      for (int j = 0; j < HALF / 8; ++j) {
        const int col = h * HALF + 8 * j;
        float v[8];
        tc::tmem_ld_x8(trow + (uint32_t)col, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fmaxf(v[i] + __ldg(&bias[col + i]), 0.f);
        if constexpr (KIND == TC_BF16) {
          uint4 o;
          o.x = pack_bf16x2(v[0], v[1]);
          o.y = pack_bf16x2(v[2], v[3]);
          o.z = pack_bf16x2(v[4], v[5]);
          o.w = pack_bf16x2(v[6], v[7]);
          if (CLAMP_IN_BOUNDS((long long)(col / 8) * n + vox, out_ext, 306)) out_act[(long long)(col / 8) * n + vox] = o;
        } else {
          float4* o4 = reinterpret_cast<float4*>(out_act);
          if (CLAMP_IN_BOUNDS((long long)(col / 4 + 1) * n + vox, out_ext, 306) &&
              CLAMP_IN_BOUNDS((long long)(col / 4) * n + vox, out_ext, 306)) {
            o4[(long long)(col / 4) * n + vox] = make_float4(v[0], v[1], v[2], v[3]);
            o4[(long long)(col / 4 + 1) * n + vox] = make_float4(v[4], v[5], v[6], v[7]);
          }
        }
      }
    }
    // every TMEM read of this tile completes before the next tile's first MMA overwrites it
    tc::fence_before_sync();
    __syncthreads();
    tile = next;
  }
  if (aborted && tid == 0) {
    if (err) atomicOr(err, 2);
    // the chunk's MMAs may still be in flight: give them a bounded wait before TMEM is freed
    tc::mbar_wait_bounded(mbar, phase & 1u, kWaitLimit);
  }
  asm volatile("cp.async.wait_all;" ::: "memory");   // no copy may land after the CTA exits
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, Cfg::TMEM_COLS);
}

// TF32x3 at <= 32 channels: per-plane staging, three CTAs per SM.  A CTA computes 4 rows
// x 1 plane of 128-voxel tiles (one MMA spans up to three tiles of the row, N <= 96).  The
// staging unit is one (channel chunk, halo plane) step: the FP32 halo plane (2 channel
// groups x 6 rows x 130 voxels), loaded into registers and written once as TF32 hi and lo
// copies (split as in k_conv3_tc), and the hi/lo weights of the matching dz (cp.async),
// about 68 KB at 32 channels.  A step's MMAs are those of one dz, in k_conv3_tc's order.
// Each CTA stages, issues and waits step by step as k_conv3_tc does per chunk; with about
// 70 KB of shared memory and 128 TMEM columns per CTA three CTAs share an SM, so one CTA's
// staging overlaps the other CTAs' MMAs (k_conv3_tc's whole-chunk halo, hi and lo, leaves
// one CTA per SM).
template <int CIN, int NPAD>
struct TcPlaneCfg {
  static constexpr int TY = 4, HY = TY + 2, MT = TY, CTAS = 3;
  static constexpr int CHUNKS = CIN / 8, STEPS = 3 * CHUNKS;
  static constexpr int HALO_VEC = 2 * HY * TC_HX;   // per copy: [2 channel groups][HY][HX]
  static constexpr int W_VEC = 3 * 2 * 3 * NPAD;    // per copy: [dx][2 channel groups][dy = 2, 1, 0][NPAD]
  static constexpr int STAGE_VEC = 2 * (HALO_VEC + W_VEC);  // [halo hi][halo lo][w hi][w lo]
  static constexpr int ZB_VEC = 2 * NPAD;
  static constexpr int TMEM_COLS = pow2_cols(MT * NPAD);
  static constexpr size_t SMEM = 1024 + 16 * ((size_t)STAGE_VEC + ZB_VEC) + 64;
  static_assert(CIN % 8 == 0 && NPAD % 16 == 0 && TY * NPAD <= 256, "tile");
  static_assert(CTAS * (SMEM + 1024) <= 228 * 1024 && CTAS * TMEM_COLS <= 512, "three CTAs per SM");
};

template <int CIN, int NPAD>
__global__ void __launch_bounds__(TC_NT, TcPlaneCfg<CIN, NPAD>::CTAS)
    k_conv3_tc_plane(const uint4* __restrict__ in, const uint4* __restrict__ wpk, const float* __restrict__ bias,
                     uint4* __restrict__ out_act, int nx, int ny, int nz, int* err) {
  using Cfg = TcPlaneCfg<CIN, NPAD>;
  using Kd = TcKind<TC_TF32X3>;
  constexpr int TY = Cfg::TY, HY = Cfg::HY, MT = Cfg::MT;
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint4* s_stage = reinterpret_cast<uint4*>(base);              // [halo hi][halo lo][w hi][w lo]
  uint4* s_zero = s_stage + Cfg::STAGE_VEC;                      // [2][NPAD] zeros
  uint64_t* mbar = reinterpret_cast<uint64_t*>(s_zero + Cfg::ZB_VEC);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int x0 = blockIdx.x * TCX, y0 = blockIdx.y * TY, z0 = blockIdx.z;
  const long long plane = (long long)nx * ny, n = plane * nz;

  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    *abort_flag = 0;
  }
  for (int e = tid; e < Cfg::ZB_VEC; e += TC_NT) s_zero[e] = make_uint4(0u, 0u, 0u, 0u);
  if (warp == 0) {
    tc::tmem_alloc(tslot, Cfg::TMEM_COLS);
    tc::tmem_relinquish();
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t stage_s = tc::smem_addr(s_stage), z_s = tc::smem_addr(s_zero);
  constexpr uint32_t LBO_A = HY * TC_HX * 16;   // channel group 0 -> 1
  constexpr uint32_t LBO_B = 3 * NPAD * 16;     // channel group 0 -> 1 within a dx block
  uint4* s_raw = s_stage + Cfg::HALO_VEC;       // the lo copy of the halo
  uint4* s_w = s_stage + 2 * Cfg::HALO_VEC;
  bool aborted = false;
  uint32_t fail_parity = 0;

#pragma unroll 1
  for (int s = 0; s < Cfg::STEPS; ++s) {
    const int c = s / 3, dz = s % 3, gz = z0 + dz - 1;
    const bool zin = gz >= 0 && gz < nz;
#pragma unroll
    for (int sp = 0; sp < 2; ++sp) {
      const uint4* wsrc = wpk + ((long long)sp * Cfg::CHUNKS + c) * (27 * 2 * NPAD) + dz * Cfg::W_VEC;
      for (int e = tid; e < Cfg::W_VEC; e += TC_NT) cp_async16(&s_w[sp * Cfg::W_VEC + e], &wsrc[e], true);
    }
    {
      float4* hi = reinterpret_cast<float4*>(s_stage);
      float4* lo = reinterpret_cast<float4*>(s_raw);
      const float4* in4 = reinterpret_cast<const float4*>(in);
#pragma unroll 4
      for (int e = tid; e < Cfg::HALO_VEC; e += TC_NT) {
        const int xr = e % TC_HX, t = e / TC_HX;
        const int yr = t % HY, cg = t / HY;
        const int gx = x0 + xr - 1, gy = y0 + yr - 1;
        const bool inb = zin && gx >= 0 && gx < nx && gy >= 0 && gy < ny;
        float4 f = make_float4(0.f, 0.f, 0.f, 0.f);
        const long long ii = (long long)(2 * c + cg) * n + (long long)gz * plane + (long long)gy * nx + gx;
        if (inb && CLAMP_IN_BOUNDS(ii, (long long)(CIN / 4) * n, 341)) f = __ldg(&in4[ii]);
        const float4 h = make_float4(tf32_rn(f.x), tf32_rn(f.y), tf32_rn(f.z), tf32_rn(f.w));
        hi[e] = h;
        lo[e] = make_float4(tf32_rn(f.x - h.x), tf32_rn(f.y - h.y), tf32_rn(f.z - h.z), tf32_rn(f.w - h.w));
      }
    }
    cp_async_wait_all();
    tc::fence_proxy_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after_sync();
      const uint64_t a_hi = tc::make_desc(stage_s, LBO_A, 128);
      const uint64_t a_lo = a_hi + (uint64_t)Cfg::HALO_VEC;   // start address in 16-byte units
      const uint64_t b_hi = tc::make_desc(stage_s + 2u * Cfg::HALO_VEC * 16u, LBO_B, 128);
      const uint64_t b_lo = b_hi + (uint64_t)Cfg::W_VEC;
      if (s == 0) {  // clear every accumulator: D = A x 0
        const uint64_t bz = tc::make_desc(z_s, NPAD * 16, 128);
#pragma unroll
        for (int mt = 0; mt < MT; ++mt)
          mma_kind(TC_TF32X3, tbase + (uint32_t)(mt * NPAD), a_hi, bz, Kd::idesc(128, NPAD), 0u);
      }
#pragma unroll
      for (int hy = 0; hy < HY; ++hy) {
        // tiles ty_lo..ty_hi read halo row hy with taps dy = hy - ty
        const int ty_lo = hy - 2 > 0 ? hy - 2 : 0, ty_hi = hy < TY - 1 ? hy : TY - 1;
        const uint32_t idesc = Kd::idesc(128, (ty_hi - ty_lo + 1) * NPAD);
        const uint32_t dcol = tbase + (uint32_t)(ty_lo * NPAD);
        const int dyp = 2 - (hy - ty_lo);
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const uint64_t aoff = (uint64_t)(hy * TC_HX + dx);
          const uint64_t boff = (uint64_t)(dx * 6 * NPAD + dyp * NPAD);
          // TF32x3 terms: (a_lo, b_hi), (a_hi, b_lo), (a_hi, b_hi)
          mma_kind(TC_TF32X3, dcol, a_lo + aoff, b_hi + boff, idesc, 1u);
          mma_kind(TC_TF32X3, dcol, a_hi + aoff, b_lo + boff, idesc, 1u);
          mma_kind(TC_TF32X3, dcol, a_hi + aoff, b_hi + boff, idesc, 1u);
        }
      }
      tc::mma_commit(mbar);
    }
    // every thread waits for the step's MMAs: they read the buffer the next step overwrites
    if (!tc::mbar_wait_bounded(mbar, (uint32_t)(s & 1), kWaitLimit)) atomicOr(abort_flag, 1);
    __syncthreads();
    if (*abort_flag) {
      aborted = true;
      fail_parity = (uint32_t)(s & 1);
      break;
    }
  }
  tc::fence_after_sync();
  if (!aborted) {
    const int q = warp & 3, h = warp >> 2;
    float4* o4 = reinterpret_cast<float4*>(out_act);
#pragma unroll 1
    for (int mt = 0; mt < MT; ++mt) {
      const int gy = y0 + mt, gx = x0 + 32 * q + lane;
      const long long vox = (long long)z0 * plane + (long long)gy * nx + gx;
      const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(mt * NPAD);
      constexpr int HALF = NPAD / 2;
#pragma unroll
      for (int j = 0; j < HALF / 8; ++j) {
        const int col = h * HALF + 8 * j;
        float v[8];
        tc::tmem_ld_x8(trow + (uint32_t)col, v);
#pragma unroll
        for (int i = 0; i < 8; ++i) v[i] = fmaxf(v[i] + __ldg(&bias[col + i]), 0.f);
        if (CLAMP_IN_BOUNDS((long long)(col / 4 + 1) * n + vox, (long long)(NPAD / 4) * n, 342) &&
            CLAMP_IN_BOUNDS((long long)(col / 4) * n + vox, (long long)(NPAD / 4) * n, 342)) {
          o4[(long long)(col / 4) * n + vox] = make_float4(v[0], v[1], v[2], v[3]);
          o4[(long long)(col / 4 + 1) * n + vox] = make_float4(v[4], v[5], v[6], v[7]);
        }
      }
    }
  } else if (tid == 0) {
    if (err) atomicOr(err, 2);
    // the step's MMAs may still be in flight: give them a bounded wait before TMEM is freed
    tc::mbar_wait_bounded(mbar, fail_parity, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, Cfg::TMEM_COLS);
}

// First layer (one input channel): out[co] = ReLU(b[co] + sum_taps W[co][tap] x(v + tap)), written
// in 16-byte channel groups.  BF16: x and W are BF16-rounded and the output is BF16.
// SIMT: K = 27 is too small for the tensor path.  A CTA stages its input tile with a
// one-voxel halo (zeros outside the volume) in shared memory; a thread computes the two
// voxels (z, z + 1) of a column, so each weight load feeds both.  Taps accumulate in the
// same order for every voxel.
template <int C, bool BF16>
__device__ __forceinline__ void store_first(uint4* out, long long n, long long v, float (&acc)[C]) {
#pragma unroll
  for (int co = 0; co < C; ++co) acc[co] = fmaxf(acc[co], 0.f);
  if constexpr (BF16) {
#pragma unroll
    for (int g = 0; g < C / 8; ++g) {
      uint4 o;
      o.x = pack_bf16x2(acc[8 * g + 0], acc[8 * g + 1]);
      o.y = pack_bf16x2(acc[8 * g + 2], acc[8 * g + 3]);
      o.z = pack_bf16x2(acc[8 * g + 4], acc[8 * g + 5]);
      o.w = pack_bf16x2(acc[8 * g + 6], acc[8 * g + 7]);
      out[(long long)g * n + v] = o;
    }
  } else {
    float4* o4 = reinterpret_cast<float4*>(out);
#pragma unroll
    for (int g = 0; g < C / 4; ++g)
      o4[(long long)g * n + v] = make_float4(acc[4 * g], acc[4 * g + 1], acc[4 * g + 2], acc[4 * g + 3]);
  }
}

constexpr int CF_X = 32, CF_Y = 8, CF_Z = 2;   // CTA tile; a thread computes one (x, y) and CF_Z planes
constexpr int CF_HX = CF_X + 2, CF_HY = CF_Y + 2, CF_HZ = CF_Z + 2;
template <int C, bool BF16>
__global__ void __launch_bounds__(NT) k_conv_first(const float* __restrict__ in, const float* __restrict__ w,
                                                   const float* __restrict__ bias, uint4* __restrict__ out, int nx,
                                                   int ny, int nz) {
  static_assert(CF_X * CF_Y == NT && CF_Z == 2, "one thread per (x, y) column of two planes");
  __shared__ float4 s_w[27 * C / 4];                 // [tap][co]
  __shared__ float s_b[C];
  __shared__ float s_in[CF_HZ * CF_HY * CF_HX];      // input tile with a one-voxel halo, zeros outside
  const int tid = threadIdx.x, tx = tid % CF_X, ty = tid / CF_X;
  const int x0 = blockIdx.x * CF_X, y0 = blockIdx.y * CF_Y, z0 = blockIdx.z * CF_Z;
  const long long plane = (long long)nx * ny, n = plane * nz;
  for (int e = tid; e < 27 * C; e += NT) {
    const int co = e % C, tap = e / C;
    reinterpret_cast<float*>(s_w)[e] = w[co * 27 + tap];
  }
  for (int e = tid; e < C; e += NT) s_b[e] = bias[e];
  for (int e = tid; e < CF_HZ * CF_HY * CF_HX; e += NT) {
    const int xr = e % CF_HX, t = e / CF_HX;
    const int yr = t % CF_HY, zr = t / CF_HY;
    const int gx = x0 + xr - 1, gy = y0 + yr - 1, gz = z0 + zr - 1;
    float v = 0.f;
    if (gx >= 0 && gx < nx && gy >= 0 && gy < ny && gz >= 0 && gz < nz) {
      v = __ldg(&in[(long long)gz * plane + (long long)gy * nx + gx]);
      if (BF16) v = __bfloat162float(__float2bfloat16_rn(v));
    }
    s_in[e] = v;
  }
  __syncthreads();
  const int x = x0 + tx, y = y0 + ty;
  if (x >= nx || y >= ny) return;
  float a0[C], a1[C];
#pragma unroll
  for (int co = 0; co < C; ++co) a0[co] = a1[co] = s_b[co];
  // taps in order tap = 9 dz + 3 dy + dx; dy and dx unrolled, so every shared-memory
  // offset but the plane's is a constant
#pragma unroll 1
  for (int dz = 0; dz < 3; ++dz) {
    const float* pl = s_in + dz * CF_HY * CF_HX + ty * CF_HX + tx;
    const float4* wz = s_w + dz * 9 * (C / 4);
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const float x0v = pl[dy * CF_HX + dx], x1v = pl[CF_HY * CF_HX + dy * CF_HX + dx];
#pragma unroll
        for (int q = 0; q < C / 4; ++q) {
          const float4 wv = wz[(dy * 3 + dx) * (C / 4) + q];
          a0[4 * q + 0] = fmaf(x0v, wv.x, a0[4 * q + 0]);
          a0[4 * q + 1] = fmaf(x0v, wv.y, a0[4 * q + 1]);
          a0[4 * q + 2] = fmaf(x0v, wv.z, a0[4 * q + 2]);
          a0[4 * q + 3] = fmaf(x0v, wv.w, a0[4 * q + 3]);
          a1[4 * q + 0] = fmaf(x1v, wv.x, a1[4 * q + 0]);
          a1[4 * q + 1] = fmaf(x1v, wv.y, a1[4 * q + 1]);
          a1[4 * q + 2] = fmaf(x1v, wv.z, a1[4 * q + 2]);
          a1[4 * q + 3] = fmaf(x1v, wv.w, a1[4 * q + 3]);
        }
      }
    }
  }
  const long long v = (long long)z0 * plane + (long long)y * nx + x;
  store_first<C, BF16>(out, n, v, a0);
  if (z0 + 1 < nz) store_first<C, BF16>(out, n, v + plane, a1);
}

// Last layer of the FP32 residual CNN (C -> 1) on FP32 CUDA cores, reading the tensor
// path's [C/4][nz][ny][nx][4] activations: out = x + b + sum_{c, tap} W[c][tap] act_c(v + tap).
// A TF32x3 tensor-core tile would pad the single output channel to 16 columns and stage
// the same hi/lo halo as a hidden layer for 1/C of its useful work.  CTA tile: 64
// x-voxels x 4 rows x CL_Z planes, 128 threads; a thread computes x-voxels tx and tx + 32
// (so a warp's shared-memory row reads are consecutive) on CL_Z planes.  One 4-channel
// group of the halo (CL_Z + 2 planes, 38 KB) is staged with cp.async at a time, each
// staged row feeding every output plane it borders; four CTAs share an SM, so one
// CTA's staging overlaps the others' arithmetic.
constexpr int CL_X = 64, CL_Y = 4, CL_Z = 4, CL_NT = 128;
constexpr int CL_HX = CL_X + 2, CL_HY = CL_Y + 2, CL_HZ = CL_Z + 2;
constexpr size_t CL_SMEM = sizeof(float4) * CL_HZ * CL_HY * CL_HX;
template <int C>
__global__ void __launch_bounds__(CL_NT, 4) k_conv_last(const float4* __restrict__ act, const float* __restrict__ w,
                                                     const float* __restrict__ bias, const float* __restrict__ resid,
                                                     float* __restrict__ out, int nx, int ny, int nz) {
  constexpr int G = C / 4;
  extern __shared__ float4 s_h[];     // [CL_HZ][CL_HY][CL_HX]
  __shared__ float4 s_w[27 * G];      // [tap][channel group]: 4 channels' weights
  const int tid = threadIdx.x, tx = tid % 32, ty = tid / 32;
  const int x0 = blockIdx.x * CL_X, y0 = blockIdx.y * CL_Y, z0 = blockIdx.z * CL_Z;
  const long long plane = (long long)nx * ny, n = plane * nz;
  for (int e = tid; e < 27 * G; e += CL_NT) {
    const int g = e % G, tap = e / G;
    s_w[e] = make_float4(w[(4 * g) * 27 + tap], w[(4 * g + 1) * 27 + tap], w[(4 * g + 2) * 27 + tap],
                         w[(4 * g + 3) * 27 + tap]);
  }
  float acc[CL_Z][2];
#pragma unroll
  for (int zo = 0; zo < CL_Z; ++zo) acc[zo][0] = acc[zo][1] = 0.f;
#pragma unroll 1
  for (int g = 0; g < G; ++g) {
    __syncthreads();   // the previous group's reads of the halo are done
    // one warp per halo row (z, y), lanes along x: the row's index arithmetic once per row
    for (int row = tid / 32; row < CL_HZ * CL_HY; row += CL_NT / 32) {
      const int yr = row % CL_HY, zr = row / CL_HY;
      const int gy = y0 + yr - 1, gz = z0 + zr - 1;
      const bool rin = gy >= 0 && gy < ny && gz >= 0 && gz < nz;
      const float4* rsrc = act + (long long)g * n + (long long)gz * plane + (long long)gy * nx;
      for (int xr = tid % 32; xr < CL_HX; xr += 32) {
        const int gx = x0 + xr - 1;
        const bool inb = rin && gx >= 0 && gx < nx;
        cp_async16(&s_h[row * CL_HX + xr], inb ? rsrc + gx : act, inb);
      }
    }
    cp_async_wait_all();
    __syncthreads();
#pragma unroll
    for (int pz = 0; pz < CL_HZ; ++pz) {
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const float4* row = s_h + (pz * CL_HY + ty + dy) * CL_HX + tx;
        const float4 f[6] = {row[0], row[1], row[2], row[32], row[33], row[34]};
#pragma unroll
        for (int dz = 0; dz < 3; ++dz) {
          const int zo = pz - dz;   // output plane this staged plane feeds with tap dz
          if (zo < 0 || zo >= CL_Z) continue;
#pragma unroll
          for (int dx = 0; dx < 3; ++dx) {
            const float4 wv = s_w[(dz * 9 + dy * 3 + dx) * G + g];
            acc[zo][0] = fmaf(wv.x, f[dx].x, fmaf(wv.y, f[dx].y, fmaf(wv.z, f[dx].z, fmaf(wv.w, f[dx].w, acc[zo][0]))));
            acc[zo][1] = fmaf(wv.x, f[dx + 3].x,
                              fmaf(wv.y, f[dx + 3].y, fmaf(wv.z, f[dx + 3].z, fmaf(wv.w, f[dx + 3].w, acc[zo][1]))));
          }
        }
      }
    }
  }
  const int gy = y0 + ty;
  if (gy >= ny) return;
  const float b = __ldg(&bias[0]);
#pragma unroll
  for (int zo = 0; zo < CL_Z; ++zo) {
    const int gz = z0 + zo;
    if (gz >= nz) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int gx = x0 + tx + 32 * j;
      if (gx >= nx) continue;
      const long long vox = (long long)gz * plane + (long long)gy * nx + gx;
      out[vox] = acc[zo][j] + b + resid[vox];
    }
  }
}

// Self-check of the bounded mbarrier wait the tensor-core kernels use instead of an
// unbounded spin: barrier 0 receives its one arrival, so its wait must succeed; nothing
// arrives on barrier 1, so its wait must give up after `limit` polls.
__global__ void k_wait_selftest(uint32_t limit, int* out) {
  __shared__ uint64_t mbar[2];
  if (threadIdx.x == 0) {
    tc::mbar_init(&mbar[0], 1);
    tc::mbar_init(&mbar[1], 1);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(tc::smem_addr(&mbar[0]))
                 : "memory");
    out[0] = tc::mbar_wait_bounded(&mbar[0], 0u, limit) ? 1 : 0;
    out[1] = tc::mbar_wait_bounded(&mbar[1], 0u, limit) ? 1 : 0;
  }
}

// One-tile GEMM on the tensor core: D[128][N] = A[128][K] B[N][K]^T, FP32 out.  BF16 operands
// (KIND = BF16) or FP32 operands through the TF32x3 split.  Checks the descriptor,
// instruction-descriptor and TMEM conventions the conv kernels rely on.
template <int KIND>
__global__ void __launch_bounds__(128, 1) k_tc_gemm(const void* __restrict__ Av, const void* __restrict__ Bv,
                                                    float* __restrict__ D, int N, int K) {
  using Kd = TcKind<KIND>;
  constexpr int EPV = Kd::EPV, ES = 16 / EPV;  // elements per vector, bytes per element
  extern __shared__ unsigned char g_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)g_smem_raw + 1023) & ~(uintptr_t)1023);
  const size_t a_bytes = (size_t)K * 128 * ES, b_bytes = (size_t)K * N * ES;
  unsigned char* sA = base;                        // [SPLIT][K/EPV][128][EPV]
  unsigned char* sB = base + Kd::SPLIT * a_bytes;  // [SPLIT][K/EPV][N][EPV]
  uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + Kd::SPLIT * b_bytes);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  for (int e = tid; e < 128 * K; e += 128) {
    const int m = e / K, k = e % K;
    const size_t off = ((size_t)(k / EPV) * 128 + m) * EPV + k % EPV;
    if constexpr (KIND == TC_BF16) {
      reinterpret_cast<unsigned short*>(sA)[off] = static_cast<const unsigned short*>(Av)[e];
    } else {
      const float x = static_cast<const float*>(Av)[e], h = tf32_rn(x);
      reinterpret_cast<float*>(sA)[off] = h;
      reinterpret_cast<float*>(sA + a_bytes)[off] = tf32_rn(x - h);
    }
  }
  for (int e = tid; e < N * K; e += 128) {
    const int nn = e / K, k = e % K;
    const size_t off = ((size_t)(k / EPV) * N + nn) * EPV + k % EPV;
    if constexpr (KIND == TC_BF16) {
      reinterpret_cast<unsigned short*>(sB)[off] = static_cast<const unsigned short*>(Bv)[e];
    } else {
      const float x = static_cast<const float*>(Bv)[e], h = tf32_rn(x);
      reinterpret_cast<float*>(sB)[off] = h;
      reinterpret_cast<float*>(sB + b_bytes)[off] = tf32_rn(x - h);
    }
  }
  const uint32_t ncols = (uint32_t)pow2_cols(N);
  if (tid == 0) tc::mbar_init(mbar, 1);
  if (warp == 0) {
    tc::tmem_alloc(tslot, ncols);
    tc::tmem_relinquish();
  }
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  if (tid == 0) {
    const uint32_t a_s = tc::smem_addr(sA), b_s = tc::smem_addr(sB);
    const uint32_t idesc = Kd::idesc(128, N);
    for (int kk = 0; kk < K / (2 * EPV); ++kk) {
      const uint64_t ah = tc::make_desc(a_s + kk * 2 * 128 * 16, 128 * 16, 128);
      const uint64_t bh = tc::make_desc(b_s + kk * 2 * N * 16, N * 16, 128);
      if constexpr (KIND == TC_BF16) {
        mma_kind(KIND, tbase, ah, bh, idesc, kk > 0 ? 1u : 0u);
      } else {
        const uint64_t al = tc::make_desc(a_s + (uint32_t)a_bytes + kk * 2 * 128 * 16, 128 * 16, 128);
        const uint64_t bl = tc::make_desc(b_s + (uint32_t)b_bytes + kk * 2 * N * 16, N * 16, 128);
        mma_kind(KIND, tbase, al, bh, idesc, kk > 0 ? 1u : 0u);
        mma_kind(KIND, tbase, ah, bl, idesc, 1u);
        mma_kind(KIND, tbase, ah, bh, idesc, 1u);
      }
    }
    tc::mma_commit(mbar);
  }
  const bool ok = __all_sync(0xffffffffu, tc::mbar_wait_bounded(mbar, 0u, kWaitLimit));
  tc::fence_after_sync();
  if (ok) {
    const int m = 32 * warp + lane;
    for (int c = 0; c < N; c += 8) {
      float v[8];
      tc::tmem_ld_x8(tbase + ((uint32_t)(32 * warp) << 16) + (uint32_t)c, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) D[m * N + c + i] = v[i];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, ncols);
}

// ---------------------------------------------------------------- host side

static uint16_t bf16_bits(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u = (u + 0x7FFFu + ((u >> 16) & 1u)) >> 16;  // round to nearest even (finite inputs)
  return (uint16_t)u;
}
static float bits_to_float(uint32_t u) {
  float r;
  memcpy(&r, &u, 4);
  return r;
}
float bf16_round_value(float f) { return bits_to_float((uint32_t)bf16_bits(f) << 16); }
static float tf32_rn_host(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0xFFFu + ((u >> 13) & 1u);
  return bits_to_float(u & 0xFFFFE000u);
}

template <int KIND, int CIN, int NPAD, bool LAST, bool TAPS = false>
static cudaError_t run_tc(const uint4* in, const uint4* wpk, const float* bias, uint4* out_act, float* out_f32,
                          const float* resid, int nx, int ny, int nz, int* err, cudaStream_t st,
                          const uint4* wtaps = nullptr, float* P = nullptr) {
  using Cfg = TcCfg<KIND, CIN, NPAD>;
  auto kern = k_conv3_tc<KIND, CIN, NPAD, LAST, TAPS>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
  if (e != cudaSuccess) return e;
  // persistent: MIN_CTAS CTAs per SM, each walking tiles
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)(nx / TCX) * (ny / Cfg::TY) * (nz / Cfg::TZ);
  const int grid = (int)std::min<long long>(ntiles, (long long)sms * TcKind<KIND>::MIN_CTAS);
  kern<<<grid, TC_NT, Cfg::SMEM, st>>>(in, wpk, bias, out_act, out_f32, resid, nx, ny, nz, err, wtaps, P);
  return cudaGetLastError();
}

template <int CIN, int NPAD>
static cudaError_t run_tc_plane(const uint4* in, const uint4* wpk, const float* bias, uint4* out_act, int nx, int ny,
                                int nz, int* err, cudaStream_t st) {
  using Cfg = TcPlaneCfg<CIN, NPAD>;
  auto kern = k_conv3_tc_plane<CIN, NPAD>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Cfg::SMEM);
  if (e != cudaSuccess) return e;
  dim3 grid(nx / TCX, ny / Cfg::TY, nz);
  kern<<<grid, TC_NT, Cfg::SMEM, st>>>(in, wpk, bias, out_act, nx, ny, nz, err);
  return cudaGetLastError();
}

template <int C, bool BF16>
static cudaError_t run_first(const float* in, const float* w, const float* b, uint4* out, int nx, int ny, int nz,
                             cudaStream_t st) {
  dim3 grid((nx + CF_X - 1) / CF_X, (ny + CF_Y - 1) / CF_Y, (nz + CF_Z - 1) / CF_Z);
  k_conv_first<C, BF16><<<grid, NT, 0, st>>>(in, w, b, out, nx, ny, nz);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- first BF16 layer (1 -> C) on tensor cores

// With one input channel the 27 taps are the GEMM's K: a CTA builds, per 128-voxel output
// row, the im2col tile A[v][k] = x[v + tap k] (k = 9 dz + 3 dy + dx < 27, zero for
// 27 <= k < 32) in BF16 from its input halo, and two K = 16 MMAs against the packed weights
// B[co][k] give all C outputs in TMEM; the epilogue is the hidden layers'.  Tiles of 2 rows
// x 2 planes, as k_conv3_tc<BF16> (tiles of 2 rows x 1 plane, four CTAs per SM by TMEM,
// measured slower).  Layouts (no-swizzle K-major): element (row, k) of A at
// (row / 8) * 512 + (k / 8) * 128 + (row % 8) * 16 + (k % 8) * 2, the same for B with co.
//
// Persistent: each CTA takes its TMEM and weights once and walks the tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...; the next tile's FP32 halo is copied (cp.async, 4-byte
// elements: the halo row starts at x0 - 1) into a raw buffer while the current tile's
// im2col, MMAs and epilogue run.  The four tile rows are multiplied and written in two
// rounds of two, so a CTA holds 2 C TMEM columns (128 at 48 channels) and four CTAs share
// an SM.
constexpr int CF1_TY = 2, CF1_TZ = 2, CF1_MT = CF1_TY * CF1_TZ;
constexpr int CF1_HY = CF1_TY + 2, CF1_HZ = CF1_TZ + 2, CF1_HROWS = CF1_HY * CF1_HZ;
constexpr int CF1_A_BYTES = 128 * 64;                               // one im2col tile (K = 32)
constexpr int CF1_HALF = CF1_MT / 2;   // tile rows per MMA round (their accumulators share TMEM)
__host__ __device__ constexpr size_t cf1_smem(int C) {
  // im2col tiles, weights, BF16 halo, FP32 raw halo, mbarrier + TMEM slot + abort flag
  return 1024 + (size_t)CF1_MT * CF1_A_BYTES + (size_t)C * 64 + 2 * CF1_HROWS * TC_HX + 4 * CF1_HROWS * TC_HX + 64;
}

template <int C>
__global__ void __launch_bounds__(TC_NT) k_conv_first_tc(const float* __restrict__ in, const uint4* __restrict__ wpk,
                                                         const float* __restrict__ bias, uint4* __restrict__ out,
                                                         int nx, int ny, int nz, int* err) {
  static_assert(C % 16 == 0 && C <= 64, "channels");
  constexpr int TMEM_COLS = pow2_cols(CF1_HALF * C);
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* s_a = base;                                            // [MT][8 KB]
  uint4* s_w = reinterpret_cast<uint4*>(s_a + CF1_MT * CF1_A_BYTES);    // C * 64 bytes
  uint16_t* s_x = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(s_w) + C * 64);  // [HZ][HY][HX]
  float* s_raw = reinterpret_cast<float*>(s_x + CF1_HROWS * TC_HX);     // [HZ][HY][HX], FP32
  uint64_t* mbar = reinterpret_cast<uint64_t*>(s_raw + CF1_HROWS * TC_HX);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  int* abort_flag = reinterpret_cast<int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long plane = (long long)nx * ny, n = plane * nz;
  const int tiles_x = nx / TCX, tiles_y = ny / CF1_TY, ntiles = tiles_x * tiles_y * (nz / CF1_TZ);
  auto origin = [&](int t, int& x0, int& y0, int& z0) {
    x0 = (t % tiles_x) * TCX;
    t /= tiles_x;
    y0 = (t % tiles_y) * CF1_TY;
    z0 = (t / tiles_y) * CF1_TZ;
  };
  // the FP32 input halo of tile t into s_raw, zeros outside: a warp per halo row, lanes along x
  auto stage_raw = [&](int t) {
    int x0, y0, z0;
    origin(t, x0, y0, z0);
    for (int r = warp; r < CF1_HROWS; r += TC_NT / 32) {
      const int yr = r % CF1_HY, zr = r / CF1_HY;
      const int gy = y0 + yr - 1, gz = z0 + zr - 1;
      const bool rin = gy >= 0 && gy < ny && gz >= 0 && gz < nz;
      const long long rbase = (long long)gz * plane + (long long)gy * nx;
      for (int xr = lane; xr < TC_HX; xr += 32) {
        const int gx = x0 + xr - 1;
        const bool inb = rin && gx >= 0 && gx < nx && CLAMP_IN_BOUNDS(rbase + gx, n, 311);
        cp_async4(&s_raw[r * TC_HX + xr], inb ? &in[rbase + gx] : in, inb);
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };

  if (tid == 0) {
    tc::mbar_init(mbar, 1);
    *abort_flag = 0;
  }
  if (warp == 0) {
    tc::tmem_alloc(tslot, TMEM_COLS);
    tc::tmem_relinquish();
  }
  for (int e = tid; e < C * 4; e += TC_NT) cp_async16(&s_w[e], &wpk[e], true);
  if ((int)blockIdx.x < ntiles) stage_raw(blockIdx.x);   // commits the weights with the first halo
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  const uint32_t a_s = tc::smem_addr(s_a), w_s = tc::smem_addr(s_w);
  uint32_t phase = 0;   // MMA commits completed so far (the mbarrier's phase parity)
  bool aborted = false;

#pragma unroll 1
  for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
    int x0, y0, z0;
    origin(tile, x0, y0, z0);
    asm volatile("cp.async.wait_group 0;" ::: "memory");   // this tile's raw halo (and, first, the weights)
    __syncthreads();
    for (int e = tid; e < CF1_HROWS * TC_HX; e += TC_NT) s_x[e] = __bfloat16_as_ushort(__float2bfloat16_rn(s_raw[e]));
    __syncthreads();   // s_raw is free again and s_x complete
    if (tile + (int)gridDim.x < ntiles) stage_raw(tile + (int)gridDim.x);
    // im2col: a thread builds whole rows (128-voxel tile row, all four 8-tap groups), so
    // every tap offset is a compile-time constant.  s_a is free: the previous tile's MMAs
    // completed before its epilogue.
    for (int e = tid; e < CF1_MT * 128; e += TC_NT) {
      const int row = e % 128, mt = e / 128;
      const int ty = mt % CF1_TY, tz = mt / CF1_TY;
      const uint16_t* xs = s_x + (tz * CF1_HY + ty) * TC_HX + row;
      unsigned char* arow = s_a + mt * CF1_A_BYTES + (row / 8) * 512 + (row % 8) * 16;
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        uint32_t w4[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          uint32_t pair = 0;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int k = 8 * g + 2 * j + h;
            if (k < 27) pair |= (uint32_t)xs[((k / 9) * CF1_HY + (k / 3) % 3) * TC_HX + k % 3] << (16 * h);
          }
          w4[j] = pair;
        }
        *reinterpret_cast<uint4*>(arow + g * 128) = make_uint4(w4[0], w4[1], w4[2], w4[3]);
      }
    }
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    // two rounds of CF1_HALF tile rows: half the TMEM per CTA, so four CTAs share an SM
#pragma unroll 1
    for (int round = 0; round < CF1_MT / CF1_HALF; ++round) {
      if (tid == 0) {
        tc::fence_after_sync();
#pragma unroll
        for (int m = 0; m < CF1_HALF; ++m) {
          const int mt = round * CF1_HALF + m;
#pragma unroll
          for (int h = 0; h < 2; ++h)
            tc::mma_bf16(tbase + (uint32_t)(m * C), tc::make_desc(a_s + mt * CF1_A_BYTES + h * 256, 128, 512),
                         tc::make_desc(w_s + h * 256, 128, 512), TcKind<TC_BF16>::idesc(128, C), h ? 1u : 0u);
        }
        tc::mma_commit(mbar);
        if (!tc::mbar_wait_bounded(mbar, phase & 1u, kWaitLimit)) *abort_flag = 1;
      }
      __syncthreads();
      if (*abort_flag) {
        aborted = true;
        break;
      }
      ++phase;
      tc::fence_after_sync();
      const int q = warp & 3, hh = warp >> 2;
#pragma unroll 1
      for (int m = 0; m < CF1_HALF; ++m) {
        const int mt = round * CF1_HALF + m;
        const int gy = y0 + mt % CF1_TY, gz = z0 + mt / CF1_TY, gx = x0 + 32 * q + lane;
        const long long vox = (long long)gz * plane + (long long)gy * nx + gx;
        const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(m * C);
        constexpr int HALF = C / 2;
#pragma unroll
        for (int j = 0; j < HALF / 8; ++j) {
          const int col = hh * HALF + 8 * j;
          float v[8];
          tc::tmem_ld_x8(trow + (uint32_t)col, v);
#pragma unroll
          for (int i = 0; i < 8; ++i) v[i] = fmaxf(v[i] + __ldg(&bias[col + i]), 0.f);
          uint4 o;
          o.x = pack_bf16x2(v[0], v[1]);
          o.y = pack_bf16x2(v[2], v[3]);
          o.z = pack_bf16x2(v[4], v[5]);
          o.w = pack_bf16x2(v[6], v[7]);
          if (CLAMP_IN_BOUNDS((long long)(col / 8) * n + vox, (long long)(C / 8) * n, 312))
            out[(long long)(col / 8) * n + vox] = o;
        }
      }
      // TMEM reads complete before the next round's MMAs overwrite the accumulators
      tc::fence_before_sync();
      __syncthreads();
    }
    if (aborted) break;
  }
  asm volatile("cp.async.wait_group 0;" ::: "memory");   // a prefetch still in flight after an abort
  if (aborted && tid == 0) {
    if (err) atomicOr(err, 2);
    tc::mbar_wait_bounded(mbar, phase & 1u, kWaitLimit);   // give the MMAs a bounded wait before TMEM is freed
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, TMEM_COLS);
}

template <int C>
static cudaError_t run_first_tc(const float* in, const uint4* wpk, const float* b, uint4* out, int nx, int ny, int nz,
                                int* err, cudaStream_t st) {
  // CTAs per SM: TMEM (512 columns) and shared memory (about 49 KB each) allow at most four;
  // where TMEM allows fewer, the shared-memory request is raised so that no further CTA
  // lands on an SM (it would wait for TMEM while other SMs idle)
  constexpr int per_sm = 512 / pow2_cols(CF1_HALF * C) < 4 ? 512 / pow2_cols(CF1_HALF * C) : 4;
  const size_t smem = std::max(cf1_smem(C), per_sm < 4 ? (size_t)(227 * 1024 / (per_sm + 1)) : (size_t)0);
  cudaError_t e = cudaFuncSetAttribute(k_conv_first_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int dev = 0, sms = 0;
  if (e == cudaSuccess) e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long ntiles = (long long)(nx / TCX) * (ny / CF1_TY) * (nz / CF1_TZ);
  const int grid = (int)std::min<long long>(ntiles, (long long)sms * per_sm);
  k_conv_first_tc<C><<<grid, TC_NT, smem, st>>>(in, wpk, b, out, nx, ny, nz, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- last BF16 layer (C -> 1)

// out[v] = x[v] + b + sum_tap sum_c W[tap][c] h[v + tap][c] is split into a pointwise GEMM,
// P_tap[u] = sum_c W[tap][c] h[u][c] for the 27 taps of every voxel u (tensor cores: M = 128
// voxels, K = C channels, N = 27 taps padded to 32, FP32 accumulators), and a gather
// out[v] = x[v] + b + sum_tap P_tap[v + tap] (zero outside the volume).  The GEMM reads each
// activation once with no halo: in the [C/8][n][8] BF16 layout 128 consecutive voxels of one
// channel group are 16 no-swizzle K-major core matrices back to back, so a tile is copied
// as is.  B (the weights, BF16) is [C/8][32 taps][8]: element (tap, c) at (c / 8) * 512 +
// tap * 16 + (c % 8) * 2.  P is FP32 [27][n] (tap-major).
constexpr int CL2_MT = 4;   // 128-voxel tiles per CTA

// Bytes of each of the prior's two activation buffers: C channels per voxel, and for BF16 at
// least the last layer's tap sums P (27 FP32 values per voxel), which go to whichever
// buffer the last hidden layer did not write.
static size_t tc_buffer_bytes(bool bf16, int C, size_t n) {
  const size_t act = ((size_t)C * n * (bf16 ? 2 : 4) + 255) & ~(size_t)255;
  return bf16 ? std::max(act, (27 * n * 4 + 255) & ~(size_t)255) : act;
}

template <int C>
__global__ void __launch_bounds__(TC_NT) k_last_taps_tc(const uint4* __restrict__ act, const uint4* __restrict__ wpk,
                                                        float* __restrict__ P, long long n, int* err) {
  constexpr int G = C / 8, KSTEPS = C / 16, TMEM_COLS = pow2_cols(CL2_MT * 32);
  extern __shared__ unsigned char tc_smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(((uintptr_t)tc_smem_raw + 1023) & ~(uintptr_t)1023);
  uint4* s_a = reinterpret_cast<uint4*>(base);                  // [MT][G][128 voxels] x 16 B
  uint4* s_w = s_a + CL2_MT * G * 128;                          // [G][32 taps] x 16 B
  uint64_t* mbar = reinterpret_cast<uint64_t*>(s_w + G * 32);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const long long v0 = (long long)blockIdx.x * (CL2_MT * 128);
  if (tid == 0) tc::mbar_init(mbar, 1);
  if (warp == 0) {
    tc::tmem_alloc(tslot, TMEM_COLS);
    tc::tmem_relinquish();
  }
  for (int e = tid; e < CL2_MT * G * 128; e += TC_NT) {
    const int vv = e % 128, g = (e / 128) % G, mt = e / (128 * G);
    cp_async16(&s_a[e], &act[(long long)g * n + v0 + mt * 128 + vv],
               CLAMP_IN_BOUNDS((long long)g * n + v0 + mt * 128 + vv, (long long)G * n, 321));
  }
  for (int e = tid; e < G * 32; e += TC_NT) cp_async16(&s_w[e], &wpk[e], true);
  cp_async_wait_all();
  tc::fence_proxy_async();
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tbase = *tslot;
  if (tid == 0) {
    const uint32_t a_s = tc::smem_addr(s_a), w_s = tc::smem_addr(s_w);
#pragma unroll
    for (int mt = 0; mt < CL2_MT; ++mt)
#pragma unroll
      for (int ks = 0; ks < KSTEPS; ++ks)
        tc::mma_bf16(tbase + (uint32_t)(mt * 32),
                     tc::make_desc(a_s + (uint32_t)((mt * G + 2 * ks) * 128 * 16), 128 * 16, 128),
                     tc::make_desc(w_s + (uint32_t)(2 * ks * 32 * 16), 32 * 16, 128), TcKind<TC_BF16>::idesc(128, 32),
                     ks ? 1u : 0u);
    tc::mma_commit(mbar);
  }
  const bool done = tc::mbar_wait_bounded(mbar, 0u, kWaitLimit);
  tc::fence_after_sync();
  if (done) {
    const int q = warp & 3, hh = warp >> 2;
#pragma unroll 1
    for (int mt = 0; mt < CL2_MT; ++mt) {
      const long long v = v0 + mt * 128 + 32 * q + lane;
      const uint32_t trow = tbase + ((uint32_t)(32 * q) << 16) + (uint32_t)(mt * 32);
#pragma unroll
      for (int j = 0; j < 2; ++j) {
        const int col = hh * 16 + 8 * j;
        float t[8];
        tc::tmem_ld_x8(trow + (uint32_t)col, t);
#pragma unroll
        for (int i = 0; i < 8; ++i)
          if (col + i < 27 && CLAMP_IN_BOUNDS((long long)(col + i) * n + v, 27 * n, 322))
            P[(long long)(col + i) * n + v] = t[i];
      }
    }
  } else if (tid == 0) {
    if (err) atomicOr(err, 2);
    tc::mbar_wait_bounded(mbar, 0u, kWaitLimit);
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, TMEM_COLS);
}

// out[v] = resid[v] + bias + sum over the 27 taps of P_tap[v + tap] inside the volume.
// Branch-free: every tap loads at coordinates clamped into the volume (always a valid
// address) and a tap outside the volume adds 0, so all 27 loads of a thread are issued
// before the first add.  The sum runs in tap order.
__global__ void __launch_bounds__(NT) k_last_gather(const float* __restrict__ P, const float* __restrict__ bias,
                                                    const float* __restrict__ resid, float* __restrict__ out, int nx,
                                                    int ny, int nz) {
  const long long plane = (long long)nx * ny, n = plane * nz;
  const long long v = (long long)blockIdx.x * NT + threadIdx.x;
  if (v >= n) return;
  const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / plane);
  float t[27];
  unsigned inside = 0u;   // bit tap: the tap's voxel lies in the volume
#pragma unroll
  for (int dz = 0; dz < 3; ++dz) {
    const int zz = z + dz - 1, zc = min(max(zz, 0), nz - 1);
#pragma unroll
    for (int dy = 0; dy < 3; ++dy) {
      const int yy = y + dy - 1, yc = min(max(yy, 0), ny - 1);
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) {
        const int xx = x + dx - 1, xc = min(max(xx, 0), nx - 1);
        const int tap = 9 * dz + 3 * dy + dx;
        const long long pi = (long long)tap * n + (long long)zc * plane + (long long)yc * nx + xc;
        t[tap] = CLAMP_IN_BOUNDS(pi, 27 * n, 331) ? __ldg(&P[pi]) : 0.f;
        if (zz == zc && yy == yc && xx == xc) inside |= 1u << tap;
      }
    }
  }
  float acc = __ldg(&bias[0]) + resid[v];
#pragma unroll
  for (int tap = 0; tap < 27; ++tap) acc += (inside >> tap) & 1u ? t[tap] : 0.f;
  out[v] = acc;
}

template <int C>
static cudaError_t run_last_tc(const uint4* act, const uint4* wpk, const float* b, const float* resid, float* out,
                               float* P, int nx, int ny, int nz, int* err, cudaStream_t st) {
  const long long n = (long long)nx * ny * nz;
  const size_t smem = 1024 + (size_t)16 * (CL2_MT * (C / 8) * 128 + (C / 8) * 32) + 64;
  cudaError_t e = cudaFuncSetAttribute(k_last_taps_tc<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_last_taps_tc<C><<<(unsigned)(n / (CL2_MT * 128)), TC_NT, smem, st>>>(act, wpk, P, n, err);
  k_last_gather<<<(unsigned)((n + NT - 1) / NT), NT, 0, st>>>(P, b, resid, out, nx, ny, nz);
  return cudaGetLastError();
}

template <int KIND, int C>
static cudaError_t apply_tc_c(const clamp_denoiser* d, const float* in, float* out, int nx, int ny, int nz, void* ws,
                              int* err, cudaStream_t st) {
  const size_t n = (size_t)nx * ny * nz;
  uint4* A = static_cast<uint4*>(ws);
  uint4* B = reinterpret_cast<uint4*>(static_cast<char*>(ws) + tc_buffer_bytes(KIND == TC_BF16, C, n));
  cudaError_t e = (KIND == TC_BF16 && d->w16[0])
                      ? run_first_tc<C>(in, static_cast<const uint4*>(d->w16[0]), d->b[0], A, nx, ny, nz, err, st)
                      : run_first<C, KIND == TC_BF16>(in, d->w[0], d->b[0], A, nx, ny, nz, st);
  if (e != cudaSuccess) return e;
  uint4* cur = A;
  // BF16 with at least one hidden layer and C >= 32: the last hidden layer also forms the
  // last layer's tap sums (k_conv3_tc<..., TAPS>), so the last layer is only the gather
  constexpr bool kFuse = KIND == TC_BF16 && C >= 32 && !tc_tall(KIND, C);
  const bool fuse = kFuse && d->layers >= 3;
  for (int i = 1; i < d->layers; ++i) {
    const uint4* wp = static_cast<const uint4*>(d->w16[i]);
    if (i == d->layers - 1) {
      if constexpr (KIND == TC_BF16) {
        if (fuse) {   // cur holds the tap sums P
          k_last_gather<<<(unsigned)((n + NT - 1) / NT), NT, 0, st>>>(reinterpret_cast<const float*>(cur), d->b[i],
                                                                      in, out, nx, ny, nz);
          e = cudaGetLastError();
        } else {
          // per-voxel tap sums on the tensor cores, then a gather (no halo staging)
          float* P = reinterpret_cast<float*>(cur == A ? B : A);
          e = run_last_tc<C>(cur, static_cast<const uint4*>(d->w_last), d->b[i], in, out, P, nx, ny, nz, err, st);
        }
      } else {
        // TF32x3: the padded tile costs as much as a hidden layer; CUDA cores instead
        e = cudaFuncSetAttribute(k_conv_last<C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM);
        if (e != cudaSuccess) return e;
        dim3 grid((nx + CL_X - 1) / CL_X, (ny + CL_Y - 1) / CL_Y, (nz + CL_Z - 1) / CL_Z);
        k_conv_last<C><<<grid, CL_NT, CL_SMEM, st>>>(reinterpret_cast<const float4*>(cur), d->w[i], d->b[i], in,
                                                     out, nx, ny, nz);
        e = cudaGetLastError();
      }
    } else {
      uint4* dst = cur == A ? B : A;
      if constexpr (tc_tall(KIND, C)) {
        e = run_tc_plane<C, C>(cur, wp, d->b[i], dst, nx, ny, nz, err, st);
      } else if constexpr (kFuse) {
        if (fuse && i == d->layers - 2)   // P (FP32 [27][n]) goes to dst
          e = run_tc<KIND, C, C, false, true>(cur, wp, d->b[i], nullptr, nullptr, nullptr, nx, ny, nz, err, st,
                                              static_cast<const uint4*>(d->w_last), reinterpret_cast<float*>(dst));
        else
          e = run_tc<KIND, C, C, false>(cur, wp, d->b[i], dst, nullptr, nullptr, nx, ny, nz, err, st);
      } else {
        e = run_tc<KIND, C, C, false>(cur, wp, d->b[i], dst, nullptr, nullptr, nx, ny, nz, err, st);
      }
      cur = dst;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

bool tc_denoiser_supports(const clamp_denoiser* d, int nx, int ny, int nz) {
  const bool bf = d->dtype == CLAMP_DENOISER_BF16;
  const int C = d->channels;
  const bool ch = bf ? (C == 16 || C == 32 || C == 48 || C == 64) : (C == 16 || C == 32 || C == 48);
  const bool tall = tc_tall(bf ? TC_BF16 : TC_TF32X3, C);
  const int ty = tall ? 4 : bf ? TcKind<TC_BF16>::TY : TcKind<TC_TF32X3>::TY;
  const int tz = tall ? 1 : bf ? TcKind<TC_BF16>::TZ : TcKind<TC_TF32X3>::TZ;
  return ch && nx % TCX == 0 && ny % ty == 0 && nz % tz == 0;
}

size_t tc_denoise_ws_bytes(const clamp_denoiser* d, int nx, int ny, int nz) {
  return 2 * tc_buffer_bytes(d->dtype == CLAMP_DENOISER_BF16, d->channels, (size_t)nx * ny * nz);
}

cudaError_t tc_denoise_apply(const clamp_denoiser* d, const float* in, float* out, int nx, int ny, int nz, void* ws,
                             int* err, cudaStream_t st) {
  if (d->dtype == CLAMP_DENOISER_BF16) {
    switch (d->channels) {
      case 16: return apply_tc_c<TC_BF16, 16>(d, in, out, nx, ny, nz, ws, err, st);
      case 32: return apply_tc_c<TC_BF16, 32>(d, in, out, nx, ny, nz, ws, err, st);
      case 48: return apply_tc_c<TC_BF16, 48>(d, in, out, nx, ny, nz, ws, err, st);
      case 64: return apply_tc_c<TC_BF16, 64>(d, in, out, nx, ny, nz, ws, err, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (d->channels) {
    case 16: return apply_tc_c<TC_TF32X3, 16>(d, in, out, nx, ny, nz, ws, err, st);
    case 32: return apply_tc_c<TC_TF32X3, 32>(d, in, out, nx, ny, nz, ws, err, st);
    case 48: return apply_tc_c<TC_TF32X3, 48>(d, in, out, nx, ny, nz, ws, err, st);
    default: return cudaErrorInvalidValue;
  }
}

// Packs layer weights W[cout][cin][27] (float, tap = 9 dz + 3 dy + dx) for the
// tensor-core kernels: per chunk of input channels [dz][dx][2 channel groups]
// [dy = 2, 1, 0][npad][epv].  BF16: BF16 (RNE), epv = 8.  TF32x3: hi copy then lo copy,
// FP32, epv = 4.  Output channels >= cout are zero.
std::vector<uint8_t> pack_last_tc_weights(const float* W, int cin) {
  std::vector<uint8_t> p((size_t)cin * 64, 0);
  uint16_t* h = reinterpret_cast<uint16_t*>(p.data());
  for (int c = 0; c < cin; ++c)
    for (int tap = 0; tap < 27; ++tap) h[((c / 8) * 512 + tap * 16 + (c % 8) * 2) / 2] = bf16_bits(W[c * 27 + tap]);
  return p;
}

std::vector<uint8_t> pack_first_tc_weights(const float* W, int cout) {
  std::vector<uint8_t> p((size_t)cout * 64, 0);
  uint16_t* h = reinterpret_cast<uint16_t*>(p.data());
  for (int co = 0; co < cout; ++co)
    for (int k = 0; k < 27; ++k)
      h[((co / 8) * 512 + (k / 8) * 128 + (co % 8) * 16 + (k % 8) * 2) / 2] = bf16_bits(W[co * 27 + k]);
  return p;
}

std::vector<uint8_t> pack_tc_weights(const float* W, int cin, int cout, int npad, bool bf16) {
  const int epv = bf16 ? 8 : 4, ch = 2 * epv, chunks = cin / ch;
  const size_t per = (size_t)chunks * 27 * 2 * npad * epv;  // elements per copy
  std::vector<uint8_t> p(bf16 ? per * 2 : per * 8, 0);
  for (int c = 0; c < chunks; ++c)
    for (int tap = 0; tap < 27; ++tap)
      for (int cg = 0; cg < 2; ++cg)
        for (int co = 0; co < cout; ++co)
          for (int e = 0; e < epv; ++e) {
            const int ci = ch * c + epv * cg + e;
            const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
            const size_t blk = ((size_t)c * 9 + dz * 3 + dx) * 2 + cg;
            const size_t dst = ((blk * 3 + (2 - dy)) * npad + co) * epv + e;
            const float w = W[((size_t)co * cin + ci) * 27 + tap];
            if (bf16) {
              reinterpret_cast<uint16_t*>(p.data())[dst] = bf16_bits(w);
            } else {
              const float h = tf32_rn_host(w);
              reinterpret_cast<float*>(p.data())[dst] = h;
              reinterpret_cast<float*>(p.data())[per + dst] = tf32_rn_host(w - h);
            }
          }
  return p;
}

cudaError_t bounds_site_tc(unsigned int* site, bool reset) { return bounds_site_local(site, reset); }

}  // namespace clamp

extern "C" clamp_status clamp_tc_gemm_bf16(int32_t n, int32_t k, const void* a, const void* b, float* d,
                                           void* stream) {
  if (n < 16 || n > 256 || n % 16 || k < 16 || k > 256 || k % 16 || !a || !b || !d) return CLAMP_EINVAL;
  const size_t smem = 1024 + (size_t)k * 128 * 2 + (size_t)k * n * 2 + 64;
  auto kern = clamp::k_tc_gemm<clamp::TC_BF16>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return CLAMP_ECUDA;
  kern<<<1, 128, smem, (cudaStream_t)stream>>>(a, b, d, n, k);
  return cudaGetLastError() == cudaSuccess ? CLAMP_OK : CLAMP_ECUDA;
}

extern "C" clamp_status clamp_tc_gemm_tf32x3(int32_t n, int32_t k, const float* a, const float* b, float* d,
                                             void* stream) {
  if (n < 16 || n > 256 || n % 16 || k < 8 || k > 192 || k % 8 || !a || !b || !d) return CLAMP_EINVAL;
  const size_t smem = 1024 + 2 * ((size_t)k * 128 * 4 + (size_t)k * n * 4) + 64;
  if (smem > 227 * 1024) return CLAMP_EINVAL;
  auto kern = clamp::k_tc_gemm<clamp::TC_TF32X3>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return CLAMP_ECUDA;
  kern<<<1, 128, smem, (cudaStream_t)stream>>>(a, b, d, n, k);
  return cudaGetLastError() == cudaSuccess ? CLAMP_OK : CLAMP_ECUDA;
}

extern "C" clamp_status clamp_selftest_bounded_wait(int32_t limit, int32_t* result) {
  if (!result || limit < 1 || limit > (1 << 20)) return CLAMP_EINVAL;
  int* d = nullptr;
  if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) return CLAMP_ENOMEM;
  cudaError_t e = cudaMemset(d, 0xff, 2 * sizeof(int));
  if (e == cudaSuccess) {
    clamp::k_wait_selftest<<<1, 32>>>((uint32_t)limit, d);
    e = cudaGetLastError();
  }
  int h[2] = {-1, -1};
  if (e == cudaSuccess) e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return CLAMP_ECUDA;
  result[0] = h[0];
  result[1] = h[1];
  return CLAMP_OK;
}
