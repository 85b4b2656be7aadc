// fft_core.cuh -- shared-memory staged FFT building blocks for sm_103a.
//
// A CTA holds a tile of LT lines x N points in shared memory, laid out
// s[line * (N + 1) + i].  The odd line stride makes every access in which the
// line index varies fastest across a half-warp conflict-free, whatever the
// point index pattern, so all radix stages use a (line fast, butterfly slow)
// thread mapping.  Each stage is a Stockham autosort radix-R pass: thread j
// takes R points spaced N/R apart, applies the stage twiddles, does an
// in-register R-point DFT and writes them Ns apart (Ns = product of earlier
// radices); the output is in natural order after the last stage.
//
// Stage twiddles exp(-2 pi i m / N) come from a table computed on the host in
// double precision (libm) and rounded once to float; the in-register DFT uses
// the exact constants cos(pi/4) and cos/sin(pi/8).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

namespace clamp {

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
__device__ __forceinline__ float2 cscale(float2 a, float s) { return make_float2(a.x * s, a.y * s); }
__device__ __forceinline__ float cabs2(float2 a) { return fmaf(a.x, a.x, a.y * a.y); }

// Multiply by W16^m = exp(-+ 2 pi i m / 16) for compile-time m in [0, 8) (after unrolling).
template <bool INV>
__device__ __forceinline__ float2 w16mul(float2 x, int m) {
  constexpr float C1 = 0.92387953251128674f;  // cos(pi/8)
  constexpr float S1 = 0.38268343236508977f;  // sin(pi/8)
  constexpr float C2 = 0.70710678118654752f;  // cos(pi/4)
  float c, s;  // W = c - i s (forward), c + i s (inverse)
  switch (m) {
    case 0: return x;
    case 4: return INV ? make_float2(-x.y, x.x) : make_float2(x.y, -x.x);
    case 1: c = C1; s = S1; break;
    case 2: c = C2; s = C2; break;
    case 3: c = S1; s = C1; break;
    case 5: c = -S1; s = C1; break;
    case 6: c = -C2; s = C2; break;
    default: c = -C1; s = S1; break;  // m = 7
  }
  if (INV) s = -s;
  return make_float2(fmaf(x.x, c, x.y * s), fmaf(x.y, c, -x.x * s));
}

template <int R>
__device__ __forceinline__ constexpr int bitrev(int i) {
  int r = 0;
  for (int b = 1, t = R >> 1; b < R; b <<= 1, t >>= 1)
    if (i & b) r |= t;
  return r;
}

// v[i] <- v[bitrev(i)], with every index a compile-time constant so the array stays in registers.
template <int R, int... I>
__device__ __forceinline__ void bitrev_permute(float2 (&v)[R], std::integer_sequence<int, I...>) {
  const float2 t[R] = {v[std::integral_constant<int, bitrev<R>(I)>::value]...};
  ((v[I] = t[I]), ...);
}

// Radix-2 decimation-in-time butterfly levels LEN, 2 LEN, ..., R on bit-reversed input.
// Compile-time recursion over the level keeps every index constant, so the array stays
// in registers.
template <int R, bool INV, int LEN>
__device__ __forceinline__ void dit_stages(float2 (&v)[R]) {
  if constexpr (LEN <= R) {
#pragma unroll
    for (int i = 0; i < R / LEN; ++i) {
#pragma unroll
      for (int k = 0; k < LEN / 2; ++k) {
        const float2 t = w16mul<INV>(v[i * LEN + k + LEN / 2], k * (16 / LEN));
        v[i * LEN + k + LEN / 2] = csub(v[i * LEN + k], t);
        v[i * LEN + k] = cadd(v[i * LEN + k], t);
      }
    }
    dit_stages<R, INV, 2 * LEN>(v);
  }
}

// In-place R-point DFT in registers, natural order in and out.
// Forward: V[s] = sum_r v[r] exp(-2 pi i r s / R); inverse uses +.
template <int R, bool INV>
__device__ __forceinline__ void dft(float2 (&v)[R]) {
  if constexpr (R == 1) {
    return;
  } else if constexpr (R == 3) {
    constexpr float H = 0.86602540378443865f;  // sin(2 pi / 3)
    float2 s = cadd(v[1], v[2]);
    float2 d = csub(v[1], v[2]);
    float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
    // forward: -i * H * d ; inverse: +i * H * d
    float2 t = INV ? make_float2(-H * d.y, H * d.x) : make_float2(H * d.y, -H * d.x);
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, t);
    v[2] = csub(m, t);
  } else {
    static_assert(R == 2 || R == 4 || R == 8 || R == 16, "radix");
    bitrev_permute(v, std::make_integer_sequence<int, R>{});
    dit_stages<R, INV, 2>(v);
  }
}

// Radix plans: N = R1 * R2 (* R3).  R1 is applied first.
template <int N> struct Plan;
template <> struct Plan<8>   { static constexpr int R1 = 4,  R2 = 2,  R3 = 1; };
template <> struct Plan<16>  { static constexpr int R1 = 4,  R2 = 4,  R3 = 1; };
template <> struct Plan<32>  { static constexpr int R1 = 8,  R2 = 4,  R3 = 1; };
template <> struct Plan<64>  { static constexpr int R1 = 8,  R2 = 8,  R3 = 1; };
template <> struct Plan<128> { static constexpr int R1 = 16, R2 = 8,  R3 = 1; };
template <> struct Plan<256> { static constexpr int R1 = 16, R2 = 16, R3 = 1; };
template <> struct Plan<96>  { static constexpr int R1 = 8,  R2 = 4,  R3 = 3; };
template <> struct Plan<192> { static constexpr int R1 = 16, R2 = 4,  R3 = 3; };

// Alternative radix plans (the autotuner's variant 1).
template <int N> struct PlanB;
template <> struct PlanB<8>   { static constexpr int R1 = 2,  R2 = 4,  R3 = 1; };
template <> struct PlanB<16>  { static constexpr int R1 = 16, R2 = 1,  R3 = 1; };
template <> struct PlanB<32>  { static constexpr int R1 = 4,  R2 = 8,  R3 = 1; };
template <> struct PlanB<64>  { static constexpr int R1 = 16, R2 = 4,  R3 = 1; };
template <> struct PlanB<96>  { static constexpr int R1 = 4,  R2 = 8,  R3 = 3; };
template <> struct PlanB<128> { static constexpr int R1 = 8,  R2 = 16, R3 = 1; };
template <> struct PlanB<192> { static constexpr int R1 = 8,  R2 = 8,  R3 = 3; };
template <> struct PlanB<256> { static constexpr int R1 = 8,  R2 = 8,  R3 = 4; };

// Offset of the length-N twiddle table inside the packed table (N = 8..256 powers of two, 96, 192).
__host__ __device__ constexpr int tw_offset(int N) {
  return N == 8 ? 0 : N == 16 ? 8 : N == 32 ? 24 : N == 64 ? 56 : N == 128 ? 120 : N == 256 ? 248 : N == 96 ? 504 : 600;
}
constexpr int kTwTotal = 792;
constexpr int kFftLengths[] = {8, 16, 32, 64, 96, 128, 192, 256};

// One Stockham stage over all LT lines of the tile.
template <int N, int R, int NS, int LT, int NT, bool INV>
__device__ __forceinline__ void stockham_stage(float2* __restrict__ s, const float2* __restrict__ tw) {
  constexpr int LD = N + 1;
  constexpr int NB = N / R;          // butterflies per line
  constexpr int TOTAL = LT * NB;
  constexpr int PER = (TOTAL + NT - 1) / NT;
  float2 v[PER][R];
  const int t = threadIdx.x;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int idx = t + p * NT;
    if (TOTAL % NT == 0 || idx < TOTAL) {
      const int line = idx % LT;
      const int j = idx / LT;
#pragma unroll
      for (int r = 0; r < R; ++r) v[p][r] = s[line * LD + j + r * NB];
    }
  }
  __syncthreads();
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int idx = t + p * NT;
    if (TOTAL % NT == 0 || idx < TOTAL) {
      const int line = idx % LT;
      const int j = idx / LT;
      const int k = j % NS;
      if constexpr (NS > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const float2 w = __ldg(&tw[r * k * (N / (NS * R))]);
          v[p][r] = INV ? cmulc(v[p][r], w) : cmul(v[p][r], w);
        }
      }
      dft<R, INV>(v[p]);
      const int base = (j / NS) * NS * R + k;
#pragma unroll
      for (int r = 0; r < R; ++r) s[line * LD + base + r * NS] = v[p][r];
    }
  }
  __syncthreads();
}

// Full N-point FFT (unnormalised) of every line of the tile with radix plan P; tw points
// at the length-N table.  Must be called by all NT threads; ends with a barrier.
template <int N, int LT, int NT, bool INV, class P = Plan<N>>
__device__ __forceinline__ void fft_tile(float2* __restrict__ s, const float2* __restrict__ tw) {
  stockham_stage<N, P::R1, 1, LT, NT, INV>(s, tw);
  if constexpr (P::R2 > 1) stockham_stage<N, P::R2, P::R1, LT, NT, INV>(s, tw);
  if constexpr (P::R3 > 1) stockham_stage<N, P::R3, P::R1 * P::R2, LT, NT, INV>(s, tw);
}

}  // namespace clamp
