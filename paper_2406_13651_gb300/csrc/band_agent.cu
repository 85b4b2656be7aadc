// band_agent.cu -- the forward agents' gradient on the aperture's support only.
//
// The gradient direction of Eq. (h-gradient) splits as
//     d = F^H [ a (y - a M) ] / sigma_w^2 - D mu,      M = F mu,
// because F^H F = I.  The bracket is zero wherever the aperture a is, so only the
// support of the lateral pupil (about 10 % of the (ky, kx) columns at a radius of 0.35
// Nyquist) ever needs the z and y transforms, and the x transform of a row only needs
// the band of kx columns the pupil touches.  The step size of Eq. (mu-update) needs
// ||A d||^2 = ||a F d||^2, again on the support only, and the next iteration's spectrum
// is M + gamma F d (F is linear), so F mu itself is formed once per call.
//
// Per look and iteration (state mu, r' in HBM; spectra on the support S = {(ky, kx):
// pupil != 0}, enumerated row by row; the band B = {kx: some pupil(ky, kx) != 0}):
//   P1 z pass on S   : M += gamma_prev F d_prev;  G = a (y - a M) / sigma_w^2;
//                      S4 = ||a y||^2;  inverse z-FFT of G              -> Gz [kz->z][S]
//   P2 y pass on B   : inverse y-FFT of Gz (zero off S)                 -> E  [z][y][B]
//   P3 x pass, rows  : e = inverse x-FFT of E (zero off B);  d = e - D mu -> d [z][y][x];
//                      S1 = ||d||^2, S3 = sum D |d|^2;  forward x-FFT of d, kept on B
//   P4 y pass on B   : forward y-FFT, kept on S                         -> [z][S]
//   P5 z pass on S   : forward z-FFT -> F d on S;  S2 = ||a F d||^2
// then gamma = S1 / (S2 / sigma_w^2 + S3) and the elementwise pass C.  Only P3 touches
// every voxel: it reads mu, r' and writes d, plus two band rows.
#include "clamp_kernels.cuh"
#include "fft_core.cuh"

#include <math.h>

#include <type_traits>

#include <vector>

namespace clamp {
namespace {

extern __shared__ float4 band_smem[];

constexpr int BC = 16;   // support / band columns per CTA in the y and z passes

__device__ __forceinline__ float warp_sum_b(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 per thread and warp, FP64 across warps in fixed order; writes out[k][idx].
template <int NV>
__device__ __forceinline__ void block_sums(const float (&v)[NV], double* const (&out)[NV], long long idx) {
  __shared__ double red[NT / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const float s = warp_sum_b(v[k]);
    if (lane == 0) red[warp][k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double acc = 0.0;
    for (int w = 0; w < NT / 32; ++w) acc += red[w][threadIdx.x];
    out[threadIdx.x][idx] = acc;
  }
}

// ---------------------------------------------------------------- support tables

// One CTA builds the tables of the support and the band from the pupil, in the order the
// host counted them (row by row, kx ascending; band columns by ascending kx).
__global__ void __launch_bounds__(1024) k_band_tables(const float* __restrict__ pupil, int nx, int ny, BandTables t) {
  __shared__ int s_bpos[256];
  __shared__ int s_rowcnt[256];
  __shared__ int s_rowstart[256];
  const int tid = threadIdx.x;
  if (tid < nx) {
    int any = 0;
    for (int ky = 0; ky < ny; ++ky) any |= pupil[ky * nx + tid] != 0.0f;
    s_bpos[tid] = any;
  }
  if (tid < ny) {
    int c = 0;
    for (int kx = 0; kx < nx; ++kx) c += pupil[tid * nx + kx] != 0.0f;
    s_rowcnt[tid] = c;
  }
  __syncthreads();
  if (tid == 0) {
    int b = 0;
    for (int kx = 0; kx < nx; ++kx) {
      if (s_bpos[kx]) {
        t.bx[b] = kx;
        s_bpos[kx] = b++;
      } else {
        s_bpos[kx] = -1;
      }
    }
    for (; b < t.nbxp; ++b) t.bx[b] = -1;
    int s = 0;
    for (int ky = 0; ky < ny; ++ky) {
      s_rowstart[ky] = s;
      s += s_rowcnt[ky];
    }
  }
  __syncthreads();
  if (tid < nx) t.bpos[tid] = s_bpos[tid];
  if (tid < ny) {
    int* row = t.sidx + (long long)tid * t.nbxp;
    for (int b = 0; b < t.nbxp; ++b) row[b] = -1;
    int s = s_rowstart[tid];
    for (int kx = 0; kx < nx; ++kx) {
      const float pv = pupil[tid * nx + kx];
      if (pv != 0.0f) {
        t.s_kykx[s] = tid * nx + kx;
        t.s_pup[s] = pv;
        row[s_bpos[kx]] = s;
        ++s;
      }
    }
  }
  __syncthreads();
  for (int s = t.nS + tid; s < t.nSp; s += blockDim.x) {   // padding columns: a = 0
    t.s_kykx[s] = 0;
    t.s_pup[s] = 0.0f;
  }
}

// ---------------------------------------------------------------- P1: z pass on the support (inverse)

template <int N>
__global__ void __launch_bounds__(NT) k_band_z_inv(BandArgs a, const float2* __restrict__ tw) {
  [[maybe_unused]] const long long nL = (long long)a.L * a.n, sL = (long long)a.L * a.nz * a.t.nSp,
                                   bL = (long long)a.L * a.nz * a.ny * a.t.nbxp;   // buffer extents
  constexpr int LD = N + 1, CNT = BC * N, PER = (CNT + NT - 1) / NT;
  float2* sm = reinterpret_cast<float2*>(band_smem);
  const int s0 = blockIdx.x * BC, l = blockIdx.y;
  const long long cbase = (long long)l * N * a.t.nSp + s0;   // compact [l][kz][s]
  const long long ybase = (long long)l * a.n;
  const float gp = a.gamma_prev ? __ldg(&a.gamma_prev[l]) : 0.0f;
  float2 mv[PER], fv[PER], yv[PER];
  float av[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int col = e % BC, kz = e / BC;
      const long long ci = cbase + (long long)kz * a.t.nSp + col;
      const int s = s0 + col;
      const bool valid = s < a.t.nS;   // padding columns hold stale values: read as zero
      mv[p] = valid && CLAMP_IN_BOUNDS(ci, sL, 101) ? a.Ms[ci] : make_float2(0.f, 0.f);
      fv[p] = (valid && a.gamma_prev && CLAMP_IN_BOUNDS(ci, sL, 102)) ? a.Fd[ci] : make_float2(0.f, 0.f);
      av[p] = __ldg(&a.t.s_pup[s]) * __ldg(&a.window[kz]);
      const long long yi = ybase + (long long)kz * a.plane + __ldg(&a.t.s_kykx[s]);
      yv[p] = CLAMP_IN_BOUNDS(yi, nL, 103) ? a.y[yi] : make_float2(0.f, 0.f);
    }
  }
  float acc[1] = {0.f};
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int col = e % BC, kz = e / BC;
      float2 M = mv[p];
      if (a.gamma_prev && s0 + col < a.t.nS) {   // the previous step's spectrum update M += gamma F d
        M.x = fmaf(gp, fv[p].x, M.x);
        M.y = fmaf(gp, fv[p].y, M.y);
        const long long mi = cbase + (long long)kz * a.t.nSp + col;
        if (CLAMP_IN_BOUNDS(mi, sL, 104)) a.Ms[mi] = M;
      }
      const float f = av[p] * a.inv_nv;
      sm[col * LD + kz] = make_float2(f * fmaf(-av[p], M.x, yv[p].x), f * fmaf(-av[p], M.y, yv[p].y));
      acc[0] += av[p] * av[p] * cabs2(yv[p]);
    }
  }
  __syncthreads();
  fft_tile<N, BC, NT, true>(sm, tw);
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int col = e % BC, z = e / BC;
      const long long fi = cbase + (long long)z * a.t.nSp + col;
      if (CLAMP_IN_BOUNDS(fi, sL, 105)) a.Fd[fi] = cscale(sm[col * LD + z], a.sc_z);   // Gz, in place
    }
  }
  double* const outs[1] = {a.s4};
  block_sums<1>(acc, outs, (long long)l * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------- P2 / P4: y passes on the band

// INV: Gz on the support -> E on the band (zero off the support).  !INV: band -> support.
template <int N, bool INV>
__global__ void __launch_bounds__(NT) k_band_y(BandArgs a, const float2* __restrict__ tw) {
  [[maybe_unused]] const long long nL = (long long)a.L * a.n, sL = (long long)a.L * a.nz * a.t.nSp,
                                   bL = (long long)a.L * a.nz * a.ny * a.t.nbxp;   // buffer extents
  constexpr int LD = N + 1, CNT = BC * N, PER = (CNT + NT - 1) / NT;
  float2* sm = reinterpret_cast<float2*>(band_smem);
  const int b0 = blockIdx.x * BC, z = blockIdx.y, l = blockIdx.z;
  const long long cplane = ((long long)l * a.nz + z) * a.t.nSp;             // compact [l][z][s]
  const long long bbase = (((long long)l * a.nz + z) * N) * a.t.nbxp + b0;  // band [l][z][y][b]
  float2 iv[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int col = e % BC, yi = e / BC;
      if constexpr (INV) {
        const int s = __ldg(&a.t.sidx[yi * a.t.nbxp + b0 + col]);
        iv[p] = s >= 0 && CLAMP_IN_BOUNDS(cplane + s, sL, 111) ? a.Fd[cplane + s] : make_float2(0.f, 0.f);
      } else {
        const long long bi = bbase + (long long)yi * a.t.nbxp + col;
        iv[p] = CLAMP_IN_BOUNDS(bi, bL, 112) ? a.band[bi] : make_float2(0.f, 0.f);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) sm[(e % BC) * LD + e / BC] = iv[p];
  }
  __syncthreads();
  fft_tile<N, BC, NT, INV>(sm, tw);
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int col = e % BC, yi = e / BC;
      const float2 v = cscale(sm[col * LD + yi], a.sc_y);
      if constexpr (INV) {
        const long long bi = bbase + (long long)yi * a.t.nbxp + col;
        if (CLAMP_IN_BOUNDS(bi, bL, 113)) a.band[bi] = v;
      } else {
        const int s = __ldg(&a.t.sidx[yi * a.t.nbxp + b0 + col]);
        if (s >= 0 && CLAMP_IN_BOUNDS(cplane + s, sL, 114)) a.Fd[cplane + s] = v;
      }
    }
  }
}

// ---------------------------------------------------------------- P3: x pass over whole rows

enum BandRowMode { BAND_GRAD = 0, BAND_SPEC = 1 };

// BAND_GRAD: e = inverse x-FFT of the band row, d = e - D mu (written), S1/S3, forward x-FFT
// of d kept on the band.  BAND_SPEC: forward x-FFT of mu kept on the band (F mu's first axis).
// Launch variant V = 0: rows_per_cta(N) rows per CTA, two CTAs per SM (at most 128
// registers: with no occupancy bound the compiler takes about 180 and one CTA runs per SM,
// 0.5 ms slower per iteration at 256x256x128, L = 32); V = 1: half as many rows, so a
// thread holds half the prefetched values and three CTAs share an SM (at N = 256 with the
// 8 x 8 x 4 radix plan, whose stages keep all threads of an 8-row tile busy); V = 2: the
// tile of V = 0 with mu and r' not held in registers across the inverse transform: the CTA
// first prefetches their lines into L2 (no registers held) and reads them after the
// transform, so three CTAs share an SM.
template <int N, int MODE, int V>
__global__ void __launch_bounds__(NT, V == 0 ? 2 : 3) k_band_x(BandArgs a, const float2* __restrict__ tw) {
  [[maybe_unused]] const long long nL = (long long)a.L * a.n, sL = (long long)a.L * a.nz * a.t.nSp,
                                   bL = (long long)a.L * a.nz * a.ny * a.t.nbxp;   // buffer extents
  constexpr int LX = V == 1 ? variant_rows(N, 2) : rows_per_cta(N), LD = N + 1, CNT = LX * N,
                PER = (CNT + NT - 1) / NT;
  constexpr bool LATE = V == 2 && MODE == BAND_GRAD;   // mu, r' read after the inverse transform
  using PL = std::conditional_t<V == 1 && N == 256, PlanB<N>, Plan<N>>;
  float2* sm = reinterpret_cast<float2*>(band_smem);
  const long long row0 = (long long)blockIdx.x * LX;   // rows over [L][nz][ny]
  const long long e0 = row0 * N;
  float2 mv[LATE ? 1 : PER], ev[PER];
  float rv[LATE ? 1 : PER];
  if constexpr (LATE) {   // 128-byte lines of the tile's mu (8 B per element) and r' (4 B)
    static_assert(CNT % 32 == 0, "tile");
    for (int i = threadIdx.x; i < CNT / 16; i += NT)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.mu + e0 + 16 * i));
    for (int i = threadIdx.x; i < CNT / 32; i += NT)
      asm volatile("prefetch.global.L2 [%0];" ::"l"(a.rprev + e0 + 32 * i));
  }
  // with NT a multiple of N every element a thread touches is in the same column
  constexpr bool FIXED_COL = NT % N == 0;
  const int b_fixed = FIXED_COL && MODE == BAND_GRAD ? __ldg(&a.t.bpos[threadIdx.x % N]) : -1;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      if constexpr (!LATE) mv[p] = CLAMP_IN_BOUNDS(e0 + e, nL, 121) ? a.mu[e0 + e] : make_float2(0.f, 0.f);
      if constexpr (MODE == BAND_GRAD) {
        if constexpr (!LATE) rv[p] = CLAMP_IN_BOUNDS(e0 + e, nL, 122) ? a.rprev[e0 + e] : 1.0f;
        const int line = e / N, i = e - line * N;
        const int b = FIXED_COL ? b_fixed : __ldg(&a.t.bpos[i]);
        ev[p] = b >= 0 && CLAMP_IN_BOUNDS((row0 + line) * a.t.nbxp + b, bL, 123) ? a.band[(row0 + line) * a.t.nbxp + b]
                                                                               : make_float2(0.f, 0.f);
      }
    }
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e / N, i = e - line * N;
      sm[line * LD + i] = MODE == BAND_GRAD ? ev[p] : mv[LATE ? 0 : p];
    }
  }
  __syncthreads();
  float acc[2] = {0.f, 0.f};
  if constexpr (MODE == BAND_GRAD) {
    fft_tile<N, LX, NT, true, PL>(sm, tw);
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = threadIdx.x + p * NT;
      if (CNT % NT == 0 || e < CNT) {
        const int line = e / N, i = e - line * N;
        const float2 ee = cscale(sm[line * LD + i], a.sc_x);
        const bool ok = !LATE || CLAMP_IN_BOUNDS(e0 + e, nL, 124);
        const float2 m = LATE ? (ok ? a.mu[e0 + e] : make_float2(0.f, 0.f)) : mv[LATE ? 0 : p];
        const float D = __frcp_rn((LATE ? (ok ? a.rprev[e0 + e] : 1.0f) : rv[LATE ? 0 : p]) + a.floor);
        const float2 dv = make_float2(fmaf(-D, m.x, ee.x), fmaf(-D, m.y, ee.y));
        if (CLAMP_IN_BOUNDS(e0 + e, nL, 126)) a.d[e0 + e] = dv;
        const float d2 = cabs2(dv);
        acc[0] += d2;
        acc[1] += D * d2;
        sm[line * LD + i] = dv;
      }
    }
    __syncthreads();
  }
  fft_tile<N, LX, NT, false, PL>(sm, tw);
  // band of the forward transform: LX rows x nbxp columns (padding columns get zeros)
  // (a warp per row at a time, lanes over the band columns: no division by nbxp)
  const int nbxp = a.t.nbxp;
  for (int line = threadIdx.x >> 5; line < LX; line += NT / 32) {
    float2* brow = a.band + (row0 + line) * nbxp;
    for (int b = threadIdx.x & 31; b < nbxp; b += 32) {
      const int kx = __ldg(&a.t.bx[b]);
      if (CLAMP_IN_BOUNDS((row0 + line) * nbxp + b, bL, 127))
        brow[b] = kx >= 0 ? cscale(sm[line * LD + kx], a.sc_x) : make_float2(0.f, 0.f);
    }
  }
  if constexpr (MODE == BAND_GRAD) {
    double* const outs[2] = {a.s1, a.s3};
    const long long rows_per_look = (long long)a.nz * a.ny;
    const long long look = row0 / rows_per_look;
    block_sums<2>(acc, outs, look * a.px + (row0 - look * rows_per_look) / LX);
  }
}

// ---------------------------------------------------------------- P5: z pass on the support (forward)

// BAND_GRAD: F d on the support (in place) and S2 = ||a F d||^2.  BAND_SPEC: writes M.
template <int N, int MODE>
__global__ void __launch_bounds__(NT) k_band_z_fwd(BandArgs a, const float2* __restrict__ tw) {
  [[maybe_unused]] const long long nL = (long long)a.L * a.n, sL = (long long)a.L * a.nz * a.t.nSp,
                                   bL = (long long)a.L * a.nz * a.ny * a.t.nbxp;   // buffer extents
  constexpr int LD = N + 1, CNT = BC * N, PER = (CNT + NT - 1) / NT;
  float2* sm = reinterpret_cast<float2*>(band_smem);
  const int s0 = blockIdx.x * BC, l = blockIdx.y;
  const long long cbase = (long long)l * N * a.t.nSp + s0;
  float2 iv[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const long long fi = cbase + (long long)(e / BC) * a.t.nSp + e % BC;
      iv[p] = s0 + e % BC < a.t.nS && CLAMP_IN_BOUNDS(fi, sL, 131) ? a.Fd[fi] : make_float2(0.f, 0.f);
    }
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) sm[(e % BC) * LD + e / BC] = iv[p];
  }
  __syncthreads();
  fft_tile<N, BC, NT, false>(sm, tw);
  float acc[1] = {0.f};
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int col = e % BC, kz = e / BC;
      const float2 v = cscale(sm[col * LD + kz], a.sc_z);
      const long long ci = cbase + (long long)kz * a.t.nSp + col;
      if constexpr (MODE == BAND_GRAD) {
        if (CLAMP_IN_BOUNDS(ci, sL, 132)) a.Fd[ci] = v;
        const float av = __ldg(&a.t.s_pup[s0 + col]) * __ldg(&a.window[kz]);
        acc[0] += av * av * cabs2(v);
      } else {
        if (CLAMP_IN_BOUNDS(ci, sL, 133)) a.Ms[ci] = v;
      }
    }
  }
  if constexpr (MODE == BAND_GRAD) {
    double* const outs[1] = {a.s2};
    block_sums<1>(acc, outs, (long long)l * gridDim.x + blockIdx.x);
  }
}

// gamma_l = S1 / (S2 / sigma_w^2 + S3) and the floored mu-residual sqrt(S1) / (sqrt(S4) / sigma_w^2).
__global__ void __launch_bounds__(NT) k_band_gamma(BandArgs a, int pS, float nv, float* gamma, double* mures) {
  const int l = blockIdx.x;
  __shared__ double red[NT][4];
  double v1 = 0, v2 = 0, v3 = 0, v4 = 0;
  for (int i = threadIdx.x; i < a.px; i += NT) {
    v1 += a.s1[(long long)l * a.px + i];
    v3 += a.s3[(long long)l * a.px + i];
  }
  for (int i = threadIdx.x; i < pS; i += NT) {
    v2 += a.s2[(long long)l * pS + i];
    v4 += a.s4[(long long)l * pS + i];
  }
  red[threadIdx.x][0] = v1;
  red[threadIdx.x][1] = v2;
  red[threadIdx.x][2] = v3;
  red[threadIdx.x][3] = v4;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o)
      for (int k = 0; k < 4; ++k) red[threadIdx.x][k] += red[threadIdx.x + o][k];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double S1 = red[0][0], S2 = red[0][1], S3 = red[0][2], S4 = red[0][3];
    const double den = S2 / (double)nv + S3;
    gamma[l] = den > 0 ? (float)(S1 / den) : 0.0f;
    mures[l] = S4 > 0 ? sqrt(S1) / (sqrt(S4) / (double)nv) : 0.0;
  }
}

template <class F>
cudaError_t dispatch_n(int N, F&& f) {
  switch (N) {
    case 8: return f(std::integral_constant<int, 8>{});
    case 16: return f(std::integral_constant<int, 16>{});
    case 32: return f(std::integral_constant<int, 32>{});
    case 64: return f(std::integral_constant<int, 64>{});
    case 96: return f(std::integral_constant<int, 96>{});
    case 128: return f(std::integral_constant<int, 128>{});
    case 192: return f(std::integral_constant<int, 192>{});
    case 256: return f(std::integral_constant<int, 256>{});
    default: return cudaErrorInvalidValue;
  }
}

#define BAND_TRY(x)                   \
  do {                                \
    cudaError_t _e = (x);             \
    if (_e != cudaSuccess) return _e; \
  } while (0)

template <class K>
cudaError_t smem_attr(K kern, size_t smem) {
  return cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

cudaError_t run_z(const BandArgs& a, int L, bool inverse, int mode, cudaStream_t st) {
  return dispatch_n(a.nz, [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    const size_t smem = (size_t)BC * (N + 1) * sizeof(float2);
    const dim3 grid(a.t.nSp / BC, L);
    if (inverse) {
      BAND_TRY(smem_attr(k_band_z_inv<N>, smem));
      k_band_z_inv<N><<<grid, NT, smem, st>>>(a, twiddle_table(N));
    } else if (mode == BAND_GRAD) {
      BAND_TRY(smem_attr(k_band_z_fwd<N, BAND_GRAD>, smem));
      k_band_z_fwd<N, BAND_GRAD><<<grid, NT, smem, st>>>(a, twiddle_table(N));
    } else {
      BAND_TRY(smem_attr(k_band_z_fwd<N, BAND_SPEC>, smem));
      k_band_z_fwd<N, BAND_SPEC><<<grid, NT, smem, st>>>(a, twiddle_table(N));
    }
    return cudaGetLastError();
  });
}

cudaError_t run_y(const BandArgs& a, int L, bool inverse, cudaStream_t st) {
  return dispatch_n(a.ny, [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    const size_t smem = (size_t)BC * (N + 1) * sizeof(float2);
    const dim3 grid(a.t.nbxp / BC, a.nz, L);
    if (inverse) {
      BAND_TRY(smem_attr(k_band_y<N, true>, smem));
      k_band_y<N, true><<<grid, NT, smem, st>>>(a, twiddle_table(N));
    } else {
      BAND_TRY(smem_attr(k_band_y<N, false>, smem));
      k_band_y<N, false><<<grid, NT, smem, st>>>(a, twiddle_table(N));
    }
    return cudaGetLastError();
  });
}

cudaError_t run_x(const BandArgs& a, int L, int mode, int variant, cudaStream_t st) {
  return dispatch_n(a.nx, [&](auto NC) -> cudaError_t {
    constexpr int N = decltype(NC)::value;
    if (mode == BAND_GRAD && variant == 1) {
      constexpr int LX = variant_rows(N, 2);
      const size_t smem = (size_t)LX * (N + 1) * sizeof(float2);
      BAND_TRY(smem_attr(k_band_x<N, BAND_GRAD, 1>, smem));
      k_band_x<N, BAND_GRAD, 1><<<(unsigned)((long long)L * a.nz * a.ny / LX), NT, smem, st>>>(a, twiddle_table(N));
      return cudaGetLastError();
    }
    if (mode == BAND_GRAD && variant == 2) {
      constexpr int LX = rows_per_cta(N);
      const size_t smem = (size_t)LX * (N + 1) * sizeof(float2);
      BAND_TRY(smem_attr(k_band_x<N, BAND_GRAD, 2>, smem));
      k_band_x<N, BAND_GRAD, 2><<<(unsigned)((long long)L * a.nz * a.ny / LX), NT, smem, st>>>(a, twiddle_table(N));
      return cudaGetLastError();
    }
    constexpr int LX = rows_per_cta(N);
    const size_t smem = (size_t)LX * (N + 1) * sizeof(float2);
    const unsigned grid = (unsigned)((long long)L * a.nz * a.ny / LX);
    if (mode == BAND_GRAD) {
      BAND_TRY(smem_attr(k_band_x<N, BAND_GRAD, 0>, smem));
      k_band_x<N, BAND_GRAD, 0><<<grid, NT, smem, st>>>(a, twiddle_table(N));
    } else {
      BAND_TRY(smem_attr(k_band_x<N, BAND_SPEC, 0>, smem));
      k_band_x<N, BAND_SPEC, 0><<<grid, NT, smem, st>>>(a, twiddle_table(N));
    }
    return cudaGetLastError();
  });
}

}  // namespace

BandShape band_shape(const float* pupil_host, int nx, int ny) {
  BandShape b{};
  int nS = 0, nbx = 0;
  for (int kx = 0; kx < nx; ++kx) {
    bool any = false;
    for (int ky = 0; ky < ny; ++ky) {
      const bool nz = pupil_host[ky * nx + kx] != 0.0f;
      any |= nz;
      nS += nz;
    }
    nbx += any;
  }
  b.nS = nS;
  b.nSp = (nS + BC - 1) / BC * BC;
  b.nbx = nbx;
  b.nbxp = (nbx + BC - 1) / BC * BC;
  return b;
}

size_t band_table_bytes(const BandShape& b, int nx, int ny) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  return al(sizeof(int) * (size_t)ny * b.nbxp) + al(sizeof(int) * (size_t)b.nSp) + al(sizeof(float) * (size_t)b.nSp) +
         al(sizeof(int) * (size_t)b.nbxp) + al(sizeof(int) * (size_t)nx);
}

BandTables band_tables_at(const BandShape& b, int nx, int ny, void* base) {
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  char* p = static_cast<char*>(base);
  BandTables t{};
  t.nS = b.nS;
  t.nSp = b.nSp;
  t.nbx = b.nbx;
  t.nbxp = b.nbxp;
  t.sidx = reinterpret_cast<int*>(p);
  p += al(sizeof(int) * (size_t)ny * b.nbxp);
  t.s_kykx = reinterpret_cast<int*>(p);
  p += al(sizeof(int) * (size_t)b.nSp);
  t.s_pup = reinterpret_cast<float*>(p);
  p += al(sizeof(float) * (size_t)b.nSp);
  t.bx = reinterpret_cast<int*>(p);
  p += al(sizeof(int) * (size_t)b.nbxp);
  t.bpos = reinterpret_cast<int*>(p);
  return t;
}

int band_pS(const BandShape& b) { return b.nSp / BC; }
int band_px(int nx, int ny, int nz, int x_variant) {
  return (int)((long long)nz * ny / (x_variant == 1 ? variant_rows(nx, 2) : rows_per_cta(nx)));
}

cudaError_t launch_band_tables(const float* pupil, int nx, int ny, const BandTables& t, cudaStream_t st) {
  k_band_tables<<<1, 1024, 0, st>>>(pupil, nx, ny, t);
  return cudaGetLastError();
}

cudaError_t launch_band_spectrum(const BandArgs& a0, int L, cudaStream_t st) {
  BandArgs a = a0;
  a.L = L;
  BAND_TRY(run_x(a, L, BAND_SPEC, 0, st));
  BAND_TRY(run_y(a, L, false, st));
  return run_z(a, L, false, BAND_SPEC, st);
}

cudaError_t launch_band_agent(const BandArgs& a, int L, float nv, float* gamma, double* mures, int x_variant,
                              cudaStream_t st) {
  BandArgs b = a;
  b.L = L;
  b.px = band_px(a.nx, a.ny, a.nz, x_variant);
  BAND_TRY(run_z(b, L, true, BAND_GRAD, st));
  BAND_TRY(run_y(b, L, true, st));
  BAND_TRY(run_x(b, L, BAND_GRAD, x_variant, st));
  BAND_TRY(run_y(b, L, false, st));
  BAND_TRY(run_z(b, L, false, BAND_GRAD, st));
  k_band_gamma<<<L, NT, 0, st>>>(b, band_pS(BandShape{a.t.nS, a.t.nSp, a.t.nbx, a.t.nbxp}), nv, gamma, mures);
  return cudaGetLastError();
}

cudaError_t bounds_site_band(unsigned int* site, bool reset) { return bounds_site_local(site, reset); }

}  // namespace clamp
