// clamp_kernels.cu -- CLAMP forward-agent, MACE and set-up passes for sm_103a.
//
// Per look and iteration the forward agent needs F(mu), F(D mu) and F^H of the
// frequency-domain gradient (Eq. h-gradient).  The 3D transforms are split in
// axis passes over HBM, with the agent arithmetic fused into them:
//   A_x : read mu, r'  -> x-FFT of mu and D mu             -> T (float4 per voxel)
//   A_y : T            -> y-FFT of both                    -> T (in place)
//   ABz : T, y, a      -> z-FFT of both; Fd = a(y - aM)/sigma_w^2 - P;
//                         S1 = ||Fd||^2, S2 = ||a Fd||^2, S4 = ||a y||^2;
//                         inverse z-FFT of Fd              -> U
//   B_y : U            -> inverse y-FFT                    -> U (in place)
//   B_x : U, r'        -> inverse x-FFT = d; S3 = sum |d|^2 D -> U holds d
// then gamma = S1 / (S2/sigma_w^2 + S3) (Parseval: ||d|| = ||Fd||, ||Ad|| = ||a Fd||)
// and one elementwise pass C over all looks of a voxel does the mu update,
// the App. A prox and the Mann step.
#include "clamp_kernels.cuh"
#include "fft_core.cuh"

#include <math.h>

#include <type_traits>
#include <vector>

namespace clamp {

__device__ float2 g_tw[kTwTotal];

cudaError_t upload_twiddles() {
  std::vector<float2> h(kTwTotal);
  for (int N : kFftLengths) {
    const int off = tw_offset(N);
    for (int m = 0; m < N; ++m) {
      const double ang = -2.0 * M_PI * (double)m / (double)N;
      h[off + m] = make_float2((float)cos(ang), (float)sin(ang));
    }
  }
  return cudaMemcpyToSymbol(g_tw, h.data(), sizeof(float2) * kTwTotal);
}

static const float2* tw_ptr(int N) {
  void* p = nullptr;
  cudaGetSymbolAddress(&p, g_tw);
  return reinterpret_cast<const float2*>(p) + tw_offset(N);
}

const float2* twiddle_table(int N) { return tw_ptr(N); }

extern __shared__ float4 dyn_smem[];

// ---------------------------------------------------------------- reductions

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-reduces NV float partials (per-thread FP32, warp FP32, across warps FP64
// in fixed order) and writes them to out[k][idx].  All threads must call.
template <int NV>
__device__ __forceinline__ void block_reduce_store(const float (&v)[NV], double* const (&out)[NV], long long idx) {
  __shared__ double red[NT / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    float s = warp_sum(v[k]);
    if (lane == 0) red[warp][k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double acc = 0.0;
    for (int wi = 0; wi < (int)(blockDim.x / 32); ++wi) acc += red[wi][threadIdx.x];
    out[threadIdx.x][idx] = acc;
  }
}

// ---------------------------------------------------------------- pass A_x

template <int N, int V>
__global__ void __launch_bounds__(NT) k_a_x(Geom g, AgentScalars s, const float2* __restrict__ mu,
                                            const float* __restrict__ rprev, float4* __restrict__ T,
                                            const float2* __restrict__ tw) {
  constexpr int LX = variant_rows(N, V), LT = 2 * LX, LD = N + 1;
  using PL = std::conditional_t<V == 1, PlanB<N>, Plan<N>>;
  float2* sm = reinterpret_cast<float2*>(dyn_smem);
  constexpr int CNT = LX * N, PER = (CNT + NT - 1) / NT;
  const long long e0 = (long long)blockIdx.x * LX * N;  // first element of the tile
  // all of a thread's loads are issued before any shared-memory store
  float2 mv[PER];
  float rv[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      mv[p] = mu[e0 + e];
      rv[p] = rprev[e0 + e];
    }
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e / N, i = e - line * N;
      sm[line * LD + i] = mv[p];
      sm[(LX + line) * LD + i] = cscale(mv[p], 1.0f / (rv[p] + s.floor));
    }
  }
  __syncthreads();
  fft_tile<N, LT, NT, false, PL>(sm, tw);
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e / N, i = e - line * N;
      const float2 a = cscale(sm[line * LD + i], s.sc_x);
      const float2 b = cscale(sm[(LX + line) * LD + i], s.sc_x);
      T[e0 + e] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
}

// ---------------------------------------------------------------- pass A_y (in place on T)

template <int N, int V>
__global__ void __launch_bounds__(NT) k_a_y(Geom g, AgentScalars s, float4* __restrict__ T,
                                            const float2* __restrict__ tw) {
  constexpr int LCV = variant_cols(V), LT = 2 * LCV, LD = N + 1;
  using PL = std::conditional_t<V == 1, PlanB<N>, Plan<N>>;
  float2* sm = reinterpret_cast<float2*>(dyn_smem);
  const long long S = g.nx;
  constexpr int CNT = LCV * N, PER = (CNT + NT - 1) / NT;
  const long long base = (long long)blockIdx.z * g.n + (long long)blockIdx.y * g.ny * g.nx + blockIdx.x * LCV;
  float4 tv[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) tv[p] = T[base + (e / LCV) * S + e % LCV];
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e % LCV, i = e / LCV;
      sm[line * LD + i] = make_float2(tv[p].x, tv[p].y);
      sm[(LCV + line) * LD + i] = make_float2(tv[p].z, tv[p].w);
    }
  }
  __syncthreads();
  fft_tile<N, LT, NT, false, PL>(sm, tw);
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e % LCV, i = e / LCV;
      const float2 a = cscale(sm[line * LD + i], s.sc_y);
      const float2 b = cscale(sm[(LCV + line) * LD + i], s.sc_y);
      T[base + i * S + line] = make_float4(a.x, a.y, b.x, b.y);
    }
  }
}

// ---------------------------------------------------------------- fused z pass (A_z + gradient + B_z)

template <int N, int V>
__global__ void __launch_bounds__(NT) k_ab_z(Geom g, AgentScalars s, const float4* __restrict__ T,
                                             const float2* __restrict__ y, const float* __restrict__ pupil,
                                             const float* __restrict__ window, float2* __restrict__ U,
                                             Partials p, const float2* __restrict__ tw) {
  constexpr int LCV = variant_cols(V), LT = 2 * LCV, LD = N + 1;
  using PL = std::conditional_t<V == 1, PlanB<N>, Plan<N>>;
  float2* sm = reinterpret_cast<float2*>(dyn_smem);
  const long long S = (long long)g.nx * g.ny;
  const int x0 = blockIdx.x * LCV, ky = blockIdx.y, l = blockIdx.z;
  const long long base = (long long)l * g.n + (long long)ky * g.nx + x0;
  constexpr int CNT = LCV * N, PER = (CNT + NT - 1) / NT;
  float4 tv[PER];
  float2 yvs[PER];   // the data for the epilogue is fetched together with T
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      tv[p] = T[base + (e / LCV) * S + e % LCV];
      yvs[p] = y[base + (e / LCV) * S + e % LCV];
    }
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e % LCV, i = e / LCV;
      sm[line * LD + i] = make_float2(tv[p].x, tv[p].y);
      sm[(LCV + line) * LD + i] = make_float2(tv[p].z, tv[p].w);
    }
  }
  __syncthreads();
  fft_tile<N, LT, NT, false, PL>(sm, tw);
  // frequency-domain gradient: Fd = a (y - a M) / sigma_w^2 - P
  float acc[3] = {0.f, 0.f, 0.f};
  const float inv_nv = 1.0f / s.nv;
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (!(CNT % NT == 0 || e < CNT)) continue;
    const int line = e % LCV, kz = e / LCV;
    const float2 M = cscale(sm[line * LD + kz], s.sc_z);
    const float2 P = cscale(sm[(LCV + line) * LD + kz], s.sc_z);
    const float av = __ldg(&pupil[ky * g.nx + x0 + line]) * __ldg(&window[kz]);
    const float2 yv = yvs[p];
    const float2 res = make_float2(fmaf(-av, M.x, yv.x), fmaf(-av, M.y, yv.y));
    const float f = av * inv_nv;
    const float2 fd = make_float2(fmaf(f, res.x, -P.x), fmaf(f, res.y, -P.y));
    const float fd2 = cabs2(fd), a2 = av * av;
    acc[0] += fd2;
    acc[1] += a2 * fd2;
    acc[2] += a2 * cabs2(yv);
    sm[line * LD + kz] = fd;
  }
  __syncthreads();
  fft_tile<N, LCV, NT, true, PL>(sm, tw);
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e % LCV, i = e / LCV;
      U[base + i * S + line] = cscale(sm[line * LD + i], s.sc_z);
    }
  }
  double* const outs[3] = {p.s1, p.s2, p.s4};
  block_reduce_store<3>(acc, outs, (long long)l * p.pz + (long long)blockIdx.y * gridDim.x + blockIdx.x);
}

// ---------------------------------------------------------------- generic single-transform passes

enum RowMode { ROW_PLAIN = 0, ROW_SIM = 1, ROW_ADJ = 2, ROW_BX = 3 };
enum ColMode { COL_PLAIN = 0, COL_SIM = 1, COL_ADJ = 2 };

struct RowArgs {
  const float2* in;
  float2* out;
  const float* rvol;   // ROW_SIM: reflectance [n]
  const float* rprev;  // ROW_BX: r' [L][n]
  float scale;         // 1/sqrt(N) (times mu_scale for ROW_ADJ)
  float floor;         // ROW_BX: sigma_w^2 / alpha
  double* s3;          // ROW_BX partials
  int px;              // ROW_BX partials per look
  long long n;
  int nx;
};

template <int N, bool INV, int MODE, int V = 0>
__global__ void __launch_bounds__(NT) k_row(RowArgs a, const float2* __restrict__ tw) {
  constexpr int LX = variant_rows(N, V), LD = N + 1;
  using PL = std::conditional_t<V == 1, PlanB<N>, Plan<N>>;
  float2* sm = reinterpret_cast<float2*>(dyn_smem);
  constexpr int CNT = LX * N, PER = (CNT + NT - 1) / NT;
  const long long e0 = (long long)blockIdx.x * LX * N;
  float2 iv[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) iv[p] = a.in[e0 + e];
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e / N, i = e - line * N;
      float2 v = iv[p];
      if constexpr (MODE == ROW_SIM) {
        const long long vox = (e0 + e) % a.n;
        v = cscale(v, sqrtf(a.rvol[vox]));
      }
      sm[line * LD + i] = v;
    }
  }
  __syncthreads();
  fft_tile<N, LX, NT, INV, PL>(sm, tw);
  float acc[1] = {0.f};
  float rpv[PER];
  if constexpr (MODE == ROW_BX) {
#pragma unroll
    for (int p = 0; p < PER; ++p) {
      const int e = threadIdx.x + p * NT;
      if (CNT % NT == 0 || e < CNT) rpv[p] = a.rprev[e0 + e];
    }
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e / N, i = e - line * N;
      const float2 v = cscale(sm[line * LD + i], a.scale);
      if constexpr (MODE == ROW_BX) acc[0] += cabs2(v) / (rpv[p] + a.floor);
      a.out[e0 + e] = v;
    }
  }
  if constexpr (MODE == ROW_BX) {
    double* const outs[1] = {a.s3};
    const long long look = e0 / a.n;
    const long long bpl = a.n / ((long long)LX * N);
    block_reduce_store<1>(acc, outs, look * a.px + (blockIdx.x - look * bpl));
  }
}

struct ColArgs {
  const float2* in;
  float2* out;
  const float* pupil;
  const float* window;
  const float2* eta;   // COL_SIM noise draws
  float sig_w;         // COL_SIM sqrt(sigma_w^2)
  float scale;
  long long n;
  long long stride;    // element stride of the FFT axis
  long long slab;      // element stride of grid.y (fixed index of the other axis)
  int nx;
  int zaxis;           // 1 when the FFT axis is z (aperture epilogue / prologue)
};

template <int N, bool INV, int MODE, int V = 0>
__global__ void __launch_bounds__(NT) k_col(ColArgs a, const float2* __restrict__ tw) {
  constexpr int LD = N + 1, LCV = variant_cols(V);
  using PL = std::conditional_t<V == 1, PlanB<N>, Plan<N>>;
  float2* sm = reinterpret_cast<float2*>(dyn_smem);
  const int x0 = blockIdx.x * LCV, fixed = blockIdx.y, l = blockIdx.z;
  const long long base = (long long)l * a.n + (long long)fixed * a.slab + x0;
  constexpr int CNT = LCV * N, PER = (CNT + NT - 1) / NT;
  float2 iv[PER];
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) iv[p] = a.in[base + (e / LCV) * a.stride + e % LCV];
  }
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (CNT % NT == 0 || e < CNT) {
      const int line = e % LCV, i = e / LCV;
      float2 v = iv[p];
      if constexpr (MODE == COL_ADJ) {  // z axis, fixed = ky
        v = cscale(v, __ldg(&a.pupil[fixed * a.nx + x0 + line]) * __ldg(&a.window[i]));
      }
      sm[line * LD + i] = v;
    }
  }
  __syncthreads();
  fft_tile<N, LCV, NT, INV, PL>(sm, tw);
#pragma unroll
  for (int p = 0; p < PER; ++p) {
    const int e = threadIdx.x + p * NT;
    if (!(CNT % NT == 0 || e < CNT)) continue;
    const int line = e % LCV, i = e / LCV;
    float2 v = cscale(sm[line * LD + i], a.scale);
    const long long gi = base + i * a.stride + line;
    if constexpr (MODE == COL_SIM) {  // z axis, fixed = ky: y = a v + sigma_w eta
      const float av = __ldg(&a.pupil[fixed * a.nx + x0 + line]) * __ldg(&a.window[i]);
      const float2 et = a.eta[gi];
      v = make_float2(fmaf(av, v.x, a.sig_w * et.x), fmaf(av, v.y, a.sig_w * et.y));
    }
    a.out[gi] = v;
  }
}

// ---------------------------------------------------------------- dispatch helpers

template <class F>
static cudaError_t dispatch_len(int N, F&& f) {
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

template <int N, bool INV, int MODE, int V = 0>
static cudaError_t run_row(const Geom& g, const RowArgs& a, cudaStream_t st) {
  constexpr int LX = variant_rows(N, V);
  const size_t smem = (size_t)LX * (N + 1) * sizeof(float2);
  auto kern = k_row<N, INV, MODE, V>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long rows = (long long)g.L * g.nz * g.ny;
  kern<<<(unsigned)(rows / LX), NT, smem, st>>>(a, tw_ptr(N));
  return cudaGetLastError();
}

template <int N, bool INV, int MODE, int V = 0>
static cudaError_t run_col(const Geom& g, const ColArgs& a, int fixed_count, cudaStream_t st) {
  constexpr int LCV = variant_cols(V);
  const size_t smem = (size_t)LCV * (N + 1) * sizeof(float2);
  auto kern = k_col<N, INV, MODE, V>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  dim3 grid(g.nx / LCV, fixed_count, g.L);
  kern<<<grid, NT, smem, st>>>(a, tw_ptr(N));
  return cudaGetLastError();
}

static ColArgs col_args(const Geom& g, bool zaxis) {
  ColArgs a{};
  a.n = g.n;
  a.nx = g.nx;
  a.zaxis = zaxis;
  if (zaxis) {
    a.stride = (long long)g.nx * g.ny;
    a.slab = g.nx;
  } else {
    a.stride = g.nx;
    a.slab = (long long)g.nx * g.ny;
  }
  return a;
}

#define CLAMP_TRY(x)                       \
  do {                                     \
    cudaError_t _e = (x);                  \
    if (_e != cudaSuccess) return _e;      \
  } while (0)

// ---------------------------------------------------------------- forward agent FFT passes

template <class F>
static cudaError_t dispatch_var(int V, F&& f) {
  switch (V) {
    case 0: return f(std::integral_constant<int, 0>{});
    case 1: return f(std::integral_constant<int, 1>{});
    case 2: return f(std::integral_constant<int, 2>{});
    default: return cudaErrorInvalidValue;
  }
}

bool variant_valid(int pass, int V, int nx, int ny, int nz) {
  if (V < 0 || V >= kVariants) return false;
  if (V == 0 || V == 1) return true;
  if (pass == 0 || pass == 4) return true;   // x passes: half the rows per CTA always divides nz * ny
  if (V == 3) return nx % 16 == 0;            // y / z passes: pipe_cols <= 16 adjacent columns
  return nx % 32 == 0;                        // y / z passes: 32 adjacent columns
}

int max_pz(int nx, int ny) { return (nx / 8) * ny; }   // the narrowest column tile is 8 (pipe_cols)
int max_px(int nx, int ny, int nz) {
  int m = 0;
  for (int V = 0; V < kVariants; ++V) {
    const int lx = variant_rows(nx, V);
    const int px = (int)((long long)nz * ny / lx);
    if (px > m) m = px;
  }
  return m;
}

cudaError_t launch_agent_pass(int pass, int V, const Geom& g, const AgentScalars& s, const float2* mu,
                              const float* rprev, const float2* y, const float* pupil, const float* window, float4* T,
                              float2* U, Partials& p, cudaStream_t st) {
  if (!variant_valid(pass, V, g.nx, g.ny, g.nz)) return cudaErrorInvalidValue;
  if (V == 3) {
    const int axis_len = (pass == 0 || pass == 4) ? g.nx : (pass == 2 ? g.nz : g.ny);
    return launch_pipe_pass(pass, g, s, mu, rprev, y, pupil, window, T, U, p, tw_ptr(axis_len), st);
  }
  switch (pass) {
    case 0:  // A_x
      return dispatch_var(V, [&](auto VC) -> cudaError_t {
        constexpr int VV = decltype(VC)::value;
        return dispatch_len(g.nx, [&](auto NC) -> cudaError_t {
          constexpr int N = decltype(NC)::value;
          constexpr int LX = variant_rows(N, VV);
          const size_t smem = (size_t)2 * LX * (N + 1) * sizeof(float2);
          CLAMP_TRY(cudaFuncSetAttribute(k_a_x<N, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          const long long rows = (long long)g.L * g.nz * g.ny;
          k_a_x<N, VV><<<(unsigned)(rows / LX), NT, smem, st>>>(g, s, mu, rprev, T, tw_ptr(N));
          return cudaGetLastError();
        });
      });
    case 1:  // A_y
      return dispatch_var(V, [&](auto VC) -> cudaError_t {
        constexpr int VV = decltype(VC)::value;
        return dispatch_len(g.ny, [&](auto NC) -> cudaError_t {
          constexpr int N = decltype(NC)::value;
          constexpr int LCV = variant_cols(VV);
          const size_t smem = (size_t)2 * LCV * (N + 1) * sizeof(float2);
          CLAMP_TRY(cudaFuncSetAttribute(k_a_y<N, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          k_a_y<N, VV><<<dim3(g.nx / LCV, g.nz, g.L), NT, smem, st>>>(g, s, T, tw_ptr(N));
          return cudaGetLastError();
        });
      });
    case 2:  // fused z pass
      return dispatch_var(V, [&](auto VC) -> cudaError_t {
        constexpr int VV = decltype(VC)::value;
        return dispatch_len(g.nz, [&](auto NC) -> cudaError_t {
          constexpr int N = decltype(NC)::value;
          constexpr int LCV = variant_cols(VV);
          const size_t smem = (size_t)2 * LCV * (N + 1) * sizeof(float2);
          CLAMP_TRY(cudaFuncSetAttribute(k_ab_z<N, VV>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
          p.pz = (g.nx / LCV) * g.ny;
          k_ab_z<N, VV><<<dim3(g.nx / LCV, g.ny, g.L), NT, smem, st>>>(g, s, T, y, pupil, window, U, p, tw_ptr(N));
          return cudaGetLastError();
        });
      });
    case 3: {  // B_y (in place on U)
      ColArgs cy = col_args(g, false);
      cy.in = U;
      cy.out = U;
      cy.scale = s.sc_y;
      return dispatch_var(V, [&](auto VC) -> cudaError_t {
        constexpr int VV = decltype(VC)::value;
        return dispatch_len(g.ny, [&](auto NC) { return run_col<decltype(NC)::value, true, COL_PLAIN, VV>(g, cy, g.nz, st); });
      });
    }
    case 4: {  // B_x (in place on U, d out, S3 partials)
      RowArgs rx{};
      rx.in = U;
      rx.out = U;
      rx.rprev = rprev;
      rx.scale = s.sc_x;
      rx.floor = s.floor;
      rx.s3 = p.s3;
      rx.n = g.n;
      rx.nx = g.nx;
      return dispatch_var(V, [&](auto VC) -> cudaError_t {
        constexpr int VV = decltype(VC)::value;
        return dispatch_len(g.nx, [&](auto NC) -> cudaError_t {
          constexpr int N = decltype(NC)::value;
          p.px = (int)((long long)g.nz * g.ny / variant_rows(N, VV));
          rx.px = p.px;
          return run_row<N, true, ROW_BX, VV>(g, rx, st);
        });
      });
    }
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t launch_agent_fft(const Geom& g, const AgentScalars& s, const float2* mu, const float* rprev,
                             const float2* y, const float* pupil, const float* window, float4* T, float2* U,
                             Partials& p, const AgentVariants& var, cudaStream_t st) {
  for (int pass = 0; pass < 5; ++pass)
    CLAMP_TRY(launch_agent_pass(pass, var.v[pass], g, s, mu, rprev, y, pupil, window, T, U, p, st));
  return cudaSuccess;
}

// ---------------------------------------------------------------- gamma (exact line search)

__global__ void __launch_bounds__(NT) k_gamma(int L, float nv, Partials p, float* gamma, double* mures) {
  const int l = blockIdx.x;
  __shared__ double red[NT][4];
  double a1 = 0, a2 = 0, a4 = 0, a3 = 0;
  for (int i = threadIdx.x; i < p.pz; i += NT) {
    a1 += p.s1[(long long)l * p.pz + i];
    a2 += p.s2[(long long)l * p.pz + i];
    a4 += p.s4[(long long)l * p.pz + i];
  }
  for (int i = threadIdx.x; i < p.px; i += NT) a3 += p.s3[(long long)l * p.px + i];
  red[threadIdx.x][0] = a1;
  red[threadIdx.x][1] = a2;
  red[threadIdx.x][2] = a3;
  red[threadIdx.x][3] = a4;
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

cudaError_t launch_gamma(const Geom& g, float nv, const Partials& p, float* gamma, double* mures, cudaStream_t st) {
  k_gamma<<<g.L, NT, 0, st>>>(g.L, nv, p, gamma, mures);
  return cudaGetLastError();
}

__global__ void k_mean(const double* v, int L, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double a = 0;
    for (int i = 0; i < L; ++i) a += v[i];
    *out = a / L;
  }
}

cudaError_t launch_mean(const double* v, int L, double* out, cudaStream_t st) {
  k_mean<<<1, 32, 0, st>>>(v, L, out);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- pass C

// App. A reflectance update for one voxel of one look: quadratic fit of the
// derivative of Q (Eq. convex-surrogate) between r' and xi, closed-form prox,
// clip to the validity interval.
// Divisions are reciprocals: 1/xi follows from 1/r' (xi = r' / beta or beta r'), and
// 1/sigma^2, 1/beta come from the host, so a voxel takes two correctly rounded reciprocals.
__device__ __forceinline__ float prox_quad(float v, float rp, float K, float s2, float inv_s2, float beta,
                                           float inv_beta) {
  const float inv = __frcp_rn(rp);
  const float qr = fmaf(-K * inv, inv, inv);           // 1/r' - K/r'^2
  const float drho = fmaf(rp - v, inv_s2, qr);
  const bool down = drho > 0.0f;                        // the minimiser lies below r'
  const float xi = down ? rp * inv_beta : beta * rp;
  const float ixi = down ? beta * inv : inv * inv_beta;
  const float aq = K * (xi + rp) * (inv * inv) * (ixi * ixi);
  const float bq = fmaf(-aq, rp, qr);
  const float rn = (v - s2 * bq) * __frcp_rn(fmaf(s2, aq, 1.0f));
  const float lo = fminf(rp, xi), hi = fmaxf(rp, xi);
  return fminf(fmaxf(rn, lo), hi);
}

// Exact prox of one voxel's EM surrogate (Sec. III-B): the positive real root of
// r^3 - v r^2 + s2 r - s2 K = 0 minimising log r + K/r + (r - v)^2 / (2 s2), in FP64
// (trigonometric form for three real roots, Cardano otherwise, one Newton polish each).
__device__ double prox_exact(double v, double K, double s2) {
  const double a2 = -v, a1 = s2, a0 = -s2 * K;
  const double q = (3.0 * a1 - a2 * a2) / 9.0;
  const double rr = (9.0 * a2 * a1 - 27.0 * a0 - 2.0 * a2 * a2 * a2) / 54.0;
  const double disc = q * q * q + rr * rr;
  double roots[3];
  int nr;
  if (disc > 0.0) {
    const double sd = sqrt(disc);
    roots[0] = cbrt(rr + sd) + cbrt(rr - sd) - a2 / 3.0;
    nr = 1;
  } else {
    const double m = 2.0 * sqrt(-q);
    const double c = fmin(fmax(rr / sqrt(-q * q * q), -1.0), 1.0);
    const double th = acos(c);
    const double twopi3 = 2.0943951023931954923;  // 2 pi / 3
    roots[0] = m * cos(th / 3.0) - a2 / 3.0;
    roots[1] = m * cos(th / 3.0 + twopi3) - a2 / 3.0;
    roots[2] = m * cos(th / 3.0 + 2.0 * twopi3) - a2 / 3.0;
    nr = 3;
  }
  double best = -1.0, best_f = 0.0;
  for (int i = 0; i < nr; ++i) {
    double r = roots[i];
    const double f = ((r + a2) * r + a1) * r + a0, df = (3.0 * r + 2.0 * a2) * r + a1;
    if (df != 0.0) r -= f / df;  // Newton polish
    if (!(r > 0.0)) continue;
    const double obj = log(r) + K / r + (r - v) * (r - v) / (2.0 * s2);
    if (best < 0.0 || obj < best_f) {
      best = r;
      best_f = obj;
    }
  }
  return best > 0.0 ? best : 1e-30;
}

// Error-free sum accumulation (Knuth two-sum) for the per-voxel look averages.
struct CSum {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    const float bp = t - s;
    c += (s - (t - bp)) + (x - bp);
    s = t;
  }
  __device__ __forceinline__ float get() const { return s + c; }
};

int passc_blocks(long long n) {
  long long b = (n + NT - 1) / NT;
  return (int)(b < 152 * 8 ? b : 152 * 8);
}

// The fused pass reads every look's r and w of a voxel twice (the look sum, then the Mann
// step), so the second read hits L2 only while the rows all resident threads hold fit in
// it: the grid keeps them near 48 MB (16 bytes per voxel pair and row), in whole waves of
// 152 SMs, between 1 and 8 CTAs per SM.  (A 64 MB grid with 64 registers per thread ran the
// pass faster but left more dirty lines in L2 for the next iteration's passes: slower overall.)
int passc_fused_blocks(long long n, int L) {
  const long long threads = (48LL << 20) / (16LL * (L + 1));
  long long b = (threads + NT - 1) / NT;
  b = (b + 151) / 152 * 152;
  if (b < 152) b = 152;
  const int cap = passc_blocks(n);
  return (int)(b < cap ? b : cap);
}

// Each thread walks the L looks of one voxel at a time.  The look loops are software-
// pipelined: look l + 1's loads are issued before look l's arithmetic and stores (the
// arrays do not alias), so two looks' loads are in flight per thread.
template <bool PROX, bool MACE, bool EXACT = false>
__global__ void __launch_bounds__(NT) k_pass_c(Geom g, PassC c) {
  const long long n = g.n;
  const int L = g.L;
  const float* __restrict__ Wi = c.w;
  float* __restrict__ Wo = c.w;
  const float* __restrict__ Ri = c.r;
  float* __restrict__ Ro = c.r;
  const float2* __restrict__ MUi = c.mu;
  float2* __restrict__ MUo = c.mu;
  const float2* __restrict__ Di = c.d;
  float acc[2] = {0.f, 0.f};
  for (long long v = (long long)blockIdx.x * NT + threadIdx.x; v < n; v += (long long)gridDim.x * NT) {
    CSum wbar_old, xbar;
    bool bad = false;
    float wl_n = Wi[v], rp_n = 0.f;
    float2 m_n = make_float2(0.f, 0.f), d_n = m_n;
    if constexpr (PROX) {
      rp_n = Ri[v];
      m_n = MUi[v];
      d_n = Di[v];
    } else {
      rp_n = Ri[v];
    }
    for (int l = 0; l < L; ++l) {
      const long long i = (long long)l * n + v;
      const float wl = wl_n, rp = rp_n;
      const float2 m0 = m_n, dd = d_n;
      if (l + 1 < L) {
        const long long in = i + n;
        wl_n = Wi[in];
        rp_n = Ri[in];
        if constexpr (PROX) {
          m_n = MUi[in];
          d_n = Di[in];
        }
      }
      float rn;
      if constexpr (PROX) {
        float2 m = m0;
        if (c.closed_mu) {  // no-aperture ablation: d holds F^H y
          const float f = 1.0f / (1.0f + c.nv / (rp + c.nv));
          m = make_float2(dd.x * f, dd.y * f);
        } else {
          const float gm = __ldg(&c.gamma[l]);
          m.x = fmaf(gm, dd.x, m.x);
          m.y = fmaf(gm, dd.y, m.y);
        }
        MUo[i] = m;
        const float cc = c.nv * rp * __frcp_rn(fmaf(c.alpha, rp, c.nv));
        const float K = cc + cabs2(m);
        if constexpr (EXACT) rn = (float)prox_exact((double)wl, (double)K, (double)c.prox_var);
        else rn = prox_quad(wl, rp, K, c.prox_var, c.inv_prox_var, c.beta, c.inv_beta);
        Ro[i] = rn;
        bad |= !isfinite(rn) || !isfinite(K);   // K covers mu: the prox's clip would hide a NaN there
      } else {
        rn = rp;
      }
      if constexpr (MACE) {
        wbar_old.add(c.ups_look * wl);
        xbar.add(c.ups_look * (2.0f * rn - wl));
      }
    }
    if constexpr (MACE) {
      const long long ip = (long long)L * n + v;
      const float rpr = Ri[ip], wpr = Wi[ip];
      wbar_old.add(c.ups_prior * wpr);
      xbar.add(c.ups_prior * (2.0f * rpr - wpr));
      const float wb = wbar_old.get(), xb = xbar.get();
      float num = 0.f;
      CSum wbar_new;
      // r and w of this voxel were just touched: these reads are L2 hits
      float rj_n = Ri[v], wj_n = Wi[v];
      for (int j = 0; j <= L; ++j) {
        const long long i = (long long)j * n + v;
        const float rj = rj_n, wj = wj_n;
        if (j < L) {
          rj_n = Ri[i + n];
          wj_n = Wi[i + n];
        }
        const float dv = rj - wb;
        num = fmaf(dv, dv, num);
        const float wn = fmaf(2.0f * c.rho, xb - rj, wj);
        Wo[i] = wn;
        wbar_new.add((j < L ? c.ups_look : c.ups_prior) * wn);
        bad |= !isfinite(wn);
      }
      c.wbar[v] = wbar_new.get();
      acc[0] += num;
      acc[1] += (float)(L + 1) * wb * wb;
    }
    if (bad && c.err) atomicOr(c.err, 1);
  }
  if constexpr (MACE) {
    double* const outs[2] = {c.part_num, c.part_den};
    block_reduce_store<2>(acc, outs, blockIdx.x);
  }
}

// Fused pass C on pairs of adjacent voxels: the same arithmetic as k_pass_c<true, true,
// false> per voxel, with 16-byte loads of mu and d and 8-byte loads of r and w, so each
// memory request carries two voxels (n even; the launcher checks the pointers'
// alignment and otherwise uses the one-voxel kernel).  The look-sum loop keeps the loads
// of the next two looks in flight and asks L2 for the look six ahead (the grid is small,
// to keep the Mann loop's re-reads in L2, so each thread needs more bytes in flight).
constexpr int kPassCPrefetch = 6;   // looks ahead that the look-sum loop prefetches into L2

__global__ void __launch_bounds__(NT) k_pass_c_pair(Geom g, PassC c) {
  const long long n2 = g.n / 2;
  const int L = g.L;
  const float2* __restrict__ Wi = reinterpret_cast<const float2*>(c.w);
  float2* __restrict__ Wo = reinterpret_cast<float2*>(c.w);
  const float2* __restrict__ Ri = reinterpret_cast<const float2*>(c.r);
  float2* __restrict__ Ro = reinterpret_cast<float2*>(c.r);
  const float4* __restrict__ MUi = reinterpret_cast<const float4*>(c.mu);
  float4* __restrict__ MUo = reinterpret_cast<float4*>(c.mu);
  const float4* __restrict__ Di = reinterpret_cast<const float4*>(c.d);
  [[maybe_unused]] const long long look_ext = (long long)L * n2, row_ext = (long long)(L + 1) * n2;   // in pairs
  float acc[2] = {0.f, 0.f};
  for (long long vp = (long long)blockIdx.x * NT + threadIdx.x; vp < n2; vp += (long long)gridDim.x * NT) {
    CSum wb0, xb0, wb1, xb1;
    bool bad = false;
    // two looks ahead in flight: slot a holds look l + 1, slot b look l + 2
    float2 w_n = Wi[vp], r_n = Ri[vp];
    float4 m_n = __ldcs(&MUi[vp]), d_n = __ldcs(&Di[vp]);
    float2 w_a = w_n, r_a = r_n;
    float4 m_a = m_n, d_a = d_n;
    if (L > 1) {
      w_a = Wi[n2 + vp];
      r_a = Ri[n2 + vp];
      m_a = __ldcs(&MUi[n2 + vp]);
      d_a = __ldcs(&Di[n2 + vp]);
    }
    float kacc = 0.f;   // sum of K over the looks: non-finite iff some K (so some mu) is
    for (int l = 0; l < L; ++l) {
      const long long i = (long long)l * n2 + vp;
      const float2 wl = w_n, rp = r_n;
      float4 m = m_n;
      const float4 dd = d_n;
      w_n = w_a;
      r_n = r_a;
      m_n = m_a;
      d_n = d_a;
      if (l + 2 < L && CLAMP_IN_BOUNDS(i + 2 * n2, look_ext, 201)) {
        w_a = Wi[i + 2 * n2];
        r_a = Ri[i + 2 * n2];
        m_a = __ldcs(&MUi[i + 2 * n2]);
        d_a = __ldcs(&Di[i + 2 * n2]);
      }
      if (l + kPassCPrefetch < L) {   // look l + kPassCPrefetch into L2: no registers held
        const long long ip = i + kPassCPrefetch * n2;
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Wi + ip));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Ri + ip));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(MUi + ip));
        asm volatile("prefetch.global.L2 [%0];" ::"l"(Di + ip));
      }
      if (c.closed_mu) {  // no-aperture ablation: d holds F^H y
        const float f0 = 1.0f / (1.0f + c.nv / (rp.x + c.nv)), f1 = 1.0f / (1.0f + c.nv / (rp.y + c.nv));
        m = make_float4(dd.x * f0, dd.y * f0, dd.z * f1, dd.w * f1);
      } else {
        const float gm = __ldg(&c.gamma[l]);
        m = make_float4(fmaf(gm, dd.x, m.x), fmaf(gm, dd.y, m.y), fmaf(gm, dd.z, m.z), fmaf(gm, dd.w, m.w));
      }
      const bool in_look = CLAMP_IN_BOUNDS(i, look_ext, 202);
      if (in_look) __stcs(&MUo[i], m);   // mu and d are not read again here: evict first
      const float c0 = c.nv * rp.x * __frcp_rn(fmaf(c.alpha, rp.x, c.nv));
      const float c1 = c.nv * rp.y * __frcp_rn(fmaf(c.alpha, rp.y, c.nv));
      const float K0 = c0 + fmaf(m.x, m.x, m.y * m.y), K1 = c1 + fmaf(m.z, m.z, m.w * m.w);
      const float2 rn = make_float2(prox_quad(wl.x, rp.x, K0, c.prox_var, c.inv_prox_var, c.beta, c.inv_beta),
                                    prox_quad(wl.y, rp.y, K1, c.prox_var, c.inv_prox_var, c.beta, c.inv_beta));
      if (in_look) Ro[i] = rn;
      kacc += K0 + K1;   // K covers mu: the prox's clip would hide a NaN there
      wb0.add(c.ups_look * wl.x);
      wb1.add(c.ups_look * wl.y);
      xb0.add(c.ups_look * (2.0f * rn.x - wl.x));
      xb1.add(c.ups_look * (2.0f * rn.y - wl.y));
    }
    const long long ip = (long long)L * n2 + vp;
    const float2 rpr = Ri[ip], wpr = Wi[ip];
    wb0.add(c.ups_prior * wpr.x);
    wb1.add(c.ups_prior * wpr.y);
    xb0.add(c.ups_prior * (2.0f * rpr.x - wpr.x));
    xb1.add(c.ups_prior * (2.0f * rpr.y - wpr.y));
    const float w0 = wb0.get(), w1 = wb1.get(), x0 = xb0.get(), x1 = xb1.get();
    float num = 0.f;
    CSum wn0, wn1;
    float2 rj_n = Ri[vp], wj_n = Wi[vp];
    float2 rj_a = Ri[n2 + vp], wj_a = Wi[n2 + vp];   // rows 0..L: L + 1 >= 2
    for (int j = 0; j <= L; ++j) {
      const long long i = (long long)j * n2 + vp;
      const float2 rj = rj_n, wj = wj_n;
      rj_n = rj_a;
      wj_n = wj_a;
      if (j + 2 <= L && CLAMP_IN_BOUNDS(i + 2 * n2, row_ext, 203)) {
        rj_a = Ri[i + 2 * n2];
        wj_a = Wi[i + 2 * n2];
      }
      const float dv0 = rj.x - w0, dv1 = rj.y - w1;
      num = fmaf(dv0, dv0, fmaf(dv1, dv1, num));
      const float2 wn = make_float2(fmaf(2.0f * c.rho, x0 - rj.x, wj.x), fmaf(2.0f * c.rho, x1 - rj.y, wj.y));
      if (CLAMP_IN_BOUNDS(i, row_ext, 204)) Wo[i] = wn;
      const float ups = j < L ? c.ups_look : c.ups_prior;
      wn0.add(ups * wn.x);
      wn1.add(ups * wn.y);
    }
    const float wbn0 = wn0.get(), wbn1 = wn1.get();
    reinterpret_cast<float2*>(c.wbar)[vp] = make_float2(wbn0, wbn1);
    // a non-finite r, w or K of any look reaches these sums (NaN and Inf propagate through
    // the adds), so one check per voxel pair replaces one per value
    bad = !isfinite(kacc) || !isfinite(x0) || !isfinite(x1) || !isfinite(w0) || !isfinite(w1) ||
          !isfinite(wbn0) || !isfinite(wbn1);
    acc[0] += num;
    acc[1] += (float)(L + 1) * (w0 * w0 + w1 * w1);
    if (bad && c.err) atomicOr(c.err, 1);
  }
  double* const outs[2] = {c.part_num, c.part_den};
  block_reduce_store<2>(acc, outs, blockIdx.x);
}

static bool aligned(const void* p, uintptr_t a) { return ((uintptr_t)p % a) == 0; }

__global__ void __launch_bounds__(NT) k_mu_update(long long n, long long total, float2* __restrict__ mu,
                                                  const float2* __restrict__ d, const float* __restrict__ gamma) {
  for (long long i = (long long)blockIdx.x * NT + threadIdx.x; i < total; i += (long long)gridDim.x * NT) {
    const float gm = __ldg(&gamma[i / n]);
    const float2 dd = d[i];
    float2 m = mu[i];
    m.x = fmaf(gm, dd.x, m.x);
    m.y = fmaf(gm, dd.y, m.y);
    mu[i] = m;
  }
}

cudaError_t launch_mu_update(const Geom& g, float2* mu, const float2* d, const float* gamma, cudaStream_t st) {
  const long long total = g.n * g.L;
  k_mu_update<<<passc_blocks(total), NT, 0, st>>>(g.n, total, mu, d, gamma);
  return cudaGetLastError();
}

cudaError_t launch_pass_c_fused(const Geom& g, const PassC& c, cudaStream_t st) {
  const bool pair = g.n % 2 == 0 && aligned(c.w, 8) && aligned(c.r, 8) && aligned(c.wbar, 8) &&
                    aligned(c.mu, 16) && aligned(c.d, 16);
  const int nb = passc_fused_blocks(g.n, g.L);
  if (c.exact_prox) k_pass_c<true, true, true><<<nb, NT, 0, st>>>(g, c);
  else if (pair) k_pass_c_pair<<<nb, NT, 0, st>>>(g, c);
  else k_pass_c<true, true><<<nb, NT, 0, st>>>(g, c);
  return cudaGetLastError();
}
cudaError_t launch_prox_only(const Geom& g, const PassC& c, cudaStream_t st) {
  if (c.exact_prox) k_pass_c<true, false, true><<<passc_blocks(g.n), NT, 0, st>>>(g, c);
  else k_pass_c<true, false><<<passc_blocks(g.n), NT, 0, st>>>(g, c);
  return cudaGetLastError();
}
cudaError_t launch_mace_only(const Geom& g, const PassC& c, cudaStream_t st) {
  k_pass_c<false, true><<<passc_blocks(g.n), NT, 0, st>>>(g, c);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(NT) k_ce_final(const double* num, const double* den, int nblk, double* ce) {
  __shared__ double rn[NT], rd[NT];
  double a = 0, b = 0;
  for (int i = threadIdx.x; i < nblk; i += NT) {
    a += num[i];
    b += den[i];
  }
  rn[threadIdx.x] = a;
  rd[threadIdx.x] = b;
  __syncthreads();
  for (int o = NT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rn[threadIdx.x] += rn[threadIdx.x + o];
      rd[threadIdx.x] += rd[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *ce = rd[0] > 0 ? sqrt(rn[0] / rd[0]) : 0.0;
}

cudaError_t launch_ce_final(const double* num, const double* den, int nblk, double* ce, cudaStream_t st) {
  k_ce_final<<<1, NT, 0, st>>>(num, den, nblk, ce);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- plain transforms, simulation, adjoint

cudaError_t launch_fft3(const Geom& g, const float2* in, float2* out, bool inverse, float sc_x, float sc_y,
                        float sc_z, cudaStream_t st) {
  RowArgs rx{};
  rx.n = g.n;
  rx.nx = g.nx;
  ColArgs cy = col_args(g, false), cz = col_args(g, true);
  cy.in = cy.out = out;
  cy.scale = sc_y;
  cz.scale = sc_z;
  rx.scale = sc_x;
  if (!inverse) {
    rx.in = in;
    rx.out = out;
    cz.in = cz.out = out;
    CLAMP_TRY(dispatch_len(g.nx, [&](auto NC) { return run_row<decltype(NC)::value, false, ROW_PLAIN>(g, rx, st); }));
    CLAMP_TRY(dispatch_len(g.ny, [&](auto NC) { return run_col<decltype(NC)::value, false, COL_PLAIN>(g, cy, g.nz, st); }));
    CLAMP_TRY(dispatch_len(g.nz, [&](auto NC) { return run_col<decltype(NC)::value, false, COL_PLAIN>(g, cz, g.ny, st); }));
  } else {
    cz.in = in;
    cz.out = out;
    rx.in = rx.out = out;
    CLAMP_TRY(dispatch_len(g.nz, [&](auto NC) { return run_col<decltype(NC)::value, true, COL_PLAIN>(g, cz, g.ny, st); }));
    CLAMP_TRY(dispatch_len(g.ny, [&](auto NC) { return run_col<decltype(NC)::value, true, COL_PLAIN>(g, cy, g.nz, st); }));
    CLAMP_TRY(dispatch_len(g.nx, [&](auto NC) { return run_row<decltype(NC)::value, true, ROW_PLAIN>(g, rx, st); }));
  }
  return cudaSuccess;
}

cudaError_t launch_simulate(const Geom& g, const float* r, const float2* z, const float2* eta, const float* pupil,
                            const float* window, float sig_w, float2* y, float sc_x, float sc_y, float sc_z,
                            cudaStream_t st) {
  RowArgs rx{};
  rx.in = z;
  rx.out = y;
  rx.rvol = r;
  rx.scale = sc_x;
  rx.n = g.n;
  rx.nx = g.nx;
  ColArgs cy = col_args(g, false), cz = col_args(g, true);
  cy.in = cy.out = y;
  cy.scale = sc_y;
  cz.in = cz.out = y;
  cz.scale = sc_z;
  cz.pupil = pupil;
  cz.window = window;
  cz.eta = eta;
  cz.sig_w = sig_w;
  CLAMP_TRY(dispatch_len(g.nx, [&](auto NC) { return run_row<decltype(NC)::value, false, ROW_SIM>(g, rx, st); }));
  CLAMP_TRY(dispatch_len(g.ny, [&](auto NC) { return run_col<decltype(NC)::value, false, COL_PLAIN>(g, cy, g.nz, st); }));
  CLAMP_TRY(dispatch_len(g.nz, [&](auto NC) { return run_col<decltype(NC)::value, false, COL_SIM>(g, cz, g.ny, st); }));
  return cudaSuccess;
}

cudaError_t launch_adjoint(const Geom& g, const float2* y, const float* pupil, const float* window, float mu_scale,
                           float2* mu, float sc_x, float sc_y, float sc_z, cudaStream_t st) {
  ColArgs cz = col_args(g, true), cy = col_args(g, false);
  cz.in = y;
  cz.out = mu;
  cz.pupil = pupil;
  cz.window = window;
  cz.scale = sc_z;
  cy.in = cy.out = mu;
  cy.scale = sc_y;
  RowArgs rx{};
  rx.in = rx.out = mu;
  rx.scale = sc_x * mu_scale;
  rx.n = g.n;
  rx.nx = g.nx;
  if (pupil)
    CLAMP_TRY(dispatch_len(g.nz, [&](auto NC) { return run_col<decltype(NC)::value, true, COL_ADJ>(g, cz, g.ny, st); }));
  else
    CLAMP_TRY(dispatch_len(g.nz, [&](auto NC) { return run_col<decltype(NC)::value, true, COL_PLAIN>(g, cz, g.ny, st); }));
  CLAMP_TRY(dispatch_len(g.ny, [&](auto NC) { return run_col<decltype(NC)::value, true, COL_PLAIN>(g, cy, g.nz, st); }));
  CLAMP_TRY(dispatch_len(g.nx, [&](auto NC) { return run_row<decltype(NC)::value, true, ROW_PLAIN>(g, rx, st); }));
  return cudaSuccess;
}

// ---------------------------------------------------------------- initial state

__global__ void __launch_bounds__(NT) k_speckle_avg(Geom g, const float2* __restrict__ mu, float inv_scale2,
                                                    const float* __restrict__ r_init, float* __restrict__ r0,
                                                    float* __restrict__ max_part) {
  float mx = 0.f;
  for (long long v = (long long)blockIdx.x * NT + threadIdx.x; v < g.n; v += (long long)gridDim.x * NT) {
    float val;
    if (r_init) {
      val = r_init[v];
    } else {
      float a = 0.f;
      for (int l = 0; l < g.L; ++l) a += cabs2(mu[(long long)l * g.n + v]);
      val = a * inv_scale2 / (float)g.L;
    }
    r0[v] = val;
    mx = fmaxf(mx, val);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  __shared__ float red[NT / 32];
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int i = 0; i < NT / 32; ++i) m = fmaxf(m, red[i]);
    max_part[blockIdx.x] = m;
  }
}

__global__ void __launch_bounds__(NT) k_broadcast_init(Geom g, const float* __restrict__ max_part, int nblk,
                                                       float* __restrict__ r, float* __restrict__ w) {
  __shared__ float s_floor;
  if (threadIdx.x == 0) {
    float m = 0.f;
    for (int i = 0; i < nblk; ++i) m = fmaxf(m, max_part[i]);
    s_floor = 1e-12f * m;
  }
  __syncthreads();
  const float fl = s_floor;
  const float* r0 = r + (long long)g.L * g.n;  // staged in the prior row
  for (long long v = (long long)blockIdx.x * NT + threadIdx.x; v < g.n; v += (long long)gridDim.x * NT) {
    const float val = fmaxf(r0[v], fl);
    for (int j = 0; j <= g.L; ++j) {
      r[(long long)j * g.n + v] = val;
      w[(long long)j * g.n + v] = val;
    }
  }
}

cudaError_t launch_init_state(const Geom& g, const float2* mu, float mu_scale, const float* r_init, float* r, float* w,
                              float* max_part, int* nblk_out, cudaStream_t st) {
  const int nb = passc_blocks(g.n);
  float* r0 = r + (long long)g.L * g.n;
  k_speckle_avg<<<nb, NT, 0, st>>>(g, mu, 1.0f / (mu_scale * mu_scale), r_init, r0, max_part);
  CLAMP_TRY(cudaGetLastError());
  k_broadcast_init<<<nb, NT, 0, st>>>(g, max_part, nb, r, w);
  if (nblk_out) *nblk_out = nb;
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Gaussian prior agent

__global__ void __launch_bounds__(NT) k_gauss3(int nx, int ny, int nz, const float* __restrict__ in,
                                               float* __restrict__ out, float g0, float g1) {
  const long long n = (long long)nx * ny * nz;
  for (long long v = (long long)blockIdx.x * NT + threadIdx.x; v < n; v += (long long)gridDim.x * NT) {
    const int x = (int)(v % nx);
    const int y = (int)((v / nx) % ny);
    const int z = (int)(v / ((long long)nx * ny));
    float acc = 0.f;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = z + dz;
      if (zz < 0 || zz >= nz) continue;
      const float wz = dz == 0 ? g1 : g0;
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy;
        if (yy < 0 || yy >= ny) continue;
        const float wzy = wz * (dy == 0 ? g1 : g0);
        const float* row = in + ((long long)zz * ny + yy) * nx;
        float s = g1 * __ldg(&row[x]);
        if (x > 0) s = fmaf(g0, __ldg(&row[x - 1]), s);
        if (x + 1 < nx) s = fmaf(g0, __ldg(&row[x + 1]), s);
        acc = fmaf(wzy, s, acc);
      }
    }
    out[v] = acc;
  }
}

cudaError_t launch_gauss3(int nx, int ny, int nz, const float* in, float* out, float g0, float g1, cudaStream_t st) {
  const long long n = (long long)nx * ny * nz;
  long long b = (n + NT - 1) / NT;
  if (b > 152 * 16) b = 152 * 16;
  k_gauss3<<<(unsigned)b, NT, 0, st>>>(nx, ny, nz, in, out, g0, g1);
  return cudaGetLastError();
}

__global__ void k_nonfinite(const float* x, long long count, int* err) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) atomicOr(err, 1);
}

cudaError_t launch_nonfinite_check(const float* x, long long count, int* err, cudaStream_t st) {
  k_nonfinite<<<152 * 4, NT, 0, st>>>(x, count, err);
  return cudaGetLastError();
}

cudaError_t bounds_site_kernels(unsigned int* site, bool reset) { return bounds_site_local(site, reset); }

}  // namespace clamp
