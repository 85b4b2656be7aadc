// fft_pipe.cu -- software-pipelined, persistent versions of the forward-agent FFT passes
// (launch variant 3 of every pass; same arithmetic as the one-tile-per-CTA kernels).
//
// A one-tile-per-CTA pass loads its tile, synchronises and computes, so an SM's HBM
// queue drains while it runs the shared-memory FFT.  Here each CTA owns tiles
// t = blockIdx.x, blockIdx.x + G, ... (G = resident CTAs) and keeps two tile buffers
// in shared memory: the next tile's loads are issued with cp.async straight into the
// padded FFT layout of one buffer before the FFT and epilogue of the current tile run
// on the other, so the loads are in flight during the compute.  Tiles never overlap,
// so the in-place passes can prefetch tile t + G while storing tile t.
#include "clamp_kernels.cuh"
#include "fft_core.cuh"

#include <type_traits>

namespace clamp {
namespace {

extern __shared__ float4 pipe_smem[];

__device__ __forceinline__ uint32_t sptr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void cp8(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sptr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp4(void* s, const void* g) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sptr(s)), "l"(g) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// Waits until at most one (the most recent) of this thread's groups is still pending.
__device__ __forceinline__ void cp_wait_prev() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// FP32 per thread and warp, FP64 across warps in fixed order; writes out[k][idx].
// All threads must call; the caller separates consecutive calls by a barrier.
template <int NV>
__device__ __forceinline__ void tile_reduce_store(const float (&v)[NV], double* const (&out)[NV], long long idx) {
  __shared__ double red[NT / 32][NV];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    const float s = warp_sum(v[k]);
    if (lane == 0) red[warp][k] = (double)s;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double acc = 0.0;
    for (int wi = 0; wi < NT / 32; ++wi) acc += red[wi][threadIdx.x];
    out[threadIdx.x][idx] = acc;
  }
}

#define ELEMS(CNT, PER)                      \
  _Pragma("unroll") for (int p = 0; p < PER; ++p) \
    if (const int e = threadIdx.x + p * NT; (CNT) % NT == 0 || e < (CNT))

// ---------------------------------------------------------------- A_x: mu, r' -> x-FFT of mu and D mu -> T

template <int N>
__global__ void __launch_bounds__(NT, 2) k_a_x_pipe(Geom g, AgentScalars s, const float2* __restrict__ mu,
                                                 const float* __restrict__ rprev, float4* __restrict__ T,
                                                 const float2* __restrict__ tw, int ntiles) {
  constexpr int LX = variant_rows(N, 3), LT = 2 * LX, LD = N + 1;
  constexpr int CNT = LX * N, PER = (CNT + NT - 1) / NT;
  constexpr int STAGE = 2 * LT * LD + CNT;  // floats: two float2 arrays, then r'
  float* smem = reinterpret_cast<float*>(pipe_smem);
  auto issue = [&](int t, float* st) {
    float2* sm = reinterpret_cast<float2*>(st);
    float* rb = st + 2 * LT * LD;
    const long long e0 = (long long)t * CNT;
    ELEMS(CNT, PER) {
      const int line = e / N, i = e - line * N;
      cp8(&sm[line * LD + i], &mu[e0 + e]);
      cp4(&rb[e], &rprev[e0 + e]);
    }
  };
  int stage = 0, t = blockIdx.x;
  if (t < ntiles) issue(t, smem);
  cp_commit();
  for (; t < ntiles; t += gridDim.x) {
    if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x, smem + (stage ^ 1) * STAGE);
    cp_commit();
    cp_wait_prev();
    float* st = smem + stage * STAGE;
    float2* sm = reinterpret_cast<float2*>(st);
    const float* rb = st + 2 * LT * LD;
    ELEMS(CNT, PER) {  // each thread scales the elements it copied itself
      const int line = e / N, i = e - line * N;
      sm[(LX + line) * LD + i] = cscale(sm[line * LD + i], 1.0f / (rb[e] + s.floor));
    }
    __syncthreads();
    fft_tile<N, LT, NT, false>(sm, tw);
    const long long e0 = (long long)t * CNT;
    ELEMS(CNT, PER) {
      const int line = e / N, i = e - line * N;
      const float2 a = cscale(sm[line * LD + i], s.sc_x);
      const float2 b = cscale(sm[(LX + line) * LD + i], s.sc_x);
      T[e0 + e] = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    stage ^= 1;
  }
}

// ---------------------------------------------------------------- A_y: y-FFT of both halves of T (in place)

template <int N>
__global__ void __launch_bounds__(NT, 2) k_a_y_pipe(Geom g, AgentScalars s, float4* __restrict__ T,
                                                 const float2* __restrict__ tw, int ntiles) {
  constexpr int LCV = pipe_cols(N), LT = 2 * LCV, LD = N + 1;
  constexpr int CNT = LCV * N, PER = (CNT + NT - 1) / NT;
  constexpr int STAGE = 2 * LT * LD;
  float* smem = reinterpret_cast<float*>(pipe_smem);
  const int nbx = g.nx / LCV;
  auto tile_base = [&](int t) {
    const int bx = t % nbx, rest = t / nbx, z = rest % g.nz, l = rest / g.nz;
    return (long long)l * g.n + (long long)z * g.ny * g.nx + (long long)bx * LCV;
  };
  auto issue = [&](int t, float* st) {
    float2* sm = reinterpret_cast<float2*>(st);
    const long long base = tile_base(t);
    ELEMS(CNT, PER) {
      const int line = e % LCV, i = e / LCV;
      const float2* src = reinterpret_cast<const float2*>(T + base + (long long)i * g.nx + line);
      cp8(&sm[line * LD + i], src);
      cp8(&sm[(LCV + line) * LD + i], src + 1);
    }
  };
  int stage = 0, t = blockIdx.x;
  if (t < ntiles) issue(t, smem);
  cp_commit();
  for (; t < ntiles; t += gridDim.x) {
    if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x, smem + (stage ^ 1) * STAGE);
    cp_commit();
    cp_wait_prev();
    __syncthreads();
    float2* sm = reinterpret_cast<float2*>(smem + stage * STAGE);
    fft_tile<N, LT, NT, false>(sm, tw);
    const long long base = tile_base(t);
    ELEMS(CNT, PER) {
      const int line = e % LCV, i = e / LCV;
      const float2 a = cscale(sm[line * LD + i], s.sc_y);
      const float2 b = cscale(sm[(LCV + line) * LD + i], s.sc_y);
      T[base + (long long)i * g.nx + line] = make_float4(a.x, a.y, b.x, b.y);
    }
    __syncthreads();
    stage ^= 1;
  }
}

// ---------------------------------------------------------------- fused z pass

template <int N>
__global__ void __launch_bounds__(NT, 2) k_ab_z_pipe(Geom g, AgentScalars s, const float4* __restrict__ T,
                                                  const float2* __restrict__ y, const float* __restrict__ pupil,
                                                  const float* __restrict__ window, float2* __restrict__ U,
                                                  Partials pp, const float2* __restrict__ tw, int ntiles) {
  constexpr int LCV = pipe_cols(N), LT = 2 * LCV, LD = N + 1;
  constexpr int CNT = LCV * N, PER = (CNT + NT - 1) / NT;
  constexpr int STAGE = 2 * LT * LD + 2 * CNT;  // floats: two float2 arrays, then y
  float* smem = reinterpret_cast<float*>(pipe_smem);
  const int nbx = g.nx / LCV;
  const long long S = (long long)g.nx * g.ny;
  auto tile_base = [&](int t) {
    const int bx = t % nbx, rest = t / nbx, ky = rest % g.ny, l = rest / g.ny;
    return (long long)l * g.n + (long long)ky * g.nx + (long long)bx * LCV;
  };
  auto issue = [&](int t, float* st) {
    float2* sm = reinterpret_cast<float2*>(st);
    float2* yb = reinterpret_cast<float2*>(st + 2 * LT * LD);
    const long long base = tile_base(t);
    ELEMS(CNT, PER) {
      const int line = e % LCV, i = e / LCV;
      const long long gi = base + (long long)i * S + line;
      const float2* src = reinterpret_cast<const float2*>(T + gi);
      cp8(&sm[line * LD + i], src);
      cp8(&sm[(LCV + line) * LD + i], src + 1);
      cp8(&yb[e], &y[gi]);
    }
  };
  const float inv_nv = 1.0f / s.nv;
  int stage = 0, t = blockIdx.x;
  if (t < ntiles) issue(t, smem);
  cp_commit();
  for (; t < ntiles; t += gridDim.x) {
    if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x, smem + (stage ^ 1) * STAGE);
    cp_commit();
    cp_wait_prev();
    __syncthreads();
    float* st = smem + stage * STAGE;
    float2* sm = reinterpret_cast<float2*>(st);
    const float2* yb = reinterpret_cast<const float2*>(st + 2 * LT * LD);
    fft_tile<N, LT, NT, false>(sm, tw);
    const int bx = t % nbx, rest = t / nbx, ky = rest % g.ny, l = rest / g.ny;
    const int x0 = bx * LCV;
    // frequency-domain gradient: Fd = a (y - a M) / sigma_w^2 - P
    float acc[3] = {0.f, 0.f, 0.f};
    ELEMS(CNT, PER) {
      const int line = e % LCV, kz = e / LCV;
      const float2 M = cscale(sm[line * LD + kz], s.sc_z);
      const float2 P = cscale(sm[(LCV + line) * LD + kz], s.sc_z);
      const float av = __ldg(&pupil[ky * g.nx + x0 + line]) * __ldg(&window[kz]);
      const float2 yv = yb[e];
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
    fft_tile<N, LCV, NT, true>(sm, tw);
    const long long base = tile_base(t);
    ELEMS(CNT, PER) {
      const int line = e % LCV, i = e / LCV;
      U[base + (long long)i * S + line] = cscale(sm[line * LD + i], s.sc_z);
    }
    double* const outs[3] = {pp.s1, pp.s2, pp.s4};
    tile_reduce_store<3>(acc, outs, (long long)l * pp.pz + (long long)ky * nbx + bx);
    __syncthreads();
    stage ^= 1;
  }
}

// ---------------------------------------------------------------- B_y: inverse y-FFT of U (in place)

template <int N>
__global__ void __launch_bounds__(NT, 2) k_b_y_pipe(Geom g, float sc, float2* __restrict__ U,
                                                 const float2* __restrict__ tw, int ntiles) {
  constexpr int LCV = pipe_cols(N), LD = N + 1;
  constexpr int CNT = LCV * N, PER = (CNT + NT - 1) / NT;
  constexpr int STAGE = 2 * LCV * LD;
  float* smem = reinterpret_cast<float*>(pipe_smem);
  const int nbx = g.nx / LCV;
  auto tile_base = [&](int t) {
    const int bx = t % nbx, rest = t / nbx, z = rest % g.nz, l = rest / g.nz;
    return (long long)l * g.n + (long long)z * g.ny * g.nx + (long long)bx * LCV;
  };
  auto issue = [&](int t, float* st) {
    float2* sm = reinterpret_cast<float2*>(st);
    const long long base = tile_base(t);
    ELEMS(CNT, PER) {
      const int line = e % LCV, i = e / LCV;
      cp8(&sm[line * LD + i], &U[base + (long long)i * g.nx + line]);
    }
  };
  int stage = 0, t = blockIdx.x;
  if (t < ntiles) issue(t, smem);
  cp_commit();
  for (; t < ntiles; t += gridDim.x) {
    if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x, smem + (stage ^ 1) * STAGE);
    cp_commit();
    cp_wait_prev();
    __syncthreads();
    float2* sm = reinterpret_cast<float2*>(smem + stage * STAGE);
    fft_tile<N, LCV, NT, true>(sm, tw);
    const long long base = tile_base(t);
    ELEMS(CNT, PER) {
      const int line = e % LCV, i = e / LCV;
      U[base + (long long)i * g.nx + line] = cscale(sm[line * LD + i], sc);
    }
    __syncthreads();
    stage ^= 1;
  }
}

// ---------------------------------------------------------------- B_x: inverse x-FFT = d, S3 = sum |d|^2 D

template <int N>
__global__ void __launch_bounds__(NT, 2) k_b_x_pipe(Geom g, AgentScalars s, float2* __restrict__ U,
                                                 const float* __restrict__ rprev, double* __restrict__ s3, int px,
                                                 const float2* __restrict__ tw, int ntiles) {
  constexpr int LX = variant_rows(N, 3), LD = N + 1;
  constexpr int CNT = LX * N, PER = (CNT + NT - 1) / NT;
  constexpr int STAGE = 2 * LX * LD + CNT;  // floats: one float2 array, then r'
  float* smem = reinterpret_cast<float*>(pipe_smem);
  auto issue = [&](int t, float* st) {
    float2* sm = reinterpret_cast<float2*>(st);
    float* rb = st + 2 * LX * LD;
    const long long e0 = (long long)t * CNT;
    ELEMS(CNT, PER) {
      const int line = e / N, i = e - line * N;
      cp8(&sm[line * LD + i], &U[e0 + e]);
      cp4(&rb[e], &rprev[e0 + e]);
    }
  };
  const long long bpl = g.n / CNT;  // tiles per look
  int stage = 0, t = blockIdx.x;
  if (t < ntiles) issue(t, smem);
  cp_commit();
  for (; t < ntiles; t += gridDim.x) {
    if (t + (int)gridDim.x < ntiles) issue(t + gridDim.x, smem + (stage ^ 1) * STAGE);
    cp_commit();
    cp_wait_prev();
    __syncthreads();
    float* st = smem + stage * STAGE;
    float2* sm = reinterpret_cast<float2*>(st);
    const float* rb = st + 2 * LX * LD;
    fft_tile<N, LX, NT, true>(sm, tw);
    const long long e0 = (long long)t * CNT;
    float acc[1] = {0.f};
    ELEMS(CNT, PER) {
      const int line = e / N, i = e - line * N;
      const float2 v = cscale(sm[line * LD + i], s.sc_x);
      acc[0] += cabs2(v) / (rb[e] + s.floor);
      U[e0 + e] = v;
    }
    const long long look = t / bpl;
    double* const outs[1] = {s3};
    tile_reduce_store<1>(acc, outs, look * px + (t - look * bpl));
    __syncthreads();
    stage ^= 1;
  }
}

#undef ELEMS

template <class F>
cudaError_t by_len(int N, F&& f) {
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

// Persistent grid: resident CTAs per SM x SMs, at most one CTA per tile.
template <class K>
cudaError_t persistent_grid(K kern, size_t smem, int ntiles, unsigned* grid) {
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, occ = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, NT, smem)) != cudaSuccess) return e;
  if (occ < 1) return cudaErrorInvalidConfiguration;
  const long long want = (long long)occ * sms;
  *grid = (unsigned)(ntiles < want ? ntiles : want);
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_pipe_pass(int pass, const Geom& g, const AgentScalars& s, const float2* mu, const float* rprev,
                             const float2* y, const float* pupil, const float* window, float4* T, float2* U,
                             Partials& p, const float2* tw, cudaStream_t st) {
  unsigned grid = 0;
  switch (pass) {
    case 0:
      return by_len(g.nx, [&](auto NC) -> cudaError_t {
        constexpr int N = decltype(NC)::value, LX = variant_rows(N, 3);
        const size_t smem = 2 * sizeof(float) * (2 * 2 * LX * (N + 1) + LX * N);
        const int ntiles = (int)((long long)g.L * g.nz * g.ny / LX);
        cudaError_t e = persistent_grid(k_a_x_pipe<N>, smem, ntiles, &grid);
        if (e != cudaSuccess) return e;
        k_a_x_pipe<N><<<grid, NT, smem, st>>>(g, s, mu, rprev, T, tw, ntiles);
        return cudaGetLastError();
      });
    case 1:
      return by_len(g.ny, [&](auto NC) -> cudaError_t {
        constexpr int N = decltype(NC)::value, LCV = pipe_cols(N);
        const size_t smem = 2 * sizeof(float) * (2 * 2 * LCV * (N + 1));
        const int ntiles = (g.nx / LCV) * g.nz * g.L;
        cudaError_t e = persistent_grid(k_a_y_pipe<N>, smem, ntiles, &grid);
        if (e != cudaSuccess) return e;
        k_a_y_pipe<N><<<grid, NT, smem, st>>>(g, s, T, tw, ntiles);
        return cudaGetLastError();
      });
    case 2:
      return by_len(g.nz, [&](auto NC) -> cudaError_t {
        constexpr int N = decltype(NC)::value, LCV = pipe_cols(N);
        const size_t smem = 2 * sizeof(float) * (2 * 2 * LCV * (N + 1) + 2 * LCV * N);
        const int ntiles = (g.nx / LCV) * g.ny * g.L;
        p.pz = (g.nx / LCV) * g.ny;
        cudaError_t e = persistent_grid(k_ab_z_pipe<N>, smem, ntiles, &grid);
        if (e != cudaSuccess) return e;
        k_ab_z_pipe<N><<<grid, NT, smem, st>>>(g, s, T, y, pupil, window, U, p, tw, ntiles);
        return cudaGetLastError();
      });
    case 3:
      return by_len(g.ny, [&](auto NC) -> cudaError_t {
        constexpr int N = decltype(NC)::value, LCV = pipe_cols(N);
        const size_t smem = 2 * sizeof(float) * (2 * LCV * (N + 1));
        const int ntiles = (g.nx / LCV) * g.nz * g.L;
        cudaError_t e = persistent_grid(k_b_y_pipe<N>, smem, ntiles, &grid);
        if (e != cudaSuccess) return e;
        k_b_y_pipe<N><<<grid, NT, smem, st>>>(g, s.sc_y, U, tw, ntiles);
        return cudaGetLastError();
      });
    case 4:
      return by_len(g.nx, [&](auto NC) -> cudaError_t {
        constexpr int N = decltype(NC)::value, LX = variant_rows(N, 3);
        const size_t smem = 2 * sizeof(float) * (2 * LX * (N + 1) + LX * N);
        const int ntiles = (int)((long long)g.L * g.nz * g.ny / LX);
        p.px = (int)((long long)g.nz * g.ny / LX);
        cudaError_t e = persistent_grid(k_b_x_pipe<N>, smem, ntiles, &grid);
        if (e != cudaSuccess) return e;
        k_b_x_pipe<N><<<grid, NT, smem, st>>>(g, s, U, rprev, p.s3, p.px, tw, ntiles);
        return cudaGetLastError();
      });
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace clamp
