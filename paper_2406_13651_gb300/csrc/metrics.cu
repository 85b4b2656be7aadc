// metrics.cu -- point-cloud metrics of a reconstruction (Sec. IV-B, Eqs. pc-distance, nrmse).
//
// P = voxels of r_hat above the threshold (the noise floor sigma_w^2 / alpha), Q = voxels
// of r_true above zero; both carry voxel-grid coordinates.  For every p in P the nearest
// q in Q is found by scanning Chebyshev shells k = 0, 1, ... around p until k exceeds the
// best Euclidean distance found (every point of a later shell is at least k away); ties
// in distance go to the smallest linear index.  Points farther than max_dist are removed
// (false positives).  Sums are FP64: block partials, then one fixed-order final pass.
#include "../../include/clamp.h"
#include "clamp_internal.cuh"

#include <math.h>

namespace clamp {
namespace {

constexpr int MT = 256;
constexpr int kMetricBlocks = 152 * 8;
constexpr int kSums = 7;   // kept, removed, sum d, sum rh*rq, sum rh^2, sum rq^2, sum rq*rq (unused pad)

__global__ void __launch_bounds__(MT) k_pc_metrics(const float* __restrict__ rh, const float* __restrict__ rt, int nx,
                                                   int ny, int nz, float thr, float max_dist, double* __restrict__ part) {
  const long long plane = (long long)nx * ny, n = plane * nz;
  const int kmax = (int)ceilf(max_dist);
  const float md2 = max_dist * max_dist;
  double acc[6] = {0, 0, 0, 0, 0, 0};
  for (long long v = (long long)blockIdx.x * MT + threadIdx.x; v < n; v += (long long)gridDim.x * MT) {
    const float rp = rh[v];
    if (!(rp > thr)) continue;
    const int x = (int)(v % nx), y = (int)((v / nx) % ny), z = (int)(v / plane);
    int best_d2 = 0x7fffffff;
    long long best_i = -1;
    for (int k = 0; k <= kmax; ++k) {
      if (best_i >= 0 && (long long)k * k > best_d2) break;   // later shells are all farther
      for (int dz = -k; dz <= k; ++dz) {
        const int zz = z + dz;
        if (zz < 0 || zz >= nz) continue;
        for (int dy = -k; dy <= k; ++dy) {
          const int yy = y + dy;
          if (yy < 0 || yy >= ny) continue;
          const bool face = (dz == -k || dz == k || dy == -k || dy == k);
          const int step = face ? 1 : 2 * k;   // interior rows of the shell: only dx = +-k
          for (int dx = -k; dx <= k; dx += (k == 0 ? 1 : step)) {
            const int xx = x + dx;
            if (xx < 0 || xx >= nx) continue;
            const long long i = (long long)zz * plane + (long long)yy * nx + xx;
            if (!(rt[i] > 0.f)) continue;
            const int d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best_d2 || (d2 == best_d2 && i < best_i)) {
              best_d2 = d2;
              best_i = i;
            }
          }
        }
      }
    }
    if (best_i >= 0 && (float)best_d2 <= md2) {
      const double rq = rt[best_i];
      acc[0] += 1.0;
      acc[2] += sqrt((double)best_d2);
      acc[3] += (double)rp * rq;
      acc[4] += (double)rp * rp;
      acc[5] += rq * rq;
    } else {
      acc[1] += 1.0;
    }
  }
  __shared__ double red[MT];
  for (int k = 0; k < 6; ++k) {
    red[threadIdx.x] = acc[k];
    __syncthreads();
    for (int o = MT / 2; o > 0; o >>= 1) {
      if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[(long long)k * gridDim.x + blockIdx.x] = red[0];
    __syncthreads();
  }
}

__global__ void k_pc_final(const double* part, int nb, double* sums) {
  const int k = threadIdx.x;
  if (k < 6) {
    double a = 0.0;
    for (int b = 0; b < nb; ++b) a += part[(long long)k * nb + b];
    sums[k] = a;
  }
}

}  // namespace
}  // namespace clamp

extern "C" size_t clamp_point_cloud_workspace_size(void) {
  return sizeof(double) * (6 * (size_t)clamp::kMetricBlocks + 8);
}

extern "C" clamp_status clamp_point_cloud_metrics(const float* r_hat, const float* r_true, int32_t nx, int32_t ny,
                                                  int32_t nz, float threshold, float max_dist, double* out,
                                                  void* ws, size_t ws_bytes, void* stream) {
  if (!r_hat || !r_true || !out || nx < 1 || ny < 1 || nz < 1 || !(max_dist >= 0.f) || max_dist > 64.f)
    return api_fail(CLAMP_EINVAL, "clamp_point_cloud_metrics: bad arguments (max_dist must be in [0, 64])");
  if (!ws || ws_bytes < clamp_point_cloud_workspace_size())
    return api_fail(CLAMP_ENOMEM, "clamp_point_cloud_metrics: workspace too small");
  cudaStream_t st = (cudaStream_t)stream;
  double* part = static_cast<double*>(ws);
  double* sums = part + 6 * clamp::kMetricBlocks;
  const long long n = (long long)nx * ny * nz;
  long long blocks = (n + clamp::MT - 1) / clamp::MT;
  if (blocks > clamp::kMetricBlocks) blocks = clamp::kMetricBlocks;
  clamp::k_pc_metrics<<<(unsigned)blocks, clamp::MT, 0, st>>>(r_hat, r_true, nx, ny, nz, threshold, max_dist, part);
  clamp::k_pc_final<<<1, 32, 0, st>>>(part, (int)blocks, sums);
  double h[6];
  cudaError_t e = cudaMemcpyAsync(h, sums, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return api_fail(CLAMP_ECUDA, "clamp_point_cloud_metrics: %s", cudaGetErrorString(e));
  const double kept = h[0], removed = h[1], total = kept + removed;
  const double beta = h[4] > 0 ? h[3] / h[4] : 0.0;                 // argmin_b sum (b rh - rq)^2
  const double resid = h[5] - (h[4] > 0 ? h[3] * h[3] / h[4] : 0.0);  // sum (beta rh - rq)^2
  out[0] = kept > 0 ? h[2] / kept : 0.0;                            // mean Euclidean distance (voxels)
  out[1] = total > 0 ? removed / total : 0.0;                       // false positive rate
  out[2] = h[5] > 0 ? sqrt(fmax(resid, 0.0) / h[5]) : 0.0;           // NRMSE(beta* r_hat, r)
  out[3] = kept;
  out[4] = removed;
  out[5] = beta;
  return CLAMP_OK;
}
