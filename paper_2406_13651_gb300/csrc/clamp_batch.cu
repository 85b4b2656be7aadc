// clamp_batch.cu -- many CLAMP reconstructions in one CUDA graph launch.
//
// Each scene becomes an independent branch of one captured graph: a fork from the
// capture origin stream to a per-scene stream, the Alg. 2 initialisation and all its
// iterations, and a join back.  One cudaGraphLaunch then runs the whole batch; the
// branches' kernels overlap on the GPU, so small volumes fill it together.  A one-thread
// kernel stamps the GPU global timer at the start of the graph and at the end of every
// branch (events recorded inside a graph cannot be timed).
#include "../../include/clamp.h"
#include "clamp_kernels.cuh"
#include "clamp_internal.cuh"
#include "denoise.cuh"

#include <array>
#include <string>
#include <vector>

using namespace clamp;

__global__ void k_stamp(unsigned long long* slot) {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  *slot = t;
}

struct clamp_batch {
  unsigned long long* stamps = nullptr;  // device [count + 1]: start, then each scene's end (ns)
  std::vector<clamp_scene> scenes;
  std::vector<size_t> ws_off;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev_end;
  std::vector<cudaEvent_t> ev_fork;
  cudaEvent_t ev_start = nullptr;
  cudaStream_t origin = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  void* ws = nullptr;
  const clamp_denoiser* den = nullptr;
};

extern "C" size_t clamp_batch_workspace_size(const clamp_scene* scenes, int32_t count, const clamp_denoiser* den) {
  if (!scenes || count < 1) return 0;
  size_t total = 0;
  for (int i = 0; i < count; ++i) {
    const size_t b = clamp_reconstruct_workspace_size(&scenes[i].p, den);
    if (b == 0) return 0;
    total += (b + 255) & ~(size_t)255;
  }
  return total;
}

extern "C" void clamp_batch_destroy(clamp_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  for (auto s : b->streams) cudaStreamDestroy(s);
  for (auto e : b->ev_end) cudaEventDestroy(e);
  for (auto e : b->ev_fork) cudaEventDestroy(e);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->stamps) cudaFree(b->stamps);
  if (b->origin) cudaStreamDestroy(b->origin);
  delete b;
}

extern "C" clamp_status clamp_batch_create(const clamp_scene* scenes, int32_t count, const clamp_denoiser* den,
                                           void* ws, size_t ws_bytes, clamp_batch** out) {
  if (!out || !scenes || count < 1 || !den) return api_fail(CLAMP_EINVAL, "clamp_batch_create: bad arguments");
  *out = nullptr;
  const size_t need = clamp_batch_workspace_size(scenes, count, den);
  if (need == 0) return api_fail(CLAMP_EINVAL, "clamp_batch_create: a scene has invalid parameters");
  if (!ws || ws_bytes < need || ((uintptr_t)ws & 255))
    return api_fail(CLAMP_ENOMEM, "clamp_batch_create: workspace %zu bytes < %zu needed (256-byte aligned)", ws_bytes,
                    need);
  for (int i = 0; i < count; ++i) {
    const clamp_scene& sc = scenes[i];
    if (!sc.y || !sc.pupil || !sc.window || !sc.r_out)
      return api_fail(CLAMP_EINVAL, "clamp_batch_create: scene %d has a NULL buffer", i);
    if (sc.p.max_iters < 1) return api_fail(CLAMP_EINVAL, "clamp_batch_create: scene %d has max_iters < 1", i);
    if (!denoise_supports(den, sc.p.nx, sc.p.ny, sc.p.nz))
      return api_fail(CLAMP_EUNSUPPORTED, "clamp_batch_create: the prior agent does not support scene %d", i);
  }
  clamp_status st = api_ensure_device();
  if (st != CLAMP_OK) return st;
  clamp_batch* b = new clamp_batch();
  b->scenes.assign(scenes, scenes + count);
  b->ws = ws;
  b->den = den;
  size_t off = 0;
  for (int i = 0; i < count; ++i) {
    b->ws_off.push_back(off);
    off += (clamp_reconstruct_workspace_size(&scenes[i].p, den) + 255) & ~(size_t)255;
  }
  auto cu = [&](cudaError_t e, const char* what) -> bool {
    if (e == cudaSuccess) return true;
    api_fail(CLAMP_ECUDA, "clamp_batch_create: %s: %s", what, cudaGetErrorString(e));
    return false;
  };
  bool ok = cu(cudaStreamCreateWithFlags(&b->origin, cudaStreamNonBlocking), "stream") &&
            cu(cudaEventCreateWithFlags(&b->ev_start, cudaEventDisableTiming), "event") &&
            cu(cudaMalloc(&b->stamps, sizeof(unsigned long long) * (count + 1)), "timer slots");
  for (int i = 0; ok && i < count; ++i) {
    cudaStream_t s;
    cudaEvent_t e1, e2;
    ok = cu(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking), "stream") &&
         cu(cudaEventCreateWithFlags(&e1, cudaEventDisableTiming), "event") &&
         cu(cudaEventCreateWithFlags(&e2, cudaEventDisableTiming), "event");
    if (ok) {
      b->streams.push_back(s);
      b->ev_end.push_back(e1);
      b->ev_fork.push_back(e2);
    }
  }
  // Everything that synchronises (aperture statistics) happens before the capture, and one
  // un-captured iteration per scene loads every kernel and sets its launch attributes.
  std::vector<ReconPlan> plans(count);
  std::vector<std::array<int, 4>> tuned;
  for (int i = 0; ok && i < count; ++i) {
    st = recon_prepare(&b->scenes[i].p, b->scenes[i].pupil, b->scenes[i].window, b->streams[i], &plans[i]);
    const clamp_params& sp = b->scenes[i].p;
    const std::array<int, 4> key{sp.nx, sp.ny, sp.nz, sp.looks};
    bool seen = false;
    for (auto& k : tuned) seen |= (k == key);
    if (st == CLAMP_OK && !seen) {   // one autotuning run per distinct geometry, on this scene's agent scratch
      char* agent_ws = static_cast<char*>(ws) + b->ws_off[i] + recon_agent_offset(&sp, den);
      st = autotune_agent(&sp, plans[i], b->scenes[i].y, b->scenes[i].pupil, b->scenes[i].window, agent_ws,
                          b->streams[i], nullptr);
      tuned.push_back(key);
    }
    if (st == CLAMP_OK) {
      clamp_params one = b->scenes[i].p;
      one.max_iters = 1;
      st = recon_enqueue(&one, plans[i], b->scenes[i].y, b->scenes[i].pupil, b->scenes[i].window, den, nullptr,
                         b->scenes[i].r_out, static_cast<char*>(ws) + b->ws_off[i], b->streams[i]);
    }
    if (st == CLAMP_OK && cudaStreamSynchronize(b->streams[i]) != cudaSuccess)
      st = api_fail(CLAMP_ECUDA, "clamp_batch_create: warm-up of scene %d failed", i);
    if (st != CLAMP_OK) {
      clamp_batch_destroy(b);
      return st;
    }
  }
  if (ok) ok = cu(cudaStreamBeginCapture(b->origin, cudaStreamCaptureModeThreadLocal), "begin capture");
  if (ok) {
    k_stamp<<<1, 1, 0, b->origin>>>(b->stamps);
    ok = cu(cudaGetLastError(), "start stamp");
  }
  for (int i = 0; ok && i < count; ++i) {
    const clamp_scene& sc = b->scenes[i];
    ok = cu(cudaEventRecord(b->ev_fork[i], b->origin), "fork") &&
         cu(cudaStreamWaitEvent(b->streams[i], b->ev_fork[i], 0), "fork");
    if (!ok) break;
    st = recon_enqueue(&sc.p, plans[i], sc.y, sc.pupil, sc.window, den, nullptr, sc.r_out,
                       static_cast<char*>(ws) + b->ws_off[i], b->streams[i]);
    if (st != CLAMP_OK) ok = false;
    if (ok) {
      k_stamp<<<1, 1, 0, b->streams[i]>>>(b->stamps + 1 + i);
      ok = cu(cudaGetLastError(), "end stamp") && cu(cudaEventRecord(b->ev_end[i], b->streams[i]), "event record") &&
           cu(cudaStreamWaitEvent(b->origin, b->ev_end[i], 0), "join");
    }
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(b->origin, &g);
  if (ok) ok = cu(ec, "end capture");
  b->graph = g;
  if (ok) ok = cu(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
  if (!ok) {
    clamp_batch_destroy(b);
    return st != CLAMP_OK ? st : CLAMP_ECUDA;
  }
  *out = b;
  return CLAMP_OK;
}

extern "C" clamp_status clamp_batch_launch(clamp_batch* b, void* stream) {
  if (!b || !b->exec) return api_fail(CLAMP_EINVAL, "clamp_batch_launch: no plan");
  const cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return api_fail(CLAMP_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
  return CLAMP_OK;
}

extern "C" clamp_status clamp_batch_latencies(clamp_batch* b, void* stream, float* latency_ms) {
  if (!b || !latency_ms) return api_fail(CLAMP_EINVAL, "clamp_batch_latencies: bad arguments");
  std::vector<unsigned long long> t(b->scenes.size() + 1);
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e == cudaSuccess)
    e = cudaMemcpy(t.data(), b->stamps, sizeof(unsigned long long) * t.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return api_fail(CLAMP_ECUDA, "clamp_batch_latencies: %s", cudaGetErrorString(e));
  for (size_t i = 0; i < b->scenes.size(); ++i) latency_ms[i] = (float)((double)(t[i + 1] - t[0]) * 1e-6);
  return CLAMP_OK;
}

extern "C" clamp_status clamp_batch_residuals(clamp_batch* b, void* stream, double* ce) {
  if (!b || !ce) return api_fail(CLAMP_EINVAL, "clamp_batch_residuals: bad arguments");
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  for (size_t i = 0; e == cudaSuccess && i < b->scenes.size(); ++i) {
    const double* ring = recon_ce_ring(&b->scenes[i].p, b->den, static_cast<char*>(b->ws) + b->ws_off[i]);
    e = cudaMemcpy(&ce[i], ring + b->scenes[i].p.max_iters - 1, sizeof(double), cudaMemcpyDeviceToHost);
  }
  if (e != cudaSuccess) return api_fail(CLAMP_ECUDA, "clamp_batch_residuals: %s", cudaGetErrorString(e));
  return CLAMP_OK;
}
