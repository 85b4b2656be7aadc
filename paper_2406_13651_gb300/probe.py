"""Profiling driver for the CLAMP kernels (one GPU; no timing contract, for ncu captures).

  python -m paper_2406_13651_gb300.probe agent --shape 256,256,128 --looks 4 --iters 3 \\
      [--schedule auto|band|full] [--prior gauss|cnn-bf16|cnn-fp32]
  python -m paper_2406_13651_gb300.probe prior --shape 256,256,64 --dtype bf16 --reps 3
  python -m paper_2406_13651_gb300.probe e2e --shape 256,256,128 --looks 32 --iters 20 --prior cnn-bf16
  python -m paper_2406_13651_gb300.probe unet --shape 64,64,32 --batch 24 --reps 3 [--cuda-cores]

``agent`` runs ``--iters`` CLAMP iterations (after one untimed iteration) on seeded random
data with a circular pupil of radius 0.35 Nyquist and a Hann range window; ``prior`` runs
the residual CNN prior agent (8 x 48 BF16 or 5 x 32 FP32) on a seeded random volume;
``e2e`` splits one clamp_reconstruct_host call on pinned host buffers into its parts: a
plain upload of y, a call with no iterations (upload, initialisation, download) and a call
with ``--iters`` iterations (wall clock); ``unet`` times the BF16 16/32/64 U-Net's forward
pass and training step (forward, backward, Adam) on a seeded batch, with its 3x3x3 convs
on the tensor cores or (``--cuda-cores``) on the CUDA cores.  Each prints one JSON line
with the mean milliseconds per repetition.
"""
from __future__ import annotations

import argparse
import json


def main(argv=None) -> int:
    import numpy as np
    import torch

    from . import build as B
    from . import clamp as C
    from . import inputs as I

    ap = argparse.ArgumentParser()
    ap.add_argument("what", choices=["agent", "prior", "e2e", "unet"])
    ap.add_argument("--shape", default="256,256,128", help="nx,ny,nz")
    ap.add_argument("--looks", type=int, default=4)
    ap.add_argument("--iters", type=int, default=3)
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--schedule", choices=["auto", "band", "full"], default="auto")
    ap.add_argument("--prior", choices=["gauss", "cnn-bf16", "cnn-fp32"], default="gauss")
    ap.add_argument("--band-row", type=int, choices=[-1, 0, 1, 2], default=-1,
                    help="band-limited row pass variant (0 default row tile, 1 half-height tiles, "
                         "2 mu and r' read late; -1 autotune)")
    ap.add_argument("--dtype", choices=["fp32", "bf16"], default="bf16")
    ap.add_argument("--batch", type=int, default=24)
    ap.add_argument("--cuda-cores", action="store_true", help="unet: 3x3x3 convs on the CUDA cores")
    a = ap.parse_args(argv)
    B.build()
    C.load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    nx, ny, nz = (int(v) for v in a.shape.split(","))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if a.what == "unet":
        ch = (16, 32, 64)
        net = C.UNet(*ch, params=I.unet_params(ch, seed=1), dtype="bf16")
        net.set_tensor_cores(not a.cuda_cores)
        g = torch.Generator(device=dev).manual_seed(3)
        x = torch.rand((a.batch, nz, ny, nx), generator=g, device=dev) * 2
        t = torch.rand((a.batch, nz, ny, nx), generator=g, device=dev)
        loss = torch.zeros((), dtype=torch.float64, device=dev)
        out = {"probe": "unet", "shape": [nx, ny, nz], "batch": a.batch, "tensor_cores": not a.cuda_cores}
        for name, fn in (("forward", lambda: net.forward(x)),
                         ("train_step", lambda: (net.backward(x, t, loss), net.adam(1e-3)))):
            fn()
            torch.cuda.synchronize()
            e0.record()
            for _ in range(a.reps):
                fn()
            e1.record()
            torch.cuda.synchronize()
            out[name + "_ms"] = e0.elapsed_time(e1) / a.reps
        net.check()
        print(json.dumps(out), flush=True)
        return 0
    if a.what == "prior":
        layers, ch = (8, 48) if a.dtype == "bf16" else (5, 32)
        ws_, bs_ = I.cnn_weights(layers, ch, seed=1)
        den = C.Denoiser.cnn(ws_, bs_, a.dtype)
        x = torch.rand((nz, ny, nx), generator=torch.Generator(device=dev).manual_seed(3), device=dev)
        out = torch.empty_like(x)
        wsb = C._ws(den.workspace_size(nx, ny, nz))
        C.denoise(den, x, out, ws=wsb)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(a.reps):
            C.denoise(den, x, out, ws=wsb)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / a.reps
        macs = 27 * (ch + (layers - 2) * ch * ch + ch)
        print(json.dumps({"probe": "prior", "shape": [nx, ny, nz], "dtype": a.dtype, "ms": ms,
                          "tflops": 2 * macs * nx * ny * nz / ms / 1e9}), flush=True)
        return 0
    L = a.looks
    if a.what == "e2e":
        import ctypes
        import time
        lib = C.load()
        pupil_pin = torch.from_numpy(I.circular_pupil(nx, ny, 0.35)).pin_memory()
        window_pin = torch.from_numpy(I.hann_window(nz)).pin_memory()
        y_pin = torch.empty((L, nz, ny, nx), dtype=torch.complex64, pin_memory=True)
        y_pin.copy_(torch.complex(torch.randn(y_pin.shape), torch.randn(y_pin.shape)) *
                    (pupil_pin[None, None] * window_pin[None, :, None, None]))
        rout_pin = torch.empty((nz, ny, nx), dtype=torch.float32, pin_memory=True)
        if a.prior == "gauss":
            den = C.Denoiser.gauss(0.8)
        else:
            dt = a.prior.split("-")[1]
            layers, ch = (8, 48) if dt == "bf16" else (5, 32)
            w_, b_ = I.cnn_weights(layers, ch, seed=1)
            den = C.Denoiser.cnn(w_, b_, dt)
        st = torch.cuda.current_stream()
        out = {"probe": "e2e", "shape": [nx, ny, nz], "looks": L, "prior": a.prior, "iters": a.iters}
        yd = torch.empty(y_pin.shape, dtype=y_pin.dtype, device=dev)
        for name, iters in (("upload_only", None), ("zero_iterations", 0), ("with_iterations", a.iters)):
            def call():
                if iters is None:
                    yd.copy_(y_pin, non_blocking=True)
                    return
                p = C.make_params(nx, ny, nz, L, 1e-3, 1e-4, max_iters=iters)
                rep = C.Report(0, 0, 0.0, 0.0, None, None)
                C._check(lib.clamp_reconstruct_host(ctypes.byref(p), y_pin.data_ptr(), pupil_pin.data_ptr(),
                                                    window_pin.data_ptr(), den.handle, None, rout_pin.data_ptr(),
                                                    ctypes.byref(rep), st.cuda_stream), "clamp_reconstruct_host")
            call()
            torch.cuda.synchronize()
            ts, gs = [], []
            for _ in range(a.reps):
                g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                t0 = time.perf_counter()
                g0.record(st)
                call()
                g1.record(st)
                torch.cuda.synchronize()
                ts.append((time.perf_counter() - t0) * 1e3)
                gs.append(g0.elapsed_time(g1))
            out[name + "_ms"] = sum(ts) / len(ts)
            out[name + "_ms_each"] = [round(t, 2) for t in ts]
            out[name + "_gpu_ms_each"] = [round(t, 2) for t in gs]   # events on the stream around the call
        print(json.dumps(out), flush=True)
        return 0
    pupil = torch.from_numpy(I.circular_pupil(nx, ny, 0.35)).to(dev)
    window = torch.from_numpy(I.hann_window(nz)).to(dev)
    flags = {"auto": 0, "band": C.FLAG_BAND_SPECTRUM, "full": C.FLAG_FULL_SPECTRUM}[a.schedule]
    p = C.make_params(nx, ny, nz, L, 1e-3, 1e-4, flags=flags)
    g = torch.Generator(device=dev).manual_seed(5)
    shape = (L, nz, ny, nx)
    y = torch.complex(torch.randn(shape, generator=g, device=dev), torch.randn(shape, generator=g, device=dev))
    y *= (pupil[None, None] * window[None, :, None, None])
    if a.prior == "gauss":
        den = C.Denoiser.gauss(0.8)
    else:
        dt = a.prior.split("-")[1]
        layers, ch = (8, 48) if dt == "bf16" else (5, 32)
        w_, b_ = I.cnn_weights(layers, ch, seed=1)
        den = C.Denoiser.cnn(w_, b_, dt)
    if a.band_row < 0:
        C.autotune(p, y, pupil, window)
    else:
        C.autotune_set_band(p, a.band_row)
    mu, r, w = C.init(p, y, pupil, window)
    wbar = torch.empty((nz, ny, nx), device=dev)
    ws = C.iterate_workspace(p, den)
    C.iterate(p, 1, 1, y, pupil, window, den, mu, r, w, wbar, ws=ws)
    torch.cuda.synchronize()
    e0.record()
    C.iterate(p, 2, a.iters, y, pupil, window, den, mu, r, w, wbar, ws=ws)
    e1.record()
    torch.cuda.synchronize()
    sched = C.agent_schedule(p, pupil, window)
    print(json.dumps({"probe": "agent", "shape": [nx, ny, nz], "looks": L, "schedule": sched, "prior": a.prior,
                      "band_row": a.band_row,
                      "ms_per_iteration": e0.elapsed_time(e1) / a.iters}), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
