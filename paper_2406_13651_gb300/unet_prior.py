"""The 3D U-Net prior agent (Sec. III-C): a U-Net trained as a denoiser of 3D surface
images with 10 % additive white Gaussian noise, used as the prior agent H of Alg. 2 in
place of the Gaussian smoother or a random CNN.

The paper trains on ShapeNet renderings (not available); here the clean images are the
seeded synthetic scenes (column surfaces and facets, 32^3 patches), the noise is drawn on
the device, and training runs on the library's U-Net kernels with Adam (Sec. III-C
recipe: batch 24, MSE, decaying learning rate, best-validation weights).  As a prior,
H(w) = m max(U(w / m), floor) with m = sum(w) / (nx ny) (clamp_denoiser_create_unet).

    python -m paper_2406_13651_gb300.unet_prior --scenes 2000 --steps 3000 \\
        --out paper_2406_13651_gb300/weights/unet_prior.npz
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

from . import clamp as C
from . import inputs as I
from . import warmstart as W

CHANNELS = (16, 32, 64)
NOISE = 0.1          # standard deviation of the additive noise, on reflectance in [0, 1]
WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_prior.npz")


def denoiser_pairs(count: int, dev, seed: int = 31, n: int = 32, noise: float = NOISE) -> W.Dataset:
    """x = (clean + noise N(0, 1)) / m, t = clean / m with m = sum(noisy) / n^2 per sample."""
    import torch
    t0 = time.perf_counter()
    clean = torch.from_numpy(I.prior_training_scenes(count, seed, n)).to(dev)
    gen = torch.Generator(device=dev).manual_seed(seed)
    noisy = clean + noise * torch.randn(clean.shape, generator=gen, device=dev)
    C.unet_normalize(noisy, clean)
    torch.cuda.synchronize()
    return W.Dataset(noisy, clean, np.zeros(count), time.perf_counter() - t0)


def scene_for_eval(spec: dict, dev):
    """(params, y, pupil, window, r_true) of one held-out reconstruction problem."""
    p, y, pu, wi = W.scene_data(spec, dev)
    r_true = I.batch_scene(spec, with_draws=False).r_true
    return p, y, pu, wi, r_true


def compare_priors(net: C.UNet, specs, dev, iters: int = 150, tol: float = 1e-3) -> list:
    """CLAMP with the Gaussian prior and with the U-Net prior on the same data: iterations to
    CE <= tol (0: not reached), final CE, PSNR (Sec. IV-B) and point-cloud metrics."""
    import torch
    out = []
    gauss = C.Denoiser.gauss(0.8)
    unet = C.Denoiser.unet(net)
    for sp in specs:
        p, y, pu, wi, r_true = scene_for_eval(sp, dev)
        q = C.make_params(p.nx, p.ny, p.nz, p.looks, p.noise_var, p.prox_var, max_iters=iters)
        alpha = float(np.mean(wi.cpu().numpy().astype(np.float64) ** 2) * np.mean(pu.cpu().numpy().astype(np.float64) ** 2))
        rt = torch.from_numpy(r_true.astype(np.float32)).to(dev)
        row = {"spec": {k: sp[k] for k in ("nx", "ny", "nz", "looks", "radius", "snr", "seed")}}
        for name, den in (("gauss", gauss), ("unet", unet)):
            res = C.reconstruct(q, y, pu, wi, den)
            rh = res.r.cpu().numpy()
            b = float(rh.ravel().astype(np.float64) @ r_true.ravel()) / max(float((rh.astype(np.float64) ** 2).sum()), 1e-300)
            pc = C.point_cloud_metrics(res.r, rt, p.noise_var / alpha / b, 3.0 * 1.22 / sp["radius"])
            row[name] = dict(psnr=W.psnr(rh, r_true), iters_to_tol=W.first_below(res.ce_hist, tol),
                             ce_final=float(res.ce_hist[-1]), point_cloud=pc)
        out.append(row)
    return out


def eval_specs(count: int = 3, seed: int = 57, nx: int = 64, nz: int = 32, looks: int = 16, snr: float = 7.5):
    specs = I.warmstart_specs(count, seed=seed, nx=nx, ny=nx, nz=nz, looks=looks, iters=150)
    for sp in specs:
        sp["snr"] = snr
    return specs


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--dtype", choices=("bf16", "fp32"), default="bf16")
    ap.add_argument("--out", default="")
    ap.add_argument("--eval", type=int, default=3, help="held-out reconstructions to compare priors on")
    a = ap.parse_args(argv)
    import torch
    from . import build as B
    B.build()
    dev = torch.device("cuda")
    log = lambda s: print(s, file=sys.stderr, flush=True)   # noqa: E731
    data = denoiser_pairs(a.scenes, dev)
    n_train = a.scenes - max(1, a.scenes // 10)
    xv, tv = data.x[n_train:].double(), data.t[n_train:].double()
    identity = float(((xv - tv) ** 2).mean())
    net = C.UNet(*CHANNELS, params=I.unet_params(CHANNELS, seed=7), dtype=a.dtype)
    tl = W.train(net, data, n_train, W.TrainConfig(steps=a.steps, lr=a.lr), log=log)
    summary = dict(scenes=a.scenes, patch=32, noise=NOISE, steps=a.steps, lr=a.lr, dtype=a.dtype,
                   train_seconds=round(tl.seconds, 1), best_val=tl.best_val, best_step=tl.best_step,
                   val_identity_mse=identity)
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        W.save(a.out, net, summary)
    del data
    if a.eval:
        summary["compare"] = compare_priors(net, eval_specs(a.eval), dev)
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    sys.exit(main())
