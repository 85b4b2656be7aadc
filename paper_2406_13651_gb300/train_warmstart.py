"""Trains the warm-start U-Net on the GPU and writes its parameters.

    python -m paper_2406_13651_gb300.train_warmstart --scenes 2000 --steps 3000 \
        --out paper_2406_13651_gb300/weights/unet_warmstart.npz

Scenes: column surfaces of 64x64x32 with 32 looks, pupil radius U[0.3, 0.5] Nyquist,
SNR U[5, 20] dB (``inputs.warmstart_specs``); targets: plain CLAMP with the Gaussian
prior run for ``--iters`` iterations in batched CUDA graphs; the last 10% of the
scenes are the validation set.  Prints one JSON summary line.
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time


def main(argv=None) -> int:
    ap = argparse.ArgumentParser()
    ap.add_argument("--scenes", type=int, default=2000)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--batch", type=int, default=24)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--iters", type=int, default=80, help="CLAMP iterations of each target")
    ap.add_argument("--nx", type=int, default=64)
    ap.add_argument("--nz", type=int, default=32)
    ap.add_argument("--looks", type=int, default=32)
    ap.add_argument("--dtype", choices=("bf16", "fp32"), default="bf16")
    ap.add_argument("--seed", type=int, default=11)
    ap.add_argument("--out", default="")
    ap.add_argument("--quiet", action="store_true")
    a = ap.parse_args(argv)

    import numpy as np
    import torch

    from . import build as B
    from . import clamp as C
    from . import inputs as I
    from . import warmstart as W

    B.build()
    dev = torch.device("cuda")
    log = None if a.quiet else (lambda s: print(s, file=sys.stderr, flush=True))
    specs = I.warmstart_specs(a.scenes, seed=a.seed, nx=a.nx, ny=a.nx, nz=a.nz, looks=a.looks, iters=a.iters)
    data = W.make_dataset(specs, dev, log=log)
    n_train = a.scenes - max(1, a.scenes // 10)
    net = C.UNet(*W.CHANNELS, params=I.unet_params(W.CHANNELS, seed=5), dtype=a.dtype)
    cfg = W.TrainConfig(steps=a.steps, batch=a.batch, lr=a.lr)
    t0 = time.perf_counter()
    tl = W.train(net, data, n_train, cfg, log=log)
    summary = dict(scenes=a.scenes, size=[a.nx, a.nx, a.nz], looks=a.looks, target_iters=a.iters,
                   target_ce_max=float(data.target_ce.max()), target_ce_median=float(np.median(data.target_ce)),
                   data_seconds=round(data.seconds, 2), train_seconds=round(time.perf_counter() - t0, 2),
                   steps=a.steps, batch=a.batch, lr=a.lr, dtype=a.dtype, best_val=tl.best_val, best_step=tl.best_step,
                   first_train_loss=tl.train_loss[0], last_train_loss=tl.train_loss[-1])
    if a.out:
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        W.save(a.out, net, summary)
    print(json.dumps(summary))
    return 0


if __name__ == "__main__":
    sys.exit(main())
