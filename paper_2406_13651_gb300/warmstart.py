"""Learned warm start for CLAMP: a 3D U-Net maps the speckle-averaged image r0 (the
initial image of Alg. 2) to an initial reflectance closer to the CLAMP solution.

Every numerical step runs in the CUDA library: scene data come from the forward
model (``clamp_simulate``), inputs from ``clamp_speckle_average``, training targets
from plain CLAMP reconstructions run as one captured CUDA graph per group of
scenes (``clamp_batch_*``), and the network is trained with the library's U-Net
forward/backward kernels and Adam (``clamp_unet_*``).  PyTorch holds the device
buffers and gathers mini-batches.

Input and target of one training pair are both divided by m = sum(r0) / (nx ny), the
energy of r0 per (x, y) column (unlike mean(r0) it does not change with the range
extent nz, so a network trained on 64x64x32 volumes sees the same value scale on
256x256x128); the warm start maps back with r_init = m * max(U(r0 / m), floor).
"""
from __future__ import annotations

import math
import os
import time
from dataclasses import dataclass, field

import numpy as np

from . import clamp as C
from . import inputs as I

CHANNELS = (16, 32, 64)
FLOOR = 1e-3
MU_STEPS = 6       # mu refinement steps after the warm start (clamp_params.init_mu_steps)


@dataclass
class TrainConfig:
    steps: int = 2000
    batch: int = 24
    lr: float = 1e-3
    lr_decay: float = 0.975      # multiplied in every `decay_every` steps
    decay_every: int = 100
    val_every: int = 100
    seed: int = 5


@dataclass
class Dataset:
    x: object                    # device float32 [N, nz, ny, nx], r0 / m
    t: object                    # device float32 [N, nz, ny, nx], r* / m
    target_ce: np.ndarray        # final CE residual of every target reconstruction
    seconds: float = 0.0


@dataclass
class TrainLog:
    steps: list = field(default_factory=list)
    train_loss: list = field(default_factory=list)
    val_steps: list = field(default_factory=list)
    val_loss: list = field(default_factory=list)
    best_val: float = math.inf
    best_step: int = 0
    seconds: float = 0.0


def device_draws(shape, seed: int, dev):
    """Circular complex Gaussian speckle and noise, CN(0, 1), drawn on the device (seeded)."""
    import torch
    gen = torch.Generator(device=dev)
    gen.manual_seed(seed)
    s = 0.5 ** 0.5
    spk = torch.complex(torch.randn(shape, generator=gen, device=dev), torch.randn(shape, generator=gen, device=dev)) * s
    eta = torch.complex(torch.randn(shape, generator=gen, device=dev), torch.randn(shape, generator=gen, device=dev)) * s
    return spk, eta


def scene_data(spec: dict, dev):
    """(params, y, pupil, window) of one warm-start scene: column-surface reflectance and
    aperture from the seeded generators, looks simulated by the library's forward model."""
    import torch
    wl = I.batch_scene(spec, with_draws=False)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=spec["iters"])
    pu = torch.from_numpy(wl.pupil).to(dev)
    wi = torch.from_numpy(wl.window).to(dev)
    spk, eta = device_draws((wl.looks, wl.nz, wl.ny, wl.nx), spec["seed"], dev)
    y = C.simulate(p, torch.from_numpy(wl.r_true.astype(np.float32)).to(dev), spk, eta, pu, wi)
    return p, y, pu, wi


def make_dataset(specs, dev, group: int = 24, den: C.Denoiser | None = None, log=None) -> Dataset:
    """Training pairs for every spec: x = r0 / m, t = r* / m (m = sum(r0) / (nx ny)), where r* is the
    plain CLAMP reconstruction after spec['iters'] iterations (Gaussian prior)."""
    import torch
    den = den or C.Denoiser.gauss(0.8)
    s0 = specs[0]
    shape = (s0["nz"], s0["ny"], s0["nx"])
    N = len(specs)
    X = torch.empty((N,) + shape, dtype=torch.float32, device=dev)
    T = torch.empty_like(X)
    ce = np.zeros(N)
    t0 = time.perf_counter()
    ws = None
    for g0 in range(0, N, group):
        chunk = specs[g0:g0 + group]
        scenes = []
        for i, sp in enumerate(chunk):
            p, y, pu, wi = scene_data(sp, dev)
            if ws is None:
                ws = C.workspace(p)
            C.speckle_average(p, y, pu, wi, out=X[g0 + i], ws=ws)
            scenes.append((p, y, pu, wi, T[g0 + i]))
        batch = C.Batch(scenes, den)
        batch.launch()
        ce[g0:g0 + len(chunk)] = batch.residuals()
        batch.close()
        del scenes, batch
        C.unet_normalize(X[g0:g0 + len(chunk)], T[g0:g0 + len(chunk)])
        if log:
            log(f"data {g0 + len(chunk)}/{N}: max target CE {ce[g0:g0 + len(chunk)].max():.2e}")
    torch.cuda.synchronize()
    return Dataset(X, T, ce, time.perf_counter() - t0)


def train(net: C.UNet, data: Dataset, n_train: int, cfg: TrainConfig, log=None) -> TrainLog:
    """Adam on mean squared error over mini-batches of the first n_train pairs; the rest is
    the validation set.  The parameters with the lowest validation loss are kept."""
    import torch
    dev = data.x.device
    N = data.x.shape[0]
    rng = np.random.default_rng(cfg.seed)
    loss_d = torch.zeros((), dtype=torch.float64, device=dev)
    out = TrainLog()
    best = net.get("params")
    order = rng.permutation(n_train)
    pos = 0
    lr = cfg.lr
    t0 = time.perf_counter()

    def val_loss():
        tot, cnt = 0.0, 0
        for v0 in range(n_train, N, cfg.batch):
            v1 = min(N, v0 + cfg.batch)
            net.loss(data.x[v0:v1], data.t[v0:v1], loss_d)
            tot += float(loss_d.item()) * (v1 - v0)
            cnt += v1 - v0
        return tot / max(cnt, 1)

    for step in range(1, cfg.steps + 1):
        if pos + cfg.batch > n_train:
            order = rng.permutation(n_train)
            pos = 0
        idx = torch.from_numpy(order[pos:pos + cfg.batch]).to(dev)
        pos += cfg.batch
        xb = data.x.index_select(0, idx)
        tb = data.t.index_select(0, idx)
        net.backward(xb, tb, loss_d)
        net.adam(lr)
        if step % cfg.decay_every == 0:
            lr *= cfg.lr_decay
        if step % 20 == 0 or step == 1:
            out.steps.append(step)
            out.train_loss.append(float(loss_d.item()))
        if n_train < N and (step % cfg.val_every == 0 or step == cfg.steps):
            vl = val_loss()
            out.val_steps.append(step)
            out.val_loss.append(vl)
            if vl < out.best_val:
                out.best_val, out.best_step = vl, step
                best = net.get("params")
            if log:
                log(f"step {step}: train {out.train_loss[-1]:.4e} val {vl:.4e} lr {lr:.2e}")
    torch.cuda.synchronize()
    out.seconds = time.perf_counter() - t0
    if n_train < N:
        net.set(best, "params")
    return out


def warm_start(net: C.UNet, p: C.Params, y, pupil, window, ws=None, floor: float = FLOOR):
    """r_init for clamp_reconstruct: the U-Net applied fully convolutionally to r0."""
    r0 = C.speckle_average(p, y, pupil, window, ws=ws)
    return net.warm_start(r0, floor)


def first_below(ce_hist: np.ndarray, tol: float) -> int:
    """1-based iteration at which the CE residual first reaches tol (0 if never)."""
    hit = np.nonzero(np.asarray(ce_hist) <= tol)[0]
    return int(hit[0]) + 1 if hit.size else 0


def psnr(r_hat: np.ndarray, r_true: np.ndarray) -> float:
    """PSNR of the optimally scaled reconstruction (Sec. IV-B): 10 log10(n / ||b r_hat - r||^2)
    with b = r_hat . r / ||r_hat||^2."""
    rh = np.asarray(r_hat, np.float64).ravel()
    rt = np.asarray(r_true, np.float64).ravel()
    b = float(rh @ rt) / max(float(rh @ rh), 1e-300)
    return float(10.0 * np.log10(rt.size / max(float(np.sum((b * rh - rt) ** 2)), 1e-300)))


def trajectory(p: C.Params, y, pupil, window, den: C.Denoiser, ref, iters: int, r_init=None, ws=None):
    """Runs ``iters`` iterations one at a time on a fresh state (speckle-average init, or
    ``r_init`` with p.init_mu_steps mu refinement steps) and returns per iteration the
    convergence error and the relative L2 distance of the output wbar to ``ref`` (device)."""
    import torch
    mu, r, w = C.init(p, y, pupil, window, r_init=r_init)
    wbar = torch.empty((p.nz, p.ny, p.nx), dtype=torch.float32, device=y.device)
    ce = torch.zeros(iters, dtype=torch.float64, device=y.device)
    dist = torch.zeros(iters, dtype=torch.float64, device=y.device)
    ws = C.iterate_workspace(p, den) if ws is None else ws
    nref = torch.linalg.vector_norm(ref.double())
    for k in range(iters):
        C.iterate(p, k + 1 + p.k0, 1, y, pupil, window, den, mu, r, w, wbar, ce_out=ce[k:k + 1], ws=ws)
        dist[k] = torch.linalg.vector_norm((wbar - ref).double()) / nref
    return ce.cpu().numpy(), dist.cpu().numpy()


def compare(net: C.UNet, p_plain: C.Params, y, pupil, window, den: C.Denoiser, tol: float = 1e-3,
            max_iters: int = 300, ref_iters: int = 0, warm_k0: int = 0, r_true: np.ndarray | None = None,
            pc_threshold: float | None = None, pc_max_dist: float | None = None, warm_mu_steps: int = MU_STEPS):
    """Wall time to CE <= tol at the same reflectance error, from the speckle-average init and
    from the warm start (which includes r0, the U-Net inference, the mapping and the mu
    refinement steps), on the same data.

    The judge of the error is the plain solution run for ``ref_iters`` iterations (4 x the
    plain count to CE <= tol when 0).  The plain run stops at its first iteration with
    CE <= tol; its distance to the reference there, e_plain, is the error both runs must
    reach: the warm run stops at its first iteration with CE <= tol and distance <= e_plain
    (``warm``); ``warm_ce_only`` is the warm run stopped at CE <= tol alone.  Iteration
    counts come from per-iteration trajectories; the wall times are of fixed-count runs
    (clamp_reconstruct with max_iters = that count, no residual read-backs).  Given r_true,
    every result also gets its PSNR and (with pc_threshold and pc_max_dist) its point-cloud
    metrics (Sec. IV-B).  warm_k0 starts the warm run's beta_k schedule at k = warm_k0 + 1."""
    import torch
    mk = lambda n, **kw: C.make_params(p_plain.nx, p_plain.ny, p_plain.nz, p_plain.looks, p_plain.noise_var,  # noqa: E731
                                       p_plain.prox_var, max_iters=n, **kw)
    aws = C.workspace(mk(0))
    # plain run to CE <= tol (iteration count), then the reference solution
    p_tol = mk(max_iters, tol=tol, check_every=1)
    res = C.reconstruct(p_tol, y, pupil, window, den)
    k_plain = first_below(res.ce_hist, tol) or max_iters
    n_ref = ref_iters or 4 * k_plain
    ws = C.reconstruct_workspace(mk(max(max_iters, n_ref, 1)), den)   # the residual ring grows with max_iters
    ref = C.reconstruct(mk(n_ref), y, pupil, window, den, ws=ws).r.clone()
    r_init = warm_start(net, mk(0), y, pupil, window, ws=aws)
    pw_traj = mk(0, k0=warm_k0, init_mu_steps=warm_mu_steps)
    ce_p, d_p = trajectory(mk(0), y, pupil, window, den, ref, k_plain)
    ce_w, d_w = trajectory(pw_traj, y, pupil, window, den, ref, max_iters, r_init=r_init)
    e_plain = float(d_p[k_plain - 1])
    hit = np.nonzero((ce_w <= tol) & (d_w <= e_plain))[0]
    k_warm = int(hit[0]) + 1 if hit.size else 0
    k_warm_ce = first_below(ce_w, tol)
    r_out = torch.empty((p_plain.nz, p_plain.ny, p_plain.nx), dtype=torch.float32, device=y.device)

    def timed(n, warm):
        if n <= 0:
            return None, None
        p_run = mk(n, k0=warm_k0, init_mu_steps=warm_mu_steps) if warm else mk(n)
        for rep in range(2):   # the first run warms up (autotune, module load)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            ri = warm_start(net, p_run, y, pupil, window, ws=aws) if warm else None
            C.reconstruct(p_run, y, pupil, window, den, r_init=ri, ws=ws, r_out=r_out, report=False)
            torch.cuda.synchronize()
            sec = time.perf_counter() - t0
        return sec, r_out.cpu().numpy()

    out = {"tol": tol, "ref_iters": n_ref, "error_target": e_plain}
    rt_dev = None
    if r_true is not None and pc_threshold is not None:
        rt_dev = torch.from_numpy(np.ascontiguousarray(r_true, np.float32)).to(y.device)
    nref = float(torch.linalg.vector_norm(ref.double()))
    for name, n, warm, ce, dd in (("plain", k_plain, False, ce_p, d_p), ("warm", k_warm, True, ce_w, d_w),
                                  ("warm_ce_only", k_warm_ce, True, ce_w, d_w)):
        sec, rh = timed(n, warm)
        if sec is None:
            out[name] = {"reached": False, "iters_run": int(len(ce))}
            continue
        o = dict(seconds=sec, iters=n, reached=True, ce_final=float(ce[n - 1]), rel_err_vs_ref=float(dd[n - 1]),
                 rel_err_timed_run=float(np.linalg.norm(rh - ref.cpu().numpy()) / nref))
        if r_true is not None:
            o["psnr"] = psnr(rh, r_true)
        if rt_dev is not None:
            # points where the optimally scaled reconstruction b r_hat (the scale of the PSNR
            # and NRMSE of Sec. IV-B) exceeds the noise floor
            rhd, rtd = rh.astype(np.float64).ravel(), np.asarray(r_true, np.float64).ravel()
            b = float(rhd @ rtd) / max(float(rhd @ rhd), 1e-300)
            o["point_cloud"] = C.point_cloud_metrics(torch.from_numpy(rh).to(y.device), rt_dev, pc_threshold / b,
                                                     pc_max_dist)
        out[name] = o
    if r_true is not None:
        out["ref_psnr"] = psnr(ref.cpu().numpy(), r_true)
    return out


WEIGHTS = os.path.join(os.path.dirname(os.path.abspath(__file__)), "weights", "unet_warmstart.npz")


def warm_workload_report(dev, seed: int = 1, weights: str = WEIGHTS, tol: float = 1e-3) -> dict:
    """The warm-start comparison at 256x256x128, L = 32 (inputs.make_workload('warm')):
    wall time to CE <= tol at the same reflectance error (compare), plain vs warm start,
    with PSNR and point-cloud metrics against the ground truth."""
    import torch
    net = load(weights, dtype="bf16")
    wl = I.make_workload("warm", seed=seed, with_draws=False)
    den = C.Denoiser.from_desc(wl.denoiser)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var)
    pu, wi = torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev)
    spk, eta = device_draws((wl.looks, wl.nz, wl.ny, wl.nx), 1233 + seed, dev)
    y = C.simulate(p, torch.from_numpy(wl.r_true.astype(np.float32)).to(dev), spk, eta, pu, wi)
    del spk, eta
    # point clouds (Sec. IV-B): threshold = noise floor sigma_w^2 / alpha, outliers beyond 3x
    # the lateral Rayleigh distance 1.22 / R voxels (pupil radius R x Nyquist)
    alpha = float(np.mean(wl.window.astype(np.float64) ** 2) * np.mean(wl.pupil.astype(np.float64) ** 2))
    c = compare(net, p, y, pu, wi, den, tol=tol, max_iters=wl.iters, r_true=wl.r_true,
                pc_threshold=wl.noise_var / alpha, pc_max_dist=3.0 * 1.22 / 0.4)
    c["speedup_wall"] = (c["plain"]["seconds"] / c["warm"]["seconds"]) if c["warm"].get("reached") else None
    c["workload"] = ("256x256x128 complex64, L=32, column-surface scene, pupil R=0.4, Hann window, "
                     "SNR 1.5 dB (per-surface-voxel SNR of 7.5 dB at nz=32), Gaussian prior sigma 0.8")
    c["network"] = ("3-level 3D U-Net 16/32/64, BF16 operands / FP32 accumulation, trained by the library's "
                    "kernels on 2000 scenes of 64x64x32 (L=32, R~U[0.3,0.5], SNR~U[5,20] dB)")
    return c


def save(path: str, net: C.UNet, meta: dict) -> None:
    np.savez_compressed(path, params=net.get("params"), channels=np.array(net.channels),
                        meta=np.array(repr(meta)))


def load(path: str, dtype: str = "bf16") -> C.UNet:
    z = np.load(path)
    c1, c2, c3 = (int(v) for v in z["channels"])
    return C.UNet(c1, c2, c3, params=z["params"], dtype=dtype)
