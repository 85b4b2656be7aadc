"""The learned warm start against plain CLAMP: the U-Net trained by the library's own
kernels (weights in paper_2406_13651_gb300/weights/) must reach the convergence error
1e-3 at the same reflectance error as the speckle-average initialisation (distance to
the long plain solution no larger than the plain run's at its own CE 1e-3 stop) in fewer
iterations and less wall time, on held-out scenes and at 256x256x128; and a short
training run from scratch must learn (validation loss far below that of the identity
map)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
WEIGHTS = os.path.join(ROOT, "paper_2406_13651_gb300", "weights", "unet_warmstart.npz")


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp, inputs, warmstart
    build.build()
    clamp.load()
    return clamp, inputs, warmstart


def test_short_training_learns(env):
    C, I, W = env
    dev = torch.device("cuda")
    specs = I.warmstart_specs(96, seed=21, nx=32, ny=32, nz=16, looks=16, iters=120)
    data = W.make_dataset(specs, dev)
    n_train = 84
    xv, tv = data.x[n_train:].double(), data.t[n_train:].double()
    identity = float(((xv - tv) ** 2).mean())
    net = C.UNet(*W.CHANNELS, params=I.unet_params(W.CHANNELS, seed=5), dtype="bf16")
    log = W.train(net, data, n_train, W.TrainConfig(steps=240, batch=12, val_every=60))
    assert np.isfinite(log.val_loss).all()
    assert log.best_val < 0.2 * identity, (log.best_val, identity)
    assert log.val_loss[-1] < log.val_loss[0]


def _trained(C, W):
    assert os.path.exists(WEIGHTS), "trained warm-start weights are missing"
    return W.load(WEIGHTS, dtype="bf16")


def test_warm_start_gain_heldout_64(env):
    C, I, W = env
    net = _trained(C, W)
    den = C.Denoiser.gauss(0.8)
    dev = torch.device("cuda")
    gains = []
    for sp in I.warmstart_specs(3, seed=77, iters=400):     # seeds outside the training set
        sp["snr"] = 7.5
        p, y, pu, wi = W.scene_data(sp, dev)
        c = W.compare(net, p, y, pu, wi, den, tol=1e-3, max_iters=400)
        assert c["plain"]["reached"] and c["warm"]["reached"], c
        assert c["warm"]["iters"] < c["plain"]["iters"], c
        assert c["warm"]["rel_err_vs_ref"] <= c["plain"]["rel_err_vs_ref"], c
        assert c["warm"]["ce_final"] <= 1e-3, c
        gains.append(1 - c["warm"]["iters"] / c["plain"]["iters"])
    assert np.mean(gains) > 0.15, gains


def test_warm_start_gain_256(env):
    C, I, W = env
    net = _trained(C, W)
    wl = I.make_workload("warm", seed=1, with_draws=False)
    den = C.Denoiser.from_desc(wl.denoiser)
    dev = torch.device("cuda")
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var)
    pu, wi = torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev)
    spk, eta = W.device_draws((wl.looks, wl.nz, wl.ny, wl.nx), 1234, dev)
    y = C.simulate(p, torch.from_numpy(wl.r_true.astype(np.float32)).to(dev), spk, eta, pu, wi)
    del spk, eta
    c = W.compare(net, p, y, pu, wi, den, tol=1e-3, max_iters=wl.iters, r_true=wl.r_true)
    print({k: c[k] for k in ("plain", "warm", "warm_ce_only", "error_target")})
    assert c["plain"]["reached"] and c["warm"]["reached"], c
    assert c["warm"]["iters"] < c["plain"]["iters"], c
    assert c["warm"]["seconds"] < c["plain"]["seconds"], c
    assert c["warm"]["rel_err_vs_ref"] <= c["plain"]["rel_err_vs_ref"], c
    assert c["warm"]["ce_final"] <= 1e-3, c
    assert c["warm"]["psnr"] > c["plain"]["psnr"] - 0.5, c
