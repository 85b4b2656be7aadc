"""The U-Net prior agent (Sec. III-C) on the GPU against the oracle: as a denoiser
(clamp_denoise with clamp_denoiser_create_unet) and inside whole reconstructions
(Alg. 2 with H the U-Net)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import clamp_oracle as O  # noqa: E402
from paper_2406_13651_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    clamp.load()
    return clamp


def rel(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _params(ch, seed):
    p = I.unet_params(ch, seed=seed)
    p[-1] = 0.3
    return p


@pytest.mark.parametrize("dtype,tol", [("fp32", 1e-5), ("bf16", 2e-3)])
def test_unet_prior_denoise_matches_oracle(C, dtype, tol):
    ch = (4, 8, 16)
    p = _params(ch, 3)
    net = C.UNet(*ch, params=p, dtype=dtype)
    den = C.Denoiser.unet(net, 1e-3)
    x = np.random.default_rng(4).uniform(0.0, 0.05, size=(16, 32, 64)).astype(np.float32)
    out = torch.empty((16, 32, 64), device="cuda")
    C.denoise(den, torch.from_numpy(x).cuda(), out)
    torch.cuda.synchronize()
    ref = O.apply_prior(x.astype(np.float64), den.desc)
    assert rel(out.cpu().numpy(), ref) < tol


def test_unet_prior_rejects_unsupported_volume(C):
    net = C.UNet(2, 4, 8, params=_params((2, 4, 8), 5), dtype="fp32")
    den = C.Denoiser.unet(net)
    x = torch.zeros((6, 8, 16), device="cuda")
    with pytest.raises(C.ClampError) as e:
        C.denoise(den, x, torch.empty_like(x))
    assert e.value.status == 7


def test_reconstruct_with_unet_prior_matches_oracle(C):
    ch = (2, 4, 8)
    wl = I.make_workload("tiny", seed=6, iters=6)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    net = C.UNet(*ch, params=_params(ch, 7), dtype="fp32")
    den = C.Denoiser.unet(net, 1e-3)
    ref, st = O.reconstruct(y32.astype(np.complex128), wl.pupil, wl.window, den.desc, wl.noise_var, wl.prox_var, 6)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=6)
    dev = torch.device("cuda")
    res = C.reconstruct(p, torch.from_numpy(y32).to(dev), torch.from_numpy(wl.pupil).to(dev),
                        torch.from_numpy(wl.window).to(dev), den)
    assert rel(res.r.cpu().numpy(), ref) < 1e-4
    np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)
