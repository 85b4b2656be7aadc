"""Tensor-core (tcgen05) path: the one-tile BF16 GEMM check and the BF16 residual CNN
prior against the oracle (BF16-rounded weights and layer inputs, FP64 products)."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import clamp_oracle as O  # noqa: E402
from paper_2406_13651_gb300 import inputs as I  # noqa: E402

TOL_BF16 = 1e-2


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


# K = 256 keeps every operand read inside the kernel's shared-memory allocation.
@pytest.mark.parametrize("n,k", [(256, 256), (48, 256), (16, 256), (64, 256)])
def test_tc_gemm_bf16(C, n, k):
    g = torch.Generator().manual_seed(n * 1000 + k)
    a = torch.randn(128, k, generator=g).to(torch.bfloat16)
    b = torch.randn(n, k, generator=g).to(torch.bfloat16)
    ref = a.double() @ b.double().T
    ad, bd = a.cuda(), b.cuda()
    d = torch.full((128, n), float("nan"), dtype=torch.float32, device="cuda")
    st = C.load().clamp_tc_gemm_bf16(n, k, ad.data_ptr(), bd.data_ptr(), d.data_ptr(),
                                     torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    got = d.cpu().double()
    assert torch.isfinite(got).all()
    assert rel(got.numpy(), ref.numpy()) < 1e-5


@pytest.mark.parametrize("n,k", [(48, 64), (32, 96), (16, 64), (128, 32)])
def test_tc_gemm_tf32x3(C, n, k):
    g = torch.Generator().manual_seed(n * 1000 + k + 7)
    a = torch.randn(128, k, generator=g, dtype=torch.float32)
    b = torch.randn(n, k, generator=g, dtype=torch.float32)
    ref = a.double() @ b.double().T
    ad, bd = a.cuda(), b.cuda()   # keep both alive: a temporary could be reused for the other
    d = torch.full((128, n), float("nan"), dtype=torch.float32, device="cuda")
    st = C.load().clamp_tc_gemm_tf32x3(n, k, ad.data_ptr(), bd.data_ptr(), d.data_ptr(),
                                       torch.cuda.current_stream().cuda_stream)
    assert st == 0
    torch.cuda.synchronize()
    got = d.cpu().double()
    assert torch.isfinite(got).all()
    assert rel(got.numpy(), ref.numpy()) < 2e-6   # FP32-level, far below plain TF32 (~1e-3)


@pytest.mark.parametrize("shape,layers,channels", [((4, 8, 128), 5, 32), ((2, 2, 256), 4, 16),
                                                   ((3, 4, 256), 4, 16), ((2, 4, 128), 3, 48),
                                                   ((16, 32, 256), 3, 48)])
def test_fp32_cnn_tensor_path_matches_oracle(C, shape, layers, channels):
    """FP32 CNN prior on the tensor cores (TF32x3): FP32-level agreement with the oracle
    (at 16 x 32 x 256 and 48 channels the persistent hidden-layer kernel has 256 tiles for
    at most one CTA per SM, so CTAs walk two)."""
    ws, bs = I.cnn_weights(layers, channels, seed=layers + channels, last_scale=0.3)
    rng = np.random.default_rng(3)
    bs = [b + 0.02 * rng.standard_normal(b.shape).astype(np.float32) for b in bs]
    x = rng.uniform(0, 1, shape).astype(np.float32)
    den = C.Denoiser.cnn(ws, bs, "fp32")
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    C.denoise(den, xd, out)
    torch.cuda.synchronize()
    ref = O.denoise_cnn(x.astype(np.float64), ws, bs)
    got = out.cpu().numpy()
    # products are FP32-exact to ~2^-21 (TF32x3); the tensor core's FP32 accumulation over
    # 27 x Cin x 3 MMAs per output leaves ~2e-5 on the CNN branch (plain TF32 would be ~1e-3)
    assert rel(got - x, ref - x) < 5e-5
    assert rel(got, ref) < 5e-5


def _bf16_cnn(layers, channels, seed, last_scale=0.3):
    ws, bs = I.cnn_weights(layers, channels, seed=seed, last_scale=last_scale)
    rng = np.random.default_rng(seed)
    bs = [b + 0.02 * rng.standard_normal(b.shape).astype(np.float32) for b in bs]
    return ws, bs


@pytest.mark.parametrize("shape,layers,channels", [((4, 8, 128), 8, 48), ((2, 4, 256), 4, 48),
                                                   ((4, 8, 128), 4, 16), ((2, 8, 128), 4, 32),
                                                   ((2, 4, 128), 3, 64), ((4, 12, 256), 3, 48),
                                                   ((16, 64, 256), 3, 48), ((32, 64, 256), 3, 16)])
def test_bf16_cnn_matches_oracle(C, shape, layers, channels):
    """Tiles at every volume edge (x0 - 1 < 0, the last rows and planes); 3, 4 and 8 layers
    (the last layer's tap sums land in either activation buffer); 512 and 1024 tiles, more
    than the persistent hidden-layer kernel's CTAs, so CTAs walk several tiles."""
    ws, bs = _bf16_cnn(layers, channels, seed=layers * 7 + channels)
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, shape).astype(np.float32)
    den = C.Denoiser.cnn(ws, bs, "bf16")
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    C.denoise(den, xd, out)
    torch.cuda.synchronize()
    ref = O.denoise_cnn(x.astype(np.float64), ws, bs, bf16=True)
    got = out.cpu().numpy()
    assert np.isfinite(got).all()
    assert rel(got - x, ref - x) < TOL_BF16     # the CNN branch
    assert rel(got, ref) < 1e-3


def test_bf16_cnn_rejects_unsupported_volume(C):
    ws, bs = _bf16_cnn(3, 16, seed=2)
    den = C.Denoiser.cnn(ws, bs, "bf16")
    x = torch.zeros((4, 8, 64), device="cuda")
    with pytest.raises(C.ClampError) as e:
        C.denoise(den, x, torch.empty_like(x))
    assert e.value.status == 7


def test_reconstruct_with_bf16_prior(C):
    wl = I.make_workload("cfg1", seed=5, nx=128, ny=16, nz=8, looks=3, iters=6)
    ws, bs = I.cnn_weights(8, 48, seed=5)
    den_desc = {"kind": "cnn", "weights": ws, "biases": bs, "dtype": "bf16"}
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    ref, _ = O.reconstruct(y32.astype(np.complex128), wl.pupil, wl.window, den_desc, wl.noise_var, wl.prox_var, 6)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=6)
    res = C.reconstruct(p, torch.from_numpy(y32).cuda(), torch.from_numpy(wl.pupil).cuda(),
                        torch.from_numpy(wl.window).cuda(), C.Denoiser.from_desc(den_desc))
    assert rel(res.r.cpu().numpy(), ref) < TOL_BF16
