"""GPU U-Net kernels against the FP64 oracle: forward pass, MSE loss, every layer's
gradient, the Adam update, per-sample normalisation and the warm-start map; FP32 and
BF16 modes.  Shapes are ragged against the conv tiles (32 x-voxels, 8 or 16 rows per
CTA) and span several tiles."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import unet_oracle as U  # noqa: E402
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
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _problem(ch, shape, B, seed):
    p = I.unet_params(ch, seed=seed)
    p[-1] = 0.5                                   # output bias
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, 2.0, size=(B,) + shape).astype(np.float32)
    t = rng.uniform(0.0, 1.5, size=(B,) + shape).astype(np.float32)
    return p, x, t


def _layer_slices(ch):
    out, off = [], 0
    for kind, ci, co in U.layer_specs(*ch):
        nw = co * ci * (27 if kind == "conv3" else 8 if kind == "tconv" else 1)
        out.append((kind, slice(off, off + nw), slice(off + nw, off + nw + co)))
        off += nw + co
    return out


@pytest.mark.parametrize("shape", [(8, 20, 40), (12, 12, 36)])
def test_forward_fp32(C, shape):
    ch = (4, 8, 16)
    p, x, _ = _problem(ch, shape, 2, 1)
    net = C.UNet(*ch, params=p, dtype="fp32")
    got = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref = U.forward(p.astype(np.float64), x.astype(np.float64), ch).numpy()
    assert rel(got, ref) < 1e-5


def test_forward_bf16(C):
    ch = (4, 8, 16)
    p, x, _ = _problem(ch, (8, 20, 40), 2, 2)
    net = C.UNet(*ch, params=p, dtype="bf16")
    got = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref_bf = U.forward(p.astype(np.float64), x.astype(np.float64), ch, bf16=True).numpy()
    ref = U.forward(p.astype(np.float64), x.astype(np.float64), ch).numpy()
    assert rel(got, ref_bf) < 2e-3      # same rounding points, FP32 accumulation order
    assert rel(got, ref) < 2e-2         # against exact arithmetic


# BF16 against exact FP64 gradients: operand rounding alone moves them by up to about
# 2.4e-2 on this problem (tests/test_bf16_tolerances.py measures it on the CPU)
@pytest.mark.parametrize("dtype,tol", [("fp32", 1e-4), ("bf16", 3e-2)])
def test_loss_and_gradients(C, dtype, tol):
    ch = (4, 8, 16)
    shape = (8, 12, 36)
    p, x, t = _problem(ch, shape, 2, 3)
    net = C.UNet(*ch, params=p, dtype=dtype)
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), loss)
    g = net.get("grads")
    lref, gref = U.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), ch)
    assert abs(float(loss.item()) - lref) <= (1e-5 if dtype == "fp32" else 1e-2) * lref
    for i, (kind, ws, bs) in enumerate(_layer_slices(ch)):
        assert rel(g[ws], gref[ws]) < tol, (i, kind, "weights", rel(g[ws], gref[ws]))
        assert rel(g[bs], gref[bs]) < tol, (i, kind, "biases", rel(g[bs], gref[bs]))
    # loss-only entry agrees with the backward pass's loss
    l2 = torch.zeros((), dtype=torch.float64, device="cuda")
    net.loss(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), l2)
    assert float(l2.item()) == float(loss.item())


def test_adam_matches_oracle(C):
    ch = (2, 4, 8)
    p, x, t = _problem(ch, (8, 8, 8), 1, 4)
    net = C.UNet(*ch, params=p, dtype="fp32")
    rng = np.random.default_rng(5)
    m = rng.normal(size=p.size).astype(np.float32) * 1e-3
    v = np.abs(rng.normal(size=p.size)).astype(np.float32) * 1e-6
    net.set(m, "adam_m")
    net.set(v, "adam_v")
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), loss)
    g = net.get("grads")
    net.step = 6                          # next step is t = 7
    net.adam(2e-3, 0.9, 0.999, 1e-8)
    # the library receives beta1, beta2 as float32: the oracle uses those same values
    b1, b2 = float(np.float32(0.9)), float(np.float32(0.999))
    pr, mr, vr = U.adam_step(p.astype(np.float64), g.astype(np.float64), m.astype(np.float64),
                             v.astype(np.float64), 7, 2e-3, b1, b2, 1e-8)
    # FP32 rounding of beta1 m + (1 - beta1) g: ~1e-7 of the larger term (|m| ~ 1e-3, |v| ~ 1e-6)
    np.testing.assert_allclose(net.get("adam_m"), mr, rtol=1e-5, atol=1e-9)
    np.testing.assert_allclose(net.get("adam_v"), vr, rtol=1e-5, atol=1e-12)
    np.testing.assert_allclose(net.get("params"), pr, rtol=1e-5, atol=1e-7)


def test_training_steps_track_oracle(C):
    """Five Adam steps on one batch: GPU parameters follow the oracle's (FP32 mode)."""
    ch = (2, 4, 8)
    p, x, t = _problem(ch, (8, 8, 16), 2, 6)
    net = C.UNet(*ch, params=p, dtype="fp32")
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    pr = p.astype(np.float64)
    mr = np.zeros_like(pr)
    vr = np.zeros_like(pr)
    for step in range(1, 6):
        net.backward(xd, td, loss)
        net.adam(1e-3)
        _, gr = U.loss_and_grad(pr, x.astype(np.float64), t.astype(np.float64), ch)
        pr, mr, vr = U.adam_step(pr, gr, mr, vr, step, 1e-3)
    assert rel(net.get("params"), pr) < 1e-4


def test_normalize_and_warm_map(C):
    rng = np.random.default_rng(7)
    x = rng.uniform(0.0, 3.0, size=(3, 8, 16, 32)).astype(np.float32)
    t = rng.uniform(0.0, 1.0, size=(3, 8, 16, 32)).astype(np.float32)
    xd, td = torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()
    C.unet_normalize(xd, td)
    m = (x.reshape(3, -1).astype(np.float64).sum(axis=1) / (16 * 32))[:, None, None, None]
    np.testing.assert_allclose(xd.cpu().numpy(), x / m, rtol=1e-6)
    np.testing.assert_allclose(td.cpu().numpy(), t / m, rtol=1e-6)
    # warm start: r_init = m * max(U(r0 / m), floor), m = sum(r0) / (nx ny)
    ch = (2, 4, 8)
    p = I.unet_params(ch, seed=8)
    p[-1] = -0.05                          # push part of the output below the floor
    net = C.UNet(*ch, params=p, dtype="fp32")
    r0 = x[0]
    got = net.warm_start(torch.from_numpy(r0).cuda(), 1e-3).cpu().numpy()
    m0 = r0.astype(np.float64).sum() / (16 * 32)
    out = U.forward(p.astype(np.float64), (r0 / m0)[None].astype(np.float64), ch).numpy()[0]
    ref = m0 * np.maximum(out, 1e-3)
    assert (out < 1e-3).any()
    assert rel(got, ref) < 1e-5


# BF16: FP32 against FP64 accumulation with the same rounding points differs by about 8e-3
# at this size (rounding flips grow through the layers; tests/test_bf16_tolerances.py)
@pytest.mark.parametrize("dtype,oracle_bf16,tol", [("fp32", False, 2e-5), ("bf16", True, 2e-2)])
def test_fullsize_forward_crop(C, dtype, oracle_bf16, tol):
    """16/32/64 network at 256x256x128 (the warm start's inference size) on one sample:
    an interior crop of the output against the oracle on the crop plus a 32-voxel halo
    (beyond the receptive field of about 28 voxels; offsets aligned to the 4-voxel
    pooling grid).  FP32 mode pins the indexing at full size; BF16 mode (same rounding
    points as the oracle's BF16 mode, FP32 accumulation) states the precision."""
    ch = (16, 32, 64)
    p = I.unet_params(ch, seed=9)
    p[-1] = 1.0
    shape = (128, 256, 256)
    xd = torch.rand(shape, generator=torch.Generator(device="cuda").manual_seed(11), device="cuda") * 2
    net = C.UNet(*ch, params=p, dtype=dtype)
    got = net.forward(xd[None])[0]
    z0, y0, x0, h, s = 48, 100, 120, 32, 16
    assert z0 % 4 == 0 and y0 % 4 == 0 and x0 % 4 == 0 and h % 4 == 0
    crop = xd[z0 - h:z0 + s + h, y0 - h:y0 + s + h, x0 - h:x0 + s + h].cpu().numpy().astype(np.float64)
    ref = U.forward(p.astype(np.float64), crop[None], ch, bf16=oracle_bf16).numpy()[0][h:-h, h:-h, h:-h]
    g = got[z0:z0 + s, y0:y0 + s, x0:x0 + s].cpu().numpy()
    print(f"full-size crop {dtype}: rel-L2 {rel(g, ref):.3e}")
    assert rel(g, ref) < tol
