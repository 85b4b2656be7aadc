"""The U-Net's 3x3x3 convs on the tensor cores (BF16 networks): forward outputs and every
layer's gradients against the CUDA-core BF16 path (the same operand rounding, other FP32
summation order) and against the FP64 oracle with BF16 rounding points, at the training
size (levels 64, 32, 16 wide: several rows per 128-voxel tile) and at an inference width
(levels 256, 128, 64: tiles of one row, then of two)."""
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


def _layer_slices(ch):
    out, off = [], 0
    for kind, ci, co in U.layer_specs(*ch):
        nw = co * ci * (27 if kind == "conv3" else 8 if kind == "tconv" else 1)
        out.append((kind, slice(off, off + nw), slice(off + nw, off + nw + co)))
        off += nw + co
    return out


def _both_paths(C, ch, p, run):
    """run(net) on a BF16 network with the tensor cores on, then off."""
    outs = []
    for on in (True, False):
        net = C.UNet(*ch, params=p, dtype="bf16")
        net.set_tensor_cores(on)
        outs.append(run(net))
        net.check()
        net.close()
    return outs


def test_tensor_core_forward_and_gradients_match_oracle(C):
    """16/16/16 network on 8 x 16 x 32 (levels 32 and 16 on the tensor cores, the 8-wide
    bottleneck on the CUDA cores) against the FP64 oracle with the same BF16 rounding
    points, and against exact gradients within the BF16 operand-rounding effect."""
    ch = (16, 16, 16)
    p = I.unet_params(ch, seed=25)
    p[-1] = 0.5
    rng = np.random.default_rng(26)
    shape = (8, 16, 32)
    x = rng.uniform(0.0, 2.0, size=(1,) + shape).astype(np.float32)
    t = rng.uniform(0.0, 1.5, size=(1,) + shape).astype(np.float32)
    net = C.UNet(*ch, params=p, dtype="bf16")
    got = net.forward(torch.from_numpy(x).cuda()).cpu().numpy()
    ref_bf = U.forward(p.astype(np.float64), x.astype(np.float64), ch, bf16=True).numpy()
    print(f"tensor-core forward vs BF16 oracle: rel-L2 {rel(got, ref_bf):.2e}")
    assert rel(got, ref_bf) < 2e-3
    loss = torch.zeros((), dtype=torch.float64, device="cuda")
    net.backward(torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda(), loss)
    net.check()
    gg = net.get("grads")
    lref, gref = U.loss_and_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), ch)
    assert abs(float(loss.item()) - lref) <= 1e-2 * lref
    for i, (kind, ws, bs) in enumerate(_layer_slices(ch)):
        assert rel(gg[ws], gref[ws]) < 3e-2, (i, kind, "weights", rel(gg[ws], gref[ws]))
        assert rel(gg[bs], gref[bs]) < 3e-2, (i, kind, "biases", rel(gg[bs], gref[bs]))
    print("tensor-core gradients vs exact: worst layer rel", max(rel(gg[ws], gref[ws]) for _, ws, _ in _layer_slices(ch)))


@pytest.mark.parametrize("shape,B", [((32, 64, 64), 2), ((16, 32, 256), 1)])
def test_forward_tensor_cores_match_cuda_cores(C, shape, B):
    ch = (16, 32, 64)
    p = I.unet_params(ch, seed=21)
    p[-1] = 0.5
    x = torch.rand((B,) + shape, generator=torch.Generator(device="cuda").manual_seed(22), device="cuda") * 2
    tc, cc = _both_paths(C, ch, p, lambda net: net.forward(x).cpu().numpy())
    # same BF16 operands, FP32 sums in another order: a difference at the FP32 rounding level
    # flips the BF16 rounding of some activations and, through ReLU and the max-pool argmax,
    # grows with depth.  The CUDA-core path itself sits 8e-3 from the oracle's FP64 sums at
    # the 256^2 x 128 inference size (test_gpu_unet.py); a wrong tap, channel or row would
    # be of order 1.
    r = rel(tc, cc)
    print(f"forward {shape} x {B}: tensor vs CUDA cores rel-L2 {r:.2e}")
    assert r < 1.5e-2
    assert np.all(np.isfinite(tc))


def test_gradients_tensor_cores_match_cuda_cores(C):
    ch = (16, 32, 64)
    p = I.unet_params(ch, seed=23)
    p[-1] = 0.5
    shape = (32, 64, 64)
    g = torch.Generator(device="cuda").manual_seed(24)
    x = torch.rand((2,) + shape, generator=g, device="cuda") * 2
    t = torch.rand((2,) + shape, generator=g, device="cuda") * 1.5

    def run(net):
        loss = torch.zeros((), dtype=torch.float64, device="cuda")
        net.backward(x, t, loss)
        return float(loss.item()), net.get("grads")

    (l_tc, g_tc), (l_cc, g_cc) = _both_paths(C, ch, p, run)
    assert abs(l_tc - l_cc) <= 1e-2 * l_cc
    # the gradients of both paths sit within the BF16 operand-rounding effect of the exact
    # ones (3e-2, test_gpu_unet.py): the same bound between them
    for i, (kind, ws, bs) in enumerate(_layer_slices(ch)):
        assert rel(g_tc[ws], g_cc[ws]) < 3e-2, (i, kind, "weights", rel(g_tc[ws], g_cc[ws]))
        assert rel(g_tc[bs], g_cc[bs]) < 3e-2, (i, kind, "biases", rel(g_tc[bs], g_cc[bs]))
    print("gradients: worst layer rel", max(rel(g_tc[ws], g_cc[ws]) for _, ws, _ in _layer_slices(ch)))
