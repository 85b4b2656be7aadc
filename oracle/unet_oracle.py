"""FP64 CPU oracle for the learned warm start: a 3-level 3D U-Net, its MSE loss, its
gradients and the Adam update.

TEST INFRASTRUCTURE ONLY.  This module is the plain reference that the CUDA U-Net
kernels are checked against; only the test-suite and the benchmark's CPU-baseline
leg may import it.  It shares no code with the CUDA library.  Plain PyTorch CPU
operators in float64 serve as steps (``conv3d``, ``max_pool3d``,
``conv_transpose3d``, autograd for the gradients); the tests pin those steps to
brute-force loops and the gradients to central finite differences.

The network follows the encoder-decoder pattern of the paper's prior (Sec. III-C):
per level two 3x3x3 convolutions with ReLU, 2x2x2 max-pooling on the way down,
a 2x2x2 stride-2 transposed convolution on the way up, the encoder's output
concatenated after the upsampled channels, and a final 1x1x1 convolution.  The
paper's channel counts sit in a figure that is not available; the warm start uses
c1/c2/c3 = 16/32/64.  Batch normalisation is omitted (reading U1: three levels of
ReLU convolutions train without it, and the network is then one fixed map at any
volume size).

Parameter layout (flat float vector), layer by layer, weights then biases:
  3x3x3 conv  W[c_out][c_in][3][3][3]  (cross-correlation, zero padding 1)
  transposed  W[c_in][c_out][2][2][2]  out[2v + d] = b + sum_ci W[ci][co][d] in[v]
  1x1x1 conv  W[1][c1]
Layers: conv 1->c1, c1->c1, c1->c2, c2->c2, c2->c3, c3->c3, tconv c3->c2,
conv 2c2->c2, c2->c2, tconv c2->c1, conv 2c1->c1, c1->c1, 1x1 c1->1.

BF16 mode (``bf16=True``) rounds every convolution's weights and inputs to bfloat16
(round to nearest even) before the float64 arithmetic, as the BF16 GPU kernels do.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as Fn


def layer_specs(c1: int, c2: int, c3: int):
    """(kind, c_in, c_out) for the 13 layers; kind in {'conv3', 'tconv', 'conv1'}."""
    return [("conv3", 1, c1), ("conv3", c1, c1), ("conv3", c1, c2), ("conv3", c2, c2),
            ("conv3", c2, c3), ("conv3", c3, c3), ("tconv", c3, c2), ("conv3", 2 * c2, c2),
            ("conv3", c2, c2), ("tconv", c2, c1), ("conv3", 2 * c1, c1), ("conv3", c1, c1),
            ("conv1", c1, 1)]


def _wshape(kind, ci, co):
    if kind == "conv3":
        return (co, ci, 3, 3, 3)
    if kind == "tconv":
        return (ci, co, 2, 2, 2)
    return (co, ci, 1, 1, 1)


def param_count(c1: int, c2: int, c3: int) -> int:
    return sum(int(np.prod(_wshape(k, ci, co))) + co for k, ci, co in layer_specs(c1, c2, c3))


def unpack(params, channels):
    """Flat parameter vector -> list of (kind, W, b) torch float64 tensors (views of one tensor)."""
    flat = params if isinstance(params, torch.Tensor) else torch.as_tensor(np.asarray(params, np.float64))
    out, off = [], 0
    for kind, ci, co in layer_specs(*channels):
        shp = _wshape(kind, ci, co)
        nw = int(np.prod(shp))
        out.append((kind, flat[off:off + nw].reshape(shp), flat[off + nw:off + nw + co]))
        off += nw + co
    assert off == flat.numel()
    return out


def _bf(t: torch.Tensor, bf16: bool) -> torch.Tensor:
    return t.to(torch.bfloat16).to(torch.float64) if bf16 else t


def forward(params, x, channels, bf16: bool = False) -> torch.Tensor:
    """U-Net output for x [B, nz, ny, nx] (float64 torch tensor or array) -> [B, nz, ny, nx]."""
    L = unpack(params, channels)
    h = torch.as_tensor(np.asarray(x, np.float64)) if not isinstance(x, torch.Tensor) else x
    h = h[:, None]

    def conv(i, t):
        _, W, b = L[i]
        return Fn.relu(Fn.conv3d(_bf(t, bf16), _bf(W, bf16), b, padding=1))

    def tconv(i, t):
        _, W, b = L[i]
        return Fn.conv_transpose3d(_bf(t, bf16), _bf(W, bf16), b, stride=2)

    s1 = conv(1, conv(0, h))
    s2 = conv(3, conv(2, Fn.max_pool3d(s1, 2)))
    b2 = conv(5, conv(4, Fn.max_pool3d(s2, 2)))
    d2 = conv(8, conv(7, torch.cat([tconv(6, b2), s2], dim=1)))
    d1 = conv(11, conv(10, torch.cat([tconv(9, d2), s1], dim=1)))
    _, W, b = L[12]
    return Fn.conv3d(_bf(d1, bf16), _bf(W, bf16), b)[:, 0]


def mse(pred: torch.Tensor, target) -> torch.Tensor:
    """Mean squared error over every output value."""
    t = torch.as_tensor(np.asarray(target, np.float64)) if not isinstance(target, torch.Tensor) else target
    return ((pred - t) ** 2).mean()


def loss_and_grad(params, x, target, channels):
    """(loss, d loss / d params) in float64 by reverse-mode differentiation of ``forward``."""
    p = torch.tensor(np.asarray(params, np.float64), requires_grad=True)
    loss = mse(forward(p, x, channels), target)
    loss.backward()
    return float(loss.detach()), p.grad.numpy().copy()


def loss_only(params, x, target, channels) -> float:
    with torch.no_grad():
        return float(mse(forward(torch.as_tensor(np.asarray(params, np.float64)), x, channels), target))


def adam_step(p, g, m, v, t: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1): biased moments, their bias
    correction by 1 - beta^t, and p - lr * m_hat / (sqrt(v_hat) + eps).  Returns (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v
