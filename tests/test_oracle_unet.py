"""Pins of the U-Net oracle to things other than itself: brute-force loops of the
convolution, transposed convolution and pooling definitions (weight layouts
included), networks with hand-set weights whose output is known in closed form
(which fixes the layer order and the concatenation order), central finite
differences of the loss for the gradients, and closed forms of the Adam update."""
import itertools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import unet_oracle as U  # noqa: E402
from paper_2406_13651_gb300 import inputs as I  # noqa: E402

CH = (2, 4, 8)


def brute_conv3(x, W, b):
    """out[co][z][y][x] = b[co] + sum_ci sum_d W[co][ci][dz][dy][dx] x[ci][z+dz-1][y+dy-1][x+dx-1] (zero outside)."""
    ci_n, nz, ny, nx = x.shape
    co_n = W.shape[0]
    out = np.zeros((co_n, nz, ny, nx))
    for co, z, y, xx in itertools.product(range(co_n), range(nz), range(ny), range(nx)):
        acc = b[co]
        for ci, dz, dy, dx in itertools.product(range(ci_n), range(3), range(3), range(3)):
            zz, yy, xi = z + dz - 1, y + dy - 1, xx + dx - 1
            if 0 <= zz < nz and 0 <= yy < ny and 0 <= xi < nx:
                acc += W[co, ci, dz, dy, dx] * x[ci, zz, yy, xi]
        out[co, z, y, xx] = acc
    return out


def test_conv3_step_matches_definition():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 4, 5, 6))
    W = rng.normal(size=(2, 3, 3, 3, 3))
    b = rng.normal(size=2)
    got = torch.nn.functional.conv3d(torch.tensor(x)[None], torch.tensor(W), torch.tensor(b), padding=1)[0].numpy()
    np.testing.assert_allclose(got, brute_conv3(x, W, b), rtol=1e-12, atol=1e-12)


def test_tconv_step_matches_definition():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(3, 2, 3, 4))
    W = rng.normal(size=(3, 2, 2, 2, 2))     # [c_in][c_out][d]
    b = rng.normal(size=2)
    ref = np.zeros((2, 4, 6, 8)) + b[:, None, None, None]
    for ci, co, z, y, xx, dz, dy, dx in itertools.product(range(3), range(2), range(2), range(3), range(4),
                                                          range(2), range(2), range(2)):
        ref[co, 2 * z + dz, 2 * y + dy, 2 * xx + dx] += W[ci, co, dz, dy, dx] * x[ci, z, y, xx]
    got = torch.nn.functional.conv_transpose3d(torch.tensor(x)[None], torch.tensor(W), torch.tensor(b),
                                               stride=2)[0].numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_maxpool_step_matches_definition():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(2, 4, 6, 8))
    ref = x.reshape(2, 2, 2, 3, 2, 4, 2).max(axis=(2, 4, 6))
    got = torch.nn.functional.max_pool3d(torch.tensor(x)[None], 2)[0].numpy()
    np.testing.assert_array_equal(got, ref)


def _zero_params(ch):
    return np.zeros(U.param_count(*ch))


def _set(params, ch, layer, w_index, value, bias=False):
    """Writes one weight (or bias) of one layer in the flat vector."""
    views = U.unpack(torch.tensor(params), ch)
    t = views[layer][2] if bias else views[layer][1]
    t[w_index] = value
    return torch.cat([torch.cat([v[1].reshape(-1), v[2]]) for v in views]).numpy()


def _centre(ci, co):
    return (co, ci, 1, 1, 1)


def test_skip_path_identity():
    """Channel 0 through both full-resolution encoder convs (centre taps 1), then the skip
    half of the concatenation (input channel c1 of layer 10), then layer 11 and the 1x1 conv:
    output == x for x >= 0.  Fixes the layer order and puts the skip after the upsampled
    channels in the concatenation."""
    ch = CH
    p = _zero_params(ch)
    p = _set(p, ch, 0, _centre(0, 0), 1.0)
    p = _set(p, ch, 1, _centre(0, 0), 1.0)
    p = _set(p, ch, 10, _centre(ch[0], 0), 1.0)
    p = _set(p, ch, 11, _centre(0, 0), 1.0)
    p = _set(p, ch, 12, (0, 0, 0, 0, 0), 1.0)
    x = np.random.default_rng(3).uniform(0, 1, size=(2, 8, 8, 8))
    np.testing.assert_allclose(U.forward(p, x, ch).numpy(), x, rtol=0, atol=1e-15)


def test_deep_path_is_blockwise_max():
    """Channel 0 down both pooling levels and back up through the transposed convs
    (all eight taps 1, i.e. nearest upsampling), entering the decoders through the
    upsampled half of the concatenation: output = max of x over its aligned 4^3 block."""
    ch = CH
    p = _zero_params(ch)
    for layer in (0, 1):
        p = _set(p, ch, layer, _centre(0, 0), 1.0)
    for layer in (2, 3, 4, 5):
        p = _set(p, ch, layer, _centre(0, 0), 1.0)
    for d in itertools.product(range(2), range(2), range(2)):
        p = _set(p, ch, 6, (0, 0) + d, 1.0)
        p = _set(p, ch, 9, (0, 0) + d, 1.0)
    p = _set(p, ch, 7, _centre(0, 0), 1.0)     # upsampled channel 0 comes first
    p = _set(p, ch, 8, _centre(0, 0), 1.0)
    p = _set(p, ch, 10, _centre(0, 0), 1.0)
    p = _set(p, ch, 11, _centre(0, 0), 1.0)
    p = _set(p, ch, 12, (0, 0, 0, 0, 0), 1.0)
    x = np.random.default_rng(4).uniform(0, 1, size=(1, 8, 12, 16))
    blk = x.reshape(1, 2, 4, 3, 4, 4, 4).max(axis=(2, 4, 6))
    ref = blk.repeat(4, axis=1).repeat(4, axis=2).repeat(4, axis=3)
    np.testing.assert_allclose(U.forward(p, x, ch).numpy(), ref, rtol=0, atol=1e-15)


def test_biases_and_output_layer():
    """All weights zero: the output is the 1x1 layer's bias; with the last hidden layer's
    bias b and 1x1 weights w it is w . relu(b) + b_out."""
    ch = CH
    p = _zero_params(ch)
    p = _set(p, ch, 12, 0, 0.25, bias=True)
    x = np.random.default_rng(5).uniform(0, 1, size=(1, 4, 4, 4))
    np.testing.assert_allclose(U.forward(p, x, ch).numpy(), 0.25, atol=1e-15)
    p = _set(p, ch, 11, 0, 2.0, bias=True)
    p = _set(p, ch, 11, 1, -3.0, bias=True)
    p = _set(p, ch, 12, (0, 0, 0, 0, 0), 0.5)
    p = _set(p, ch, 12, (0, 1, 0, 0, 0), 7.0)
    np.testing.assert_allclose(U.forward(p, x, ch).numpy(), 0.25 + 0.5 * 2.0, atol=1e-15)


def _tiny_problem(seed=6):
    ch = CH
    p = I.unet_params(ch, seed=seed).astype(np.float64)
    rng = np.random.default_rng(seed)
    p[U.param_count(*ch) - 1] = 0.3
    x = rng.uniform(0.1, 2.0, size=(2, 8, 8, 8))
    t = rng.uniform(0.0, 1.5, size=(2, 8, 8, 8))
    return ch, p, x, t


def test_gradient_matches_finite_differences_per_layer():
    """<grad, u> against (loss(p + h u) - loss(p - h u)) / 2h for a random direction u
    confined to each layer's weights and to each layer's biases in turn."""
    ch, p, x, t = _tiny_problem()
    _, g = U.loss_and_grad(p, x, t, ch)
    rng = np.random.default_rng(7)
    off = 0
    h = 1e-7
    for kind, ci, co in U.layer_specs(*ch):
        nw = co * ci * (27 if kind == "conv3" else 8 if kind == "tconv" else 1)
        for lo, hi in ((off, off + nw), (off + nw, off + nw + co)):
            u = np.zeros_like(p)
            u[lo:hi] = rng.normal(size=hi - lo)
            fd = (U.loss_only(p + h * u, x, t, ch) - U.loss_only(p - h * u, x, t, ch)) / (2 * h)
            an = float(g @ u)
            # central-difference rounding: ~ loss * 1e-16 / h ~ 1e-9 per unit of |u|
            assert abs(fd - an) <= 1e-6 * abs(an) + 1e-8 * np.linalg.norm(u), (kind, lo, fd, an)
        off += nw + co
    assert off == p.size


def test_gradient_single_coordinates():
    ch, p, x, t = _tiny_problem(8)
    _, g = U.loss_and_grad(p, x, t, ch)
    rng = np.random.default_rng(9)
    h = 1e-7
    for i in rng.choice(p.size, 12, replace=False):
        e = np.zeros_like(p)
        e[i] = h
        fd = (U.loss_only(p + e, x, t, ch) - U.loss_only(p - e, x, t, ch)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * abs(g[i]) + 1e-8, (i, fd, g[i])


def test_mse_is_the_mean_of_squares():
    rng = np.random.default_rng(10)
    a = rng.normal(size=(2, 3, 4, 5))
    b = rng.normal(size=(2, 3, 4, 5))
    assert abs(float(U.mse(torch.tensor(a), b)) - np.sum((a - b) ** 2) / a.size) < 1e-14


def test_adam_closed_forms():
    """First step moves every parameter by lr * g / (|g| + eps); under a constant gradient the
    bias-corrected moments equal g and g^2 at every step, so each step is the same."""
    g = np.array([0.3, -2.0, 1e-3, 5.0])
    p = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 0.01, 1e-8
    p1, m, v = U.adam_step(p, g, m, v, 1, lr, eps=eps)
    np.testing.assert_allclose(p1, -lr * g / (np.abs(g) + eps), rtol=1e-12)
    pk = p1
    for t in range(2, 30):
        prev = pk
        pk, m, v = U.adam_step(pk, g, m, v, t, lr, eps=eps)
        np.testing.assert_allclose(pk - prev, -lr * g / (np.abs(g) + eps), rtol=1e-9)


def test_bf16_rounding_is_nearest_even():
    one = 1.0
    vals = torch.tensor([one + 2 ** -8, one + 3 * 2 ** -8, one + 2 ** -9, -(one + 2 ** -8)], dtype=torch.float64)
    got = U._bf(vals, True).numpy()
    np.testing.assert_array_equal(got, [1.0, 1.0 + 2 ** -6, 1.0, -1.0])


def test_param_count_matches_generator():
    for ch in (CH, (16, 32, 64)):
        assert I.unet_params(ch, seed=1).size == U.param_count(*ch)
