"""Seeded synthetic inputs for CLAMP reconstructions (scenes, speckle, noise, apertures).

This module holds no arithmetic of the reconstruction method itself: it draws
random numbers and builds the scene, aperture and denoiser-weight inputs that
both the CUDA path and the FP64 oracle consume.  The data simulation
``y = A g + eta`` (the forward model of Sec. II-B, Eqs. (forward-model),
(g-given-r)) is done by each side on its own from the draws produced here.

Random numbers come from a counter-based SplitMix64 generator (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014) turned
into normals by the Box-Muller transform, so the same seed gives the same
values on every machine and numpy version.

Layouts: volumes are ``[nz][ny][nx]`` with x fastest; frequency-domain arrays
(pupil, window) are in unshifted FFT order with DC at index 0.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def _mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (finaliser) applied elementwise to uint64."""
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def _stream_key(seed: int, stream: int) -> np.uint64:
    k = np.array([(seed * 0x100000001B3 + stream * 0x9E3779B1 + 0x1234567) & (2**64 - 1)], dtype=np.uint64)
    return _mix64(k)[0]


def uniform(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` doubles in [0, 1) from counters offset+1 .. offset+count of stream (seed, stream)."""
    with np.errstate(over="ignore"):
        i = np.arange(offset + 1, offset + count + 1, dtype=np.uint64)
        z = _mix64(_stream_key(seed, stream) + i * _GOLDEN)
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def normal(seed: int, stream: int, count: int, offset: int = 0) -> np.ndarray:
    """``count`` standard normal doubles (Box-Muller on pairs of uniforms); ``offset`` (even)
    is the index of the first normal within the stream, so chunks concatenate to one draw."""
    assert offset % 2 == 0
    m = (count + 1) // 2
    u = uniform(seed, stream, 2 * m, offset)
    u1 = 1.0 - u[0::2]  # in (0, 1], keeps log finite
    u2 = u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * m)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:count]


def complex_normal(seed: int, stream: int, shape, offset: int = 0) -> np.ndarray:
    """Circular complex Gaussian CN(0, 1): E|z|^2 = 1, real and imaginary parts N(0, 1/2).
    ``offset`` is the index of the first complex value within the stream."""
    cnt = int(np.prod(shape))
    v = normal(seed, stream, 2 * cnt, 2 * offset)
    return ((v[0::2] + 1j * v[1::2]) * math.sqrt(0.5)).reshape(shape)


def look_draws(wl: "Workload", seed: int, look: int):
    """Speckle and noise draws of one look, equal to look ``look`` of the full draws
    make_workload(..., with_draws=True) returns."""
    n = wl.nx * wl.ny * wl.nz
    shape = (wl.nz, wl.ny, wl.nx)
    return complex_normal(seed, 20, shape, look * n), complex_normal(seed, 21, shape, look * n)


# ----------------------------------------------------------------------------- apertures

def signed_freq(n: int) -> np.ndarray:
    """Signed DFT bin index in unshifted order: k for k < n/2, else k - n."""
    k = np.arange(n)
    return np.where(k <= (n - 1) // 2, k, k - n).astype(np.float64)


def circular_pupil(nx: int, ny: int, radius: float) -> np.ndarray:
    """Binary lateral pupil ``p[ky][kx]``: 1 inside a circle of ``radius`` x Nyquist.

    The aperture is a centred circle in the pupil plane (Sec. IV-B: diameter 50 %
    of the grid length, i.e. radius 0.5 Nyquist).  Bin (kx, ky) is inside iff
    (2 fx / nx)^2 + (2 fy / ny)^2 <= radius^2 with signed bins fx, fy.
    """
    fx = 2.0 * signed_freq(nx) / nx
    fy = 2.0 * signed_freq(ny) / ny
    return ((fy[:, None] ** 2 + fx[None, :] ** 2) <= radius * radius + 1e-12).astype(np.float32)


def hann_window(nz: int) -> np.ndarray:
    """Periodic Hann range window centred on DC: h = 0.5 (1 + cos(2 pi fz / nz))."""
    fz = signed_freq(nz)
    return (0.5 * (1.0 + np.cos(2.0 * math.pi * fz / nz))).astype(np.float32)


def band_window(nz: int, q: float) -> np.ndarray:
    """Range window of data zero-padded by ``q`` (Sec. II-B): the periodic Hann window of
    the measured band of m = nz / q bins, centred on DC, embedded in the padded spectrum,
    zero outside it.  q = 1 gives ``hann_window(nz)``."""
    m = nz / q
    fz = signed_freq(nz)
    h = np.where(np.abs(fz) <= m / 2.0, 0.5 * (1.0 + np.cos(2.0 * math.pi * fz / m)), 0.0)
    return h.astype(np.float32)


def rect_window(nz: int) -> np.ndarray:
    """All-pass range window (binary aperture along range)."""
    return np.ones(nz, dtype=np.float32)


# ----------------------------------------------------------------------------- scenes

def _periodic_smooth(field: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic Gaussian smoothing of a 2D field (scene texture only)."""
    ny, nx = field.shape
    fy = signed_freq(ny)[:, None] / ny
    fx = signed_freq(nx)[None, :] / nx
    h = np.exp(-2.0 * (math.pi * sigma) ** 2 * (fx * fx + fy * fy))
    return np.real(np.fft.ifft2(np.fft.fft2(field) * h))


def column_surface_scene(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """One surface per (x, y) column at a depth from a smooth random field.

    Depth: white noise smoothed (periodic Gaussian, sigma = n/8), min-max mapped to
    [0.2, 0.8] nz and rounded half up.  Reflectance per column ~ U[0.2, 1].
    Returns float64 r[nz][ny][nx] (zero off the surface).
    """
    noise = normal(seed, 1, nx * ny).reshape(ny, nx)
    depth = _periodic_smooth(noise, max(nx, ny) / 8.0)
    lo, hi = depth.min(), depth.max()
    t = (depth - lo) / (hi - lo if hi > lo else 1.0)
    zi = np.floor((0.2 + 0.6 * t) * nz + 0.5).astype(np.int64)
    zi = np.clip(zi, 0, nz - 1)
    refl = 0.2 + 0.8 * uniform(seed, 2, nx * ny).reshape(ny, nx)
    r = np.zeros((nz, ny, nx))
    yy, xx = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r[zi, yy, xx] = refl
    return r


def facet_scene(nx: int, ny: int, nz: int, seed: int) -> np.ndarray:
    """3 to 6 planar facets z = p x + q y + c over random rectangles, with occlusion.

    A back plane sits at 0.9 nz; in every (x, y) column the nearest surface wins
    (z-buffer).  Per-facet reflectance ~ U[0.2, 1].  Returns float64 r[nz][ny][nx].
    """
    u = uniform(seed, 3, 64)
    nf = 3 + int(u[0] * 4) % 4
    zbuf = np.full((ny, nx), 0.9 * nz)
    rbuf = np.full((ny, nx), 0.2 + 0.8 * u[1])
    yy, xx = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    for f in range(nf):
        v = uniform(seed, 10 + f, 8)
        x0, x1 = sorted((v[0] * nx, v[1] * nx))
        y0, y1 = sorted((v[2] * ny, v[3] * ny))
        x1 = max(x1, x0 + nx / 8)
        y1 = max(y1, y0 + ny / 8)
        p = (v[4] - 0.5) * 0.5 * nz / nx
        q = (v[5] - 0.5) * 0.5 * nz / ny
        c = (0.15 + 0.6 * v[6]) * nz
        cx, cy = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
        z = c + p * (xx - cx) + q * (yy - cy)
        inside = (xx >= x0) & (xx < x1) & (yy >= y0) & (yy < y1) & (z >= 0) & (z < zbuf)
        zbuf = np.where(inside, z, zbuf)
        rbuf = np.where(inside, 0.2 + 0.8 * v[7], rbuf)
    zi = np.clip(np.floor(zbuf + 0.5).astype(np.int64), 0, nz - 1)
    r = np.zeros((nz, ny, nx))
    iy, ix = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r[zi, iy, ix] = rbuf
    return r


def noise_variance_for_snr(r: np.ndarray, pupil: np.ndarray, window: np.ndarray, snr_db: float) -> float:
    """Noise variance sigma_w^2 giving ``snr_db`` over the aperture support.

    Signal power per in-aperture sample is its expectation under the speckle model,
    E|a_k (F g)_k|^2 = a_k^2 mean(r) (F orthonormal, g ~ CN(0, D(r))), averaged over
    the support of a; sigma_w^2 = P_s / 10^(snr/10).
    """
    a2 = (window.astype(np.float64)[:, None, None] * pupil.astype(np.float64)[None, :, :]) ** 2
    support = np.count_nonzero(a2)
    ps = float(r.mean()) * float(a2.sum()) / max(support, 1)
    return ps / (10.0 ** (snr_db / 10.0))


def cnn_weights(layers: int, channels: int, seed: int, last_scale: float = 0.01):
    """Seeded He-normal 3x3x3 conv weights for the residual CNN denoiser.

    Layer i maps c_in -> c_out (1 -> C -> ... -> C -> 1); weight layout
    ``[c_out][c_in][3][3][3]`` (dz, dy, dx), std sqrt(2 / (27 c_in)); the last
    layer is scaled by ``last_scale``; biases are zero.  Returns lists of float32.
    """
    ws, bs = [], []
    for i in range(layers):
        cin = 1 if i == 0 else channels
        cout = 1 if i == layers - 1 else channels
        std = math.sqrt(2.0 / (27.0 * cin))
        w = normal(seed, 100 + i, cout * cin * 27).reshape(cout, cin, 3, 3, 3) * std
        if i == layers - 1:
            w = w * last_scale
        ws.append(w.astype(np.float32))
        bs.append(np.zeros(cout, dtype=np.float32))
    return ws, bs


def unet_layer_shapes(c1: int, c2: int, c3: int):
    """(weight shape, fan-in, c_out) of the 13 warm-start U-Net layers in parameter order
    (3x3x3 conv [c_out][c_in][3][3][3], transposed conv [c_in][c_out][2][2][2], 1x1 [1][c1])."""
    conv = lambda ci, co: ((co, ci, 3, 3, 3), 27 * ci, co)   # noqa: E731
    tconv = lambda ci, co: ((ci, co, 2, 2, 2), ci, co)        # noqa: E731
    return [conv(1, c1), conv(c1, c1), conv(c1, c2), conv(c2, c2), conv(c2, c3), conv(c3, c3), tconv(c3, c2),
            conv(2 * c2, c2), conv(c2, c2), tconv(c2, c1), conv(2 * c1, c1), conv(c1, c1), ((1, c1, 1, 1, 1), c1, 1)]


def unet_params(channels=(16, 32, 64), seed: int = 5) -> np.ndarray:
    """Seeded He-normal initial U-Net parameters (std sqrt(2 / fan_in), zero biases), flat float32."""
    parts = []
    for i, (shape, fan_in, co) in enumerate(unet_layer_shapes(*channels)):
        parts.append(normal(seed, 300 + i, int(np.prod(shape))) * math.sqrt(2.0 / fan_in))
        parts.append(np.zeros(co))
    return np.concatenate(parts).astype(np.float32)


def warmstart_specs(count: int = 2000, seed: int = 11, nx: int = 64, ny: int = 64, nz: int = 32, looks: int = 32,
                    iters: int = 80):
    """Training scenes of the warm start: column-surface scenes of one size, pupil radius
    U[0.3, 0.5] Nyquist, SNR U[5, 20] dB, each with its own seed."""
    u = uniform(seed, 600, 2 * count).reshape(count, 2)
    return [dict(nx=nx, ny=ny, nz=nz, looks=looks, radius=0.3 + 0.2 * u[i, 0], snr=5.0 + 15.0 * u[i, 1],
                 seed=seed * 100000 + i, iters=iters) for i in range(count)]


def prior_training_scenes(count: int, seed: int = 31, n: int = 32) -> np.ndarray:
    """Clean n^3 volumes for training the U-Net prior agent: alternating column-surface and
    facet scenes, each with its own seed.  float32 [count][n][n][n]."""
    out = np.empty((count, n, n, n), np.float32)
    for i in range(count):
        sd = seed * 100000 + i
        out[i] = column_surface_scene(n, n, n, sd) if i % 2 == 0 else facet_scene(n, n, n, sd)
    return out


# ----------------------------------------------------------------------------- workloads

@dataclass
class Workload:
    """One synthetic reconstruction problem: scene, looks' random draws and parameters."""
    name: str
    nx: int
    ny: int
    nz: int
    looks: int
    r_true: np.ndarray               # float64 [nz][ny][nx]
    speckle: np.ndarray              # complex128 [L][nz][ny][nx], CN(0,1)
    noise: np.ndarray                # complex128 [L][nz][ny][nx], CN(0,1)
    pupil: np.ndarray                # float32 [ny][nx]
    window: np.ndarray               # float32 [nz]
    noise_var: float                 # sigma_w^2
    prox_var: float                  # sigma^2
    rho: float = 0.5
    prior_weight: float = 0.5
    iters: int = 20
    denoiser: dict = field(default_factory=lambda: {"kind": "gauss", "sigma": 0.8})


def make_workload(name: str, seed: int = 1, *, nx=None, ny=None, nz=None, looks=None,
                  iters=None, with_draws: bool = True, q: float = 1.0) -> Workload:
    """Build one of the named synthetic workloads.

    ``tiny``      16x16x8, L=2, Gaussian denoiser (unit tests).
    ``cfg1``      32x32x16, L=4, pupil R=0.5, Hann window, 10 dB, Gaussian sigma 0.8, 20 iterations.
    ``cfg2``      128x128x64, L=16, R=0.4, 15 dB, residual CNN 5 layers x 32 ch FP32, 50 iterations.
    ``cfg3``      256x256x128, L=32, facets, R=0.35, 10 dB, residual CNN 8 layers x 48 ch.
    ``warm``      256x256x128, L=32, columns, R=0.4, 1.5 dB, Gaussian sigma 0.8 (warm-start comparison;
                  the SNR is relative to mean(r), so 1.5 dB at nz = 128 is the per-surface-voxel SNR
                  of 7.5 dB at nz = 32).
    Size keywords override the shape (same generator and parameters).  ``q`` > 1 is the
    zero-padding factor (Sec. II-B, Sec. IV): the shape is the padded grid, the measured
    band is 1/q of it in every dimension (pupil radius R / q of the padded Nyquist,
    ``band_window(nz, q)``), and the scene lives on the padded (finer) grid.
    """
    presets = {
        "tiny": dict(nx=16, ny=16, nz=8, looks=2, radius=0.5, snr=10.0, scene="columns",
                     den={"kind": "gauss", "sigma": 0.8}, iters=5),
        "cfg1": dict(nx=32, ny=32, nz=16, looks=4, radius=0.5, snr=10.0, scene="columns",
                     den={"kind": "gauss", "sigma": 0.8}, iters=20),
        "cfg2": dict(nx=128, ny=128, nz=64, looks=16, radius=0.4, snr=15.0, scene="columns",
                     den={"kind": "cnn", "layers": 5, "channels": 32, "dtype": "fp32"}, iters=50),
        "cfg3": dict(nx=256, ny=256, nz=128, looks=32, radius=0.35, snr=10.0, scene="facets",
                     den={"kind": "cnn", "layers": 8, "channels": 48, "dtype": "bf16"}, iters=20),
        "warm": dict(nx=256, ny=256, nz=128, looks=32, radius=0.4, snr=1.5, scene="columns",
                     den={"kind": "gauss", "sigma": 0.8}, iters=400),
    }
    p = dict(presets[name])
    nx = nx or p["nx"]
    ny = ny or p["ny"]
    nz = nz or p["nz"]
    L = looks or p["looks"]
    if p["scene"] == "columns":
        r = column_surface_scene(nx, ny, nz, seed)
    else:
        r = facet_scene(nx, ny, nz, seed)
    pupil = circular_pupil(nx, ny, p["radius"] / q)
    window = band_window(nz, q)
    nv = noise_variance_for_snr(r, pupil, window, p["snr"])
    shape = (L, nz, ny, nx)
    if with_draws:
        spk = complex_normal(seed, 20, shape)
        eta = complex_normal(seed, 21, shape)
    else:
        spk = eta = None
    den = dict(p["den"])
    if den["kind"] == "cnn":
        den["weights"], den["biases"] = cnn_weights(den["layers"], den["channels"], seed)
    return Workload(name=name, nx=nx, ny=ny, nz=nz, looks=L, r_true=r, speckle=spk, noise=eta,
                    pupil=pupil, window=window, noise_var=float(nv), prox_var=1e-4,
                    iters=iters or p["iters"], denoiser=den)


def batch_specs(count: int = 24, seed: int = 7, lateral=(64, 96, 128, 192, 256), rng_z=(32, 64, 128),
                looks=(4, 32), iters: int = 10):
    """Seeded shapes and parameters of a batch of uneven scenes: square lateral size from
    ``lateral``, range size from ``rng_z``, looks uniform in ``looks`` (inclusive), pupil
    radius U[0.3, 0.5] Nyquist, SNR U[5, 20] dB."""
    u = uniform(seed, 500, 6 * count).reshape(count, 6)
    specs = []
    for i in range(count):
        nxy = lateral[int(u[i, 0] * len(lateral)) % len(lateral)]
        nz = rng_z[int(u[i, 1] * len(rng_z)) % len(rng_z)]
        L = looks[0] + int(u[i, 2] * (looks[1] - looks[0] + 1)) % (looks[1] - looks[0] + 1)
        specs.append(dict(nx=nxy, ny=nxy, nz=nz, looks=L, radius=0.3 + 0.2 * u[i, 3], snr=5.0 + 15.0 * u[i, 4],
                          seed=seed * 1000 + i, iters=iters))
    return specs


def batch_scene(spec: dict, with_draws: bool = True) -> Workload:
    """One scene of a batch (column-surface scene, Gaussian prior) from a spec of batch_specs."""
    nx, ny, nz, L, seed = spec["nx"], spec["ny"], spec["nz"], spec["looks"], spec["seed"]
    r = column_surface_scene(nx, ny, nz, seed)
    pupil = circular_pupil(nx, ny, spec["radius"])
    window = hann_window(nz)
    nv = noise_variance_for_snr(r, pupil, window, spec["snr"])
    shape = (L, nz, ny, nx)
    spk = complex_normal(seed, 20, shape) if with_draws else None
    eta = complex_normal(seed, 21, shape) if with_draws else None
    return Workload(name="batch", nx=nx, ny=ny, nz=nz, looks=L, r_true=r, speckle=spk, noise=eta, pupil=pupil,
                    window=window, noise_var=float(nv), prox_var=1e-4, iters=spec["iters"],
                    denoiser={"kind": "gauss", "sigma": 0.8})
