"""Thin Python binding of the CLAMP C ABI (``include/clamp.h``).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays are torch tensors on the current CUDA device (complex data as
``torch.complex64`` or trailing-dimension-2 ``float32``), passed by pointer;
streams are torch streams.  Loading fails loudly when the library has not been
built -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libclamp.so")
# the bounds-checking test build (build.build(checked=True)); load() takes it when the
# environment sets CLAMP_BOUNDS_CHECK=1
LIB_CHECKED_PATH = os.path.join(_PKG, "_lib", "libclamp_checked.so")

CLAMP_OK = 0
STATUS = {0: "CLAMP_OK", 1: "CLAMP_EINVAL", 2: "CLAMP_ENOMEM", 3: "CLAMP_ECUDA", 4: "CLAMP_ENOTCONV",
          5: "CLAMP_ETIMEOUT", 6: "CLAMP_ENONFINITE", 7: "CLAMP_EUNSUPPORTED"}
FLAG_MU_INIT_NO_ALPHA = 0x1
FLAG_EXACT_PROX = 0x2
FLAG_NO_APERTURE = 0x4
FLAG_PRIOR_CONCURRENT = 0x8
FLAG_PRIOR_SERIAL = 0x10
FLAG_FULL_SPECTRUM = 0x20
FLAG_BAND_SPECTRUM = 0x40
DENOISER_FP32 = 0
DENOISER_BF16 = 1

EXPORTS = [
    "clamp_last_error", "clamp_version", "clamp_supported_length", "clamp_check_params",
    "clamp_workspace_size", "clamp_reconstruct_workspace_size", "clamp_fft3", "clamp_simulate",
    "clamp_init", "clamp_forward_prox", "clamp_denoise", "clamp_mace_step",
    "clamp_denoiser_create_gauss", "clamp_denoiser_create_cnn", "clamp_denoiser_destroy", "clamp_denoiser_create_l21",
    "clamp_denoise_workspace_size", "clamp_reconstruct", "clamp_reconstruct_host", "clamp_release_cache",
    "clamp_iterate", "clamp_iterate_workspace_size", "clamp_mace_step_noalloc",
    "clamp_tc_gemm_bf16", "clamp_tc_gemm_tf32x3",
    "clamp_batch_workspace_size", "clamp_batch_create", "clamp_batch_launch", "clamp_batch_latencies",
    "clamp_batch_residuals", "clamp_batch_destroy", "clamp_autotune", "clamp_autotune_set", "clamp_agent_schedule", "clamp_autotune_set_band",
    "clamp_unet_create", "clamp_unet_destroy", "clamp_unet_param_count", "clamp_unet_get", "clamp_unet_set",
    "clamp_unet_workspace_size", "clamp_unet_forward", "clamp_unet_backward", "clamp_unet_adam",
    "clamp_speckle_average", "clamp_unet_normalize", "clamp_unet_warm_start", "clamp_unet_loss",
    "clamp_point_cloud_workspace_size", "clamp_point_cloud_metrics", "clamp_denoiser_create_unet",
    "clamp_selftest_bounded_wait", "clamp_prior_concurrent", "clamp_unet_set_tensor_cores", "clamp_unet_check",
    "clamp_bounds_check", "clamp_host_alloc", "clamp_host_free",
]


class ClampError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(ctypes.Structure):
    """Mirror of ``clamp_params``."""
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32),
                ("looks", ctypes.c_int32), ("noise_var", ctypes.c_float), ("prox_var", ctypes.c_float),
                ("rho", ctypes.c_float), ("prior_weight", ctypes.c_float), ("max_iters", ctypes.c_int32),
                ("k0", ctypes.c_int32), ("flags", ctypes.c_int32), ("check_every", ctypes.c_int32),
                ("tol", ctypes.c_double), ("init_mu_steps", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class Scene(ctypes.Structure):
    """Mirror of ``clamp_scene``."""
    _fields_ = [("p", Params), ("y", ctypes.c_void_p), ("pupil", ctypes.c_void_p), ("window", ctypes.c_void_p),
                ("r_out", ctypes.c_void_p)]


class Report(ctypes.Structure):
    """Mirror of ``clamp_report``."""
    _fields_ = [("iters", ctypes.c_int32), ("converged", ctypes.c_int32), ("ce_residual", ctypes.c_double),
                ("mu_residual", ctypes.c_double), ("ce_hist", ctypes.POINTER(ctypes.c_double)),
                ("mu_hist", ctypes.POINTER(ctypes.c_double))]


_lib = None


def load(path: str | None = None) -> ctypes.CDLL:
    """Loads libclamp.so (raises if it is missing: build it with ``__graft_entry__.build()``);
    with CLAMP_BOUNDS_CHECK=1 in the environment, the bounds-checking libclamp_checked.so."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = LIB_CHECKED_PATH if os.environ.get("CLAMP_BOUNDS_CHECK") == "1" else LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"CLAMP CUDA library not built: {path} is missing "
                           "(run `python -c 'import __graft_entry__ as g; g.build()'`)")
    lib = ctypes.CDLL(path)
    P, S, V, I, D = ctypes.c_void_p, ctypes.c_size_t, None, ctypes.c_int32, ctypes.c_double
    PP = ctypes.POINTER(Params)
    sig = {
        "clamp_last_error": (ctypes.c_char_p, []),
        "clamp_version": (ctypes.c_char_p, []),
        "clamp_supported_length": (I, [I]),
        "clamp_check_params": (I, [PP]),
        "clamp_prior_concurrent": (I, [PP]),
        "clamp_workspace_size": (S, [PP]),
        "clamp_reconstruct_workspace_size": (S, [PP, P]),
        "clamp_fft3": (I, [I, I, I, I, P, P, I, P]),
        "clamp_simulate": (I, [PP, P, P, P, P, P, P, P]),
        "clamp_init": (I, [PP, P, P, P, P, P, P, P, P, S, P]),
        "clamp_forward_prox": (I, [PP, I, P, P, P, P, P, P, P, P, S, P]),
        "clamp_denoise": (I, [P, P, P, I, I, I, P, S, P]),
        "clamp_mace_step": (I, [PP, P, P, P, P, P, S, P]),
        "clamp_denoiser_create_gauss": (I, [ctypes.c_float, ctypes.POINTER(P)]),
        "clamp_denoiser_create_l21": (I, [ctypes.c_float, ctypes.POINTER(P)]),
        "clamp_denoiser_create_cnn": (I, [I, I, I, P, P, ctypes.POINTER(P)]),
        "clamp_denoiser_destroy": (V, [P]),
        "clamp_denoise_workspace_size": (S, [P, I, I, I]),
        "clamp_reconstruct": (I, [PP, P, P, P, P, P, P, ctypes.POINTER(Report), P, S, P]),
        "clamp_reconstruct_host": (I, [PP, P, P, P, P, P, P, ctypes.POINTER(Report), P]),
        "clamp_release_cache": (V, []),
        "clamp_iterate_workspace_size": (S, [PP, P]),
        "clamp_iterate": (I, [PP, I, I, P, P, P, P, P, P, P, P, P, P, P, S, P, P]),
        "clamp_mace_step_noalloc": (I, [PP, P, P, P, P, P]),
        "clamp_tc_gemm_bf16": (I, [I, I, P, P, P, P]),
        "clamp_tc_gemm_tf32x3": (I, [I, I, P, P, P, P]),
        "clamp_batch_workspace_size": (S, [ctypes.POINTER(Scene), I, P]),
        "clamp_batch_create": (I, [ctypes.POINTER(Scene), I, P, P, S, ctypes.POINTER(P)]),
        "clamp_batch_launch": (I, [P, P]),
        "clamp_batch_latencies": (I, [P, P, ctypes.POINTER(ctypes.c_float)]),
        "clamp_batch_residuals": (I, [P, P, ctypes.POINTER(ctypes.c_double)]),
        "clamp_batch_destroy": (V, [P]),
        "clamp_autotune": (I, [PP, P, P, P, P, S, P, ctypes.POINTER(ctypes.c_int32)]),
        "clamp_autotune_set": (I, [PP, ctypes.POINTER(ctypes.c_int32)]),
        "clamp_agent_schedule": (I, [PP, P, P, P, ctypes.POINTER(ctypes.c_int32)]),
        "clamp_autotune_set_band": (I, [PP, I]),
        "clamp_unet_create": (I, [I, I, I, I, P, ctypes.POINTER(P)]),
        "clamp_unet_destroy": (V, [P]),
        "clamp_unet_param_count": (ctypes.c_int64, [P]),
        "clamp_unet_get": (I, [P, I, P]),
        "clamp_unet_set": (I, [P, I, P]),
        "clamp_unet_workspace_size": (S, [P, I, I, I, I, I]),
        "clamp_unet_forward": (I, [P, P, P, I, I, I, I, P, S, P]),
        "clamp_unet_backward": (I, [P, P, P, I, I, I, I, P, P, S, P]),
        "clamp_unet_adam": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, I, P]),
        "clamp_speckle_average": (I, [PP, P, P, P, P, P, S, P]),
        "clamp_unet_normalize": (I, [I, ctypes.c_int64, ctypes.c_int64, P, P, P, P, P]),
        "clamp_unet_set_tensor_cores": (I, [P, I]),
        "clamp_unet_check": (I, [P]),
        "clamp_unet_warm_start": (I, [P, I, I, I, P, ctypes.c_float, P, P, S, P]),
        "clamp_unet_loss": (I, [P, P, P, I, I, I, I, P, P, S, P]),
        "clamp_point_cloud_workspace_size": (S, []),
        "clamp_denoiser_create_unet": (I, [P, ctypes.c_float, ctypes.POINTER(P)]),
        "clamp_selftest_bounded_wait": (I, [I, ctypes.POINTER(ctypes.c_int32)]),
        "clamp_bounds_check": (I, [I, ctypes.POINTER(ctypes.c_uint32)]),
        "clamp_host_alloc": (I, [S, ctypes.POINTER(P)]),
        "clamp_host_free": (V, [P]),
        "clamp_point_cloud_metrics": (I, [P, P, I, I, I, ctypes.c_float, ctypes.c_float, P, P, S, P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != CLAMP_OK:
        raise ClampError(status, where, load().clamp_last_error().decode())


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    return t.data_ptr()


def _stream(stream) -> int | None:
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


def make_params(nx, ny, nz, looks, noise_var, prox_var, rho=0.5, prior_weight=0.5, max_iters=0, k0=0,
                flags=0, check_every=10, tol=0.0, init_mu_steps=0) -> Params:
    return Params(nx, ny, nz, looks, noise_var, prox_var, rho, prior_weight, max_iters, k0, flags,
                  check_every, tol, init_mu_steps, 0)


class Denoiser:
    """Owns a ``clamp_denoiser`` handle (created on the current CUDA device)."""

    def __init__(self, handle: int, desc: dict):
        self.handle = handle
        self.desc = desc

    @classmethod
    def gauss(cls, sigma: float = 0.8) -> "Denoiser":
        h = ctypes.c_void_p()
        _check(load().clamp_denoiser_create_gauss(sigma, ctypes.byref(h)), "clamp_denoiser_create_gauss")
        return cls(h.value, {"kind": "gauss", "sigma": sigma})

    @classmethod
    def l21(cls, lam: float) -> "Denoiser":
        """The l2,1 prior agent: each range bin's cross-range plane shrunk in l2 norm by lam."""
        h = ctypes.c_void_p()
        _check(load().clamp_denoiser_create_l21(lam, ctypes.byref(h)), "clamp_denoiser_create_l21")
        return cls(h.value, {"kind": "l21", "lam": lam})

    @classmethod
    def cnn(cls, weights, biases, dtype: str = "fp32") -> "Denoiser":
        layers = len(weights)
        channels = int(weights[0].shape[0])
        w = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).ravel() for x in weights]))
        b = np.ascontiguousarray(np.concatenate([np.asarray(x, np.float32).ravel() for x in biases]))
        h = ctypes.c_void_p()
        dt = DENOISER_BF16 if dtype == "bf16" else DENOISER_FP32
        _check(load().clamp_denoiser_create_cnn(layers, channels, dt, w.ctypes.data, b.ctypes.data,
                                                ctypes.byref(h)), "clamp_denoiser_create_cnn")
        return cls(h.value, {"kind": "cnn", "layers": layers, "channels": channels, "dtype": dtype})

    @classmethod
    def unet(cls, net: "UNet", floor: float = 1e-3) -> "Denoiser":
        """The U-Net prior agent H(w) = m max(U(w / m), floor), m = sum(w) / (nx ny)."""
        h = ctypes.c_void_p()
        _check(load().clamp_denoiser_create_unet(net.handle, floor, ctypes.byref(h)), "clamp_denoiser_create_unet")
        d = cls(h.value, {"kind": "unet", "params": net.get("params"), "channels": net.channels,
                          "dtype": net.dtype, "floor": floor})
        d._net = net   # the denoiser borrows the network: keep it alive as long as the denoiser
        return d

    @classmethod
    def from_desc(cls, desc: dict) -> "Denoiser":
        if desc["kind"] == "gauss":
            return cls.gauss(desc["sigma"])
        if desc["kind"] == "l21":
            return cls.l21(desc["lam"])
        if desc["kind"] == "unet":
            net = UNet(*desc["channels"], params=desc["params"], dtype=desc.get("dtype", "bf16"))
            return cls.unet(net, desc.get("floor", 1e-3))
        return cls.cnn(desc["weights"], desc["biases"], desc.get("dtype", "fp32"))

    def workspace_size(self, nx, ny, nz) -> int:
        return load().clamp_denoise_workspace_size(self.handle, nx, ny, nz)

    def close(self):
        if self.handle:
            load().clamp_denoiser_destroy(self.handle)
            self.handle = None
        self._net = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------ device-buffer calls

def _ws(nbytes: int):
    import torch
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device="cuda")


def workspace(p: Params):
    n = load().clamp_workspace_size(ctypes.byref(p))
    if n == 0:
        _check(load().clamp_check_params(ctypes.byref(p)), "clamp_workspace_size")
    return _ws(n)


def autotune(p: Params, y, pupil, window, ws=None, stream=None) -> list:
    """Times the forward-agent pass variants for this geometry and caches the fastest;
    returns the chosen variant of each of the 5 passes."""
    ws = workspace(p) if ws is None else ws
    out = (ctypes.c_int32 * 5)()
    _check(load().clamp_autotune(ctypes.byref(p), _ptr(y), _ptr(pupil), _ptr(window), _ptr(ws), ws.numel(),
                                 _stream(stream), out), "clamp_autotune")
    return list(out)


def autotune_set(p: Params, variants) -> None:
    arr = (ctypes.c_int32 * 5)(*variants)
    _check(load().clamp_autotune_set(ctypes.byref(p), arr), "clamp_autotune_set")


class _HostBlock:
    """Owns one clamp_host_alloc block; freed when the last tensor viewing it goes away."""

    def __init__(self, nbytes: int):
        ptr = ctypes.c_void_p()
        _check(load().clamp_host_alloc(nbytes, ctypes.byref(ptr)), "clamp_host_alloc")
        self.ptr = ptr.value
        self.nbytes = nbytes

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.clamp_host_free(self.ptr)
            self.ptr = None


def host_empty(shape, dtype):
    """A CPU torch tensor in huge-page, page-locked host memory from clamp_host_alloc (zeroed):
    the staging buffers for clamp_reconstruct_host."""
    import torch
    n = 1
    for d in shape:
        n *= int(d)
    esize = torch.empty((), dtype=dtype).element_size()
    blk = _HostBlock(max(n * esize, 1))
    arr = (ctypes.c_char * blk.nbytes).from_address(blk.ptr)
    arr._owner = blk   # the array (held by the tensor) keeps the block alive
    return torch.frombuffer(arr, dtype=dtype, count=n).view(tuple(int(d) for d in shape))


def bounds_check(reset: bool = True) -> tuple[bool, int]:
    """(checked build?, first out-of-range site code recorded, 0 if none); clears the
    record when ``reset``.  Only the bounds-checking build records anything."""
    site = ctypes.c_uint32(0)
    r = load().clamp_bounds_check(1 if reset else 0, ctypes.byref(site))
    if r < 0:
        _check(-r, "clamp_bounds_check")
    return bool(r), int(site.value)


def autotune_set_band(p: Params, row_variant: int) -> None:
    """Band-limited schedule's row pass for this geometry: 0 the default row tile, 1 half-height
    tiles, 2 the default tile with mu and r' read after the inverse transform."""
    _check(load().clamp_autotune_set_band(ctypes.byref(p), row_variant), "clamp_autotune_set_band")


def agent_schedule(p: Params, pupil, window, stream=None) -> dict:
    """The forward-agent schedule iterations with these parameters run, and the aperture's
    support and band column counts."""
    info = (ctypes.c_int32 * 5)()
    _check(load().clamp_agent_schedule(ctypes.byref(p), _ptr(pupil), _ptr(window), _stream(stream), info),
           "clamp_agent_schedule")
    return {"schedule": "band-limited" if info[0] else "full spectrum", "support_columns": int(info[1]),
            "band_columns": int(info[2]), "band_fits": bool(info[3]), "row_pass_variant": int(info[4])}


def fft3(x, inverse: bool = False, out=None, stream=None):
    """Orthonormal 3D DFT of complex64 x [..., nz, ny, nx] (batched over leading dims)."""
    import torch
    assert x.dtype == torch.complex64 and x.is_contiguous()
    nz, ny, nx = x.shape[-3:]
    batch = x.numel() // (nx * ny * nz)
    out = torch.empty_like(x) if out is None else out
    _check(load().clamp_fft3(nx, ny, nz, batch, _ptr(x), _ptr(out), 1 if inverse else 0, _stream(stream)),
           "clamp_fft3")
    return out


def simulate(p: Params, r, speckle, noise, pupil, window, stream=None, out=None):
    import torch
    y = torch.empty_like(speckle) if out is None else out
    _check(load().clamp_simulate(ctypes.byref(p), _ptr(r), _ptr(speckle), _ptr(noise), _ptr(pupil), _ptr(window),
                                 _ptr(y), _stream(stream)), "clamp_simulate")
    return y


def init(p: Params, y, pupil, window, r_init=None, ws=None, stream=None):
    """Returns (mu [L][n] complex64, r [L+1][n], w [L+1][n])."""
    import torch
    n = p.nx * p.ny * p.nz
    mu = torch.empty((p.looks, p.nz, p.ny, p.nx), dtype=torch.complex64, device=y.device)
    r = torch.empty((p.looks + 1, p.nz, p.ny, p.nx), dtype=torch.float32, device=y.device)
    w = torch.empty_like(r)
    ws = workspace(p) if ws is None else ws
    _check(load().clamp_init(ctypes.byref(p), _ptr(y), _ptr(pupil), _ptr(window), _ptr(r_init), _ptr(mu), _ptr(r),
                             _ptr(w), _ptr(ws), ws.numel(), _stream(stream)), "clamp_init")
    return mu, r, w


def speckle_average(p: Params, y, pupil, window, out=None, ws=None, stream=None):
    """r0 = (1/L) sum_l |A^H y_l|^2 (floored), device float32 [nz, ny, nx]."""
    import torch
    out = torch.empty((p.nz, p.ny, p.nx), dtype=torch.float32, device=y.device) if out is None else out
    ws = workspace(p) if ws is None else ws
    _check(load().clamp_speckle_average(ctypes.byref(p), _ptr(y), _ptr(pupil), _ptr(window), _ptr(out), _ptr(ws),
                                        ws.numel(), _stream(stream)), "clamp_speckle_average")
    return out


def forward_prox(p: Params, k: int, y, pupil, window, mu, r, w, mu_residual=None, ws=None, stream=None):
    ws = workspace(p) if ws is None else ws
    _check(load().clamp_forward_prox(ctypes.byref(p), k, _ptr(y), _ptr(pupil), _ptr(window), _ptr(mu), _ptr(r),
                                     _ptr(w), _ptr(mu_residual), _ptr(ws), ws.numel(), _stream(stream)),
           "clamp_forward_prox")


def denoise(den: Denoiser, w_prior, r_prior, ws=None, stream=None):
    nz, ny, nx = w_prior.shape[-3:]
    need = den.workspace_size(nx, ny, nz)
    if ws is None and need:
        ws = _ws(need)
    _check(load().clamp_denoise(den.handle, _ptr(w_prior), _ptr(r_prior), nx, ny, nz, _ptr(ws),
                                ws.numel() if ws is not None else 0, _stream(stream)), "clamp_denoise")


def mace_step(p: Params, r, w, wbar, ce_residual=None, ws=None, stream=None):
    ws = workspace(p) if ws is None else ws
    _check(load().clamp_mace_step(ctypes.byref(p), _ptr(r), _ptr(w), _ptr(wbar), _ptr(ce_residual), _ptr(ws),
                                  ws.numel(), _stream(stream)), "clamp_mace_step")


@dataclass
class Result:
    r: object
    iters: int
    converged: bool
    ce_hist: np.ndarray
    mu_hist: np.ndarray


def iterate_workspace(p: Params, den: Denoiser):
    n = load().clamp_iterate_workspace_size(ctypes.byref(p), den.handle)
    if n == 0:
        _check(load().clamp_check_params(ctypes.byref(p)), "clamp_iterate_workspace_size")
    return _ws(n)


def prior_concurrent(p: Params) -> bool:
    """Whether iterations with these parameters run the prior agent beside the forward agents."""
    v = load().clamp_prior_concurrent(ctypes.byref(p))
    if v < 0:
        raise ClampError(1, "clamp_prior_concurrent", load().clamp_last_error().decode())
    return bool(v)


def iterate(p: Params, k_first: int, iters: int, y, pupil, window, den: Denoiser, mu, r, w, wbar, ce_out=None,
            mu_out=None, ws=None, events=None, stream=None):
    """Runs ``iters`` CLAMP iterations on the caller-held state (mu, r, w); wbar receives the output.
    ``events``: optional list of 4*iters torch.cuda.Event (recorded per iteration around the phases)."""
    ws = iterate_workspace(p, den) if ws is None else ws
    ev = None
    if events is not None:
        if any(e.cuda_event == 0 for e in events):
            raise ValueError("events must have been recorded once (torch creates CUDA events lazily)")
        arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
        ev = ctypes.cast(arr, ctypes.c_void_p)
    _check(load().clamp_iterate(ctypes.byref(p), k_first, iters, _ptr(y), _ptr(pupil), _ptr(window), den.handle,
                                _ptr(mu), _ptr(r), _ptr(w), _ptr(wbar), _ptr(ce_out), _ptr(mu_out), _ptr(ws),
                                ws.numel(), ev, _stream(stream)), "clamp_iterate")


def reconstruct_workspace(p: Params, den: Denoiser):
    n = load().clamp_reconstruct_workspace_size(ctypes.byref(p), den.handle)
    if n == 0:
        _check(load().clamp_check_params(ctypes.byref(p)), "clamp_reconstruct_workspace_size")
    return _ws(n)


def reconstruct(p: Params, y, pupil, window, den: Denoiser, r_init=None, ws=None, r_out=None, report=True,
                stream=None) -> Result:
    import torch
    r_out = torch.empty((p.nz, p.ny, p.nx), dtype=torch.float32, device=y.device) if r_out is None else r_out
    rep = None
    ce = np.zeros(max(p.max_iters, 1))
    mh = np.zeros(max(p.max_iters, 1))
    if report:
        rep = Report(0, 0, 0.0, 0.0, ce.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                     mh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    wsp, wsn = (_ptr(ws), ws.numel()) if ws is not None else (None, 0)
    _check(load().clamp_reconstruct(ctypes.byref(p), _ptr(y), _ptr(pupil), _ptr(window), den.handle, _ptr(r_init),
                                    _ptr(r_out), ctypes.byref(rep) if rep else None, wsp, wsn, _stream(stream)),
           "clamp_reconstruct")
    it = rep.iters if rep else p.max_iters
    return Result(r_out, it, bool(rep.converged) if rep else False, ce[:it], mh[:it])


def reconstruct_host(p: Params, y: np.ndarray, pupil: np.ndarray, window: np.ndarray, den: Denoiser,
                     r_init: np.ndarray | None = None, r_out: np.ndarray | None = None, stream=None) -> Result:
    """Host-buffer reconstruction: numpy in, numpy out (copies inside the call)."""
    y = np.ascontiguousarray(y, dtype=np.complex64)
    pupil = np.ascontiguousarray(pupil, dtype=np.float32)
    window = np.ascontiguousarray(window, dtype=np.float32)
    ri = None if r_init is None else np.ascontiguousarray(r_init, dtype=np.float32)
    r_out = np.empty((p.nz, p.ny, p.nx), np.float32) if r_out is None else r_out
    ce = np.zeros(max(p.max_iters, 1))
    mh = np.zeros(max(p.max_iters, 1))
    rep = Report(0, 0, 0.0, 0.0, ce.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                 mh.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
    _check(load().clamp_reconstruct_host(ctypes.byref(p), y.ctypes.data, pupil.ctypes.data, window.ctypes.data,
                                         den.handle, None if ri is None else ri.ctypes.data, r_out.ctypes.data,
                                         ctypes.byref(rep), _stream(stream)), "clamp_reconstruct_host")
    return Result(r_out, rep.iters, bool(rep.converged), ce[:rep.iters], mh[:rep.iters])


class Batch:
    """Many reconstructions as one CUDA graph (``clamp_batch_*``).

    ``scenes``: list of (Params, y, pupil, window, r_out) with device tensors; they must
    stay alive while the batch is used."""

    def __init__(self, scenes, den: Denoiser):
        import torch
        self._keep = scenes
        self.den = den
        self.count = len(scenes)
        self._arr = (Scene * self.count)(*[Scene(p, _ptr(y), _ptr(pu), _ptr(wi), _ptr(ro))
                                            for (p, y, pu, wi, ro) in scenes])
        need = load().clamp_batch_workspace_size(self._arr, self.count, den.handle)
        if need == 0:
            raise ClampError(1, "clamp_batch_workspace_size", "invalid scene parameters")
        self.ws = _ws(need)
        h = ctypes.c_void_p()
        _check(load().clamp_batch_create(self._arr, self.count, den.handle, _ptr(self.ws), self.ws.numel(),
                                         ctypes.byref(h)), "clamp_batch_create")
        self.handle = h.value

    def launch(self, stream=None):
        _check(load().clamp_batch_launch(self.handle, _stream(stream)), "clamp_batch_launch")

    def latencies(self, stream=None) -> np.ndarray:
        out = np.zeros(self.count, np.float32)
        _check(load().clamp_batch_latencies(self.handle, _stream(stream),
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_float))),
               "clamp_batch_latencies")
        return out

    def residuals(self, stream=None) -> np.ndarray:
        out = np.zeros(self.count, np.float64)
        _check(load().clamp_batch_residuals(self.handle, _stream(stream),
                                            out.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
               "clamp_batch_residuals")
        return out

    def close(self):
        if self.handle:
            load().clamp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class UNet:
    """Owns a ``clamp_unet`` handle: the warm-start 3D U-Net (channels c1/c2/c3) with its
    FP32 master parameters, gradients and Adam moments on the current CUDA device."""

    STATE = {"params": 0, "grads": 1, "adam_m": 2, "adam_v": 3}

    def __init__(self, c1: int, c2: int, c3: int, params: np.ndarray | None = None, dtype: str = "bf16"):
        self.channels = (c1, c2, c3)
        self.dtype = dtype
        h = ctypes.c_void_p()
        dt = DENOISER_BF16 if dtype == "bf16" else DENOISER_FP32
        buf = None if params is None else np.ascontiguousarray(params, np.float32)
        _check(load().clamp_unet_create(c1, c2, c3, dt, None if buf is None else buf.ctypes.data, ctypes.byref(h)),
               "clamp_unet_create")
        self.handle = h.value
        self.count = int(load().clamp_unet_param_count(self.handle))
        if buf is not None and buf.size != self.count:
            self.close()
            raise ValueError(f"expected {self.count} parameters, got {buf.size}")
        self._ws = None
        self.step = 0

    def get(self, which: str = "params") -> np.ndarray:
        out = np.empty(self.count, np.float32)
        _check(load().clamp_unet_get(self.handle, self.STATE[which], out.ctypes.data), "clamp_unet_get")
        return out

    def set(self, values: np.ndarray, which: str = "params") -> None:
        buf = np.ascontiguousarray(values, np.float32)
        if buf.size != self.count:
            raise ValueError(f"expected {self.count} values, got {buf.size}")
        _check(load().clamp_unet_set(self.handle, self.STATE[which], buf.ctypes.data), "clamp_unet_set")

    def workspace(self, batch: int, nx: int, ny: int, nz: int, training: bool):
        need = load().clamp_unet_workspace_size(self.handle, batch, nx, ny, nz, int(training))
        if need == 0:
            raise ClampError(1, "clamp_unet_workspace_size", "nx, ny, nz must be multiples of 4")
        if self._ws is None or self._ws.numel() < need:
            self._ws = None
            self._ws = _ws(need)
        return self._ws

    def forward(self, x, out=None, stream=None):
        """x: float32 [B, nz, ny, nx] (or [nz, ny, nx]) on the device."""
        import torch
        shp = x.shape if x.dim() == 4 else (1,) + tuple(x.shape)
        B, nz, ny, nx = shp
        if out is None:
            out = torch.empty_like(x)
        ws = self.workspace(B, nx, ny, nz, False)
        _check(load().clamp_unet_forward(self.handle, _ptr(x), _ptr(out), B, nx, ny, nz, _ptr(ws), ws.numel(),
                                         _stream(stream)), "clamp_unet_forward")
        return out

    def backward(self, x, target, loss=None, stream=None):
        """Loss mean((U(x) - target)^2) into ``loss`` (device float64 scalar tensor, optional)
        and every parameter's gradient into the handle's gradient buffer."""
        shp = x.shape if x.dim() == 4 else (1,) + tuple(x.shape)
        B, nz, ny, nx = shp
        ws = self.workspace(B, nx, ny, nz, True)
        _check(load().clamp_unet_backward(self.handle, _ptr(x), _ptr(target), B, nx, ny, nz, _ptr(loss),
                                          _ptr(ws), ws.numel(), _stream(stream)), "clamp_unet_backward")

    def loss(self, x, target, loss, stream=None):
        """loss (device float64 scalar tensor) <- mean((U(x) - target)^2); no gradients."""
        shp = x.shape if x.dim() == 4 else (1,) + tuple(x.shape)
        B, nz, ny, nx = shp
        ws = self.workspace(B, nx, ny, nz, True)
        _check(load().clamp_unet_loss(self.handle, _ptr(x), _ptr(target), B, nx, ny, nz, _ptr(loss), _ptr(ws),
                                      ws.numel(), _stream(stream)), "clamp_unet_loss")

    def warm_start(self, r0, floor_rel: float = 1e-3, out=None, stream=None):
        """r_init = m * max(U(r0 / m), floor_rel), m = sum(r0) / (nx ny); r0 device float32 [nz, ny, nx]."""
        import torch
        nz, ny, nx = r0.shape
        out = torch.empty_like(r0) if out is None else out
        ws = self.workspace(1, nx, ny, nz, False)
        _check(load().clamp_unet_warm_start(self.handle, nx, ny, nz, _ptr(r0), floor_rel, _ptr(out), _ptr(ws),
                                            ws.numel(), _stream(stream)), "clamp_unet_warm_start")
        return out

    def adam(self, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8, stream=None):
        self.step += 1
        _check(load().clamp_unet_adam(self.handle, lr, beta1, beta2, eps, self.step, _stream(stream)),
               "clamp_unet_adam")

    def set_tensor_cores(self, on: bool) -> None:
        """BF16 networks: 3x3x3 convs on the tensor cores (default) or on the CUDA cores."""
        _check(load().clamp_unet_set_tensor_cores(self.handle, int(bool(on))), "clamp_unet_set_tensor_cores")

    def check(self) -> None:
        """Raises if a bounded tensor-core wait gave up since the last check (synchronous)."""
        _check(load().clamp_unet_check(self.handle), "clamp_unet_check")

    def close(self):
        if getattr(self, "handle", None):
            load().clamp_unet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def unet_normalize(x, t=None, x_out=None, t_out=None, stream=None):
    """Per-sample division of x [B, nz, ny, nx] (and t) by m_b = sum(x_b) / (nx ny); in place by default."""
    B = x.shape[0]
    n = x.numel() // B
    cols = x.shape[-1] * x.shape[-2]
    x_out = x if x_out is None else x_out
    if t is not None and t_out is None:
        t_out = t
    _check(load().clamp_unet_normalize(B, n, cols, _ptr(x), _ptr(t), _ptr(x_out), _ptr(t_out), _stream(stream)),
           "clamp_unet_normalize")
    return x_out, t_out


def point_cloud_metrics(r_hat, r_true, threshold: float, max_dist: float, stream=None) -> dict:
    """Point-cloud metrics (Sec. IV-B) of device volumes r_hat, r_true [nz, ny, nx]."""
    nz, ny, nx = r_hat.shape
    out = np.zeros(6, np.float64)
    ws = _ws(load().clamp_point_cloud_workspace_size())
    _check(load().clamp_point_cloud_metrics(_ptr(r_hat), _ptr(r_true), nx, ny, nz, threshold, max_dist,
                                            out.ctypes.data, _ptr(ws), ws.numel(), _stream(stream)),
           "clamp_point_cloud_metrics")
    return dict(distance=float(out[0]), false_positive_rate=float(out[1]), nrmse=float(out[2]), kept=int(out[3]),
                removed=int(out[4]), beta=float(out[5]))


def selftest_bounded_wait(limit: int = 1000) -> tuple:
    """(first wait succeeded, second wait succeeded): (1, 0) for a sound build."""
    out = (ctypes.c_int32 * 2)(-1, -1)
    _check(load().clamp_selftest_bounded_wait(limit, out), "clamp_selftest_bounded_wait")
    return int(out[0]), int(out[1])
