"""GPU parity: every CUDA entry point against the FP64 oracle on the same seeded
inputs (fp32-rounded inputs are given to both sides).

Tolerances: the FP32 FFT/MM path must match the oracle within relative L2
error 1e-4 on reflectance (the FP32 target); single FFTs within 1e-5.
"""
import ctypes
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import clamp_oracle as O  # noqa: E402
from paper_2406_13651_gb300 import inputs as I  # noqa: E402

TOL_RECON = 1e-4
TOL_FFT = 1e-5


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    clamp.load()
    return clamp


def dev():
    return torch.device("cuda")


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to(dev())


def problem(name="cfg1", seed=1, **kw):
    """Workload + fp32-rounded data y (complex64) and its fp64 copy."""
    wl = I.make_workload(name, seed=seed, **kw)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    return wl, a, y32, y32.astype(np.complex128)


def params(C, wl, **kw):
    return C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, **kw)


# ------------------------------------------------------------------ FFT (Eq. A)

@pytest.mark.parametrize("shape", [(32, 96, 96), (64, 192, 96), (32, 64, 192), (96, 16, 16), (8, 16, 16), (16, 16, 16), (16, 32, 32), (64, 128, 128), (256, 16, 16), (16, 256, 16),
                                   (16, 16, 256), (32, 64, 128), (128, 256, 256)])
def test_fft3_matches_oracle(C, shape):
    rng = np.random.default_rng(0)
    batch = 2 if np.prod(shape) < 2**22 else 1
    x = (rng.standard_normal((batch,) + shape) + 1j * rng.standard_normal((batch,) + shape)).astype(np.complex64)
    xd = to_dev(x)
    f = C.fft3(xd).cpu().numpy()
    assert rel(f, O.fft3(x.astype(np.complex128))) < TOL_FFT
    b = C.fft3(xd, inverse=True).cpu().numpy()
    assert rel(b, O.ifft3(x.astype(np.complex128))) < TOL_FFT
    # in place round trip
    C.fft3(xd, out=xd)
    C.fft3(xd, inverse=True, out=xd)
    assert rel(xd.cpu().numpy(), x) < TOL_FFT


# ------------------------------------------------------------------ simulation and initialisation

def test_simulate_matches_oracle(C):
    wl = I.make_workload("cfg1", seed=2)
    a = O.aperture(wl.pupil, wl.window)
    spk = wl.speckle.astype(np.complex64)
    eta = wl.noise.astype(np.complex64)
    r32 = wl.r_true.astype(np.float32)
    ref = O.simulate_data(r32.astype(np.float64), spk.astype(np.complex128), eta.astype(np.complex128), a,
                          wl.noise_var)
    p = params(C, wl)
    y = C.simulate(p, to_dev(r32), to_dev(spk), to_dev(eta), to_dev(wl.pupil), to_dev(wl.window))
    assert rel(y.cpu().numpy(), ref) < TOL_FFT


@pytest.mark.parametrize("with_rinit", [False, True])
def test_init_matches_oracle(C, with_rinit):
    wl, a, y32, y64 = problem("cfg1", seed=3)
    r_init = None
    if with_rinit:
        r_init = (0.05 + wl.r_true).astype(np.float32)
    st = O.init_state(y64, a, None if r_init is None else r_init.astype(np.float64))
    p = params(C, wl)
    mu, r, w = C.init(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window),
                      None if r_init is None else to_dev(r_init))
    torch.cuda.synchronize()
    assert rel(mu.cpu().numpy(), st.mu) < TOL_FFT
    assert rel(r.cpu().numpy(), st.r) < TOL_FFT
    assert rel(w.cpu().numpy(), st.w) < TOL_FFT


# ------------------------------------------------------------------ forward agent (Alg. 2 steps 5-9)

def _agent_reference(st, y64, a, wl, k):
    alpha = O.alpha_of(a)
    beta = O.beta_k(k)
    mu_new = np.empty_like(st.mu)
    r_new = np.empty_like(st.r[:wl.looks])
    for l in range(wl.looks):
        mu_new[l], r_new[l], _, _ = O.forward_agent(st.mu[l], st.r[l], st.w[l], y64[l], a, wl.noise_var,
                                                   wl.prox_var, alpha, beta)
    mres = O.mu_residual(st.mu, y64, st.r[:wl.looks], a, wl.noise_var, alpha, floored=True)
    return mu_new, r_new, mres


@pytest.mark.parametrize("k", [1, 7])
def test_forward_prox_matches_oracle(C, k):
    wl, a, y32, y64 = problem("cfg1", seed=4)
    st = O.init_state(y64, a)
    # perturb w away from r so the prox has work to do
    rng = np.random.default_rng(5)
    st.w = (st.w * (1 + 0.3 * rng.uniform(-1, 1, st.w.shape))).astype(np.float32).astype(np.float64)
    st.mu = st.mu.astype(np.complex64).astype(np.complex128)
    st.r = st.r.astype(np.float32).astype(np.float64)
    mu_ref, r_ref, mres_ref = _agent_reference(st, y64, a, wl, k)
    p = params(C, wl)
    mu = to_dev(st.mu.astype(np.complex64))
    r = to_dev(st.r.astype(np.float32))
    w = to_dev(st.w.astype(np.float32))
    mres = torch.zeros(1, dtype=torch.float64, device=dev())
    C.forward_prox(p, k, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), mu, r, w, mu_residual=mres)
    torch.cuda.synchronize()
    assert rel(mu.cpu().numpy(), mu_ref) < TOL_RECON
    assert rel(r.cpu().numpy()[:wl.looks], r_ref) < TOL_RECON
    # the prior row is untouched
    np.testing.assert_array_equal(r.cpu().numpy()[wl.looks], st.r[wl.looks].astype(np.float32))
    assert mres.item() == pytest.approx(mres_ref, rel=1e-4)


@pytest.mark.parametrize("nx,ny,nz", [(96, 96, 32), (192, 64, 32)])
def test_forward_prox_radix3_sizes(C, nx, ny, nz):
    """Lateral sizes 96 and 192 (radix-3 stages) of the batched workload."""
    wl, a, y32, y64 = problem("cfg1", seed=9, nx=nx, ny=ny, nz=nz, looks=3)
    st = O.init_state(y64, a)
    st.mu = st.mu.astype(np.complex64).astype(np.complex128)
    st.r = st.r.astype(np.float32).astype(np.float64)
    st.w = (st.w * 1.1).astype(np.float32).astype(np.float64)
    mu_ref, r_ref, _ = _agent_reference(st, y64, a, wl, 4)
    p = params(C, wl)
    mu, r, w = to_dev(st.mu.astype(np.complex64)), to_dev(st.r.astype(np.float32)), to_dev(st.w.astype(np.float32))
    C.forward_prox(p, 4, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), mu, r, w)
    torch.cuda.synchronize()
    assert rel(mu.cpu().numpy(), mu_ref) < TOL_RECON
    assert rel(r.cpu().numpy()[:wl.looks], r_ref) < TOL_RECON


def test_forward_prox_single_look_no_aperture(C):
    """Degenerate case L = 1, a == 1 (binary, everything passes)."""
    wl, _, _, _ = problem("cfg1", seed=6, looks=1)
    ones_p = np.ones_like(wl.pupil)
    ones_w = np.ones_like(wl.window)
    a = O.aperture(ones_p, ones_w)
    y64 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64).astype(np.complex128)
    st = O.init_state(y64, a)
    st.mu = st.mu.astype(np.complex64).astype(np.complex128)
    st.r = st.r.astype(np.float32).astype(np.float64)
    st.w = st.w.astype(np.float32).astype(np.float64)
    mu_ref, r_ref, _ = _agent_reference(st, y64, a, wl, 3)
    p = params(C, wl)
    mu, r, w = to_dev(st.mu.astype(np.complex64)), to_dev(st.r.astype(np.float32)), to_dev(st.w.astype(np.float32))
    C.forward_prox(p, 3, to_dev(y64.astype(np.complex64)), to_dev(ones_p), to_dev(ones_w), mu, r, w)
    torch.cuda.synchronize()
    assert rel(mu.cpu().numpy(), mu_ref) < TOL_RECON
    assert rel(r.cpu().numpy()[:1], r_ref) < TOL_RECON


# ------------------------------------------------------------------ MACE step (Eq. mann)

def test_mace_step_matches_oracle(C):
    rng = np.random.default_rng(7)
    L, shape = 5, (16, 32, 64)
    r = rng.uniform(0.01, 1, (L + 1,) + shape).astype(np.float32)
    w = rng.uniform(0.01, 1, (L + 1,) + shape).astype(np.float32)
    ups = O.consensus_weights(L, 0.5)
    ce_ref = O.convergence_error(r.astype(np.float64), w.astype(np.float64), ups)
    w_ref = O.mace_update(r.astype(np.float64), w.astype(np.float64), ups, 0.5)
    p = C.make_params(64, 32, 16, L, 1e-3, 1e-4)
    wd = to_dev(w)
    wbar = torch.empty(shape, dtype=torch.float32, device=dev())
    ce = torch.zeros(1, dtype=torch.float64, device=dev())
    C.mace_step(p, to_dev(r), wd, wbar, ce)
    torch.cuda.synchronize()
    assert rel(wd.cpu().numpy(), w_ref) < 1e-6
    assert rel(wbar.cpu().numpy(), O.G_avg(w_ref, ups)) < 1e-6
    assert ce.item() == pytest.approx(ce_ref, rel=1e-5)


# ------------------------------------------------------------------ prior agents

def test_gauss_denoiser_matches_oracle(C):
    rng = np.random.default_rng(8)
    x = rng.uniform(0, 1, (16, 32, 64)).astype(np.float32)
    den = C.Denoiser.gauss(0.8)
    out = torch.empty_like(to_dev(x))
    C.denoise(den, to_dev(x), out)
    torch.cuda.synchronize()
    assert rel(out.cpu().numpy(), O.denoise_gauss(x.astype(np.float64), 0.8)) < 1e-6


@pytest.mark.parametrize("shape", [(16, 32, 32), (20, 24, 48)])
def test_cnn_fp32_denoiser_matches_oracle(C, shape):
    ws, bs = I.cnn_weights(5, 32, seed=3, last_scale=0.3)
    rng = np.random.default_rng(9)
    bs = [b + 0.05 * rng.standard_normal(b.shape).astype(np.float32) for b in bs]
    x = rng.uniform(0, 1, shape).astype(np.float32)
    den = C.Denoiser.cnn(ws, bs, "fp32")
    out = torch.empty_like(to_dev(x))
    C.denoise(den, to_dev(x), out)
    torch.cuda.synchronize()
    ref = O.denoise_cnn(x.astype(np.float64), ws, bs)
    assert rel(out.cpu().numpy() - x, ref - x) < 1e-5   # the CNN branch itself
    assert rel(out.cpu().numpy(), ref) < 1e-6


# ------------------------------------------------------------------ end to end (Alg. 2)

@pytest.mark.parametrize("name,iters", [("tiny", 8), ("cfg1", 20)])
def test_reconstruct_matches_oracle(C, name, iters):
    wl, a, y32, y64 = problem(name, seed=1, iters=iters)
    ref, st = O.reconstruct(y64, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, iters)
    p = params(C, wl, max_iters=iters)
    den = C.Denoiser.from_desc(wl.denoiser)
    res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), den)
    torch.cuda.synchronize()
    assert res.iters == iters
    assert rel(res.r.cpu().numpy(), ref) < TOL_RECON
    np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)
    np.testing.assert_allclose(res.mu_hist, st.mu_res_hist, rtol=1e-3)


@pytest.mark.parametrize("shape,q", [((96, 96, 96), 1.5), ((64, 64, 32), 2.0)])
def test_reconstruct_zero_padded_matches_oracle(C, shape, q):
    """Data zero-padded by q (Sec. II-B, Sec. IV): the measured band is 1/q of the grid in
    every dimension (radix-3 transforms at q = 1.5)."""
    nx, ny, nz = shape
    wl = I.make_workload("cfg1", seed=4, nx=nx, ny=ny, nz=nz, looks=2, iters=6, q=q)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    ref, st = O.reconstruct(y32.astype(np.complex128), wl.pupil, wl.window, wl.denoiser, wl.noise_var,
                            wl.prox_var, 6)
    p = params(C, wl, max_iters=6)
    res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), C.Denoiser.from_desc(wl.denoiser))
    assert rel(res.r.cpu().numpy(), ref) < TOL_RECON
    np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)


@pytest.mark.parametrize("mode", ["exact_prox", "no_aperture", "both"])
def test_reconstruct_paper_variants_match_oracle(C, mode):
    """Exact cubic-root prox (Sec. III-B) and the no-aperture ablation (Sec. IV-A)."""
    exact, noap = mode in ("exact_prox", "both"), mode in ("no_aperture", "both")
    wl, a, y32, y64 = problem("tiny", seed=7, iters=8)
    ref, st = O.reconstruct(y64, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, 8,
                            exact_prox=exact, no_aperture=noap)
    flags = (C.FLAG_EXACT_PROX if exact else 0) | (C.FLAG_NO_APERTURE if noap else 0)
    p = params(C, wl, max_iters=8, flags=flags)
    res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), C.Denoiser.gauss(0.8))
    assert rel(res.r.cpu().numpy(), ref) < TOL_RECON
    np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)


def test_reconstruct_warm_start_with_mu_steps(C):
    """A given r_init with init_mu_steps: mu refined with r' = r_init held fixed before the
    first iteration, as the oracle's mu_presteps does."""
    wl, a, y32, y64 = problem("cfg1", seed=8, iters=6)
    r_init = (0.5 * wl.r_true + 0.01 + 0.004 * np.random.default_rng(8).uniform(size=wl.r_true.shape))
    r_init = r_init.astype(np.float32)
    ref, st = O.reconstruct(y64, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, 6,
                            r_init=r_init.astype(np.float64), init_mu_steps=4)
    p = params(C, wl, max_iters=6, init_mu_steps=4)
    res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), C.Denoiser.gauss(0.8),
                        r_init=to_dev(r_init))
    assert rel(res.r.cpu().numpy(), ref) < TOL_RECON
    np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)


def test_reconstruct_warm_start_and_tolerance(C):
    wl, a, y32, y64 = problem("cfg1", seed=2, iters=30)
    r_init = (wl.r_true + 0.01).astype(np.float32)
    ref, st = O.reconstruct(y64, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, 30,
                            r_init=r_init.astype(np.float64))
    p = params(C, wl, max_iters=30)
    den = C.Denoiser.gauss(0.8)
    res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), den, r_init=to_dev(r_init))
    assert rel(res.r.cpu().numpy(), ref) < TOL_RECON
    # early stop once the convergence error reaches tol
    tol = float(st.ce_hist[12]) * 1.0001
    p2 = params(C, wl, max_iters=30, tol=tol, check_every=1)
    res2 = C.reconstruct(p2, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), den, r_init=to_dev(r_init))
    first = int(np.argmax(np.asarray(st.ce_hist) <= tol)) + 1
    assert res2.converged and res2.iters == first


def test_reconstruct_host_matches_device(C):
    wl, a, y32, y64 = problem("cfg1", seed=3, iters=6)
    p = params(C, wl, max_iters=6)
    den = C.Denoiser.gauss(0.8)
    dres = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), den)
    hres = C.reconstruct_host(p, y32, wl.pupil, wl.window, den)
    np.testing.assert_array_equal(hres.r, dres.r.cpu().numpy())
    hres2 = C.reconstruct_host(p, y32, wl.pupil, wl.window, den)   # cached device buffers reused
    np.testing.assert_array_equal(hres2.r, hres.r)


def test_reconstruct_host_from_huge_page_buffers(C):
    """Staging buffers from clamp_host_alloc (huge pages, page-locked) give the same result as
    pageable numpy arrays; the blocks are zeroed, huge-page aligned, and freed with their tensors."""
    import gc
    wl, a, y32, y64 = problem("cfg1", seed=3, iters=6)
    p = params(C, wl, max_iters=6)
    den = C.Denoiser.gauss(0.8)
    ref = C.reconstruct_host(p, y32, wl.pupil, wl.window, den)
    yh = C.host_empty(y32.shape, torch.complex64)
    assert not yh.any() and yh.data_ptr() % (2 << 20) == 0
    yh.copy_(torch.from_numpy(y32))
    ph = C.host_empty(wl.pupil.shape, torch.float32)
    ph.copy_(torch.from_numpy(wl.pupil))
    wh = C.host_empty(wl.window.shape, torch.float32)
    wh.copy_(torch.from_numpy(wl.window))
    rh = C.host_empty((wl.nz, wl.ny, wl.nx), torch.float32)
    res = C.reconstruct_host(p, yh.numpy(), ph.numpy(), wh.numpy(), den, r_out=rh.numpy())
    np.testing.assert_array_equal(rh.numpy(), ref.r)
    np.testing.assert_array_equal(res.r, ref.r)
    del yh, ph, wh, rh, res
    gc.collect()
    lib = C.load()
    lib.clamp_host_free(None)                     # ignored
    lib.clamp_host_free(ctypes.c_void_p(4096))    # not from the allocator: ignored
    out = ctypes.c_void_p()
    assert lib.clamp_host_alloc(0, ctypes.byref(out)) == 1   # CLAMP_EINVAL


def test_reconstruct_cnn_prior_matches_oracle(C):
    """cfg2's prior (5-layer 32-channel FP32 residual CNN) inside the loop, on a 32x32x16 scene."""
    wl, a, y32, y64 = problem("cfg1", seed=4, iters=6)
    ws, bs = I.cnn_weights(5, 32, seed=4)
    den_desc = {"kind": "cnn", "weights": ws, "biases": bs, "dtype": "fp32"}
    ref, _ = O.reconstruct(y64, wl.pupil, wl.window, den_desc, wl.noise_var, wl.prox_var, 6)
    p = params(C, wl, max_iters=6)
    res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), C.Denoiser.from_desc(den_desc))
    assert rel(res.r.cpu().numpy(), ref) < TOL_RECON


# ------------------------------------------------------------------ full-size workload (128x128x64, L=16)

def test_full_size_forward_agent_and_mace(C):
    """One full iteration at the 128x128x64, L=16 size in the launch configuration the
    benchmark times; the forward agents are checked on every voxel (oracle in FP64),
    the CNN prior on a cropped block with a 5-voxel halo."""
    wl = I.make_workload("cfg2", seed=1)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    y64 = y32.astype(np.complex128)
    del wl.speckle, wl.noise
    st = O.init_state(y64, a)
    st.mu = st.mu.astype(np.complex64).astype(np.complex128)
    st.r = st.r.astype(np.float32).astype(np.float64)
    st.w = st.w.astype(np.float32).astype(np.float64)
    p = params(C, wl)
    mu, r, w = to_dev(st.mu.astype(np.complex64)), to_dev(st.r.astype(np.float32)), to_dev(st.w.astype(np.float32))
    C.forward_prox(p, 1, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), mu, r, w)
    torch.cuda.synchronize()
    mu_ref, r_ref, _ = _agent_reference(st, y64, a, wl, 1)
    assert rel(mu.cpu().numpy(), mu_ref) < TOL_RECON
    assert rel(r.cpu().numpy()[:wl.looks], r_ref) < TOL_RECON
    # CNN prior on a crop (receptive field of 5 layers = 5 voxels)
    den = C.Denoiser.from_desc(wl.denoiser)
    out = torch.empty_like(w[wl.looks])
    C.denoise(den, w[wl.looks].contiguous(), out)
    torch.cuda.synchronize()
    z0, y0, x0, h = 20, 40, 60, 5
    crop = st.w[wl.looks, z0 - h:z0 + 8 + h, y0 - h:y0 + 16 + h, x0 - h:x0 + 16 + h]
    ref = O.denoise_cnn(crop, wl.denoiser["weights"], wl.denoiser["biases"])[h:-h, h:-h, h:-h]
    got_all = out.cpu().numpy()
    assert rel(got_all[z0:z0 + 8, y0:y0 + 16, x0:x0 + 16], ref) < 1e-5
    # the two corners: the crop keeps the volume's own edge, so its zero padding there is
    # the volume's, and a 5-voxel halo on the inner side
    nz, ny, nx = got_all.shape
    for (z0, y0, x0) in [(0, 0, 0), (nz - 8, ny - 16, nx - 16)]:
        zl, yl, xl = max(z0 - h, 0), max(y0 - h, 0), max(x0 - h, 0)
        zh, yh, xh = min(z0 + 8 + h, nz), min(y0 + 16 + h, ny), min(x0 + 16 + h, nx)
        ref = O.denoise_cnn(st.w[wl.looks, zl:zh, yl:yh, xl:xh], wl.denoiser["weights"], wl.denoiser["biases"])
        ref = ref[z0 - zl:z0 - zl + 8, y0 - yl:y0 - yl + 16, x0 - xl:x0 - xl + 16]
        assert rel(got_all[z0:z0 + 8, y0:y0 + 16, x0:x0 + 16], ref) < 1e-5, (z0, y0, x0)


def test_prior_schedules_give_identical_results(C):
    """The prior agent beside the forward agents (second stream) or after them: the same
    kernels on the same inputs, so the reconstructions agree bit for bit."""
    wl, a, y32, y64 = problem("cfg1", seed=6, iters=5)
    ws_, bs_ = I.cnn_weights(5, 32, seed=6)
    den = C.Denoiser.from_desc({"kind": "cnn", "weights": ws_, "biases": bs_, "dtype": "fp32"})
    out = {}
    for name, flag in (("serial", C.FLAG_PRIOR_SERIAL), ("concurrent", C.FLAG_PRIOR_CONCURRENT)):
        p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=5, flags=flag)
        assert C.prior_concurrent(p) == (name == "concurrent")
        res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), den)
        out[name] = (res.r.cpu().numpy(), np.asarray(res.ce_hist))
    assert np.array_equal(out["serial"][0], out["concurrent"][0])
    assert np.array_equal(out["serial"][1], out["concurrent"][1])
