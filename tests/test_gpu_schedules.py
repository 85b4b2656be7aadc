"""Both forward-agent schedules against the FP64 oracle: the full-spectrum schedule (five
FFT passes over the whole volume) and the band-limited one (x over whole rows, y and z on
the pupil's support only, F mu advanced by gamma F d).  Pupils: the circular ones of the
workloads, a single nonzero column, a ragged random support, and one too wide for the
band-limited arrays (which must fall back to the full spectrum)."""
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
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def to_dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _pupil(kind, nx, ny, rng):
    if kind == "circle":
        return I.circular_pupil(nx, ny, 0.4)
    if kind == "one_column":
        p = np.zeros((ny, nx), np.float32)
        p[3 % ny, 5 % nx] = 1.0
        p[(ny - 2) % ny, 5 % nx] = 0.5
        return p
    if kind == "ragged":
        return ((rng.uniform(size=(ny, nx)) < 0.12) * rng.uniform(0.5, 1.0, (ny, nx))).astype(np.float32)
    if kind == "wide":
        return I.circular_pupil(nx, ny, 1.3)   # covers most of the plane: band arrays do not fit
    raise ValueError(kind)


def _problem(shape, L, pupil_kind, seed):
    nx, ny, nz = shape
    wl = I.make_workload("cfg1", seed=seed, nx=nx, ny=ny, nz=nz, looks=L, iters=6)
    rng = np.random.default_rng(seed)
    wl.pupil = _pupil(pupil_kind, nx, ny, rng)
    wl.noise_var = I.noise_variance_for_snr(wl.r_true, wl.pupil, wl.window, 10.0)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    return wl, a, y32


ROW_VARIANT = {"band": 0, "band_half_rows": 1, "band_late_loads": 2}


@pytest.mark.parametrize("flag", ["full", "band", "band_half_rows", "band_late_loads"])
@pytest.mark.parametrize("shape,L,pupil_kind", [((64, 32, 16), 2, "circle"), ((96, 96, 32), 1, "circle"),
                                                 ((16, 8, 8), 1, "one_column"), ((96, 32, 16), 3, "ragged"),
                                                 ((32, 32, 16), 2, "wide"), ((256, 16, 8), 2, "circle")])
def test_forward_prox_both_schedules(C, flag, shape, L, pupil_kind):
    wl, a, y32 = _problem(shape, L, pupil_kind, seed=sum(shape) + L)
    alpha = O.alpha_of(a)
    st = O.init_state(y32.astype(np.complex128), a)
    rng = np.random.default_rng(1)
    w = st.r[:L] * (1 + 0.3 * rng.uniform(-1, 1, st.r[:L].shape))
    mu0 = st.mu.astype(np.complex64)
    r0 = st.r[:L].astype(np.float32)
    w0 = w.astype(np.float32)
    refs = [O.forward_agent(mu0[l].astype(np.complex128), r0[l].astype(np.float64), w0[l].astype(np.float64),
                            y32[l].astype(np.complex128), a, wl.noise_var, wl.prox_var, alpha, O.beta_k(3))
            for l in range(L)]
    f = C.FLAG_FULL_SPECTRUM if flag == "full" else C.FLAG_BAND_SPECTRUM
    p = C.make_params(wl.nx, wl.ny, wl.nz, L, wl.noise_var, wl.prox_var, flags=f)
    C.autotune_set_band(p, ROW_VARIANT.get(flag, 0))
    mu, r, wd = to_dev(mu0), to_dev(r0), to_dev(w0)
    mres = torch.zeros((), dtype=torch.float64, device="cuda")
    try:
        C.forward_prox(p, 3, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), mu, r, wd, mu_residual=mres)
        torch.cuda.synchronize()
    finally:
        C.autotune_set_band(p, 0)
    for l in range(L):
        assert rel(mu[l].cpu().numpy(), refs[l][0]) < 1e-5, l
        assert rel(r[l].cpu().numpy(), refs[l][1]) < 1e-5, l
    mr = O.mu_residual(mu0.astype(np.complex128), y32.astype(np.complex128), r0.astype(np.float64), a,
                       wl.noise_var, alpha, floored=True)
    assert float(mres.item()) == pytest.approx(mr, rel=1e-4)


@pytest.mark.parametrize("shape,L,pupil_kind", [((64, 64, 32), 3, "circle"), ((16, 8, 8), 2, "one_column"),
                                                 ((64, 32, 32), 2, "ragged"), ((32, 32, 16), 2, "wide")])
def test_reconstruct_both_schedules(C, shape, L, pupil_kind):
    """Six iterations: both schedules against the oracle, and against each other."""
    wl, a, y32 = _problem(shape, L, pupil_kind, seed=7 + L)
    ref, st = O.reconstruct(y32.astype(np.complex128), wl.pupil, wl.window, wl.denoiser, wl.noise_var,
                            wl.prox_var, 6)
    out = {}
    for flag in ("full", "band", "band_half_rows", "band_late_loads"):
        f = C.FLAG_FULL_SPECTRUM if flag == "full" else C.FLAG_BAND_SPECTRUM
        p = C.make_params(wl.nx, wl.ny, wl.nz, L, wl.noise_var, wl.prox_var, max_iters=6, flags=f)
        C.autotune_set_band(p, ROW_VARIANT.get(flag, 0))
        try:
            res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), C.Denoiser.gauss(0.8))
        finally:
            C.autotune_set_band(p, 0)
        out[flag] = res.r.cpu().numpy()
        assert rel(out[flag], ref) < 1e-4, flag
        np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)
        np.testing.assert_allclose(res.mu_hist, st.mu_res_hist, rtol=1e-3)
    assert rel(out["band"], out["full"]) < 2e-5
    assert rel(out["band_half_rows"], out["band"]) < 2e-5
    assert rel(out["band_late_loads"], out["band"]) < 2e-5


def test_band_schedule_long_run_tracks_oracle(C):
    """The band-limited spectrum is advanced by gamma F d for the whole run (formed from mu
    once per call): after 40 iterations it still matches the oracle, which forms F mu
    afresh every iteration."""
    wl, a, y32 = _problem((64, 64, 32), 2, "circle", seed=3)
    ref, st = O.reconstruct(y32.astype(np.complex128), wl.pupil, wl.window, wl.denoiser, wl.noise_var,
                            wl.prox_var, 40)
    p = C.make_params(wl.nx, wl.ny, wl.nz, 2, wl.noise_var, wl.prox_var, max_iters=40, flags=C.FLAG_BAND_SPECTRUM)
    res = C.reconstruct(p, to_dev(y32), to_dev(wl.pupil), to_dev(wl.window), C.Denoiser.gauss(0.8))
    assert rel(res.r.cpu().numpy(), ref) < 1e-4
    np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)
