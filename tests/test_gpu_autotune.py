"""Autotuner: every launch variant of the full-spectrum schedule's passes matches the
oracle, and the tuner returns a valid variant for each pass (it also times the
band-limited schedule against them and caches the faster)."""
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
    a, b = np.asarray(a), np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _case(nx, ny, nz, L, seed):
    wl = I.make_workload("cfg1", seed=seed, nx=nx, ny=ny, nz=nz, looks=L)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    y64 = y32.astype(np.complex128)
    st = O.init_state(y64, a)
    st.mu = st.mu.astype(np.complex64).astype(np.complex128)
    st.r = st.r.astype(np.float32).astype(np.float64)
    st.w = (st.w * 0.9).astype(np.float32).astype(np.float64)
    alpha = O.alpha_of(a)
    ref = [O.forward_agent(st.mu[l], st.r[l], st.w[l], y64[l], a, wl.noise_var, wl.prox_var, alpha, O.beta_k(3))
           for l in range(L)]
    return wl, y32, st, np.stack([x[0] for x in ref]), np.stack([x[1] for x in ref])


@pytest.mark.parametrize("shape", [(32, 32, 16, 3), (96, 64, 32, 2), (256, 16, 16, 2)])
@pytest.mark.parametrize("variant", [0, 1, 2, 3])
def test_every_variant_matches_oracle(C, shape, variant):
    nx, ny, nz, L = shape
    wl, y32, st, mu_ref, r_ref = _case(nx, ny, nz, L, seed=nx + variant)
    # the variants belong to the full-spectrum schedule's five passes
    p = C.make_params(nx, ny, nz, L, wl.noise_var, wl.prox_var, flags=C.FLAG_FULL_SPECTRUM)
    dev = torch.device("cuda")
    C.autotune_set(p, [variant] * 5)
    try:
        mu = torch.from_numpy(st.mu.astype(np.complex64)).to(dev)
        r = torch.from_numpy(st.r.astype(np.float32)).to(dev)
        w = torch.from_numpy(st.w.astype(np.float32)).to(dev)
        C.forward_prox(p, 3, torch.from_numpy(y32).to(dev), torch.from_numpy(wl.pupil).to(dev),
                       torch.from_numpy(wl.window).to(dev), mu, r, w)
        torch.cuda.synchronize()
        assert rel(mu.cpu().numpy(), mu_ref) < 1e-4
        assert rel(r.cpu().numpy()[:L], r_ref) < 1e-4
    finally:
        C.autotune_set(p, [0] * 5)


def test_autotune_picks_valid_variants(C):
    wl, y32, _, _, _ = _case(96, 64, 32, 2, seed=5)
    p = C.make_params(96, 64, 32, 2, wl.noise_var, wl.prox_var)
    dev = torch.device("cuda")
    try:
        v = C.autotune(p, torch.from_numpy(y32).to(dev), torch.from_numpy(wl.pupil).to(dev),
                       torch.from_numpy(wl.window).to(dev))
        assert len(v) == 5 and all(x in (0, 1, 2, 3) for x in v)
    finally:
        C.autotune_set(p, [0] * 5)
