"""Full-size parity at 256x256x128, L = 32 (facet scene, BF16 CNN prior 8 x 48), in the
launch configuration the benchmark times.  The oracle computes sampled outputs one by
one: the forward agents of looks 0 and 31 on every voxel, the prior agent on a cropped
block with its receptive-field halo, the MACE step on a z-slab."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from oracle import clamp_oracle as O  # noqa: E402
from paper_2406_13651_gb300 import inputs as I  # noqa: E402

SAMPLED = (0, 31)


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    clamp.load()
    return clamp


def rel(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_fullsize_256_L32(C):
    wl = I.make_workload("cfg3", seed=1, with_draws=False)
    L, shape = wl.looks, (wl.nz, wl.ny, wl.nx)
    a = O.aperture(wl.pupil, wl.window)
    alpha = O.alpha_of(a)
    dev = torch.device("cuda")
    y = torch.zeros((L,) + shape, dtype=torch.complex64, device=dev)
    mu = torch.zeros_like(y)
    r = torch.empty((L + 1,) + shape, dtype=torch.float32, device=dev)
    w = torch.empty_like(r)
    ref = {}
    rng = np.random.default_rng(3)
    for l in SAMPLED:
        spk, eta = I.look_draws(wl, 1, l)
        y64 = O.simulate_data(wl.r_true, spk[None], eta[None], a, wl.noise_var).astype(np.complex64)
        st = O.init_state(y64.astype(np.complex128), a)
        mu0 = st.mu[0].astype(np.complex64)
        r0 = st.r[0].astype(np.float32)
        w0 = (st.r[0] * (1 + 0.3 * rng.uniform(-1, 1, shape))).astype(np.float32)
        y[l] = torch.from_numpy(y64[0]).to(dev)
        mu[l] = torch.from_numpy(mu0).to(dev)
        r[l] = torch.from_numpy(r0).to(dev)
        w[l] = torch.from_numpy(w0).to(dev)
        ref[l] = O.forward_agent(mu0.astype(np.complex128), r0.astype(np.float64), w0.astype(np.float64),
                                 y64[0].astype(np.complex128), a, wl.noise_var, wl.prox_var, alpha, O.beta_k(2))
    for l in range(L):   # looks that are not compared still carry a valid state
        if l not in SAMPLED:
            y[l], mu[l], r[l], w[l] = y[0], mu[0], r[0], w[0]
    r[L] = r[0]
    w[L] = w[0]
    p = C.make_params(wl.nx, wl.ny, wl.nz, L, wl.noise_var, wl.prox_var)
    C.forward_prox(p, 2, y, torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev), mu, r, w)
    torch.cuda.synchronize()
    for l in SAMPLED:
        mu_ref, r_ref, _, _ = ref[l]
        assert rel(mu[l].cpu().numpy(), mu_ref) < 1e-4, l
        assert rel(r[l].cpu().numpy(), r_ref) < 1e-4, l

    # prior agent (BF16 CNN, 8 layers of 48 channels) on a crop with an 8-voxel halo
    den = C.Denoiser.from_desc(wl.denoiser)
    prior_in = torch.from_numpy(rng.uniform(0.05, 1.0, shape).astype(np.float32)).to(dev)
    prior_out = torch.empty_like(prior_in)
    C.denoise(den, prior_in, prior_out)
    torch.cuda.synchronize()
    z0, y0, x0, h = 60, 100, 120, 8
    crop = prior_in.cpu().numpy()[z0 - h:z0 + 4 + h, y0 - h:y0 + 8 + h, x0 - h:x0 + 16 + h].astype(np.float64)
    cref = O.denoise_cnn(crop, wl.denoiser["weights"], wl.denoiser["biases"], bf16=True)[h:-h, h:-h, h:-h]
    got = prior_out.cpu().numpy()[z0:z0 + 4, y0:y0 + 8, x0:x0 + 16]
    src = crop[h:-h, h:-h, h:-h]
    assert rel(got - src, cref - src) < 1e-2
    assert rel(got, cref) < 1e-3

    # MACE step: every voxel is independent; compare a z-slab
    r_full = torch.from_numpy(rng.uniform(0.01, 1.0, (L + 1,) + shape).astype(np.float32)).to(dev)
    wbar = torch.empty(shape, dtype=torch.float32, device=dev)
    w_in = w.clone()
    C.mace_step(p, r_full, w, wbar)
    torch.cuda.synchronize()
    zs = slice(40, 42)
    ups = O.consensus_weights(L)
    w_ref = O.mace_update(r_full[:, zs].cpu().numpy().astype(np.float64),
                          w_in[:, zs].cpu().numpy().astype(np.float64), ups, 0.5)
    assert rel(w[:, zs].cpu().numpy(), w_ref) < 1e-6
    assert rel(wbar[zs].cpu().numpy(), O.G_avg(w_ref, ups)) < 1e-6
