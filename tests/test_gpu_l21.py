"""The l2,1 prior agent (Sec. IV comparison prior: l2 across cross-range, l1 across range)
against the FP64 oracle: the denoiser alone on planes that are kept and planes that are
zeroed, in place, on one-CTA and many-CTA planes with a ragged last CTA, and a whole CLAMP
reconstruction with it as the prior agent."""
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
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / max(np.linalg.norm(b), 1e-300))


def _lam_between_norms(x):
    """A lam halfway between two neighbouring plane norms, so that about half the planes are
    zeroed and none sits at the threshold."""
    nrm = np.sort(np.sqrt(np.sum(x.astype(np.float64) ** 2, axis=(1, 2))))
    k = len(nrm) // 2
    return float(0.5 * (nrm[k - 1] + nrm[k])) if len(nrm) > 1 else float(0.5 * nrm[0])


# plane sizes: 1920 floats (one CTA, ragged), 65536 floats (16 CTAs), 256 floats (one CTA, ragged)
@pytest.mark.parametrize("shape", [(10, 40, 48), (8, 256, 256), (3, 16, 16)])
def test_l21_denoiser_matches_oracle(C, shape):
    rng = np.random.default_rng(sum(shape))
    scale = rng.uniform(0.2, 2.0, (shape[0], 1, 1))          # planes of different energy
    x = (rng.standard_normal(shape) * scale).astype(np.float32)
    lam = _lam_between_norms(x)
    ref = O.denoise_l21(x.astype(np.float64), lam)
    den = C.Denoiser.l21(lam)
    xd = torch.from_numpy(x).cuda()
    out = torch.empty_like(xd)
    C.denoise(den, xd, out)
    got = out.cpu().numpy()
    zeroed = [z for z in range(shape[0]) if not ref[z].any()]
    assert 0 < len(zeroed) < shape[0] or shape[0] == 1
    for z in zeroed:
        assert not got[z].any()
    assert rel(got, ref) < 1e-6
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(ref))
    # in place, and lam = 0 is the identity
    C.denoise(den, xd, xd)
    np.testing.assert_array_equal(xd.cpu().numpy(), got)
    C.denoise(C.Denoiser.l21(0.0), out, xd)
    np.testing.assert_array_equal(xd.cpu().numpy(), got)


def test_reconstruct_with_l21_prior_matches_oracle(C):
    wl = I.make_workload("cfg1", seed=5, looks=3, iters=10)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    r0 = O.speckle_average(y32.astype(np.complex128), a)
    lam = 0.05 * float(np.median(np.sqrt(np.sum(r0 ** 2, axis=(1, 2)))))
    den_desc = {"kind": "l21", "lam": lam}
    ref, st = O.reconstruct(y32.astype(np.complex128), wl.pupil, wl.window, den_desc, wl.noise_var,
                            wl.prox_var, 10)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=10)
    dev = torch.device("cuda")
    res = C.reconstruct(p, torch.from_numpy(y32).to(dev), torch.from_numpy(wl.pupil).to(dev),
                        torch.from_numpy(wl.window).to(dev), C.Denoiser.from_desc(den_desc))
    assert rel(res.r.cpu().numpy(), ref) < 1e-4
    np.testing.assert_allclose(res.ce_hist, st.ce_hist, rtol=1e-3)
