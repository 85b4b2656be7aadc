"""Point-cloud metrics (Sec. IV-B) on the GPU against the oracle: the counts are
integers and must agree exactly, the mean distance is a sum of square roots of integers,
NRMSE and beta* are FP64 sums over the same matched pairs."""
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


def _check(got, ref):
    assert got["kept"] == ref["kept"] and got["removed"] == ref["removed"], (got, ref)
    assert abs(got["distance"] - ref["distance"]) <= 1e-12 * max(1.0, ref["distance"])
    assert abs(got["false_positive_rate"] - ref["false_positive_rate"]) <= 1e-15
    assert abs(got["nrmse"] - ref["nrmse"]) <= 1e-9 * max(1.0, ref["nrmse"])
    assert abs(got["beta"] - ref["beta"]) <= 1e-9 * max(1.0, abs(ref["beta"]))


def test_metrics_of_a_reconstruction(C):
    """cfg1-sized reconstruction against its ground truth, threshold = noise floor."""
    wl = I.make_workload("cfg1", seed=3, iters=20)
    a = O.aperture(wl.pupil, wl.window)
    y = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=20)
    dev = torch.device("cuda")
    res = C.reconstruct(p, torch.from_numpy(y).to(dev), torch.from_numpy(wl.pupil).to(dev),
                        torch.from_numpy(wl.window).to(dev), C.Denoiser.gauss(0.8))
    r_hat = res.r.cpu().numpy()
    thr = float(np.float32(wl.noise_var / O.alpha_of(a)))
    md = 3 * 1.22 / 0.5
    got = C.point_cloud_metrics(res.r, torch.from_numpy(wl.r_true.astype(np.float32)).to(dev), thr, md)
    ref = O.point_cloud_metrics(r_hat, wl.r_true.astype(np.float32), thr, md)
    assert got["kept"] > 100
    _check(got, ref)


@pytest.mark.parametrize("shape,density,md", [((24, 40, 72), 0.05, 4.0), ((16, 64, 64), 0.02, 9.0),
                                              ((8, 8, 8), 0.0, 2.0)])
def test_metrics_random_sparse_volumes(C, shape, density, md):
    rng = np.random.default_rng(int(md * 10))
    r_true = np.where(rng.uniform(size=shape) < density, rng.uniform(0.2, 1.0, shape), 0.0).astype(np.float32)
    r_hat = np.where(rng.uniform(size=shape) < 0.1, rng.uniform(0.0, 1.0, shape), 0.0).astype(np.float32)
    dev = torch.device("cuda")
    got = C.point_cloud_metrics(torch.from_numpy(r_hat).to(dev), torch.from_numpy(r_true).to(dev), 0.05, md)
    ref = O.point_cloud_metrics(r_hat, r_true, 0.05, md)
    _check(got, ref)
