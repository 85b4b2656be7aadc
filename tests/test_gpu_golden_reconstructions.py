"""Whole CLAMP reconstructions (Alg. 2 end to end) against the FP64 oracle at the full
configurations, in the launch configuration the benchmark times:

* 128x128x64, L = 16, residual CNN 5 x 32 FP32 prior, 50 iterations, whole volume:
  relative L2 <= 1e-4 (the FP32 path's target);
* 256x256x128, L = 32, facets, residual CNN 8 x 48 BF16 prior, 3 iterations, eight range
  planes of the volume: relative L2 <= 1e-2 (the BF16 prior's target).

The oracle's results are stored goldens (tests/golden/reconstruction_*.npz, written by
tests/golden/make_reconstruction_goldens.py from the oracle alone).  The data are
rebuilt here the way that script builds them: the oracle simulates each look from the
seeded draws and rounds it to complex64.  Besides the relative L2 error each test bounds
the largest per-voxel error against the largest value, so that a local error cannot
hide under the norm."""
import os
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.join(HERE, "golden"))

from paper_2406_13651_gb300 import inputs as I  # noqa: E402
import make_reconstruction_goldens as G  # noqa: E402


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    clamp.load()
    return clamp


# (workload, rel-L2 target, bound on max |error| / max |reference|, CE history rtol)
CASES = [("cfg2", 1e-4, 1e-3, 1e-3), ("cfg3", 1e-2, 5e-2, 1e-2)]


@pytest.mark.parametrize("name,tol,tol_max,tol_ce", CASES)
def test_reconstruction_matches_oracle_golden(C, name, tol, tol_max, tol_ce):
    g = np.load(os.path.join(HERE, "golden", f"reconstruction_{name}.npz"))
    iters = int(g["iters"])
    wl = I.make_workload(name, seed=1, with_draws=False)
    dev = torch.device("cuda")
    y = torch.from_numpy(G.looks_data(wl)).to(dev)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=iters)
    res = C.reconstruct(p, y, torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev),
                        C.Denoiser.from_desc(wl.denoiser))
    got = res.r.cpu().numpy().astype(np.float64)
    if "slab" in g.files:
        z0, z1 = (int(v) for v in g["slab"])
        got = got[z0:z1]
    ref = g["wbar"].astype(np.float64)
    rel = float(np.linalg.norm(got - ref) / np.linalg.norm(ref))
    mx = float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))
    print(f"{name}: {iters} iterations, rel-L2 {rel:.3e}, max|err|/max|ref| {mx:.3e}, "
          f"CE gpu {res.ce_hist[iters - 1]:.4e} oracle {g['ce_hist'][-1]:.4e}")
    assert rel <= tol
    assert mx <= tol_max
    np.testing.assert_allclose(res.ce_hist[:iters], g["ce_hist"], rtol=tol_ce)
