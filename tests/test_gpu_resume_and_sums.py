"""Resuming a run from its state, and the accuracy of the per-voxel look sums.

* clamp_iterate continues a run from {mu, r, w, k}: iterations 1..4 followed by 5..10 give
  what iterations 1..10 in one call give, and both equal clamp_reconstruct's output.
* The MACE pass forms wbar = sum_j upsilon_j w_j and G(x) over L + 1 = 33 rows per voxel in
  FP32 with error-free (two-sum) compensation.  With rows spanning 1e-6 .. 1 the result
  must stay within 1.5 units in the last place of the exact sum of the FP32 rows; plain
  FP32 summation in row order is off by up to 2.8 units on the same rows.
"""
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
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_resumed_iterations_equal_one_run(C):
    wl = I.make_workload("cfg1", seed=2, nx=64, ny=64, nz=32, looks=4)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    dev = torch.device("cuda")
    y = torch.from_numpy(y32).to(dev)
    pu, wi = torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev)
    den = C.Denoiser.gauss(0.8)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=10)
    ws = C.iterate_workspace(p, den)
    shape = (wl.nz, wl.ny, wl.nx)
    mu, r, w = C.init(p, y, pu, wi)
    mu2, r2, w2 = mu.clone(), r.clone(), w.clone()
    wbar = torch.empty(shape, device=dev)
    wbar2 = torch.empty(shape, device=dev)
    ce = torch.zeros(10, dtype=torch.float64, device=dev)
    ce2 = torch.zeros(10, dtype=torch.float64, device=dev)
    C.iterate(p, 1, 10, y, pu, wi, den, mu, r, w, wbar, ce_out=ce, ws=ws)
    C.iterate(p, 1, 4, y, pu, wi, den, mu2, r2, w2, wbar2, ce_out=ce2[:4], ws=ws)
    C.iterate(p, 5, 6, y, pu, wi, den, mu2, r2, w2, wbar2, ce_out=ce2[4:], ws=ws)
    torch.cuda.synchronize()
    assert rel(wbar2.cpu(), wbar.cpu()) < 1e-6
    assert rel(torch.view_as_real(mu2).cpu(), torch.view_as_real(mu).cpu()) < 1e-6
    np.testing.assert_allclose(ce2.cpu().numpy(), ce.cpu().numpy(), rtol=1e-5)
    res = C.reconstruct(p, y, pu, wi, den)
    assert rel(res.r.cpu(), wbar.cpu()) < 1e-6


def test_look_sums_are_compensated(C):
    L = 32
    nz, ny, nx = 16, 64, 64
    rng = np.random.default_rng(8)
    # rows alternate between O(1) values and values of 1e-6 .. 1e-5
    big = rng.uniform(0.5, 1.0, (L + 1, nz, ny, nx))
    small = rng.uniform(1e-6, 1e-5, (L + 1, nz, ny, nx))
    w_in = np.where((np.arange(L + 1) % 2 == 0)[:, None, None, None], big, small).astype(np.float32)
    r_in = np.where((np.arange(L + 1) % 3 == 0)[:, None, None, None], small, big).astype(np.float32)
    dev = torch.device("cuda")
    r = torch.from_numpy(r_in).to(dev)
    w = torch.from_numpy(w_in).to(dev)
    wbar = torch.empty((nz, ny, nx), device=dev)
    ce = torch.zeros(1, dtype=torch.float64, device=dev)
    p = C.make_params(nx, ny, nz, L, 1e-3, 1e-4)
    C.mace_step(p, r, w, wbar, ce)
    torch.cuda.synchronize()
    ups = O.consensus_weights(L).astype(np.float32).astype(np.float64)   # the weights as the kernel holds them
    w_new = w.cpu().numpy()
    exact = np.tensordot(ups, w_new.astype(np.float64), axes=(0, 0))        # exact sum of the FP32 rows
    got = wbar.cpu().numpy().astype(np.float64)
    ulp = np.spacing(np.abs(exact).astype(np.float32)).astype(np.float64)
    assert np.max(np.abs(got - exact) / ulp) <= 1.5
    # plain FP32 summation in row order misses that bound on the same rows
    naive = np.zeros((nz, ny, nx), np.float32)
    for j in range(L + 1):
        naive = naive + np.float32(ups[j]) * w_new[j]
    assert np.max(np.abs(naive.astype(np.float64) - exact) / ulp) > 1.5
    # the MACE update itself against the oracle on the same FP32 inputs
    w_ref = O.mace_update(r_in.astype(np.float64), w_in.astype(np.float64), O.consensus_weights(L), 0.5)
    assert rel(w_new, w_ref) < 1e-6
    assert float(ce.item()) == pytest.approx(O.convergence_error(r_in.astype(np.float64), w_in.astype(np.float64),
                                                                 O.consensus_weights(L)), rel=1e-6)
