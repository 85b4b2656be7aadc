"""Batched reconstruction: scenes of uneven size and look count in one CUDA graph launch
give the same result as one clamp_reconstruct call per scene, and match the oracle."""
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


SPECS = [dict(nx=32, ny=32, nz=16, looks=4, radius=0.5, snr=10.0, seed=11, iters=5),
         dict(nx=64, ny=64, nz=32, looks=3, radius=0.4, snr=15.0, seed=12, iters=7),
         dict(nx=96, ny=96, nz=32, looks=2, radius=0.35, snr=8.0, seed=13, iters=4)]


def test_batch_matches_single_scene_calls_and_oracle(C):
    den = C.Denoiser.gauss(0.8)
    dev = torch.device("cuda")
    scenes, wls, ys = [], [], []
    for sp in SPECS:
        wl = I.batch_scene(sp)
        a = O.aperture(wl.pupil, wl.window)
        y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
        p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=wl.iters)
        yd = torch.from_numpy(y32).to(dev)
        scenes.append((p, yd, torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev),
                       torch.empty((wl.nz, wl.ny, wl.nx), dtype=torch.float32, device=dev)))
        wls.append(wl)
        ys.append(y32)
    batch = C.Batch(scenes, den)
    for rep in range(2):   # the captured graph can be launched repeatedly
        batch.launch()
        lat = batch.latencies()
        ce = batch.residuals()
        assert np.all(np.isfinite(lat)) and np.all(lat > 0)
        for i, (p, yd, pu, wi, ro) in enumerate(scenes):
            single = C.reconstruct(p, yd, pu, wi, den)
            assert rel(ro.cpu().numpy(), single.r.cpu().numpy()) < 1e-6, i
            assert ce[i] == pytest.approx(single.ce_hist[-1], rel=1e-6)
    wl = wls[1]
    ref, _ = O.reconstruct(ys[1].astype(np.complex128), wl.pupil, wl.window, wl.denoiser, wl.noise_var,
                           wl.prox_var, wl.iters)
    assert rel(scenes[1][4].cpu().numpy(), ref) < 1e-4
    batch.close()


def test_batch_rejects_bad_scene(C):
    den = C.Denoiser.gauss(0.8)
    dev = torch.device("cuda")
    p = C.make_params(48, 32, 16, 2, 1e-3, 1e-4, max_iters=2)   # nx = 48 is not a supported length
    y = torch.zeros((2, 16, 32, 48), dtype=torch.complex64, device=dev)
    with pytest.raises(C.ClampError):
        C.Batch([(p, y, torch.ones(32 * 48, device=dev), torch.ones(16, device=dev),
                  torch.empty(16 * 32 * 48, device=dev))], den)


def test_batch_graph_with_concurrent_prior(C):
    """Scenes whose prior agent runs on the side stream: with the side stream created
    before capture (a reconstruction ran on this thread first) the fork and join become
    edges of the captured graph, and the results equal single calls on the serial
    schedule."""
    den = C.Denoiser.gauss(0.8)
    dev = torch.device("cuda")
    scenes, serial = [], []
    for sp in SPECS[:2]:
        wl = I.batch_scene(sp)
        a = O.aperture(wl.pupil, wl.window)
        y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
        mk = lambda flag: C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var,
                                        max_iters=wl.iters, flags=flag)
        pc, ps = mk(C.FLAG_PRIOR_CONCURRENT), mk(C.FLAG_PRIOR_SERIAL)
        assert C.prior_concurrent(pc) and not C.prior_concurrent(ps)
        yd, pu, wi = (torch.from_numpy(v).to(dev) for v in (y32, wl.pupil, wl.window))
        C.reconstruct(pc, yd, pu, wi, den)   # creates this thread's side stream outside capture
        scenes.append((pc, yd, pu, wi, torch.empty((wl.nz, wl.ny, wl.nx), dtype=torch.float32, device=dev)))
        serial.append(C.reconstruct(ps, yd, pu, wi, den))
    batch = C.Batch(scenes, den)
    batch.launch()
    ce = batch.residuals()
    for i, (p, yd, pu, wi, ro) in enumerate(scenes):
        assert rel(ro.cpu().numpy(), serial[i].r.cpu().numpy()) < 1e-6, i
        assert ce[i] == pytest.approx(serial[i].ce_hist[-1], rel=1e-6)
    batch.close()
