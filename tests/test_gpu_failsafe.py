"""Failure handling on the GPU without faulting it: the bounded mbarrier wait gives up
and reports when nothing arrives, and non-finite data is reported as CLAMP_ENONFINITE
rather than returned as a reconstruction."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2406_13651_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    clamp.load()
    return clamp


def test_bounded_wait_gives_up_when_nothing_arrives(C):
    assert C.selftest_bounded_wait(1000) == (1, 0)
    assert C.selftest_bounded_wait(1)[1] == 0     # one poll: still gives up, does not hang
    x = torch.ones(4, device="cuda")             # the context is still usable
    assert float((x * 2).sum().item()) == 8.0


def test_nan_data_is_reported(C):
    wl = I.make_workload("tiny", seed=3, with_draws=False)
    dev = torch.device("cuda")
    y = torch.ones((wl.looks, wl.nz, wl.ny, wl.nx), dtype=torch.complex64, device=dev)
    y[0, 1, 2, 3] = complex(float("nan"), 0.0)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=3)
    with pytest.raises(C.ClampError) as e:
        C.reconstruct(p, y, torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev),
                      C.Denoiser.gauss(0.8))
    assert e.value.status == 6                    # CLAMP_ENONFINITE
    # a clean call afterwards still works
    y[0, 1, 2, 3] = 1.0
    res = C.reconstruct(p, y, torch.from_numpy(wl.pupil).to(dev), torch.from_numpy(wl.window).to(dev),
                        C.Denoiser.gauss(0.8))
    assert np.isfinite(res.r.cpu().numpy()).all()
