"""Bounds-checking build of the hot path.  A child process loads ``libclamp_checked.so``
(every global index of the band passes, pass C and the CNN prior's tensor-core kernels
tested against its buffer's extent; an access outside is skipped and its site recorded)
and runs the forward agents in all three x-pass variants, the full-spectrum schedule, the
BF16 and FP32 CNN priors at edge, multi-tile and fused-tap shapes, and a reconstruction
with the BF16 prior.  No site may be recorded, and every output must equal the product
build's, computed here in this process on the same inputs."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2406_13651_gb300 import inputs as I  # noqa: E402

ROW_VARIANTS = (0, 1, 2)
AGENT_CASES = [((64, 32, 16), 3, "circle"), ((96, 32, 16), 2, "ragged"), ((16, 8, 8), 1, "one_column"),
               ((256, 16, 8), 2, "circle")]
CNN_CASES = [("bf16", (4, 8, 128), 8, 48), ("bf16", (4, 8, 128), 4, 16), ("bf16", (16, 64, 256), 3, 48),
             ("bf16", (2, 4, 128), 3, 64), ("bf16", (2, 8, 128), 4, 32), ("fp32", (2, 2, 256), 4, 16),
             ("fp32", (4, 8, 128), 5, 32), ("fp32", (2, 4, 128), 3, 48)]


def _pupil(kind, nx, ny, rng):
    if kind == "circle":
        return I.circular_pupil(nx, ny, 0.4)
    if kind == "one_column":
        p = np.zeros((ny, nx), np.float32)
        p[3 % ny, 5 % nx] = 1.0
        return p
    return ((rng.uniform(size=(ny, nx)) < 0.12) * rng.uniform(0.5, 1.0, (ny, nx))).astype(np.float32)


def _scene(shape, L, pupil_kind, seed):
    from oracle import clamp_oracle as O
    nx, ny, nz = shape
    wl = I.make_workload("cfg1", seed=seed, nx=nx, ny=ny, nz=nz, looks=L, iters=6)
    wl.pupil = _pupil(pupil_kind, nx, ny, np.random.default_rng(seed))
    wl.noise_var = I.noise_variance_for_snr(wl.r_true, wl.pupil, wl.window, 10.0)
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    return wl, y32


def run_cases(C):
    """Runs every case through the loaded library; returns ({name: output}, {name: site})."""
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).cuda()  # noqa: E731
    outs, sites = {}, {}
    C.bounds_check(reset=True)
    for shape, L, kind in AGENT_CASES:
        wl, y32 = _scene(shape, L, kind, seed=sum(shape) + L)
        for flag in ("full", "band"):
            for v in (ROW_VARIANTS if flag == "band" else (0,)):
                f = C.FLAG_FULL_SPECTRUM if flag == "full" else C.FLAG_BAND_SPECTRUM
                p = C.make_params(wl.nx, wl.ny, wl.nz, L, wl.noise_var, wl.prox_var, max_iters=4, flags=f)
                C.autotune_set_band(p, v)
                try:
                    res = C.reconstruct(p, dev(y32), dev(wl.pupil), dev(wl.window), C.Denoiser.gauss(0.8))
                finally:
                    C.autotune_set_band(p, 0)
                name = f"agent_{flag}{v}_{shape[0]}x{shape[1]}x{shape[2]}_L{L}_{kind}"
                outs[name] = res.r.cpu().numpy()
                sites[name] = C.bounds_check(reset=True)[1]
    for dtype, shape, layers, ch in CNN_CASES:
        ws, bs = I.cnn_weights(layers, ch, seed=layers * 7 + ch, last_scale=0.3)
        rng = np.random.default_rng(layers + ch)
        bs = [b + 0.02 * rng.standard_normal(b.shape).astype(np.float32) for b in bs]
        x = dev(rng.uniform(0, 1, shape).astype(np.float32))
        out = torch.empty_like(x)
        C.denoise(C.Denoiser.cnn(ws, bs, dtype), x, out)
        torch.cuda.synchronize()
        name = f"cnn_{dtype}_{shape[0]}x{shape[1]}x{shape[2]}_{layers}x{ch}"
        outs[name] = out.cpu().numpy()
        sites[name] = C.bounds_check(reset=True)[1]
    wl = I.make_workload("cfg1", seed=5, nx=128, ny=16, nz=8, looks=3, iters=6)
    ws, bs = I.cnn_weights(8, 48, seed=5)
    from oracle import clamp_oracle as O
    a = O.aperture(wl.pupil, wl.window)
    y32 = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var).astype(np.complex64)
    p = C.make_params(wl.nx, wl.ny, wl.nz, wl.looks, wl.noise_var, wl.prox_var, max_iters=6)
    res = C.reconstruct(p, dev(y32), dev(wl.pupil), dev(wl.window), C.Denoiser.cnn(ws, bs, "bf16"))
    outs["reconstruct_bf16_prior"] = res.r.cpu().numpy()
    sites["reconstruct_bf16_prior"] = C.bounds_check(reset=True)[1]
    return outs, sites


def _worker(out_path):
    from paper_2406_13651_gb300 import build, clamp
    assert os.environ.get("CLAMP_BOUNDS_CHECK") == "1"
    build.build(checked=True)
    clamp.load()
    checked, site = clamp.bounds_check(reset=True)
    outs, sites = run_cases(clamp)
    np.savez(out_path, **outs)
    with open(out_path + ".json", "w") as f:
        json.dump({"checked": checked, "initial_site": site, "sites": sites}, f)


@pytest.fixture(scope="module")
def C():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2406_13651_gb300 import build, clamp
    build.build()
    clamp.load()
    return clamp


def test_product_build_records_nothing(C):
    checked, site = C.bounds_check(reset=False)
    assert not checked and site == 0


def test_checked_build_in_bounds_and_identical(C, tmp_path):
    out = str(tmp_path / "checked.npz")
    env = dict(os.environ, CLAMP_BOUNDS_CHECK="1", PYTHONPATH=ROOT)
    r = subprocess.run([sys.executable, os.path.abspath(__file__), out], env=env, cwd=ROOT,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    with open(out + ".json") as f:
        meta = json.load(f)
    assert meta["checked"] is True
    assert meta["initial_site"] == 0
    bad = {k: v for k, v in meta["sites"].items() if v != 0}
    assert not bad, f"out-of-range accesses recorded (case: site code): {bad}"
    got = np.load(out)
    want, sites = run_cases(C)
    assert set(want) == set(got.files)
    assert all(v == 0 for v in sites.values())
    for k, w in want.items():
        g = got[k]
        assert np.isfinite(g).all(), k
        err = float(np.linalg.norm(g.astype(np.float64) - w) / max(np.linalg.norm(w.astype(np.float64)), 1e-300))
        assert err < 1e-6, (k, err)


if __name__ == "__main__":
    _worker(sys.argv[1])
