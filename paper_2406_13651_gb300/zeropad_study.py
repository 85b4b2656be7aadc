"""Resolution against the zero-padding factor q (Sec. II-B, Sec. IV): one synthetic scene,
one set of measurements, reconstructed on grids q = 1, 1.5 and 2 times finer than the
measurement grid.

The scene (one reflecting surface per (x, y) column, reflectance U[0.2, 1]) lives on the
finest grid, 256 x 256 x 128 (q = 2).  The looks are simulated there by the library
(clamp_simulate: speckle g = sqrt(r) z, y = a F g + eta) with the measured band the
central half of the spectrum in every dimension: pupil radius R / 2 of that grid's Nyquist
and the Hann window of the 64 measured range bins.  The data of the coarser grids are the
same spectral samples: the central 192 x 192 x 96 (q = 1.5) and 128 x 128 x 64 (q = 1)
frequencies, whose pupil (R / q) and window (band_window(nz, q)) select the same physical
band.  Each grid is reconstructed by CLAMP (Alg. 2, Gaussian prior, the same iterations
and sigma^2) and by the speckle average; every result is brought to the finest grid by
nearest-neighbour upsampling and compared with the scene: PSNR after the optimal scale
(Eq. psnr), and the depth of every (x, y) column (the range bin of its largest value, in
units of the finest grid's voxels; the scene has one surface per column) against the
true depth: mean and RMS error and the fraction of columns within one voxel.  (The
point-cloud threshold of Sec. IV-B, the noise floor sigma_w^2 / alpha, is not used here:
alpha is the band's share of the grid, so it falls as q grows and the threshold stops
being comparable across grids.)

  python -m paper_2406_13651_gb300.zeropad_study   (one GPU; prints one JSON line)
"""
from __future__ import annotations

import json
import time

import numpy as np

from . import clamp as C
from . import inputs as I

FINE = (256, 256, 128)   # nx, ny, nz of the q = 2 grid
QS = (1.0, 1.5, 2.0)


def _crop_index(n_fine: int, m: int):
    """Fine-grid bin of every bin of an m-point grid (same signed frequency)."""
    return (I.signed_freq(m).astype(np.int64) % n_fine)


def _upsample_index(n_fine: int, m: int):
    """Coarse voxel nearest to (containing) each fine voxel: floor(i m / n_fine)."""
    return (np.arange(n_fine) * m) // n_fine


def run(dev, seed: int = 1, looks: int = 16, iters: int = 200, radius: float = 0.4, snr_db: float = 1.5,
        prox_var: float = 1e-4) -> dict:
    import torch
    from .warmstart import device_draws, psnr
    nxf, nyf, nzf = FINE
    r_true = I.column_surface_scene(nxf, nyf, nzf, seed)
    pupil_f = I.circular_pupil(nxf, nyf, radius / 2.0)
    window_f = I.band_window(nzf, 2.0)
    nv = I.noise_variance_for_snr(r_true, pupil_f, window_f, snr_db)
    pf = C.make_params(nxf, nyf, nzf, looks, nv, prox_var)
    spk, eta = device_draws((looks, nzf, nyf, nxf), 4321 + seed, dev)
    y_f = C.simulate(pf, torch.from_numpy(r_true.astype(np.float32)).to(dev), spk, eta,
                     torch.from_numpy(pupil_f).to(dev), torch.from_numpy(window_f).to(dev))
    del spk, eta
    z_true = r_true.argmax(axis=0).astype(np.float64)   # one surface voxel per column
    rows = []
    for q in QS:
        nx, ny, nz = (int(round(v * q / 2.0)) for v in FINE)
        ix, iy, iz = (torch.from_numpy(_crop_index(nf, m)).to(dev) for nf, m in ((nxf, nx), (nyf, ny), (nzf, nz)))
        y = y_f.index_select(1, iz).index_select(2, iy).index_select(3, ix).contiguous()
        pupil = I.circular_pupil(nx, ny, radius / q)
        window = I.band_window(nz, q)
        pu, wi = torch.from_numpy(pupil).to(dev), torch.from_numpy(window).to(dev)
        p = C.make_params(nx, ny, nz, looks, nv, prox_var, max_iters=iters)
        den = C.Denoiser.gauss(0.8)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = C.reconstruct(p, y, pu, wi, den)
        torch.cuda.synchronize()
        seconds = time.perf_counter() - t0
        sa = C.speckle_average(p, y, pu, wi)
        ux, uy, uz = (torch.from_numpy(_upsample_index(nf, m)).to(dev) for nf, m in ((nxf, nx), (nyf, ny), (nzf, nz)))
        row = {"q": q, "grid": [nx, ny, nz], "iters": iters, "seconds": seconds,
               "ce_final": float(res.ce_hist[-1])}
        for name, img in (("clamp", res.r), ("speckle_average", sa)):
            up = img.index_select(0, uz).index_select(1, uy).index_select(2, ux).contiguous()
            rh = up.cpu().numpy().astype(np.float64)
            # depth per fine column: the coarse column's argmax, at its bin centre in fine voxels
            zc = img.argmax(dim=0).index_select(0, uy).index_select(1, ux).cpu().numpy().astype(np.float64)
            z_hat = (zc + 0.5) * (nzf / nz) - 0.5
            err = np.abs(z_hat - z_true)
            row[name] = {"psnr": psnr(rh, r_true), "depth_mean_abs_err": float(err.mean()),
                         "depth_rms_err": float(np.sqrt(np.mean(err ** 2))),
                         "depth_within_1_voxel": float(np.mean(err <= 1.0))}
        rows.append(row)
    return {"scene": f"column-surface scene on {nxf}x{nyf}x{nzf} (q = 2 grid), seed {seed}",
            "measurements": f"{looks} looks, central half of the spectrum in every dimension "
                            f"(pupil R = {radius} of the measurement grid), {snr_db} dB SNR",
            "prior": "Gaussian sigma 0.8 voxels of each grid", "rows": rows}


def main() -> int:
    import torch
    from . import build as B
    B.build()
    C.load()
    dev = torch.device("cuda", 0)
    print(json.dumps(run(dev)), flush=True)
    return 0


if __name__ == "__main__":
    raise SystemExit(main())
