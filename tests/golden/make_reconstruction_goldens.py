"""Writes the end-to-end reconstruction goldens the GPU parity tests compare with.

Calls only the FP64 oracle (``oracle.clamp_oracle``) and the seeded input generators
(``paper_2406_13651_gb300.inputs``): nothing here runs CUDA code.  For each workload the
looks' data are simulated by the oracle from the seeded draws (Eqs. forward-model,
g-given-r) and rounded to complex64, the form the GPU receives; the oracle then runs
CLAMP (Alg. 2, initialised as in Sec. IV-A) on those data and the output r* = wbar is
stored as float32 (its rounding, ~6e-8 relative, is far below the test tolerances).

  cfg2: 128x128x64, L = 16, residual CNN 5 x 32 FP32 prior, 50 iterations; whole volume.
  cfg3: 256x256x128, L = 32, facets, residual CNN 8 x 48 BF16 prior, 3 iterations; the
        eight range planes SLAB3 of the volume (the iteration couples every voxel through
        the FFTs, so the oracle computes all of it).

Usage: python tests/golden/make_reconstruction_goldens.py cfg2|cfg3   (about 40 / 60 min on
8 cores; cfg3 holds about 40 GB).
"""
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import clamp_oracle as O  # noqa: E402
from paper_2406_13651_gb300 import inputs as I  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))
ITERS = {"cfg2": 50, "cfg3": 3}
SLAB3 = (60, 68)


def looks_data(wl, seed: int = 1) -> np.ndarray:
    """complex64 [L][nz][ny][nx]: each look simulated by the oracle, then rounded."""
    a = O.aperture(wl.pupil, wl.window)
    y = np.empty((wl.looks, wl.nz, wl.ny, wl.nx), np.complex64)
    for l in range(wl.looks):
        spk, eta = I.look_draws(wl, seed, l)
        y[l] = O.simulate_data(wl.r_true, spk[None], eta[None], a, wl.noise_var)[0]
    return y


def main(name: str):
    wl = I.make_workload(name, seed=1, with_draws=False)
    t0 = time.time()
    y = looks_data(wl).astype(np.complex128)
    iters = ITERS[name]
    r_out, st = O.reconstruct(y, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, iters)
    out = dict(iters=iters, ce_hist=np.array(st.ce_hist), mu_res_hist=np.array(st.mu_res_hist),
               norm2=float(np.sum(r_out ** 2)))
    if name == "cfg3":
        out["slab"] = np.array(SLAB3)
        out["wbar"] = r_out[SLAB3[0]:SLAB3[1]].astype(np.float32)
    else:
        out["wbar"] = r_out.astype(np.float32)
    path = os.path.join(HERE, f"reconstruction_{name}.npz")
    np.savez_compressed(path, **out)
    print(f"{name}: {iters} iterations in {time.time() - t0:.0f} s -> {path}; CE {st.ce_hist[-1]:.3e}")


if __name__ == "__main__":
    main(sys.argv[1])
