"""Seeded input generators: determinism, distributions and aperture geometry."""
import math

import numpy as np
import pytest

from paper_2406_13651_gb300 import inputs as I


def test_generator_is_deterministic_and_stream_separated():
    a = I.uniform(7, 1, 1000)
    np.testing.assert_array_equal(a, I.uniform(7, 1, 1000))
    assert not np.array_equal(a, I.uniform(7, 2, 1000))
    assert not np.array_equal(a, I.uniform(8, 1, 1000))
    assert a.min() >= 0.0 and a.max() < 1.0


def test_splitmix64_reference_values():
    """SplitMix64 finaliser on known inputs (the published mixing constants)."""
    z = I._mix64(np.array([0, 1], dtype=np.uint64))
    # mixing 0 gives 0; mixing 1 is a fixed 64-bit value
    assert int(z[0]) == 0
    x = 1
    x ^= x >> 30; x = (x * 0xBF58476D1CE4E5B9) % 2**64
    x ^= x >> 27; x = (x * 0x94D049BB133111EB) % 2**64
    x ^= x >> 31
    assert int(z[1]) == x


def test_complex_normal_moments():
    z = I.complex_normal(3, 5, (200000,))
    assert abs(np.mean(np.abs(z) ** 2) - 1.0) < 0.01
    assert abs(np.mean(z)) < 0.01
    assert abs(np.mean(z * z)) < 0.01          # circular: E[z^2] = 0
    assert abs(np.var(z.real) - 0.5) < 0.01


def test_pupil_and_window_geometry():
    p = I.circular_pupil(128, 128, 0.5)
    assert p[0, 0] == 1.0                      # DC inside
    assert p[0, 32] == 1.0 and p[0, 33] == 0.0  # radius 0.5 Nyquist = 32 bins
    assert p[0, -32] == 1.0 and p[0, -33] == 0.0
    np.testing.assert_array_equal(p, p[:, ::-1][:, np.r_[-1, 0:127]])  # symmetric fx <-> -fx
    h = I.hann_window(16)
    assert h[0] == pytest.approx(1.0) and h[8] == pytest.approx(0.0, abs=1e-7)
    assert h[4] == pytest.approx(0.5)


def test_scenes_one_surface_per_column():
    r = I.column_surface_scene(32, 24, 16, seed=2)
    assert r.shape == (16, 24, 32)
    nnz = np.count_nonzero(r, axis=0)
    assert np.all(nnz == 1)
    vals = r[r > 0]
    assert vals.min() >= 0.2 and vals.max() <= 1.0
    f = I.facet_scene(64, 64, 32, seed=4)
    assert np.all(np.count_nonzero(f, axis=0) == 1)


def test_noise_variance_for_snr():
    r = I.column_surface_scene(16, 16, 8, seed=1)
    p, h = I.circular_pupil(16, 16, 0.5), I.hann_window(8)
    v10 = I.noise_variance_for_snr(r, p, h, 10.0)
    v20 = I.noise_variance_for_snr(r, p, h, 20.0)
    assert v10 / v20 == pytest.approx(10.0)


def test_workload_presets():
    wl = I.make_workload("cfg1", seed=1)
    assert (wl.nz, wl.ny, wl.nx, wl.looks) == (16, 32, 32, 4)
    assert wl.speckle.shape == (4, 16, 32, 32)
    w2 = I.make_workload("cfg2", seed=1, with_draws=False)
    assert w2.denoiser["kind"] == "cnn" and len(w2.denoiser["weights"]) == 5
    assert w2.denoiser["weights"][1].shape == (32, 32, 3, 3, 3)


def test_chunked_draws_equal_full_draw():
    full = I.complex_normal(5, 20, (3, 4, 8, 16))
    n = 4 * 8 * 16
    parts = [I.complex_normal(5, 20, (4, 8, 16), l * n) for l in range(3)]
    np.testing.assert_array_equal(np.stack(parts), full)
    wl = I.make_workload("tiny", seed=2)
    spk, eta = I.look_draws(wl, 2, 1)
    np.testing.assert_array_equal(spk, wl.speckle[1])
    np.testing.assert_array_equal(eta, wl.noise[1])


def test_band_window_for_zero_padding():
    """q = 1 is the plain Hann window; q > 1 keeps the measured band of nz / q bins (the
    Hann window of that length, DC = 1) and is zero outside it."""
    np.testing.assert_array_equal(I.band_window(32, 1.0), I.hann_window(32))
    for nz, q in ((96, 1.5), (64, 2.0)):
        h = I.band_window(nz, q)
        m = int(round(nz / q))
        f = I.signed_freq(nz)
        assert h[0] == 1.0
        assert np.all(h[np.abs(f) > m / 2] == 0.0)
        inside = np.abs(f) < m / 2
        np.testing.assert_allclose(h[inside], 0.5 * (1 + np.cos(2 * np.pi * f[inside] / m)), rtol=1e-6)
        # the embedded band equals the un-padded Hann window of length m, bin for bin
        hm = I.hann_window(m)
        fm = I.signed_freq(m)
        for k in range(m):
            if abs(fm[k]) < m / 2:
                j = int(fm[k]) % nz
                assert abs(h[j] - hm[k]) < 1e-6


def test_zero_padded_workload_shrinks_the_band():
    w1 = I.make_workload("cfg1", seed=3, nx=64, ny=64, nz=32, looks=2, with_draws=False)
    w2 = I.make_workload("cfg1", seed=3, nx=96, ny=96, nz=48, looks=2, with_draws=False, q=1.5)
    frac = lambda w: float(np.count_nonzero(w.pupil)) / w.pupil.size   # noqa: E731
    assert abs(frac(w2) / frac(w1) - 1 / 1.5 ** 2) < 0.05
    assert np.count_nonzero(w2.window) < np.count_nonzero(w1.window) * 48 / 32
