"""Pins for the FP64 oracle: each oracle function is checked against something other
than itself -- brute force, finite differences, the dense exact likelihood, closed
forms, library routines or invariants the paper states.  CPU only."""
import json
import math
import os

import numpy as np
import pytest

from oracle import clamp_oracle as O
from paper_2406_13651_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _crand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ------------------------------------------------------------------ DFT (Eq. A)

@pytest.mark.parametrize("shape", [(2, 3, 4), (4, 4, 2), (6, 6, 4), (3, 5, 2)])
def test_fft3_matches_direct_dft(shape):
    """Orthonormal 3D DFT equals the O(n^2) definition sum_j x_j e^{-2 pi i k.j / N} / sqrt(n)."""
    rng = _rng(1)
    x = _crand(rng, shape)
    nz, ny, nx = shape
    n = x.size
    kz, ky, kx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    X = np.zeros(shape, dtype=complex)
    for jz in range(nz):
        for jy in range(ny):
            for jx in range(nx):
                ph = -2j * math.pi * (kz * jz / nz + ky * jy / ny + kx * jx / nx)
                X += x[jz, jy, jx] * np.exp(ph)
    X /= math.sqrt(n)
    np.testing.assert_allclose(O.fft3(x), X, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(O.ifft3(X), x, rtol=1e-12, atol=1e-12)


def test_fft3_parseval_unitary_delta():
    rng = _rng(2)
    x = _crand(rng, (4, 8, 6))
    assert abs(np.linalg.norm(O.fft3(x)) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)
    np.testing.assert_allclose(O.ifft3(O.fft3(x)), x, atol=1e-13)
    d = np.zeros((4, 8, 6), dtype=complex)
    d[0, 0, 0] = 1.0
    np.testing.assert_allclose(O.fft3(d), np.full(d.shape, 1 / math.sqrt(d.size)), atol=1e-15)


# ------------------------------------------------------------------ aperture (Eq. A)

def _AHA(x, a):
    return O.AH_op(O.A_op(x, a), a)


def test_aperture_projection_properties():
    rng = _rng(3)
    nx, ny, nz = 8, 8, 4
    a = O.aperture(I.circular_pupil(nx, ny, 0.5), I.rect_window(nz))
    x, z = _crand(rng, (nz, ny, nx)), _crand(rng, (nz, ny, nx))
    # self-adjoint
    assert abs(np.vdot(_AHA(x, a), z) - np.vdot(x, _AHA(z, a))) < 1e-12 * np.linalg.norm(x) * np.linalg.norm(z)
    # binary aperture: idempotent projection, norm <= 1
    np.testing.assert_allclose(_AHA(_AHA(x, a), a), _AHA(x, a), atol=1e-12)
    assert np.linalg.norm(_AHA(x, a)) <= np.linalg.norm(x) * (1 + 1e-12)
    # alpha is the light fraction ||a||_1 / n for a binary aperture (Sec. III-B)
    assert O.alpha_of(a) == pytest.approx(np.abs(a).sum() / a.size, rel=1e-15)
    # a == 1 gives the identity
    ones = np.ones_like(a)
    np.testing.assert_allclose(_AHA(x, ones), x, atol=1e-12)


def test_hann_aperture_spectrum_in_unit_interval():
    nx, ny, nz = 4, 4, 4
    a = O.aperture(I.circular_pupil(nx, ny, 0.5), I.hann_window(nz))
    n = a.size
    M = np.stack([_AHA(e.reshape(a.shape), a).ravel() for e in np.eye(n)], axis=1)
    assert np.allclose(M, M.conj().T, atol=1e-12)
    ev = np.linalg.eigvalsh(M)
    assert ev.min() > -1e-12 and ev.max() < 1 + 1e-12


# ------------------------------------------------------------------ mu step (Eqs. mu-objective, h-gradient, mu-update)

def _tiny_problem(seed=4, shape=(4, 4, 4), window="hann"):
    rng = _rng(seed)
    nz, ny, nx = shape
    win = I.hann_window(nz) if window == "hann" else I.rect_window(nz)
    a = O.aperture(I.circular_pupil(nx, ny, 0.5), win)
    r_prev = rng.uniform(0.1, 1.0, shape)
    y = a * _crand(rng, shape)
    mu = _crand(rng, shape) * 0.3
    return a, r_prev, y, mu, 0.05


def test_gradient_matches_central_differences():
    """dh/dt along e at mu equals -Re <e, d> with d = -grad h (Eq. h-gradient)."""
    a, r_prev, y, mu, nv = _tiny_problem()
    alpha = O.alpha_of(a)
    d = O.grad_direction(mu, y, r_prev, a, nv, alpha)
    rng = _rng(5)
    for _ in range(6):
        e = _crand(rng, mu.shape)
        t = 1e-5
        fd = (O.h_objective(mu + t * e, y, r_prev, a, nv, alpha)
              - O.h_objective(mu - t * e, y, r_prev, a, nv, alpha)) / (2 * t)
        assert fd == pytest.approx(-np.real(np.vdot(e, d)), rel=1e-6)
    for e in (1.0, 1j):  # purely real and imaginary directions on one voxel
        E = np.zeros(mu.shape, dtype=complex)
        E[1, 2, 3] = e
        t = 1e-5
        fd = (O.h_objective(mu + t * E, y, r_prev, a, nv, alpha)
              - O.h_objective(mu - t * E, y, r_prev, a, nv, alpha)) / (2 * t)
        assert fd == pytest.approx(-np.real(np.vdot(E, d)), rel=1e-6, abs=1e-9)


def test_line_search_is_exact_minimiser():
    from scipy.optimize import minimize_scalar
    a, r_prev, y, mu, nv = _tiny_problem(6)
    alpha = O.alpha_of(a)
    d = O.grad_direction(mu, y, r_prev, a, nv, alpha)
    g = O.line_search_gamma(mu, d, y, r_prev, a, nv, alpha)
    res = minimize_scalar(lambda t: O.h_objective(mu + t * d, y, r_prev, a, nv, alpha),
                          bracket=(0.0, g * 0.5 + 1e-3), tol=1e-14)
    assert g > 0
    assert g == pytest.approx(res.x, rel=1e-6)
    # grid check: no step on a fine grid beats gamma*
    hs = O.h_objective(mu + g * d, y, r_prev, a, nv, alpha)
    for t in np.linspace(0, 3 * g, 61):
        assert hs <= O.h_objective(mu + t * d, y, r_prev, a, nv, alpha) + 1e-10 * abs(hs)


def test_mu_steps_decrease_h_and_reach_dense_solution():
    """With r' fixed, repeated gradient steps with exact line search decrease h monotonically
    and converge to the solution of (A^H A / sigma_w^2 + D) mu = A^H y / sigma_w^2."""
    a, r_prev, y, mu, nv = _tiny_problem(7, shape=(2, 4, 4))
    alpha = O.alpha_of(a)
    Am = O.dense_A(a)
    D = 1.0 / (r_prev.ravel() + nv / alpha)
    M = Am.conj().T @ Am / nv + np.diag(D)
    mu_star = np.linalg.solve(M, Am.conj().T @ y.ravel() / nv).reshape(mu.shape)
    hprev = O.h_objective(mu, y, r_prev, a, nv, alpha)
    for _ in range(3000):
        d = O.grad_direction(mu, y, r_prev, a, nv, alpha)
        mu = mu + O.line_search_gamma(mu, d, y, r_prev, a, nv, alpha) * d
        h = O.h_objective(mu, y, r_prev, a, nv, alpha)
        assert h <= hprev + 1e-12 * abs(hprev)
        hprev = h
    np.testing.assert_allclose(mu, mu_star, rtol=1e-7, atol=1e-9)


def test_no_aperture_mu_closed_form():
    """a = 1: the mu objective has the closed-form minimiser F^H y / (1 + sigma_w^2 D)
    (Sec. IV-A, no-aperture ablation), which repeated steps reach."""
    a, r_prev, y, mu, nv = _tiny_problem(8, shape=(2, 4, 4))
    a = np.ones_like(a)
    y = O.fft3(_crand(_rng(9), a.shape))
    alpha = O.alpha_of(a)
    D = 1.0 / (r_prev + nv / alpha)
    closed = O.ifft3(y) / (1.0 + nv * D)
    for _ in range(400):
        d = O.grad_direction(mu, y, r_prev, a, nv, alpha)
        mu = mu + O.line_search_gamma(mu, d, y, r_prev, a, nv, alpha) * d
    np.testing.assert_allclose(mu, closed, rtol=1e-9, atol=1e-11)


def test_c_is_exact_diagonal_when_A_is_orthogonal():
    """When A^H A = alpha I exactly (a == 1) the diagonal c equals diag(C~) of Eq. (Bi)."""
    a, r_prev, y, mu, nv = _tiny_problem(10, shape=(2, 2, 4))
    a = np.ones_like(a)
    _, C = O.exact_posterior(r_prev, y, a, nv)
    c = O.c_update(r_prev, nv, O.alpha_of(a))
    np.testing.assert_allclose(c.ravel(), np.real(np.diag(C)), rtol=1e-12)


# ------------------------------------------------------------------ EM surrogate (Eqs. em-surrogate-final, y-given-r)

@pytest.mark.parametrize("window", ["rect", "hann"])
def test_em_surrogate_majorises_exact_nll(window):
    """EM: f^(r; r') - f(r) >= f^(r'; r') - f(r') for every r > 0, with f the exact
    negative log likelihood of Eq. (y-given-r) and f^ built from the exact posterior."""
    rng = _rng(11)
    shape = (2, 2, 4)
    nz, ny, nx = shape
    win = I.hann_window(nz) if window == "hann" else I.rect_window(nz)
    a = O.aperture(I.circular_pupil(nx, ny, 0.6), win)
    nv = 0.05
    r_true = rng.uniform(0.2, 1.0, shape)
    g = np.sqrt(r_true) * _crand(rng, shape) / math.sqrt(2)
    y = O.A_op(g, a) + math.sqrt(nv) * _crand(rng, shape) / math.sqrt(2)
    r_prev = rng.uniform(0.2, 1.0, shape)
    mu, C = O.exact_posterior(r_prev, y, a, nv)
    c = np.real(np.diag(C)).reshape(shape)
    gap0 = O.em_surrogate(r_prev, mu, c) - O.exact_nll(r_prev, y, a, nv)
    for _ in range(40):
        r = rng.uniform(0.05, 2.0, shape)
        gap = O.em_surrogate(r, mu, c) - O.exact_nll(r, y, a, nv)
        assert gap >= gap0 - 1e-9
    # first-order contact at r': small perturbations change the gap only to second order
    e = rng.standard_normal(shape)
    t = 1e-4
    gp = O.em_surrogate(r_prev + t * e, mu, c) - O.exact_nll(r_prev + t * e, y, a, nv)
    gm = O.em_surrogate(r_prev - t * e, mu, c) - O.exact_nll(r_prev - t * e, y, a, nv)
    assert abs(gp - gm) / (2 * t) < 1e-5


# ------------------------------------------------------------------ prox (App. A) and the exact cubic prox

def test_cubic_prox_is_brute_force_minimiser():
    from scipy.optimize import minimize_scalar
    for v, K, s2 in [(0.5, 0.3, 0.1), (2.0, 0.01, 0.5), (0.05, 1.0, 0.01), (-0.3, 0.2, 0.2)]:
        r = O.cubic_prox(v, K, s2)
        obj = lambda t: np.log(t) + K / t + (t - v) ** 2 / (2 * s2)
        grid = np.exp(np.linspace(math.log(1e-6), math.log(10.0), 400001))
        t0 = grid[np.argmin(obj(grid))]          # global search (the objective can be non-convex)
        res = minimize_scalar(obj, bounds=(t0 * 0.999, t0 * 1.001), method="bounded",
                              options={"xatol": 1e-14})
        assert r == pytest.approx(res.x, rel=1e-6)


def _q(r, rp, K):
    """Per-voxel convex surrogate of App. A (Eq. convex-surrogate): r/r' + K/r."""
    return r / rp + K / r


def test_quadratic_prox_matches_bruteforce_surrogate_minimum():
    """The clipped closed form equals the brute-force minimiser, over the validity interval,
    of the quadratic whose derivative interpolates Q' (taken by finite differences of
    Eq. convex-surrogate) at r' and xi, plus the prox term."""
    rng = _rng(12)
    for _ in range(200):
        rp = rng.uniform(0.05, 2.0)
        K = rng.uniform(0.0, 2.0)
        v = rng.uniform(-0.5, 2.5)
        s2 = rng.choice([0.01, 0.1, 1.0])
        beta = rng.uniform(1.2, 4.0)
        got = float(O.prox_quadratic(v, rp, K, s2, beta))
        h = 1e-6
        dq = lambda r: (_q(r + h * r, rp, K) - _q(r - h * r, rp, K)) / (2 * h * r)
        drho = dq(rp) + (rp - v) / s2
        xi = rp / beta if drho > 0 else rp * beta
        s = (dq(xi) - dq(rp)) / (xi - rp)   # slope of the derivative chord
        grid = np.linspace(min(rp, xi), max(rp, xi), 20001)
        obj = 0.5 * s * (grid - rp) ** 2 + dq(rp) * (grid - rp) + (grid - v) ** 2 / (2 * s2)
        best = grid[np.argmin(obj)]
        assert got == pytest.approx(best, abs=(max(rp, xi) - min(rp, xi)) / 20000 * 1.5 + 1e-9)


def test_log_linearisation_majorises_surrogate():
    """Q(r; r') - Q(r'; r') >= f^(r) - f^(r') per voxel, equality at r = r' (App. A)."""
    rng = _rng(13)
    rp, K = rng.uniform(0.1, 2, 1000), rng.uniform(0, 2, 1000)
    r = rng.uniform(0.01, 5, 1000)
    fhat = lambda t: np.log(t) + K / t
    lhs = _q(r, rp, K) - _q(rp, rp, K)
    rhs = fhat(r) - fhat(rp)
    assert np.all(lhs >= rhs - 1e-12)


def test_iterated_quadratic_prox_reaches_cubic_root():
    """MM on one voxel: re-anchoring r' <- r with the beta_k schedule converges to the exact
    prox of the EM surrogate, the root of the cubic (Sec. III-B)."""
    for v, K, s2, r0 in [(0.5, 0.3, 0.1, 0.9), (1.5, 0.05, 0.5, 0.2), (0.2, 0.8, 0.05, 0.3)]:
        r = r0
        for k in range(1, 400):
            r = float(O.prox_quadratic(v, r, K, s2, O.beta_k(k)))
        assert r == pytest.approx(O.cubic_prox(v, K, s2), rel=1e-8)


def test_beta_schedule():
    assert O.beta_k(1) == pytest.approx(1 + 2 / math.log(2))
    b = [O.beta_k(k) for k in range(1, 300)]
    assert all(x > y > 1 for x, y in zip(b, b[1:]))


# ------------------------------------------------------------------ MACE (Eq. mann, Alg. 1, Thm. 1)

def test_mace_quadratic_agents_reach_weighted_mean():
    """Agents f_i = ||r - b_i||^2 / 2 (prox with sigma^2 = 1: (w + b_i)/2): the consensus
    equilibrium is sum_i upsilon_i b_i; with rho = 1/2, G w^{k+1} = G r^{k+1} every step."""
    rng = _rng(14)
    L = 3
    b = rng.standard_normal((L + 1, 5, 4, 3))
    ups = O.consensus_weights(L, 0.5)
    w = rng.standard_normal(b.shape)
    for _ in range(200):
        r = 0.5 * (w + b)
        w_new = O.mace_update(r, w, ups, 0.5)
        np.testing.assert_allclose(O.G_avg(w_new, ups), O.G_avg(r, ups), atol=1e-12)
        w = w_new
    r = 0.5 * (w + b)
    target = np.tensordot(ups, b, axes=(0, 0))
    np.testing.assert_allclose(O.G_avg(w, ups), target, atol=1e-9)
    assert O.convergence_error(r, w, ups) < 1e-9


def test_consensus_average_linear_idempotent():
    rng = _rng(15)
    ups = O.consensus_weights(4, 0.5)
    assert ups.sum() == pytest.approx(1.0)
    assert ups[0] == pytest.approx(1 / 8) and ups[4] == pytest.approx(0.5)
    x, z = rng.standard_normal((5, 3, 3, 3)), rng.standard_normal((5, 3, 3, 3))
    Gx = np.broadcast_to(O.G_avg(x, ups), x.shape)
    np.testing.assert_allclose(O.G_avg(Gx, ups), O.G_avg(x, ups), atol=1e-14)
    np.testing.assert_allclose(O.G_avg(2 * x + z, ups), 2 * O.G_avg(x, ups) + O.G_avg(z, ups), atol=1e-13)


# ------------------------------------------------------------------ priors

def test_gauss_denoiser_matches_scipy():
    from scipy.ndimage import gaussian_filter
    rng = _rng(16)
    x = rng.standard_normal((6, 7, 9))
    ref = gaussian_filter(x, sigma=0.8, mode="constant", cval=0.0, truncate=1.0 / 0.8)
    np.testing.assert_allclose(O.denoise_gauss(x, 0.8), ref, atol=1e-13)


def test_gauss_denoiser_is_symmetric_and_contractive():
    rng = _rng(17)
    x, z = rng.standard_normal((4, 5, 6)), rng.standard_normal((4, 5, 6))
    assert np.vdot(O.denoise_gauss(x, 0.8), z) == pytest.approx(np.vdot(x, O.denoise_gauss(z, 0.8)), rel=1e-12)
    g = O.gauss_kernel1d(0.8)
    assert g[1] - 2 * g[0] > 0  # 1D symbol positive: spectrum in (0, 1]


def test_conv3d_and_bf16_match_torch():
    torch = pytest.importorskip("torch")
    rng = _rng(18)
    x = rng.standard_normal((3, 5, 6, 7))
    w = rng.standard_normal((4, 3, 3, 3, 3))
    b = rng.standard_normal(4)
    ref = torch.nn.functional.conv3d(torch.from_numpy(x)[None], torch.from_numpy(w),
                                     torch.from_numpy(b), padding=1)[0].numpy()
    np.testing.assert_allclose(O.conv3d(x, w, b), ref, atol=1e-12)
    v = rng.standard_normal(10000).astype(np.float32) * 10
    tb = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(O.bf16_round(v), tb)


# ------------------------------------------------------------------ end to end

def test_speckle_average_textbook_case():
    """a == 1 and no noise: (1/L) sum |A^H y_l|^2 is the average of |g_l|^2 (Sec. I)."""
    rng = _rng(19)
    g = _crand(rng, (3, 4, 4, 4))
    a = np.ones((4, 4, 4))
    y = O.A_op(g, a)
    np.testing.assert_allclose(O.speckle_average(y, a), np.mean(np.abs(g) ** 2, axis=0), rtol=1e-12)


def test_reconstruct_converges_on_tiny_scene():
    wl = I.make_workload("tiny", seed=3)
    a = O.aperture(wl.pupil, wl.window)
    y = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var)
    r_out, st = O.reconstruct(y, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, 60)
    assert np.all(np.isfinite(r_out)) and r_out.min() > 0
    ce = st.ce_hist
    assert ce[-1] < 0.2 * ce[0]
    assert np.mean(ce[-10:]) < np.mean(ce[:10])
    # G w = G r after every step with rho = 1/2 (App. B)
    ups = O.consensus_weights(wl.looks)
    np.testing.assert_allclose(O.G_avg(st.w, ups), O.G_avg(st.r, ups), rtol=1e-10, atol=1e-14)


def test_psnr_optimal_scale():
    rng = _rng(20)
    r = rng.uniform(0, 1, (4, 4, 4))
    rh = 2.5 * r + 0.05 * rng.standard_normal(r.shape)
    p = O.psnr(rh, r)
    for bscale in np.linspace(0.3, 0.5, 41):
        assert p >= 10 * math.log10(r.size / np.sum((bscale * rh - r) ** 2)) - 1e-12


def test_paper_constants_fixture():
    """Constants the paper fixes (golden fixture with citations) match the oracle's defaults."""
    with open(os.path.join(GOLDEN, "paper_constants.json")) as f:
        g = json.load(f)
    L = 9
    ups = O.consensus_weights(L)
    assert ups[0] == pytest.approx(g["upsilon_look"]["value_times_2L"] / (2 * L))
    assert ups[L] == pytest.approx(g["upsilon_prior"]["value"])
    nx = 128
    pupil = I.circular_pupil(nx, nx, g["aperture_diameter_fraction"]["value"])
    # along the kx axis the disk spans 50 % of the grid
    assert pupil[0].sum() == pytest.approx(g["aperture_diameter_fraction"]["value"] * nx, abs=1)
    assert g["rho"]["value"] == 0.5


def test_no_aperture_mu_is_the_limit_of_gradient_steps():
    """The ablation's closed-form mu equals many exact-line-search steps of h with a = 1."""
    rng = _rng(21)
    shape = (2, 4, 4)
    y = O.fft3(_crand(rng, shape))
    r_prev = rng.uniform(0.1, 1.0, shape)
    nv = 0.05
    a = np.ones(shape)
    mu = np.zeros(shape, dtype=complex)
    for _ in range(400):
        d = O.grad_direction(mu, y, r_prev, a, nv, 1.0)
        mu = mu + O.line_search_gamma(mu, d, y, r_prev, a, nv, 1.0) * d
    np.testing.assert_allclose(O.no_aperture_mu(y, r_prev, nv), mu, rtol=1e-9, atol=1e-11)


def test_exact_prox_reconstruction_runs_and_converges():
    wl = I.make_workload("tiny", seed=4)
    a = O.aperture(wl.pupil, wl.window)
    y = O.simulate_data(wl.r_true, wl.speckle, wl.noise, a, wl.noise_var)
    r1, st1 = O.reconstruct(y, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, 25, exact_prox=True)
    r2, st2 = O.reconstruct(y, wl.pupil, wl.window, wl.denoiser, wl.noise_var, wl.prox_var, 25, no_aperture=True)
    assert np.all(np.isfinite(r1)) and np.all(np.isfinite(r2))
    assert st1.ce_hist[-1] < st1.ce_hist[0] and st2.ce_hist[-1] < st2.ce_hist[0]


# ---------------------------------------------------------------------- point-cloud metrics (Sec. IV-B)

def _brute_pc(r_hat, r_true, thr, max_dist):
    """All-pairs nearest neighbour with the smallest-index tie rule (independent of the k-d tree)."""
    nz, ny, nx = r_true.shape
    P = [(i, np.array([i % nx, (i // nx) % ny, i // (nx * ny)], float)) for i in np.flatnonzero(r_hat.ravel() > thr)]
    Q = [(i, np.array([i % nx, (i // nx) % ny, i // (nx * ny)], float)) for i in np.flatnonzero(r_true.ravel() > 0)]
    kept_d, rh, rq, removed = [], [], [], 0
    for ip, sp in P:
        best = min(Q, key=lambda t: (np.sum((t[1] - sp) ** 2), t[0]))
        d = float(np.sqrt(np.sum((best[1] - sp) ** 2)))
        if d <= max_dist:
            kept_d.append(d)
            rh.append(r_hat.ravel()[ip])
            rq.append(r_true.ravel()[best[0]])
        else:
            removed += 1
    rh, rq = np.array(rh), np.array(rq)
    b = rh @ rq / (rh @ rh)
    return dict(distance=float(np.mean(kept_d)), false_positive_rate=removed / len(P),
                nrmse=float(np.sqrt(np.sum((b * rh - rq) ** 2) / np.sum(rq ** 2))), kept=len(kept_d), removed=removed,
                beta=float(b))


def test_point_cloud_metrics_match_brute_force():
    rng = np.random.default_rng(11)
    r_true = np.where(rng.uniform(size=(6, 7, 8)) < 0.15, rng.uniform(0.2, 1.0, (6, 7, 8)), 0.0)
    r_hat = np.where(rng.uniform(size=(6, 7, 8)) < 0.3, rng.uniform(0.0, 1.0, (6, 7, 8)), 0.0)
    for thr, md in ((0.1, 2.5), (0.0, 1.0), (0.5, 10.0)):
        got = O.point_cloud_metrics(r_hat, r_true, thr, md)
        ref = _brute_pc(r_hat, r_true, thr, md)
        assert got["kept"] == ref["kept"] and got["removed"] == ref["removed"]
        for k in ("distance", "false_positive_rate", "nrmse", "beta"):
            assert abs(got[k] - ref[k]) < 1e-12, (k, got[k], ref[k])


def test_point_cloud_metrics_closed_forms():
    rng = np.random.default_rng(12)
    r = np.zeros((8, 8, 8))
    pts = [(1, 2, 3), (4, 4, 1), (6, 1, 6)]
    for (z, y, x) in pts:
        r[z, y, x] = rng.uniform(0.3, 1.0)
    m = O.point_cloud_metrics(r, r, 0.0, 3.0)            # identical clouds
    assert m["distance"] == 0 and m["false_positive_rate"] == 0 and m["nrmse"] < 1e-15 and abs(m["beta"] - 1) < 1e-15
    m = O.point_cloud_metrics(3.0 * r, r, 0.0, 3.0)      # scale is absorbed by beta*
    assert m["nrmse"] < 1e-15 and abs(m["beta"] - 1 / 3) < 1e-15
    shifted = np.roll(r, 1, axis=2)                       # every point one voxel off in x
    m = O.point_cloud_metrics(shifted, r, 0.0, 3.0)
    assert abs(m["distance"] - 1.0) < 1e-15 and m["nrmse"] < 1e-15
    far = r.copy()
    far[7, 7, 0] = 0.5                                    # an outlier 5+ voxels from every true point
    m = O.point_cloud_metrics(far, r, 0.0, 2.0)
    assert m["removed"] == 1 and abs(m["false_positive_rate"] - 0.25) < 1e-15


def test_mu_presteps_reach_the_exact_posterior_mean():
    """With r' held at r_init, the warm-start mu steps minimise h (floored D, reading R5),
    whose minimiser is the exact posterior mean at r' + sigma_w^2 / alpha."""
    rng = np.random.default_rng(21)
    shape = (2, 4, 4)
    a = (rng.uniform(size=shape) < 0.6).astype(float)
    y = (rng.normal(size=(1,) + shape) + 1j * rng.normal(size=(1,) + shape)) * a
    r_init = rng.uniform(0.2, 1.0, shape)
    nv = 0.05
    st = O.init_state(y, a, r_init)
    st = O.mu_presteps(st, y, a, nv, 400)
    mu_ref, _ = O.exact_posterior(st.r[0] + nv / O.alpha_of(a), y[0], a, nv)
    np.testing.assert_allclose(st.mu[0], mu_ref, rtol=1e-8, atol=1e-10)
