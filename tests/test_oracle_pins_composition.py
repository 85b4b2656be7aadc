"""Pins for the oracle functions that compose pinned pieces: the convergence error, the
mu-residual, the residual CNN prior, the forward agent's order of steps, the U-Net prior's
normalisation and the l2,1 prior agent.  Each test names the plausible slip it catches
(a dropped factor, a wrong operand, a step taken in the wrong order).  CPU only."""
import math

import numpy as np
import pytest

from oracle import clamp_oracle as O
from paper_2406_13651_gb300 import inputs as I


def _rng(seed):
    return np.random.default_rng(seed)


def _crand(rng, shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ------------------------------------------------------------------ convergence error (Eq. mace-convergence-error)

def test_convergence_error_closed_form():
    """With agent outputs r_j = (1 + eps_j) wbar, wbar = G(w), the error is
    sqrt(sum_j eps_j^2 / (L + 1)) exactly (reading R10: unweighted stacked norm over the
    L + 1 agents, normalised by sqrt(L + 1) ||wbar||).  Catches: a dropped (L + 1), the
    average of r instead of G(w), and upsilon-weighted sums."""
    rng = _rng(40)
    L = 3
    # the paper's weights (Sec. III-A): 1/(2L) per look, 1/2 for the prior
    ups = np.array([1.0 / (2 * L)] * L + [0.5])
    w = rng.uniform(0.1, 1.0, (L + 1, 4, 5, 6))
    wbar = sum(ups[j] * w[j] for j in range(L + 1))
    eps = np.array([0.1, -0.2, 0.3, 0.05])
    r = np.stack([(1.0 + eps[j]) * wbar for j in range(L + 1)])
    got = O.convergence_error(r, w, O.consensus_weights(L, 0.5))
    assert got == pytest.approx(math.sqrt(np.sum(eps ** 2) / (L + 1)), rel=1e-12)
    # the slips give different numbers on this input
    assert abs(got - math.sqrt(np.sum(eps ** 2))) > 0.1
    assert abs(got - math.sqrt(np.sum(ups * eps ** 2))) > 0.01


# ------------------------------------------------------------------ mu-residual (Eqs. residual, Bi)

def test_mu_residual_against_dense_posterior():
    """Unfloored form: (1/L) sum_l ||C~_l^{-1} mu_l - A^H y_l / sigma_w^2|| / ||A^H y_l / sigma_w^2||
    with C~^{-1} the inverse of the dense posterior covariance of Eq. (Bi).  It is zero at
    the exact posterior mean (the numerator comes from the exact solution of Eq. (mu2)).
    Floored form: zero at the posterior mean with r' + sigma_w^2/alpha, and equal to
    ||d|| sigma_w^2 / ||A^H y||.  Catches: sum instead of mean over looks, a missing
    1/sigma_w^2, D(1/r') swapped between the two forms."""
    rng = _rng(41)
    shape = (2, 2, 4)
    nz, ny, nx = shape
    a = O.aperture(I.circular_pupil(nx, ny, 0.6), I.hann_window(nz))
    nv = 0.07
    L = 2
    alpha = O.alpha_of(a)
    r_prev = rng.uniform(0.2, 1.0, (L,) + shape)
    y = np.stack([a * _crand(rng, shape) for _ in range(L)])
    Am = O.dense_A(a)
    mu = np.empty((L,) + shape, dtype=complex)
    mu[0] = O.exact_posterior(r_prev[0], y[0], a, nv)[0]
    mu[1] = _crand(rng, shape) * 0.4
    _, C1 = O.exact_posterior(r_prev[1], y[1], a, nv)
    ahy1 = Am.conj().T @ y[1].ravel() / nv
    val1 = np.linalg.norm(np.linalg.inv(C1) @ mu[1].ravel() - ahy1) / np.linalg.norm(ahy1)
    got = O.mu_residual(mu, y, r_prev, a, nv, alpha)
    assert got == pytest.approx(0.5 * val1, rel=1e-9)
    assert O.mu_residual(mu[:1], y[:1], r_prev[:1], a, nv, alpha) < 1e-10
    # floored form
    mf = O.exact_posterior(r_prev[0] + nv / alpha, y[0], a, nv)[0]
    assert O.mu_residual(mf[None], y[:1], r_prev[:1], a, nv, alpha, floored=True) < 1e-10
    d = O.grad_direction(mu[1], y[1], r_prev[1], a, nv, alpha)
    want = np.linalg.norm(d) * nv / np.linalg.norm(Am.conj().T @ y[1].ravel())
    got_f = O.mu_residual(mu[1:], y[1:], r_prev[1:], a, nv, alpha, floored=True)
    assert got_f == pytest.approx(want, rel=1e-10)


# ------------------------------------------------------------------ residual CNN prior

@pytest.mark.parametrize("bf16", [False, True])
def test_denoise_cnn_matches_torch_stack(bf16):
    """H(x) = x + CNN(x) against torch's Conv3d / ReLU modules: ReLU after every hidden
    layer, none after the last; the last layer's bias is negative, so part of the CNN
    output is below zero and a ReLU there would change it.  BF16: weights and every
    layer's input rounded by torch's own bfloat16 cast (not the oracle's bit trick)."""
    torch = pytest.importorskip("torch")
    rng = _rng(42)
    C = 6
    nl = 4
    ws, bs = [], []
    for i in range(nl):
        cin = 1 if i == 0 else C
        cout = 1 if i == nl - 1 else C
        ws.append((rng.standard_normal((cout, cin, 3, 3, 3)) * math.sqrt(2.0 / (27 * cin))).astype(np.float32))
        bs.append((rng.standard_normal(cout) * 0.1 - (0.3 if i == nl - 1 else 0.0)).astype(np.float32))
    x = rng.uniform(0.0, 1.0, (5, 6, 7))
    got = O.denoise_cnn(x, ws, bs, bf16=bf16)
    layers = []
    for i in range(nl):
        conv = torch.nn.Conv3d(ws[i].shape[1], ws[i].shape[0], 3, padding=1).double()
        w_t = torch.from_numpy(ws[i]).double()
        if bf16:
            w_t = w_t.to(torch.bfloat16).double()
        with torch.no_grad():
            conv.weight.copy_(w_t)
            conv.bias.copy_(torch.from_numpy(bs[i]).double())
        layers.append(conv)
    h = torch.from_numpy(x)[None, None]
    with torch.no_grad():
        for i, conv in enumerate(layers):
            h = conv(h.to(torch.bfloat16).double() if bf16 else h)
            if i < nl - 1:
                h = torch.nn.ReLU()(h)
    cnn = h[0, 0].numpy()
    assert (cnn < 0).mean() > 0.2          # the last layer's output really is signed
    np.testing.assert_allclose(got, x + cnn, rtol=1e-12, atol=1e-12)


# ------------------------------------------------------------------ forward agent (Alg. 2 steps 5-9)

def test_forward_agent_step_order():
    """Alg. 2 steps 5-9 in order: the mu step minimises h along d (checked by a scalar
    search, not the closed-form gamma), and the prox uses K = c + |mu_new|^2 of the
    POST-step mu with c from the old r' (checked per voxel by brute force over the
    validity interval).  Using the pre-step mu in K moves r on this input."""
    from scipy.optimize import minimize_scalar
    rng = _rng(43)
    shape = (2, 4, 4)
    nz, ny, nx = shape
    a = O.aperture(I.circular_pupil(nx, ny, 0.5), I.hann_window(nz))
    nv = 0.05
    alpha = O.alpha_of(a)
    r_prev = rng.uniform(0.1, 1.0, shape)
    y = a * _crand(rng, shape) * 2.0
    mu = _crand(rng, shape) * 0.3
    w = rng.uniform(0.05, 1.5, shape)
    s2, beta = 0.1, O.beta_k(3)
    mu_new, r_new, gamma, d = O.forward_agent(mu, r_prev, w, y, a, nv, s2, alpha, beta)
    res = minimize_scalar(lambda t: O.h_objective(mu + t * d, y, r_prev, a, nv, alpha),
                          bracket=(0.0, 1e-3), tol=1e-14)
    np.testing.assert_allclose(mu_new, mu + res.x * d, rtol=1e-6, atol=1e-9)
    c = O.c_update(r_prev, nv, alpha)

    def brute(K):
        out = np.empty(shape)
        for idx in np.ndindex(shape):
            rp, v, k = r_prev[idx], w[idx], K[idx]
            hh = 1e-6
            dq = lambda r: ((r + hh * r) / rp + k / (r + hh * r) - (r - hh * r) / rp - k / (r - hh * r)) / (2 * hh * r)
            drho = dq(rp) + (rp - v) / s2
            xi = rp / beta if drho > 0 else rp * beta
            sl = (dq(xi) - dq(rp)) / (xi - rp)
            grid = np.linspace(min(rp, xi), max(rp, xi), 20001)
            obj = 0.5 * sl * (grid - rp) ** 2 + dq(rp) * (grid - rp) + (grid - v) ** 2 / (2 * s2)
            out[idx] = grid[np.argmin(obj)]
        return out

    ref = brute(c + np.abs(mu_new) ** 2)
    width = np.abs(r_prev * beta - r_prev / beta)
    assert np.all(np.abs(r_new - ref) <= width / 20000 * 1.5 + 1e-9)
    pre = brute(c + np.abs(mu) ** 2)
    assert np.max(np.abs(pre - r_new) / width) > 1e-2


# ------------------------------------------------------------------ U-Net prior agent normalisation (Sec. III-C)

def test_denoise_unet_normalisation_closed_form():
    """With every weight zero and output bias b the U-Net is the constant b, so
    H(w) = m max(b, floor) with m = sum(w) / (nx ny) (energy per (x, y) column, not the
    mean over nz too).  With random weights H is 1-homogeneous: H(s w) = s H(w)."""
    pytest.importorskip("torch")
    from oracle import unet_oracle as U
    ch = (2, 4, 8)
    rng = _rng(44)
    x = rng.uniform(0.0, 1.0, (8, 4, 4))
    params = np.zeros(U.param_count(*ch))
    for b, floor in ((0.7, 1e-3), (-1.0, 1e-3), (0.2, 0.5)):
        params[-1] = b
        got = O.denoise_unet(x, params, ch, False, floor)
        m = x.sum() / (4 * 4)
        np.testing.assert_allclose(got, np.full(x.shape, m * max(b, floor)), rtol=1e-12)
    p = I.unet_params(ch, seed=3).astype(np.float64)
    h1 = O.denoise_unet(x, p, ch, False, 1e-3)
    h2 = O.denoise_unet(3.7 * x, p, ch, False, 1e-3)
    np.testing.assert_allclose(h2, 3.7 * h1, rtol=1e-10)


# ------------------------------------------------------------------ l2,1 prior agent (Sec. IV comparison prior)

def _l21_objective(r, x, lam):
    return 0.5 * np.sum((r - x) ** 2) + lam * sum(np.linalg.norm(r[z]) for z in range(r.shape[0]))


def test_l21_prox_is_the_minimiser():
    """The l2,1 agent returns the minimiser of 1/2 ||r - x||^2 + lam sum_z ||r_z||: it
    satisfies the optimality conditions (r_z - x_z + lam r_z / ||r_z|| = 0 for a kept plane,
    ||x_z|| <= lam for a zeroed one) and no random perturbation lowers the objective;
    lam = 0 is the identity."""
    rng = _rng(45)
    x = rng.standard_normal((6, 3, 4))
    norms = np.array([np.linalg.norm(x[z]) for z in range(6)])
    lam = float(np.median(norms))           # about half the planes are zeroed
    r = O.denoise_l21(x, lam)
    kept = 0
    for z in range(6):
        if norms[z] > lam:
            kept += 1
            np.testing.assert_allclose(r[z] - x[z] + lam * r[z] / np.linalg.norm(r[z]), 0.0, atol=1e-12)
        else:
            assert np.all(r[z] == 0.0)
    assert 0 < kept < 6
    f0 = _l21_objective(r, x, lam)
    for _ in range(200):
        assert _l21_objective(r + 1e-3 * rng.standard_normal(r.shape), x, lam) >= f0 - 1e-12
    np.testing.assert_array_equal(O.denoise_l21(x, 0.0), x)


def test_l21_prox_brute_force_small():
    """Two planes of two voxels: the prox equals a direct numerical minimisation."""
    from scipy.optimize import minimize
    rng = _rng(46)
    for _ in range(5):
        x = rng.standard_normal((2, 1, 2))
        lam = rng.uniform(0.2, 1.5)
        res = minimize(lambda v: _l21_objective(v.reshape(x.shape), x, lam), x.ravel() * 0.5,
                       method="Powell", options={"xtol": 1e-12, "ftol": 1e-14, "maxiter": 200000})
        np.testing.assert_allclose(O.denoise_l21(x, lam).ravel(), res.x, atol=2e-5)
