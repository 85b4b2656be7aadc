"""FP64 CPU oracle for CLAMP (Allen, Rabb, Buzzard, Bouman, "CLAMP: Majorized
Plug-and-Play for Coherent 3D Lidar Imaging", IEEE TCI 11, 2025).

TEST INFRASTRUCTURE ONLY.  This module is the slow, plain reference that the
CUDA path is checked against.  Only the test-suite, the package smoke check and
the benchmark's CPU-baseline leg may import it; the product path never does.
It shares no code with the CUDA library: numpy (float64 / complex128) with
``numpy.fft`` as the DFT primitive, no blocking, fusion or reordering beyond
what each cited equation states.

Notation follows the paper: n voxels in a [nz][ny][nx] grid, L looks,
``F`` the orthonormal 3D DFT, ``a`` the aperture (lateral pupil x range window),
``A = D(a) F`` (Eq. (A)), ``sigma_w^2`` the data-noise variance, ``sigma^2`` the
forward-agent proximal parameter, ``alpha`` the light fraction through the
aperture, ``mu_l`` the posterior-mean estimate, ``r_l`` the per-look anchor,
``w_j`` the MACE state.

Readings where the paper is silent or garbled (each is used below):
  R1  sigma_w^2 and sigma_eta^2 are the same data-noise variance.
  R2  mu is initialised as A^H y / alpha (Sec. IV-A, Methods), not A^H y (Alg. 2).
  R3  r_{L+3} / n(L+3) in Alg. 1-3 mean L+1 (L forward agents plus one prior).
  R4  the consensus average is  wbar = sum_j upsilon_j w_j  (the 1/(L+1) prefactor in
      Sec. III-A is dropped since the weights already sum to one).
  R5  the line search is the exact minimiser of h (Eq. mu-objective, with the
      noise floor) along +d; the D(1/r') in the printed step size is read as the
      floored D of h.
  R6  the quadratic surrogate of App. A fits the chord of the derivative of the
      Q-term 1/r' - K/r^2 between r' and xi; adding the prox term before or after
      the fit gives the same update.
  R7  beta_k = 1 + 2 / ln(k + 1) for CLAMP iteration k = 1, 2, ... (the printed
      1 + 2/log(k) is infinite at k = 1).
  R8  ties rho'(r') = 0 take xi = beta r' (both branches return r = r').
  R9  c, h and the prox anchor all use the look's own r_l from the previous iteration;
      the prox input is v = w_l.
  R10 convergence error (Eq. mace-convergence-error) is the unweighted stacked
      2-norm  sqrt(sum_j ||r_j - wbar||^2) / sqrt((L+1) ||wbar||^2), evaluated with the
      agent outputs r_j = F_j(w_j) and wbar of the same (pre-update) w.
  R11 for a non-binary aperture, A^H A = F^H D(a^2) F and alpha = mean(a^2), which
      equals ||a||_1 / n when a is binary (Sec. III-B).
  R12 the speckle-average initial image is floored at 1e-12 max to keep r > 0.
  R13 the l2,1 comparison prior (Sec. IV) groups the voxels of each range bin: the norm is
      sum_z ||r_z||_2 over the (y, x) planes r_z (l2 in cross-range, l1 in range).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "fft3", "ifft3", "aperture", "alpha_of", "A_op", "AH_op", "simulate_data",
    "speckle_average", "init_state", "c_update", "h_objective", "grad_direction",
    "line_search_gamma", "beta_k", "prox_quadratic", "forward_agent", "gauss_kernel1d",
    "denoise_gauss", "conv3d", "denoise_cnn", "mace_update", "convergence_error",
    "mu_residual", "reconstruct", "OracleState", "em_surrogate", "exact_nll",
    "exact_posterior", "cubic_prox", "psnr", "cubic_prox_field", "no_aperture_mu", "denoise_l21",
]


# ---------------------------------------------------------------------- forward model

def fft3(x: np.ndarray) -> np.ndarray:
    """Orthonormal 3D DFT F over the last three axes (Eq. (A): F is orthonormal)."""
    return np.fft.fftn(x, axes=(-3, -2, -1), norm="ortho")


def ifft3(x: np.ndarray) -> np.ndarray:
    """F^H, the inverse orthonormal 3D DFT."""
    return np.fft.ifftn(x, axes=(-3, -2, -1), norm="ortho")


def aperture(pupil: np.ndarray, window: np.ndarray) -> np.ndarray:
    """a(kz, ky, kx) = window(kz) * pupil(ky, kx): lateral pupil times range window (Eq. (A))."""
    return window.astype(np.float64)[:, None, None] * pupil.astype(np.float64)[None, :, :]


def alpha_of(a: np.ndarray) -> float:
    """Fraction of light through the aperture, used in A^H A ~ alpha I (Sec. III-B; reading R11)."""
    return float(np.mean(a * a))


def A_op(g: np.ndarray, a: np.ndarray) -> np.ndarray:
    """A g = D(a) F g (Eq. (A))."""
    return a * fft3(g)


def AH_op(y: np.ndarray, a: np.ndarray) -> np.ndarray:
    """A^H y = F^H D(a) y (adjoint of Eq. (A))."""
    return ifft3(a * y)


def simulate_data(r: np.ndarray, speckle: np.ndarray, noise: np.ndarray, a: np.ndarray,
                  noise_var: float) -> np.ndarray:
    """y_l = A g_l + eta_l with g_l = sqrt(r) z_l, z_l ~ CN(0, I), eta_l = sigma_w e_l
    (Eq. (forward-model) with the speckle model Eq. (g-given-r))."""
    g = np.sqrt(r)[None] * speckle
    return A_op(g, a) + math.sqrt(noise_var) * noise


# ---------------------------------------------------------------------- CLAMP pieces

def speckle_average(y: np.ndarray, a: np.ndarray) -> np.ndarray:
    """(1/L) sum_l |A^H y_l|^2, the conventional speckle-averaged image (Sec. I, Fig. 1(c))."""
    return np.mean(np.abs(AH_op(y, a)) ** 2, axis=0)


@dataclass
class OracleState:
    """CLAMP state: mu [L][n] complex, r [L+1][n] (r[L] = prior-agent output), w [L+1][n]."""
    mu: np.ndarray
    r: np.ndarray
    w: np.ndarray
    k: int = 0
    ce_hist: list = field(default_factory=list)
    mu_res_hist: list = field(default_factory=list)


def init_state(y: np.ndarray, a: np.ndarray, r_init: np.ndarray | None = None,
               mu_over_alpha: bool = True) -> OracleState:
    """Initialisation of Alg. 2 with Sec. IV-A (Methods): r = speckle average, w and r
    stacked copies of it, mu_l = A^H y_l / alpha (reading R2); a given r_init
    (warm start) replaces the speckle average.  Floor of reading R12."""
    L = y.shape[0]
    ahy = AH_op(y, a)
    if r_init is None:
        r0 = np.mean(np.abs(ahy) ** 2, axis=0)
    else:
        r0 = np.asarray(r_init, dtype=np.float64).copy()
    r0 = np.maximum(r0, 1e-12 * r0.max())
    mu = ahy / alpha_of(a) if mu_over_alpha else ahy
    r = np.broadcast_to(r0, (L + 1,) + r0.shape).copy()
    w = r.copy()
    return OracleState(mu=mu, r=r, w=w)


def c_update(r_prev: np.ndarray, noise_var: float, alpha: float) -> np.ndarray:
    """c_j = sigma_w^2 r'_j / (alpha r'_j + sigma_w^2): diagonal covariance under
    A^H A ~ alpha I (Sec. III-B; Alg. 2 'Update C_l')."""
    return noise_var * r_prev / (alpha * r_prev + noise_var)


def _dfloor(r_prev, noise_var, alpha):
    """Diagonal of D(1 / (r' + sigma_w^2 / alpha)) in h (Eq. mu-objective)."""
    return 1.0 / (r_prev + noise_var / alpha)


def h_objective(g, y, r_prev, a, noise_var, alpha) -> float:
    """h(g; y, r') = ||y - A g||^2 / (2 sigma_w^2) + g^H D(1/(r' + sigma_w^2/alpha)) g / 2
    (Eq. mu-objective)."""
    res = y - A_op(g, a)
    return float(0.5 / noise_var * np.sum(np.abs(res) ** 2)
                 + 0.5 * np.sum(_dfloor(r_prev, noise_var, alpha) * np.abs(g) ** 2))


def grad_direction(mu, y, r_prev, a, noise_var, alpha) -> np.ndarray:
    """d = -grad h(mu) = A^H (y - A mu) / sigma_w^2 - D mu (Eq. h-gradient; complex
    steepest-descent direction, so that dh/dt along e is -Re<e, d>)."""
    return AH_op(y - A_op(mu, a), a) / noise_var - _dfloor(r_prev, noise_var, alpha) * mu


def line_search_gamma(mu, d, y, r_prev, a, noise_var, alpha) -> float:
    """Exact step gamma* of Eq. (mu-update) in the printed form
    [Re (Ad)^H (y - A mu) - sigma_w^2 Re d^H D mu] / [d^H A^H A d + sigma_w^2 d^H D d],
    with D the floored diagonal of h (reading R5) and A d formed by a separate FFT."""
    D = _dfloor(r_prev, noise_var, alpha)
    Ad = A_op(d, a)
    num = np.real(np.vdot(Ad, y - A_op(mu, a))) - noise_var * np.real(np.vdot(d, D * mu))
    den = np.real(np.vdot(Ad, Ad)) + noise_var * np.real(np.vdot(d, D * d))
    return float(num / den)


def beta_k(k: int) -> float:
    """Interval factor beta = 1 + 2 / ln(k + 1) for iteration k >= 1 (App. A; reading R7)."""
    return 1.0 + 2.0 / math.log(k + 1.0)


def prox_quadratic(v, r_prev, K, prox_var, beta):
    """Reflectance update of App. A (Eqs. convex-surrogate, g, quadratic-surrogate,
    r-update, r-update2), elementwise.

    rho(r)  = r / r' + K / r + (r - v)^2 / (2 sigma^2),  K = c + |mu|^2
    xi      = r'/beta if rho'(r') > 0 else beta r'       (reading R8 for ties)
    a_q,b_q = chord fit of q'(r) = 1/r' - K/r^2 between r' and xi (reading R6)
    r       = (v - sigma^2 b_q) / (1 + sigma^2 a_q), clipped to [min(r', xi), max(r', xi)].
    """
    v = np.asarray(v, dtype=np.float64)
    rp = np.asarray(r_prev, dtype=np.float64)
    K = np.asarray(K, dtype=np.float64)
    drho = 1.0 / rp - K / rp ** 2 + (rp - v) / prox_var
    xi = np.where(drho > 0, rp / beta, beta * rp)
    qp_r = 1.0 / rp - K / rp ** 2
    qp_xi = 1.0 / rp - K / xi ** 2
    a_q = (qp_xi - qp_r) / (xi - rp)
    b_q = qp_r - a_q * rp
    r_new = (v - prox_var * b_q) / (1.0 + prox_var * a_q)
    lo = np.minimum(rp, xi)
    hi = np.maximum(rp, xi)
    return np.clip(r_new, lo, hi)


def forward_agent(mu_l, r_l, w_l, y_l, a, noise_var, prox_var, alpha, beta):
    """One pass of Alg. 2's inner loop for one look (C update, gradient step with
    exact line search, surrogate prox), in the algorithm's order.
    Returns (mu_new, r_new, gamma, d)."""
    c = c_update(r_l, noise_var, alpha)
    d = grad_direction(mu_l, y_l, r_l, a, noise_var, alpha)
    gamma = line_search_gamma(mu_l, d, y_l, r_l, a, noise_var, alpha)
    mu_new = mu_l + gamma * d
    K = c + np.abs(mu_new) ** 2
    r_new = prox_quadratic(w_l, r_l, K, prox_var, beta)
    return mu_new, r_new, gamma, d


# ---------------------------------------------------------------------- prior agents

def gauss_kernel1d(sigma: float) -> np.ndarray:
    """Normalised 3-tap sampled Gaussian [e, 1, e] / (1 + 2e), e = exp(-1 / (2 sigma^2))."""
    e = math.exp(-1.0 / (2.0 * sigma * sigma))
    return np.array([e, 1.0, e]) / (1.0 + 2.0 * e)


def denoise_gauss(x: np.ndarray, sigma: float) -> np.ndarray:
    """3x3x3 separable Gaussian smoother with zero padding (the fixed prior agent H)."""
    g = gauss_kernel1d(sigma)
    out = np.asarray(x, dtype=np.float64)
    for axis in range(3):
        pad = [(0, 0)] * 3
        pad[axis] = (1, 1)
        p = np.pad(out, pad)
        n = out.shape[axis]
        sl = lambda s: tuple(slice(s, s + n) if ax == axis else slice(None) for ax in range(3))
        out = g[0] * p[sl(0)] + g[1] * p[sl(1)] + g[2] * p[sl(2)]
    return out


def conv3d(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Direct 3x3x3 convolution (cross-correlation), zero padding, stride 1.
    x [Cin][nz][ny][nx], w [Cout][Cin][3][3][3] (dz, dy, dx), b [Cout]."""
    cin, nz, ny, nx = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    out = np.zeros((w.shape[0], nz, ny, nx))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                patch = xp[:, dz:dz + nz, dy:dy + ny, dx:dx + nx].reshape(cin, -1)
                out += (w[:, :, dz, dy, dx].astype(np.float64) @ patch).reshape(out.shape)
    return out + b.astype(np.float64)[:, None, None, None]


def bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float values to bfloat16 (round to nearest even), returned as float64."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def denoise_cnn(x: np.ndarray, weights, biases, bf16: bool = False) -> np.ndarray:
    """Residual CNN prior agent H(x) = x + CNN(x): 3x3x3 conv + bias + ReLU on hidden
    layers, linear last layer.  With ``bf16`` the weights and every layer input are
    rounded to bfloat16 (products accumulated in FP64 here)."""
    h = np.asarray(x, dtype=np.float64)[None]
    nl = len(weights)
    for i, (w, b) in enumerate(zip(weights, biases)):
        wi = bf16_round(w) if bf16 else w.astype(np.float64)
        hi = bf16_round(h) if bf16 else h
        h = conv3d(hi, wi, b)
        if i < nl - 1:
            h = np.maximum(h, 0.0)
    return np.asarray(x, dtype=np.float64) + h[0]


def denoise_l21(x: np.ndarray, lam: float) -> np.ndarray:
    """Prior agent of the l2,1-regularised comparison method (Sec. IV: l2 across cross-range,
    l1 across range): the proximal map of lam * sum_z ||r_z||_2, where r_z is the (y, x)
    cross-range plane of range bin z.  Each plane's group is shrunk in l2 norm by lam:
    r_z = max(0, 1 - lam / ||x_z||) x_z (reading R13)."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for z in range(x.shape[0]):
        nrm = math.sqrt(float(np.sum(x[z] * x[z])))
        if nrm > lam:
            out[z] = (1.0 - lam / nrm) * x[z]
    return out


def apply_prior(x: np.ndarray, den: dict) -> np.ndarray:
    if den["kind"] == "gauss":
        return denoise_gauss(x, den["sigma"])
    if den["kind"] == "l21":
        return denoise_l21(x, den["lam"])
    if den["kind"] == "cnn":
        return denoise_cnn(x, den["weights"], den["biases"], bf16=den.get("dtype") == "bf16")
    if den["kind"] == "identity":
        return np.asarray(x, dtype=np.float64).copy()
    if den["kind"] == "unet":
        return denoise_unet(x, den["params"], tuple(den["channels"]), den.get("dtype") == "bf16",
                            den.get("floor", 1e-3))
    raise ValueError(den["kind"])


def denoise_unet(x: np.ndarray, params, channels, bf16: bool, floor: float) -> np.ndarray:
    """U-Net prior agent (Sec. III-C): m max(U(x / m), floor) with m = sum(x) / (nx ny), the
    energy per (x, y) column (reading: the normalisation that makes one trained network
    apply at any range extent); U is the U-Net of ``oracle.unet_oracle``."""
    from . import unet_oracle
    x = np.asarray(x, dtype=np.float64)
    nz, ny, nx = x.shape
    m = x.sum() / (nx * ny)
    if not m > 0:
        m = 1.0
    u = unet_oracle.forward(np.asarray(params, np.float64), (x / m)[None], channels, bf16=bf16).numpy()[0]
    return m * np.maximum(u, floor)


# ---------------------------------------------------------------------- MACE

def consensus_weights(L: int, prior_weight: float = 0.5) -> np.ndarray:
    """upsilon_j = (1 - prior_weight)/L for the L looks and prior_weight for the prior
    (Sec. III-A uses 1/(2L) and 1/2)."""
    v = np.full(L + 1, (1.0 - prior_weight) / L)
    v[L] = prior_weight
    return v


def G_avg(x: np.ndarray, ups: np.ndarray) -> np.ndarray:
    """The weighted average xbar = sum_j upsilon_j x_j of G (Eq. mace; reading R4)."""
    return np.tensordot(ups, x, axes=(0, 0))


def mace_update(r: np.ndarray, w: np.ndarray, ups: np.ndarray, rho: float) -> np.ndarray:
    """Mann step of Alg. 1 / Alg. 2: x = 2 r - w; w <- w + 2 rho (G(x) - r)."""
    x = 2.0 * r - w
    return w + 2.0 * rho * (G_avg(x, ups)[None] - r)


def convergence_error(r: np.ndarray, w: np.ndarray, ups: np.ndarray) -> float:
    """||F(w) - G(w)|| / ||G(w)|| (Eq. mace-convergence-error; reading R10)."""
    wbar = G_avg(w, ups)
    num = np.sum((r - wbar[None]) ** 2)
    den = r.shape[0] * np.sum(wbar ** 2)
    return float(math.sqrt(num / den))


def mu_residual(mu, y, r_prev, a, noise_var, alpha, floored: bool = False) -> float:
    """(1/L) sum_l ||C~_l^{-1} mu_l - A^H y_l / sigma_w^2|| / ||A^H y_l / sigma_w^2||
    (Eq. residual) with C~^{-1} = A^H A / sigma_w^2 + D(1/r') (Eq. Bi).  With
    ``floored`` the D uses the noise floor of h, making the numerator ||d||."""
    vals = []
    for l in range(mu.shape[0]):
        ahy = AH_op(y[l], a) / noise_var
        D = _dfloor(r_prev[l], noise_var, alpha) if floored else 1.0 / r_prev[l]
        cinv_mu = AH_op(A_op(mu[l], a), a) / noise_var + D * mu[l]
        vals.append(np.linalg.norm(cinv_mu - ahy) / np.linalg.norm(ahy))
    return float(np.mean(vals))


def cubic_prox_field(v, K, prox_var) -> np.ndarray:
    """Exact prox of the EM surrogate for every voxel (cubic_prox elementwise)."""
    v = np.asarray(v, dtype=np.float64)
    K = np.broadcast_to(np.asarray(K, dtype=np.float64), v.shape)
    out = np.empty_like(v)
    for idx in np.ndindex(v.shape):
        out[idx] = cubic_prox(float(v[idx]), float(K[idx]), prox_var)
    return out


def no_aperture_mu(y_l, r_prev, noise_var) -> np.ndarray:
    """Closed-form mu step of the no-aperture ablation (Sec. IV-A, a = 1): the minimiser of
    h with A = F, mu = F^H y / (1 + sigma_w^2 D), D = 1/(r' + sigma_w^2) (alpha = 1)."""
    return ifft3(y_l) / (1.0 + noise_var / (r_prev + noise_var))


def clamp_iteration(state: OracleState, y, a, den: dict, noise_var, prox_var,
                    rho=0.5, prior_weight=0.5, exact_prox: bool = False,
                    no_aperture: bool = False) -> OracleState:
    """One iteration of Alg. 2: every forward agent (C, mu, r updates), the prior agent
    on w_{L+1}, then the MACE step.  Records the convergence error (Eq.
    mace-convergence-error) and the mu-residual (Eq. residual, floored form) of the
    iteration's starting state."""
    L = y.shape[0]
    alpha = alpha_of(a)
    k = state.k + 1
    beta = beta_k(k)
    r_new = np.empty_like(state.r)
    mu_new = np.empty_like(state.mu)
    if no_aperture:
        # Sec. IV-A ablation: a = 1 and the mu update in closed form; the prox as in Alg. 2
        state.mu_res_hist.append(0.0)
        for l in range(L):
            mu_new[l] = no_aperture_mu(y[l], state.r[l], noise_var)
            K = c_update(state.r[l], noise_var, 1.0) + np.abs(mu_new[l]) ** 2
            r_new[l] = (cubic_prox_field(state.w[l], K, prox_var) if exact_prox
                        else prox_quadratic(state.w[l], state.r[l], K, prox_var, beta))
    else:
        state.mu_res_hist.append(mu_residual(state.mu, y, state.r[:L], a, noise_var, alpha, floored=True))
        for l in range(L):
            if exact_prox:
                c = c_update(state.r[l], noise_var, alpha)
                d = grad_direction(state.mu[l], y[l], state.r[l], a, noise_var, alpha)
                mu_new[l] = state.mu[l] + line_search_gamma(state.mu[l], d, y[l], state.r[l], a, noise_var,
                                                            alpha) * d
                r_new[l] = cubic_prox_field(state.w[l], c + np.abs(mu_new[l]) ** 2, prox_var)
            else:
                mu_new[l], r_new[l], _, _ = forward_agent(state.mu[l], state.r[l], state.w[l], y[l], a,
                                                           noise_var, prox_var, alpha, beta)
    r_new[L] = apply_prior(state.w[L], den)
    ups = consensus_weights(L, prior_weight)
    state.ce_hist.append(convergence_error(r_new, state.w, ups))
    w_new = mace_update(r_new, state.w, ups, rho)
    return OracleState(mu=mu_new, r=r_new, w=w_new, k=k, ce_hist=state.ce_hist,
                       mu_res_hist=state.mu_res_hist)


def mu_presteps(st: OracleState, y, a, noise_var, steps: int) -> OracleState:
    """Warm-start refinement of mu: ``steps`` times, every look's gradient step with exact
    line search (Alg. 2 steps 6-8) with r' = r_l held fixed and no prox."""
    alpha = alpha_of(a)
    for l in range(y.shape[0]):
        for _ in range(steps):
            d = grad_direction(st.mu[l], y[l], st.r[l], a, noise_var, alpha)
            st.mu[l] = st.mu[l] + line_search_gamma(st.mu[l], d, y[l], st.r[l], a, noise_var, alpha) * d
    return st


def reconstruct(y, pupil, window, den: dict, noise_var, prox_var, iters, rho=0.5,
                prior_weight=0.5, r_init=None, tol: float = 0.0, exact_prox: bool = False,
                no_aperture: bool = False, init_mu_steps: int = 0):
    """CLAMP (Alg. 2): initialise (Sec. IV-A), iterate, output r* = wbar.
    Stops early once the convergence error falls to ``tol`` (when tol > 0).
    ``exact_prox``: the cubic-root prox of the EM surrogate instead of App. A's quadratic step.
    ``no_aperture``: the Sec. IV-A ablation (a = 1, closed-form mu update).
    ``init_mu_steps``: with ``r_init``, that many mu refinement steps (``mu_presteps``)."""
    a = np.ones((len(window), pupil.shape[0], pupil.shape[1])) if no_aperture else aperture(pupil, window)
    st = init_state(y, a, r_init)
    if r_init is not None and init_mu_steps > 0 and not no_aperture:
        st = mu_presteps(st, y, a, noise_var, init_mu_steps)
    for _ in range(iters):
        st = clamp_iteration(st, y, a, den, noise_var, prox_var, rho, prior_weight, exact_prox, no_aperture)
        if tol > 0 and st.ce_hist[-1] <= tol:
            break
    ups = consensus_weights(y.shape[0], prior_weight)
    return G_avg(st.w, ups), st


# ---------------------------------------------------------------------- pins' exact forms

def em_surrogate(r, mu, c) -> float:
    """f^(r; mu, c) = sum_j log r_j + (|mu_j|^2 + c_j) / r_j (Eq. em-surrogate-final)."""
    return float(np.sum(np.log(r) + (np.abs(mu) ** 2 + c) / r))


def dense_A(a: np.ndarray) -> np.ndarray:
    """Dense matrix of A = D(a) F for tiny volumes (columns are A e_j)."""
    n = a.size
    eye = np.eye(n).reshape((n,) + a.shape)
    return np.stack([A_op(e, a).ravel() for e in eye], axis=1)


def exact_nll(r: np.ndarray, y: np.ndarray, a: np.ndarray, noise_var: float) -> float:
    """f(r) = -log p(y | r) up to a constant: log det S + y^H S^{-1} y with
    S = A D(r) A^H + sigma_w^2 I (Eq. y-given-r)."""
    Am = dense_A(a)
    S = Am @ np.diag(r.ravel()) @ Am.conj().T + noise_var * np.eye(a.size)
    sign, logdet = np.linalg.slogdet(S)
    yv = y.ravel()
    return float(np.real(logdet) + np.real(np.vdot(yv, np.linalg.solve(S, yv))))


def exact_posterior(r_prev: np.ndarray, y: np.ndarray, a: np.ndarray, noise_var: float):
    """Exact mean and covariance of g | y, r' (Eqs. mu2, Bi) for tiny volumes."""
    Am = dense_A(a)
    Cinv = Am.conj().T @ Am / noise_var + np.diag(1.0 / r_prev.ravel())
    C = np.linalg.inv(Cinv)
    mu = C @ (Am.conj().T @ y.ravel()) / noise_var
    return mu.reshape(a.shape), C


def cubic_prox(v: float, K: float, prox_var: float) -> float:
    """Exact prox of one voxel's surrogate: argmin_r log r + K/r + (r - v)^2/(2 sigma^2),
    the positive real root of r^3 - v r^2 + sigma^2 r - sigma^2 K = 0 (Sec. III-B,
    'closed form by solving for a root of a cubic')."""
    roots = np.roots([1.0, -v, prox_var, -prox_var * K])
    real = [x.real for x in roots if abs(x.imag) < 1e-9 * max(1.0, abs(x)) and x.real > 0]
    obj = lambda r: math.log(r) + K / r + (r - v) ** 2 / (2 * prox_var)
    return min(real, key=obj)


def psnr(r_hat: np.ndarray, r: np.ndarray) -> float:
    """PSNR(beta* r_hat, r) = 10 log10(n / ||beta* r_hat - r||^2), beta* = r_hat^T r / ||r_hat||^2
    (Eq. psnr)."""
    beta = float(np.vdot(r_hat, r) / np.vdot(r_hat, r_hat))
    return 10.0 * math.log10(r.size / float(np.sum((beta * r_hat - r) ** 2)))


# ---------------------------------------------------------------------- point-cloud metrics

def point_cloud_metrics(r_hat: np.ndarray, r_true: np.ndarray, threshold: float, max_dist: float) -> dict:
    """Point-cloud metrics of Sec. IV-B (Eqs. pc-distance, nrmse).

    P = voxels of r_hat above ``threshold``, Q = voxels of r_true above 0, with voxel
    coordinates (x, y, z).  Each p is matched to its nearest q (Euclidean; ties to the
    smallest linear index of q, a reading: the paper leaves ties open); p with no q within
    ``max_dist`` is removed, and the false-positive rate is the removed fraction.  The mean
    distance and NRMSE(beta* r_hat, r) = sqrt(sum (b r_hat_p - r_q)^2 / sum r_q^2) with
    b = argmin (closed form sum r_hat r_q / sum r_hat^2) run over the kept points.
    scipy's k-d tree gives the nearest distance; a ball query at that distance applies the
    tie rule.
    """
    from scipy.spatial import cKDTree
    nz, ny, nx = r_true.shape
    qi = np.flatnonzero(r_true.ravel() > 0)
    pi = np.flatnonzero(r_hat.ravel() > threshold)

    def coords(idx):
        return np.stack([idx % nx, (idx // nx) % ny, idx // (nx * ny)], axis=1).astype(np.float64)

    if pi.size == 0 or qi.size == 0:
        return dict(distance=0.0, false_positive_rate=1.0 if pi.size else 0.0, nrmse=0.0, kept=0,
                    removed=int(pi.size), beta=0.0)
    tree = cKDTree(coords(qi))
    pc = coords(pi)
    d, _ = tree.query(pc, k=1)
    match = np.empty(pi.size, dtype=np.int64)
    for j in range(pi.size):
        cand = tree.query_ball_point(pc[j], d[j] + 1e-9)
        cand = [c for c in cand if abs(np.linalg.norm(coords(qi[[c]])[0] - pc[j]) - d[j]) < 1e-9]
        match[j] = qi[min(cand, key=lambda c: qi[c])]
    keep = d <= max_dist
    rh = r_hat.ravel()[pi[keep]].astype(np.float64)
    rq = r_true.ravel()[match[keep]].astype(np.float64)
    b = float(rh @ rq / (rh @ rh)) if rh.size else 0.0
    nrmse = float(np.sqrt(np.sum((b * rh - rq) ** 2) / np.sum(rq * rq))) if rh.size else 0.0
    return dict(distance=float(d[keep].mean()) if keep.any() else 0.0,
                false_positive_rate=float((~keep).sum() / pi.size), nrmse=nrmse, kept=int(keep.sum()),
                removed=int((~keep).sum()), beta=b)
