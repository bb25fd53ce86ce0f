"""Pins of the FP64 oracle's loss, gradient, spectral method and GD (Sec. II-B, IV).

The gradient is pinned by central finite differences, the spectral method by
the leading eigenvector of the explicitly formed covariance matrix (a library
eigensolver on a matrix the oracle never forms), GD by exact recovery on
noiseless tiny problems, and the metrics by brute force over the global phase.
"""
import json
import os

import numpy as np
import pytest

import oracle as O
import synthetic as S

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_claims.json")


def _problem(seed, n, alpha, L, signal="gaussian"):
    m = int(round(alpha * n))
    theta = S.phases(seed, L, m)
    x = S.signal_gaussian(seed, 1, n) if signal == "gaussian" else S.signal_amplitude_phase(seed, 1, n)
    fwd, adj = O.structured_ops(theta, n, m)
    y = np.abs(fwd(x)) ** 2
    return theta, x, y, fwd, adj, m


def test_gradient_matches_central_differences():
    """dL/dRe x_k = 2 Re g_k and dL/dIm x_k = 2 Im g_k, g = 2 A^H((|Ax|^2 - y) Ax)."""
    n, m = 8, 32
    theta = S.phases(1, 2, m)
    fwd, adj = O.structured_ops(theta, n, m)
    x_true = S.signal_gaussian(1, 1, n)
    y = np.abs(fwd(x_true)) ** 2
    x = S.signal_gaussian(2, 1, n)
    _, g = O.loss_and_grad(x, y, fwd, adj)
    h = 1e-6
    for k in range(n):
        for direction, part in ((1.0, np.real), (1j, np.imag)):
            xp = x.copy()
            xm = x.copy()
            xp[0, k] += h * direction
            xm[0, k] -= h * direction
            fd = (O.intensity_loss(fwd(xp), y)[0] - O.intensity_loss(fwd(xm), y)[0]) / (2 * h)
            assert np.isclose(fd, 2 * part(g[0, k]), rtol=1e-6, atol=1e-7)


def test_loss_is_brute_force_sum():
    n, m = 6, 24
    theta = S.phases(4, 2, m)
    A = O.dense_structured_matrix(theta, n, m)
    x = S.signal_gaussian(4, 1, n)[0]
    y = np.linspace(0.0, 1.0, m)
    expect = 0.0
    for i in range(m):
        zi = sum(A[i, j] * x[j] for j in range(n))
        expect += (abs(zi) ** 2 - y[i]) ** 2
    assert np.isclose(O.intensity_loss(O.forward(x, theta, m), y), expect, rtol=1e-12)


def test_gradient_vanishes_at_truth_and_loss_is_phase_blind():
    theta, x, y, fwd, adj, m = _problem(3, 16, 4, 2)
    loss, g = O.loss_and_grad(x, y, fwd, adj)
    assert loss[0] < 1e-25 and np.max(np.abs(g)) < 1e-12
    x2 = S.signal_gaussian(9, 1, 16)
    l1 = O.intensity_loss(fwd(x2), y)
    l2 = O.intensity_loss(fwd(np.exp(0.7j) * x2), y)
    assert np.allclose(l1, l2, rtol=1e-12)


def test_spectral_weights_closed_form():
    y = np.array([[0.0, 0.5, 1.0, 2.0, 4.5]])  # sum 8, m 5 -> y_hat = 5y/8
    yhat = 5 * y / 8
    assert np.allclose(O.spectral_weights(y, "identity"), yhat)
    t = O.spectral_weights(y, "optimal", lam=-1.0)
    # y_hat = [0, 0.3125, 0.625, 1.25, 2.8125]: 1 - 1/y_hat = [-inf, -2.2, -0.6, 0.2, 0.6444]
    assert np.allclose(t, [[-1.0, -1.0, -0.6, 0.2, 1 - 1 / 2.8125]])
    assert np.isclose(O.spectral_weights(y, "identity").mean(), 1.0)
    with pytest.raises(ValueError):
        O.spectral_weights(y, "nope")


@pytest.mark.parametrize("mode,lam", [("identity", -1.0), ("optimal", -1.0), ("optimal", -0.3)])
def test_power_iteration_reaches_top_eigenvector(mode, lam):
    """The iterate approaches the leading eigenvector of the explicit n x n matrix
    M = A^H diag(T) A (Eq. 3) within the power-iteration error bound
    tan(angle_T) <= tan(angle_0) * rho^T, rho = max_{i>=2}|mu_i + s| / (mu_1 + s)."""
    n, m, L = 24, 96, 2
    theta, x, y, fwd, adj, _ = _problem(5, n, 4, L)
    A = O.dense_structured_matrix(theta, n, m)
    w = O.spectral_weights(y, mode, lam)[0]
    M = A.conj().T @ (w[:, None] * A)
    mu, V = np.linalg.eigh(M)
    u1 = V[:, -1]
    s = 0.0 if mode == "identity" else -2.0 * lam
    rho = np.max(np.abs(mu[:-1] + s)) / (mu[-1] + s)
    assert rho < 1
    v0 = S.start_vector(5, 1, n)
    c0 = abs(np.vdot(u1, v0[0])) / np.linalg.norm(v0)
    tan0 = np.sqrt(1 - c0 ** 2) / c0
    for T in (5, 40, 200):
        xs = O.spectral_init(y, v0, fwd, adj, T, mode=mode, lam=lam)[0]
        assert np.isclose(np.linalg.norm(xs), np.sqrt(y.sum()), rtol=1e-12)
        v = xs / np.linalg.norm(xs)
        c = abs(np.vdot(u1, v))
        sinT = np.linalg.norm(v - u1 * np.vdot(u1, v))  # accurate for tiny angles
        assert sinT / c <= tan0 * rho ** T * (1 + 1e-6) + 1e-12


def test_gd_recovers_noiseless_tiny_problem():
    """GD from the spectral start recovers x up to a global phase at alpha = 4,
    L = 2 (full recovery by alpha ~ 3 per Sec. IV-A), with a decreasing loss."""
    errs = []
    for seed in range(6):
        theta, x, y, fwd, adj, m = _problem(seed, 32, 4, 2)
        x0 = O.spectral_init(y, S.start_vector(seed, 1, 32), fwd, adj, 50, mode="optimal")
        xT, hist = O.gradient_descent(x0, y, fwd, adj, 3000, mu0=0.1)
        errs.append(O.relative_error_global_phase(xT, x)[0])
        assert hist[-1, 0] < 1e-12 * hist[0, 0]
        assert np.all(np.diff(hist[:, 0]) <= 1e-12 * hist[0, 0])
    assert np.max(errs) < 1e-8


def test_metrics_brute_force_over_phase():
    rng = np.random.default_rng(3)
    x = rng.standard_normal(20) + 1j * rng.standard_normal(20)
    xh = x + 0.3 * (rng.standard_normal(20) + 1j * rng.standard_normal(20))
    xh = np.exp(1.1j) * xh
    phis = np.linspace(0, 2 * np.pi, 200001)
    brute = min(np.linalg.norm(np.exp(1j * p) * xh - x) for p in phis[::100])
    fine = np.min(np.linalg.norm(np.exp(1j * phis[:, None]) * xh[None] - x[None], axis=1))
    r = O.relative_error_global_phase(xh[None], x[None])[0]
    assert r <= brute / np.linalg.norm(x) + 1e-12
    assert np.isclose(r, fine / np.linalg.norm(x), rtol=1e-6)
    assert np.isclose(O.cosine_similarity(np.exp(2.0j) * 3 * x[None], x[None])[0], 1.0)
    assert np.isclose(O.relative_error_global_phase(np.exp(2.0j) * x[None], x[None])[0], 0.0, atol=1e-7)
    # orthogonal estimate: cosine 0
    e1 = np.zeros(4, complex); e1[0] = 1
    e2 = np.zeros(4, complex); e2[1] = 1j
    assert O.cosine_similarity(e1[None], e2[None])[0] == 0.0


def test_paper_claims_layers_and_alpha():
    """Qualitative claims of Sec. IV (recorded in tests/golden/paper_claims.json):
    two layers beat one by a wide margin, three layers are close to two, and
    accuracy grows with alpha. Spectral method only, as in Fig. 3."""
    claims = json.load(open(GOLDEN))
    assert "two_layers_beat_one" in claims and "monotone_in_alpha" in claims

    def cos(n, alpha, L, seed):
        theta, x, y, fwd, adj, _ = _problem(seed, n, alpha, L)
        xs = O.spectral_init(y, S.start_vector(seed, 1, n), fwd, adj, 300, mode="optimal")
        return O.cosine_similarity(xs, x)[0]

    seeds = range(6)
    c = {(a, L): np.mean([cos(64, a, L, s) for s in seeds]) for a in (2, 3, 4) for L in (1, 2, 3)}
    for a in (3, 4):
        assert c[(a, 2)] > c[(a, 1)] + 0.25
        assert abs(c[(a, 3)] - c[(a, 2)]) < 0.1
    assert c[(2, 2)] < c[(3, 2)] < c[(4, 2)]


def test_step_ramp_and_gd_with_warmup():
    """ramp_t = 1 - exp(-(t+1)/tau0): closed form at chosen t; constant when tau0 = 0;
    GD with the warm-up still recovers the tiny noiseless problem."""
    assert O.step_ramp(0, 0.0) == 1.0 and O.step_ramp(123, 0.0) == 1.0
    assert np.isclose(O.step_ramp(99, 100.0), 1 - np.exp(-1.0))
    assert np.isclose(O.step_ramp(0, 1.0), 1 - np.exp(-1.0))
    assert O.step_ramp(5, 10.0) < O.step_ramp(6, 10.0) < 1.0
    theta, x, y, fwd, adj, m = _problem(2, 32, 4, 2)
    x0 = O.spectral_init(y, S.start_vector(2, 1, 32), fwd, adj, 50, mode="optimal")
    # one step by hand: x1 = x0 - (1 - e^{-1/tau0}) * mu0 * m / sum(y) * g(x0)
    _, g0 = O.loss_and_grad(x0, y, fwd, adj)
    x1, _ = O.gradient_descent(x0, y, fwd, adj, 1, mu0=0.15, tau0=20.0)
    assert np.allclose(x1, x0 - (1 - np.exp(-1 / 20.0)) * 0.15 * m / y.sum() * g0, atol=1e-12)
    xT, hist = O.gradient_descent(x0, y, fwd, adj, 3000, mu0=0.15, tau0=100.0)
    assert O.relative_error_global_phase(xT, x)[0] < 1e-8


def _linearised_gradient_matrix(Adense, z):
    """Real 2n x 2n matrix of delta -> 4 A^H(z * Re(conj(z) * A delta)), the first-order
    change of g = 2 A^H((|Ax|^2 - y) Ax) at the solution (where |Ax|^2 = y),
    acting on delta = a + i b stored as [a; b]; formed from the explicit matrix A."""
    n = Adense.shape[1]
    J = np.zeros((2 * n, 2 * n))
    for j in range(2 * n):
        d = np.zeros(n, complex)
        d[j % n] = 1.0 if j < n else 1j
        u = 4.0 * (Adense.conj().T @ (z * np.real(np.conj(z) * (Adense @ d))))
        J[:n, j], J[n:, j] = u.real, u.imag
    return J


@pytest.mark.parametrize("seed,L", [(3, 2), (4, 1)])
def test_gd_step_stability_threshold(seed, L):
    """Linear stability of GD at the solution. Near x*, x_{t+1} - x* ~ (I - mu J)(x_t - x*)
    with J the linearised gradient map (symmetric positive semidefinite in the real
    inner product, with the global-phase direction i x* in its kernel), so GD with
    mu = mu0 m / sum(y) is stable iff mu0 < 2 sum(y) / (m lambda_max(J)). J is formed
    from the explicit dense A (not the oracle's FFT path); the oracle's
    gradient_descent, started at x* + eps v_max, must shrink the deviation at 0.9 of the
    threshold and grow it at 1.1. A dropped factor 2 in the gradient or a step scaled
    by the mean of y instead of its sum moves the threshold and fails one side."""
    n, alpha = 8, 4
    theta, x, y, fwd, adj, m = _problem(seed, n, alpha, L)
    Ad = O.dense_structured_matrix(theta, n, m)
    z = (Ad @ x[0])
    J = _linearised_gradient_matrix(Ad, z)
    assert np.allclose(J, J.T, atol=1e-12)
    ev, V = np.linalg.eigh(J)
    assert ev[0] > -1e-12
    ix = np.concatenate([-x[0].imag, x[0].real])  # i x* as a real vector
    assert np.linalg.norm(J @ ix) <= 1e-12 * np.linalg.norm(J) * np.linalg.norm(ix)
    v = V[:, -1]
    dmax = (v[:n] + 1j * v[n:])[None]
    mu0_crit = 2.0 * y.sum() / (m * ev[-1])
    eps = 1e-7 * np.linalg.norm(x)
    T = 40
    for f, grows in ((0.9, False), (1.1, True)):
        xT, _ = O.gradient_descent(x + eps * dmax, y, fwd, adj, T, mu0=f * mu0_crit, tau0=0.0)
        ratio = np.linalg.norm(xT - x) / eps
        expected = abs(1.0 - 2.0 * f) ** T  # 0.8^40 or 1.2^40
        assert (ratio > 1.0) == grows, (f, ratio)
        assert 0.5 * expected <= ratio <= 2.0 * expected, (f, ratio, expected)


def test_gd_warmup_ramp_follows_the_linearised_product():
    """The warm-up ramp over many steps: near x*, along the top eigenvector v of
    the linearised gradient map J, GD with mu_t = mu0 ramp_t m / sum(y) scales
    the deviation by prod_t |1 - mu_t lambda_max|, ramp_t = 1 - exp(-(t+1)/tau0).
    At mu0 = 0.4 of the stability limit every factor lies in (0, 1); the
    oracle's GD must follow the product within 5% over 20 steps, which tells it
    apart from a ramp shifted by one step (a factor 2 off)."""
    n, alpha, L, seed, tau0, T = 8, 4, 2, 3, 20.0, 20
    theta, x, y, fwd, adj, m = _problem(seed, n, alpha, L)
    Ad = O.dense_structured_matrix(theta, n, m)
    J = _linearised_gradient_matrix(Ad, Ad @ x[0])
    ev, V = np.linalg.eigh(J)
    dmax = (V[:n, -1] + 1j * V[n:, -1])[None]
    mu0 = 0.4 * 2.0 * y.sum() / (m * ev[-1])
    mu = mu0 * m / y.sum()
    eps = 1e-7 * np.linalg.norm(x)
    xT, _ = O.gradient_descent(x + eps * dmax, y, fwd, adj, T, mu0=mu0, tau0=tau0)
    expected = np.prod([abs(1.0 - mu * (1.0 - np.exp(-(t + 1) / tau0)) * ev[-1]) for t in range(T)])
    shifted = np.prod([abs(1.0 - mu * (1.0 - np.exp(-(t + 2) / tau0)) * ev[-1]) for t in range(T)])
    ratio = np.linalg.norm(xT - x) / eps
    assert abs(ratio / expected - 1.0) <= 0.05, (ratio, expected)
    assert abs(ratio / shifted - 1.0) > 0.5, (ratio, shifted)
