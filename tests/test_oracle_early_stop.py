"""Pins of the oracle's early-stopping GD against plain GD (pinned in
test_oracle_recovery.py) and a brute-force scan of its loss history: the rule
stops at the first multiple of check_every where every problem's last
relative loss change is within rel_tol, and returns exactly the iterate of
plain GD run for that many iterations."""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def _problem(B=3, n=32, m=128, L=2, seed=8):
    """Noisy measurements: the loss levels off, so its relative change decays
    and the rule stops. (Noiseless GD converges linearly, the loss shrinking by
    a few percent per iteration to zero, and a relative-change rule with a
    smaller tolerance than that rate never fires.)"""
    th = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(th, n, m)
    x_true = S.signal_gaussian(seed, B, n)
    y0 = np.abs(fwd(x_true)) ** 2
    y = np.maximum(y0 + S.gaussian_noise(seed, y0.shape, 0.05 * y0.mean()), 0.0)
    x0 = O.spectral_init(y, S.start_vector(seed, B, n), fwd, adj, 30, mode="optimal")
    return y, x0, fwd, adj


def test_zero_tolerance_runs_every_iteration():
    y, x0, fwd, adj = _problem()
    x, h, t = O.gradient_descent_early_stop(x0, y, fwd, adj, 60, 0.0, 10, mu0=0.1, tau0=5.0)
    xr, hr = O.gradient_descent(x0, y, fwd, adj, 60, mu0=0.1, tau0=5.0)
    assert t == 60 and np.array_equal(x, xr) and np.array_equal(h, hr)


def test_huge_tolerance_stops_at_first_check():
    y, x0, fwd, adj = _problem()
    x, h, t = O.gradient_descent_early_stop(x0, y, fwd, adj, 60, 10.0, 7, mu0=0.1, tau0=5.0)
    xr, hr = O.gradient_descent(x0, y, fwd, adj, 7, mu0=0.1, tau0=5.0)
    assert t == 7 and np.array_equal(x, xr) and np.array_equal(h, hr)


@pytest.mark.parametrize("tol,every", [(1e-2, 5), (1e-3, 10), (1e-4, 4)])
def test_stop_matches_brute_force_scan(tol, every):
    y, x0, fwd, adj = _problem()
    T = 400
    _, hr = O.gradient_descent(x0, y, fwd, adj, T, mu0=0.1, tau0=5.0)
    want = T
    for t in range(every - 1, T - 1, every):
        if all(abs(hr[t - 1, b] - hr[t, b]) <= tol * hr[t - 1, b] for b in range(hr.shape[1])):
            want = t + 1
            break
    x, h, got = O.gradient_descent_early_stop(x0, y, fwd, adj, T, tol, every, mu0=0.1, tau0=5.0)
    assert got == want and every < got < T  # the rule fires, and not at the first check
    xr, _ = O.gradient_descent(x0, y, fwd, adj, got, mu0=0.1, tau0=5.0)
    assert np.array_equal(x, xr) and np.array_equal(h, hr[:got])


def test_check_every_must_allow_two_losses():
    y, x0, fwd, adj = _problem()
    with pytest.raises(ValueError):
        O.gradient_descent_early_stop(x0, y, fwd, adj, 10, 1e-3, 1)


def test_relative_change_is_taken_against_the_previous_loss():
    """At the first check the last change is r = |L_{t-1} - L_t| / L_{t-1}; a
    tolerance between r and r / (1 - r) stops there only when the change is
    divided by the previous loss (as the rule states), not by the current one."""
    y, x0, fwd, adj = _problem(B=1)
    every = 6
    _, hr = O.gradient_descent(x0, y, fwd, adj, every, mu0=0.1, tau0=5.0)
    t = every - 1
    r = abs(hr[t - 1, 0] - hr[t, 0]) / hr[t - 1, 0]
    assert 0.01 < r < 0.9
    tol = 0.5 * (r + r / (1.0 - r))
    assert r <= tol < abs(hr[t - 1, 0] - hr[t, 0]) / hr[t, 0]
    _, _, got = O.gradient_descent_early_stop(x0, y, fwd, adj, 100, tol, every, mu0=0.1, tau0=5.0)
    assert got == every


# ------------------------------------------------------------ power iteration

def _spec_problem(B=2, n=24, m=96, L=2, seed=4):
    th = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(th, n, m)
    y = np.abs(fwd(S.signal_gaussian(seed, B, n))) ** 2
    return th, y, S.start_vector(seed, B, n), fwd, adj


@pytest.mark.parametrize("mode", ["identity", "optimal"])
def test_power_iteration_zero_and_huge_tolerance(mode):
    th, y, v0, fwd, adj = _spec_problem()
    x, lams, run = O.spectral_init_early_stop(y, v0, fwd, adj, 40, 0.0, 8, mode=mode)
    assert run == 40 and np.array_equal(x, O.spectral_init(y, v0, fwd, adj, 40, mode=mode))
    x, lams, run = O.spectral_init_early_stop(y, v0, fwd, adj, 40, 10.0, 8, mode=mode)
    assert run == 8 and np.array_equal(x, O.spectral_init(y, v0, fwd, adj, 8, mode=mode))


def test_power_iteration_estimates_by_brute_force_and_top_eigenvalue():
    """lambda_t recomputed from scratch: v_t from t plain power steps, then
    ||M v_t + s v_t|| with M formed explicitly; the stop point is the first
    check where every change is within rel_tol; lambda converges to the top
    eigenvalue of M + s I (dense eigensolver)."""
    th, y, v0, fwd, adj = _spec_problem()
    n, m, lam = 24, 96, -1.0
    A = O.dense_structured_matrix(th, n, m)
    w = O.spectral_weights(y, "optimal", lam)
    s_ = -2.0 * lam
    T, tol, every = 120, 1e-4, 6
    x, lams, run = O.spectral_init_early_stop(y, v0, fwd, adj, T, tol, every, mode="optimal", lam=lam)
    brute = np.zeros((run, y.shape[0]))
    for t in range(run):
        vt = O.spectral_init(y, v0, fwd, adj, t, mode="optimal", lam=lam) / np.sqrt(np.sum(y, -1, keepdims=True))
        for b in range(y.shape[0]):
            M = A.conj().T @ (w[b][:, None] * A) + s_ * np.eye(n)
            brute[t, b] = np.linalg.norm(M @ vt[b])
    assert np.allclose(lams, brute, rtol=1e-10)
    want = T
    for t in range(every - 1, T - 1, every):
        if t < run and np.all(np.abs(brute[t - 1] - brute[t]) <= tol * brute[t - 1]):
            want = t + 1
            break
    assert run == want and every < run < T
    for b in range(y.shape[0]):
        M = A.conj().T @ (w[b][:, None] * A) + s_ * np.eye(n)
        top = np.max(np.linalg.eigvalsh(M))
        assert abs(lams[-1, b] - top) <= 1e-2 * top
