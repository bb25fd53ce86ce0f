"""Loss, gradient, spectral initialisation, gradient descent and metrics (FP64).

Test infrastructure only (see the package docstring).

Every solver takes the sensing operator as a pair of callables
``fwd(x) -> A x`` and ``adj(z) -> A^H z`` so the same plain code serves the
structured model (Sec. III) and the dense i.i.d. model (Sec. II-A).

Readings of the paper used here:
* Eq. 2 prints diag(x_hat); that is dimensionally inconsistent, and the
  gradient of the loss of Sec. II-B-1 is taken with diag(A x_hat):
  grad = -2 A^H diag(A x_hat)(y - |A x_hat|^2) = 2 A^H((|A x_hat|^2 - y) * A x_hat),
  the Wirtinger derivative dL/d conj(x). The derivative with respect to the
  real and imaginary parts is twice its real and imaginary parts.
* The loss is the sum (not the mean) of squared intensity residuals.
* Step size (the paper gives none): mu_t = mu0 * ramp_t * m / sum(y), with
  sum(y) = ||x||^2 for the unitary model setting the scale and
  ramp_t = 1 - exp(-(t+1)/tau0) a warm-up in the manner of the Wirtinger-flow
  schedule (Candes, Li and Soltanolkotabi, 2015); tau0 = 0 means a constant
  step (ramp_t = 1). A constant mu0 = 0.1 diverges from poor spectral starts.
* Spectral weights: y_hat = m * y / sum(y) (mean one). The default weight is
  the identity, T(y_hat) = y_hat, i.e. M = A^H diag(y_hat) A; the optional
  weight is the preprocessing T(y_hat) = max(1 - 1/y_hat, lambda) of Sec. II-B-2
  (lambda < 0, T = lambda where y_hat <= 0). The 1/m factor of Eq. 3 is dropped
  (a positive scale does not change the eigenvector; with A^H A = I the
  spectrum of M then lies in [lambda, 1], the range the shift of Eq. 4 assumes).
* Power iteration (Eq. 4): u = M v - 2*lambda*v for the preprocessed weight and
  u = M v for the identity weight; v is normalised to unit norm every
  iteration (including the start vector), and the estimate is
  x0 = sqrt(sum(y)) * v, the exact scale for noiseless y since sum(y) = ||x||^2.
"""
from __future__ import annotations

import numpy as np

from .operator import adjoint, forward

MU0_DEFAULT = 0.1


def structured_ops(theta: np.ndarray, n: int, m: int):
    """(fwd, adj) callables of the structured operator of Eq. 5."""
    return (lambda x: forward(x, theta, m)), (lambda z: adjoint(z, theta, n))


def intensity_loss(z: np.ndarray, y: np.ndarray) -> np.ndarray:
    """L = || |z|^2 - y ||^2 per problem (sum over the last axis) (Sec. II-B-1)."""
    r = np.abs(z) ** 2 - y
    return np.sum(r * r, axis=-1)


def loss_and_grad(x: np.ndarray, y: np.ndarray, fwd, adj):
    """Loss and gradient 2 A^H((|Ax|^2 - y) * Ax) of Eq. 2 (read with diag(Ax))."""
    z = fwd(x)
    r = np.abs(z) ** 2 - y
    loss = np.sum(r * r, axis=-1)
    grad = 2.0 * adj(r * z)
    return loss, grad


def step_ramp(t: int, tau0: float) -> float:
    """Warm-up factor of step t: 1 - exp(-(t+1)/tau0), or 1 when tau0 == 0."""
    return 1.0 if tau0 == 0 else 1.0 - np.exp(-(t + 1) / tau0)


def gradient_descent(x0: np.ndarray, y: np.ndarray, fwd, adj, iters: int,
                     mu0: float = MU0_DEFAULT, tau0: float = 0.0):
    """x_{t+1} = x_t - mu_t * grad(x_t), mu_t = mu0 * ramp_t * m / sum(y) (Sec. II-B-1, Sec. IV-A).

    Returns (x_T, loss history [iters, ...]); entry t is the loss at x_t.
    """
    x = np.array(x0, dtype=np.complex128, copy=True)
    y = np.asarray(y, dtype=np.float64)
    m = y.shape[-1]
    mu = (mu0 * m / np.sum(y, axis=-1))[..., None]
    hist = []
    for t in range(iters):
        loss, g = loss_and_grad(x, y, fwd, adj)
        hist.append(loss)
        x = x - (step_ramp(t, tau0) * mu) * g
    return x, np.array(hist)


def gradient_descent_early_stop(x0: np.ndarray, y: np.ndarray, fwd, adj, max_iters: int, rel_tol: float,
                                check_every: int, mu0: float = MU0_DEFAULT, tau0: float = 0.0):
    """Gradient descent with early stopping (Sec. IV-A runs GD "with early
    stopping" without stating the rule). Reading: after every `check_every`
    iterations, stop once every problem's loss changed over the last
    iteration by at most rel_tol of its previous value,
    |L(x_{t-1}) - L(x_t)| <= rel_tol * L(x_{t-1}), where t is the chunk's
    last iteration and L(x_t) the loss at the iterate that iteration updates.

    Returns (x, loss history [iterations run, ...], iterations run).
    """
    if check_every < 2:
        raise ValueError("check_every must be >= 2")
    x = np.array(x0, dtype=np.complex128, copy=True)
    y = np.asarray(y, dtype=np.float64)
    m = y.shape[-1]
    mu = (mu0 * m / np.sum(y, axis=-1))[..., None]
    hist = []
    for t in range(max_iters):
        loss, g = loss_and_grad(x, y, fwd, adj)
        hist.append(loss)
        x = x - (step_ramp(t, tau0) * mu) * g
        if (t + 1) % check_every == 0 and t + 1 < max_iters:
            if np.all(np.abs(hist[t - 1] - hist[t]) <= rel_tol * hist[t - 1]):
                return x, np.array(hist), t + 1
    return x, np.array(hist), max_iters


def spectral_weights(y: np.ndarray, mode: str = "identity", lam: float = -1.0) -> np.ndarray:
    """Weights of the covariance of Eq. 3 on y_hat = m*y/sum(y).

    mode "identity": T(y_hat) = y_hat. mode "optimal": T(y_hat) = max(1 - 1/y_hat, lam)
    (Sec. II-B-2), with T = lam where y_hat <= 0.
    """
    y = np.asarray(y, dtype=np.float64)
    m = y.shape[-1]
    yhat = m * y / np.sum(y, axis=-1, keepdims=True)
    if mode == "identity":
        return yhat
    if mode == "optimal":
        pos = yhat > 0
        t = np.full_like(yhat, lam)
        t[pos] = np.maximum(1.0 - 1.0 / yhat[pos], lam)
        return t
    raise ValueError(f"unknown spectral weight mode {mode!r}")


def spectral_init(y: np.ndarray, v0: np.ndarray, fwd, adj, iters: int,
                  mode: str = "identity", lam: float = -1.0):
    """Leading eigenvector of M = A^H diag(T(y_hat)) A by shifted power iteration (Eq. 3-4).

    Returns x0 = sqrt(sum(y)) * v_T with ||v_T|| = 1.
    """
    y = np.asarray(y, dtype=np.float64)
    w = spectral_weights(y, mode, lam)
    shift = 0.0 if mode == "identity" else -2.0 * lam
    v = np.array(v0, dtype=np.complex128, copy=True)
    v = v / np.linalg.norm(v, axis=-1, keepdims=True)
    for _ in range(iters):
        u = adj(w * fwd(v)) + shift * v
        v = u / np.linalg.norm(u, axis=-1, keepdims=True)
    return np.sqrt(np.sum(y, axis=-1, keepdims=True)) * v


def spectral_init_early_stop(y: np.ndarray, v0: np.ndarray, fwd, adj, max_iters: int, rel_tol: float,
                             check_every: int, mode: str = "identity", lam: float = -1.0):
    """Power iteration of Eq. 3-4 with early stopping (Sec. IV-A runs it "with
    early stopping" without stating the rule). Reading: lambda_t = ||u_t||,
    u_t = M v_t + s v_t with unit v_t, estimates the top eigenvalue of M + s I;
    after every `check_every` steps stop once every problem has
    |lambda_{t-1} - lambda_t| <= rel_tol * lambda_{t-1} (t the chunk's last step).

    Returns (x0 = sqrt(sum y) v, [lambda_0 .. lambda_{run-1}], steps run).
    """
    if check_every < 2:
        raise ValueError("check_every must be >= 2")
    y = np.asarray(y, dtype=np.float64)
    w = spectral_weights(y, mode, lam)
    shift = 0.0 if mode == "identity" else -2.0 * lam
    v = np.array(v0, dtype=np.complex128, copy=True)
    v = v / np.linalg.norm(v, axis=-1, keepdims=True)
    lams = []
    run = max_iters
    for t in range(max_iters):
        u = adj(w * fwd(v)) + shift * v
        nrm = np.linalg.norm(u, axis=-1, keepdims=True)
        lams.append(nrm[..., 0])
        v = u / nrm
        if (t + 1) % check_every == 0 and t + 1 < max_iters:
            if np.all(np.abs(lams[t - 1] - lams[t]) <= rel_tol * lams[t - 1]):
                run = t + 1
                break
    return np.sqrt(np.sum(y, axis=-1, keepdims=True)) * v, np.array(lams), run


def cosine_similarity(xh: np.ndarray, x: np.ndarray) -> np.ndarray:
    """|<x_hat, x>| / (||x_hat|| ||x||), <a, b> = a^H b (Sec. IV-A, Eq. 6)."""
    inner = np.sum(np.conj(xh) * x, axis=-1)
    return np.abs(inner) / (np.linalg.norm(xh, axis=-1) * np.linalg.norm(x, axis=-1))


def relative_error_global_phase(xh: np.ndarray, x: np.ndarray) -> np.ndarray:
    """min over phi of ||exp(i phi) x_hat - x|| / ||x||.

    Expanding the norm, the minimum is attained where exp(-i phi) <x_hat, x>
    is real and positive, i.e. exp(i phi) = <x_hat, x> / |<x_hat, x>|; the
    distance is then evaluated directly (the expanded form
    sqrt(||x_hat||^2 + ||x||^2 - 2|<x_hat, x>|) loses half the digits to
    cancellation near zero).
    """
    inner = np.sum(np.conj(xh) * x, axis=-1, keepdims=True)
    mag = np.abs(inner)
    phase = np.where(mag > 0, inner / np.where(mag > 0, mag, 1.0), 1.0)
    return np.linalg.norm(phase * xh - x, axis=-1) / np.linalg.norm(x, axis=-1)
