"""Pins of the oracle's backward pass (gradients with respect to x and the
diffuser phases theta_l) by central finite differences on a real loss, and by
the adjoint special case G_x = A^H G_z."""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def _loss_and_gz(z, c, w):
    """L = Re(c^H z) + sum w |z|^2 and its complex gradient G_z = c + 2 w z."""
    loss = np.real(np.sum(np.conj(c) * z)) + np.sum(w * np.abs(z) ** 2)
    return loss, c + 2 * w * z


@pytest.mark.parametrize("n,m,L,B", [(6, 16, 2, 2), (5, 12, 1, 1), (8, 32, 3, 2)])
def test_theta_gradient_matches_central_differences(n, m, L, B):
    theta = S.phases(3, L, m)
    x = S.signal_gaussian(4, B, n)
    c = S.complex_gaussian(5, (B, m), S.STREAM_NOISE)
    w = np.abs(S.complex_gaussian(6, (B, m), S.STREAM_NOISE))
    z = O.forward(x, theta, m)
    _, gz = _loss_and_gz(z, c, w)
    gx, gth = O.autodiff.backward(x, gz, theta, n, m)
    h = 1e-6
    for l in range(L):
        for k in range(0, m, max(1, m // 6)):
            tp = theta.copy(); tp[l, k] += h
            tm = theta.copy(); tm[l, k] -= h
            fd = (_loss_and_gz(O.forward(x, tp, m), c, w)[0] - _loss_and_gz(O.forward(x, tm, m), c, w)[0]) / (2 * h)
            assert np.isclose(gth[l, k], fd, rtol=1e-6, atol=1e-7)
    # x-gradient in the same convention: dL/dRe x + i dL/dIm x
    for b in range(B):
        for k in range(n):
            for d, part in ((1.0, np.real), (1j, np.imag)):
                xp = x.copy(); xp[b, k] += h * d
                xm = x.copy(); xm[b, k] -= h * d
                fd = (_loss_and_gz(O.forward(xp, theta, m), c, w)[0] -
                      _loss_and_gz(O.forward(xm, theta, m), c, w)[0]) / (2 * h)
                assert np.isclose(part(gx[b, k]), fd, rtol=1e-6, atol=1e-7)


def test_x_gradient_is_the_adjoint():
    n, m, L = 20, 64, 2
    theta = S.phases(8, L, m)
    x = S.signal_gaussian(1, 3, n)
    gz = S.complex_gaussian(2, (3, m), S.STREAM_NOISE)
    gx, _ = O.autodiff.backward(x, gz, theta, n, m)
    assert np.allclose(gx, O.adjoint(gz, theta, n), atol=1e-12)


def test_theta_gradient_vanishes_for_phase_blind_loss_of_one_layer():
    # L = 1, loss = sum |z|^2 = ||x||^2 does not depend on theta (A is an isometry)
    n, m = 7, 28
    theta = S.phases(9, 1, m)
    x = S.signal_gaussian(3, 2, n)
    z = O.forward(x, theta, m)
    _, gth = O.autodiff.backward(x, 2 * z, theta, n, m)
    assert np.max(np.abs(gth)) < 1e-12
