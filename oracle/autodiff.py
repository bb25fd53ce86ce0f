"""Backward pass of z = A x with respect to x and the diffuser phases (FP64).

Test infrastructure only (see the package docstring).

A = F D_L ... F D_1 U (Sec. III, Eq. 5) with D_l = diag(exp(i theta_l)); the
phases theta_l are the real parameters of the model (Sec. III) and are
differentiated here as the differentiable operator (autograd) of the library does.

Gradient convention (the one of PyTorch for complex tensors): for a real loss
L, the gradient of a complex variable w is G_w = dL/dRe(w) + i dL/dIm(w)
= 2 dL/d conj(w). Then for the linear map z = A x, G_x = A^H G_z. Writing
q_1 = U x, p_l = D_l q_l, q_{l+1} = F p_l (so z = q_{L+1}), and h_l = G_{p_l},
the chain rule gives h_L = F^H G_z, h_{l-1} = F^H D_l^H h_l, G_x = U^H D_1^H h_1,
and, since dp_l/dtheta_l = i p_l elementwise,
    dL/dtheta_l[k] = Re(conj(G_{p_l}[k]) * i p_l[k]) = Im(conj(p_l[k]) h_l[k]),
summed over the batch (the phases are shared by all problems).
"""
from __future__ import annotations

import numpy as np

from .operator import unitary_fft, unitary_ifft, zero_pad


def backward(x: np.ndarray, gz: np.ndarray, theta: np.ndarray, n: int, m: int):
    """(G_x [B, n], dL/dtheta [L, m]) for z = A x given G_z [B, m]."""
    x = np.atleast_2d(np.asarray(x, dtype=np.complex128))
    gz = np.atleast_2d(np.asarray(gz, dtype=np.complex128))
    L = theta.shape[0]
    # forward, keeping p_l = D_l q_l
    q = zero_pad(x, m)
    p = []
    for l in range(L):
        pl = np.exp(1j * theta[l]) * q
        p.append(pl)
        q = unitary_fft(pl)
    # backward
    h = unitary_ifft(gz)  # h_L = F^H G_z
    gtheta = np.zeros((L, m))
    for l in reversed(range(L)):
        gtheta[l] = np.sum(np.imag(np.conj(p[l]) * h), axis=0)
        g_q = np.exp(-1j * theta[l]) * h  # G_{q_l} = D_l^H h_l
        if l > 0:
            h = unitary_ifft(g_q)  # h_{l-1} = F^H G_{q_l}
    gx = g_q[:, :n].copy()  # U^H
    return gx, gtheta
