"""Two-dimensional structured random operator A = F2 D_L ... F2 D_1 U2 (FP64).

Test infrastructure only (see the package docstring).

The experiments of Sec. IV run the model on images with a 2D FFT (Sec. IV,
implementation paragraph): the signal is an h x w image, oversampling zero-pads
it to an S x S grid (Sec. III, the paragraph after Eq. 5), and every F of Eq. 5
is the unitary 2D DFT of that grid.

Readings used here (the paper does not fix them):
* Vectors are the row-major flattening of the image: pixel (r, c) of the h x w
  signal is x[r*w + c], entry (r, c) of the S x S grid is v[r*S + c].
* U2 places the image in the top-left corner (rows 0..h-1, columns 0..w-1), the
  2D form of the 1D reading (x in entries 0..n-1); U2^H keeps that corner.
* F2[(a, b), (r, c)] = S^{-1} exp(-2*pi*i*(r*a + c*b)/S), the unitary 2D DFT.
* D_l = diag(exp(i*theta_l)) with theta_l indexed like the grid (row-major).
"""
from __future__ import annotations

import numpy as np


def unitary_fft2(v: np.ndarray, S: int) -> np.ndarray:
    """Unitary 2D DFT of row-major S x S grids along the last axis (library FFT as a step)."""
    g = np.asarray(v, dtype=np.complex128).reshape(v.shape[:-1] + (S, S))
    return np.fft.fft2(g, norm="ortho").reshape(v.shape[:-1] + (S * S,))


def unitary_ifft2(v: np.ndarray, S: int) -> np.ndarray:
    """Inverse unitary 2D DFT F2^H of row-major S x S grids."""
    g = np.asarray(v, dtype=np.complex128).reshape(v.shape[:-1] + (S, S))
    return np.fft.ifft2(g, norm="ortho").reshape(v.shape[:-1] + (S * S,))


def zero_pad_2d(x: np.ndarray, h: int, w: int, S: int) -> np.ndarray:
    """U2: h x w image (row-major, [..., h*w]) into the top-left of an S x S grid."""
    if h > S or w > S:
        raise ValueError("zero padding needs h, w <= S")
    x = np.asarray(x, dtype=np.complex128)
    out = np.zeros(x.shape[:-1] + (S, S), dtype=np.complex128)
    out[..., :h, :w] = x.reshape(x.shape[:-1] + (h, w))
    return out.reshape(x.shape[:-1] + (S * S,))


def crop_2d(v: np.ndarray, h: int, w: int, S: int) -> np.ndarray:
    """U2^H: the top-left h x w corner of S x S grids, row-major [..., h*w]."""
    g = np.asarray(v).reshape(v.shape[:-1] + (S, S))
    return g[..., :h, :w].reshape(v.shape[:-1] + (h * w,)).copy()


def forward_2d(x: np.ndarray, theta: np.ndarray, h: int, w: int, S: int) -> np.ndarray:
    """z = A x with A = F2 D_L ... F2 D_1 U2 (Eq. 5 with the 2D DFT of Sec. IV).

    x: [..., h*w]; theta: [L, S*S]; returns [..., S*S] (row-major grid).
    """
    v = zero_pad_2d(x, h, w, S)
    for l in range(theta.shape[0]):
        v = unitary_fft2(np.exp(1j * theta[l]) * v, S)
    return v


def adjoint_2d(z: np.ndarray, theta: np.ndarray, h: int, w: int, S: int) -> np.ndarray:
    """A^H z = U2^H D_1^H F2^H ... D_L^H F2^H z; returns [..., h*w]."""
    v = np.asarray(z, dtype=np.complex128)
    for l in reversed(range(theta.shape[0])):
        v = np.exp(-1j * theta[l]) * unitary_ifft2(v, S)
    return crop_2d(v, h, w, S)


def dense_structured_matrix_2d(theta: np.ndarray, h: int, w: int, S: int) -> np.ndarray:
    """Explicit (S*S) x (h*w) matrix of the 2D model (tiny sizes).

    F2 is formed entry by entry from its definition, U2 from the index rule
    (r*w + c) -> (r*S + c); no FFT is involved.
    """
    r = np.arange(S)
    a = r[:, None, None, None]
    b = r[None, :, None, None]
    rr = r[None, None, :, None]
    cc = r[None, None, None, :]
    ph = (rr * a + cc * b) % S  # exact integer phase index
    F2 = (np.exp(-2j * np.pi * ph / S) / S).reshape(S * S, S * S)
    U2 = np.zeros((S * S, h * w), dtype=np.complex128)
    for i in range(h):
        for j in range(w):
            U2[i * S + j, i * w + j] = 1.0
    A = U2
    for l in range(theta.shape[0]):
        A = F2 @ (np.diag(np.exp(1j * theta[l])) @ A)
    return A


def structured_ops_2d(theta: np.ndarray, h: int, w: int, S: int):
    """(fwd, adj) callables of the 2D model, for the recovery routines."""
    return (lambda x: forward_2d(x, theta, h, w, S)), (lambda z: adjoint_2d(z, theta, h, w, S))
