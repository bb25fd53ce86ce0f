"""Structured random sensing operator A = F D_L ... F D_1 U and its adjoint (FP64).

Test infrastructure only (see the package docstring).

Readings of the paper used here (Sec. III, Eq. 5, alpha > 1 branch):
* D_1 acts first: A = F D_L ... F D_1 U, matching the optical order of Fig. 1
  (diffuser, lens, diffuser, lens).
* F is the unitary DFT, F[k, j] = m^{-1/2} exp(-2*pi*i*j*k/m); the paper calls
  the structured matrix unitary (Sec. IV-A), which fixes the 1/sqrt(m).
* D_l = diag(exp(i*theta_l)), theta_l ~ U[0, 2*pi) (Sec. III).
* U zero-pads x in C^n to C^m by placing x in entries 0..n-1.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(m: int) -> np.ndarray:
    """Naive unitary DFT matrix F[k, j] = m^{-1/2} exp(-2*pi*i*j*k/m) (Sec. III, Eq. 5)."""
    jk = np.outer(np.arange(m), np.arange(m)) % m  # exact integer phase index
    return np.exp(-2j * np.pi * jk / m) / np.sqrt(m)


def dft_naive(v: np.ndarray) -> np.ndarray:
    """Unitary DFT along the last axis by the O(m^2) matrix product."""
    m = v.shape[-1]
    return v @ dft_matrix(m).T


def unitary_fft(v: np.ndarray) -> np.ndarray:
    """Unitary DFT along the last axis (library FFT as one step, O(m log m))."""
    return np.fft.fft(v, axis=-1, norm="ortho")


def unitary_ifft(v: np.ndarray) -> np.ndarray:
    """Inverse unitary DFT F^H along the last axis."""
    return np.fft.ifft(v, axis=-1, norm="ortho")


def zero_pad(x: np.ndarray, m: int) -> np.ndarray:
    """U: C^n -> C^m, x placed in entries 0..n-1, zeros after (Sec. III)."""
    n = x.shape[-1]
    if n > m:
        raise ValueError("zero padding needs n <= m")
    out = np.zeros(x.shape[:-1] + (m,), dtype=np.complex128)
    out[..., :n] = x
    return out


def forward(x: np.ndarray, theta: np.ndarray, m: int, fft=unitary_fft) -> np.ndarray:
    """z = A x with A = F D_L ... F D_1 U (Sec. III, Eq. 5, alpha > 1).

    x: [..., n] complex; theta: [L, m] phases of the diagonals; returns [..., m].
    """
    v = zero_pad(np.asarray(x, dtype=np.complex128), m)
    for l in range(theta.shape[0]):
        v = fft(np.exp(1j * theta[l]) * v)
    return v


def adjoint(z: np.ndarray, theta: np.ndarray, n: int, ifft=unitary_ifft) -> np.ndarray:
    """A^H z = U^H D_1^H F^H ... D_L^H F^H z (conjugate transpose of Eq. 5).

    z: [..., m]; returns the first n entries, [..., n].
    """
    v = np.asarray(z, dtype=np.complex128)
    for l in reversed(range(theta.shape[0])):
        v = np.exp(-1j * theta[l]) * ifft(v)
    return v[..., :n].copy()


def dense_structured_matrix(theta: np.ndarray, n: int, m: int) -> np.ndarray:
    """Explicit m x n matrix of A, formed as the product of its factors (tiny sizes).

    Built from the naive DFT matrix and explicit diagonal matrices only, so it
    shares no code path with ``forward`` beyond the definition itself.
    """
    F = dft_matrix(m)
    U = np.eye(m, n, dtype=np.complex128)
    A = U
    for l in range(theta.shape[0]):
        A = F @ (np.diag(np.exp(1j * theta[l])) @ A)
    return A
