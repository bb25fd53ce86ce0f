"""Structured random sensing operator A = F D_L ... F D_1 U and its adjoint (FP64).

Test infrastructure only (see the package docstring).

Readings of the paper used here (Sec. III, Eq. 5, alpha > 1 branch):
* D_1 acts first: A = F D_L ... F D_1 U, matching the optical order of Fig. 1
  (diffuser, lens, diffuser, lens).
* F is the unitary DFT, F[k, j] = m^{-1/2} exp(-2*pi*i*j*k/m); the paper calls
  the structured matrix unitary (Sec. IV-A), which fixes the 1/sqrt(m).
* D_l = diag(exp(i*theta_l)), theta_l ~ U[0, 2*pi) (Sec. III).
* U zero-pads x in C^n to C^m by placing x in entries 0..n-1.
* alpha < 1 (m < n, Sec. III, the undersampling paragraph after Eq. 5): the
  DFTs have length n (no padding) and S "trims the edges" of the result,
  read as keeping the m central entries off .. off+m-1 with
  off = floor((n - m) / 2); theta then has shape [L, n].
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


def trim_offset(n: int, m: int) -> int:
    """First kept entry of S: the m central entries of a length-n vector."""
    return (n - m) // 2


def trim(v: np.ndarray, m: int) -> np.ndarray:
    """S: C^n -> C^m, keeps entries off .. off+m-1 (Sec. III, alpha < 1)."""
    off = trim_offset(v.shape[-1], m)
    return v[..., off:off + m].copy()


def untrim(w: np.ndarray, n: int) -> np.ndarray:
    """S^H: C^m -> C^n, w placed at entries off .. off+m-1, zeros elsewhere."""
    m = w.shape[-1]
    off = trim_offset(n, m)
    out = np.zeros(w.shape[:-1] + (n,), dtype=np.complex128)
    out[..., off:off + m] = w
    return out


def forward(x: np.ndarray, theta: np.ndarray, m: int, fft=unitary_fft) -> np.ndarray:
    """z = A x with A = F D_L ... F D_1 U (Sec. III, Eq. 5, alpha >= 1), or
    A = S F D_L ... F D_1 when m < n (alpha < 1).

    x: [..., n] complex; theta: [L, max(n, m)] phases of the diagonals; returns [..., m].
    """
    x = np.asarray(x, dtype=np.complex128)
    n = x.shape[-1]
    v = zero_pad(x, m) if m >= n else x
    for l in range(theta.shape[0]):
        v = fft(np.exp(1j * theta[l]) * v)
    return v if m >= n else trim(v, m)


def adjoint(z: np.ndarray, theta: np.ndarray, n: int, ifft=unitary_ifft) -> np.ndarray:
    """A^H z = U^H D_1^H F^H ... D_L^H F^H z (conjugate transpose of Eq. 5), or
    D_1^H F^H ... D_L^H F^H S^H z when m < n.

    z: [..., m]; returns [..., n].
    """
    v = np.asarray(z, dtype=np.complex128)
    m = v.shape[-1]
    if m < n:
        v = untrim(v, n)
    for l in reversed(range(theta.shape[0])):
        v = np.exp(-1j * theta[l]) * ifft(v)
    return v[..., :n].copy()


def dense_structured_matrix(theta: np.ndarray, n: int, m: int) -> np.ndarray:
    """Explicit m x n matrix of A, formed as the product of its factors (tiny sizes).

    Built from the naive DFT matrix and explicit diagonal matrices only, so it
    shares no code path with ``forward`` beyond the definition itself.
    """
    N = max(n, m)
    F = dft_matrix(N)
    A = np.eye(N, n, dtype=np.complex128)  # U (the identity when m < n)
    for l in range(theta.shape[0]):
        A = F @ (np.diag(np.exp(1j * theta[l])) @ A)
    if m < n:  # S: rows off .. off+m-1
        off = (n - m) // 2
        Sm = np.zeros((m, n), dtype=np.complex128)
        for i in range(m):
            Sm[i, off + i] = 1.0
        A = Sm @ A
    return A
