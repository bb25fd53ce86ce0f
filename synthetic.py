"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the benchmark.

This module holds no arithmetic of the phase-retrieval method: it only draws
random numbers. Everything random that the method consumes -- the diffuser
phases theta_l of the diagonals D_l (Sec. III, Eq. 5), the signals x (Sec. II-A),
the power-iteration start vector (Sec. II-B-2) and measurement noise -- comes
from one counter-based generator, Philox4x32-10 (Salmon, Moraes, Dror and Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written here from its
published definition. The CUDA library's plan implements the same generator
independently (in C) so that ``sr_plan_create(n, m, L, seed)`` produces
exactly the phases ``phases(seed, L, m)`` returns; a CPU test checks the two
bit for bit.

Counter convention (one Philox block per drawn element):
    ctr = (index mod 2^32, index div 2^32, sub, stream),  key = (seed mod 2^32, seed div 2^32)
Streams: 0 signal x, 1 phases theta, 2 start vector v0, 3 noise, 4 dense i.i.d. matrix,
5 phase-image ellipses.
A uniform draw is u = (word >> 8) * 2^-24, exact in float64, in [0, 1).
"""
from __future__ import annotations

import numpy as np

STREAM_SIGNAL = 0
STREAM_THETA = 1
STREAM_START = 2
STREAM_NOISE = 3
STREAM_DENSE = 4
STREAM_IMAGE = 5

# Philox4x32 constants as published: the two round multipliers and the two
# Weyl-sequence key increments (golden ratio and sqrt(3)-1 in 0.32 fixed point).
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint32(0x9E3779B9)
_W1 = np.uint32(0xBB67AE85)
_LO = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox4x32 rounds on uint32 counter words (arrays) under key (k0, k1).

    Each round multiplies words 0 and 2 by the round constants (64-bit product),
    and forms the new counter (hi1^c1^k0, lo1, hi0^c3^k1, lo0); the key is
    advanced by the Weyl increments between rounds.
    """
    c0 = np.asarray(c0, dtype=np.uint32)
    c1 = np.asarray(c1, dtype=np.uint32)
    c2 = np.asarray(c2, dtype=np.uint32)
    c3 = np.asarray(c3, dtype=np.uint32)
    k0 = np.uint32(k0)
    k1 = np.uint32(k1)
    with np.errstate(over="ignore"):
        for _ in range(10):
            p0 = _M0 * c0.astype(np.uint64)
            p1 = _M1 * c2.astype(np.uint64)
            hi0 = (p0 >> _S32).astype(np.uint32)
            lo0 = (p0 & _LO).astype(np.uint32)
            hi1 = (p1 >> _S32).astype(np.uint32)
            lo1 = (p1 & _LO).astype(np.uint32)
            c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
            k0 = np.uint32(k0 + _W0)
            k1 = np.uint32(k1 + _W1)
    return c0, c1, c2, c3


def _blocks(seed: int, count: int, sub: int, stream: int):
    """Philox output words for element indices 0..count-1 of (sub, stream)."""
    idx = np.arange(count, dtype=np.uint64)
    lo = (idx & _LO).astype(np.uint32)
    hi = (idx >> _S32).astype(np.uint32)
    sub_w = np.full(count, sub, dtype=np.uint32)
    st_w = np.full(count, stream, dtype=np.uint32)
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    return philox4x32_10(lo, hi, sub_w, st_w, seed & 0xFFFFFFFF, seed >> 32)


def uniform_from_word(w) -> np.ndarray:
    """u = (w >> 8) * 2^-24 in [0, 1), exact in float64."""
    return (np.asarray(w, dtype=np.uint32) >> np.uint32(8)).astype(np.float64) * 2.0 ** -24


def phases(seed: int, L: int, m: int) -> np.ndarray:
    """Diffuser phases theta[l, k] = 2*pi*u, u ~ U[0, 1): float64 [L, m] (Sec. III, Eq. 5)."""
    out = np.empty((L, m), dtype=np.float64)
    for l in range(L):
        w0, _, _, _ = _blocks(seed, m, l, STREAM_THETA)
        out[l] = 2.0 * np.pi * uniform_from_word(w0)
    return out


def complex_gaussian(seed: int, shape, stream: int, sub: int = 0, var: float = 1.0) -> np.ndarray:
    """CN(0, var) draws by Box-Muller on words 0 and 1 of each block: complex128."""
    count = int(np.prod(shape))
    w0, w1, _, _ = _blocks(seed, count, sub, stream)
    u1 = ((np.asarray(w0) >> np.uint32(8)).astype(np.float64) + 1.0) * 2.0 ** -24  # (0, 1]
    u2 = uniform_from_word(w1)
    rad = np.sqrt(-np.log(u1) * var)  # |g|^2 ~ Exp(var): E|g|^2 = var
    g = rad * np.exp(2j * np.pi * u2)
    return g.reshape(shape)


def uniform(seed: int, shape, stream: int, sub: int = 0, word: int = 0) -> np.ndarray:
    count = int(np.prod(shape))
    words = _blocks(seed, count, sub, stream)
    return uniform_from_word(words[word]).reshape(shape)


def signal_gaussian(seed: int, B: int, n: int) -> np.ndarray:
    """Signals x ~ CN(0, I_n), shape [B, n] (complex Gaussian test signals)."""
    return complex_gaussian(seed, (B, n), STREAM_SIGNAL)


def signal_amplitude_phase(seed: int, B: int, n: int) -> np.ndarray:
    """Image-like signals x_k = a_k exp(i phi_k), a ~ U[0, 1], phi ~ U[0, 2*pi): [B, n]."""
    count = B * n
    w0, w1, _, _ = _blocks(seed, count, 0, STREAM_SIGNAL)
    a = uniform_from_word(w0)
    phi = 2.0 * np.pi * uniform_from_word(w1)
    return (a * np.exp(1j * phi)).reshape(B, n)


def phase_image_ellipses(seed: int, B: int, h: int, w: int, count: int = 10) -> np.ndarray:
    """Phantom-like phase images, [B, h*w] row-major, unit magnitude.

    Stands in for the paper's benchmark image (Sec. IV-A: a Shepp-Logan phantom
    whose grey levels in [0, 1) become phases in [-pi/2, pi/2)): each image sums
    `count` random filled ellipses (centre, semi-axes, rotation and grey-level
    increment drawn from Philox stream 5, sub-stream = image index), clips the
    grey level to [0, 1) and maps it linearly to a phase phi in [-pi/2, pi/2),
    x = exp(i phi).
    """
    yy, xx = np.meshgrid((np.arange(h) + 0.5) / h * 2.0 - 1.0, (np.arange(w) + 0.5) / w * 2.0 - 1.0,
                         indexing="ij")
    out = np.empty((B, h * w), dtype=np.complex128)
    for b in range(B):
        w0, w1, w2, w3 = _blocks(seed, 2 * count, b, STREAM_IMAGE)
        u = np.stack([uniform_from_word(w0), uniform_from_word(w1), uniform_from_word(w2),
                      uniform_from_word(w3)])  # [4, 2 * count]
        grey = np.zeros((h, w))
        for e in range(count):
            cy, cx = 1.2 * u[0, e] - 0.6, 1.2 * u[1, e] - 0.6
            ay, ax = 0.1 + 0.6 * u[2, e], 0.1 + 0.6 * u[3, e]
            rot = np.pi * u[0, count + e]
            inc = 0.1 + 0.4 * u[1, count + e]
            cs, sn = np.cos(rot), np.sin(rot)
            dy, dx = yy - cy, xx - cx
            py, px = cs * dy + sn * dx, -sn * dy + cs * dx
            grey += inc * ((py / ay) ** 2 + (px / ax) ** 2 <= 1.0)
        grey = np.clip(grey, 0.0, np.nextafter(1.0, 0.0))
        out[b] = np.exp(1j * np.pi * (grey - 0.5)).reshape(-1)
    return out


def start_vector(seed: int, B: int, n: int) -> np.ndarray:
    """Random power-iteration start v0 ~ CN(0, I_n), shape [B, n] (Sec. II-B-2)."""
    return complex_gaussian(seed, (B, n), STREAM_START)


def dense_iid_matrix(seed: int, m: int, n: int) -> np.ndarray:
    """Dense i.i.d. sensing matrix with entries CN(0, 1/m), shape [m, n] (Sec. II-A)."""
    return complex_gaussian(seed, (m, n), STREAM_DENSE, var=1.0 / m)


def round_to_bf16(a: np.ndarray) -> np.ndarray:
    """Nearest-even rounding of float values to the BF16 grid (8-bit significand),
    returned as float64. Used to define a dense matrix whose entries are exactly
    representable in BF16 (the stored form of the dense comparison model)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    bias = ((u >> np.uint32(16)) & np.uint32(1)) + np.uint32(0x7FFF)
    with np.errstate(over="ignore"):
        r = (u + bias) & np.uint32(0xFFFF0000)
    return r.view(np.float32).astype(np.float64)


def dense_iid_matrix_bf16(seed: int, m: int, n: int) -> np.ndarray:
    """CN(0, 1/m) dense matrix with real and imaginary parts on the BF16 grid: [m, n]."""
    A = dense_iid_matrix(seed, m, n)
    return round_to_bf16(A.real) + 1j * round_to_bf16(A.imag)


def round_to_tf32(a: np.ndarray) -> np.ndarray:
    """Rounding of float values to the TF32 grid (11-bit significand: 10
    fraction bits) to nearest with ties away from zero, returned as float64.
    Defines a dense matrix whose entries are exactly representable in TF32
    (the stored form of the TF32 dense comparison model)."""
    u = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    with np.errstate(over="ignore"):
        r = (u + np.uint32(0x1000)) & np.uint32(0xFFFFE000)
    return r.view(np.float32).astype(np.float64)


def dense_iid_matrix_tf32(seed: int, m: int, n: int) -> np.ndarray:
    """CN(0, 1/m) dense matrix with real and imaginary parts on the TF32 grid: [m, n]."""
    A = dense_iid_matrix(seed, m, n)
    return round_to_tf32(A.real) + 1j * round_to_tf32(A.imag)


def gaussian_noise(seed: int, shape, sigma) -> np.ndarray:
    """Real N(0, sigma^2) noise via Box-Muller (real part of a CN(0, 2) draw)."""
    g = complex_gaussian(seed, shape, STREAM_NOISE, var=2.0)
    return np.asarray(sigma)[..., None] * g.real if np.ndim(sigma) else sigma * g.real


def poisson_counts(seed: int, lam: np.ndarray) -> np.ndarray:
    """Poisson(lam) draws (elementwise), by inversion of the CDF on a Philox uniform.

    Inversion walks the CDF from k = 0; for large means it starts at the mode
    region via a normal approximation guard so that the walk stays short.
    """
    lam = np.asarray(lam, dtype=np.float64)
    flat = lam.reshape(-1)
    u = uniform(seed, flat.shape, STREAM_NOISE, sub=1)
    out = np.empty(flat.shape, dtype=np.float64)
    for i, (mu, ui) in enumerate(zip(flat, u)):
        if mu <= 0.0:
            out[i] = 0.0
            continue
        # Walk up from k=0 in log space to stay stable for moderate means.
        k = 0
        logp = -mu
        cdf = np.exp(logp)
        while cdf < ui and k < 100000:
            k += 1
            logp += np.log(mu) - np.log(k)
            cdf += np.exp(logp)
        out[i] = k
    return out.reshape(lam.shape)
