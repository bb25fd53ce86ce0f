"""Pins of the dense i.i.d. comparison model (Sec. II-A) and of the seeded inputs."""
import numpy as np

import oracle as O
import synthetic as S


def test_dense_ops_are_triple_loops():
    m, n = 7, 4
    A = S.dense_iid_matrix(3, m, n)
    x = S.signal_gaussian(3, 2, n)
    w = S.complex_gaussian(4, (2, m), S.STREAM_NOISE)
    z = O.dense_forward(A, x)
    g = O.dense_adjoint(A, w)
    for b in range(2):
        for i in range(m):
            assert abs(z[b, i] - sum(A[i, k] * x[b, k] for k in range(n))) < 1e-13
        for k in range(n):
            assert abs(g[b, k] - sum(np.conj(A[i, k]) * w[b, i] for i in range(m))) < 1e-13


def test_dense_iid_entry_statistics():
    m, n = 512, 256
    A = S.dense_iid_matrix(11, m, n)
    p = np.abs(A) ** 2
    assert abs(p.mean() * m - 1.0) < 0.01  # E|A_ik|^2 = 1/m
    assert abs(np.mean(A.real) * np.sqrt(m)) < 0.01
    assert abs(np.mean(A.real * A.imag) * m) < 0.01
    # |A_ik|^2 * m ~ Exp(1): variance 1
    assert abs(np.var(p * m) - 1.0) < 0.03


def test_philox_streams_are_deterministic_and_distinct():
    a = S.phases(123, 2, 1000)
    b = S.phases(123, 2, 1000)
    c = S.phases(124, 2, 1000)
    assert np.array_equal(a, b)
    assert not np.any(a == c)
    assert not np.any(a[0] == a[1])
    assert a.min() >= 0 and a.max() < 2 * np.pi


def test_uniform_draws_are_uniform():
    u = S.uniform(5, (200000,), S.STREAM_THETA)
    hist, _ = np.histogram(u, bins=50, range=(0, 1))
    expected = len(u) / 50
    chi2 = np.sum((hist - expected) ** 2 / expected)
    assert chi2 < 100  # 49 dof: mean 49, sd ~ 10
    assert abs(u.mean() - 0.5) < 0.003 and abs(u.var() - 1 / 12) < 0.002


def test_philox_counter_words_feed_every_output_bit():
    # Flipping one counter bit changes about half the output bits (avalanche).
    base = S.philox4x32_10([0], [0], [0], [0], 1, 2)
    flips = []
    for word in range(4):
        for bit in (0, 13, 31):
            c = [[0], [0], [0], [0]]
            c[word] = [1 << bit]
            out = S.philox4x32_10(*c, 1, 2)
            flips.append(sum(bin(int(o[0]) ^ int(b[0])).count("1") for o, b in zip(out, base)))
    assert 40 < np.mean(flips) < 88


def test_signal_generators_shapes_and_moments():
    x = S.signal_gaussian(1, 4, 5000)
    assert x.shape == (4, 5000) and abs(np.mean(np.abs(x) ** 2) - 1) < 0.03
    xa = S.signal_amplitude_phase(1, 2, 5000)
    a = np.abs(xa)
    assert a.max() <= 1 and abs(a.mean() - 0.5) < 0.02
    lam = np.full(4000, 100.0)
    k = S.poisson_counts(2, lam)
    assert abs(k.mean() - 100) < 1.0 and abs(k.var() - 100) < 10


def test_round_to_bf16_grid():
    # exactly representable values are kept; others go to the nearest 8-bit significand, ties to even
    vals = np.array([1.0, -2.5, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -8, 1.0 + 2 ** -9, 3.0e-3], dtype=np.float64)
    r = S.round_to_bf16(vals)
    assert r[0] == 1.0 and r[1] == -2.5
    assert r[2] == 1.0          # halfway between 1 and 1 + 2^-7: ties to even (1.0)
    assert r[3] == 1.0 + 2 ** -6  # halfway between 1 + 2^-7 and 1 + 2^-6: to even (1 + 2^-6)
    assert r[4] == 1.0
    m, e = np.frexp(r[5])
    assert np.isclose(r[5], 3.0e-3, rtol=2 ** -8) and (m * 2 ** 8) == np.round(m * 2 ** 8)
    A = S.dense_iid_matrix_bf16(1, 64, 32)
    assert np.array_equal(S.round_to_bf16(A.real), A.real)


def test_round_to_tf32_grid():
    # exactly representable values are kept; others go to the nearest 11-bit significand
    # (10 fraction bits), ties away from zero
    vals = np.array([1.0, -2.5, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, -(1.0 + 2 ** -11), 1.0 + 2 ** -12, 3.0e-3])
    r = S.round_to_tf32(vals)
    assert r[0] == 1.0 and r[1] == -2.5
    assert r[2] == 1.0 + 2 ** -10      # halfway between 1 and 1 + 2^-10: away from zero
    assert r[3] == 1.0 + 2 ** -9       # halfway between 1 + 2^-10 and 1 + 2^-9: away from zero
    assert r[4] == -(1.0 + 2 ** -10)   # negative ties move away from zero too
    assert r[5] == 1.0
    m, e = np.frexp(r[6])
    assert np.isclose(r[6], 3.0e-3, rtol=2 ** -11) and (m * 2 ** 11) == np.round(m * 2 ** 11)
    A = S.dense_iid_matrix_tf32(1, 64, 32)
    assert np.array_equal(S.round_to_tf32(A.imag), A.imag)
    assert np.max(np.abs(A - S.dense_iid_matrix(1, 64, 32))) <= 2 ** -11 * np.max(np.abs(A))
