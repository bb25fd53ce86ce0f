"""Pins of the FP64 oracle's DFT and structured operator (Sec. III, Eq. 5).

Each test checks the oracle against something other than itself: closed forms,
brute-force sums written from the definition, an explicitly formed dense
matrix, or invariants fixed by the mathematics.
"""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def _rand_c(rng, *shape):
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


# ---------------------------------------------------------------- DFT F

@pytest.mark.parametrize("m", [1, 2, 8, 48, 256])
def test_dft_matrix_unitary(m):
    F = O.dft_matrix(m)
    assert np.allclose(F.conj().T @ F, np.eye(m), atol=1e-12)


@pytest.mark.parametrize("m", [8, 64, 256])
def test_dft_of_delta_is_flat(m):
    # F e_0 = m^{-1/2} (1, ..., 1): closed form of the unitary DFT of a delta.
    d = np.zeros(m, complex)
    d[0] = 1
    for f in (O.dft_naive, O.unitary_fft):
        assert np.allclose(f(d), np.full(m, m ** -0.5), atol=1e-13)


@pytest.mark.parametrize("m,k0", [(16, 3), (256, 17), (96, 95)])
def test_dft_of_tone_is_scaled_delta(m, k0):
    # x_j = exp(+2 pi i k0 j / m) => F x = sqrt(m) e_{k0} with the exp(-2 pi i jk/m) sign.
    j = np.arange(m)
    tone = np.exp(2j * np.pi * k0 * j / m)
    expect = np.zeros(m, complex)
    expect[k0] = np.sqrt(m)
    for f in (O.dft_naive, O.unitary_fft):
        assert np.allclose(f(tone), expect, atol=1e-11)


@pytest.mark.parametrize("m", [12, 256, 1536])
def test_library_fft_matches_naive_dft(m):
    rng = np.random.default_rng(m)
    v = _rand_c(rng, 3, m)
    assert np.allclose(O.unitary_fft(v), O.dft_naive(v), atol=1e-10 * np.sqrt(m))
    assert np.allclose(O.unitary_ifft(O.unitary_fft(v)), v, atol=1e-12)


def test_parseval():
    rng = np.random.default_rng(1)
    v = _rand_c(rng, 1024)
    assert np.isclose(np.linalg.norm(O.unitary_fft(v)), np.linalg.norm(v), rtol=1e-13)


# ---------------------------------------------------------------- structured A

@pytest.mark.parametrize("n,m,L", [(8, 32, 1), (16, 64, 2), (12, 48, 3), (64, 256, 2), (5, 5, 2)])
def test_structured_matches_dense_materialised(n, m, L):
    theta = S.phases(7, L, m)
    A = O.dense_structured_matrix(theta, n, m)
    rng = np.random.default_rng(n + m)
    x = _rand_c(rng, 4, n)
    z = _rand_c(rng, 4, m)
    assert np.allclose(O.forward(x, theta, m), x @ A.T, atol=1e-11)
    assert np.allclose(O.adjoint(z, theta, n), z @ A.conj(), atol=1e-11)
    # the naive-DFT route through forward agrees too
    assert np.allclose(O.forward(x, theta, m, fft=O.dft_naive), x @ A.T, atol=1e-11)


@pytest.mark.parametrize("n,m", [(4, 16), (6, 12)])
def test_two_layer_column_brute_force(n, m):
    """A e_j for L=2 written as a double sum from the definition (D_1 first).

    [A e_j]_k = (1/m) exp(i theta1_j) sum_q exp(i theta2_q) exp(-2 pi i q (j + k)/m)
    -- fails if the diagonals are applied in the other order, if the DFT sign
    is flipped, if the normalisation is wrong, or if x is padded elsewhere.
    """
    theta = S.phases(3, 2, m)
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        col = O.forward(e, theta, m)
        for k in range(m):
            s = 0j
            for q in range(m):
                s += np.exp(1j * theta[1, q]) * np.exp(-2j * np.pi * q * (j + k) / m)
            expect = np.exp(1j * theta[0, j]) * s / m
            assert abs(col[k] - expect) < 1e-12


def test_one_layer_column_closed_form():
    # L=1: [A e_j]_k = m^{-1/2} exp(i theta_j) exp(-2 pi i j k / m).
    n, m = 8, 32
    theta = S.phases(11, 1, m)
    k = np.arange(m)
    for j in range(n):
        e = np.zeros(n, complex)
        e[j] = 1
        expect = np.exp(1j * theta[0, j]) * np.exp(-2j * np.pi * j * k / m) / np.sqrt(m)
        assert np.allclose(O.forward(e, theta, m), expect, atol=1e-13)


@pytest.mark.parametrize("n,m,L", [(16, 64, 2), (50, 200, 3), (7, 7, 1)])
def test_adjoint_identity(n, m, L):
    theta = S.phases(5, L, m)
    rng = np.random.default_rng(2)
    x = _rand_c(rng, n)
    z = _rand_c(rng, m)
    lhs = np.vdot(O.forward(x, theta, m), z)  # <Ax, z>
    rhs = np.vdot(x, O.adjoint(z, theta, n))  # <x, A^H z>
    assert abs(lhs - rhs) < 1e-11 * np.linalg.norm(x) * np.linalg.norm(z)


@pytest.mark.parametrize("n,m,L", [(16, 64, 2), (30, 90, 1), (32, 32, 4)])
def test_isometry(n, m, L):
    # The paper calls the structured matrix unitary (Sec. IV-A): A^H A = I_n for alpha >= 1.
    theta = S.phases(9, L, m)
    A = O.dense_structured_matrix(theta, n, m)
    assert np.allclose(A.conj().T @ A, np.eye(n), atol=1e-12)
    x = S.signal_gaussian(4, 2, n)
    y = np.abs(O.forward(x, theta, m)) ** 2
    assert np.allclose(y.sum(-1), (np.abs(x) ** 2).sum(-1), rtol=1e-12)


def test_zero_phase_one_layer_is_autocorrelation():
    """theta = 0, L = 1: y = |F U x|^2, whose inverse DFT is the circular
    autocorrelation of U x (Wiener-Khinchin); for alpha >= 2 it equals the
    linear autocorrelation, computed here by a direct double loop."""
    n, m = 10, 24
    x = S.signal_gaussian(1, 1, n)[0]
    y = np.abs(O.forward(x, np.zeros((1, m)), m)) ** 2
    # inverse *unnormalised* DFT of y / ... : sum_k y_k e^{2 pi i k s / m} / sqrt(m) * sqrt(m)
    k = np.arange(m)
    acf = np.array([np.sum(y * np.exp(2j * np.pi * k * s / m)) for s in range(m)])
    direct = np.zeros(m, complex)
    for s in range(m):
        for j in range(n):
            if 0 <= j - s < n:
                direct[s] += x[j] * np.conj(x[j - s])
            if 0 <= j - s + m < n:  # wrap-around term, zero when m >= 2n
                direct[s] += x[j] * np.conj(x[j - s + m])
    assert np.allclose(acf, direct, atol=1e-12)


def test_zero_phase_two_layers_is_time_reversal():
    # theta = 0, L = 2: F^2 is the index reversal v_k -> v_{-k mod m}.
    n, m = 6, 16
    x = S.signal_gaussian(2, 1, n)[0]
    z = O.forward(x, np.zeros((2, m)), m)
    v = O.zero_pad(x, m)
    assert np.allclose(z, v[(-np.arange(m)) % m], atol=1e-13)


def test_zero_pad_places_signal_first():
    x = np.arange(1, 4) + 0j
    assert np.array_equal(O.zero_pad(x, 6), np.array([1, 2, 3, 0, 0, 0], complex))
    with pytest.raises(ValueError):
        O.zero_pad(np.ones(5), 4)
