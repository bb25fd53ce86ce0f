"""Pins of the oracle's alpha < 1 branch, A = S F D_L ... F D_1 with S keeping
the m central entries of the length-n result (Sec. III, the undersampling
paragraph after Eq. 5), against an explicit matrix built entry by entry, a
closed-form tone, the m = n special case and invariants. None of them calls
the oracle's forward to check itself.

A plausible mistake (window off by one or at the start, padding instead of
trimming, S^H placing w wrongly, D after F, theta of length m) fails one of these."""
import numpy as np
import pytest

import oracle as O
import synthetic as S


def test_trim_window_rule():
    for n, m in ((8, 5), (8, 6), (9, 4), (16, 16), (7, 1)):
        off = (n - m) // 2
        assert O.trim_offset(n, m) == off
        v = np.arange(n) + 1.0
        assert np.array_equal(O.trim(v, m), v[off:off + m])
        w = np.arange(m) + 1.0
        u = O.untrim(w, n)
        assert np.array_equal(u[off:off + m], w)
        assert np.count_nonzero(u) == m


@pytest.mark.parametrize("n,m,L", [(8, 5, 1), (16, 7, 2), (12, 12, 2), (16, 1, 3), (12, 9, 1)])
def test_forward_adjoint_match_explicit_matrix(n, m, L):
    th = S.phases(3 + n + m, L, n)
    # explicit S F D_L ... F D_1 from the DFT definition, entry by entry
    jk = np.outer(np.arange(n), np.arange(n))
    F = np.exp(-2j * np.pi * (jk % n) / n) / np.sqrt(n)
    A = np.eye(n, dtype=np.complex128)
    for l in range(L):
        A = F @ (np.exp(1j * th[l])[:, None] * A)
    off = (n - m) // 2
    A = A[off:off + m]
    assert np.allclose(O.dense_structured_matrix(th, n, m), A, atol=1e-12)
    x = S.complex_gaussian(1, (3, n), S.STREAM_SIGNAL)
    w = S.complex_gaussian(2, (3, m), S.STREAM_NOISE)
    assert np.allclose(O.forward(x, th, m), x @ A.T, atol=1e-12)
    assert np.allclose(O.adjoint(w, th, n), w @ A.conj(), atol=1e-12)


@pytest.mark.parametrize("k0", [0, 3, 5, 7, 12, 15])
def test_tone_lands_in_or_out_of_the_window(k0):
    """L = 1, theta = 0: the unitary DFT of exp(2 pi i k0 j / n) is sqrt(n) at
    k0; S keeps it at position k0 - off when off <= k0 < off + m, else z = 0."""
    n, m = 16, 6
    off = (n - m) // 2  # 5
    x = np.exp(2j * np.pi * k0 * np.arange(n) / n)
    z = O.forward(x, np.zeros((1, n)), m)
    want = np.zeros(m, dtype=np.complex128)
    if off <= k0 < off + m:
        want[k0 - off] = np.sqrt(n)
    assert np.allclose(z, want, atol=1e-12)


def test_m_equals_n_is_the_plain_model():
    n, L = 16, 2
    th = S.phases(5, L, n)
    x = S.complex_gaussian(4, (2, n), S.STREAM_SIGNAL)
    v = x.copy()
    for l in range(L):
        v = O.dft_naive(np.exp(1j * th[l]) * v)
    assert np.allclose(O.forward(x, th, n), v, atol=1e-12)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_rows_are_orthonormal(L):
    """A A^H = S S^H = I_m: F D_l is unitary and S keeps m distinct entries."""
    n, m = 32, 11
    th = S.phases(7, L, n)
    w = S.complex_gaussian(8, (3, m), S.STREAM_NOISE)
    assert np.allclose(O.forward(O.adjoint(w, th, n), th, m), w, atol=1e-12)
    x = S.complex_gaussian(9, (3, n), S.STREAM_SIGNAL)
    lhs = np.sum(O.forward(x, th, m) * w.conj(), axis=1)
    rhs = np.sum(x * O.adjoint(w, th, n).conj(), axis=1)
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_gradient_by_finite_differences_alpha_below_one():
    n, m, L = 16, 10, 2
    th = S.phases(21, L, n)
    fwd, adj = O.structured_ops(th, n, m)
    y = np.abs(fwd(S.complex_gaussian(1, (1, n), S.STREAM_SIGNAL))) ** 2
    x = S.complex_gaussian(2, (1, n), S.STREAM_SIGNAL)
    _, g = O.loss_and_grad(x, y, fwd, adj)
    d = S.complex_gaussian(3, (1, n), S.STREAM_NOISE)
    h = 1e-6
    lp = O.intensity_loss(fwd(x + h * d), y)
    lm = O.intensity_loss(fwd(x - h * d), y)
    # dL/dRe x_k = 2 Re g_k and dL/dIm x_k = 2 Im g_k, so along d: 2 Re sum conj(g) d
    fd = (lp - lm) / (2 * h)
    assert np.allclose(fd, 2 * np.real(np.sum(g.conj() * d, axis=1)), rtol=1e-6)
