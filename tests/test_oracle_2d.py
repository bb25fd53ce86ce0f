"""Pins of the 2D oracle (oracle/operator2d.py) against brute-force sums, closed
forms and invariants, none of which call the oracle's own 2D routines.

A plausible mistake in the oracle (transposed padding, a swapped DFT axis, a
wrong sign or scale, D applied after instead of before the DFT, a dropped
layer) fails at least one of these."""
import numpy as np
import pytest

import oracle as O
import synthetic as S

pytestmark = pytest.mark.filterwarnings("ignore")


def brute_dft2(img):
    """sum_{r,c} img[r, c] exp(-2 pi i (r a + c b) / S) / S by explicit loops."""
    S_ = img.shape[0]
    out = np.zeros((S_, S_), dtype=np.complex128)
    for a in range(S_):
        for b in range(S_):
            acc = 0j
            for r in range(S_):
                for c in range(S_):
                    acc += img[r, c] * np.exp(-2j * np.pi * ((r * a + c * b) % S_) / S_)
            out[a, b] = acc / S_
    return out


@pytest.mark.parametrize("S_", [1, 2, 4, 6])
def test_fft2_equals_brute_force_sum(S_):
    img = S.complex_gaussian(7, (S_, S_), S.STREAM_SIGNAL)
    got = O.unitary_fft2(img.reshape(-1), S_).reshape(S_, S_)
    assert np.allclose(got, brute_dft2(img), atol=1e-12)
    back = O.unitary_ifft2(got.reshape(-1), S_).reshape(S_, S_)
    assert np.allclose(back, img, atol=1e-12)


def test_fft2_orientation_plane_wave():
    """exp(+2 pi i (r a0 + c b0)/S) / S transforms to a unit spike at row a0,
    column b0, i.e. flat index a0 * S + b0 (not b0 * S + a0)."""
    S_, a0, b0 = 8, 3, 5
    r, c = np.meshgrid(np.arange(S_), np.arange(S_), indexing="ij")
    img = np.exp(2j * np.pi * (r * a0 + c * b0) / S_) / S_
    z = O.unitary_fft2(img.reshape(-1), S_)
    want = np.zeros(S_ * S_, dtype=np.complex128)
    want[a0 * S_ + b0] = 1.0
    assert np.allclose(z, want, atol=1e-12)


def test_pad_and_crop_index_rule():
    h, w, S_ = 3, 5, 8
    x = np.arange(h * w) + 1.0
    v = O.zero_pad_2d(x, h, w, S_)
    for r in range(S_):
        for c in range(S_):
            want = r * w + c + 1.0 if (r < h and c < w) else 0.0
            assert v[r * S_ + c] == want
    assert np.array_equal(O.crop_2d(v, h, w, S_), x)


def test_single_pixel_closed_form():
    """x = one pixel at (0, 0): after D_1 and F2 every entry is exp(i theta_1[0]) / S;
    the second layer is then F2 of exp(i theta_2) times that constant (brute force)."""
    S_ = 4
    th = S.phases(11, 2, S_ * S_)
    z1 = O.forward_2d(np.array([1.0 + 0j]), th[:1], 1, 1, S_)
    assert np.allclose(z1, np.exp(1j * th[0, 0]) / S_, atol=1e-14)
    z2 = O.forward_2d(np.array([1.0 + 0j]), th, 1, 1, S_)
    want = brute_dft2(np.exp(1j * th[1]).reshape(S_, S_) * np.exp(1j * th[0, 0]) / S_).reshape(-1)
    assert np.allclose(z2, want, atol=1e-12)


def test_single_row_reduces_to_1d_dft():
    """L = 1, theta = 0, a 1 x w image: every row a of the 2D spectrum is the
    unitary 1D DFT (pinned naive matrix) of the padded row, over sqrt(S)."""
    S_, w = 8, 5
    row = S.complex_gaussian(3, (w,), S.STREAM_SIGNAL)
    z = O.forward_2d(row, np.zeros((1, S_ * S_)), 1, w, S_).reshape(S_, S_)
    d1 = O.dft_naive(np.concatenate([row, np.zeros(S_ - w)])) / np.sqrt(S_)
    for a in range(S_):
        assert np.allclose(z[a], d1, atol=1e-12)


@pytest.mark.parametrize("h,w,S_,L", [(2, 3, 4, 1), (3, 2, 4, 2), (4, 4, 4, 3), (1, 5, 6, 2)])
def test_forward_adjoint_match_dense_matrix(h, w, S_, L):
    th = S.phases(5 + L, L, S_ * S_)
    A = O.dense_structured_matrix_2d(th, h, w, S_)
    x = S.complex_gaussian(1, (3, h * w), S.STREAM_SIGNAL)
    z = S.complex_gaussian(2, (3, S_ * S_), S.STREAM_NOISE)
    assert np.allclose(O.forward_2d(x, th, h, w, S_), x @ A.T, atol=1e-12)
    assert np.allclose(O.adjoint_2d(z, th, h, w, S_), z @ A.conj(), atol=1e-12)


@pytest.mark.parametrize("L", [1, 2, 3])
def test_unitary_without_padding_and_adjoint_identity(L):
    S_ = 8
    th = S.phases(9, L, S_ * S_)
    x = S.complex_gaussian(4, (2, S_ * S_), S.STREAM_SIGNAL)
    z = O.forward_2d(x, th, S_, S_, S_)
    assert np.allclose(np.linalg.norm(z, axis=1), np.linalg.norm(x, axis=1), rtol=1e-12)
    assert np.allclose(O.adjoint_2d(z, th, S_, S_, S_), x, atol=1e-12)
    h, w = 5, 3
    xs = S.complex_gaussian(6, (2, h * w), S.STREAM_SIGNAL)
    ws = S.complex_gaussian(8, (2, S_ * S_), S.STREAM_NOISE)
    lhs = np.sum(O.forward_2d(xs, th, h, w, S_) * ws.conj(), axis=1)
    rhs = np.sum(xs * O.adjoint_2d(ws, th, h, w, S_).conj(), axis=1)
    assert np.allclose(lhs, rhs, atol=1e-12)


def test_layer_order_d1_first():
    """A = F2 D_2 F2 D_1 U2: swapping the two phase layers changes the result
    unless the image is a single pixel at the origin and D_1 = 1 there."""
    S_ = 4
    th = S.phases(13, 2, S_ * S_)
    x = S.complex_gaussian(1, (S_ * S_,), S.STREAM_SIGNAL)
    z = O.forward_2d(x, th, S_, S_, S_)
    F2 = O.dense_structured_matrix_2d(np.zeros((1, S_ * S_)), S_, S_, S_)
    want = F2 @ (np.exp(1j * th[1]) * (F2 @ (np.exp(1j * th[0]) * x)))
    assert np.allclose(z, want, atol=1e-12)
    assert not np.allclose(z, O.forward_2d(x, th[::-1], S_, S_, S_), atol=1e-6)


def test_phase_images_are_unit_modulus_phantoms():
    x = S.phase_image_ellipses(20240905, 3, 32, 24)
    assert x.shape == (3, 32 * 24)
    assert np.allclose(np.abs(x), 1.0)
    phi = np.angle(x)
    assert phi.min() >= -np.pi / 2 - 1e-12 and phi.max() < np.pi / 2
    # piecewise constant: a handful of grey levels, and the images differ
    assert all(len(np.unique(np.round(p, 9))) < 200 for p in phi)
    assert not np.allclose(x[0], x[1])
    assert np.array_equal(x, S.phase_image_ellipses(20240905, 3, 32, 24))
