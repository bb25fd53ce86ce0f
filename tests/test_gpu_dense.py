"""GPU parity of the dense i.i.d. comparison model (tcgen05 GEMM, BF16 and
TF32 operands) against the FP64 oracle's matrix products, with the same
BF16-exact or TF32-exact matrix on both sides.

Tolerance: the vector operand is split into high and low parts of the
operand format (about 2^-17 relative each entry in BF16, 2^-22 in TF32) and
products accumulate in FP32, so one product is within 2e-5 relative of the
FP64 result, and every entry within 1e-4 of the RMS."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def DenseModel():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2409_05734_gb300 import buildlib
    buildlib.build()
    from paper_2409_05734_gb300 import DenseModel as D
    return D


def dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


MATRIX = {"bf16": S.dense_iid_matrix_bf16, "tf32": S.dense_iid_matrix_tf32}
ROUND = {"bf16": S.round_to_bf16, "tf32": S.round_to_tf32}
FORMATS = ["bf16", "tf32"]


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("n,m,B", [(64, 128, 8), (128, 512, 16), (256, 1024, 40), (512, 2048, 64)])
def test_dense_forward_adjoint(DenseModel, n, m, B, fmt):
    A = MATRIX[fmt](n + m, m, n)
    model = DenseModel(A, format=fmt)
    x = S.signal_gaussian(1, B, n)
    z = model.forward(dev(x)).cpu().numpy()
    model.check()
    zo = O.dense_forward(A, x)
    assert rel(z, zo) <= 2e-5
    assert np.max(np.abs(z - zo)) <= 1e-4 * np.sqrt(np.mean(np.abs(zo) ** 2))
    w = S.complex_gaussian(2, (B, m), S.STREAM_NOISE)
    xa = model.adjoint(dev(w)).cpu().numpy()
    model.check()
    xo = O.dense_adjoint(A, w)
    assert rel(xa, xo) <= 2e-5
    assert np.max(np.abs(xa - xo)) <= 1e-4 * np.sqrt(np.mean(np.abs(xo) ** 2))


@pytest.mark.parametrize("fmt", FORMATS)
def test_dense_gradient_descent(DenseModel, fmt):
    n, m, B = 128, 512, 8
    A = MATRIX[fmt](7, m, n)
    model = DenseModel(A, format=fmt)
    fwd, adj = O.dense_ops(A)
    xt = S.signal_gaussian(3, B, n)
    y = np.abs(fwd(xt)) ** 2
    x0 = O.spectral_init(y, S.start_vector(3, B, n), fwd, adj, 30, mode="optimal")
    xT, hist = O.gradient_descent(x0, y, fwd, adj, 40, mu0=0.1, tau0=10.0)
    x = dev(x0)
    _, h = model.gd_solve(dev(y, torch.float32), x, 40, mu0=0.1, tau0=10.0, record_loss=True)
    model.check()
    assert rel(x.cpu().numpy(), xT) <= 1e-4
    assert np.max(np.abs(x.cpu().numpy() - xT)) <= 1e-3 * np.sqrt(np.mean(np.abs(xT) ** 2))
    hh = h.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(hh - hist) / hist) <= 1e-3


@pytest.mark.parametrize("fmt", FORMATS)
@pytest.mark.parametrize("weight", ["identity", "optimal"])
def test_dense_spectral_init(DenseModel, weight, fmt):
    n, m, B, T = 128, 512, 8, 40
    A = MATRIX[fmt](9, m, n)
    model = DenseModel(A, format=fmt)
    fwd, adj = O.dense_ops(A)
    xt = S.signal_gaussian(5, B, n)
    y = np.abs(fwd(xt)) ** 2
    v0 = S.start_vector(5, B, n)
    ref = O.spectral_init(y, v0, fwd, adj, T, mode=weight, lam=-1.0)
    got = model.spectral_init(dev(y, torch.float32), dev(v0), T, weight=weight, lam=-1.0).cpu().numpy()
    model.check()
    for b in range(B):
        assert rel(got[b], ref[b]) <= 1e-4
        assert np.max(np.abs(got[b] - ref[b])) <= 1e-3 * np.sqrt(np.mean(np.abs(ref[b]) ** 2))
    got0 = model.spectral_init(dev(y, torch.float32), dev(v0), 0).cpu().numpy()
    assert rel(got0, O.spectral_init(y, v0, fwd, adj, 0)) <= 1e-6


@pytest.mark.parametrize("fmt", FORMATS)
def test_dense_comparison_size_sampled(DenseModel, fmt):
    """The comparison shape: n = 4096, m = 16384, B = 64; sampled output rows."""
    n, m, B = 4096, 16384, 64
    rng = np.random.default_rng(5)
    A = ROUND[fmt](rng.standard_normal((m, n)) / np.sqrt(2 * m)) + \
        1j * ROUND[fmt](rng.standard_normal((m, n)) / np.sqrt(2 * m))
    model = DenseModel(A, format=fmt)
    x = S.signal_amplitude_phase(2, B, n)
    z = model.forward(dev(x)).cpu().numpy()
    model.check()
    rows = rng.integers(0, m, 256)
    zo = x @ A[rows].T
    assert rel(z[:, rows], zo) <= 2e-5
    assert np.max(np.abs(z[:, rows] - zo)) <= 1e-4 * np.sqrt(np.mean(np.abs(zo) ** 2))
    w = S.complex_gaussian(4, (B, m), S.STREAM_NOISE)
    xa = model.adjoint(dev(w)).cpu().numpy()
    model.check()
    cols = rng.integers(0, n, 128)
    xo = w @ np.conj(A[:, cols])
    assert rel(xa[:, cols], xo) <= 2e-5
    assert np.max(np.abs(xa[:, cols] - xo)) <= 1e-4 * np.sqrt(np.mean(np.abs(xo) ** 2))


def test_dense_tf32_rounds_the_matrix_itself(DenseModel):
    """The TF32 model rounds the caller's FP32 entries (to nearest, ties away
    from zero): a matrix off the TF32 grid gives the products of its rounded
    copy, not of the original."""
    n, m, B = 64, 128, 8
    A = S.dense_iid_matrix(11, m, n)
    Ar = S.round_to_tf32(A.real.astype(np.float32)) + 1j * S.round_to_tf32(A.imag.astype(np.float32))
    model = DenseModel(A, format="tf32")
    x = S.signal_gaussian(2, B, n)
    z = model.forward(dev(x)).cpu().numpy()
    model.check()
    assert rel(z, O.dense_forward(Ar, x)) <= 2e-5
    assert rel(O.dense_forward(A, x), O.dense_forward(Ar, x)) > 1e-4  # the rounding is visible


def test_dense_rejects_unknown_format(DenseModel):
    with pytest.raises(ValueError):
        DenseModel(S.dense_iid_matrix_bf16(1, 128, 64), format="fp8")
