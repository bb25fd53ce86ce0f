"""GPU parity of the 2D model (h x w images in an S x S grid, unitary 2D DFTs;
the form Sec. IV runs) against the FP64 oracle of oracle/operator2d.py, which
is pinned in test_oracle_2d.py.

Same tolerances as the 1D parity tests (test_gpu_parity.py): the 2D path runs
the same four-step passes with unit four-step twiddles, so its FP32 error is
that of two line FFTs per DFT. Odd L matters separately: the kernels then end
the forward on the transposed grid and transpose y for the epilogue."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sr():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2409_05734_gb300 import buildlib
    buildlib.build()
    import paper_2409_05734_gb300 as pkg
    return pkg


def dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def assert_close_elementwise(got, ref, tol_norm=1e-5, tol_elem=2e-5):
    assert rel(got, ref) <= tol_norm, rel(got, ref)
    rms = np.sqrt(np.mean(np.abs(ref) ** 2))
    worst = np.max(np.abs(got - ref)) / rms
    assert worst <= tol_elem, worst


CASES = [
    # (h, w, S, L, B): smallest grid, h != w both ways, no padding, odd and even L,
    # several tiles per pass, the 128 x 128 image at alpha = 4, largest grid
    (1, 1, 2, 1, 1),
    (2, 1, 2, 2, 3),
    (3, 5, 8, 1, 2),
    (5, 3, 8, 2, 2),
    (8, 8, 8, 3, 1),
    (7, 16, 16, 3, 5),
    (20, 30, 32, 2, 3),
    (64, 64, 64, 1, 2),
    (100, 128, 128, 3, 2),
    (60, 50, 64, 4, 1),
    (128, 128, 256, 2, 2),
    (128, 128, 256, 3, 1),
    (300, 512, 512, 2, 1),
    (1000, 700, 1024, 1, 1),
    (2048, 1500, 2048, 2, 1),
    (4096, 3000, 4096, 1, 1),
    (5, 9, 16, 2, 700),
]


@pytest.mark.parametrize("h,w,S_,L,B", CASES)
def test_2d_forward_adjoint(sr, h, w, S_, L, B):
    seed = 4000 + h + 7 * w + S_ + L
    plan = sr.Plan2D(h, w, S_, L, seed)
    theta = S.phases(seed, L, S_ * S_)
    assert np.array_equal(plan.phases, theta)
    x = S.signal_gaussian(seed, B, h * w)
    z = host(plan.forward(dev(x)))
    plan.check()
    assert_close_elementwise(z, O.forward_2d(x, theta, h, w, S_))
    wv = S.complex_gaussian(seed + 1, (B, S_ * S_), S.STREAM_NOISE)
    xa = host(plan.adjoint(dev(wv)))
    plan.check()
    assert_close_elementwise(xa, O.adjoint_2d(wv, theta, h, w, S_))


@pytest.mark.parametrize("L", [1, 2, 3])
def test_2d_loss_grad(sr, L):
    h, w, S_, B = 24, 20, 32, 3
    seed = 77 + L
    plan = sr.Plan2D(h, w, S_, L, seed)
    fwd, adj = O.structured_ops_2d(S.phases(seed, L, S_ * S_), h, w, S_)
    y = np.abs(fwd(S.phase_image_ellipses(seed, B, h, w))) ** 2
    x = S.signal_gaussian(seed + 1, B, h * w)
    loss_o, g_o = O.loss_and_grad(x, y, fwd, adj)
    loss, g = plan.loss_grad(dev(x), dev(y, torch.float32))
    plan.check()
    assert np.max(np.abs(host(loss) - loss_o) / loss_o) <= 1e-5
    assert_close_elementwise(host(g), g_o)


@pytest.mark.parametrize("L,weight", [(2, "optimal"), (3, "optimal"), (1, "identity")])
def test_2d_spectral_init(sr, L, weight):
    h, w, S_, B, T = 16, 16, 32, 2, 40
    seed = 20240905 + L
    plan = sr.Plan2D(h, w, S_, L, seed)
    fwd, adj = O.structured_ops_2d(S.phases(seed, L, S_ * S_), h, w, S_)
    y = np.abs(fwd(S.phase_image_ellipses(seed, B, h, w))) ** 2
    v0 = S.start_vector(seed, B, h * w)
    ref = O.spectral_init(y, v0, fwd, adj, T, mode=weight, lam=-1.0)
    got = host(plan.spectral_init(dev(y, torch.float32), dev(v0), T, weight=weight, lam=-1.0))
    plan.check()
    for b in range(B):
        assert rel(got[b], ref[b]) <= 1e-4


@pytest.mark.parametrize("L", [2, 3])
def test_2d_gradient_descent_phase_images(sr, L):
    """Phantom-like phase images (Sec. IV-A recipe), alpha = 4 (16 x 16 in 32 x 32):
    spectral start, then GD with the warm-up schedule; the reconstruction error
    (up to a global phase) and the loss history follow the oracle."""
    h = w = 16
    S_, B = 32, 2
    seed = 20240905
    plan = sr.Plan2D(h, w, S_, L, seed)
    fwd, adj = O.structured_ops_2d(S.phases(seed, L, S_ * S_), h, w, S_)
    x_true = S.phase_image_ellipses(seed, B, h, w)
    y = np.abs(fwd(x_true)) ** 2
    v0 = S.start_vector(seed, B, h * w)
    x0_o = O.spectral_init(y, v0, fwd, adj, 50, mode="optimal")
    xT_o, hist_o = O.gradient_descent(x0_o, y, fwd, adj, 200, mu0=0.1, tau0=20.0)
    x = dev(x0_o)
    _, hist = plan.gd_solve(dev(y, torch.float32), x, 200, mu0=0.1, tau0=20.0, record_loss=True)
    plan.check()
    err_o = O.relative_error_global_phase(xT_o, x_true)
    err_g = O.relative_error_global_phase(host(x), x_true)
    assert np.all(np.abs(err_g - err_o) <= 1e-4)
    h_ = host(hist)
    assert np.max(np.abs(h_[:20] - hist_o[:20]) / hist_o[:20]) <= 1e-3


def test_2d_rejects_unsupported(sr):
    with pytest.raises(Exception):
        sr.Plan2D(4, 4, 12, 2, 1)  # S not a power of two
    with pytest.raises(Exception):
        sr.Plan2D(9, 4, 8, 2, 1)  # h > S
    plan = sr.Plan2D(4, 4, 8, 2, 1)
    with pytest.raises(Exception):
        plan.set_phases_device(torch.zeros(2 * 64, device="cuda"))
    x = torch.zeros((1, 16), dtype=torch.complex64, device="cuda")
    with pytest.raises(Exception):
        plan.backward(x, torch.zeros((1, 64), dtype=torch.complex64, device="cuda"))
    # the plan still works after the refusals
    theta = S.phases(1, 2, 64)
    xs = S.signal_gaussian(3, 1, 16)
    assert_close_elementwise(host(plan.forward(dev(xs))), O.forward_2d(xs, theta, 4, 4, 8))
