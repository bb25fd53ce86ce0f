"""GPU parity of the radix-3 lengths m = 3 * 2^a (oversampling alpha in {1.5, 3,
6, ...}) against the FP64 oracle, whose DFT of those lengths is pinned against
the naive O(m^2) DFT in test_oracle_operator.py. Same tolerances as the
power-of-two parity tests: one radix-3 step adds a few FP32 roundings per
element to the power-of-two transform."""
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
    # (n, m, L, B): smallest length, ragged n, alpha = 1.5 / 3 / 6 at the sweep's n = 2^16, L up to 4
    (10, 12, 2, 1),
    (5, 24, 3, 2),
    (40, 48, 1, 3),
    (100, 384, 2, 2),
    (1000, 3072, 2, 2),
    (3 * 2 ** 11, 3 * 2 ** 12, 4, 2),
    (2 ** 16, 3 * 2 ** 15, 2, 1),
    (2 ** 16, 3 * 2 ** 16, 3, 1),
    (2 ** 16, 3 * 2 ** 17, 2, 1),
    (7, 48, 2, 700),
    (2 ** 22 - 1, 3 * 2 ** 22, 2, 1),  # the largest radix-3 length
]


@pytest.mark.parametrize("n,m,L,B", CASES)
def test_radix3_forward_adjoint(sr, n, m, L, B):
    seed = 3000 + n + m + L
    plan = sr.Plan(n, m, L, seed)
    theta = S.phases(seed, L, m)
    assert np.array_equal(plan.phases, theta)
    x = S.signal_gaussian(seed, B, n)
    z = host(plan.forward(dev(x)))
    plan.check()
    assert_close_elementwise(z, O.forward(x, theta, m))
    w = S.complex_gaussian(seed + 1, (B, m), S.STREAM_NOISE)
    xa = host(plan.adjoint(dev(w)))
    plan.check()
    assert_close_elementwise(xa, O.adjoint(w, theta, n))


@pytest.mark.parametrize("n,m", [(64, 192), (3000, 3 * 2 ** 13)])  # inner-plan form; radix-3 lines
def test_radix3_loss_grad(sr, n, m):
    L, B = 2, 3
    seed = 11
    plan = sr.Plan(n, m, L, seed)
    theta = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(theta, n, m)
    y = np.abs(fwd(S.signal_gaussian(seed, B, n))) ** 2
    x = S.signal_gaussian(seed + 1, B, n)
    loss_o, g_o = O.loss_and_grad(x, y, fwd, adj)
    loss, g = plan.loss_grad(dev(x), dev(y, torch.float32))
    plan.check()
    assert np.max(np.abs(host(loss) - loss_o) / loss_o) <= 1e-5
    assert_close_elementwise(host(g), g_o)


@pytest.mark.parametrize("n,m", [(64, 192), (3000, 3 * 2 ** 13)])
@pytest.mark.parametrize("weight", ["identity", "optimal"])
def test_radix3_spectral_init(sr, weight, n, m):
    L, B, T = 2, 3, 50
    seed = 20240905
    plan = sr.Plan(n, m, L, seed)
    theta = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(theta, n, m)
    y = np.abs(fwd(S.signal_gaussian(seed, B, n))) ** 2
    v0 = S.start_vector(seed, B, n)
    ref = O.spectral_init(y, v0, fwd, adj, T, mode=weight, lam=-1.0)
    got = host(plan.spectral_init(dev(y, torch.float32), dev(v0), T, weight=weight, lam=-1.0))
    plan.check()
    for b in range(B):
        assert rel(got[b], ref[b]) <= 1e-4


@pytest.mark.parametrize("n,m", [(64, 192), (4096, 3 * 2 ** 12)])  # inner-plan form; radix-3 lines
def test_radix3_gradient_descent_alpha_3(sr, n, m):
    """alpha = 3 (m = 3n), L = 2: 50 power iterations, then 300 GD steps with
    the warm-up step schedule; loss history and final estimate vs the oracle."""
    L = 2
    seed = 20240905
    plan = sr.Plan(n, m, L, seed)
    theta = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(theta, n, m)
    x_true = S.signal_gaussian(seed, 2, n)
    y = np.abs(fwd(x_true)) ** 2
    v0 = S.start_vector(seed, 2, n)
    x0_o = O.spectral_init(y, v0, fwd, adj, 50, mode="optimal")
    xT_o, hist_o = O.gradient_descent(x0_o, y, fwd, adj, 300, mu0=0.1, tau0=20.0)
    yd = dev(y, torch.float32)
    x0 = plan.spectral_init(yd, dev(v0), 50, weight="optimal")
    assert rel(host(x0), x0_o) <= 1e-4
    x = dev(x0_o)
    _, hist = plan.gd_solve(yd, x, 300, mu0=0.1, tau0=20.0, record_loss=True)
    plan.check()
    xh = host(x)
    err_o = O.relative_error_global_phase(xT_o, x_true)
    err_g = O.relative_error_global_phase(xh, x_true)
    assert np.all(np.abs(err_g - err_o) <= 1e-4)
    h = host(hist)
    assert np.max(np.abs(h[:20] - hist_o[:20]) / hist_o[:20]) <= 1e-3


def test_radix3_backward(sr):
    n, m, L, B = 256, 768, 2, 3
    seed = 5
    plan = sr.Plan(n, m, L, seed)
    theta = S.phases(seed, L, m).astype(np.float32)
    plan.set_phases_device(torch.from_numpy(theta).cuda())
    th64 = theta.astype(np.float64)
    x = S.signal_gaussian(seed, B, n)
    c = S.complex_gaussian(seed + 2, (B, m), S.STREAM_NOISE)
    z = O.forward(x, th64, m)
    gz = c + 2 * z
    gx_o, gth_o = O.autodiff.backward(x, gz, th64, n, m)
    gx, gth = plan.backward(dev(x), dev(gz))
    plan.check()
    assert rel(host(gx), gx_o) <= 1e-5
    assert rel(host(gth), gth_o) <= 2e-5
