"""GPU parity of GD with early stopping (sr_gd_solve_early_stop) against the
oracle's rule (pinned in test_oracle_early_stop.py). The stop iteration is an
integer decided by floating-point losses, so each case first checks on the
oracle that the decision has a clear margin on both sides (the FP32 losses
are accurate to about 1e-6 relative, which moves a relative change of 1e-3 by
well under 1%)."""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Plan():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2409_05734_gb300 import buildlib
    buildlib.build()
    from paper_2409_05734_gb300 import Plan as P
    return P


def _noisy_problem(B, n, m, L, seed, sigma=0.05):
    th = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(th, n, m)
    x_true = S.signal_gaussian(seed, B, n)
    y0 = np.abs(fwd(x_true)) ** 2
    y = np.maximum(y0 + S.gaussian_noise(seed, y0.shape, sigma * y0.mean()), 0.0)
    x0 = O.spectral_init(y, S.start_vector(seed, B, n), fwd, adj, 30, mode="optimal")
    return y, x0, fwd, adj


@pytest.mark.parametrize("B,n,m,L,seed,tol,every", [(3, 256, 1024, 2, 8, 1e-3, 10),
                                                     (2, 1024, 4096, 2, 5, 1e-3, 10)])
def test_early_stop_matches_oracle(Plan, B, n, m, L, seed, tol, every):
    y, x0, fwd, adj = _noisy_problem(B, n, m, L, seed)
    T = 400
    x_o, h_o, t_o = O.gradient_descent_early_stop(x0, y, fwd, adj, T, tol, every, mu0=0.1, tau0=5.0)
    assert every < t_o < T
    # margins of the decision: below tol at the stop, clearly above one check earlier
    ratio = lambda t: np.max(np.abs(h_o[t - 2] - h_o[t - 1]) / h_o[t - 2]) / tol
    assert ratio(t_o) <= 0.95 and ratio(t_o - every) >= 1.05
    plan = Plan(n, m, L, seed)
    x = torch.from_numpy(x0).to(torch.complex64).cuda()
    yd = torch.from_numpy(y).float().cuda()
    _, t_g, h_g = plan.gd_solve_early_stop(yd, x, T, tol, check_every=every, mu0=0.1, tau0=5.0, record_loss=True)
    plan.check()
    assert t_g == t_o
    xg = x.cpu().numpy().astype(np.complex128)
    assert np.linalg.norm(xg - x_o) / np.linalg.norm(x_o) <= 5e-4
    hg = h_g.cpu().numpy().astype(np.float64)
    assert np.max(np.abs(hg - h_o) / h_o) <= 1e-3


def test_early_stop_without_history_and_limits(Plan):
    """Without a loss history the rule reads its internal buffer; a zero
    tolerance runs every iteration and matches sr_gd_solve (up to rounding:
    chunk boundaries replace the fused last/first kernel by the separate ones)."""
    B, n, m, L, seed = 2, 128, 512, 2, 3
    y, x0, fwd, adj = _noisy_problem(B, n, m, L, seed)
    plan = Plan(n, m, L, seed)
    yd = torch.from_numpy(y).float().cuda()
    x1 = torch.from_numpy(x0).to(torch.complex64).cuda()
    x2 = x1.clone()
    _, t, _ = plan.gd_solve_early_stop(yd, x1, 37, 0.0, check_every=5, mu0=0.1, tau0=5.0)
    plan.gd_solve(yd, x2, 37, mu0=0.1, tau0=5.0)
    plan.check()
    assert t == 37
    assert (torch.linalg.vector_norm(x1 - x2) / torch.linalg.vector_norm(x2)).item() <= 1e-6
    _, t, _ = plan.gd_solve_early_stop(yd, x1, 100, 10.0, check_every=4, mu0=0.1, tau0=5.0)
    assert t == 4
    with pytest.raises(Exception):
        plan.gd_solve_early_stop(yd, x1, 10, 1e-3, check_every=1)


@pytest.mark.parametrize("B,n,m,L,seed,tol,every", [(3, 256, 1024, 2, 8, 1e-4, 5),
                                                     (2, 1024, 4096, 2, 5, 1e-4, 6)])
def test_power_iteration_early_stop_matches_oracle(Plan, B, n, m, L, seed, tol, every):
    """The eigenvalue estimates change by ~1e-4 relative at the decision; FP32
    norms are accurate to ~1e-6, so the margin asserted on the oracle (15%)
    covers the FP32 error of the change by an order of magnitude."""
    th = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(th, n, m)
    y = np.abs(fwd(S.signal_gaussian(seed, B, n))) ** 2
    v0 = S.start_vector(seed, B, n)
    T = 400
    x_o, lams, t_o = O.spectral_init_early_stop(y, v0, fwd, adj, T, tol, every, mode="optimal")
    assert every < t_o < T
    ratio = lambda t: np.max(np.abs(lams[t - 2] - lams[t - 1]) / lams[t - 2]) / tol
    assert ratio(t_o) <= 0.9 and ratio(t_o - every) >= 1.1
    plan = Plan(n, m, L, seed)
    x, t_g = plan.spectral_init_early_stop(torch.from_numpy(y).float().cuda(),
                                           torch.from_numpy(v0).to(torch.complex64).cuda(), T, tol,
                                           check_every=every, weight="optimal")
    plan.check()
    assert t_g == t_o
    xg = x.cpu().numpy().astype(np.complex128)
    for b in range(B):
        assert np.linalg.norm(xg[b] - x_o[b]) / np.linalg.norm(x_o[b]) <= 1e-4
    # zero tolerance: every step runs and the result is that of sr_spectral_init
    x2 = plan.spectral_init(torch.from_numpy(y).float().cuda(), torch.from_numpy(v0).to(torch.complex64).cuda(),
                            37, weight="optimal")
    x3, t3 = plan.spectral_init_early_stop(torch.from_numpy(y).float().cuda(),
                                           torch.from_numpy(v0).to(torch.complex64).cuda(), 37, 0.0,
                                           check_every=every, weight="optimal")
    plan.check()
    assert t3 == 37
    assert (torch.linalg.vector_norm(x3 - x2) / torch.linalg.vector_norm(x2)).item() <= 1e-6


@pytest.mark.parametrize("kind", ["radix3", "radix3 lines", "alpha<1", "2d odd L"])
def test_early_stop_calls_on_every_plan_kind(Plan, kind):
    """With a zero tolerance both early-stopping calls run every step and give
    the plain calls' results (chunk boundaries only change the kernel split)."""
    from paper_2409_05734_gb300 import Plan2D
    plan = {"radix3": lambda: Plan(100, 384, 2, 7),
            "radix3 lines": lambda: Plan(3000, 3 * 2 ** 12, 3, 7),
            "alpha<1": lambda: Plan(512, 300, 2, 7),
            "2d odd L": lambda: Plan2D(12, 10, 16, 3, 7)}[kind]()
    B = 2
    x_true = torch.from_numpy(S.signal_gaussian(5, B, plan.n)).to(torch.complex64).cuda()
    y = (plan.forward(x_true).abs() ** 2).contiguous()
    v0 = torch.from_numpy(S.start_vector(5, B, plan.n)).to(torch.complex64).cuda()
    a = plan.spectral_init(y, v0, 13, weight="optimal")
    b, t = plan.spectral_init_early_stop(y, v0, 13, 0.0, check_every=5, weight="optimal")
    assert t == 13
    assert (torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a)).item() <= 1e-6
    x1, x2 = a.clone(), a.clone()
    plan.gd_solve(y, x1, 13, mu0=0.05, tau0=5.0)
    _, t, _ = plan.gd_solve_early_stop(y, x2, 13, 0.0, check_every=5, mu0=0.05, tau0=5.0)
    plan.check()
    assert t == 13
    assert (torch.linalg.vector_norm(x1 - x2) / torch.linalg.vector_norm(x1)).item() <= 1e-6
