"""GPU parity of the resident solver for short transforms (power-of-two
m <= 8192: whole solves inside one CTA per problem) against the FP64 oracle,
across every supported length, ragged n, L = 1..4, batches that fill the
GPU or leave most SMs idle (the two problems-per-CTA shapes), per-problem
phases, loss histories and the early-stopping forms. Tolerances as in
test_gpu_parity.py."""
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


def dev(a, dtype=torch.complex64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype).cuda()


def host(t):
    return t.detach().cpu().numpy().astype(np.complex128 if t.is_complex() else np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    # (n, m, L, B)
    (3, 4, 1, 3), (5, 8, 2, 2), (16, 16, 2, 5), (20, 32, 3, 4), (64, 64, 2, 300), (100, 128, 1, 2),
    (77, 256, 4, 9), (512, 512, 2, 2), (1000, 1024, 3, 700), (600, 2048, 2, 3), (4096, 4096, 2, 2),
    (3001, 8192, 2, 2), (2048, 8192, 3, 200),
]


@pytest.mark.parametrize("n,m,L,B", CASES)
def test_small_loss_grad_and_spectral(Plan, n, m, L, B):
    seed = 7000 + n + m + L
    plan = Plan(n, m, L, seed)
    fwd, adj = O.structured_ops(S.phases(seed, L, m), n, m)
    y = np.abs(fwd(S.signal_gaussian(seed, B, n))) ** 2
    x = S.signal_gaussian(seed + 1, B, n)
    loss_o, g_o = O.loss_and_grad(x, y, fwd, adj)
    loss, g = plan.loss_grad(dev(x), dev(y, torch.float32))
    plan.check()
    assert np.max(np.abs(host(loss) - loss_o) / loss_o) <= 1e-5
    assert rel(host(g), g_o) <= 1e-5
    v0 = S.start_vector(seed, B, n)
    ref = O.spectral_init(y, v0, fwd, adj, 15, mode="optimal")
    got = host(plan.spectral_init(dev(y, torch.float32), dev(v0), 15, weight="optimal"))
    plan.check()
    assert max(rel(got[b], ref[b]) for b in range(B)) <= 1e-4


@pytest.mark.parametrize("n,m,L,B", [(64, 256, 2, 4), (1000, 4096, 2, 3), (2000, 8192, 2, 2)])
def test_small_gradient_descent_with_history(Plan, n, m, L, B):
    seed = 31 + m
    plan = Plan(n, m, L, seed)
    fwd, adj = O.structured_ops(S.phases(seed, L, m), n, m)
    x_true = S.signal_gaussian(seed, B, n)
    y = np.abs(fwd(x_true)) ** 2
    x0 = O.spectral_init(y, S.start_vector(seed, B, n), fwd, adj, 30, mode="optimal")
    xT_o, hist_o = O.gradient_descent(x0, y, fwd, adj, 60, mu0=0.1, tau0=10.0)
    x = dev(x0)
    _, hist = plan.gd_solve(dev(y, torch.float32), x, 60, mu0=0.1, tau0=10.0, record_loss=True)
    plan.check()
    err_o = O.relative_error_global_phase(xT_o, x_true)
    err_g = O.relative_error_global_phase(host(x), x_true)
    assert np.all(np.abs(err_g - err_o) <= 1e-4)
    h = host(hist)
    assert np.max(np.abs(h[:20] - hist_o[:20]) / hist_o[:20]) <= 1e-3


def test_small_per_problem_phases_and_early_stop(Plan):
    n, m, L = 200, 1024, 2
    seeds = [3, 14, 15, 92]
    plan = Plan(n, m, L, 1)
    plan.set_batch_seeds(seeds)
    x_true = S.signal_gaussian(8, len(seeds), n)
    ys = np.stack([np.abs(O.forward(x_true[b], S.phases(sd, L, m), m)) ** 2 for b, sd in enumerate(seeds)])
    x0 = np.stack([O.spectral_init(ys[b][None], S.start_vector(8, len(seeds), n)[b][None],
                                   *O.structured_ops(S.phases(sd, L, m), n, m), 20, mode="optimal")[0]
                   for b, sd in enumerate(seeds)])
    yd = dev(ys, torch.float32)
    x1 = dev(x0)
    plan.gd_solve(yd, x1, 25, mu0=0.1, tau0=5.0)
    for b, sd in enumerate(seeds):
        fwd, adj = O.structured_ops(S.phases(sd, L, m), n, m)
        xr, _ = O.gradient_descent(x0[b][None], ys[b][None], fwd, adj, 25, mu0=0.1, tau0=5.0)
        assert rel(host(x1)[b], xr[0]) <= 1e-4
    x2 = dev(x0)
    _, t, _ = plan.gd_solve_early_stop(yd, x2, 25, 0.0, check_every=6, mu0=0.1, tau0=5.0)
    plan.check()
    assert t == 25
    assert (torch.linalg.vector_norm(x1 - x2) / torch.linalg.vector_norm(x1)).item() <= 1e-6
