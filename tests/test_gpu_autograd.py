"""GPU parity of the differentiable operator: sr_backward, device-set phases
and the torch.autograd.Function, against the FP64 oracle's backward pass
(itself pinned by finite differences in test_oracle_autodiff.py)."""
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


def _loss_parts(seed, B, m):
    c = S.complex_gaussian(seed, (B, m), S.STREAM_NOISE)
    w = np.abs(S.complex_gaussian(seed + 1, (B, m), S.STREAM_NOISE))
    return c, w


@pytest.mark.parametrize("n,m,L,B", [(256, 1024, 2, 3), (100, 512, 1, 2), (37, 128, 3, 4), (5000, 2 ** 14, 2, 2),
                                     (3000, 3 * 2 ** 13, 2, 2), (20, 48, 2, 2)])
def test_backward_matches_oracle(sr, n, m, L, B):
    seed = n + m
    plan = sr.Plan(n, m, L, seed)
    # phases set from a device float32 tensor; the oracle uses the same float values
    theta = S.phases(seed, L, m).astype(np.float32)
    plan.set_phases_device(torch.from_numpy(theta).cuda())
    th64 = theta.astype(np.float64)
    assert np.array_equal(plan.phases, th64)
    x = S.signal_gaussian(seed, B, n)
    c, w = _loss_parts(seed + 2, B, m)
    z = O.forward(x, th64, m)
    gz = c + 2 * w * z
    gx_o, gth_o = O.autodiff.backward(x, gz, th64, n, m)
    zg = host(plan.forward(dev(x)))
    assert rel(zg, z) <= 1e-5
    gx, gth = plan.backward(dev(x), dev(gz))
    plan.check()
    assert rel(host(gx), gx_o) <= 1e-5
    # phase gradient: a batch sum of products of two transforms
    assert np.max(np.abs(host(gth) - gth_o)) <= 2e-5 * np.max(np.abs(gth_o))
    assert rel(host(gth), gth_o) <= 2e-5


def test_autograd_function_matches_oracle(sr):
    n, m, L, B = 256, 1024, 2, 3
    seed = 5
    plan = sr.Plan(n, m, L, seed)
    theta64 = S.phases(seed, L, m)
    theta = torch.tensor(theta64.astype(np.float32), device="cuda", requires_grad=True)
    x_np = S.signal_gaussian(seed, B, n)
    x = dev(x_np).requires_grad_(True)
    c, w = _loss_parts(11, B, m)
    ct, wt = dev(c), torch.from_numpy(w).float().cuda()
    z = sr.structured_random(x, theta, plan)
    loss = torch.real(torch.sum(torch.conj(ct) * z)) + torch.sum(wt * torch.abs(z) ** 2)
    loss.backward()
    th = theta.detach().cpu().numpy().astype(np.float64)
    zo = O.forward(x_np, th, m)
    gx_o, gth_o = O.autodiff.backward(x_np, c + 2 * w * zo, th, n, m)
    assert rel(host(x.grad), gx_o) <= 1e-5
    assert rel(host(theta.grad), gth_o) <= 2e-5
    # only theta requires grad
    theta.grad = None
    z2 = sr.structured_random(dev(x_np), theta, plan)
    torch.sum(torch.abs(z2) ** 2 * wt).backward()
    assert theta.grad is not None


def test_differentiable_operator_large_batch_sampled(sr):
    """B = 8 signals, n = 2^20 (1024 x 1024), alpha = 4 (m = 2^22), L = 2: forward and
    backward on the GPU; the oracle checks two problems of the batch for grad_x and the
    phase gradient summed over the batch on sampled entries."""
    n, m, L, B = 2 ** 20, 2 ** 22, 2, 8
    seed = 20240905
    plan = sr.Plan(n, m, L, seed)
    theta = S.phases(seed, L, m).astype(np.float32)
    plan.set_phases_device(torch.from_numpy(theta).cuda())
    th64 = theta.astype(np.float64)
    x = S.signal_gaussian(seed, B, n)
    c, w = _loss_parts(3, B, m)
    xd = dev(x)
    z = plan.forward(xd)
    wt = torch.from_numpy(w).float().cuda()
    gz = (dev(c) + 2 * wt * z).contiguous()
    gx, gth = plan.backward(xd, gz)
    plan.check()
    zh = host(z)
    zo = O.forward(x, th64, m)
    assert rel(zh, zo) <= 1e-5
    gz_o = c + 2 * w * zo
    gx_o, gth_o = O.autodiff.backward(x, gz_o, th64, n, m)
    gxh = host(gx)
    for b in (0, 5):
        assert rel(gxh[b], gx_o[b]) <= 1e-4
    idx = np.random.default_rng(0).integers(0, m, 4096)
    g = host(gth)
    for l in range(L):
        err = np.max(np.abs(g[l, idx] - gth_o[l, idx])) / np.max(np.abs(gth_o[l]))
        assert err <= 1e-4, err
