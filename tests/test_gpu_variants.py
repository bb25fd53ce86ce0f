"""GPU parity of the 1-layer model with an extra FFT (Sec. IV-B mentions adding
an extra FFT to the 1-layer model), read as A = F D_1 F U. It is the L = 2
plan with theta_1 = 0 (D_1 = I), so it needs no kernel of its own: the
reference here is composed from the oracle's pinned unitary FFT directly."""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.mark.parametrize("n,m,B", [(16, 64, 2), (1000, 4096, 3), (2 ** 14, 2 ** 16, 2)])
def test_one_layer_plus_extra_fft(Plan, n, m, B):
    seed = 17 + n
    plan = Plan(n, m, 2, seed)
    theta = S.phases(seed, 2, m)
    theta[0] = 0.0  # the extra FFT: F D F U
    plan.set_phases(theta)
    x = S.signal_gaussian(seed, B, n)
    want = O.unitary_fft(np.exp(1j * theta[1]) * O.unitary_fft(O.zero_pad(x, m)))
    z = plan.forward(torch.from_numpy(x).to(torch.complex64).cuda()).cpu().numpy()
    plan.check()
    assert rel(z, want) <= 1e-5
    w = S.complex_gaussian(seed + 1, (B, m), S.STREAM_NOISE)
    want_a = O.unitary_ifft(np.exp(-1j * theta[1]) * O.unitary_ifft(w))[:, :n]
    xa = plan.adjoint(torch.from_numpy(w).to(torch.complex64).cuda()).cpu().numpy()
    plan.check()
    assert rel(xa, want_a) <= 1e-5


@pytest.mark.parametrize("n,m,L", [(100, 512, 2), (64, 192, 3), (512, 300, 2), (4000, 3 * 2 ** 13, 2)])
def test_batch_seeds_give_each_problem_its_own_operator(Plan, n, m, L):
    """Problem b of the batch uses the phases of seeds[b] (power-of-two, radix-3
    and alpha < 1 plans); a call with another batch size is refused."""
    seeds = [11, 2024, 77, 5]
    B = len(seeds)
    N = max(n, m)
    plan = Plan(n, m, L, 999)
    plan.set_batch_seeds(seeds)
    x = S.signal_gaussian(3, B, n)
    z = plan.forward(torch.from_numpy(x).to(torch.complex64).cuda()).cpu().numpy()
    w = S.complex_gaussian(4, (B, m), S.STREAM_NOISE)
    xa = plan.adjoint(torch.from_numpy(w).to(torch.complex64).cuda()).cpu().numpy()
    plan.check()
    for b, sd in enumerate(seeds):
        th = S.phases(sd, L, N)
        assert rel(z[b], O.forward(x[b], th, m)) <= 1e-5
        assert rel(xa[b], O.adjoint(w[b], th, n)) <= 1e-5
    with pytest.raises(Exception):
        plan.forward(torch.from_numpy(x[:2]).to(torch.complex64).cuda())
