"""Every plan kind's solver calls can be captured in a CUDA graph once the
workspace is reserved (no allocation and no host synchronisation inside a
call), and a replay gives the eager result bit for bit: power-of-two and
radix-3 lengths, the alpha < 1 branch and the 2D model with odd L (whose
epilogues read a transposed copy of y made inside the call)."""
import numpy as np
import pytest
import torch

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


def _plans(sr):
    return [("pow2", sr.Plan(200, 1024, 2, 3)),
            ("radix3", sr.Plan(200, 768, 2, 4)),
            ("radix3 lines", sr.Plan(2000, 3 * 2 ** 13, 2, 8)),
            ("alpha<1", sr.Plan(1024, 700, 2, 5)),
            ("2d odd L", sr.Plan2D(20, 24, 32, 3, 6))]


@pytest.mark.parametrize("kind", ["pow2", "radix3", "radix3 lines", "alpha<1", "2d odd L"])
def test_solver_calls_capture_and_replay(sr, kind):
    plan = dict(_plans(sr))[kind]
    B = 3
    plan.reserve(B)
    x_true = torch.from_numpy(S.signal_gaussian(9, B, plan.n)).to(torch.complex64).cuda()
    y = (plan.forward(x_true).abs() ** 2).contiguous()
    v0 = torch.from_numpy(S.start_vector(9, B, plan.n)).to(torch.complex64).cuda()
    hist_e = torch.empty((12, B), device="cuda")
    hist_g = torch.empty((12, B), device="cuda")

    def solve(x, hist):
        plan.spectral_init(y, v0, 8, weight="optimal", out=x)
        plan.gd_solve(y, x, 12, mu0=0.05, tau0=5.0, loss_hist=hist)

    x_e = torch.empty_like(v0)
    solve(x_e, hist_e)
    x_g = torch.empty_like(v0)
    solve(x_g, hist_g)  # warm-up outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        solve(x_g, hist_g)
    x_g.zero_()
    g.replay()
    torch.cuda.synchronize()
    plan.check()
    assert torch.equal(x_e, x_g)
    assert torch.equal(hist_e, hist_g)
    assert torch.isfinite(x_g).all()
