"""Failure detection on the GPU without a GPU fault: a kernel's bounded wait on
an mbarrier that nothing completes gives up after the library's limit, records
SR_ERR_TIMEOUT, and returns; the host reads the status at the next check and
the context keeps working."""
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


def test_bounded_wait_gives_up_and_reports_timeout(sr):
    from paper_2409_05734_gb300._lib import SrError
    n, m, L = 16, 64, 2
    plan = sr.Plan(n, m, L, 3)
    plan.check()
    plan.selftest_timeout()
    with pytest.raises(SrError) as exc:
        plan.check()
    assert exc.value.status == 5  # SR_ERR_TIMEOUT
    plan.check()  # the status was cleared
    # the context is intact: the operator still matches the oracle
    x = S.signal_gaussian(1, 2, n)
    z = plan.forward(torch.from_numpy(x).to(torch.complex64).cuda()).cpu().numpy()
    zo = O.forward(x, S.phases(3, L, m), m)
    assert np.linalg.norm(z - zo) / np.linalg.norm(zo) <= 1e-5
    plan.check()


def test_ragged_queue_wait_gives_up_and_reports_timeout(sr):
    """The queue-driven ragged solve waits (bounded) for the tiles of the
    previous pass of each problem; with completion counts no pass can reach,
    every such wait gives up, the status reports SR_ERR_TIMEOUT, and the
    next solve still matches the oracle."""
    from paper_2409_05734_gb300._lib import SrError
    shapes = [(3000, 2 ** 14, 2), (5000, 2 ** 15, 1)]
    seeds = [11, 12]
    r = sr.Ragged([s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], seeds)
    r.check()
    r.selftest_timeout()
    with pytest.raises(SrError) as exc:
        r.check()
    assert exc.value.status == 5  # SR_ERR_TIMEOUT
    r.check()  # the status was cleared
    xs = [S.signal_gaussian(sd, 1, n)[0] for sd, (n, _, _) in zip(seeds, shapes)]
    ys = [np.abs(O.forward(x, S.phases(sd, L, m), m)) ** 2 for x, sd, (n, m, L) in zip(xs, seeds, shapes)]
    v0 = [S.start_vector(sd, 1, n)[0] for sd, (n, _, _) in zip(seeds, shapes)]
    y_cat = torch.from_numpy(r.pack(ys, "y")).float().cuda()
    x = r.spectral_init(y_cat, torch.from_numpy(r.pack(v0, "x")).to(torch.complex64).cuda(), 5, weight="optimal")
    r.check()
    xg = x.cpu().numpy()
    for i, (n, m, L) in enumerate(shapes):
        fwd, adj = O.structured_ops(S.phases(seeds[i], L, m), n, m)
        ref = O.spectral_init(ys[i][None], v0[i][None], fwd, adj, 5, mode="optimal")[0]
        got = xg[r.x_off[i]:r.x_off[i] + n]
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-4
