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
