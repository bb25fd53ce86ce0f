"""sr_forward_noalloc against sr_forward (GPU).

The no-allocation entry point serves callers that cannot allocate device
memory during the call, such as code capturing a CUDA graph or hosts whose
device memory belongs to their own allocator. It must give the same z = A x
as sr_forward, call after call, while reusing its fixed scratch array. This
file is collected last so that a failing run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synthetic as S

pytestmark = pytest.mark.gpu


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def test_forward_noalloc_matches_forward_on_consecutive_calls():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2409_05734_gb300 import buildlib
    buildlib.build()
    from paper_2409_05734_gb300 import Plan, _lib
    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    n, m, L, B = 3001, 2 ** 16, 2, 4   # B*m = 2^18, within the 2^19 limit; ragged n
    plan = Plan(n, m, L, 31)
    for call in range(2):
        x = torch.from_numpy(S.signal_gaussian(100 + call, B, n)).to(torch.complex64).cuda()
        z_ref = plan.forward(x)
        z = torch.full_like(z_ref, float("nan"))
        st = lib.sr_forward_noalloc(plan._h, _ptr(x), _ptr(z), B, stream)
        assert st == 0, lib.sr_last_error().decode()
        plan.check()
        got, ref = z.cpu().numpy(), z_ref.cpu().numpy()
        # same tolerance as the parity tests: 1e-5 in norm, 2e-5 of the RMS per element
        assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= 1e-5
        assert np.max(np.abs(got - ref)) <= 2e-5 * np.sqrt(np.mean(np.abs(ref) ** 2))
    # a batch beyond the static scratch is refused without launching anything
    big = torch.zeros(9, n, dtype=torch.complex64, device="cuda")
    out = torch.zeros(9, m, dtype=torch.complex64, device="cuda")
    assert lib.sr_forward_noalloc(plan._h, _ptr(big), _ptr(out), 9, stream) == 2
    assert "exceeds the static scratch" in lib.sr_last_error().decode()
    # a smaller plan afterwards reuses the same scratch
    plan2 = Plan(64, 256, 3, 5)
    x2 = torch.from_numpy(S.signal_gaussian(7, 3, 64)).to(torch.complex64).cuda()
    z2 = torch.empty(3, 256, dtype=torch.complex64, device="cuda")
    assert lib.sr_forward_noalloc(plan2._h, _ptr(x2), _ptr(z2), 3, stream) == 0
    plan2.check()
    ref2 = plan2.forward(x2).cpu().numpy()
    assert np.linalg.norm(z2.cpu().numpy() - ref2) / np.linalg.norm(ref2) <= 1e-5
