"""sr_forward_noalloc against sr_forward and the FP64 oracle (GPU).

The no-allocation entry point serves callers that cannot allocate device
memory during the call, such as code capturing a CUDA graph or hosts whose
device memory belongs to their own allocator. It must give the same z = A x
as sr_forward, call after call, while reusing its fixed scratch array, and it
must refuse (before launching anything) every call it cannot serve. This file
is collected last so that a failing run has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu

# same tolerance as the parity tests: 1e-5 in norm, 2e-5 of the RMS per element
TOL_NORM, TOL_ELEM = 1e-5, 2e-5


def _ptr(t):
    return C.c_void_p(t.data_ptr())


def _close(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) <= TOL_NORM
    assert np.max(np.abs(got - ref)) <= TOL_ELEM * np.sqrt(np.mean(np.abs(ref) ** 2))


@pytest.fixture(scope="module")
def env():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2409_05734_gb300 import buildlib
    buildlib.build()
    from paper_2409_05734_gb300 import Plan, _lib
    lib = _lib.load()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return Plan, lib, stream


def test_forward_noalloc_matches_forward_on_consecutive_calls(env):
    Plan, lib, stream = env
    n, m, L, B = 3001, 2 ** 16, 2, 4   # B*m = 2^18, within the 2^19 limit; ragged n
    plan = Plan(n, m, L, 31)
    theta = S.phases(31, L, m)
    for call in range(2):
        xh = S.signal_gaussian(100 + call, B, n)
        x = torch.from_numpy(xh).to(torch.complex64).cuda()
        z_ref = plan.forward(x)
        z = torch.full_like(z_ref, float("nan"))
        st = lib.sr_forward_noalloc(plan._h, _ptr(x), _ptr(z), B, stream)
        assert st == 0, lib.sr_last_error().decode()
        plan.check()
        got = z.cpu().numpy()
        _close(got, z_ref.cpu().numpy())
        _close(got, O.forward(xh, theta, m))
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
    _close(z2.cpu().numpy(), plan2.forward(x2).cpu().numpy())


def test_forward_noalloc_one_layer(env):
    """L = 1: the first pass goes straight to the last (one DFT)."""
    Plan, lib, stream = env
    n, m, B = 700, 2 ** 12, 5
    plan = Plan(n, m, 1, 77)
    xh = S.signal_gaussian(3, B, n)
    x = torch.from_numpy(xh).to(torch.complex64).cuda()
    for _ in range(2):
        z = torch.full((B, m), float("nan"), dtype=torch.complex64, device="cuda")
        assert lib.sr_forward_noalloc(plan._h, _ptr(x), _ptr(z), B, stream) == 0, lib.sr_last_error().decode()
        plan.check()
        _close(z.cpu().numpy(), plan.forward(x).cpu().numpy())
        _close(z.cpu().numpy(), O.forward(xh, S.phases(77, 1, m), m))


def test_forward_noalloc_per_problem_phases(env):
    """A plan with per-problem phases accepts only its batch size: another B
    would index past the [B][L][m] diagonal tables, so it is refused."""
    Plan, lib, stream = env
    n, m, L = 5000, 2 ** 16, 2
    seeds = [101, 202]
    plan = Plan(n, m, L, seeds[0])
    plan.set_batch_seeds(seeds)
    x4 = torch.zeros(4, n, dtype=torch.complex64, device="cuda")
    z4 = torch.zeros(4, m, dtype=torch.complex64, device="cuda")
    assert lib.sr_forward_noalloc(plan._h, _ptr(x4), _ptr(z4), 4, stream) == 1
    assert "per-problem phases" in lib.sr_last_error().decode()
    xh = S.signal_gaussian(9, 2, n)
    x = torch.from_numpy(xh).to(torch.complex64).cuda()
    for _ in range(2):
        z = torch.full((2, m), float("nan"), dtype=torch.complex64, device="cuda")
        assert lib.sr_forward_noalloc(plan._h, _ptr(x), _ptr(z), 2, stream) == 0, lib.sr_last_error().decode()
        plan.check()
        got = z.cpu().numpy()
        _close(got, plan.forward(x).cpu().numpy())
        for b, sd in enumerate(seeds):
            _close(got[b], O.forward(xh[b:b + 1], S.phases(sd, L, m), m)[0])


@pytest.mark.parametrize("kind", ["2d", "radix3", "subsampled"])
def test_forward_noalloc_refuses_unsupported_plans(env, kind):
    """2D plans, m = 3 * 2^a and m < n return SR_ERR_UNSUPPORTED with the reason."""
    Plan, lib, stream = env
    from paper_2409_05734_gb300 import Plan2D
    if kind == "2d":
        plan, n, m, why = Plan2D(8, 8, 16, 2, 1), 64, 256, "2D"
    elif kind == "radix3":
        plan, n, m, why = Plan(64, 192, 2, 1), 64, 192, "power-of-two"
    else:
        plan, n, m, why = Plan(256, 200, 2, 1), 256, 200, "m < n"
    x = torch.zeros(1, n, dtype=torch.complex64, device="cuda")
    z = torch.zeros(1, m, dtype=torch.complex64, device="cuda")
    assert lib.sr_forward_noalloc(plan._h, _ptr(x), _ptr(z), 1, stream) == 2
    assert why in lib.sr_last_error().decode()
