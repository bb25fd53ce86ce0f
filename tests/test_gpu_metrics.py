"""GPU parity of the device metrics (sr_metrics) against the FP64 oracle.

cosine similarity (Eq. 6) and the relative error up to a global phase of
Sec. IV-A, per problem, on the same complex64 inputs the GPU receives. The
device sums are compensated FP32 and the error is summed directly at the
optimal phase, so the only deviation is FP32 rounding of the products:
|cos_gpu - cos_oracle| <= 1e-6 and |err_gpu - err_oracle| <= 1e-6 + 1e-5 err.
"""
import numpy as np
import pytest
import torch

import oracle as O
import synthetic as S

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def metrics():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    from paper_2409_05734_gb300 import buildlib
    buildlib.build()
    from paper_2409_05734_gb300 import metrics as M
    return M


def _c64(a):
    return np.ascontiguousarray(a).astype(np.complex64)


def _check(metrics, xh, xr):
    xh, xr = _c64(xh), _c64(xr)
    cos, err = metrics(torch.from_numpy(xh).cuda(), torch.from_numpy(xr).cuda())
    cos, err = cos.cpu().numpy().astype(np.float64), err.cpu().numpy().astype(np.float64)
    a, b = xh.astype(np.complex128), xr.astype(np.complex128)
    cos_o = O.cosine_similarity(a, b)
    err_o = O.relative_error_global_phase(a, b)
    assert np.all(np.abs(cos - cos_o) <= 1e-6), np.max(np.abs(cos - cos_o))
    assert np.all(np.abs(err - err_o) <= 1e-6 + 1e-5 * err_o), np.max(np.abs(err - err_o))
    return cos, err


# (n, B): one element, ragged lengths, one CTA per problem, clusters of 2..8 CTAs
@pytest.mark.parametrize("n,B", [(1, 3), (17, 4), (1000, 7), (16384, 5), (40000, 3), (100003, 2), (2 ** 20, 1)])
def test_metrics_match_oracle(metrics, n, B):
    xr = S.signal_gaussian(n + B, B, n)
    phi = np.exp(1j * 2 * np.pi * np.arange(B) / max(B, 1))[:, None]
    # estimates from far (independent) to very close to a rotated copy of the reference
    scale = np.logspace(0, -6, B)[:, None]
    noise = S.complex_gaussian(n + B + 1, (B, n), S.STREAM_NOISE)
    xh = phi * xr + scale * noise
    _check(metrics, xh, xr)


def test_metrics_edge_cases(metrics):
    n = 3000
    xr = S.signal_gaussian(5, 3, n)
    xh = xr.copy()
    xh[0] = 0.0                      # zero estimate: relative error 1, cosine undefined (NaN)
    xh[1] = 1j * xr[1]               # a pure global phase: error 0, cosine 1
    xh[2] = -xr[2] * (1 + 1e-3)      # rotation and scale
    cos, err = metrics(torch.from_numpy(_c64(xh)).cuda(), torch.from_numpy(_c64(xr)).cuda())
    cos, err = cos.cpu().numpy(), err.cpu().numpy()
    assert np.isnan(cos[0]) and abs(err[0] - 1.0) <= 1e-6
    assert abs(cos[1] - 1.0) <= 1e-6 and err[1] <= 1e-6
    assert abs(err[2] - 1e-3) <= 1e-6
    _check(metrics, xh[1:], xr[1:])


def test_metrics_deterministic_and_phase_blind(metrics):
    n, B = 70000, 4
    xr = torch.from_numpy(_c64(S.signal_gaussian(8, B, n))).cuda()
    xh = xr + 1e-2 * torch.from_numpy(_c64(S.complex_gaussian(9, (B, n), S.STREAM_NOISE))).cuda()
    c1, e1 = metrics(xh, xr)
    c2, e2 = metrics(xh, xr)
    assert torch.equal(c1, c2) and torch.equal(e1, e2)
    c3, e3 = metrics(xh * np.exp(0.7j), xr)
    assert torch.allclose(c1, c3, rtol=0, atol=1e-6) and torch.allclose(e1, e3, rtol=1e-4, atol=0)
