"""GPU parity of every four-step split the passes support (sr_plan_set_split)
and of the split the autotuner picks, against the FP64 oracle.

A split m = m1 * m2 only changes how the DFT is factored (Sec. III states the
DFT, not its factorisation), so every split must give the oracle's A, A^H and
GD iterates within the usual tolerances: 1e-5 in norm and 2e-5 of the RMS per
element for one operator application, 1e-4 for a short GD run.
"""
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


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def close(got, ref, tol_norm=1e-5, tol_elem=2e-5):
    assert rel(got, ref) <= tol_norm, rel(got, ref)
    assert np.max(np.abs(got - ref)) <= tol_elem * np.sqrt(np.mean(np.abs(ref) ** 2))


# (n, m, L, B, m1): the balanced split and its neighbours; odd and even log2(m);
# several tiles per pass and a ragged n
SPLITS = [(3000, 2 ** 14, 2, 3, m1) for m1 in (64, 128, 256)] + \
         [(5000, 2 ** 15, 3, 2, m1) for m1 in (128, 256, 512)] + \
         [(20000, 2 ** 16, 2, 2, m1) for m1 in (128, 256, 512)] + \
         [(40000, 2 ** 17, 1, 2, m1) for m1 in (256, 512, 1024)]


@pytest.mark.parametrize("n,m,L,B,m1", SPLITS)
def test_split_operator_and_gd_match_oracle(sr, n, m, L, B, m1):
    seed = 7 + m1
    plan = sr.Plan(n, m, L, seed)
    plan.set_split(m1)
    got_m1, got_m2, _ = plan.tuning
    assert (got_m1, got_m2) == (m1, m // m1)
    th = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(th, n, m)
    x = S.signal_gaussian(seed, B, n)
    z = plan.forward(dev(x)).cpu().numpy()
    plan.check()
    close(z, fwd(x))
    w = S.complex_gaussian(seed, (B, m), S.STREAM_NOISE)
    close(plan.adjoint(dev(w)).cpu().numpy(), adj(w))
    # a short GD run from a point near the signal
    y = np.abs(fwd(x)) ** 2
    x0 = x + 0.3 * S.complex_gaussian(seed + 1, (B, n), S.STREAM_NOISE)
    xg = dev(x0)
    plan.gd_solve(dev(y, torch.float32), xg, 10, mu0=0.1)
    plan.check()
    xo, _ = O.gradient_descent(x0, y, fwd, adj, 10, mu0=0.1)
    assert rel(xg.cpu().numpy(), xo) <= 1e-4


def test_autotune_picks_a_supported_split_and_keeps_results(sr):
    n, m, L, B, seed = 30000, 2 ** 17, 2, 4, 99
    plan = sr.Plan(n, m, L, seed)
    plan.reserve(B)
    plan.autotune(B)
    m1, m2, c = plan.tuning
    assert m1 * m2 == m and m1 in (256, 512, 1024) and c >= 1
    th = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(th, n, m)
    x = S.signal_gaussian(seed, B, n)
    close(plan.forward(dev(x)).cpu().numpy(), fwd(x))
    plan.check()


def test_split_on_radix3_plan(sr):
    n, m, L, B, seed = 2000, 3 * 2 ** 14, 2, 2, 5
    plan = sr.Plan(n, m, L, seed)
    assert plan.tuning[:2] == (192, 256)  # the default: radix-3 lines of 192 in layout X
    plan.set_split(256)   # lines of 256 in layout X, radix-3 lines of 192 in layout Y
    assert plan.tuning[:2] == (256, 192)
    fwd, adj = O.structured_ops(S.phases(seed, L, m), n, m)
    x = S.signal_gaussian(seed, B, n)
    close(plan.forward(dev(x)).cpu().numpy(), fwd(x))
    plan.check()


def test_split_keeps_per_problem_phases_and_capacity(sr):
    n, m, L, seeds = 5000, 2 ** 16, 2, [11, 12, 13]
    plan = sr.Plan(n, m, L, seeds[0])
    plan.set_batch_seeds(seeds)
    plan.reserve(3)
    plan.set_split(512)
    x = S.signal_gaussian(4, 3, n)
    z = plan.forward(dev(x)).cpu().numpy()
    plan.check()
    for b, sd in enumerate(seeds):
        close(z[b], O.forward(x[b:b + 1], S.phases(sd, L, m), m)[0])


def test_unsupported_splits_are_refused(sr):
    from paper_2409_05734_gb300._lib import SrError
    plan = sr.Plan(3000, 2 ** 14, 2, 1)
    for bad in (3, 2 ** 15, 1):
        with pytest.raises(SrError):
            plan.set_split(bad)
    assert plan.tuning[:2] == (128, 128)  # unchanged
    with pytest.raises(SrError):
        sr.Plan2D(8, 8, 16, 2, 1).set_split(8)


# Radix-3 lengths on the four-step passes: lines of 192, 384 or 768 points (a
# radix-3 step inside the line FFT) in either layout, several tiles per pass,
# ragged n, L = 1 .. 3.
R3_SPLITS = [(3000, 3 * 2 ** 14, 2, 3, m1) for m1 in (192, 256, 384)] + \
            [(30000, 3 * 2 ** 16, 3, 2, m1) for m1 in (384, 512, 768)] + \
            [(9000, 3 * 2 ** 13, 1, 2, 192), (2 ** 16, 3 * 2 ** 17, 2, 1, 768)]


@pytest.mark.parametrize("n,m,L,B,m1", R3_SPLITS)
def test_radix3_line_splits_match_oracle(sr, n, m, L, B, m1):
    seed = 50 + m1 + L
    plan = sr.Plan(n, m, L, seed)
    plan.set_split(m1)
    got_m1, got_m2, _ = plan.tuning
    assert (got_m1, got_m2) == (m1, m // m1)
    th = S.phases(seed, L, m)
    fwd, adj = O.structured_ops(th, n, m)
    x = S.signal_gaussian(seed, B, n)
    close(plan.forward(dev(x)).cpu().numpy(), fwd(x))
    plan.check()
    w = S.complex_gaussian(seed, (B, m), S.STREAM_NOISE)
    close(plan.adjoint(dev(w)).cpu().numpy(), adj(w))
    y = np.abs(fwd(x)) ** 2
    x0 = x + 0.3 * S.complex_gaussian(seed + 1, (B, n), S.STREAM_NOISE)
    xg = dev(x0)
    plan.gd_solve(dev(y, torch.float32), xg, 10, mu0=0.1)
    plan.check()
    xo, _ = O.gradient_descent(x0, y, fwd, adj, 10, mu0=0.1)
    assert rel(xg.cpu().numpy(), xo) <= 1e-4
    # the power iteration (spectral epilogue between the forward and inverse DFTs)
    v0 = S.start_vector(seed, B, n)
    xs = plan.spectral_init(dev(y, torch.float32), dev(v0), 5, weight="optimal", lam=-1.0).cpu().numpy()
    plan.check()
    assert rel(xs, O.spectral_init(y, v0, fwd, adj, 5, mode="optimal", lam=-1.0)) <= 1e-4
