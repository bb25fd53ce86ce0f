"""FP64 CPU oracle for the structured random phase-retrieval model (arXiv 2409.05734).

TEST INFRASTRUCTURE ONLY. Nothing in the product path imports, calls or links
this package: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline
leg of ``bench.py`` may use it. It shares no code with the CUDA library; the
only module both sides use is ``synthetic`` (seeded random draws, none of the
method's arithmetic).

What it computes, in float64 / complex128, following the paper step by step:

* ``operator``  -- the unitary DFT F (naive O(m^2) matrix, and the library FFT as
  a step), the structured sensing operator A = F D_L ... F D_1 U of Sec. III,
  Eq. 5 (alpha > 1 branch) and its adjoint, and an explicitly materialised
  dense copy of A for tiny sizes.
* ``operator2d`` -- the same model on h x w images with the unitary 2D DFT of
  an S x S zero-padded grid (the form the experiments of Sec. IV run).
* ``recovery``  -- the l2 intensity loss and its gradient (Sec. II-B-1, Eq. 2),
  the spectral initialisation by shifted power iteration on the weighted
  covariance (Sec. II-B-2, Eq. 3-4), gradient descent (Sec. IV-A), and the
  accuracy metrics (cosine similarity, Eq. 6; relative error up to a global
  phase).
* ``dense_iid`` -- the i.i.d. random comparison model (Sec. II-A) as plain
  matrix products.
* ``autodiff`` -- the backward pass of z = A x with respect to x and the
  diffuser phases theta_l, by the chain rule written out layer by layer.

Pins: every function here is checked by ``tests/test_oracle_*.py`` against
closed forms, invariants, brute-force sums and library special cases (not
against itself). The recovery-rate-versus-alpha curves of Sec. IV are only
qualitative in the paper (its figures are not reproduced in the text), so
their parity is unpinned beyond the monotonicity and layer-count checks.
"""
from .operator import (
    dft_matrix,
    dft_naive,
    unitary_fft,
    unitary_ifft,
    zero_pad,
    trim,
    untrim,
    trim_offset,
    forward,
    adjoint,
    dense_structured_matrix,
)
from .recovery import (
    intensity_loss,
    loss_and_grad,
    spectral_weights,
    spectral_init,
    spectral_init_early_stop,
    gradient_descent,
    gradient_descent_early_stop,
    step_ramp,
    cosine_similarity,
    relative_error_global_phase,
    structured_ops,
)
from .operator2d import (
    unitary_fft2,
    unitary_ifft2,
    zero_pad_2d,
    crop_2d,
    forward_2d,
    adjoint_2d,
    dense_structured_matrix_2d,
    structured_ops_2d,
)
from .dense_iid import dense_forward, dense_adjoint, dense_ops
from . import autodiff

__all__ = [
    "dft_matrix", "dft_naive", "unitary_fft", "unitary_ifft", "zero_pad", "trim", "untrim", "trim_offset", "forward",
    "adjoint", "dense_structured_matrix", "intensity_loss", "loss_and_grad",
    "spectral_weights", "spectral_init", "spectral_init_early_stop", "gradient_descent", "gradient_descent_early_stop", "step_ramp", "cosine_similarity",
    "relative_error_global_phase", "structured_ops", "dense_forward", "dense_adjoint",
    "dense_ops", "autodiff", "unitary_fft2", "unitary_ifft2", "zero_pad_2d", "crop_2d",
    "forward_2d", "adjoint_2d", "dense_structured_matrix_2d", "structured_ops_2d",
]
