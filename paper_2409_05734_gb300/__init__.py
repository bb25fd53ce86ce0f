"""GB300-native structured random phase retrieval (arXiv 2409.05734).

The operator A = F D_L ... F D_1 U of Sec. III (Eq. 5), its adjoint, the
loss/gradient of Eq. 2, the spectral initialisation of Eq. 3-4 and gradient
descent run in hand-written CUDA kernels for sm_103a behind a C ABI
(include/sr.h, libsr.so). This package is the thin Python binding.
"""
from .buildlib import build, library_path
from .plan import Plan, Plan2D, metrics, phases
from .autograd import StructuredRandomOp, structured_random
from .dense import DenseModel
from .ragged import Ragged

__all__ = ["Plan", "Plan2D", "metrics", "phases", "build", "library_path", "StructuredRandomOp", "structured_random",
           "DenseModel", "Ragged"]
