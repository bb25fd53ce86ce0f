"""Dense i.i.d. random comparison model (Sec. II-A), FP64.

Test infrastructure only (see the package docstring).

A in C^{m x n} with i.i.d. entries (CN(0, 1/m) in the tests); the forward
model is the plain product z = A x and the adjoint is A^H w. These are the
operations the paper compares against in Sec. IV (accuracy, Fig. 2; cost,
Fig. 4).
"""
from __future__ import annotations

import numpy as np


def dense_forward(A: np.ndarray, x: np.ndarray) -> np.ndarray:
    """z = A x for x of shape [..., n]; returns [..., m]."""
    return np.asarray(x, dtype=np.complex128) @ A.T


def dense_adjoint(A: np.ndarray, w: np.ndarray) -> np.ndarray:
    """A^H w for w of shape [..., m]; returns [..., n]."""
    return np.asarray(w, dtype=np.complex128) @ np.conj(A)


def dense_ops(A: np.ndarray):
    """(fwd, adj) callables of the dense model."""
    return (lambda x: dense_forward(A, x)), (lambda w: dense_adjoint(A, w))
