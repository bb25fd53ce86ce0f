"""Python binding of the dense i.i.d. comparison model (Sec. II-A) of the C ABI.

Argument marshalling only; the products run in the library's tcgen05 GEMM.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from .plan import _p, _stream_handle


FORMATS = {"bf16": 0, "tf32": 1}


class DenseModel:
    """Dense A in C^{m x n}, the caller's entries rounded once to the operand
    format: "bf16" (to nearest even, tcgen05 kind::f16) or "tf32" (10 fraction
    bits, to nearest with ties away from zero, tcgen05 kind::tf32)."""

    def __init__(self, A: np.ndarray, device=None, format: str = "bf16"):
        if format not in FORMATS:
            raise ValueError(f"format must be one of {sorted(FORMATS)}")
        self.format = format
        A = np.asarray(A)
        if A.ndim != 2 or not np.iscomplexobj(A):
            raise ValueError("A must be a complex [m, n] array")
        self.m, self.n = A.shape
        self._lib = _lib.load()
        host = np.ascontiguousarray(np.stack([A.real, A.imag], axis=-1).astype(np.float32))
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        h = C.c_void_p()
        with torch.cuda.device(dev):
            _lib.check(self._lib.sr_dense_create_format(self.n, self.m, host.ctypes.data_as(C.c_void_p),
                                                        FORMATS[format], C.byref(h)), "sr_dense_create_format")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sr_dense_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self):
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_dense_check(self._h), "sr_dense_check")

    def forward(self, x: torch.Tensor) -> torch.Tensor:
        B = x.shape[0]
        z = torch.empty((B, self.m), dtype=torch.complex64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_dense_forward(self._h, _p(x.contiguous()), _p(z), B, _stream_handle()),
                       "sr_dense_forward")
        return z

    def adjoint(self, w: torch.Tensor) -> torch.Tensor:
        B = w.shape[0]
        x = torch.empty((B, self.n), dtype=torch.complex64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_dense_adjoint(self._h, _p(w.contiguous()), _p(x), B, _stream_handle()),
                       "sr_dense_adjoint")
        return x

    def spectral_init(self, y: torch.Tensor, v0: torch.Tensor, iters: int, weight: str = "optimal",
                      lam: float = -1.0, out: torch.Tensor | None = None) -> torch.Tensor:
        """Power iteration on M = A^H diag(T(y_hat)) A from v0 (Eq. 3-4); returns sqrt(sum y) v."""
        B = v0.shape[0]
        mode = {"identity": _lib.SR_WEIGHT_IDENTITY, "optimal": _lib.SR_WEIGHT_OPTIMAL}[weight]
        opts = _lib.SpectralOpts(mode, float(lam))
        x = out if out is not None else torch.empty_like(v0)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_dense_spectral_init(self._h, _p(y.contiguous()), _p(v0.contiguous()), int(iters),
                                                        C.byref(opts), _p(x), B, _stream_handle()),
                       "sr_dense_spectral_init")
        return x

    def gd_solve(self, y: torch.Tensor, x: torch.Tensor, iters: int, mu0: float = 0.1, tau0: float = 0.0,
                 record_loss: bool = False):
        B = x.shape[0]
        hist = torch.empty((int(iters), B), dtype=torch.float32, device=self.device) if record_loss else None
        opts = _lib.GdOpts(float(mu0), float(tau0))
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_dense_gd_solve(self._h, _p(y), _p(x), int(iters), C.byref(opts), _p(hist), B,
                                                   _stream_handle()), "sr_dense_gd_solve")
        return x, hist
