"""Python binding of the ragged-batch API of the C ABI: many independent
problems with their own sizes and phases (the recovery experiments of Sec. IV
solve many independent problems). Argument marshalling only."""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from .plan import _p, _stream_handle


class Ragged:
    """Independent problems i = 0..count-1 with sizes n[i], m[i], L[i] and phase
    seeds seeds[i], bucketed by shape inside the library."""

    def __init__(self, n, m, L, seeds, autotune: bool = False, device=None):
        self._lib = _lib.load()
        self.n = np.ascontiguousarray(n, dtype=np.int64)
        self.m = np.ascontiguousarray(m, dtype=np.int64)
        self.L = np.ascontiguousarray(L, dtype=np.int32)
        self.seeds = np.ascontiguousarray(seeds, dtype=np.uint64)
        self.count = len(self.n)
        if not (len(self.m) == len(self.L) == len(self.seeds) == self.count):
            raise ValueError("n, m, L and seeds must have the same length")
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.device = dev
        h = C.c_void_p()
        with torch.cuda.device(dev):
            _lib.check(self._lib.sr_ragged_create(
                self.count, self.n.ctypes.data_as(C.POINTER(C.c_int64)), self.m.ctypes.data_as(C.POINTER(C.c_int64)),
                self.L.ctypes.data_as(C.POINTER(C.c_int)), self.seeds.ctypes.data_as(C.POINTER(C.c_uint64)),
                int(bool(autotune)), C.byref(h)), "sr_ragged_create")
        self._h = h
        self.x_off = np.empty(self.count, dtype=np.int64)
        self.y_off = np.empty(self.count, dtype=np.int64)
        xt, yt, nb = C.c_int64(), C.c_int64(), C.c_int()
        _lib.check(self._lib.sr_ragged_layout(h, self.x_off.ctypes.data_as(C.POINTER(C.c_int64)),
                                              self.y_off.ctypes.data_as(C.POINTER(C.c_int64)), C.byref(xt),
                                              C.byref(yt), C.byref(nb)), "sr_ragged_layout")
        self.x_total, self.y_total, self.buckets = xt.value, yt.value, nb.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sr_ragged_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -------------------------------------------------------- concatenation
    def pack(self, arrays, kind: str) -> np.ndarray:
        """Concatenated host buffer in the library's layout from per-problem arrays."""
        off, size, total = (self.x_off, self.n, self.x_total) if kind == "x" else (self.y_off, self.m, self.y_total)
        dtype = np.result_type(*[np.asarray(a).dtype for a in arrays])
        out = np.zeros(total, dtype=dtype)
        for i, a in enumerate(arrays):
            out[off[i]:off[i] + size[i]] = np.asarray(a).reshape(-1)
        return out

    def unpack(self, flat, kind: str):
        off, size = (self.x_off, self.n) if kind == "x" else (self.y_off, self.m)
        return [flat[off[i]:off[i] + size[i]] for i in range(self.count)]

    # -------------------------------------------------------------- compute
    def check(self):
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_ragged_check(self._h), "sr_ragged_check")

    def selftest_timeout(self):
        """Run the queue-driven solve's failure-path probe: the next check() raises SR_ERR_TIMEOUT."""
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_ragged_selftest_timeout(self._h, _stream_handle()), "sr_ragged_selftest_timeout")

    def forward(self, x_cat: torch.Tensor) -> torch.Tensor:
        z = torch.empty(self.y_total, dtype=torch.complex64, device=self.device)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_ragged_forward(self._h, _p(x_cat), _p(z), _stream_handle()), "sr_ragged_forward")
        return z

    def spectral_init(self, y_cat: torch.Tensor, v0_cat: torch.Tensor, iters: int, weight: str = "optimal",
                      lam: float = -1.0, out: torch.Tensor | None = None) -> torch.Tensor:
        mode = {"identity": _lib.SR_WEIGHT_IDENTITY, "optimal": _lib.SR_WEIGHT_OPTIMAL}[weight]
        opts = _lib.SpectralOpts(mode, float(lam))
        x = out if out is not None else torch.empty_like(v0_cat)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_ragged_spectral_init(self._h, _p(y_cat), _p(v0_cat), int(iters), C.byref(opts),
                                                         _p(x), _stream_handle()), "sr_ragged_spectral_init")
        return x

    def reserve(self, iters: int):
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_ragged_reserve(self._h, int(iters)), "sr_ragged_reserve")

    def gd_solve(self, y_cat: torch.Tensor, x_cat: torch.Tensor, iters: int, mu0: float = 0.1, tau0: float = 0.0,
                 record_loss: bool = False, loss_hist: torch.Tensor | None = None):
        hist = loss_hist
        if hist is None and record_loss:
            self.reserve(iters)
            hist = torch.empty((int(iters), self.count), dtype=torch.float32, device=self.device)
        opts = _lib.GdOpts(float(mu0), float(tau0))
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_ragged_gd_solve(self._h, _p(y_cat), _p(x_cat), int(iters), C.byref(opts),
                                                    _p(hist), _stream_handle()), "sr_ragged_gd_solve")
        return x_cat, hist
