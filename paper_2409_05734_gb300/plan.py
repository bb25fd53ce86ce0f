"""Python binding of the C ABI: torch tensors in, torch tensors out.

Argument marshalling only -- every step of the operator and of the solvers
runs in the CUDA kernels of libsr.so. Complex arrays are torch.complex64
(interleaved re/im, the ABI's c64), real arrays torch.float32, all on the
plan's CUDA device and C-contiguous. Calls are enqueued on the current torch
stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib


def _stream_handle(stream=None) -> C.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


def _p(t) -> C.c_void_p:
    return C.c_void_p(t.data_ptr()) if t is not None else C.c_void_p(0)


class Plan:
    """Structured random operator A = F D_L ... F D_1 U (Sec. III, Eq. 5) on one GPU.

    m < n selects the alpha < 1 branch A = S F D_L ... F D_1: DFTs of length n,
    S keeping the m central entries. The phases have shape [L, N] with
    N = max(n, m), the DFT length."""

    def __init__(self, n: int, m: int, L: int = 2, seed: int = 0, device=None):
        self._lib = _lib.load()
        self.n, self.m, self.L, self.seed = int(n), int(m), int(L), int(seed)
        self.N = max(self.n, self.m)
        self._set_device(device)
        h = C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_create(self.n, self.m, self.L, self.seed, C.byref(h)), "sr_plan_create")
        self._h = h

    def _set_device(self, device):
        dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        if dev.type != "cuda":
            raise ValueError("a plan lives on a CUDA device")
        self.device = torch.device("cuda", dev.index if dev.index is not None else torch.cuda.current_device())

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sr_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ----------------------------------------------------------------- phases
    @property
    def phases(self) -> np.ndarray:
        out = np.empty((self.L, self.N), dtype=np.float64)
        _lib.check(self._lib.sr_plan_get_phases(self._h, out.ctypes.data_as(C.POINTER(C.c_double))),
                   "sr_plan_get_phases")
        return out

    def set_phases(self, theta) -> None:
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(self.L, self.N)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_set_phases(self._h, th.ctypes.data_as(C.POINTER(C.c_double))),
                       "sr_plan_set_phases")

    def set_batch_seeds(self, seeds) -> None:
        """Give problem b of every later call its own phases sr_phases(seeds[b], L, N)
        (independent random operators in one batch); later calls must use B = len(seeds)."""
        arr = (C.c_uint64 * len(seeds))(*[int(v) for v in seeds])
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_set_batch_phases(self._h, len(seeds), arr), "sr_plan_set_batch_phases")

    def check(self) -> None:
        """Synchronise and raise if a kernel of this plan recorded a device-side error."""
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_check(self._h), "sr_plan_check")

    def set_phases_device(self, theta: torch.Tensor) -> None:
        """Phases from a device float32 tensor [L, N]; tables rebuilt on the current stream."""
        if theta.dtype != torch.float32 or theta.device != self.device or tuple(theta.shape) != (self.L, self.N):
            raise ValueError(f"theta must be a float32 [{self.L}, {self.N}] tensor on {self.device}")
        theta = theta.contiguous()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_set_phases_device(self._h, _p(theta), _stream_handle()),
                       "sr_plan_set_phases_device")

    def backward(self, x: torch.Tensor, gz: torch.Tensor, need_x: bool = True, need_theta: bool = True):
        """(grad_x [B, n] or None, grad_theta [L, m] or None) of z = A x for the
        gradient gz of a real loss with respect to z (PyTorch's complex convention)."""
        x = self._c64(x, self.n, "x")
        gz = self._c64(gz, self.m, "gz")
        B = self._batch(x)
        gx = torch.empty_like(x) if need_x else None
        gth = torch.empty((self.L, self.m), dtype=torch.float32, device=self.device) if need_theta else None
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_backward(self._h, _p(x), _p(gz), _p(gx), _p(gth), B, _stream_handle()),
                       "sr_backward")
        return gx, gth

    def selftest_timeout(self) -> None:
        """Launch the failure-path probe: the next check() raises SR_ERR_TIMEOUT."""
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_selftest_timeout(self._h, _stream_handle()), "sr_plan_selftest_timeout")

    def autotune(self, B: int) -> None:
        """Choose the four-step split and the persistent grid size of the pass kernels for
        batches of B (timed on the GPU)."""
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_autotune(self._h, int(B), _stream_handle()), "sr_plan_autotune")

    def set_split(self, m1: int) -> None:
        """Factor the DFT length as m1 * (m / m1) (lines of m1 and m / m1 points)."""
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_set_split(self._h, int(m1)), "sr_plan_set_split")

    @property
    def tuning(self):
        """(m1, m2, CTAs per SM) of the four-step passes; CTAs per SM 0 = the kernels' occupancy."""
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        _lib.check(self._lib.sr_plan_tuning(self._h, C.byref(a), C.byref(b), C.byref(c)), "sr_plan_tuning")
        return a.value, b.value, c.value

    def reserve(self, B: int) -> None:
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_reserve(self._h, int(B)), "sr_plan_reserve")

    # ---------------------------------------------------------------- helpers
    def _c64(self, t, last: int, name: str):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex64:
            raise TypeError(f"{name} must be a torch.complex64 tensor")
        if t.device != self.device:
            raise ValueError(f"{name} must live on {self.device}")
        if t.shape[-1] != last or t.dim() not in (1, 2):
            raise ValueError(f"{name} must have shape [B, {last}] or [{last}]")
        if not t.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return t

    def _f32(self, t, last: int, name: str):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.float32:
            raise TypeError(f"{name} must be a torch.float32 tensor")
        if t.device != self.device or t.shape[-1] != last or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous [B, {last}] tensor on {self.device}")
        return t

    @staticmethod
    def _batch(t) -> int:
        return 1 if t.dim() == 1 else t.shape[0]

    # ------------------------------------------------------------- operators
    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """z = A x; x: complex64 [B, n] -> z: complex64 [B, m]."""
        x = self._c64(x, self.n, "x")
        B = self._batch(x)
        z = out if out is not None else torch.empty(x.shape[:-1] + (self.m,), dtype=torch.complex64, device=self.device)
        self._c64(z, self.m, "out")
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_forward(self._h, _p(x), _p(z), B, _stream_handle()), "sr_forward")
        return z

    def adjoint(self, z: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """x = A^H z; z: complex64 [B, m] -> x: complex64 [B, n]."""
        z = self._c64(z, self.m, "z")
        B = self._batch(z)
        x = out if out is not None else torch.empty(z.shape[:-1] + (self.n,), dtype=torch.complex64, device=self.device)
        self._c64(x, self.n, "out")
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_adjoint(self._h, _p(z), _p(x), B, _stream_handle()), "sr_adjoint")
        return x

    def loss_grad(self, x: torch.Tensor, y: torch.Tensor):
        """(loss [B], grad [B, n]) of L = || |Ax|^2 - y ||^2, grad = 2 A^H((|Ax|^2 - y) Ax) (Eq. 2)."""
        x = self._c64(x, self.n, "x")
        y = self._f32(y, self.m, "y")
        B = self._batch(x)
        loss = torch.empty(B, dtype=torch.float32, device=self.device)
        grad = torch.empty_like(x)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_loss_grad(self._h, _p(x), _p(y), _p(loss), _p(grad), B, _stream_handle()),
                       "sr_loss_grad")
        return loss, grad

    def spectral_init(self, y: torch.Tensor, v0: torch.Tensor, iters: int, weight: str = "optimal",
                      lam: float = -1.0, out: torch.Tensor | None = None) -> torch.Tensor:
        """Power iteration on M = A^H diag(T(y_hat)) A from v0 (Eq. 3-4); returns sqrt(sum y) v."""
        y = self._f32(y, self.m, "y")
        v0 = self._c64(v0, self.n, "v0")
        B = self._batch(v0)
        mode = {"identity": _lib.SR_WEIGHT_IDENTITY, "optimal": _lib.SR_WEIGHT_OPTIMAL}[weight]
        opts = _lib.SpectralOpts(mode, float(lam))
        x = out if out is not None else torch.empty_like(v0)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_spectral_init(self._h, _p(y), _p(v0), int(iters), C.byref(opts), _p(x), B,
                                                  _stream_handle()), "sr_spectral_init")
        return x

    def spectral_init_early_stop(self, y: torch.Tensor, v0: torch.Tensor, max_iters: int, rel_tol: float,
                                 check_every: int = 50, weight: str = "optimal", lam: float = -1.0,
                                 out: torch.Tensor | None = None):
        """Power iteration with early stopping: every check_every steps, stop once
        every problem's eigenvalue estimate ||M v + s v|| changed by <= rel_tol
        relative. Synchronises at each check. Returns (x, steps run)."""
        y = self._f32(y, self.m, "y")
        v0 = self._c64(v0, self.n, "v0")
        B = self._batch(v0)
        mode = {"identity": _lib.SR_WEIGHT_IDENTITY, "optimal": _lib.SR_WEIGHT_OPTIMAL}[weight]
        opts = _lib.SpectralOpts(mode, float(lam))
        x = out if out is not None else torch.empty_like(v0)
        run = C.c_int(0)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_spectral_init_early_stop(self._h, _p(y), _p(v0), int(max_iters), C.byref(opts),
                                                             float(rel_tol), int(check_every), _p(x), C.byref(run),
                                                             B, _stream_handle()), "sr_spectral_init_early_stop")
        return x, run.value

    def gd_solve(self, y: torch.Tensor, x: torch.Tensor, iters: int, mu0: float = 0.1, tau0: float = 0.0,
                 record_loss: bool = False, loss_hist: torch.Tensor | None = None):
        """In-place GD on x (Sec. II-B-1), step mu0 (1 - exp(-(t+1)/tau0)) m / sum(y)
        (constant when tau0 == 0); returns (x, loss history [iters, B] or None)."""
        y = self._f32(y, self.m, "y")
        x = self._c64(x, self.n, "x")
        B = self._batch(x)
        hist = loss_hist
        if hist is None and record_loss:
            hist = torch.empty((int(iters), B), dtype=torch.float32, device=self.device)
        opts = _lib.GdOpts(float(mu0), float(tau0))
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_gd_solve(self._h, _p(y), _p(x), int(iters), C.byref(opts), _p(hist), B,
                                             _stream_handle()), "sr_gd_solve")
        return x, hist

    def gd_solve_early_stop(self, y: torch.Tensor, x: torch.Tensor, max_iters: int, rel_tol: float,
                            check_every: int = 50, mu0: float = 0.1, tau0: float = 0.0, record_loss: bool = False):
        """GD with early stopping: every check_every iterations, stop once every
        problem's last relative loss change is <= rel_tol. Synchronises at each
        check. Returns (x, iterations run, loss history [run, B] or None)."""
        y = self._f32(y, self.m, "y")
        x = self._c64(x, self.n, "x")
        B = self._batch(x)
        hist = torch.empty((int(max_iters), B), dtype=torch.float32, device=self.device) if record_loss else None
        opts = _lib.GdOpts(float(mu0), float(tau0))
        run = C.c_int(0)
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_gd_solve_early_stop(self._h, _p(y), _p(x), int(max_iters), C.byref(opts),
                                                        float(rel_tol), int(check_every), _p(hist), C.byref(run),
                                                        B, _stream_handle()), "sr_gd_solve_early_stop")
        return x, run.value, (hist[:run.value] if hist is not None else None)


def phases(seed: int, L: int, m: int) -> np.ndarray:
    """Host-side phases a plan with this seed uses (sr_phases): float64 [L, m]."""
    lib = _lib.load()
    out = np.empty((L, m), dtype=np.float64)
    _lib.check(lib.sr_phases(int(seed), int(L), int(m), out.ctypes.data_as(C.POINTER(C.c_double))), "sr_phases")
    return out


def metrics(x_hat: torch.Tensor, x_ref: torch.Tensor):
    """(cosine similarity of Eq. 6, relative error up to a global phase) per
    problem of two complex64 [B, n] device tensors, as float32 [B] tensors on
    the same device (sr_metrics)."""
    lib = _lib.load()
    for name, t in (("x_hat", x_hat), ("x_ref", x_ref)):
        if not isinstance(t, torch.Tensor) or t.dtype != torch.complex64 or not t.is_cuda:
            raise TypeError(f"{name} must be a complex64 CUDA tensor")
    if x_hat.shape != x_ref.shape or x_hat.device != x_ref.device:
        raise ValueError("x_hat and x_ref must have the same shape and device")
    a = x_hat.reshape(-1, x_hat.shape[-1]).contiguous()
    b = x_ref.reshape(-1, x_ref.shape[-1]).contiguous()
    B, n = a.shape
    cos = torch.empty(B, dtype=torch.float32, device=a.device)
    err = torch.empty(B, dtype=torch.float32, device=a.device)
    with torch.cuda.device(a.device):
        _lib.check(lib.sr_metrics(_p(a), _p(b), n, B, _p(cos), _p(err), _stream_handle()), "sr_metrics")
    return cos, err


class Plan2D(Plan):
    """The 2D form of the operator (Sec. IV runs it with a 2D FFT on images):
    A = F2 D_L ... F2 D_1 U2 on h x w images (row-major, n = h*w) zero-padded
    into the top-left of an S x S grid (m = S*S, row-major). Same calls as
    Plan, except set_phases_device and backward."""

    def __init__(self, h: int, w: int, S: int, L: int = 2, seed: int = 0, device=None):
        self._lib = _lib.load()
        self.h, self.w, self.S = int(h), int(w), int(S)
        self.n, self.m, self.L, self.seed = self.h * self.w, self.S * self.S, int(L), int(seed)
        self.N = self.m
        self._set_device(device)
        hd = C.c_void_p()
        with torch.cuda.device(self.device):
            _lib.check(self._lib.sr_plan_create_2d(self.h, self.w, self.S, self.L, self.seed, C.byref(hd)),
                       "sr_plan_create_2d")
        self._h = hd
