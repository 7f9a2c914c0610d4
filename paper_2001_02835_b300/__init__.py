"""Thin Python binding of libnspt.so, the B300 (sm_103a) NSPT polynomial-matrix library.

The library computes the truncated product of polynomial matrices
C_k = sum_{l<=k} A_l B_{k-l} (Eq. 5) naively or by FFT-CONV (Sec. 2, Steps 1-5),
its backward (truncated correlations), and one NSPT Langevin step of the
twisted Eguchi-Kawai model (Eqs. 1-3).  This module only marshals arguments:
it passes torch CUDA tensors' device pointers, sizes and the current stream to
the C ABI declared in include/nspt.h, and raises when a call fails.  Every
step of the path runs in the library's CUDA kernels; there is no CPU or
PyTorch fallback, and importing the package without the built library raises.

Series tensors are complex128, contiguous, shaped (batch, T+1, N, N) or
(T+1, N, N); link tensors for the Langevin step are (batch, 4, T+1, N, N).
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional

import torch

__all__ = [
    "lib", "library_path", "Opts", "NsptError",
    "polymat_mul", "polymat_mul_host", "polymat_mul_backward", "tek_langevin_step", "tek_md_trajectory", "tek_wilson_loops",
    "tek_unitarize", "tek_noise", "order_fft", "order_ifft",
    "workspace_size", "star", "PolymatMul",
    "ALGO_NAIVE", "ALGO_FFT", "ALGO_AUTO", "PREC_FP64", "PREC_SPLIT", "RESCALE_AUTO",
]

ALGO_NAIVE, ALGO_FFT, ALGO_AUTO = 0, 1, 2
PREC_FP64, PREC_SPLIT = 0, 1
OP_MUL, OP_MUL_BACKWARD, OP_LANGEVIN, OP_MD, OP_UNITARIZE = 0, 1, 2, 3, 4
RESCALE_AUTO = -1000

_HERE = os.path.dirname(os.path.abspath(__file__))
library_path = os.path.join(_HERE, "libnspt.so")
_lib = None


class NsptError(RuntimeError):
    """A libnspt call returned a negative status."""


class PolymatDesc(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("B", ctypes.c_void_p), ("C", ctypes.c_void_p),
                ("N", ctypes.c_int), ("T", ctypes.c_int), ("batch", ctypes.c_int)]


class Opts(ctypes.Structure):
    _fields_ = [
        ("algo", ctypes.c_int),
        ("prec", ctypes.c_int),
        ("fft_len", ctypes.c_int),
        ("slices", ctypes.c_int),
        ("complex_mode", ctypes.c_int),
        ("rescale_log2r", ctypes.c_int),
        ("workspace", ctypes.c_void_p),
        ("workspace_bytes", ctypes.c_size_t),
    ]


_vp, _i, _d, _sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
_SIGS = {
    "nspt_opts_default": (None, [ctypes.POINTER(Opts)]),
    "nspt_init": (_i, []),
    "nspt_workspace_size": (_sz, [_i, _i, _i, _i, ctypes.POINTER(Opts)]),
    "nspt_workspace_size_wilson": (_sz, [_i, _i, _i, _i, ctypes.POINTER(Opts)]),
    "nspt_workspace_size_host": (_sz, [_i, _i, _i, ctypes.POINTER(Opts)]),
    "nspt_debug_wait_budget": (_i, [ctypes.c_longlong]),
    "nspt_debug_pair_schedule": (_i, [_i, _i, ctypes.POINTER(ctypes.c_int), _i]),
    "nspt_polymat_mul_host": (_i, [_vp, _vp, _vp, _i, _i, _i, ctypes.POINTER(Opts), _vp]),
    "nspt_tek_wilson_loops": (_i, [_vp, _i, _i, _i, _i, _i, _vp, ctypes.POINTER(Opts), _vp]),
    "nspt_polymat_mul": (_i, [_vp, _vp, _vp, _i, _i, _i, ctypes.POINTER(Opts), _vp]),
    "nspt_polymat_mul_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, ctypes.POINTER(Opts), _vp]),
    "nspt_tek_langevin_step": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _d, ctypes.POINTER(Opts), _vp]),
    "nspt_tek_md_trajectory": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _d, _i, ctypes.POINTER(Opts), _vp]),
    "nspt_tek_unitarize": (_i, [_vp, _i, _i, _i, _i, ctypes.POINTER(Opts), _vp]),
    "nspt_tek_noise": (_i, [_vp, _i, _i, ctypes.c_ulonglong, ctypes.c_ulonglong, _vp, _vp]),
    "nspt_order_fft": (_i, [_vp, _vp, _i, _i, _i, _i, _vp]),
    "nspt_order_ifft": (_i, [_vp, _vp, _i, _i, _i, _i, _vp]),
    "nspt_status_string": (ctypes.c_char_p, [_i]),
    "nspt_launch_count": (ctypes.c_longlong, []),
    "nspt_profile_begin": (_i, [_i]),
    "nspt_profile_end": (_i, [_i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong)]),
    "nspt_stage_name": (ctypes.c_char_p, [_i]),
    "nspt_last_error": (ctypes.c_char_p, []),
    "nspt_device_status": (_i, [ctypes.POINTER(Opts), _vp]),
    "nspt_split_slices": (_i, [_vp, _vp, _vp, _i, _i, _i, _i, _i, _i, _vp]),
    "nspt_split_mode_gemm": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _i, _i, _vp, _vp]),
    "nspt_polymat_mul_fft_noalloc": (_i, [_vp, _vp, _vp, _i, _i, _i, _vp]),
    "nspt_workspace_size_grouped": (_sz, [_vp, _i, ctypes.POINTER(Opts)]),
    "nspt_polymat_mul_grouped": (_i, [_vp, _i, ctypes.POINTER(Opts), _vp]),
    "nspt_autotune_grouped": (_i, [_vp, _i, ctypes.POINTER(Opts), ctypes.c_char_p, ctypes.POINTER(ctypes.c_int), _vp]),
}


def lib() -> ctypes.CDLL:
    """Loads libnspt.so from the package directory (built by `build.py`)."""
    global _lib
    if _lib is None:
        if not os.path.exists(library_path):
            raise ImportError("libnspt.so is not built; run `python -m paper_2001_02835_b300.build`")
        L = ctypes.CDLL(library_path)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc: int, what: str):
    if rc != 0:
        L = lib()
        msg = L.nspt_status_string(rc).decode()
        if rc == -5:
            msg += " (" + L.nspt_last_error().decode() + ")"
        raise NsptError("%s failed: %s [%d]" % (what, msg, rc))


def _algo(a) -> int:
    return {"naive": ALGO_NAIVE, "fft": ALGO_FFT, "auto": ALGO_AUTO}.get(a, a)


def _prec(p) -> int:
    return {"fp64": PREC_FP64, "split": PREC_SPLIT}.get(p, p)


def make_opts(algo="auto", prec="fp64", fft_len=0, slices=0, rescale_log2r=0, complex_mode=0) -> Opts:
    o = Opts()
    lib().nspt_opts_default(ctypes.byref(o))
    o.algo = _algo(algo)
    o.prec = _prec(prec)
    o.fft_len = int(fft_len)
    o.slices = int(slices)
    o.rescale_log2r = int(rescale_log2r)
    o.complex_mode = int(complex_mode)
    return o


_ws_cache: dict = {}


def _workspace(nbytes: int, device: torch.device, tag: str = "") -> Optional[torch.Tensor]:
    if nbytes == 0:
        return None
    key = (device.index, torch.cuda.current_stream(device).cuda_stream, tag)
    buf = _ws_cache.get(key)
    if buf is None or buf.numel() < nbytes:
        buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        _ws_cache[key] = buf
    return buf


def _series_dims(X: torch.Tensor):
    if X.dim() == 3:
        return 1, X.shape[0] - 1, X.shape[1]
    if X.dim() == 4:
        return X.shape[0], X.shape[1] - 1, X.shape[2]
    raise ValueError("series tensor must be (batch, T+1, N, N) or (T+1, N, N)")


def _check_tensor(X: torch.Tensor, name: str):
    if not isinstance(X, torch.Tensor) or not X.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if X.dtype != torch.complex128:
        raise ValueError("%s must be complex128" % name)
    if not X.is_contiguous():
        raise ValueError("%s must be contiguous" % name)


def _stream_ptr(device) -> int:
    return torch.cuda.current_stream(device).cuda_stream


def workspace_size(op: int, N: int, T: int, batch: int, opts: Opts) -> int:
    return int(lib().nspt_workspace_size(op, N, T, batch, ctypes.byref(opts)))


def _with_ws(op, N, T, batch, opts, device):
    nbytes = workspace_size(op, N, T, batch, opts)
    ws = _workspace(nbytes, device)
    if ws is not None:
        opts.workspace = ws.data_ptr()
        opts.workspace_bytes = ws.numel()
    return ws


def polymat_mul(A: torch.Tensor, B: torch.Tensor, C: Optional[torch.Tensor] = None, **kw) -> torch.Tensor:
    """C = A star B (Eq. 5) through nspt_polymat_mul; kw: algo, prec, fft_len, slices, rescale_log2r,
    complex_mode (split form: 4, or 3 for three real products per complex product).  Both forms
    (algo "naive" or "fft") take prec "split"."""
    _check_tensor(A, "A")
    _check_tensor(B, "B")
    if A.shape != B.shape:
        raise ValueError("A and B must have the same shape")
    batch, T, N = _series_dims(A)
    if C is None:
        C = torch.empty_like(A)
    _check_tensor(C, "C")
    opts = make_opts(**kw)
    ws = _with_ws(OP_MUL, N, T, batch, opts, A.device)  # noqa: F841  (kept alive for the call)
    rc = lib().nspt_polymat_mul(A.data_ptr(), B.data_ptr(), C.data_ptr(), N, T, batch, ctypes.byref(opts),
                                _stream_ptr(A.device))
    _check(rc, "nspt_polymat_mul")
    return C


def polymat_mul_host(A: torch.Tensor, B: torch.Tensor, C: Optional[torch.Tensor] = None, device=None,
                     **kw) -> torch.Tensor:
    """C = A star B for CPU tensors (pinned for the copies to overlap the products) through
    nspt_polymat_mul_host on `device` (default: the current CUDA device); queued on that
    device's current stream -- synchronise it before reading C."""
    for t, name in ((A, "A"), (B, "B")):
        if t.device.type != "cpu" or t.dtype != torch.complex128 or not t.is_contiguous():
            raise ValueError("%s must be a contiguous complex128 CPU tensor" % name)
    if A.shape != B.shape:
        raise ValueError("A and B must have the same shape")
    batch, T, N = _series_dims(A)
    if C is None:
        C = torch.empty_like(A).pin_memory()
    dev = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
    opts = make_opts(**kw)
    nbytes = lib().nspt_workspace_size_host(N, T, batch, ctypes.byref(opts))
    # a workspace of its own: consecutive calls chain through its device slots
    ws = _workspace(nbytes, dev, "host")  # noqa: F841
    if ws is not None:
        opts.workspace = ws.data_ptr()
        opts.workspace_bytes = ws.numel()
    rc = lib().nspt_polymat_mul_host(A.data_ptr(), B.data_ptr(), C.data_ptr(), N, T, batch, ctypes.byref(opts),
                                     _stream_ptr(dev))
    _check(rc, "nspt_polymat_mul_host")
    return C


def polymat_mul_backward(A, B, gC, need_gA=True, need_gB=True, **kw):
    """(gA, gB) of C = A star B for upstream gradient gC (truncated correlations)."""
    for X, n in ((A, "A"), (B, "B"), (gC, "gC")):
        _check_tensor(X, n)
    batch, T, N = _series_dims(A)
    gA = torch.empty_like(A) if need_gA else None
    gB = torch.empty_like(B) if need_gB else None
    opts = make_opts(**kw)
    ws = _with_ws(OP_MUL_BACKWARD, N, T, batch, opts, A.device)  # noqa: F841
    rc = lib().nspt_polymat_mul_backward(A.data_ptr(), B.data_ptr(), gC.data_ptr(),
                                         gA.data_ptr() if gA is not None else None,
                                         gB.data_ptr() if gB is not None else None,
                                         N, T, batch, ctypes.byref(opts), _stream_ptr(A.device))
    _check(rc, "nspt_polymat_mul_backward")
    return gA, gB


def tek_langevin_step(U: torch.Tensor, eta: torch.Tensor, flux: int, eps: float, want_drift: bool = False, **kw):
    """One Langevin step in place on U (batch, 4, T+1, N, N) with noise eta (batch, 4, N, N).
    Returns (U, F) with F the drift of the input links when want_drift.  kw: algo, prec, fft_len,
    slices, rescale_log2r (per-order rescale of the step's order transforms; RESCALE_AUTO fits it)."""
    _check_tensor(U, "U")
    _check_tensor(eta, "eta")
    if U.dim() != 5 or U.shape[1] != 4:
        raise ValueError("U must be (batch, 4, T+1, N, N)")
    batch, T, N = U.shape[0], U.shape[2] - 1, U.shape[3]
    if tuple(eta.shape) != (batch, 4, N, N):
        raise ValueError("eta must be (batch, 4, N, N)")
    F = torch.empty_like(U) if want_drift else None
    opts = make_opts(**kw)
    ws = _with_ws(OP_LANGEVIN, N, T, batch, opts, U.device)  # noqa: F841
    rc = lib().nspt_tek_langevin_step(U.data_ptr(), eta.data_ptr(), F.data_ptr() if F is not None else None,
                                      N, T, batch, int(flux), float(eps), ctypes.byref(opts), _stream_ptr(U.device))
    _check(rc, "nspt_tek_langevin_step")
    return U, F


def tek_noise(N: int, count: int, seed: int, counter: int = 0, d_counter: Optional[torch.Tensor] = None,
              out: Optional[torch.Tensor] = None, device="cuda") -> torch.Tensor:
    """`count` traceless Hermitian N x N noise matrices (complex128, (count, N, N)) from the
    counter-based generator of nspt_tek_noise, keyed by seed and counter; with d_counter (a
    one-element int64 tensor on the device) the counter is counter + d_counter, advanced by one
    per call on the device, so that a captured graph draws fresh noise at every replay."""
    if out is None:
        out = torch.empty((count, N, N), dtype=torch.complex128, device=device)
    _check_tensor(out, "out")
    if tuple(out.shape[-3:]) != (count, N, N) or out.numel() != count * N * N:
        raise ValueError("out must hold (count, N, N) complex128")
    if d_counter is not None and (d_counter.dtype != torch.int64 or d_counter.numel() != 1
                                  or d_counter.device != out.device):
        raise ValueError("d_counter must be a one-element int64 tensor on the output's device")
    rc = lib().nspt_tek_noise(out.data_ptr(), int(N), int(count), int(seed) & (2 ** 64 - 1),
                              int(counter) & (2 ** 64 - 1), d_counter.data_ptr() if d_counter is not None else None,
                              _stream_ptr(out.device))
    _check(rc, "nspt_tek_noise")
    return out


def tek_md_trajectory(U: torch.Tensor, P: torch.Tensor, flux: int, eps: float, nsteps: int,
                      eta: Optional[torch.Tensor] = None, **kw):
    """Leapfrog molecular dynamics in place on U and P (batch, 4, T+1, N, N); with eta
    (batch, 4, N, N) the momentum is refreshed to P^(1) = eta first.  Returns (U, P).  kw as for
    tek_langevin_step; with rescale_log2r=RESCALE_AUTO every phase fits its own rescale (one
    stream synchronisation per phase)."""
    _check_tensor(U, "U")
    _check_tensor(P, "P")
    if U.shape != P.shape or U.dim() != 5 or U.shape[1] != 4:
        raise ValueError("U and P must be (batch, 4, T+1, N, N)")
    batch, T, N = U.shape[0], U.shape[2] - 1, U.shape[3]
    if eta is not None:
        _check_tensor(eta, "eta")
        if tuple(eta.shape) != (batch, 4, N, N):
            raise ValueError("eta must be (batch, 4, N, N)")
    opts = make_opts(**kw)
    ws = _with_ws(OP_MD, N, T, batch, opts, U.device)  # noqa: F841
    rc = lib().nspt_tek_md_trajectory(U.data_ptr(), P.data_ptr(), eta.data_ptr() if eta is not None else None, N, T,
                                      batch, int(flux), float(eps), int(nsteps), ctypes.byref(opts),
                                      _stream_ptr(U.device))
    _check(rc, "nspt_tek_md_trajectory")
    return U, P


def tek_unitarize(U: torch.Tensor, special: bool = False, **kw) -> torch.Tensor:
    """Unitarity projection in place: every series of U ((..., T+1, N, N), e.g. links
    (batch, 4, T+1, N, N)) becomes its polar factor U * (U^+ U)^(-1/2) in the truncated ring,
    order 0 kept; with special=True its U(1) phase is removed too (det U = det U^(0) through
    order T; see include/nspt.h).  kw: algo, prec, fft_len, slices, rescale_log2r."""
    _check_tensor(U, "U")
    if U.dim() < 3 or U.shape[-1] != U.shape[-2]:
        raise ValueError("U must be (..., T+1, N, N)")
    T, N = U.shape[-3] - 1, U.shape[-1]
    nser = U.numel() // ((T + 1) * N * N)
    opts = make_opts(**kw)
    ws = _with_ws(OP_UNITARIZE, N, T, nser, opts, U.device)  # noqa: F841
    rc = lib().nspt_tek_unitarize(U.data_ptr(), N, T, nser, int(bool(special)), ctypes.byref(opts),
                                  _stream_ptr(U.device))
    _check(rc, "nspt_tek_unitarize")
    return U


def tek_wilson_loops(U: torch.Tensor, flux: int, amax: int, **kw) -> torch.Tensor:
    """Perturbative Wilson loops W (batch, amax, amax, T+1) complex128 of the links U
    (batch, 4, T+1, N, N), W[b, a-1, c-1, k] = W(a, c)^(k) (see include/nspt.h)."""
    _check_tensor(U, "U")
    if U.dim() != 5 or U.shape[1] != 4:
        raise ValueError("U must be (batch, 4, T+1, N, N)")
    batch, T, N = U.shape[0], U.shape[2] - 1, U.shape[3]
    W = torch.empty((batch, amax, amax, T + 1), dtype=torch.complex128, device=U.device)
    opts = make_opts(**kw)
    nbytes = lib().nspt_workspace_size_wilson(N, T, batch, int(amax), ctypes.byref(opts))
    if nbytes == 0:
        raise ValueError("unsupported Wilson-loop sizes")
    ws = _workspace(nbytes, U.device)  # noqa: F841
    if ws is not None:
        opts.workspace = ws.data_ptr()
        opts.workspace_bytes = ws.numel()
    rc = lib().nspt_tek_wilson_loops(U.data_ptr(), N, T, batch, int(flux), int(amax), W.data_ptr(),
                                     ctypes.byref(opts), _stream_ptr(U.device))
    _check(rc, "nspt_tek_wilson_loops")
    return W


def order_fft(A: torch.Tensor, M: int) -> torch.Tensor:
    """Steps 1-2: zero-pad to M and transform along the order axis (w = exp(+2 pi i/M))."""
    _check_tensor(A, "A")
    batch, T, N = _series_dims(A)
    At = torch.empty((batch, M, N, N), dtype=A.dtype, device=A.device)
    _check(lib().nspt_order_fft(A.data_ptr(), At.data_ptr(), N, T, batch, M, _stream_ptr(A.device)), "nspt_order_fft")
    return At


def order_ifft(Ct: torch.Tensor, T: int) -> torch.Tensor:
    """Steps 4-5: inverse transform with 1/M and keep orders 0..T."""
    _check_tensor(Ct, "Ct")
    batch, M, N = Ct.shape[0], Ct.shape[1], Ct.shape[2]
    C = torch.empty((batch, T + 1, N, N), dtype=Ct.dtype, device=Ct.device)
    _check(lib().nspt_order_ifft(Ct.data_ptr(), C.data_ptr(), N, T, batch, M, _stream_ptr(Ct.device)),
           "nspt_order_ifft")
    return C


NSTAGES = 10


def launch_count() -> int:
    """Kernel launches enqueued by the library since it was loaded."""
    return int(lib().nspt_launch_count())


def profile_begin(max_records: int = 100000):
    """Bracket every library kernel launch with CUDA events on its own stream."""
    _check(lib().nspt_profile_begin(int(max_records)), "nspt_profile_begin")


def profile_end() -> dict:
    """Per-stage totals since profile_begin: {stage: (total_ms, launches)}."""
    ms = (ctypes.c_double * NSTAGES)()
    n = (ctypes.c_longlong * NSTAGES)()
    rc = lib().nspt_profile_end(NSTAGES, ms, n)
    if rc < 0:
        _check(rc, "nspt_profile_end")
    return {lib().nspt_stage_name(i).decode(): (ms[i], int(n[i])) for i in range(NSTAGES) if n[i]}


def split_slices(X: torch.Tensor, S: int, trans: bool = False, conj: bool = False, right: bool = False):
    """Stage entry: digit slices (bf16 (Q, S, P, N, Kp), P = 3 for a right operand, else 2)
    and row exponents (int32 (Q, N)) of the Q matrices X (Q, N, N) complex128 (see include/nspt.h)."""
    _check_tensor(X, "X")
    Q, N = X.shape[0], X.shape[1]
    Kp = (N + 7) // 8 * 8
    sl = torch.zeros((Q, S, 3 if right else 2, N, Kp), dtype=torch.bfloat16, device=X.device)
    ex = torch.empty((Q, N), dtype=torch.int32, device=X.device)
    _check(lib().nspt_split_slices(X.data_ptr(), sl.data_ptr(), ex.data_ptr(), N, Q, S, int(trans), int(conj),
                                   int(right), _stream_ptr(X.device)), "nspt_split_slices")
    return sl, ex


def split_mode_gemm(slA: torch.Tensor, slB: torch.Tensor, expA: torch.Tensor, expB: torch.Tensor, N: int,
                    S: int) -> torch.Tensor:
    """Stage entry: mode GEMMs from digit slices (see include/nspt.h).
    Returns Ct as float32 (Q, N, N, 4) = (re_hi, re_lo, im_hi, im_lo)."""
    Q = expA.shape[0]
    Ct = torch.empty((Q, N, N, 4), dtype=torch.float32, device=slA.device)
    err = torch.zeros(1, dtype=torch.int32, device=slA.device)
    rc = lib().nspt_split_mode_gemm(slA.data_ptr(), slB.data_ptr(), expA.data_ptr(), expB.data_ptr(), Ct.data_ptr(),
                                    N, Q, S, err.data_ptr(), _stream_ptr(slA.device))
    _check(rc, "nspt_split_mode_gemm")
    if int(err.item()) != 0:
        raise NsptError("nspt_split_mode_gemm: device wait timed out (code %d)" % int(err.item()))
    return Ct


def _group_descs(As, Bs, Cs):
    if not (len(As) == len(Bs) == len(Cs)) or not As:
        raise ValueError("need equally many A, B, C tensors")
    arr = (PolymatDesc * len(As))()
    for i, (A, B, C) in enumerate(zip(As, Bs, Cs)):
        for X, n in ((A, "A"), (B, "B"), (C, "C")):
            _check_tensor(X, n)
        if A.shape != B.shape or A.shape != C.shape:
            raise ValueError("product %d: A, B, C shapes differ" % i)
        batch, T, N = _series_dims(A)
        arr[i] = PolymatDesc(A.data_ptr(), B.data_ptr(), C.data_ptr(), N, T, batch)
    return arr


def _group_ws(arr, count, opts, device):
    nbytes = int(lib().nspt_workspace_size_grouped(arr, count, ctypes.byref(opts)))
    ws = _workspace(nbytes, device)
    if ws is not None:
        opts.workspace = ws.data_ptr()
        opts.workspace_bytes = ws.numel()
    return ws


def polymat_mul_grouped(As, Bs, Cs=None, **kw):
    """C_i = A_i star B_i for a list of products of uneven (N, T) (nspt_polymat_mul_grouped);
    kw: prec ('split' runs all mode GEMMs in one persistent tensor-core launch), slices, rescale_log2r."""
    if Cs is None:
        Cs = [torch.empty_like(A) for A in As]
    arr = _group_descs(As, Bs, Cs)
    opts = make_opts(algo="fft", **kw)
    ws = _group_ws(arr, len(As), opts, As[0].device)  # noqa: F841
    _check(lib().nspt_polymat_mul_grouped(arr, len(As), ctypes.byref(opts), _stream_ptr(As[0].device)),
           "nspt_polymat_mul_grouped")
    return Cs


def autotune_grouped(As, Bs, cache_path=None, **kw) -> int:
    """Times the tile widths of the split form's grouped GEMM for this group and keeps the
    fastest for later calls with the same signature; returns the chosen width."""
    Cs = [torch.empty_like(A) for A in As]
    arr = _group_descs(As, Bs, Cs)
    opts = make_opts(algo="fft", prec="split", **kw)
    ws = _group_ws(arr, len(As), opts, As[0].device)  # noqa: F841
    chosen = ctypes.c_int(0)
    path = cache_path.encode() if cache_path else None
    _check(lib().nspt_autotune_grouped(arr, len(As), ctypes.byref(opts), path, ctypes.byref(chosen),
                                       _stream_ptr(As[0].device)), "nspt_autotune_grouped")
    return int(chosen.value)


class PolymatMul(torch.autograd.Function):
    """Autograd wrapper: forward = nspt_polymat_mul, backward = nspt_polymat_mul_backward
    (PyTorch's convention grad = dL/dRe + i dL/dIm)."""

    @staticmethod
    def forward(ctx, A, B, kw):
        A = A.contiguous()
        B = B.contiguous()
        ctx.save_for_backward(A, B)
        ctx.kw = kw
        return polymat_mul(A, B, **kw)

    @staticmethod
    def backward(ctx, gC):
        A, B = ctx.saved_tensors
        gA, gB = polymat_mul_backward(A, B, gC.contiguous(), ctx.needs_input_grad[0], ctx.needs_input_grad[1], **ctx.kw)
        return gA, gB, None


def star(A: torch.Tensor, B: torch.Tensor, **kw) -> torch.Tensor:
    """Differentiable truncated product A star B."""
    return PolymatMul.apply(A, B, kw)
