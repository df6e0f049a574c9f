"""Thin ctypes binding of ``libhs.so`` (argument marshalling only).

The functions keep the C names (``hs_plan``, ``hs_assemble``, ...).  Tensors
are torch CUDA tensors in the ABI's column-major layout:

* ``A``, ``B``: complex128, shape ``(K, N_G)``, strides ``(1, ld)`` with
  ``ld >= K`` (e.g. ``torch.empty(N_G, K, dtype=torch.complex128).T``);
* ``T_AA``, ``T_AB``, ``T_BB``: complex128, shape ``(N_A, N_L, N_L)``,
  strides ``(N_L*N_L, 1, N_L)`` (each block column-major);
* ``U``: float64, shape ``(N_A, N_L)``, contiguous;
* ``H``, ``S``: complex128, shape ``(N_G, N_G)``, strides ``(1, N_G)``.

``to_device_*`` helpers move numpy arrays (natural orientation) into that
layout.  Every computation happens in the library; there is no fallback:
importing this module without a built ``libhs.so`` raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libhs.so")

HS_OK, HS_PENDING = 0, 1
HS_EINVAL, HS_ENOMEM, HS_ECUDA, HS_EBUSY, HS_ETIMEDOUT, HS_EDEVICE, HS_ENOTSUP = (
    -1, -2, -3, -4, -5, -6, -7)
HS_ESCRATCH = -8
HS_ENOTPD = -9
HS_FP64, HS_SPLIT_BF16 = 0, 1
HS_REAL = 0x100
PRECISIONS = {"fp64": HS_FP64, "split_bf16": HS_SPLIT_BF16,
              "fp64_real": HS_FP64 | HS_REAL, "split_bf16_real": HS_SPLIT_BF16 | HS_REAL}


class hs_info(C.Structure):
    _fields_ = [("n_fallback", C.c_int), ("slices", C.c_int), ("ms_total", C.c_double),
                ("ms_factor", C.c_double), ("ms_atoms", C.c_double), ("ms_slice", C.c_double),
                ("ms_S", C.c_double), ("ms_H", C.c_double), ("ms_finalize", C.c_double),
                ("ms_queue", C.c_double), ("ms_latency", C.c_double),
                ("inflight_bytes", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class hs_reduce_info(C.Structure):
    _fields_ = [("fail_col", C.c_int), ("ms_total", C.c_double), ("ms_cholesky", C.c_double),
                ("ms_inverse", C.c_double), ("ms_p", C.c_double), ("ms_g", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


# exported symbol -> (restype, argtypes)
_VP, _I, _SZ, _I64 = C.c_void_p, C.c_int, C.c_size_t, C.c_int64
SIGNATURES = {
    "hs_plan": (_I, [C.POINTER(_VP), _I, _I, _I, _I, _I, _SZ, _VP]),
    "hs_footprint": (_SZ, [_VP, _I]),
    "hs_set_t": (_I, [_VP, _VP, _VP, _VP]),
    "hs_assemble": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _VP, _VP,
                         C.POINTER(hs_info)]),
    "hs_assemble_host": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _VP, _VP,
                              C.POINTER(hs_info)]),
    "hs_submit": (_I, [_VP, _VP, _VP, _I, _VP, _I, _VP, _VP, C.POINTER(_I64)]),
    "hs_assemble_partial": (_I, [_VP, _VP, _VP, _I, _VP, _VP, _VP, _VP, _I, _I, _I, _VP, _VP,
                                 C.POINTER(hs_info)]),
    "hs_finalize": (_I, [_VP, _VP, _VP, _I]),
    "hs_poll": (_I, [_VP, _I64, _I64, C.POINTER(hs_info)]),
    "hs_fallback_flags": (_I, [_VP, C.POINTER(_I)]),
    "hs_destroy": (_I, [_VP]),
    "hs_strerror": (C.c_char_p, [_I]),
    "hs_assemble_static": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _VP, _VP, _VP]),
    "hs_set_t_real": (_I, [_VP, _VP, _VP, _VP]),
    "hs_assemble_real": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _I, _VP, _VP,
                              C.POINTER(hs_info)]),
    "hs_reduce": (_I, [_VP, _VP, _VP, _I, C.POINTER(hs_reduce_info)]),
    "hs_reduce_real": (_I, [_VP, _VP, _VP, _I, C.POINTER(hs_reduce_info)]),
    "hs_matching": (_I, [_VP, _VP, _VP, _VP, C.c_double, _I, _I, _I, _VP, _VP, _I, _VP]),
}


def load(path: str = _LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise RuntimeError(
            f"libhs.so not found at {path}: build it first "
            "(python -m paper_1611_00606_gb300.build); there is no CPU fallback")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = load()


class HSError(RuntimeError):
    def __init__(self, code: int, where: str):
        super().__init__(f"{where}: {_lib.hs_strerror(code).decode()} ({code})")
        self.code = code


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise HSError(rc, where)
    return rc


# ---------------------------------------------------------------- marshalling

def _ptr(t) -> int:
    return t.data_ptr()


def _check_coef(X, K, N_G, name):
    import torch
    if X.dtype != torch.complex128 or not X.is_cuda:
        raise ValueError(f"{name}: complex128 CUDA tensor required")
    if X.shape[0] != K or X.shape[1] < N_G or X.stride(0) != 1 or X.stride(1) < K:
        raise ValueError(f"{name}: shape (K, N_G) column-major with ld >= K required")
    return X.stride(1)


def _check_T(T, N_A, N_L, name):
    import torch
    if T.dtype != torch.complex128 or not T.is_cuda or tuple(T.shape) != (N_A, N_L, N_L) or \
            tuple(T.stride()) != (N_L * N_L, 1, N_L):
        raise ValueError(f"{name}: (N_A, N_L, N_L) complex128 CUDA tensor, column-major blocks")


def _check_out(X, N_G, name):
    import torch
    if X.dtype != torch.complex128 or not X.is_cuda or tuple(X.shape) != (N_G, N_G) or \
            tuple(X.stride()) != (1, N_G):
        raise ValueError(f"{name}: (N_G, N_G) complex128 CUDA tensor, column-major")


def empty_hs(N_G: int, device="cuda"):
    """Column-major (N_G, N_G) complex128 output tensor."""
    import torch
    return torch.empty((N_G, N_G), dtype=torch.complex128, device=device).T


def to_device_coef(X: np.ndarray, device="cuda"):
    """numpy (K, N_G) complex -> column-major CUDA tensor of the same shape."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X).T)).to(device).T


def to_device_T(T: np.ndarray, device="cuda"):
    """numpy (N_A, N_L, N_L) natural orientation -> column-major-block CUDA tensor."""
    import torch
    buf = np.ascontiguousarray(np.swapaxes(np.asarray(T), -1, -2))
    return torch.from_numpy(buf).to(device).transpose(1, 2)


def to_device_U(U: np.ndarray, device="cuda"):
    import torch
    return torch.from_numpy(np.ascontiguousarray(U, dtype=np.float64)).to(device)


# ---------------------------------------------------------------- C names

def hs_plan(N_A: int, N_L: int, N_G_max: int, precision="fp64", slices: int = 0,
            hbm_budget_bytes: int = 0, stream=None) -> int:
    """Create a plan; returns the opaque handle (int).  stream: torch.cuda.Stream or None
    (None = torch's current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    h = C.c_void_p()
    _check(_lib.hs_plan(C.byref(h), N_A, N_L, N_G_max, prec, slices, hbm_budget_bytes,
                        C.c_void_p(stream.cuda_stream)), "hs_plan")
    return h.value


def hs_footprint(plan: int, N_G: int) -> int:
    return int(_lib.hs_footprint(plan, N_G))


def hs_set_t(plan: int, T_AA, T_AB, T_BB) -> None:
    _check(_lib.hs_set_t(plan, _ptr(T_AA), _ptr(T_AB), _ptr(T_BB)), "hs_set_t")


def hs_assemble(plan: int, A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int, N_G: int,
                H=None, S=None) -> tuple:
    """Assemble H, S (device tensors, written in place or allocated); returns (H, S, info)."""
    K = N_A * N_L
    ld = _check_coef(A, K, N_G, "A")
    if _check_coef(B, K, N_G, "B") != ld or ld != K:
        raise ValueError("hs_assemble: A and B must have leading dimension K")
    for T, n in ((T_AA, "T_AA"), (T_AB, "T_AB"), (T_BB, "T_BB")):
        _check_T(T, N_A, N_L, n)
    if H is None:
        H = empty_hs(N_G, A.device)
    if S is None:
        S = empty_hs(N_G, A.device)
    _check_out(H, N_G, "H")
    _check_out(S, N_G, "S")
    info = hs_info()
    _check(_lib.hs_assemble(plan, _ptr(A), _ptr(B), _ptr(T_AA), _ptr(T_AB), _ptr(T_BB),
                            _ptr(U), N_A, N_L, N_G, _ptr(H), _ptr(S), C.byref(info)),
           "hs_assemble")
    return H, S, info.as_dict()


def hs_assemble_host(plan: int, A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int, N_G: int,
                     H, S) -> dict:
    """Host-buffer variant: every argument is a host (CPU, ideally pinned) torch tensor
    in the ABI layout; H and S are written in place.  Returns info."""
    info = hs_info()
    _check(_lib.hs_assemble_host(plan, _ptr(A), _ptr(B), _ptr(T_AA), _ptr(T_AB), _ptr(T_BB),
                                 _ptr(U), N_A, N_L, N_G, _ptr(H), _ptr(S), C.byref(info)),
           "hs_assemble_host")
    return info.as_dict()


def hs_assemble_partial(plan: int, A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int, N_G: int,
                        H, S) -> dict:
    """Terms of one atom range (the plan's N_A atoms), lower triangles of H and S only.
    A, B: row views (N_A*N_L, >= N_G) of the full stacked arrays (leading dimension
    >= N_A*N_L); T_*: (N_A, N_L, N_L) views of the range's blocks; U: (N_A, N_L)."""
    K = N_A * N_L
    ld = _check_coef(A, K, N_G, "A")
    if _check_coef(B, K, N_G, "B") != ld:
        raise ValueError("hs_assemble_partial: A and B must share a leading dimension")
    for T, n in ((T_AA, "T_AA"), (T_AB, "T_AB"), (T_BB, "T_BB")):
        _check_T(T, N_A, N_L, n)
    _check_out(H, N_G, "H")
    _check_out(S, N_G, "S")
    info = hs_info()
    _check(_lib.hs_assemble_partial(plan, _ptr(A), _ptr(B), ld, _ptr(T_AA), _ptr(T_AB),
                                    _ptr(T_BB), _ptr(U), N_A, N_L, N_G, _ptr(H), _ptr(S),
                                    C.byref(info)), "hs_assemble_partial")
    return info.as_dict()


def hs_finalize(plan: int, H, S, N_G: int) -> None:
    """Upper triangles := conjugates of the lower ones, Im(diag) := 0 (after the partial
    sums of all atom ranges were added up)."""
    _check_out(H, N_G, "H")
    _check_out(S, N_G, "S")
    _check(_lib.hs_finalize(plan, _ptr(H), _ptr(S), N_G), "hs_finalize")


def hs_submit(plan: int, A, B, U, N_G: int, H, S) -> int:
    """Enqueue a serving request; A, B may be column-truncated views (ld >= K)."""
    ld = A.stride(1)
    if B.stride(1) != ld:
        raise ValueError("hs_submit: A and B must share a leading dimension")
    _check_out(H, N_G, "H")
    _check_out(S, N_G, "S")
    t = C.c_int64()
    _check(_lib.hs_submit(plan, _ptr(A), _ptr(B), ld, _ptr(U), N_G, _ptr(H), _ptr(S),
                          C.byref(t)), "hs_submit")
    return t.value


def hs_poll(plan: int, ticket: int, timeout_us: int = -1):
    """Returns (code, info dict or None); code is HS_OK, HS_PENDING or HS_ETIMEDOUT."""
    info = hs_info()
    rc = _lib.hs_poll(plan, ticket, timeout_us, C.byref(info))
    if rc in (HS_PENDING, HS_ETIMEDOUT):
        return rc, None
    _check(rc, "hs_poll")
    return rc, info.as_dict()


def hs_fallback_flags(plan: int, N_A: int) -> np.ndarray:
    buf = (C.c_int * N_A)()
    _check(_lib.hs_fallback_flags(plan, buf), "hs_fallback_flags")
    return np.array(buf[:], dtype=np.int32)


def hs_destroy(plan: int) -> None:
    _check(_lib.hs_destroy(plan), "hs_destroy")


def hs_assemble_static(A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int, N_G: int, H, S,
                       stream=None) -> None:
    """Allocation-free FP64 assembly (no plan): intermediates live in the library's
    static device scratch.  For callers that must not allocate device memory; see
    include/hs.h for the size limit and the rule that overlapping calls race."""
    import torch
    K = N_A * N_L
    if _check_coef(A, K, N_G, "A") != K or _check_coef(B, K, N_G, "B") != K:
        raise ValueError("hs_assemble_static: A and B must have leading dimension K")
    for T, n in ((T_AA, "T_AA"), (T_AB, "T_AB"), (T_BB, "T_BB")):
        _check_T(T, N_A, N_L, n)
    _check_out(H, N_G, "H")
    _check_out(S, N_G, "S")
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib.hs_assemble_static(_ptr(A), _ptr(B), _ptr(T_AA), _ptr(T_AB), _ptr(T_BB),
                                   _ptr(U), N_A, N_L, N_G, _ptr(H), _ptr(S),
                                   C.c_void_p(stream.cuda_stream)), "hs_assemble_static")


def _check_f64(X, shape, name):
    import torch
    if X.dtype != torch.float64 or not X.is_cuda or tuple(X.shape) != shape or \
            not X.is_contiguous():
        raise ValueError(f"{name}: contiguous float64 CUDA tensor of shape {shape} required")


def hs_matching(Kvec, tau, R, ufun, omega: float, l_max: int, A=None, B=None,
                stream=None):
    """Matching coefficients A, B (Sec. 1.1) of N_G plane waves (Kvec: (N_G, 3)) on N_A
    spheres (tau: (N_A, 3), R: (N_A,), ufun: (N_A, l_max + 1, 4) = u, u', udot, udot'
    at R), float64 CUDA tensors.  Returns A, B as (N_A N_L, N_G) column-major complex128
    tensors, allocated here unless given (any leading dimension >= N_A N_L)."""
    import torch
    N_G, N_A = int(Kvec.shape[0]), int(tau.shape[0])
    N_L = (l_max + 1) ** 2
    K = N_A * N_L
    _check_f64(Kvec, (N_G, 3), "Kvec")
    _check_f64(tau, (N_A, 3), "tau")
    _check_f64(R, (N_A,), "R")
    _check_f64(ufun, (N_A, l_max + 1, 4), "ufun")
    if A is None:
        A = torch.empty((N_G, K), dtype=torch.complex128, device=Kvec.device).T
    if B is None:
        B = torch.empty((N_G, K), dtype=torch.complex128, device=Kvec.device).T
    ld = _check_coef(A, K, N_G, "A")
    if _check_coef(B, K, N_G, "B") != ld:
        raise ValueError("hs_matching: A and B must share one leading dimension")
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(_lib.hs_matching(_ptr(Kvec), _ptr(tau), _ptr(R), _ptr(ufun), float(omega), N_A,
                            l_max, N_G, _ptr(A), _ptr(B), ld, C.c_void_p(stream.cuda_stream)),
           "hs_matching")
    return A, B


# ---------------------------------------------------------------- real-symmetric variant

def _check_real(X, shape, strides, name):
    import torch
    if X.dtype != torch.float64 or not X.is_cuda or tuple(X.shape) != shape or \
            tuple(X.stride()) != strides:
        raise ValueError(f"{name}: float64 CUDA tensor of shape {shape}, strides {strides}")


def to_device_real(X: np.ndarray, device="cuda"):
    """numpy real (rows, cols) -> column-major float64 CUDA tensor of the same shape."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(np.asarray(X, dtype=np.float64).T)).to(device).T


def to_device_T_real(T: np.ndarray, device="cuda"):
    """numpy real (N_A, N_L, N_L) natural orientation -> column-major-block CUDA tensor."""
    import torch
    buf = np.ascontiguousarray(np.swapaxes(np.asarray(T, dtype=np.float64), -1, -2))
    return torch.from_numpy(buf).to(device).transpose(1, 2)


def empty_hs_real(N_G: int, device="cuda"):
    """Column-major (N_G, N_G) float64 output tensor."""
    import torch
    return torch.empty((N_G, N_G), dtype=torch.float64, device=device).T


def hs_set_t_real(plan: int, T_AA, T_AB, T_BB) -> None:
    _check(_lib.hs_set_t_real(plan, _ptr(T_AA), _ptr(T_AB), _ptr(T_BB)), "hs_set_t_real")


def hs_assemble_real(plan: int, A, B, T_AA, T_AB, T_BB, U, N_A: int, N_L: int, N_G: int,
                     H=None, S=None) -> tuple:
    """Real-symmetric variant (plan made with a *_real precision): real H, S."""
    K = N_A * N_L
    _check_real(A, (K, N_G), (1, K), "A")
    _check_real(B, (K, N_G), (1, K), "B")
    for T, n in ((T_AA, "T_AA"), (T_AB, "T_AB"), (T_BB, "T_BB")):
        _check_real(T, (N_A, N_L, N_L), (N_L * N_L, 1, N_L), n)
    if H is None:
        H = empty_hs_real(N_G, A.device)
    if S is None:
        S = empty_hs_real(N_G, A.device)
    _check_real(H, (N_G, N_G), (1, N_G), "H")
    _check_real(S, (N_G, N_G), (1, N_G), "S")
    info = hs_info()
    _check(_lib.hs_assemble_real(plan, _ptr(A), _ptr(B), _ptr(T_AA), _ptr(T_AB), _ptr(T_BB),
                                 _ptr(U), N_A, N_L, N_G, _ptr(H), _ptr(S), C.byref(info)),
           "hs_assemble_real")
    return H, S, info.as_dict()


def hs_reduce(plan: int, H, S, N_G: int = None) -> dict:
    """Generalized-eigenproblem reduction in place: S <- L (S = L L^H), H <- L^-1 H L^-H.
    H, S: (N_G, N_G) column-major complex128 CUDA tensors.  Returns the info dict;
    raises HSError (code HS_ENOTPD, ``fail_col`` attribute) when S is not positive
    definite."""
    N_G = H.shape[0] if N_G is None else N_G
    _check_out(H, N_G, "H")
    _check_out(S, N_G, "S")
    info = hs_reduce_info()
    rc = _lib.hs_reduce(plan, _ptr(H), _ptr(S), N_G, C.byref(info))
    if rc < 0:
        err = HSError(rc, "hs_reduce")
        err.fail_col = info.fail_col
        raise err
    return info.as_dict()


def hs_reduce_real(plan: int, H, S, N_G: int = None) -> dict:
    """Real-symmetric form of hs_reduce (plan made with "fp64_real"): float64 (N_G, N_G)
    column-major CUDA tensors, reduced in place.  Returns the info dict; raises HSError
    (HS_ENOTPD with ``fail_col``) when S is not positive definite."""
    N_G = H.shape[0] if N_G is None else N_G
    _check_real(H, (N_G, N_G), (1, N_G), "H")
    _check_real(S, (N_G, N_G), (1, N_G), "S")
    info = hs_reduce_info()
    rc = _lib.hs_reduce_real(plan, _ptr(H), _ptr(S), N_G, C.byref(info))
    if rc < 0:
        err = HSError(rc, "hs_reduce_real")
        err.fail_col = info.fail_col
        raise err
    return info.as_dict()


def hs_strerror(code: int) -> str:
    return _lib.hs_strerror(code).decode()


class Plan:
    """Context-managed plan handle."""

    def __init__(self, N_A, N_L, N_G_max, precision="fp64", slices=0, hbm_budget_bytes=0,
                 stream=None):
        self.N_A, self.N_L, self.N_G_max = N_A, N_L, N_G_max
        self.h = hs_plan(N_A, N_L, N_G_max, precision, slices, hbm_budget_bytes, stream)

    def assemble(self, A, B, T_AA, T_AB, T_BB, U, N_G=None, H=None, S=None):
        N_G = A.shape[1] if N_G is None else N_G
        return hs_assemble(self.h, A, B, T_AA, T_AB, T_BB, U, self.N_A, self.N_L, N_G, H, S)

    def assemble_real(self, A, B, T_AA, T_AB, T_BB, U, N_G=None, H=None, S=None):
        N_G = A.shape[1] if N_G is None else N_G
        return hs_assemble_real(self.h, A, B, T_AA, T_AB, T_BB, U, self.N_A, self.N_L, N_G, H, S)

    def reduce(self, H, S, N_G=None):
        return hs_reduce(self.h, H, S, N_G)

    def close(self):
        if self.h:
            hs_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
