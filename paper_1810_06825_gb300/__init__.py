"""frPCA / frPCAt on GB300: Python binding of the ``libfrpca.so`` C ABI.

Fast randomized PCA for sparse data (Feng, Xie, Song, Yu, Tang, ACML 2018):
``frpca_run`` computes a rank-k truncated SVD of a CSR matrix with q passes
over it (Alg. 5 for wide, Alg. 6 for tall matrices), every step in this
package's CUDA kernels.  This module only marshals arguments: the functions
named like the C entry points take raw device pointers; ``FrPCA`` and the
helpers below take torch CUDA tensors and pass their pointers and the current
stream.  There is no CPU fallback: without the built library every call raises.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfrpca.so")

FRPCA_OK = 0
STATUS_NAMES = {
    0: "OK", 1: "INVALID_ARG", 2: "INVALID_CSR", 3: "OOM", 4: "CUDA", 5: "SINGULAR_PIVOT",
    6: "RANK_DEFICIENT", 7: "TIMEOUT", 8: "NOT_CONVERGED", 9: "UNSUPPORTED",
}
FRPCA_F32, FRPCA_F64 = 0, 1
FRPCA_I64, FRPCA_I32 = 0, 1
PREC = {"fp64": 0, "fp32": 1, "fp32_splitgram": 2, "fp32_dfgram": 3}

EXPORTED = [
    "frpca_create", "frpca_destroy", "frpca_last_error", "frpca_run", "frpca_run_async", "frpca_sync",
    "frpca_refresh", "frpca_set_timing", "frpca_get_stats", "frpca_reset_stats",
    "frpca_gaussian", "frpca_spmm", "frpca_get_transpose", "frpca_lu", "frpca_gram", "frpca_eig",
    "frpca_eigsvd", "frpca_backward", "frpca_gram_splitbf16", "frpca_lu_tournament", "frpca_set_wait_limit",
    "frpca_trim_memory",
]


class FrpcaError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class frpca_csr(ctypes.Structure):
    _fields_ = [("m", ctypes.c_int64), ("n", ctypes.c_int64), ("nnz", ctypes.c_int64),
                ("rowptr", ctypes.c_void_p), ("colidx", ctypes.c_void_p), ("values", ctypes.c_void_p),
                ("dtype", ctypes.c_int), ("on_device", ctypes.c_int), ("rowptr_type", ctypes.c_int)]


class frpca_create_opts(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("borrow", ctypes.c_int), ("validate", ctypes.c_int),
                ("hot_columns", ctypes.c_int), ("max_device_bytes", ctypes.c_int64), ("panel_rows", ctypes.c_int),
                ("fused_sweep", ctypes.c_int)]


class frpca_run_opts(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("l", ctypes.c_int), ("q", ctypes.c_int), ("seed", ctypes.c_uint64),
                ("precision", ctypes.c_int), ("alg", ctypes.c_int), ("center", ctypes.c_int),
                ("scheme", ctypes.c_int)]


class frpca_stats(ctypes.Structure):
    _fields_ = [("runs", ctypes.c_int64), ("kernel_launches", ctypes.c_int64), ("spmm_passes", ctypes.c_int64),
                ("spmm_ms", ctypes.c_double), ("spmm_bytes", ctypes.c_double), ("spmm_flops", ctypes.c_double),
                ("lu_calls", ctypes.c_int64), ("lu_ms", ctypes.c_double), ("eigsvd_calls", ctypes.c_int64),
                ("gram_ms", ctypes.c_double), ("eig_ms", ctypes.c_double), ("apply_ms", ctypes.c_double),
                ("gaussian_ms", ctypes.c_double), ("transpose_ms", ctypes.c_double), ("finish_ms", ctypes.c_double),
                ("spmm_a_passes", ctypes.c_int64), ("spmm_t_passes", ctypes.c_int64), ("spmm_a_ms", ctypes.c_double),
                ("spmm_t_ms", ctypes.c_double), ("fused_sweeps", ctypes.c_int64), ("qr_calls", ctypes.c_int64)]

    def as_dict(self) -> dict:
        return {name: getattr(self, name) for name, _ in self._fields_}


_lib = None


def library() -> ctypes.CDLL:
    """The loaded C library; raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1810_06825_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, I64, U64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
    sig = {
        "frpca_create": [P, P, P],
        "frpca_destroy": [P],
        "frpca_run": [P, P, P, P, P],
        "frpca_run_async": [P, P, P, P, P],
        "frpca_sync": [P],
        "frpca_refresh": [P],
        "frpca_set_timing": [P, I],
        "frpca_get_stats": [P, P],
        "frpca_reset_stats": [P],
        "frpca_set_wait_limit": [P, I64],
        "frpca_trim_memory": [],
        "frpca_gaussian": [P, I64, I, I64, U64, I, P],
        "frpca_spmm": [P, I, I, P, I64, P, I64, I],
        "frpca_get_transpose": [P, P, P, P],
        "frpca_lu": [P, I64, I, P, I64, I, P],
        "frpca_lu_noalloc": [I64, I, P, I64, I, P, P],
        "frpca_gram": [P, I64, I, P, I64, I, P],
        "frpca_eig": [P, I, P, P, P],
        "frpca_eigsvd": [P, I64, I, P, I64, I, P, P],
        "frpca_backward": [P, I, P, P, P, P, P, P, I, P],
        "frpca_gram_splitbf16": [P, I64, I, P, I64, P],
        "frpca_lu_tournament": [P, I64, I, P, I64, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.frpca_last_error.argtypes = [P]
    lib.frpca_last_error.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(status: int, handle) -> None:
    if status != FRPCA_OK:
        msg = library().frpca_last_error(handle)
        raise FrpcaError(status, msg.decode() if msg else "")


# ---------------------------------------------------------------- raw C-ABI calls
def frpca_create(csr, opts) -> int:
    h = ctypes.c_void_p()
    st = library().frpca_create(ctypes.byref(csr) if csr is not None else None, ctypes.byref(opts), ctypes.byref(h))
    _check(st, None)
    return h.value


def frpca_destroy(h) -> None:
    library().frpca_destroy(h)


def frpca_last_error(h) -> str:
    m = library().frpca_last_error(h)
    return m.decode() if m else ""


def frpca_run(h, opts, U, S, V) -> None:
    _check(library().frpca_run(h, ctypes.byref(opts), U, S, V), h)


def frpca_run_async(h, opts, U, S, V) -> None:
    _check(library().frpca_run_async(h, ctypes.byref(opts), U, S, V), h)


def frpca_sync(h) -> None:
    _check(library().frpca_sync(h), h)


def frpca_refresh(h) -> None:
    _check(library().frpca_refresh(h), h)


def frpca_set_timing(h, enable: bool) -> None:
    _check(library().frpca_set_timing(h, 1 if enable else 0), h)


def frpca_get_stats(h) -> frpca_stats:
    st = frpca_stats()
    _check(library().frpca_get_stats(h, ctypes.byref(st)), h)
    return st


def frpca_reset_stats(h) -> None:
    _check(library().frpca_reset_stats(h), h)


def frpca_trim_memory() -> None:
    """Give back the device memory the library's pool keeps for later handles."""
    _check(library().frpca_trim_memory(), None)


def frpca_set_wait_limit(h, cycles: int) -> None:
    _check(library().frpca_set_wait_limit(h, cycles), h)


def frpca_gaussian(h, R, l, ld, seed, dtype, out) -> None:
    _check(library().frpca_gaussian(h, R, l, ld, seed, dtype, out), h)


def frpca_spmm(h, trans, l, X, ldx, Y, ldy, dtype) -> None:
    _check(library().frpca_spmm(h, trans, l, X, ldx, Y, ldy, dtype), h)


def frpca_get_transpose(h, rowptrT, colidxT, valuesT) -> None:
    _check(library().frpca_get_transpose(h, rowptrT, colidxT, valuesT), h)


def frpca_lu(h, R, l, M, ld, dtype, piv) -> None:
    _check(library().frpca_lu(h, R, l, M, ld, dtype, piv), h)


def frpca_lu_noalloc(R, l, M, ld, dtype, piv, stream) -> None:
    """frpca_lu without device allocation (static scratch); see include/frpca.h."""
    _check(library().frpca_lu_noalloc(R, l, M, ld, dtype, piv, stream), None)


def frpca_gram(h, R, l, M, ld, dtype, B) -> None:
    _check(library().frpca_gram(h, R, l, M, ld, dtype, B), h)


def frpca_eig(h, n, B, w, V) -> None:
    _check(library().frpca_eig(h, n, B, w, V), h)


def frpca_eigsvd(h, R, l, M, ld, dtype, S, V) -> None:
    _check(library().frpca_eigsvd(h, R, l, M, ld, dtype, S, V), h)


# ---------------------------------------------------------------- torch helpers
def frpca_lu_tournament(h, R, l, M, ld, piv) -> None:
    _check(library().frpca_lu_tournament(h, R, l, M, ld, piv), h)


def frpca_gram_splitbf16(h, R, l, M, ld, B) -> None:
    _check(library().frpca_gram_splitbf16(h, R, l, M, ld, B), h)


def frpca_backward(h, k, U, S, V, dU, dS, dV, dtype, dvalues) -> None:
    _check(library().frpca_backward(h, k, U, S, V, dU, dS, dV, dtype, dvalues), h)


def _torch():
    import torch
    return torch


def _dtype_code(t) -> int:
    torch = _torch()
    if t.dtype == torch.float32:
        return FRPCA_F32
    if t.dtype == torch.float64:
        return FRPCA_F64
    raise TypeError(f"unsupported dtype {t.dtype}")


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


def _need_cuda(*ts):
    for t in ts:
        if not t.is_cuda:
            raise ValueError("tensors must be on a CUDA device")


def padded_ld(l: int) -> int:
    """Row length (elements) used for dense blocks: a multiple of 4, so every row starts on 16 bytes."""
    return (l + 3) // 4 * 4


def empty_block(R: int, l: int, dtype, device) -> "torch.Tensor":
    """R x l view of a zeroed R x padded_ld(l) buffer (rows 16-byte aligned)."""
    torch = _torch()
    return torch.zeros((R, padded_ld(l)), dtype=dtype, device=device)[:, :l]


class _Context:
    """Matrix-less handle per (device, stream) for the step-level entry points."""
    _cache: dict = {}

    @classmethod
    def get(cls, stream=None) -> int:
        torch = _torch()
        s = stream if stream is not None else torch.cuda.current_stream()
        key = (s.device.index, s.cuda_stream)
        h = cls._cache.get(key)
        if h is None:
            opts = frpca_create_opts(stream=s.cuda_stream, borrow=0, validate=1)
            h = frpca_create(None, opts)
            cls._cache[key] = h
        return h


class FrPCA:
    """A sparse matrix resident on the GPU, ready for frPCA runs.

    ``indptr`` (int64 or int32, m+1), ``indices`` (int32, nnz, sorted and
    unique per row) and ``values`` (float32/float64, nnz) are CUDA tensors; by
    default they are borrowed (kept alive by this object) and A^T is built on
    the device.  ``FrPCA.from_host`` takes host arrays instead, which the
    library copies to the device itself.  ``hot_columns``: 0 keeps every
    nonzero on the CSR kernel; -1 picks the densest columns automatically and
    > 0 that many (multiples of 128, at most 256) for a dense block whose share
    of each pass runs on the tensor cores.  ``max_device_bytes`` caps the
    device memory the handle allocates for itself (0: no cap).  ``panel_rows``:
    the panel height of the pass that gathers rows of the larger dense block
    (0 automatic, -1 off); ``fused_sweep`` 1 runs each power-iteration pair of
    passes as one panel-by-panel sweep (0: two passes).
    """

    def __init__(self, indptr, indices, values, shape, stream=None, borrow=True, validate=True, hot_columns=0,
                 max_device_bytes=0, panel_rows=0, fused_sweep=0):
        torch = _torch()
        _need_cuda(indptr, indices, values)
        if indptr.dtype not in (torch.int64, torch.int32):
            indptr = indptr.to(torch.int64)
        self._keep = (indptr.contiguous(), indices.contiguous().to(torch.int32), values.contiguous())
        self.indptr, self.indices, self.values = self._keep
        self._setup(self.indptr.data_ptr(), self.indices.data_ptr() if self.indices.numel() else None,
                    self.values.data_ptr() if self.values.numel() else None, int(self.indices.numel()),
                    self.indptr.dtype == torch.int32, self.values.dtype, shape, 1, self.values.device, stream,
                    borrow, validate, hot_columns, max_device_bytes, panel_rows, fused_sweep)

    def _setup(self, p_indptr, p_indices, p_values, nnz, rp32, dtype, shape, on_device, device, stream, borrow,
               validate, hot_columns, max_device_bytes, panel_rows=0, fused_sweep=0):
        torch = _torch()
        self.m, self.n = int(shape[0]), int(shape[1])
        self._nnz = nnz
        self.dtype = dtype
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        csr = frpca_csr(m=self.m, n=self.n, nnz=nnz, rowptr=p_indptr, colidx=p_indices, values=p_values,
                        dtype=FRPCA_F32 if dtype == torch.float32 else FRPCA_F64, on_device=on_device,
                        rowptr_type=FRPCA_I32 if rp32 else FRPCA_I64)
        opts = frpca_create_opts(stream=self.stream.cuda_stream, borrow=1 if borrow else 0,
                                 validate=1 if validate else 0, hot_columns=int(hot_columns),
                                 max_device_bytes=int(max_device_bytes), panel_rows=int(panel_rows),
                                 fused_sweep=int(fused_sweep))
        self.handle = frpca_create(csr, opts)

    @classmethod
    def from_host(cls, indptr, indices, values, shape, device="cuda", stream=None, validate=True, hot_columns=0,
                  max_device_bytes=0, panel_rows=0, fused_sweep=0):
        """From host arrays (numpy or CPU tensors; pinned memory copies fastest):
        the C ABI's own host path (``on_device = 0``) copies them to the
        device and validates them there."""
        import numpy as np
        torch = _torch()
        to_np = lambda a: a.numpy() if hasattr(a, "numpy") and not isinstance(a, np.ndarray) else a  # noqa: E731
        ip, ix, va = (to_np(a) for a in (indptr, indices, values))
        if ip.dtype not in (np.int64, np.int32):
            ip = ip.astype(np.int64)
        ip = np.ascontiguousarray(ip)
        ix = np.ascontiguousarray(ix, dtype=np.int32)
        va = np.ascontiguousarray(va)
        if va.dtype not in (np.float32, np.float64):
            raise TypeError(f"unsupported dtype {va.dtype}")
        self = cls.__new__(cls)
        self._keep = None
        self.indptr = self.indices = self.values = None
        dev = torch.device(device)
        if dev.index is None:
            dev = torch.device("cuda", torch.cuda.current_device())
        with torch.cuda.device(dev):
            self._setup(ip.ctypes.data, ix.ctypes.data if ix.size else None, va.ctypes.data if va.size else None,
                        int(ix.size), ip.dtype == np.int32,
                        torch.float32 if va.dtype == np.float32 else torch.float64, shape, 0, dev, stream,
                        False, validate, hot_columns, max_device_bytes, panel_rows, fused_sweep)
        return self

    @classmethod
    def from_csr(cls, csr, device="cuda", dtype=None, **kw):
        """From an object with m, n, indptr, indices, data (numpy), e.g. synthetic.CSR."""
        torch = _torch()
        data = csr.data if dtype is None else csr.data.astype(dtype)
        return cls(torch.from_numpy(csr.indptr).to(device), torch.from_numpy(csr.indices).to(device),
                   torch.from_numpy(data).to(device), (csr.m, csr.n), **kw)

    @property
    def nnz(self) -> int:
        return self._nnz

    def close(self):
        if getattr(self, "handle", None):
            frpca_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def run(self, k: int, l: int, q: int, seed: int = 0, precision: str = "fp32", alg: int = 0, out=None,
            sync: bool = True, center: bool = False, scheme: str = "frpca"):
        """Rank-k frPCA (Alg. 5/6); returns (U m x k, S k descending float64, V n x k).
        ``center=True`` factors the column-centered matrix (PCA proper);
        ``scheme="qr"`` runs the basic randomized PCA with QR (Alg. 1/4)."""
        torch = _torch()
        dt = torch.float64 if precision == "fp64" else torch.float32
        dev = self.device
        if out is None:
            U = torch.empty((self.m, k), dtype=dt, device=dev)
            S = torch.empty((k,), dtype=torch.float64, device=dev)
            V = torch.empty((self.n, k), dtype=dt, device=dev)
        else:
            U, S, V = out
        opts = frpca_run_opts(k=k, l=l, q=q, seed=seed, precision=PREC[precision], alg=alg, center=int(center),
                              scheme={"frpca": 0, "qr": 1}[scheme])
        fn = frpca_run if sync else frpca_run_async
        fn(self.handle, opts, U.data_ptr(), S.data_ptr(), V.data_ptr())
        return U, S, V

    def spmm(self, X, trans: bool = False, out=None):
        """A X (or A^T X) for a dense block X whose rows start on 16 bytes."""
        torch = _torch()
        l = X.shape[1]
        rows = self.n if trans else self.m
        Y = out if out is not None else empty_block(rows, l, X.dtype, X.device)
        frpca_spmm(self.handle, 1 if trans else 0, l, X.data_ptr(), X.stride(0), Y.data_ptr(), Y.stride(0),
                   _dtype_code(X))
        return Y

    def refresh(self):
        """Rebuild A^T on the device (after the borrowed values changed in place)."""
        frpca_refresh(self.handle)

    def set_timing(self, enable: bool = True):
        frpca_set_timing(self.handle, enable)

    def stats(self) -> dict:
        return frpca_get_stats(self.handle).as_dict()

    def reset_stats(self):
        frpca_reset_stats(self.handle)

    def backward(self, U, S, V, dU=None, dS=None, dV=None, out=None):
        """Gradient with respect to the nnz CSR values of a loss of the rank-k
        result (U, S, V), given its cotangents (any may be None = zero): the
        thin-SVD adjoint sampled at A's nonzeros (``frpca_backward``)."""
        torch = _torch()
        k = S.shape[0]
        dt = U.dtype
        for t, rows in ((U, self.m), (V, self.n), (dU, self.m), (dV, self.n)):
            if t is not None and (t.shape != (rows, k) or t.dtype != dt or not t.is_contiguous()):
                raise ValueError("U, V, dU, dV must be contiguous (rows x k) tensors of one dtype")
        for t in (S, dS):
            if t is not None and (t.shape != (k,) or t.dtype != torch.float64 or not t.is_contiguous()):
                raise ValueError("S and dS must be contiguous float64 vectors of length k")
        out = out if out is not None else torch.empty(self.nnz, dtype=dt, device=U.device)
        ptr = lambda t: t.data_ptr() if t is not None else None  # noqa: E731
        frpca_backward(self.handle, k, U.data_ptr(), S.data_ptr(), V.data_ptr(), ptr(dU), ptr(dS), ptr(dV),
                       _dtype_code(U), out.data_ptr() if self.nnz else None)
        return out

    def set_wait_limit(self, cycles: int):
        """Bound (SM clock cycles) of the LU and eigensolver grid-barrier waits; <= 0 restores the default."""
        frpca_set_wait_limit(self.handle, int(cycles))

    def transpose(self):
        torch = _torch()
        dev = self.device
        pT = torch.empty(self.n + 1, dtype=torch.int64, device=dev)
        cT = torch.empty(max(self.nnz, 1), dtype=torch.int32, device=dev)
        vT = torch.empty(max(self.nnz, 1), dtype=self.dtype, device=dev)
        frpca_get_transpose(self.handle, pT.data_ptr(), cT.data_ptr(), vT.data_ptr())
        return pT, cT[: self.nnz], vT[: self.nnz]


def gaussian(R: int, l: int, seed: int, dtype=None, device="cuda"):
    torch = _torch()
    dtype = dtype or torch.float64
    out = empty_block(R, l, dtype, device)
    frpca_gaussian(_Context.get(), R, l, out.stride(0), seed, _dtype_code(out), out.data_ptr())
    return out


def lu(M):
    """P^T L of Alg. 5/6's lu() (in a copy of M) and the pivot rows."""
    torch = _torch()
    _need_cuda(M)
    R, l = M.shape
    A = empty_block(R, l, M.dtype, M.device)
    A.copy_(M)
    piv = torch.empty(l, dtype=torch.int64, device=M.device)
    frpca_lu(_Context.get(), R, l, A.data_ptr(), A.stride(0), _dtype_code(A), piv.data_ptr())
    return A, piv


def gram(M):
    torch = _torch()
    _need_cuda(M)
    R, l = M.shape
    if M.stride(1) != 1:
        M = M.contiguous()
    B = torch.empty((l, l), dtype=torch.float64, device=M.device)
    frpca_gram(_Context.get(), R, l, M.data_ptr(), M.stride(0), _dtype_code(M), B.data_ptr())
    return B


def gram_splitbf16(M):
    """B = M^T M (float64) of an FP32 block on the tensor cores (split BF16)."""
    torch = _torch()
    _need_cuda(M)
    R, l = M.shape
    if M.dtype != torch.float32:
        raise TypeError("gram_splitbf16 takes float32 blocks")
    if M.stride(1) != 1 or M.stride(0) % 4 or M.data_ptr() % 16:
        M = empty_block(R, l, torch.float32, M.device).copy_(M)
    B = torch.empty((l, l), dtype=torch.float64, device=M.device)
    frpca_gram_splitbf16(_Context.get(), R, l, M.data_ptr(), M.stride(0), B.data_ptr())
    return B


def eig(B):
    torch = _torch()
    _need_cuda(B)
    n = B.shape[0]
    B = B.to(torch.float64).contiguous()
    w = torch.empty(n, dtype=torch.float64, device=B.device)
    V = torch.empty((n, n), dtype=torch.float64, device=B.device)
    frpca_eig(_Context.get(), n, B.data_ptr(), w.data_ptr(), V.data_ptr())
    return w, V


def eigsvd(M):
    """Alg. 2 on a copy of M: (U, S ascending, V)."""
    torch = _torch()
    _need_cuda(M)
    R, l = M.shape
    U = empty_block(R, l, M.dtype, M.device)
    U.copy_(M)
    S = torch.empty(l, dtype=torch.float64, device=M.device)
    V = torch.empty((l, l), dtype=torch.float64, device=M.device)
    frpca_eigsvd(_Context.get(), R, l, U.data_ptr(), U.stride(0), _dtype_code(U), S.data_ptr(), V.data_ptr())
    return U, S, V


def _make_svd_function():
    torch = _torch()

    class FrpcaSVD(torch.autograd.Function):
        """(U, S, V) = frPCA of the CSR matrix whose values are the input.

        The forward runs ``frpca_run`` on a handle that borrows ``values``
        (A^T is rebuilt on every call, so in-place updates are seen); the
        backward runs ``frpca_backward``.  Nothing from the q passes is kept:
        the adjoint needs only U, S, V and the cotangents."""

        @staticmethod
        def forward(ctx, values, indptr, indices, shape, k, l, q, seed, mat):
            precision = "fp64" if values.dtype == torch.float64 else "fp32"
            if mat is None:
                mat = FrPCA(indptr, indices, values.detach(), shape, borrow=True)
            else:
                if mat.values.data_ptr() != values.data_ptr() or mat.dtype != values.dtype:
                    raise ValueError("mat must borrow the same values tensor")
                mat.refresh()
            U, S, V = mat.run(k, l, q, seed=seed, precision=precision)
            ctx.mat = mat
            ctx.set_materialize_grads(False)
            ctx.save_for_backward(U, S, V)
            return U, S, V

        @staticmethod
        def backward(ctx, dU, dS, dV):
            U, S, V = ctx.saved_tensors
            c = lambda t, dt: None if t is None else t.to(dt).contiguous()  # noqa: E731
            dvalues = ctx.mat.backward(U, S, V, c(dU, U.dtype), c(dS, torch.float64), c(dV, V.dtype))
            return dvalues, None, None, None, None, None, None, None, None

    return FrpcaSVD


_svd_fn = None


def frpca_svd(values, indptr, indices, shape, k: int, l: int, q: int, seed: int = 0, mat=None):
    """Differentiable rank-k frPCA: returns (U, S, V) with gradients flowing to
    ``values`` (the CSR values, float32 -> FP32 path, float64 -> FP64 path).
    ``mat`` may be an ``FrPCA`` that borrows ``values`` (reused across calls)."""
    global _svd_fn
    if _svd_fn is None:
        _svd_fn = _make_svd_function()
    return _svd_fn.apply(values, indptr, indices, shape, k, l, q, seed, mat)
