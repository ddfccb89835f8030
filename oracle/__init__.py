"""FP64 CPU oracle for fast randomized PCA on sparse data (frPCA / frPCAt).

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import this
package.  The CUDA path never reaches it, and it imports nothing from the CUDA
path.

The arithmetic lives in ``frpca_oracle.c`` (plain C, double precision, the
paper's algorithms step by step); this module only marshals numpy arrays.
Parity status of every function is listed in ``PINS`` below; each one is pinned
by a ``-m "not gpu"`` test against something other than itself.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "frpca_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, ERR_INVALID_ARG, ERR_OOM, ERR_SINGULAR_PIVOT, ERR_RANK_DEFICIENT, ERR_NOT_CONVERGED = 0, 1, 3, 5, 6, 8

# What pins each oracle function (see tests/test_oracle_*.py).
PINS = {
    "philox4x64": "bit-exact against numpy.random.Philox raw output",
    "gaussian": "Kolmogorov-Smirnov and moment tests; Box-Muller values recomputed from numpy's Philox words",
    "csr_transpose": "bit-exact against scipy.sparse .T.tocsr() and a dense transpose",
    "spmm / spmm_t": "dense numpy products on small matrices",
    "lu_ptl": "scipy.linalg.lu(permute_l=True); Lemma 3 range equality; |entries| <= 1",
    "eig_sym": "numpy.linalg.eigh; orthogonality and residual",
    "eigsvd": "Lemma 1 against numpy.linalg.svd",
    "frpca": "exact-rank closed form, planted spectra, Theorems 1-2 vs the QR scheme, exact identities",
    "frpca (center)": "the uncentered method on the explicitly centered matrix stored dense; closed form for an "
                      "exactly rank-l centered matrix",
}


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile ``frpca_oracle.c`` into ``liboracle.so`` next to it (gcc, OpenMP if available)."""
    with _lock:
        if not force and os.path.exists(_LIB_PATH) and os.path.getmtime(_LIB_PATH) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "frpca_oracle.h"))
        ):
            return _LIB_PATH
        base = ["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC", "-shared", _SRC, "-o", _LIB_PATH + ".tmp", "-lm"]
        for extra in (["-fopenmp"], []):
            r = subprocess.run(base[:-1] + extra + ["-lm"], capture_output=True, text=True)
            if r.returncode == 0:
                break
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
        if verbose:
            print(" ".join(base), file=sys.stderr)
        os.replace(_LIB_PATH + ".tmp", _LIB_PATH)
        return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB_PATH)
    P = ctypes.c_void_p
    I64 = ctypes.c_int64
    U64 = ctypes.c_uint64
    lib.or_philox4x64.argtypes = [P, P, P]
    lib.or_philox4x64.restype = None
    lib.or_gaussian.argtypes = [I64, I64, U64, P]
    lib.or_csr_transpose.argtypes = [I64, I64, P, P, P, P, P, P]
    lib.or_spmm.argtypes = [I64, I64, P, P, P, I64, P, I64, P, I64]
    lib.or_spmm_t.argtypes = [I64, I64, P, P, P, I64, P, I64, P, I64]
    lib.or_lu_ptl.argtypes = [I64, I64, P, I64, P]
    lib.or_eig_sym.argtypes = [I64, P, P, P, P]
    lib.or_gram.argtypes = [I64, I64, P, I64, P]
    lib.or_eigsvd.argtypes = [I64, I64, P, I64, P, I64, P, P]
    lib.or_frpca.argtypes = [ctypes.c_int, I64, I64, P, P, P, I64, I64, I64, U64, P, P, P]
    lib.or_frpca_ex.argtypes = [ctypes.c_int, I64, I64, P, P, P, I64, I64, I64, U64, ctypes.c_int, ctypes.c_int,
                                P, P, P]
    lib.or_svd_adjoint_sddmm.argtypes = [I64, I64, P, P, I64, P, P, P, P, P, P, P]
    lib.or_num_threads.argtypes = []
    for name in ("or_gaussian", "or_csr_transpose", "or_spmm", "or_spmm_t", "or_lu_ptl", "or_eig_sym",
                 "or_gram", "or_eigsvd", "or_frpca", "or_frpca_ex", "or_svd_adjoint_sddmm", "or_num_threads"):
        getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


class OracleError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: oracle status {status}")
        self.status = status


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(st: int, what: str):
    if st != OK:
        raise OracleError(st, what)


def _csr(indptr, indices, data):
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    data = np.ascontiguousarray(data, dtype=np.float64)
    return indptr, indices, data


def num_threads() -> int:
    return _load().or_num_threads()


def philox4x64(counter, key) -> np.ndarray:
    """One Philox4x64-10 block: four uint64 words for a 4-word counter and 2-word key."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    _load().or_philox4x64(_p(c), _p(k), _p(out))
    return out


def gaussian(R: int, l: int, seed: int) -> np.ndarray:
    out = np.empty((R, l), dtype=np.float64)
    _check(_load().or_gaussian(R, l, seed, _p(out)), "gaussian")
    return out


def csr_transpose(m: int, n: int, indptr, indices, data):
    indptr, indices, data = _csr(indptr, indices, data)
    nnz = int(indptr[-1])
    pT = np.empty(n + 1, dtype=np.int64)
    cT = np.empty(nnz, dtype=np.int32)
    vT = np.empty(nnz, dtype=np.float64)
    _check(_load().or_csr_transpose(m, n, _p(indptr), _p(indices), _p(data), _p(pT), _p(cT), _p(vT)), "csr_transpose")
    return pT, cT, vT


def spmm(m: int, n: int, indptr, indices, data, X: np.ndarray) -> np.ndarray:
    indptr, indices, data = _csr(indptr, indices, data)
    X = np.ascontiguousarray(X, dtype=np.float64)
    l = X.shape[1]
    Y = np.empty((m, l), dtype=np.float64)
    _check(_load().or_spmm(m, n, _p(indptr), _p(indices), _p(data), l, _p(X), l, _p(Y), l), "spmm")
    return Y


def spmm_t(m: int, n: int, indptr, indices, data, X: np.ndarray) -> np.ndarray:
    indptr, indices, data = _csr(indptr, indices, data)
    X = np.ascontiguousarray(X, dtype=np.float64)
    l = X.shape[1]
    Y = np.empty((n, l), dtype=np.float64)
    _check(_load().or_spmm_t(m, n, _p(indptr), _p(indices), _p(data), l, _p(X), l, _p(Y), l), "spmm_t")
    return Y


def lu_ptl(M: np.ndarray):
    """Returns (P^T L, pivot rows); raises OracleError(ERR_SINGULAR_PIVOT) on a zero column."""
    M = np.array(M, dtype=np.float64, order="C", copy=True)
    R, l = M.shape
    piv = np.empty(l, dtype=np.int64)
    _check(_load().or_lu_ptl(R, l, _p(M), l, _p(piv)), "lu_ptl")
    return M, piv


def eig_sym(B: np.ndarray):
    B = np.ascontiguousarray(B, dtype=np.float64)
    n = B.shape[0]
    w = np.empty(n, dtype=np.float64)
    V = np.empty((n, n), dtype=np.float64)
    sweeps = ctypes.c_int(0)
    _check(_load().or_eig_sym(n, _p(B), _p(w), _p(V), ctypes.byref(sweeps)), "eig_sym")
    return w, V


def gram(M: np.ndarray) -> np.ndarray:
    M = np.ascontiguousarray(M, dtype=np.float64)
    R, l = M.shape
    B = np.empty((l, l), dtype=np.float64)
    _check(_load().or_gram(R, l, _p(M), l, _p(B)), "gram")
    return B


def eigsvd(M: np.ndarray):
    """Alg. 2: returns (U, S ascending, V)."""
    M = np.ascontiguousarray(M, dtype=np.float64)
    R, l = M.shape
    U = np.empty((R, l), dtype=np.float64)
    S = np.empty(l, dtype=np.float64)
    V = np.empty((l, l), dtype=np.float64)
    _check(_load().or_eigsvd(R, l, _p(M), l, _p(U), l, _p(S), _p(V)), "eigsvd")
    return U, S, V


def frpca(m: int, n: int, indptr, indices, data, k: int, l: int, q: int, seed: int, alg: int | None = None,
          stabilize: bool = False, center: bool = False):
    """Alg. 5 / Alg. 6.  ``alg=None`` applies the shape rule (Alg. 6 when m >= n).

    ``stabilize=True`` runs the last power-iteration orthonormalization as
    eigSVD(lu(M)) (same range by Lemma 3, same result in exact arithmetic).
    ``center=True`` factors the column-centered A - 1 mu^T (PCA proper,
    Sec. 2.1) through rank-1 corrections of every product.
    """
    indptr, indices, data = _csr(indptr, indices, data)
    if alg is None:
        alg = 6 if m >= n else 5
    U = np.empty((m, k), dtype=np.float64)
    S = np.empty(k, dtype=np.float64)
    V = np.empty((n, k), dtype=np.float64)
    _check(_load().or_frpca_ex(alg, m, n, _p(indptr), _p(indices), _p(data), k, l, q, seed, int(stabilize),
                               int(center), _p(U), _p(S), _p(V)), "frpca")
    return U, S, V


def svd_adjoint_sddmm(m: int, n: int, indptr, indices, U, S, V, dU=None, dS=None, dV=None):
    """Gradient with respect to the CSR values of a loss of the rank-k truncated
    SVD (U, S, V) with cotangents (dU, dS, dV), each optional: the thin-SVD
    adjoint (Townsend 2016) sampled at the nonzeros.  Not part of the paper."""
    indptr = np.ascontiguousarray(indptr, dtype=np.int64)
    indices = np.ascontiguousarray(indices, dtype=np.int32)
    f64 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    U, S, V, dU, dS, dV = map(f64, (U, S, V, dU, dS, dV))
    k = S.shape[0]
    assert U.shape == (m, k) and V.shape == (n, k)
    assert dU is None or dU.shape == (m, k)
    assert dV is None or dV.shape == (n, k)
    out = np.empty(int(indptr[-1]), dtype=np.float64)
    opt = lambda a: None if a is None else _p(a)  # noqa: E731
    _check(_load().or_svd_adjoint_sddmm(m, n, _p(indptr), _p(indices), k, _p(U), _p(S), _p(V), opt(dU),
                                        opt(dS), opt(dV), _p(out)), "svd_adjoint_sddmm")
    return out
