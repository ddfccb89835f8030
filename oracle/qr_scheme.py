"""Basic rPCA (Alg. 1) and basic rPCAt (Alg. 4) with QR orthonormalization.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).  These are the comparison
algorithms of Theorems 1 and 2: frPCA with an even pass count q equals basic
rPCA with power parameter p = (q-2)/2 in exact arithmetic, and the modified
power iteration of Sec. 3.2 (Q = Omega = randn(m, k+s), one pass fewer) covers
odd q.  orth() is numpy's Householder QR, svd() numpy's LAPACK SVD, and the
sparse products come from the oracle, so a mistake in the oracle's LU, Jacobi
or eigSVD code cannot hide behind a shared routine.
"""
from __future__ import annotations

import numpy as np

from . import gaussian, spmm, spmm_t


def _orth(X: np.ndarray) -> np.ndarray:
    Q, _ = np.linalg.qr(X, mode="reduced")
    return Q


def rpca_t(m, n, indptr, indices, data, k, l, p, seed, modified=False):
    """Alg. 4 (random matrix on the left of A).

    ``modified=True`` replaces Steps 1-2 by Q = Omega = randn(n, k+s) (the
    Sec. 3.2 variant written for Alg. 4's roles), giving 2p+1 passes.
    Returns U (m x k), S (k, descending), V (n x k).
    """
    A = (m, n, indptr, indices, data)
    if modified:
        Q = gaussian(n, l, seed)
    else:
        G = gaussian(m, l, seed)          # row i = column i of randn(k+s, m)
        Q = _orth(spmm_t(*A, G))          # orth((Omega A)^T)
    for _ in range(p):
        Gq = _orth(spmm(*A, Q))           # G = orth(A Q)
        Q = _orth(spmm_t(*A, Gq))         # Q = orth(A^T G)
    B = spmm(*A, Q).T                     # B = (A Q)^T, l x m
    Uh, Sh, Vht = np.linalg.svd(B, full_matrices=False)
    V = Q @ Uh                            # V = Q U^
    U = Vht.T                             # U = V^(:, 1:k)
    return U[:, :k], Sh[:k], V[:, :k]


def rpca(m, n, indptr, indices, data, k, l, p, seed, modified=False):
    """Alg. 1 (random matrix on the right of A); ``modified`` as in Sec. 3.2."""
    A = (m, n, indptr, indices, data)
    if modified:
        Q = gaussian(m, l, seed)          # Q = Omega = randn(m, k+s)
    else:
        Om = gaussian(n, l, seed)
        Q = _orth(spmm(*A, Om))
    for _ in range(p):
        G = _orth(spmm_t(*A, Q))
        Q = _orth(spmm(*A, G))
    B = spmm_t(*A, Q).T                   # B = Q^T A, l x n
    Ub, Sb, Vbt = np.linalg.svd(B, full_matrices=False)
    U = Q @ Ub
    return U[:, :k], Sb[:k], Vbt.T[:, :k]
