"""Comparison metrics shared by the tests (no frPCA arithmetic)."""
import numpy as np


def orthonormal_basis(X):
    Q, _ = np.linalg.qr(np.asarray(X, dtype=np.float64), mode="reduced")
    return Q


def max_principal_sine(X, Y, orthonormalize=True):
    """sin of the largest principal angle between range(X) and range(Y)."""
    if orthonormalize:
        X, Y = orthonormal_basis(X), orthonormal_basis(Y)
    if X.shape[1] != Y.shape[1]:
        raise ValueError("bases of different dimension")
    # sin of the largest angle = || (I - X X^T) Y ||_2 (accurate near 0).
    R = Y - X @ (X.T @ Y)
    return float(np.linalg.norm(R, 2)) if R.size else 0.0


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.max(np.abs(a - b) / np.maximum(np.abs(b), 1e-300)))


def dense_svd_topk(A, k):
    U, S, Vt = np.linalg.svd(A, full_matrices=False)
    return U[:, :k], S[:k], Vt[:k].T
