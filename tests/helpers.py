"""Comparison metrics shared by the tests (no frPCA arithmetic)."""
import numpy as np

import synthetic


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


def block_rank_csr(m, n, blocks, seed, scales=None):
    """Sum of `blocks` disjoint rank-1 blocks x_b y_b^T * scale_b: its SVD is
    known in closed form (sigma_b = scale_b |x_b| |y_b|)."""
    rng = np.random.default_rng(seed)
    rperm, cperm = rng.permutation(m), rng.permutation(n)
    rsplit = np.array_split(rperm, blocks)
    csplit = np.array_split(cperm, blocks)
    if scales is None:
        scales = 2.0 ** (-0.5 * np.arange(blocks))
    rows, cols, vals, sig, U, V = [], [], [], [], np.zeros((m, blocks)), np.zeros((n, blocks))
    for b in range(blocks):
        x = rng.uniform(0.5, 1.5, size=rsplit[b].size) * rng.choice([-1, 1], size=rsplit[b].size)
        y = rng.uniform(0.5, 1.5, size=csplit[b].size) * rng.choice([-1, 1], size=csplit[b].size)
        rr, cc = np.meshgrid(rsplit[b], csplit[b], indexing="ij")
        rows.append(rr.ravel()); cols.append(cc.ravel()); vals.append((np.outer(x, y) * scales[b]).ravel())
        sig.append(scales[b] * np.linalg.norm(x) * np.linalg.norm(y))
        U[rsplit[b], b] = x / np.linalg.norm(x)
        V[csplit[b], b] = y / np.linalg.norm(y)
    A = synthetic.from_coo(m, n, np.concatenate(rows), np.concatenate(cols), np.concatenate(vals))
    order = np.argsort(-np.array(sig), kind="stable")
    return A, np.array(sig)[order], U[:, order], V[:, order]
