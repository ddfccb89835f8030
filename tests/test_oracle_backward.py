"""Pins for the oracle's backward (the thin-SVD adjoint sampled at A's
nonzeros), each against something other than the oracle: PyTorch's autograd
of a dense FP64 SVD, central finite differences of the top-k functional, and
the closed form d sigma_a / dA = u_a v_a^T.
"""
import numpy as np
import pytest
import torch

import synthetic
from tests.helpers import block_rank_csr


def _dense(A):
    return A.to_dense().astype(np.float64)


def _canon(U, V):
    """Sign convention of this build: largest-|.| entry of each v_j positive."""
    idx = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[idx, np.arange(V.shape[1])])
    sgn[sgn == 0] = 1.0
    return U * sgn, V * sgn


def _topk(D, k):
    U, S, Vt = np.linalg.svd(D, full_matrices=False)
    U, V = _canon(U[:, :k], Vt[:k].T)
    return U, S[:k], V


@pytest.mark.parametrize("shape,density", [((14, 9), 1.0), ((23, 11), 0.6), ((9, 14), 0.7)])
def test_adjoint_full_thin_svd_matches_torch(oracle_lib, shape, density):
    """k = min(m, n): the truncated adjoint is the full thin-SVD adjoint, which
    torch.linalg.svd's autograd computes independently (FP64)."""
    m, n = shape
    rng = np.random.default_rng(7 + m)
    D = rng.standard_normal((m, n)) * (rng.random((m, n)) < density)
    A = synthetic.from_dense(D)
    k = min(m, n)
    At = torch.tensor(_dense(A), dtype=torch.float64, requires_grad=True)
    U, S, Vh = torch.linalg.svd(At, full_matrices=False)
    V = Vh.mT
    gU = torch.tensor(rng.standard_normal((m, k)))
    gS = torch.tensor(rng.standard_normal(k))
    gV = torch.tensor(rng.standard_normal((n, k)))
    loss = (U * gU).sum() + (S * gS).sum() + (V * gV).sum()
    loss.backward()
    G = At.grad.numpy()
    out = oracle_lib.svd_adjoint_sddmm(m, n, A.indptr, A.indices, U.detach().numpy(), S.detach().numpy(),
                                       V.detach().numpy(), gU.numpy(), gS.numpy(), gV.numpy())
    ref = G[A.row_ids(), A.indices]
    assert np.max(np.abs(out - ref)) <= 1e-9 * np.max(np.abs(ref))


def test_adjoint_sigma_term_closed_form(oracle_lib):
    """d(sum_a c_a sigma_a)/dA = sum_a c_a u_a v_a^T for simple singular values,
    with no gap needed between sigma_k and sigma_{k+1}: checked against the
    autograd of a dense FP64 SVD on the generator's 300 x 200 instance."""
    A = synthetic.powerlaw_csr(300, 200, 10, 1.1, "tfidf", seed=5, dtype=np.float64)
    k = 32
    D = _dense(A)
    At = torch.tensor(D, requires_grad=True)
    S = torch.linalg.svdvals(At)
    c = torch.linspace(1.0, 2.0, k, dtype=torch.float64)
    (S[:k] * c).sum().backward()
    U, Sk, V = _topk(D, k)
    out = oracle_lib.svd_adjoint_sddmm(A.m, A.n, A.indptr, A.indices, U, Sk, V, None, c.numpy(), None)
    ref = At.grad.numpy()[A.row_ids(), A.indices]
    assert np.max(np.abs(out - ref)) <= 1e-10 * np.max(np.abs(ref))


def _loss_parts(D, k, Y, Z):
    U, S, V = _topk(D, k)
    return S.sum() + np.sum((U.T @ Y) ** 2) + np.sum((V.T @ Z) ** 2)


@pytest.mark.parametrize("shape", [(300, 200), (120, 180)])
def test_adjoint_planted_rank_k_finite_differences(oracle_lib, shape):
    """Planted rank-k sparse A (k disjoint rank-1 blocks, distinct scales): the
    discarded spectrum is zero, so the truncated adjoint is the exact gradient
    of loss = sum sigma + ||U^T Y||^2 + ||V^T Z||^2; central differences with
    h = 1e-6 max|a| at sampled nonzeros agree to 1e-6 relative."""
    m, n = shape
    k = 8
    A, sig, _, _ = block_rank_csr(m, n, k, seed=11, scales=1.3 ** -np.arange(k))
    rng = np.random.default_rng(3)
    Y = rng.standard_normal((m, 3))
    Z = rng.standard_normal((n, 2))
    D = _dense(A)
    U, S, V = _topk(D, k)
    dU = 2.0 * Y @ (Y.T @ U)
    dV = 2.0 * Z @ (Z.T @ V)
    out = oracle_lib.svd_adjoint_sddmm(m, n, A.indptr, A.indices, U, S, V, dU, np.ones(k), dV)
    h = 1e-6 * np.max(np.abs(A.data))
    rows = A.row_ids()
    sample = rng.choice(A.nnz, size=40, replace=False)
    fd = np.empty(sample.size)
    for t, e in enumerate(sample):
        Dp, Dm = D.copy(), D.copy()
        Dp[rows[e], A.indices[e]] += h
        Dm[rows[e], A.indices[e]] -= h
        fd[t] = (_loss_parts(Dp, k, Y, Z) - _loss_parts(Dm, k, Y, Z)) / (2 * h)
    scale = np.max(np.abs(fd))
    assert np.max(np.abs(out[sample] - fd)) <= 1e-6 * scale


def test_adjoint_missing_cotangents_are_zero(oracle_lib):
    """No cotangent at all gives a zero gradient; dU alone and dV alone add up
    to the gradient with both (the adjoint is linear in the cotangents)."""
    A = synthetic.powerlaw_csr(120, 80, 8, 1.1, "tfidf", seed=2, dtype=np.float64)
    k = 6
    U, S, V = _topk(_dense(A), k)
    rng = np.random.default_rng(0)
    dU, dV = rng.standard_normal((A.m, k)), rng.standard_normal((A.n, k))
    f = lambda *c: oracle_lib.svd_adjoint_sddmm(A.m, A.n, A.indptr, A.indices, U, S, V, *c)  # noqa: E731
    assert np.all(f(None, None, None) == 0.0)
    both = f(dU, None, dV)
    assert np.allclose(f(dU, None, None) + f(None, None, dV), both, rtol=1e-12, atol=1e-12 * np.abs(both).max())


def test_adjoint_invalid_args(oracle_lib):
    A = synthetic.powerlaw_csr(20, 10, 3, 1.1, "tfidf", seed=2, dtype=np.float64)
    U, S, V = np.zeros((20, 2)), np.array([1.0, 0.0]), np.zeros((10, 2))
    with pytest.raises(Exception):
        oracle_lib.svd_adjoint_sddmm(20, 10, A.indptr, A.indices, U, S, V)
