"""Backward (the SVD adjoint + SDDMM kernels and the autograd Function) on the
GPU, through the C ABI.

Parity: ``frpca_backward`` against the oracle's adjoint on the same (U, S, V,
dU, dS, dV), element by element: FP64 within 1e-11 and FP32 within 2e-5 of the
largest gradient entry (FP32 forms 2k-term dot products of factors computed in
float from an FP64 k x k algebra).  End to end: the autograd gradient of
loss = sum(S) + ||U^T Y||^2 + ||V^T Z||^2 against central finite differences of
a dense FP64 SVD on a planted rank-k instance (exact adjoint), within 1e-6
(FP64) and 1e-3 (FP32) relative, and the sigma-sum gradient against PyTorch's
dense SVD autograd on the generator's 300 x 200 instance.
"""
import numpy as np
import pytest

import synthetic
from tests.helpers import block_rank_csr

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1810_06825_gb300 as frpca  # noqa: E402

DEV = "cuda:0"
PTOL = {torch.float64: 1e-11, torch.float32: 2e-5}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _orth(rng, r, k):
    Q, _ = np.linalg.qr(rng.standard_normal((r, k)))
    return Q


def _inputs(A, k, seed, with_u=True, with_s=True, with_v=True):
    rng = np.random.default_rng(seed)
    U, V = _orth(rng, A.m, k), _orth(rng, A.n, k)
    S = np.sort(rng.uniform(1.0, 3.0, k))[::-1] * (1.0 + 0.05 * np.arange(k))[::-1]
    dU = rng.standard_normal((A.m, k)) if with_u else None
    dS = rng.standard_normal(k) if with_s else None
    dV = rng.standard_normal((A.n, k)) if with_v else None
    return U, np.ascontiguousarray(S), V, dU, dS, dV


def _gpu_backward(mat, dt, U, S, V, dU, dS, dV):
    t = lambda a, d: None if a is None else torch.tensor(a, dtype=d, device=DEV).contiguous()  # noqa: E731
    out = mat.backward(t(U, dt), t(S, torch.float64), t(V, dt), t(dU, dt), t(dS, torch.float64), t(dV, dt))
    return out.double().cpu().numpy()


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
@pytest.mark.parametrize("k", [1, 5, 16, 33, 64])
def test_backward_matches_oracle(dt, k):
    A = synthetic.powerlaw_csr(3000, 800, 20, 1.1, "tfidf", seed=4, dtype=np.float64)
    U, S, V, dU, dS, dV = _inputs(A, k, seed=k)
    ref = oracle.svd_adjoint_sddmm(A.m, A.n, A.indptr, A.indices, U, S, V, dU, dS, dV)
    mat = frpca.FrPCA.from_csr(A, device=DEV, dtype=np.float32 if dt == torch.float32 else np.float64)
    got = _gpu_backward(mat, dt, U, S, V, dU, dS, dV)
    mat.close()
    assert np.max(np.abs(got - ref)) <= PTOL[dt] * np.max(np.abs(ref))


@pytest.mark.parametrize("which", [(True, False, False), (False, True, False), (False, False, True),
                                   (False, False, False)])
def test_backward_partial_cotangents(which):
    A = synthetic.powerlaw_csr(1500, 700, 12, 1.1, "tfidf", seed=6, dtype=np.float64)
    U, S, V, dU, dS, dV = _inputs(A, 12, 3, *which)
    ref = oracle.svd_adjoint_sddmm(A.m, A.n, A.indptr, A.indices, U, S, V, dU, dS, dV)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    got = _gpu_backward(mat, torch.float64, U, S, V, dU, dS, dV)
    mat.close()
    scale = max(np.max(np.abs(ref)), 1e-300)
    assert np.max(np.abs(got - ref)) <= 1e-11 * scale


def test_backward_empty_rows_and_long_rows():
    """Rows without entries, a 1,400-entry row and a hot column."""
    rng = np.random.default_rng(2)
    m, n = 900, 1500
    rows, cols = [], []
    for i in range(m):
        if i % 7 == 0:
            continue
        d = 1400 if i == 5 else rng.integers(1, 30)
        c = np.unique(np.concatenate([[0], rng.choice(n, size=d, replace=False)]))
        rows.append(np.full(c.size, i)); cols.append(c)
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    A = synthetic.from_coo(m, n, rows, cols, rng.standard_normal(rows.size))
    U, S, V, dU, dS, dV = _inputs(A, 20, 9)
    ref = oracle.svd_adjoint_sddmm(A.m, A.n, A.indptr, A.indices, U, S, V, dU, dS, dV)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    got = _gpu_backward(mat, torch.float64, U, S, V, dU, dS, dV)
    mat.close()
    assert np.max(np.abs(got - ref)) <= 1e-11 * np.max(np.abs(ref))


def test_backward_rejects_bad_sigma():
    A = synthetic.powerlaw_csr(400, 200, 8, 1.1, "tfidf", seed=1, dtype=np.float64)
    U, S, V, dU, dS, dV = _inputs(A, 6, 1)
    S[3] = 0.0
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    with pytest.raises(frpca.FrpcaError) as ei:
        _gpu_backward(mat, torch.float64, U, S, V, dU, dS, dV)
    assert ei.value.status == 1
    mat.close()


def _canon(U, V):
    idx = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[idx, np.arange(V.shape[1])])
    return U * sgn, V * sgn


def _dense_loss(D, k, Y, Z):
    U, S, Vt = np.linalg.svd(D, full_matrices=False)
    U, V = _canon(U[:, :k], Vt[:k].T)
    return S[:k].sum() + np.sum((U.T @ Y) ** 2) + np.sum((V.T @ Z) ** 2)


@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-6), (torch.float32, 1e-3)])
@pytest.mark.parametrize("q", [3, 4])
def test_autograd_planted_rank_k_finite_differences(dt, tol, q):
    """frPCA with l = k on an exactly rank-k matrix is the exact top-k SVD, and
    the adjoint is exact: the autograd gradient matches central differences of
    the dense SVD's loss."""
    m, n, k = 300, 200, 8
    A, _, _, _ = block_rank_csr(m, n, k, seed=11, scales=1.3 ** -np.arange(k))
    rng = np.random.default_rng(3)
    Y, Z = rng.standard_normal((m, 3)), rng.standard_normal((n, 2))
    npdt = np.float64 if dt == torch.float64 else np.float32
    vals = torch.tensor(A.data.astype(npdt), device=DEV, requires_grad=True)
    ip = torch.tensor(A.indptr, device=DEV)
    ix = torch.tensor(A.indices, device=DEV)
    U, S, V = frpca.frpca_svd(vals, ip, ix, (m, n), k, k, q, seed=0)
    Yt, Zt = torch.tensor(Y, dtype=dt, device=DEV), torch.tensor(Z, dtype=dt, device=DEV)
    loss = S.sum() + ((U.T @ Yt) ** 2).sum().double() + ((V.T @ Zt) ** 2).sum().double()
    loss.backward()
    g = vals.grad.double().cpu().numpy()
    D = A.to_dense().astype(np.float64)
    h = 1e-6 * np.max(np.abs(A.data))
    rows = A.row_ids()
    sample = rng.choice(A.nnz, size=30, replace=False)
    fd = np.empty(sample.size)
    for t, e in enumerate(sample):
        Dp, Dm = D.copy(), D.copy()
        Dp[rows[e], A.indices[e]] += h
        Dm[rows[e], A.indices[e]] -= h
        fd[t] = (_dense_loss(Dp, k, Y, Z) - _dense_loss(Dm, k, Y, Z)) / (2 * h)
    assert np.max(np.abs(g[sample] - fd)) <= tol * np.max(np.abs(fd))


def test_autograd_sigma_sum_matches_dense_autograd():
    """d(sum of the top-k sigma)/d values on the generator's 300 x 200,
    ~3,000-nnz instance against torch.linalg.svdvals autograd (FP64): exact for
    simple singular values whatever the gap, up to the frPCA error in U, V."""
    A = synthetic.powerlaw_csr(300, 200, 10, 1.1, "tfidf", seed=5, dtype=np.float64)
    k, l, q = 32, 48, 61
    vals = torch.tensor(A.data, device=DEV, requires_grad=True)
    U, S, V = frpca.frpca_svd(vals, torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV),
                              (A.m, A.n), k, l, q, seed=0)
    S.sum().backward()
    g = vals.grad.cpu().numpy()
    Dt = torch.tensor(A.to_dense(), dtype=torch.float64, requires_grad=True)
    torch.linalg.svdvals(Dt)[:k].sum().backward()
    ref = Dt.grad.numpy()[A.row_ids(), A.indices]
    # sigma_49 / sigma_32 = 0.82 here: the top-k subspaces from q = 61 passes
    # agree with the exact ones to ~0.82^61 = 4e-6.
    assert np.max(np.abs(g - ref)) <= 1e-4 * np.max(np.abs(ref))


def test_autograd_reuses_borrowing_handle():
    A = synthetic.powerlaw_csr(2000, 600, 15, 1.1, "tfidf", seed=8, dtype=np.float32)
    vals = torch.tensor(A.data, device=DEV, requires_grad=True)
    ip, ix = torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV)
    mat = frpca.FrPCA(ip, ix, vals.detach(), (A.m, A.n))
    g = []
    for _ in range(2):
        vals.grad = None
        U, S, V = frpca.frpca_svd(vals, ip, ix, (A.m, A.n), 10, 20, 4, mat=mat)
        S.sum().backward()
        g.append(vals.grad.clone())
    assert torch.equal(g[0], g[1])
    with torch.no_grad():
        vals.mul_(2.0)
    U2, S2, V2 = frpca.frpca_svd(vals, ip, ix, (A.m, A.n), 10, 20, 4, mat=mat)
    assert torch.allclose(S2, 2.0 * S, rtol=1e-5)
    mat.close()


def test_backward_workload_100000x20000_sampled():
    """The differentiation workload (100,000 x 20,000, ~5M nnz, k=32, l=48,
    q=4): loss = sum(S) + ||U^T Y||^2 with Y 100,000 x 8.  The GPU gradient
    (FP32) against the oracle's adjoint of the GPU's own (U, S, V) and the
    same cotangents, on every nonzero."""
    A = synthetic.make_workload("powerlaw_100000x20000_deg50")
    k, l, q = 32, 48, 4
    vals = torch.tensor(A.data, device=DEV, requires_grad=True)
    ip, ix = torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV)
    U, S, V = frpca.frpca_svd(vals, ip, ix, (A.m, A.n), k, l, q, seed=0)
    Y = torch.tensor(np.random.default_rng(2).standard_normal((A.m, 8)), dtype=torch.float32, device=DEV)
    loss = S.sum() + ((U.T @ Y) ** 2).sum().double()
    loss.backward()
    g = vals.grad.double().cpu().numpy()
    Un, Sn, Vn, Yn = (t.detach().double().cpu().numpy() for t in (U, S, V, Y))
    dU = 2.0 * Yn @ (Yn.T @ Un)
    ref = oracle.svd_adjoint_sddmm(A.m, A.n, A.indptr, A.indices, Un, Sn, Vn, dU, np.ones(k), None)
    # dU is formed by torch in float on the GPU and in double here: allow that too.
    assert np.max(np.abs(g - ref)) <= 1e-4 * np.max(np.abs(ref))
