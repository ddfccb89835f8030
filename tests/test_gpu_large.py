"""The large sparse PCA workload at full size: 12,000,000 x 320,000, ~480M nnz
(row degrees log-normal mean 40, column Zipf s=1.05, binary tf-idf values),
FP32, int32 indices, A and A^T both resident on the GPU; k=100, l=120, q=5
(Alg. 6, the odd-pass scheme).

test_large_powerlaw_matches_oracle runs the whole FP64 oracle on the same
matrix and Gaussian test matrix and gates the FP32 path at the stated
tolerances: singular values within 1e-4 relative, element by element, and the
largest principal-angle sines of U and V within 1e-3.

test_large_powerlaw_12000000x320000_fp32 checks what holds at any size (Alg.
6's final step and the orthonormality of its factors) plus the convergence of
the leading triplet, with the oracle forming single outputs:

- A V = U diag(S) on seeded rows: the final step gives U = A Q V^ diag(1./S^)
  and V = Q V^, so the identity holds up to float rounding of the last pass
  and the applies; the oracle forms A(i,:) V for the sampled rows.
- U^T U = V^T V = I (both are orthonormal by construction: eigSVD's U and
  V = Q V^ with an orthonormal Q).
- S positive and descending (ind = k+s : -1 : s+1).
- A^T U(:, 1) = S(1) V(:, 1) on seeded columns of A taken from the oracle's
  transpose: the leading singular value of this matrix stands about 4x above
  the next, so q = 5 passes converge its triplet (the next ones sit in a flat
  stretch of the spectrum, where single triplets are not determined and only
  the subspace is).
"""
import numpy as np
import pytest

import synthetic

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1810_06825_gb300 as frpca  # noqa: E402

DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _sub_rows(indptr, indices, data, rows):
    """CSR of the given rows (in order) of a CSR matrix."""
    starts, ends = indptr[rows], indptr[rows + 1]
    lens = ends - starts
    sub_ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    np.cumsum(lens, out=sub_ptr[1:])
    take = np.concatenate([np.arange(s, e) for s, e in zip(starts, ends)]) if len(rows) else np.zeros(0, np.int64)
    return sub_ptr, indices[take], data[take]


def _gram64(X, chunk=1 << 20):
    """X^T X in FP64, by row chunks (X may be large and float32)."""
    G = np.zeros((X.shape[1], X.shape[1]))
    for r in range(0, X.shape[0], chunk):
        Xc = X[r:r + chunk].astype(np.float64)
        G += Xc.T @ Xc
    return G


@pytest.fixture(scope="module")
def large():
    return synthetic.make_workload("powerlaw_12000000x320000_deg40")


def _sine_from_grams(X, Y, chunk=1 << 20):
    """Largest principal-angle sine between range(X) and range(Y) for tall X, Y
    (same width), from FP64 Gram-sized products only: with X^T X = Lx Lx^T and
    Y^T Y = Ly Ly^T, the cosines of the principal angles are the singular
    values of Lx^-1 X^T Y Ly^-T."""
    k = X.shape[1]
    Gx, Gy, C = np.zeros((k, k)), np.zeros((k, k)), np.zeros((k, k))
    for r in range(0, X.shape[0], chunk):
        Xc, Yc = X[r:r + chunk].astype(np.float64), Y[r:r + chunk].astype(np.float64)
        Gx += Xc.T @ Xc
        Gy += Yc.T @ Yc
        C += Xc.T @ Yc
    Lx, Ly = np.linalg.cholesky(Gx), np.linalg.cholesky(Gy)
    Mx = np.linalg.solve(Lx, C)
    Mxy = np.linalg.solve(Ly, Mx.T).T
    cmin = float(np.linalg.svd(Mxy, compute_uv=False).min())
    return float(np.sqrt(max(0.0, 1.0 - min(cmin, 1.0) ** 2)))


def test_large_powerlaw_matches_oracle(large):
    """FP32 GPU path vs the FP64 oracle at full size (Alg. 6, q = 5, same
    Philox Omega): sigma within 1e-4 relative element by element, principal-
    angle sines of U and V within 1e-3."""
    A = large
    k, l, q = 100, 120, 5
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    U, S, V = mat.run(k, l, q, seed=0, precision="fp32")
    U, S, V = U.cpu().numpy(), S.cpu().numpy(), V.cpu().numpy()
    mat.close()
    del mat
    torch.cuda.empty_cache()
    Uo, So, Vo = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), k, l, q, 0)
    es = float(np.max(np.abs(S - So) / So))
    eu = _sine_from_grams(U, Uo)
    ev = _sine_from_grams(V, Vo)
    print(f"large workload vs oracle: sigma rel {es:.2e}, sine U {eu:.2e}, sine V {ev:.2e}")
    assert es <= 1e-4
    assert eu <= 1e-3 and ev <= 1e-3


def test_large_powerlaw_12000000x320000_fp32(large):
    A = large
    k, l, q = 100, 120, 5
    assert A.nnz > 400_000_000
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    U, S, V = mat.run(k, l, q, seed=0, precision="fp32")
    # A second run, timed on the device (A^T rebuild + the whole method).
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(mat.stream)
    mat.refresh()
    mat.run(k, l, q, seed=0, precision="fp32", out=(U, S, V), sync=False)
    t1.record(mat.stream)
    torch.cuda.synchronize()
    print(f"refresh + run: {t0.elapsed_time(t1):.1f} ms")
    U = U.cpu().numpy()
    S = S.double().cpu().numpy()
    V = V.cpu().numpy()
    mat.close()
    del mat
    torch.cuda.empty_cache()

    assert np.all(np.isfinite(U)) and np.all(np.isfinite(S)) and np.all(np.isfinite(V))
    assert np.all(S > 0) and np.all(np.diff(S) <= 0)
    # Orthonormal factors (float storage of a 12M-row block: a few 1e-6).
    eu = np.max(np.abs(_gram64(U) - np.eye(k)))
    ev = np.max(np.abs(_gram64(V) - np.eye(k)))
    print(f"|U^T U - I| {eu:.2e}, |V^T V - I| {ev:.2e}")
    assert eu <= 1e-4 and ev <= 1e-4

    # A V = U diag(S) on 2,000 seeded rows, A(i,:) V by the oracle.
    rows = np.sort(np.random.default_rng(5).choice(A.m, size=2000, replace=False))
    sp, si, sd = _sub_rows(A.indptr, A.indices, A.data, rows)
    AV = oracle.spmm(len(rows), A.n, sp, si, sd.astype(np.float64), V.astype(np.float64))
    US = U[rows].astype(np.float64) * S
    row_norm = np.sqrt(np.add.reduceat(sd.astype(np.float64) ** 2, sp[:-1])) if sp[-1] else np.zeros(len(rows))
    err = np.linalg.norm(AV - US, axis=1) / np.maximum(row_norm, 1e-30)
    print(f"A V = U S on sampled rows: max rel residual {err.max():.2e}")
    assert err.max() <= 1e-4

    # A^T U(:, 1) = S(1) V(:, 1) on 2,000 seeded columns of A (rows of the
    # oracle's transpose).
    pT, cT, vT = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64))
    cols = np.sort(np.random.default_rng(6).choice(A.n, size=2000, replace=False))
    tp, ti, td = _sub_rows(pT, cT, vT, cols)
    lead = 1
    assert S[0] > 2.0 * S[1]  # the gap that converges the leading triplet
    ATU = oracle.spmm(len(cols), A.m, tp, ti, td, U[:, :lead].astype(np.float64))
    SV = V[cols, :lead].astype(np.float64) * S[:lead]
    # Residual over the sampled coordinates, relative to S(1) times the
    # sampled part of a unit vector (sqrt(2000 / n)).
    res = np.linalg.norm(ATU - SV, axis=0) / (S[:lead] * np.sqrt(len(cols) / A.n))
    print(f"A^T u_1 = s_1 v_1, sampled rel residual: {res[0]:.2e}")
    assert np.all(res <= 1e-2)
