"""GPU parity of each step of the path against the FP64 CPU oracle, through the C ABI.

Tolerances: integer/index work bit-exact; the Gaussian generator's words
bit-exact (checked through the normals to within libm/CUDA rounding); FP64
SpMM within the summation bound d * eps * (|A||X|); FP32 SpMM within
(d + 2) * eps32 * (|A||X|); FP64 LU bit-exact (same operations, no fused
multiply-add); eigensolver within a few eps * ||B||.
"""
import numpy as np
import pytest

import synthetic
from tests.helpers import max_principal_sine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1810_06825_gb300 as frpca  # noqa: E402

EPS64 = np.finfo(np.float64).eps
EPS32 = np.finfo(np.float32).eps
DEV = "cuda:0"


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cpu(t):
    return t.detach().double().cpu().numpy()


# ---------------------------------------------------------------- Gaussian
@pytest.mark.parametrize("R,l", [(1, 1), (7, 5), (33, 20), (1000, 120), (50_000, 120), (4097, 13)])
@pytest.mark.parametrize("seed", [0, 12345])
def test_gaussian_matches_oracle(R, l, seed):
    ref = oracle.gaussian(R, l, seed)
    g64 = _cpu(frpca.gaussian(R, l, seed, dtype=torch.float64, device=DEV))
    # Same words; libm vs CUDA log/cos differ by a few ulps of r <= 8.6.
    assert np.max(np.abs(g64 - ref)) <= 200 * EPS64
    g32 = _cpu(frpca.gaussian(R, l, seed, dtype=torch.float32, device=DEV))
    # Float evaluation of the same formula: uniform rounding moves the angle by
    # at most 2 pi 2^-24, and ln(u) keeps relative accuracy at both ends.
    assert np.max(np.abs(g32 - ref)) <= 8e-6 + 4 * EPS32 * np.max(np.abs(ref))


# ---------------------------------------------------------------- transpose
def _mats():
    rng = np.random.default_rng(0)
    out = []
    # empty rows and columns, a dense row longer than one SpMM segment, a hot column
    m, n = 3000, 1500
    rows, cols = [], []
    for i in range(m):
        if i % 97 == 0:
            continue
        c = rng.choice(n, size=rng.integers(1, 12), replace=False)
        rows.append(np.full(c.size, i)); cols.append(c)
    rows.append(np.full(1400, 5)); cols.append(rng.choice(n, 1400, replace=False))
    hot = np.setdiff1d(np.arange(m), [5])
    rows.append(hot); cols.append(np.full(hot.size, 7))
    r = np.concatenate(rows); c = np.concatenate(cols)
    key = np.unique(r * n + c)
    r, c = key // n, key % n
    out.append(synthetic.from_coo(m, n, r, c, rng.standard_normal(r.size)))
    out.append(synthetic.powerlaw_csr(20_000, 3_000, 20, 1.1, "tfidf", seed=2, dtype=np.float64))
    out.append(synthetic.uniform_csr(2000, 1000, 20000, seed=1))
    # Row lengths at the edges of the SpMM work split: runs of empty rows (at
    # the start, inside and at the end), runs of one-entry rows longer than a
    # 32-row group, rows of 31-33 entries (one 32-entry chunk and a ragged
    # tail) and of 1,023-1,025 and 2,049 entries (a whole row at the segment
    # length, segments and their fix-up).
    m, n = 1200, 3000
    lens = np.zeros(m, dtype=np.int64)
    lens[40:120] = 1
    lens[130:200] = rng.integers(1, 4, 70)
    lens[[210, 211, 212, 300, 301, 302, 400]] = [31, 32, 33, 1023, 1024, 1025, 2049]
    lens[500:1100] = rng.integers(0, 40, 600)
    r = np.repeat(np.arange(m), lens)
    c = np.concatenate([np.sort(rng.choice(n, k, replace=False)) for k in lens if k])
    out.append(synthetic.from_coo(m, n, r, c, rng.standard_normal(r.size)))
    return out


MATS = _mats()


@pytest.mark.parametrize("idx", range(len(MATS)))
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_transpose_bit_exact(idx, dtype):
    A = MATS[idx].astype(dtype)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    pT, cT, vT = mat.transpose()
    rp, ci, va = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64))
    assert np.array_equal(pT.cpu().numpy(), rp)
    assert np.array_equal(cT.cpu().numpy(), ci)
    assert np.array_equal(vT.cpu().numpy(), va.astype(dtype))
    mat.close()


# ---------------------------------------------------------------- SpMM
def _spmm_bound(A, X, trans, eps, hot_block=False):
    """Element-wise bound on |Y - Y_exact|: a sum of d products in the CSR
    order rounds at most (d + 2) eps * (|A| |X|) (d additions, one product
    each, and the final store).  With the densest columns as a dense block on
    the tensor cores (hot_block), FP32 accumulation also rounds once per
    16-column K-step with a nonzero product (at most once per entry), plus the
    split remainder (< 2^-26 per product) and the sums of the correction
    accumulator and of the cold part: (2 d + 8) eps * (|A| |X|)."""
    Aabs = synthetic.CSR(A.m, A.n, A.indptr, A.indices, np.abs(A.data.astype(np.float64)))
    f = oracle.spmm_t if trans else oracle.spmm
    mag = f(Aabs.m, Aabs.n, Aabs.indptr, Aabs.indices, Aabs.data, np.abs(X))
    deg = np.diff(A.indptr) if not trans else np.bincount(A.indices, minlength=A.n)
    if hot_block:
        return (2 * deg[:, None] + 8) * eps * mag + 1e-300
    return (deg[:, None] + 2) * eps * mag + 1e-300


@pytest.mark.parametrize("idx", range(len(MATS)))
@pytest.mark.parametrize("l", [1, 5, 20, 48, 120, 160])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
@pytest.mark.parametrize("trans", [0, 1])
def test_spmm_matches_oracle(idx, l, dtype, trans):
    A = MATS[idx].astype(dtype)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    rng = np.random.default_rng(l)
    X = rng.standard_normal((A.m if trans else A.n, l)).astype(dtype)
    Xg = frpca.empty_block(X.shape[0], l, torch.float64 if dtype == np.float64 else torch.float32, DEV)
    Xg.copy_(torch.from_numpy(X))
    Y = _cpu(mat.spmm(Xg, trans=bool(trans)))
    f = oracle.spmm_t if trans else oracle.spmm
    ref = f(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), X.astype(np.float64))
    eps = EPS64 if dtype == np.float64 else EPS32
    bound = _spmm_bound(A, X.astype(np.float64), trans, eps)
    assert np.all(np.abs(Y - ref) <= bound)
    mat.close()


def _hot_matrix(m, n, seed):
    """Power-law CSR whose densest columns hold 5-60 % of the rows."""
    return synthetic.powerlaw_csr(m, n, 40, 1.1, "tfidf", seed=seed, dtype=np.float32)


@pytest.mark.parametrize("hot", [-1, 0, 128, 256])
@pytest.mark.parametrize("l", [1, 48, 120, 128])
@pytest.mark.parametrize("trans", [0, 1])
def test_spmm_hot_columns_match_oracle(hot, l, trans):
    """A X and A^T X with the densest columns on the tensor cores (forced
    block sizes, automatic (-1), and off (0)) against the oracle; rows of A^T at hot
    columns come from the dense block, the rest from the CSR of A^T."""
    A = _hot_matrix(9000, 2500, 3)
    mat = frpca.FrPCA.from_csr(A, device=DEV, hot_columns=hot)
    X = np.random.default_rng(l + trans).standard_normal((A.m if trans else A.n, l)).astype(np.float32)
    Xg = frpca.empty_block(X.shape[0], l, torch.float32, DEV)
    Xg.copy_(torch.from_numpy(X))
    Y = _cpu(mat.spmm(Xg, trans=bool(trans)))
    f = oracle.spmm_t if trans else oracle.spmm
    ref = f(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), X.astype(np.float64))
    assert np.all(np.abs(Y - ref) <= _spmm_bound(A, X.astype(np.float64), trans, EPS32, hot_block=hot != 0))
    mat.close()


def test_spmm_hot_columns_refresh_and_determinism():
    """After the values change in place, frpca_refresh rebuilds the dense block
    and the cold values; results stay deterministic."""
    A = _hot_matrix(6000, 1200, 4)
    vals = torch.tensor(A.data, device=DEV)
    mat = frpca.FrPCA(torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV), vals, (A.m, A.n),
                      hot_columns=128)
    X = frpca.empty_block(A.n, 64, torch.float32, DEV)
    X.copy_(torch.randn(A.n, 64, generator=torch.Generator().manual_seed(0)))
    Y1 = mat.spmm(X).clone()
    with torch.no_grad():
        vals.mul_(3.0)
    mat.refresh()
    Y3 = mat.spmm(X).clone()
    assert torch.allclose(Y3, 3.0 * Y1, rtol=1e-5, atol=1e-5 * float(Y1.abs().max()))
    assert torch.equal(mat.spmm(X), Y3)
    mat.close()


def test_spmm_is_deterministic():
    A = MATS[1].astype(np.float32)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    X = frpca.empty_block(A.m, 120, torch.float32, DEV)
    X.copy_(torch.randn(A.m, 120, generator=torch.Generator().manual_seed(0)))
    Y1 = mat.spmm(X, trans=True).clone()
    Y2 = mat.spmm(X, trans=True).clone()
    assert torch.equal(Y1, Y2)
    mat.close()


# ---------------------------------------------------------------- LU
@pytest.mark.parametrize("R,l", [(1, 1), (7, 7), (50, 8), (1000, 33), (20_000, 120), (5000, 160), (333, 17)])
def test_lu_fp64_bit_exact(R, l):
    M = np.random.default_rng(R + l).standard_normal((R, l))
    ref, piv_ref = oracle.lu_ptl(M)
    Mg = torch.from_numpy(M).to(DEV)
    PL, piv = frpca.lu(Mg)
    assert np.array_equal(piv.cpu().numpy(), piv_ref)
    assert np.array_equal(_cpu(PL), ref)


@pytest.mark.parametrize("R,l", [(50, 8), (20_000, 120), (4099, 48)])
def test_lu_fp32_spans_same_range(R, l):
    M = np.random.default_rng(R).standard_normal((R, l)).astype(np.float32)
    PL, piv = frpca.lu(torch.from_numpy(M).to(DEV))
    P = _cpu(PL)
    piv = piv.cpu().numpy()
    assert len(set(piv.tolist())) == l
    assert np.max(np.abs(P)) <= 1.0 + 1e-6
    for j, p in enumerate(piv):
        assert P[p, j] == 1.0 and np.all(P[p, j + 1:] == 0.0)
    assert max_principal_sine(P, M.astype(np.float64)) < 1e-4


def test_lu_singular_pivot_reports():
    M = np.random.default_rng(0).standard_normal((100, 6))
    M[:, 3] = 0.0
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.lu(torch.from_numpy(M).to(DEV))
    assert ei.value.status == 5


# ---------------------------------------------------------------- Gram / eig / eigSVD
@pytest.mark.parametrize("R,l", [(1, 1), (100, 20), (5000, 120), (200_000, 120), (777, 160)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_gram_matches_oracle(R, l, dtype):
    M = np.random.default_rng(R).standard_normal((R, l)).astype(dtype)
    B = _cpu(frpca.gram(torch.from_numpy(M).to(DEV)))
    ref = oracle.gram(M.astype(np.float64))
    scale = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
    eps = EPS64 if dtype == np.float64 else EPS32
    chunk = R if dtype == np.float64 else min(R, 4096)
    assert np.all(np.abs(B - ref) <= (chunk + 2) * eps * scale + 1e-300)
    assert np.array_equal(B, B.T)


@pytest.mark.parametrize("n", [1, 2, 5, 20, 64, 120, 121, 160])
def test_eig_matches_oracle(n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((3 * n, n))
    B = X.T @ X
    w, V = frpca.eig(torch.from_numpy(B).to(DEV))
    w, V = _cpu(w), _cpu(V)
    wr, Vr = oracle.eig_sym(B)
    nb = np.linalg.norm(B, 2)
    assert np.max(np.abs(w - wr)) <= 64 * EPS64 * nb
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-12)
    assert np.max(np.abs(B @ V - V * w)) <= 256 * EPS64 * nb
    gaps = np.diff(wr)
    for j in range(n):
        gap = min(gaps[j - 1] if j > 0 else np.inf, gaps[j] if j < n - 1 else np.inf)
        if gap > 1e-6 * nb:
            assert abs(abs(V[:, j] @ Vr[:, j]) - 1) <= 1e-9


def test_eig_clustered_and_indefinite():
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((40, 40)))
    d = np.concatenate([np.full(10, 2.0), np.linspace(-1, 1, 20), np.full(10, 5.0 + 1e-9)])
    B = (Q * d) @ Q.T
    B = (B + B.T) / 2
    w, V = frpca.eig(torch.from_numpy(B).to(DEV))
    w, V = _cpu(w), _cpu(V)
    assert np.allclose(np.sort(d), w, atol=1e-12)
    assert np.allclose(V.T @ V, np.eye(40), atol=1e-12)
    assert np.allclose(B @ V, V * w, atol=1e-11)


@pytest.mark.parametrize("R,l,cond", [(500, 20, 10.0), (20_000, 120, 100.0), (3000, 160, 30.0)])
@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_eigsvd_matches_oracle(R, l, cond, dtype):
    rng = np.random.default_rng(R)
    Uq, _ = np.linalg.qr(rng.standard_normal((R, l)))
    Vq, _ = np.linalg.qr(rng.standard_normal((l, l)))
    M = ((Uq * np.geomspace(1, 1 / cond, l)) @ Vq.T).astype(dtype)
    U, S, V = frpca.eigsvd(torch.from_numpy(M).to(DEV))
    Uo, So, Vo = oracle.eigsvd(M.astype(np.float64))
    S, U = _cpu(S), _cpu(U)
    tol = 1e-10 if dtype == np.float64 else 1e-4
    assert np.max(np.abs(S - So) / So) <= tol
    assert np.allclose(U.T @ U, np.eye(l), atol=(1e-10 if dtype == np.float64 else 1e-3))
    assert max_principal_sine(U, Uo) <= (1e-10 if dtype == np.float64 else 1e-3)


@pytest.mark.parametrize("R,l", [(1, 1), (127, 7), (129, 64), (300, 65), (1000, 128), (4097, 120), (40000, 33),
                                 (60001, 120)])
def test_eigsvd_apply_step_elementwise(R, l):
    """Step 5 of Alg. 2 in FP32 (U = M V spdiags(1./S), on the tensor cores for
    l <= 128): every entry of U against the product formed in FP64 from the
    returned S and V, with the float accumulation bound of an l-term sum;
    covers ragged 128-row tiles, ragged 32-column chunks and (R > 152 x 128)
    several tiles per CTA."""
    rng = np.random.default_rng(R + l)
    Uq, _ = np.linalg.qr(rng.standard_normal((R, l)))
    Vq, _ = np.linalg.qr(rng.standard_normal((l, l)))
    M = ((Uq * np.geomspace(1, 0.1, l)) @ Vq.T).astype(np.float32)
    U, S, V = frpca.eigsvd(torch.from_numpy(M).to(DEV))
    U, S, V = _cpu(U), _cpu(S), _cpu(V)
    W = (V / S).astype(np.float32).astype(np.float64)  # the float W the step multiplies by
    Md = M.astype(np.float64)
    ref = Md @ W
    bound = (l + 8) * 2.0**-23 * (np.abs(Md) @ np.abs(W))
    assert np.all(np.abs(U - ref) <= bound)


def test_eigsvd_rank_deficient_reports():
    M = np.random.default_rng(0).standard_normal((300, 8))
    M[:, 7] = M[:, 0] - M[:, 2]
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.eigsvd(torch.from_numpy(M).to(DEV))
    assert ei.value.status == 6


def test_invalid_csr_rejected_on_device():
    A = synthetic.uniform_csr(50, 40, 300, seed=3)
    bad = A.indices.copy()
    s = A.indptr[7]
    bad[s], bad[s + 1] = bad[s + 1], bad[s]  # unsorted row
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.FrPCA(torch.from_numpy(A.indptr).to(DEV), torch.from_numpy(bad).to(DEV),
                    torch.from_numpy(A.data).to(DEV), (A.m, A.n))
    assert ei.value.status == 2
    bad = A.indices.copy()
    bad[3] = 40  # column out of range
    with pytest.raises(frpca.FrpcaError):
        frpca.FrPCA(torch.from_numpy(A.indptr).to(DEV), torch.from_numpy(bad).to(DEV),
                    torch.from_numpy(A.data).to(DEV), (A.m, A.n))


# ---------------------------------------------------------------- LU, tournament pivoting (FP32 path)
def _lu_tournament(M):
    R, l = M.shape
    A = frpca.empty_block(R, l, torch.float32, DEV)
    A.copy_(torch.from_numpy(M).to(DEV))
    piv = torch.empty(l, dtype=torch.int64, device=DEV)
    frpca.frpca_lu_tournament(frpca._Context.get(), R, l, A.data_ptr(), A.stride(0), piv.data_ptr())
    return _cpu(A), piv.cpu().numpy()


@pytest.mark.parametrize("R,l", [(50, 8), (300, 45), (4099, 48), (20_000, 120), (50_000, 120), (9_000, 160),
                                 (1000, 1), (33, 33), (100_003, 120), (320_000, 120), (600_001, 37)])
def test_lu_tournament_structure_and_range(R, l):
    """Lemma 3 for any pivot rows: range(P^T L) = range(M); the pivot row of
    column j holds 1 at j and 0 right of j; the unit lower factor stays
    moderate (tournament pivoting does not bound it by 1).  Up to 512 rows per
    block the rows are cached in shared memory; the larger cases (100,003 to
    600,001 rows) take the form that updates them in place in global memory."""
    M = np.random.default_rng(R + 7 * l).standard_normal((R, l)).astype(np.float32)
    P, piv = _lu_tournament(M)
    assert len(set(piv.tolist())) == l and piv.min() >= 0 and piv.max() < R
    for j, p in enumerate(piv):
        assert P[p, j] == 1.0 and np.all(P[p, j + 1:] == 0.0)
    assert np.all(np.isfinite(P)) and np.max(np.abs(P)) <= 16.0
    assert max_principal_sine(P, M.astype(np.float64)) < 1e-4


def test_lu_tournament_matches_partial_pivoting_range():
    """Same range as the partial-pivoting factor of the same block, on an ill-
    conditioned block like the power iteration's (columns nearly aligned)."""
    rng = np.random.default_rng(5)
    base = rng.standard_normal((30_000, 1))
    M = (base + 1e-3 * rng.standard_normal((30_000, 96))) * np.logspace(0, -2, 96)
    M = M.astype(np.float32)
    P_t, _ = _lu_tournament(M)
    P_p, _ = frpca.lu(torch.from_numpy(M).to(DEV))
    assert max_principal_sine(P_t, _cpu(P_p)) < 1e-3


def test_lu_tournament_singular_pivot_reports():
    M = np.random.default_rng(1).standard_normal((500, 20)).astype(np.float32)
    M[:, 11] = 0.0
    with pytest.raises(frpca.FrpcaError) as ei:
        _lu_tournament(M)
    assert ei.value.status == 5


# ---------------------------------------------------------------- SpMM by panels of the gathered block
def _panel_bound(A, X, trans, eps):
    """Each panel's part of a row is summed from zero in CSR order and then
    added to the row once, so a product passes through at most d + 1
    additions plus the fix-up's additions of the 1,024-entry segments of a
    long row within a panel: (d + 4 + d / 512) eps (|A| |X|)."""
    Aabs = synthetic.CSR(A.m, A.n, A.indptr, A.indices, np.abs(A.data.astype(np.float64)))
    f = oracle.spmm_t if trans else oracle.spmm
    mag = f(Aabs.m, Aabs.n, Aabs.indptr, Aabs.indices, Aabs.data, np.abs(X))
    deg = np.diff(A.indptr) if not trans else np.bincount(A.indices, minlength=A.n)
    return (deg[:, None] + 4 + deg[:, None] // 512) * eps * mag + 1e-300


def _wide(A):
    pT, cT, vT = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64))
    return synthetic.CSR(A.n, A.m, pT, cT, vT)


@pytest.mark.parametrize("idx", range(len(MATS)))
@pytest.mark.parametrize("shape", ["tall", "wide"])
@pytest.mark.parametrize("panel_rows", [64, 700])
@pytest.mark.parametrize("l,dtype", [(120, np.float32), (5, np.float32), (48, np.float64)])
def test_spmm_panels_match_oracle(idx, shape, panel_rows, l, dtype):
    """The pass that gathers rows of the larger block (A^T X for a tall A, A X
    for a wide one) run panel by panel: every entry within the summation
    bound of the oracle's product; the other pass and the A^T values are
    unaffected."""
    A = (MATS[idx] if shape == "tall" else _wide(MATS[idx])).astype(dtype)
    mat = frpca.FrPCA.from_csr(A, device=DEV, panel_rows=panel_rows)
    trans = 1 if A.m >= A.n else 0
    rng = np.random.default_rng(l + idx)
    X = rng.standard_normal((A.m if trans else A.n, l)).astype(dtype)
    Xg = frpca.empty_block(X.shape[0], l, torch.float64 if dtype == np.float64 else torch.float32, DEV)
    Xg.copy_(torch.from_numpy(X))
    Y = _cpu(mat.spmm(Xg, trans=bool(trans)))
    f = oracle.spmm_t if trans else oracle.spmm
    ref = f(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), X.astype(np.float64))
    eps = EPS64 if dtype == np.float64 else EPS32
    assert np.all(np.abs(Y - ref) <= _panel_bound(A, X.astype(np.float64), trans, eps))
    assert torch.equal(mat.spmm(Xg, trans=bool(trans)), mat.spmm(Xg, trans=bool(trans)))
    pT, cT, vT = mat.transpose()
    rp, ci, va = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64))
    assert np.array_equal(cT.cpu().numpy(), ci) and np.array_equal(vT.cpu().numpy(), va.astype(dtype))
    mat.close()


def test_spmm_panels_refresh():
    """After the values change in place, frpca_refresh updates the panel form
    (and A^T's own values when they are next read)."""
    A = MATS[1].astype(np.float32)
    vals = torch.tensor(A.data, device=DEV)
    mat = frpca.FrPCA(torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV), vals, (A.m, A.n),
                      panel_rows=1000)
    X = frpca.empty_block(A.m, 64, torch.float32, DEV)
    X.copy_(torch.randn(A.m, 64, generator=torch.Generator().manual_seed(0)))
    Y1 = mat.spmm(X, trans=True).clone()
    with torch.no_grad():
        vals.mul_(2.0)
    mat.refresh()
    Y2 = mat.spmm(X, trans=True).clone()
    assert torch.equal(Y2, 2.0 * Y1)  # scaling by 2 is exact
    _, _, vT = mat.transpose()
    _, _, va = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, 2.0 * A.data.astype(np.float64))
    assert np.array_equal(vT.cpu().numpy(), va.astype(np.float32))
    mat.close()
