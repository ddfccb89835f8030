"""Pins for the FP64 CPU oracle, each against something other than the oracle.

Philox against numpy's independent Philox4x64 implementation; the sparse
kernels against scipy and dense numpy; LU against LAPACK getrf (through scipy)
and Lemma 3; Jacobi against LAPACK syevd; eigSVD against LAPACK gesdd
(Lemma 1); the whole method against closed-form spectra, the QR scheme of
Alg. 1 / Alg. 4 (Theorems 1 and 2) and exact identities.
"""
import numpy as np
import pytest
import scipy.linalg
import scipy.sparse as sp
import scipy.stats

import synthetic
from tests.helpers import block_rank_csr, dense_svd_topk, max_principal_sine, rel_err

pytestmark = pytest.mark.usefixtures("oracle_lib")


def _np_philox_block(seed, b, stream=0):
    """Block b of the generator, taken from numpy's Philox (which increments
    its 256-bit counter before emitting), so counter b-1 yields block b."""
    prev = (b - 1) % (1 << 256)
    ctr = np.array([(prev >> (64 * i)) & ((1 << 64) - 1) for i in range(4)], dtype=np.uint64)
    bg = np.random.Philox(key=np.array([seed, stream], dtype=np.uint64), counter=ctr)
    return bg.random_raw(4)


# ----------------------------------------------------------------- Philox / randn
@pytest.mark.parametrize("seed", [0, 1, 7, 2**63 + 12345, 2**64 - 1])
@pytest.mark.parametrize("block", [0, 1, 2, 3, 1000, 2**33 + 5])
def test_philox_matches_numpy(oracle_lib, seed, block):
    ours = oracle_lib.philox4x64([block, 0, 0, 0], [seed, 0])
    assert np.array_equal(ours, _np_philox_block(seed, block))


def test_gaussian_layout_from_numpy_words(oracle_lib):
    """Element e uses word e%4 of block e//4; Box-Muller on word pairs."""
    R, l, seed = 7, 5, 3
    G = oracle_lib.gaussian(R, l, seed).ravel()
    for e in range(R * l):
        w = _np_philox_block(seed, e // 4)
        u = ((w >> np.uint64(12)).astype(np.float64) + 0.5) * 2.0 ** -52
        pair = (e % 4) // 2
        r = np.sqrt(-2.0 * np.log(u[2 * pair]))
        ang = 2.0 * np.pi * u[2 * pair + 1]
        ref = r * (np.cos(ang) if e % 2 == 0 else np.sin(ang))
        assert abs(G[e] - ref) <= 1e-14 * max(1.0, abs(ref))


def test_gaussian_distribution(oracle_lib):
    G = oracle_lib.gaussian(50_000, 4, 11).ravel()
    assert abs(G.mean()) < 5 * (1 / np.sqrt(G.size))
    assert abs(G.var() - 1.0) < 5 * np.sqrt(2.0 / G.size)
    assert scipy.stats.kstest(G, "norm").pvalue > 1e-3
    # Box-Muller partners are independent N(0,1): correlation ~ 0.
    pairs = G.reshape(-1, 2)
    assert abs(np.corrcoef(pairs[:, 0], pairs[:, 1])[0, 1]) < 5 / np.sqrt(pairs.shape[0])


def test_gaussian_seeds_differ_and_repeat(oracle_lib):
    a = oracle_lib.gaussian(10, 3, 5)
    assert np.array_equal(a, oracle_lib.gaussian(10, 3, 5))
    assert not np.allclose(a, oracle_lib.gaussian(10, 3, 6))
    # A longer matrix starts with the same numbers (counter-based, layout flat).
    b = oracle_lib.gaussian(20, 3, 5)
    assert np.array_equal(a.ravel(), b.ravel()[:30])


# ----------------------------------------------------------------- CSR transpose
def _random_csr(m, n, density, seed, empty_rows=True):
    rng = np.random.default_rng(seed)
    A = sp.random(m, n, density=density, random_state=rng, format="csr", dtype=np.float64)
    if empty_rows and m > 3:
        A = A.tolil()
        A[1, :] = 0
        A[m - 1, :] = 0
        A = A.tocsr()
    A.sort_indices()
    A.eliminate_zeros()
    return synthetic.CSR(m, n, A.indptr.astype(np.int64), A.indices.astype(np.int32), A.data)


@pytest.mark.parametrize("m,n,density", [(1, 1, 1.0), (5, 9, 0.3), (40, 17, 0.2), (300, 257, 0.02), (17, 400, 0.05)])
def test_csr_transpose_matches_scipy(oracle_lib, m, n, density):
    A = _random_csr(m, n, density, seed=m * 31 + n)
    pT, cT, vT = oracle_lib.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data)
    ref = sp.csr_matrix((A.data, A.indices, A.indptr), shape=(m, n)).T.tocsr()
    ref.sort_indices()
    assert np.array_equal(pT, ref.indptr)
    assert np.array_equal(cT, ref.indices)
    assert np.array_equal(vT, ref.data)
    back = synthetic.CSR(n, m, pT, cT, vT).to_dense()
    assert np.array_equal(back, A.to_dense().T)


def test_csr_transpose_powerlaw(oracle_lib):
    A = synthetic.powerlaw_csr(3000, 500, 20, 1.1, "tfidf", seed=3, dtype=np.float64)
    pT, cT, vT = oracle_lib.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data)
    ref = sp.csr_matrix((A.data, A.indices, A.indptr), shape=(A.m, A.n)).T.tocsr()
    ref.sort_indices()
    assert np.array_equal(pT, ref.indptr) and np.array_equal(cT, ref.indices) and np.array_equal(vT, ref.data)


# ----------------------------------------------------------------- SpMM
@pytest.mark.parametrize("m,n,l", [(1, 1, 1), (40, 17, 5), (300, 257, 20), (64, 500, 33)])
def test_spmm_against_dense(oracle_lib, m, n, l):
    A = _random_csr(m, n, 0.1, seed=m + n + l)
    Ad = A.to_dense()
    rng = np.random.default_rng(l)
    X = rng.standard_normal((n, l))
    Y = oracle_lib.spmm(m, n, A.indptr, A.indices, A.data, X)
    assert np.allclose(Y, Ad @ X, rtol=1e-13, atol=1e-13)
    Z = rng.standard_normal((m, l))
    W = oracle_lib.spmm_t(m, n, A.indptr, A.indices, A.data, Z)
    assert np.allclose(W, Ad.T @ Z, rtol=1e-13, atol=1e-13)


# ----------------------------------------------------------------- LU
@pytest.mark.parametrize("R,l", [(1, 1), (7, 7), (50, 8), (400, 33), (1000, 20)])
def test_lu_matches_lapack(oracle_lib, R, l):
    rng = np.random.default_rng(R * 7 + l)
    M = rng.standard_normal((R, l))
    PL, piv = oracle_lib.lu_ptl(M)
    ref = scipy.linalg.lu(M, permute_l=True)[0]
    assert np.allclose(PL, ref, rtol=1e-12, atol=1e-12)
    assert np.max(np.abs(PL)) <= 1.0 + 1e-15
    # Pivot rows carry the unit diagonal and zeros to their right.
    for j, p in enumerate(piv):
        assert PL[p, j] == 1.0 and np.all(PL[p, j + 1:] == 0.0)
    assert len(set(piv.tolist())) == l
    # Lemma 3: range(P^T L) = range(M).
    assert max_principal_sine(PL, M) < 1e-12


def test_lu_tie_takes_smallest_row(oracle_lib):
    M = np.array([[1.0, 0.0], [-2.0, 1.0], [2.0, 5.0], [0.5, 3.0]])
    _, piv = oracle_lib.lu_ptl(M)
    assert piv[0] == 1


def test_lu_zero_column_is_singular(oracle_lib):
    import oracle
    M = np.random.default_rng(0).standard_normal((20, 4))
    M[:, 2] = 0.0
    with pytest.raises(oracle.OracleError) as ei:
        oracle_lib.lu_ptl(M)
    assert ei.value.status == oracle.ERR_SINGULAR_PIVOT


# ----------------------------------------------------------------- eig / eigSVD
@pytest.mark.parametrize("n", [1, 2, 5, 20, 64, 121])
def test_eig_matches_lapack(oracle_lib, n):
    rng = np.random.default_rng(n)
    X = rng.standard_normal((n, n))
    B = X + X.T
    w, V = oracle_lib.eig_sym(B)
    wr, Vr = np.linalg.eigh(B)
    scale = max(1.0, np.abs(wr).max())
    assert np.all(np.diff(w) >= 0)
    assert np.max(np.abs(w - wr)) <= 1e-13 * scale
    assert np.allclose(V.T @ V, np.eye(n), atol=1e-13)
    assert np.max(np.abs(B @ V - V * w)) <= 1e-12 * scale
    # Eigenvectors agree with LAPACK's up to sign (spectrum is simple here).
    dots = np.abs(np.sum(V * Vr, axis=0))
    assert np.all(dots > 1 - 1e-9)


def test_eig_repeated_eigenvalues(oracle_lib):
    Q, _ = np.linalg.qr(np.random.default_rng(1).standard_normal((10, 10)))
    d = np.array([1, 1, 1, 2, 3, 3, 4, 5, 5, 5], dtype=float)
    B = (Q * d) @ Q.T
    w, V = oracle_lib.eig_sym(B)
    assert np.allclose(w, d, atol=1e-13)
    assert np.allclose(V.T @ V, np.eye(10), atol=1e-13)
    assert np.allclose(B @ V, V * w, atol=1e-12)


@pytest.mark.parametrize("R,l,cond", [(30, 5, 10.0), (500, 40, 1e3), (2000, 120, 1e2)])
def test_eigsvd_lemma1(oracle_lib, R, l, cond):
    rng = np.random.default_rng(R + l)
    Uq, _ = np.linalg.qr(rng.standard_normal((R, l)))
    Vq, _ = np.linalg.qr(rng.standard_normal((l, l)))
    s = np.geomspace(1.0, 1.0 / cond, l)
    M = (Uq * s) @ Vq.T
    U, S, V = oracle_lib.eigsvd(M)
    Ur, Sr, Vrt = np.linalg.svd(M, full_matrices=False)
    assert np.all(np.diff(S) >= 0)                        # ascending, Sec. 3.1
    assert rel_err(S[::-1], Sr) <= 1e-12 * cond
    assert np.allclose(U.T @ U, np.eye(l), atol=1e-12 * cond ** 2)
    assert np.allclose((U * S) @ V.T, M, atol=1e-12 * cond)
    assert np.allclose(oracle_lib.gram(M), M.T @ M, rtol=1e-13, atol=1e-13)


def test_eigsvd_rank_deficient(oracle_lib):
    import oracle
    M = np.random.default_rng(2).standard_normal((50, 6))
    M[:, 5] = M[:, 0] + M[:, 1]
    with pytest.raises(oracle.OracleError) as ei:
        oracle_lib.eigsvd(M)
    assert ei.value.status == oracle.ERR_RANK_DEFICIENT


# ----------------------------------------------------------------- the method
@pytest.mark.parametrize("q", [2, 3, 4, 5, 6])
@pytest.mark.parametrize("tall", [True, False])
@pytest.mark.parametrize("alg", [None, 5, 6])
def test_frpca_exact_rank_closed_form(oracle_lib, q, tall, alg):
    """Pin 1: rank(A) = l, so range(A Omega) = range(A) and any q is exact,
    for the shape rule's algorithm and for either one forced (Table 3 runs
    both on each shape)."""
    l, k = 10, 6
    m, n = (140, 90) if tall else (90, 140)
    A, sig, Ut, Vt = block_rank_csr(m, n, l, seed=q)
    U, S, V = oracle_lib.frpca(m, n, A.indptr, A.indices, A.data, k, l, q, seed=0, alg=alg)
    # eigSVD squares the condition number (Sec. 3.1), so rounding reaches
    # eps * kappa(M)^2 ~ 1e-12 when a power step squares the spread of sigma.
    # Off the shape rule the power step's block lives on the longer side and
    # its A^T A Omega carries kappa ~ (sigma_1 / sigma_l)^2 ~ 5e2, so eps *
    # kappa^2 ~ 6e-11 moves the subspaces by a few 1e-10.
    tol = 1e-10 if alg is None else 2e-9
    assert rel_err(S, sig[:k]) <= 1e-10
    assert max_principal_sine(U, Ut[:, :k]) <= tol
    assert max_principal_sine(V, Vt[:, :k]) <= tol


@pytest.mark.parametrize("alg_tall", [True, False])
def test_frpca_planted_spectrum(oracle_lib, alg_tall):
    """Pin 2: sigma_i = 0.5^i planted in a dense-stored CSR; q = 9 resolves the
    top k to rounding since (sigma_{l+1}/sigma_k)^(q-1) ~ 1e-15."""
    rng = np.random.default_rng(5)
    m, n = (60, 40) if alg_tall else (40, 60)
    r = min(m, n)
    Uq, _ = np.linalg.qr(rng.standard_normal((m, r)))
    Vq, _ = np.linalg.qr(rng.standard_normal((n, r)))
    sig = 0.5 ** np.arange(r)
    Ad = (Uq * sig) @ Vq.T
    A = synthetic.from_dense(Ad, keep_zeros=True)
    k, l = 5, 10
    U, S, V = oracle_lib.frpca(m, n, A.indptr, A.indices, A.data, k, l, 9, seed=1)
    assert rel_err(S, sig[:k]) <= 1e-10
    for j in range(k):
        assert abs(abs(U[:, j] @ Uq[:, j]) - 1) < 1e-10
        assert abs(abs(V[:, j] @ Vq[:, j]) - 1) < 1e-10


def _theorem_case(tall):
    A = synthetic.powerlaw_csr(400, 250, 12, 1.1, "tfidf", seed=9, dtype=np.float64)
    if not tall:
        import oracle
        pT, cT, vT = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data)
        A = synthetic.CSR(A.n, A.m, pT, cT, vT)
    return A


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("tall", [True, False])
@pytest.mark.parametrize("stabilize", [False, True])
def test_frpca_equals_qr_scheme(oracle_lib, q, tall, stabilize):
    """Pin 3: Theorem 2 (Alg. 6 vs Alg. 4) and Theorem 1 (Alg. 5 vs Alg. 1) with
    p = (q-2)/2 on the same Omega; odd q against the modified power iteration.
    The stabilized schedule (an extra lu() before the last eigSVD, Lemma 3)
    must give the same result."""
    from oracle import qr_scheme
    A = _theorem_case(tall)
    k, l = 8, 14
    U, S, V = oracle_lib.frpca(A.m, A.n, A.indptr, A.indices, A.data, k, l, q, seed=4, stabilize=stabilize)
    base = qr_scheme.rpca_t if tall else qr_scheme.rpca
    if q % 2 == 0:
        Ur, Sr, Vr = base(A.m, A.n, A.indptr, A.indices, A.data, k, l, (q - 2) // 2, seed=4)
    else:
        Ur, Sr, Vr = base(A.m, A.n, A.indptr, A.indices, A.data, k, l, (q - 1) // 2, seed=4, modified=True)
    assert rel_err(S, Sr) <= 1e-10
    assert max_principal_sine(U, Ur) <= 1e-8
    assert max_principal_sine(V, Vr) <= 1e-8


@pytest.mark.parametrize("q", [3, 4])
@pytest.mark.parametrize("tall", [True, False])
def test_frpca_identities(oracle_lib, q, tall):
    """Pin 4: A V = U diag(S) (Alg. 6) or A^T U = V diag(S) (Alg. 5); U, V
    orthonormal; S descending; ||A - U S V^T||_F^2 = ||A||_F^2 - sum S^2; signs."""
    A = _theorem_case(tall)
    Ad = A.to_dense()
    k, l = 8, 14
    U, S, V = oracle_lib.frpca(A.m, A.n, A.indptr, A.indices, A.data, k, l, q, seed=2)
    if tall:
        assert np.allclose(Ad @ V, U * S, atol=1e-12 * S[0])
    else:
        assert np.allclose(Ad.T @ U, V * S, atol=1e-12 * S[0])
    assert np.allclose(U.T @ U, np.eye(k), atol=1e-11)
    assert np.allclose(V.T @ V, np.eye(k), atol=1e-11)
    assert np.all(np.diff(S) <= 0)
    res = np.linalg.norm(Ad - (U * S) @ V.T) ** 2
    assert abs(res - (np.linalg.norm(Ad) ** 2 - np.sum(S ** 2))) <= 1e-10 * np.linalg.norm(Ad) ** 2
    X = V if A.m >= A.n else U
    idx = np.argmax(np.abs(X), axis=0)
    assert np.all(X[idx, np.arange(k)] > 0)
    # Eq. 3 style: the rank-k residual is within a few percent of optimal.
    opt = np.sum(np.linalg.svd(Ad, compute_uv=False)[k:] ** 2)
    assert res <= 1.1 * opt


def test_frpca_more_passes_more_accurate(oracle_lib):
    """Eq. 9 direction: q = 5 (odd scheme) is at least as accurate as q = 4."""
    A = _theorem_case(True)
    Ad = A.to_dense()
    k, l = 8, 10
    _, Sr, _ = dense_svd_topk(Ad, k)
    errs = []
    for q in (2, 3, 4, 5, 7):
        _, S, _ = oracle_lib.frpca(A.m, A.n, A.indptr, A.indices, A.data, k, l, q, seed=3)
        errs.append(rel_err(S, Sr))
    assert errs[-1] <= errs[0]
    assert errs[3] <= errs[2] * 1.5 + 1e-14


def test_frpca_uniform_2000x1000(oracle_lib):
    """Pin 5 (brute force): the uniform 2,000 x 1,000 workload against dense
    LAPACK.  Its spectrum is flat below sigma_1, so at q = 3 the estimates are
    rough (printed, not gated).  Gated: Ritz values of A on range(Q) never
    exceed the true ones (interlacing), and sigma_1 converges as q grows, at the
    rate the power iteration gives it."""
    w = synthetic.WORKLOADS["uniform_2000x1000_nnz20000"]
    A = synthetic.make_workload("uniform_2000x1000_nnz20000")
    Sr = np.linalg.svd(A.to_dense(), compute_uv=False)[: w["k"]]
    errs = {}
    for q in (w["q"], 9, 25):
        _, S, _ = oracle_lib.frpca(A.m, A.n, A.indptr, A.indices, A.data, w["k"], w["l"], q, seed=0)
        assert np.all(S <= Sr * (1 + 1e-12))
        errs[q] = np.abs(S - Sr) / Sr
    print("uniform 2000x1000 q=3 sigma rel err:", errs[w["q"]])
    assert errs[9][0] < 1e-3 and errs[25][0] < 1e-10
    assert np.all(errs[25] <= errs[w["q"]])


@pytest.mark.parametrize("k,l,q", [(0, 5, 3), (6, 5, 3), (3, 5, 1), (3, 500, 3)])
def test_frpca_invalid_args(oracle_lib, k, l, q):
    import oracle
    A = _theorem_case(True)
    with pytest.raises(oracle.OracleError) as ei:
        oracle_lib.frpca(A.m, A.n, A.indptr, A.indices, A.data, k, l, q, seed=0)
    assert ei.value.status == oracle.ERR_INVALID_ARG


# ----------------------------------------------------------------- implicit centering
@pytest.mark.parametrize("q", [2, 3, 4, 5])
@pytest.mark.parametrize("tall", [True, False])
def test_frpca_centered_equals_explicit_centering(oracle_lib, q, tall):
    """The centered method (rank-1 corrections of every product) equals the
    plain method run on the centered matrix A - 1 mu^T stored as a dense CSR
    (every entry kept): the same algorithm on the same matrix and Omega, so
    the results agree to rounding."""
    A = synthetic.powerlaw_csr(300, 120, 8, 1.1, "tfidf", seed=11, dtype=np.float64)
    if not tall:
        pT, cT, vT = oracle_lib.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data)
        A = synthetic.CSR(A.n, A.m, pT, cT, vT)
    Ad = A.to_dense()
    Ac = Ad - Ad.mean(axis=0, keepdims=True)
    D = synthetic.from_dense(Ac, keep_zeros=True)
    k, l = 6, 12
    U, S, V = oracle_lib.frpca(A.m, A.n, A.indptr, A.indices, A.data, k, l, q, seed=2, center=True)
    Ue, Se, Ve = oracle_lib.frpca(D.m, D.n, D.indptr, D.indices, D.data, k, l, q, seed=2)
    assert rel_err(S, Se) <= 1e-10
    assert max_principal_sine(U, Ue) <= 1e-8 and max_principal_sine(V, Ve) <= 1e-8
    # Centered columns: U is orthogonal to the all-ones vector (Abar^T 1 = 0,
    # and U spans part of range(Abar)).
    assert np.max(np.abs(U.sum(axis=0))) <= 1e-8 * np.sqrt(A.m)


def test_frpca_centered_closed_form(oracle_lib):
    """A matrix whose centered version has rank exactly l: a rank-l matrix plus
    a constant row added to every row (the offset the centering removes),
    both sparse patterns stored in full.  Any q returns the exact top-k SVD
    of the centered matrix."""
    rng = np.random.default_rng(3)
    m, n, r, k = 200, 80, 8, 5
    B = (rng.standard_normal((m, r)) * 0.8 ** np.arange(r)) @ rng.standard_normal((r, n))
    B -= B.mean(axis=0, keepdims=True)
    Ad = B + rng.standard_normal(n)[None, :]
    A = synthetic.from_dense(Ad, keep_zeros=True)
    Ut, St, Vt = np.linalg.svd(B, full_matrices=False)
    for q in (2, 3, 4):
        U, S, V = oracle_lib.frpca(m, n, A.indptr, A.indices, A.data, k, r, q, seed=1, center=True)
        assert rel_err(S, St[:k]) <= 1e-10
        assert max_principal_sine(U, Ut[:, :k]) <= 1e-9 and max_principal_sine(V, Vt[:k].T) <= 1e-9
