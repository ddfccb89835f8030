"""End-to-end GPU frPCA (Alg. 5 / Alg. 6) against the FP64 CPU oracle on the same
Philox Gaussian test matrix.

Gates: singular values rel. error <= 1e-10 (FP64 path) / 1e-4 (FP32 path);
largest principal-angle sine between GPU and oracle U_k and V_k subspaces <=
1e-8 (FP64) / 1e-3 (FP32); the sign convention agrees wherever it is decided
by a clear margin.
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

DEV = "cuda:0"
TOL = {"fp64": (1e-10, 1e-8), "fp32": (1e-4, 1e-3)}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cpu(t):
    return t.detach().double().cpu().numpy()


def _compare(A, k, l, q, seed, prec, alg=None, mat=None, stabilize=False, angle_tol=None):
    Uo, So, Vo = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), k, l, q, seed, alg=alg,
                              stabilize=stabilize)
    own = mat is None
    if own:
        mat = frpca.FrPCA.from_csr(A, device=DEV)
    U, S, V = mat.run(k, l, q, seed=seed, precision=prec, alg=alg or 0)
    U, S, V = _cpu(U), _cpu(S), _cpu(V)
    if own:
        mat.close()
    stol, atol = TOL[prec]
    atol = angle_tol or atol
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(S - So) / So) <= stol, np.max(np.abs(S - So) / So)
    assert max_principal_sine(U, Uo) <= atol
    assert max_principal_sine(V, Vo) <= atol
    # Sign convention: the min(m, n)-length factor's largest entry is positive.
    X, Xo = (V, Vo) if A.m >= A.n else (U, Uo)
    srt = np.sort(np.abs(Xo), axis=0)
    clear = (srt[-1] - srt[-2]) > 1e-3 * srt[-1]
    gaps = np.abs(np.diff(So))
    sep = np.ones(k, dtype=bool)
    sep[:-1] &= gaps > 1e-3 * So[0]
    sep[1:] &= gaps > 1e-3 * So[0]
    cos = np.sum(X * Xo, axis=0)
    assert np.all(cos[clear & sep] > 0)
    return S, So


SMALL_TALL = synthetic.powerlaw_csr(3000, 800, 12, 1.1, "tfidf", seed=1, dtype=np.float64)


def _transposed(A):
    pT, cT, vT = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data)
    return synthetic.CSR(A.n, A.m, pT, cT, vT)


SMALL_WIDE = _transposed(SMALL_TALL)


@pytest.mark.parametrize("q", [2, 3, 4, 5, 6, 7])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["tall", "wide"])
def test_frpca_small(q, prec, shape):
    A = SMALL_TALL if shape == "tall" else SMALL_WIDE
    _compare(A.astype(np.float64 if prec == "fp64" else np.float32), 10, 24, q, 7, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["tall", "wide"])
def test_frpca_panels(prec, shape):
    """The whole method with the larger block's pass run by panels (250 rows
    each, so a dozen panels at this size)."""
    A = SMALL_TALL if shape == "tall" else SMALL_WIDE
    A = A.astype(np.float64 if prec == "fp64" else np.float32)
    mat = frpca.FrPCA.from_csr(A, device=DEV, panel_rows=250, fused_sweep=1)
    for q in (3, 4, 5):
        _compare(A, 10, 24, q, 7, prec, mat=mat)
    mat.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["tall", "wide"])
def test_fused_sweep_matches_two_passes(prec, shape):
    """Alg. 6's loop body M = A^T (A Q) (Alg. 5: A (A^T Q)) as one sweep: panel b of A Q is made into an L2-resident slot and gathered from
    there at once.  Every row is formed by the same kernel in the same order
    as in the two-pass form, so U, S and V agree bit for bit."""
    A = SMALL_TALL if shape == "tall" else SMALL_WIDE
    A = A.astype(np.float64 if prec == "fp64" else np.float32)
    m1 = frpca.FrPCA.from_csr(A, device=DEV, panel_rows=250, fused_sweep=1)
    m2 = frpca.FrPCA.from_csr(A, device=DEV, panel_rows=250)
    for q in (3, 5, 6):
        m1.reset_stats()
        r1 = [t.clone() for t in m1.run(10, 24, q, seed=5, precision=prec)]
        r2 = [t.clone() for t in m2.run(10, 24, q, seed=5, precision=prec)]
        for a, b in zip(r1, r2):
            assert torch.equal(a, b)
        assert m1.stats()["fused_sweeps"] == (q - 1) // 2
    m1.close()
    m2.close()


@pytest.mark.parametrize("shape", ["tall", "wide"])
@pytest.mark.parametrize("fused", [0, 1])
def test_refresh_then_run_matches_new_handle(shape, fused):
    """After the values change in place and frpca_refresh, a run reads the
    new values in every pass: A^T's own values are refreshed for the passes
    that read them (the producing pass of a wide matrix's fused sweep, the
    A^T pass without panels) and may be left stale by the others.  The same
    kernels run on the same data, so U, S and V equal a new handle's bit for
    bit."""
    A = (SMALL_TALL if shape == "tall" else SMALL_WIDE).astype(np.float32)
    vals = torch.tensor(A.data, device=DEV)
    m1 = frpca.FrPCA(torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV), vals, (A.m, A.n),
                     panel_rows=250, fused_sweep=fused)
    m1.run(10, 24, 5, seed=3, precision="fp32")
    with torch.no_grad():
        vals.mul_(torch.linspace(0.5, 2.0, vals.numel(), device=DEV))
    m1.refresh()
    r1 = [t.clone() for t in m1.run(10, 24, 5, seed=3, precision="fp32")]
    m2 = frpca.FrPCA(torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV), vals.clone(),
                     (A.m, A.n), panel_rows=250, fused_sweep=fused)
    r2 = [t.clone() for t in m2.run(10, 24, 5, seed=3, precision="fp32")]
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    m1.close()
    m2.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_frpca_uniform_2000x1000(prec):
    """The uniform 2,000 x 1,000 workload, k = 10, l = 20, 3 passes, seed 0."""
    w = synthetic.WORKLOADS["uniform_2000x1000_nnz20000"]
    A = synthetic.make_workload("uniform_2000x1000_nnz20000")
    _compare(A if prec == "fp64" else A.astype(np.float32), w["k"], w["l"], w["q"], 0, prec)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["tall", "wide"])
@pytest.mark.parametrize("alg", [5, 6])
def test_frpca_forced_alg_either_shape(prec, shape, alg):
    """Table 3 runs Alg. 5 and Alg. 6 on tall and on wide matrices: either
    algorithm, forced on either shape, matches the oracle's same algorithm
    (and the sign convention follows the shorter factor whatever the
    algorithm)."""
    A = SMALL_TALL if shape == "tall" else SMALL_WIDE
    A = A.astype(np.float64 if prec == "fp64" else np.float32)
    for q in (4, 5):
        _compare(A, 10, 24, q, 7, prec, alg=alg)


def test_frpca_square_alg5_forced():
    """m == n with Alg. 5 forced: the sign is decided on V, the apply side."""
    A = synthetic.powerlaw_csr(900, 900, 10, 1.1, "tfidf", seed=4, dtype=np.float64)
    _compare(A, 6, 12, 4, 3, "fp64", alg=5)
    _compare(A, 6, 12, 4, 3, "fp64", alg=6)


def test_frpca_exact_rank():
    """rank(A) = l exactly: every q returns the exact top-k SVD (closed form).
    Block scales decay as 0.85^b, so that the power step's eigSVD input stays
    within double precision's reach (a faster decay makes kappa(M)^2 exceed
    1e13 at q = 3, where no FP64 evaluation of eigSVD holds 1e-10)."""
    from tests.helpers import block_rank_csr
    A, sig, _, _ = block_rank_csr(600, 300, 16, seed=3, scales=0.85 ** np.arange(16))
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    for q in (2, 3, 4):
        U, S, V = mat.run(10, 16, q, seed=1, precision="fp64")
        assert np.max(np.abs(_cpu(S) - sig[:10]) / sig[:10]) <= 1e-10
    mat.close()


def test_frpca_deterministic():
    A = SMALL_TALL.astype(np.float32)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    r1 = [t.clone() for t in mat.run(10, 24, 5, seed=3)]
    r2 = [t.clone() for t in mat.run(10, 24, 5, seed=3)]
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    mat.close()


def test_frpca_invalid_args():
    mat = frpca.FrPCA.from_csr(SMALL_TALL, device=DEV)
    for k, l, q in [(0, 5, 3), (6, 5, 3), (3, 5, 1), (3, 900, 3)]:
        with pytest.raises(frpca.FrpcaError) as ei:
            mat.run(k, l, q, precision="fp64")
        assert ei.value.status == 1
    with pytest.raises(frpca.FrpcaError) as ei:
        mat.run(3, 5, 3, alg=7)  # only Alg. 5 and Alg. 6 exist
    assert ei.value.status == 1
    mat.close()


def test_frpca_rank_deficient_reports():
    """Fewer than l nonzero rows: range(A Q) has dimension < l and eigSVD refuses it."""
    A = synthetic.from_dense(np.vstack([np.random.default_rng(0).standard_normal((5, 40)), np.zeros((95, 40))]))
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    with pytest.raises(frpca.FrpcaError) as ei:
        mat.run(4, 8, 3, precision="fp64")
    assert ei.value.status in (5, 6)
    mat.close()


# -------------------------------------------------------------- full-size workload
@pytest.fixture(scope="module")
def powerlaw_200k():
    return synthetic.make_workload("powerlaw_200000x50000_deg100")


@pytest.mark.parametrize("q", [4, 5])
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_frpca_powerlaw_200000x50000(powerlaw_200k, q, prec):
    """The 200,000 x 50,000 (~20M nnz) power-law workload, k=100, l=120, FP32
    and FP64 paths, against the FP64 oracle on the same Gaussian test matrix.

    Here the last power-iteration block A^T A Q has condition number 6e3-1e4,
    so the oracle's plain FP64 eigSVD returns a basis orthonormal only to
    eps * kappa^2 ~ 1e-8, which moves its singular values by up to ~5e-10.
    The FP64 path is therefore held to 1e-10 against the oracle's stabilized
    schedule (lu() before that eigSVD; Lemma 3, identical in exact
    arithmetic) and to 1e-8 against the plain one.  sigma_100 and sigma_101
    are only ~1e-3 apart in relative terms, so the top-100 subspaces are
    compared at 1e-6 in FP64 (rounding-level perturbations over that gap)."""
    A = powerlaw_200k if prec == "fp32" else powerlaw_200k.astype(np.float64)
    if prec == "fp64":
        S, So = _compare(A, 100, 120, q, 0, prec, stabilize=True, angle_tol=1e-6)
        _, So_plain, _ = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data, 100, 120, q, 0)
        dev = np.max(np.abs(S - So_plain) / So_plain)
        print(f"fp64 q={q} vs plain-schedule oracle {dev:.3e}")
        assert dev <= 1e-8
    else:
        S, So = _compare(A, 100, 120, q, 0, prec)
    print(f"{prec} q={q} max sigma rel err {np.max(np.abs(S - So) / So):.3e}")


def test_precision_form_powerlaw_1000000x200000():
    """The precision-form workload: 1,000,000 x 200,000, ~100M nnz, k=100,
    l=120, q=5.  FP32 SpMM with the split-BF16 tensor-core Gram
    (FP32_SPLITGRAM) and the plain FP64 GPU path, both against the FP64
    oracle (stabilized schedule) on the same Gaussian test matrix: singular
    values in full, V in full and U on a seeded 10% row subsample (each
    restricted basis re-orthonormalized).  Gates: the FP32 path's 1e-4 on
    sigma and 1e-3 on the principal-angle sines for the precision form; the
    FP64 path's 1e-10 on sigma and 1e-5 on the sines (sigma_100 and sigma_101
    are close, so the FP64 subspaces carry rounding over that gap)."""
    A = synthetic.make_workload("powerlaw_1000000x200000_deg100")
    k, l, q = 100, 120, 5
    Uo, So, Vo = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), k, l, q, 0,
                              stabilize=True)
    rows = np.sort(np.random.default_rng(10).choice(A.m, size=A.m // 10, replace=False))
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    for prec, stol, atol in (("fp32_splitgram", 1e-4, 1e-3), ("fp64", 1e-10, 1e-5)):
        U, S, V = (_cpu(t) for t in mat.run(k, l, q, seed=0, precision=prec))
        es = np.max(np.abs(S - So) / So)
        eu = max_principal_sine(U[rows], Uo[rows])
        ev = max_principal_sine(V, Vo)
        print(f"{prec}: sigma rel {es:.2e}, sine U (10% rows) {eu:.2e}, sine V {ev:.2e}")
        assert es <= stol and eu <= atol and ev <= atol
    mat.close()
