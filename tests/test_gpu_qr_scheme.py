"""The basic randomized PCA with QR (Alg. 1 / Alg. 4, orth() after every
product, here CholeskyQR2 on the GPU) that frPCA is compared with in
Theorems 1-2 and Table 2:

- against the oracle's QR scheme (numpy Householder QR and LAPACK SVD on the
  oracle's products, the same Gaussian test matrix): sigma within 1e-10 /
  1e-4 relative (FP64 / FP32) and principal-angle sines within 1e-8 / 1e-3;
- Theorems 1-2 on the GPU: the QR scheme and frPCA with the same passes give
  the same singular values and subspaces (to rounding in FP64)."""
import numpy as np
import pytest

import synthetic
from tests.helpers import max_principal_sine

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
from oracle import qr_scheme  # noqa: E402
import paper_1810_06825_gb300 as frpca  # noqa: E402

DEV = "cuda:0"
TALL = synthetic.powerlaw_csr(3000, 800, 12, 1.1, "tfidf", seed=1, dtype=np.float64)


def _wide(A):
    pT, cT, vT = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data)
    return synthetic.CSR(A.n, A.m, pT, cT, vT)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cpu(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["tall", "wide"])
@pytest.mark.parametrize("q", [2, 3, 4, 5, 6])
def test_qr_scheme_matches_oracle(prec, shape, q):
    A = TALL if shape == "tall" else _wide(TALL)
    A = A.astype(np.float64 if prec == "fp64" else np.float32)
    k, l, seed = 10, 24, 7
    p, modified = ((q - 2) // 2, False) if q % 2 == 0 else ((q - 1) // 2, True)
    f = qr_scheme.rpca_t if A.m >= A.n else qr_scheme.rpca
    Uo, So, Vo = f(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), k, l, p, seed, modified=modified)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    U, S, V = (_cpu(t) for t in mat.run(k, l, q, seed=seed, precision=prec, scheme="qr"))
    st, at = (1e-10, 1e-8) if prec == "fp64" else (1e-4, 1e-3)
    assert np.all(np.diff(S) <= 0)
    assert np.max(np.abs(S - So) / So) <= st
    assert max_principal_sine(U, Uo) <= at and max_principal_sine(V, Vo) <= at
    assert mat.stats()["qr_calls"] >= (1 if q % 2 == 0 else 0)
    mat.close()


@pytest.mark.parametrize("shape", ["tall", "wide"])
@pytest.mark.parametrize("q", [2, 4, 5, 6])
def test_qr_scheme_equals_frpca(shape, q):
    """Theorem 2 (Alg. 6 vs Alg. 4) and Theorem 1 (Alg. 5 vs Alg. 1), both
    schemes run by the library in FP64 on the same Omega."""
    A = TALL if shape == "tall" else _wide(TALL)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    U1, S1, V1 = (_cpu(t) for t in mat.run(10, 24, q, seed=3, precision="fp64"))
    U2, S2, V2 = (_cpu(t) for t in mat.run(10, 24, q, seed=3, precision="fp64", scheme="qr"))
    assert np.max(np.abs(S1 - S2) / S2) <= 1e-10
    assert max_principal_sine(U1, U2) <= 1e-8 and max_principal_sine(V1, V2) <= 1e-8
    mat.close()
