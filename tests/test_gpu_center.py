"""Implicit centering on the GPU: PCA proper (Sec. 2.1 assumes centered data)
of A - 1 mu^T, mu the column means, without forming it (every product gets
its rank-1 correction).  Against the oracle's centered method on the same
Gaussian test matrix, at the usual gates (sigma rel. 1e-10 / 1e-4 for FP64 /
FP32, principal-angle sines 1e-8 / 1e-3), for Alg. 6 and Alg. 5 and with the
panel form; and the property the centering guarantees: the left singular
vectors are orthogonal to the all-ones vector."""
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


def _check(A, prec, k, l, q, seed, mat, stol=None, atol=None):
    Uo, So, Vo = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), k, l, q, seed, center=True)
    U, S, V = (t.double().cpu().numpy() for t in mat.run(k, l, q, seed=seed, precision=prec, center=True))
    st, at = (1e-10, 1e-8) if prec == "fp64" else (1e-4, 1e-3)
    es = float(np.max(np.abs(S - So) / So))
    eu, ev = max_principal_sine(U, Uo), max_principal_sine(V, Vo)
    print(f"centered {prec} {A.m}x{A.n} q={q}: sigma {es:.2e}, sine U {eu:.2e}, V {ev:.2e}")
    assert es <= (stol or st) and eu <= (atol or at) and ev <= (atol or at)
    ones = np.ones(A.m) / np.sqrt(A.m)
    assert np.max(np.abs(ones @ U)) <= (1e-8 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("shape", ["tall", "wide"])
@pytest.mark.parametrize("panel_rows", [0, 250])
def test_centered_matches_oracle(prec, shape, panel_rows):
    A = TALL if shape == "tall" else _wide(TALL)
    A = A.astype(np.float64 if prec == "fp64" else np.float32)
    mat = frpca.FrPCA.from_csr(A, device=DEV, panel_rows=panel_rows)
    for q in (2, 3, 4, 5):
        _check(A, prec, 10, 24, q, 7, mat)
    mat.close()


def test_centered_refresh_recomputes_means():
    """After the values change in place, the column means follow."""
    A = TALL.astype(np.float32)
    vals = torch.tensor(A.data, device=DEV)
    mat = frpca.FrPCA(torch.tensor(A.indptr, device=DEV), torch.tensor(A.indices, device=DEV), vals, (A.m, A.n))
    _check(A, "fp32", 10, 24, 5, 3, mat)
    with torch.no_grad():
        vals.copy_(torch.tensor(np.sqrt(A.data), device=DEV))
    mat.refresh()
    B = synthetic.CSR(A.m, A.n, A.indptr, A.indices, np.sqrt(A.data))
    _check(B, "fp32", 10, 24, 5, 3, mat)
    mat.close()


def test_centered_powerlaw_200000x50000():
    A = synthetic.make_workload("powerlaw_200000x50000_deg100")
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    _check(A, "fp32", 100, 120, 5, 0, mat)
    mat.close()
