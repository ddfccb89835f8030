"""The precision form FRPCA_PREC_FP32_SPLITGRAM: the Gram matrix of eigSVD
(Alg. 2, step 1) on the tcgen05 tensor cores from split-BF16 operands.

Kernel parity against the oracle's FP64 Gram of the same float block, entry by
entry, within 64 * 2^-24 * (|M|^T |M|)_ij: the three-term split leaves at most
~5 * 2^-27 |x||y| per product (split remainder and the dropped products), FP32
accumulation in tensor memory spans at most 512 rows (32 MMAs of K = 16, each
rounding the running sum once) before the sum moves to double-float, and the
other 32 units cover each MMA's own summation of its 16 products.  End to end, frPCA with the form against the FP64
oracle at the FP32 path's gates (sigma rel. error <= 1e-4, principal-angle sine
<= 1e-3), and the measured errors are printed.
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


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _block(R, l, seed, scale_cols=False, pad_nan=True):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((R, l)).astype(np.float32)
    if scale_cols:
        X *= (10.0 ** rng.uniform(-3, 3, l)).astype(np.float32)
    ld = (l + 31) // 32 * 32
    buf = torch.full((R, ld), float("nan") if pad_nan else 0.0, dtype=torch.float32, device=DEV)
    buf[:, :l] = torch.from_numpy(X).to(DEV)
    return X, buf


@pytest.mark.parametrize("R,l", [(1, 1), (1, 128), (100, 7), (128, 64), (129, 120), (1000, 128), (5000, 33),
                                 (50000, 120), (200001, 120), (77_953, 128), (1_000_000, 120)])
def test_gram_splitbf16_matches_oracle(R, l):
    X, buf = _block(R, l, seed=R + l, scale_cols=(R % 2 == 1))
    B = torch.empty((l, l), dtype=torch.float64, device=DEV)
    frpca.frpca_gram_splitbf16(frpca._Context.get(), R, l, buf.data_ptr(), buf.stride(0), B.data_ptr())
    B = B.cpu().numpy()
    X64 = X.astype(np.float64)
    ref = oracle.gram(X64)
    bound = 64 * 2.0 ** -24 * (np.abs(X64).T @ np.abs(X64))
    assert np.all(np.abs(B - ref) <= bound), np.max(np.abs(B - ref) / bound)
    assert np.array_equal(B, B.T)


def test_gram_splitbf16_deterministic_and_rejects_large_l():
    X, buf = _block(30000, 120, seed=3)
    a = frpca.gram_splitbf16(buf[:, :120])
    b = frpca.gram_splitbf16(buf[:, :120])
    assert torch.equal(a, b)
    big = torch.zeros((300, 160), dtype=torch.float32, device=DEV)
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.gram_splitbf16(big)
    assert ei.value.status == 9


def _run(A, k, l, q, prec):
    mat = frpca.FrPCA.from_csr(A, device=DEV, dtype=np.float32)
    U, S, V = mat.run(k, l, q, seed=0, precision=prec)
    out = tuple(t.double().cpu().numpy() for t in (U, S, V))
    mat.close()
    return out


@pytest.mark.parametrize("shape,q", [((3000, 800), 4), ((3000, 800), 5), ((800, 3000), 5)])
def test_frpca_splitgram_small(shape, q):
    m, n = shape
    A = synthetic.powerlaw_csr(m, n, 20, 1.1, "tfidf", seed=7, dtype=np.float32)
    k, l = 16, 32
    Uo, So, Vo = oracle.frpca(m, n, A.indptr, A.indices, A.data.astype(np.float64), k, l, q, 0)
    U, S, V = _run(A, k, l, q, "fp32_splitgram")
    err = np.max(np.abs(S - So) / So)
    print(f"splitgram {shape} q={q}: sigma rel {err:.2e}, sine U {max_principal_sine(U, Uo):.2e}, "
          f"V {max_principal_sine(V, Vo):.2e}")
    assert err <= 1e-4
    assert max_principal_sine(U, Uo) <= 1e-3 and max_principal_sine(V, Vo) <= 1e-3


@pytest.mark.parametrize("q", [4, 5])
def test_frpca_splitgram_powerlaw_200000x50000(q):
    A = synthetic.make_workload("powerlaw_200000x50000_deg100")
    k, l = 100, 120
    Uo, So, Vo = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), k, l, q, 0,
                              stabilize=True)
    U, S, V = _run(A, k, l, q, "fp32_splitgram")
    _, S32, _ = _run(A, k, l, q, "fp32")
    err = np.max(np.abs(S - So) / So)
    err32 = np.max(np.abs(S32 - So) / So)
    su, sv = max_principal_sine(U, Uo), max_principal_sine(V, Vo)
    print(f"splitgram q={q}: sigma rel {err:.2e} (fp32 path {err32:.2e}), sine U {su:.2e}, V {sv:.2e}")
    assert err <= 1e-4
    assert su <= 1e-3 and sv <= 1e-3


def test_frpca_splitgram_rejects_l_above_128():
    A = synthetic.powerlaw_csr(3000, 800, 20, 1.1, "tfidf", seed=7, dtype=np.float32)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    with pytest.raises(frpca.FrpcaError) as ei:
        mat.run(100, 140, 4, precision="fp32_splitgram")
    assert ei.value.status == 9
    mat.close()
