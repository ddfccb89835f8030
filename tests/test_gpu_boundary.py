"""The C-ABI boundary around frpca_create / frpca_run (the problem statement of
Alg. 5/6: A in R^{m x n} in CSR, k, l = k + s, q passes), exercised on the GPU:

- host arrays (on_device = 0): the library copies the CSR to the device and
  validates it there; the result matches the FP64 oracle like the device path;
- int32 row pointers (rowptr_type = FRPCA_I32), from host and device arrays;
- an invalid CSR given as host arrays is refused with FRPCA_ERR_INVALID_CSR;
- a cap on the handle's own device memory (max_device_bytes) makes an
  allocation fail with FRPCA_ERR_OOM, at create or at run;
- a bounded device-side wait given a very short limit runs out: the LU and
  eigensolver grid barriers return FRPCA_ERR_TIMEOUT, and the same handle then
  serves normal calls whose results match the oracle.
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
A64 = synthetic.powerlaw_csr(3000, 800, 12, 1.1, "tfidf", seed=1, dtype=np.float64)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)


def _cpu(t):
    return t.detach().double().cpu().numpy()


def _check_against_oracle(mat, A, prec, k=10, l=24, q=5, seed=7):
    Uo, So, Vo = oracle.frpca(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64), k, l, q, seed)
    U, S, V = (_cpu(t) for t in mat.run(k, l, q, seed=seed, precision=prec))
    stol, atol = (1e-10, 1e-8) if prec == "fp64" else (1e-4, 1e-3)
    assert np.max(np.abs(S - So) / So) <= stol
    assert max_principal_sine(U, Uo) <= atol
    assert max_principal_sine(V, Vo) <= atol


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("rowptr", ["i64", "i32"])
def test_create_from_host_arrays(prec, rowptr):
    A = A64 if prec == "fp64" else A64.astype(np.float32)
    ip = A.indptr if rowptr == "i64" else A.indptr.astype(np.int32)
    mat = frpca.FrPCA.from_host(ip, A.indices, A.data, (A.m, A.n), device=DEV)
    pT, cT, vT = mat.transpose()
    rp, ci, va = oracle.csr_transpose(A.m, A.n, A.indptr, A.indices, A.data.astype(np.float64))
    assert np.array_equal(pT.cpu().numpy(), rp) and np.array_equal(cT.cpu().numpy(), ci)
    assert np.array_equal(vT.cpu().numpy(), va.astype(A.data.dtype))
    _check_against_oracle(mat, A, prec)
    mat.close()


def test_create_from_pinned_host_tensors():
    A = A64.astype(np.float32)
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    mat = frpca.FrPCA.from_host(pin(A.indptr), pin(A.indices), pin(A.data), (A.m, A.n), device=DEV)
    _check_against_oracle(mat, A, "fp32")
    mat.close()


@pytest.mark.parametrize("borrow", [True, False])
def test_int32_rowptr_on_device(borrow):
    A = A64.astype(np.float32)
    mat = frpca.FrPCA(torch.from_numpy(A.indptr.astype(np.int32)).to(DEV), torch.from_numpy(A.indices).to(DEV),
                      torch.from_numpy(A.data).to(DEV), (A.m, A.n), borrow=borrow)
    _check_against_oracle(mat, A, "fp32")
    mat.close()


def test_host_invalid_csr_rejected():
    A = synthetic.uniform_csr(50, 40, 300, seed=3)
    bad = A.indices.copy()
    s = A.indptr[7]
    bad[s], bad[s + 1] = bad[s + 1], bad[s]  # unsorted row
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.FrPCA.from_host(A.indptr, bad, A.data, (A.m, A.n), device=DEV)
    assert ei.value.status == 2
    ip = A.indptr.copy()
    ip[-1] -= 1  # rowptr[m] != nnz
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.FrPCA.from_host(ip, A.indices, A.data, (A.m, A.n), device=DEV)
    assert ei.value.status == 2
    ip = A.indptr.astype(np.int32)
    ip[10], ip[11] = ip[11], ip[10]  # non-monotone
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.FrPCA.from_host(ip, A.indices, A.data, (A.m, A.n), device=DEV)
    assert ei.value.status == 2


def test_device_memory_cap_reports_oom():
    A = A64.astype(np.float32)
    # Too small for the handle's own status word and copies: create fails.
    with pytest.raises(frpca.FrpcaError) as ei:
        frpca.FrPCA.from_host(A.indptr, A.indices, A.data, (A.m, A.n), device=DEV, max_device_bytes=4096)
    assert ei.value.status == 3
    # Enough to create (copies, A^T, plans) but not for the run's blocks.
    mat = frpca.FrPCA.from_host(A.indptr, A.indices, A.data, (A.m, A.n), device=DEV, max_device_bytes=2_000_000)
    with pytest.raises(frpca.FrpcaError) as ei:
        mat.run(10, 24, 5, seed=7, precision="fp32")
    assert ei.value.status == 3
    mat.close()
    # Without the cap the same matrix runs.
    mat = frpca.FrPCA.from_host(A.indptr, A.indices, A.data, (A.m, A.n), device=DEV)
    _check_against_oracle(mat, A, "fp32")
    mat.close()


def test_bounded_waits_time_out_then_recover():
    """The grid-wide barriers of the LU kernels and of the eigensolver's
    refinement, given a one-cycle limit, run out (every block that arrives
    before the last one gives up and leaves the kernel); each call returns
    TIMEOUT and the handle then serves normal calls."""
    h = frpca._Context.get()
    rng = np.random.default_rng(11)
    M64 = rng.standard_normal((50_000, 120))
    Mg = torch.from_numpy(M64).to(DEV)
    Mf = torch.from_numpy(M64.astype(np.float32)).to(DEV)
    X = rng.standard_normal((360, 120))
    B = torch.from_numpy(X.T @ X).to(DEV)
    try:
        frpca.frpca_set_wait_limit(h, 1)
        for call in (lambda: frpca.lu(Mg), lambda: frpca.lu(Mf), lambda: frpca.eig(B)):
            with pytest.raises(frpca.FrpcaError) as ei:
                call()
            assert ei.value.status == 7
        A = frpca.empty_block(50_000, 120, torch.float32, DEV)
        A.copy_(Mf)
        piv = torch.empty(120, dtype=torch.int64, device=DEV)
        with pytest.raises(frpca.FrpcaError) as ei:
            frpca.frpca_lu_tournament(h, 50_000, 120, A.data_ptr(), A.stride(0), piv.data_ptr())
        assert ei.value.status == 7
    finally:
        frpca.frpca_set_wait_limit(h, 0)
    PL, piv = frpca.lu(Mg)
    ref, piv_ref = oracle.lu_ptl(M64)
    assert np.array_equal(piv.cpu().numpy(), piv_ref) and np.array_equal(_cpu(PL), ref)
    w, V = frpca.eig(B)
    wr, _ = oracle.eig_sym(X.T @ X)
    assert np.max(np.abs(_cpu(w) - wr)) <= 64 * np.finfo(np.float64).eps * np.linalg.norm(X.T @ X, 2)
    # A handle whose run timed out serves the next run.
    mat = frpca.FrPCA.from_csr(A64.astype(np.float32), device=DEV)
    mat.set_wait_limit(1)
    with pytest.raises(frpca.FrpcaError) as ei:
        mat.run(10, 24, 5, seed=7, precision="fp32")
    assert ei.value.status == 7
    mat.set_wait_limit(0)
    _check_against_oracle(mat, A64.astype(np.float32), "fp32")
    mat.close()


def test_trim_memory_returns_the_pool():
    """A destroyed handle's memory stays mapped in the library's pool for the
    next handle; frpca_trim_memory gives it back to the device."""
    A = synthetic.powerlaw_csr(200_000, 50_000, 20, 1.1, "tfidf", seed=2, dtype=np.float32)
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    mat.run(10, 24, 3, seed=1, precision="fp32")
    mat.close()
    torch.cuda.synchronize()
    free_kept, _ = torch.cuda.mem_get_info()
    frpca.frpca_trim_memory()
    free_trimmed, _ = torch.cuda.mem_get_info()
    assert free_trimmed > free_kept
    # A handle created after the trim works as before.
    mat = frpca.FrPCA.from_csr(A, device=DEV)
    U, S, V = mat.run(10, 24, 3, seed=1, precision="fp32")
    assert torch.all(S > 0)
    mat.close()
