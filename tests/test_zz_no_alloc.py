"""frpca_lu_noalloc: the LU entry point for callers that cannot call cudaMalloc
(for example a process whose device memory is already reserved by another
allocator, or a loop that must not take cudaMalloc's device-wide
synchronization).  It keeps its scratch in a static device array instead of
handle-owned buffers.  Through the C ABI this checks that it returns exactly
what frpca_lu returns (and, in FP64, exactly the oracle's P^T L), on two calls
in a row (the shared scratch must be cleared between calls); that the calls
after a warm-up call leave the device's free memory and torch's reserved
memory unchanged; and that oversized requests are refused with the status
frpca_lu gives them.

The file name makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import oracle  # noqa: E402
import paper_1810_06825_gb300 as frpca  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    from paper_1810_06825_gb300 import build
    build.build()
    oracle.build()
    torch.cuda.set_device(0)
    return frpca.library()


def _lu_reference(M):
    """frpca_lu through the C ABI on a handle (handle-owned scratch)."""
    R, l = M.shape
    A = frpca.empty_block(R, l, M.dtype, M.device)
    A.copy_(M)
    piv = torch.empty(l, dtype=torch.int64, device=M.device)
    frpca.frpca_lu(frpca._Context.get(), R, l, A.data_ptr(), A.stride(0), frpca._dtype_code(A), piv.data_ptr())
    return A, piv


def _call_noalloc(lib, A, piv):
    R, l = A.shape
    stream = torch.cuda.current_stream().cuda_stream
    return lib.frpca_lu_noalloc(ctypes.c_int64(R), ctypes.c_int(l), ctypes.c_void_p(A.data_ptr()),
                                ctypes.c_int64(A.stride(0)), ctypes.c_int(frpca._dtype_code(A)),
                                ctypes.c_void_p(piv.data_ptr()), ctypes.c_void_p(stream))


def _lu_noalloc(lib, M):
    R, l = M.shape
    A = frpca.empty_block(R, l, M.dtype, M.device)
    A.copy_(M)
    piv = torch.empty(l, dtype=torch.int64, device=M.device)
    st = _call_noalloc(lib, A, piv)
    assert st == 0, lib.frpca_last_error(None)
    return A, piv


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("R,l", [(5000, 120), (333, 17)])
def test_noalloc_matches_lu_twice(lib, dtype, R, l):
    gen = torch.Generator().manual_seed(R + l)
    M = torch.randn(R, l, generator=gen, dtype=torch.float64).to(dtype).cuda()
    ref, piv_ref = _lu_reference(M)
    for _ in range(2):
        out, piv = _lu_noalloc(lib, M)
        torch.cuda.synchronize()
        assert torch.equal(piv, piv_ref)
        # Same kernel and the same operation order: the tolerance of the LU
        # parity tests (bit-exact) applies.
        assert torch.equal(out, ref)
        if dtype == torch.float64:
            PL, piv_o = oracle.lu_ptl(M.cpu().numpy())
            assert np.array_equal(piv.cpu().numpy(), piv_o)
            assert np.array_equal(out.cpu().numpy(), PL)


def test_noalloc_allocates_nothing(lib):
    """After a warm-up call (which may load the library's device code into the
    context), further calls change neither the free device memory the driver
    reports nor the memory torch's caching allocator holds."""
    gen = torch.Generator().manual_seed(3)
    M = torch.randn(20_000, 120, generator=gen, dtype=torch.float64).cuda()
    A = frpca.empty_block(20_000, 120, torch.float64, "cuda")
    piv = torch.empty(120, dtype=torch.int64, device="cuda")
    A.copy_(M)
    assert _call_noalloc(lib, A, piv) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        A.copy_(M)
        assert _call_noalloc(lib, A, piv) == 0, lib.frpca_last_error(None)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_rejects_oversize(lib):
    M = torch.zeros((8, 200), dtype=torch.float64, device="cuda")
    st = lib.frpca_lu_noalloc(ctypes.c_int64(200), ctypes.c_int(200), ctypes.c_void_p(M.data_ptr()),
                              ctypes.c_int64(200), ctypes.c_int(1), None, None)
    assert st == 9  # FRPCA_ERR_UNSUPPORTED, as frpca_lu returns for l > 160
    assert b"l > 160" in lib.frpca_last_error(None)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    st = lib.frpca_lu_noalloc(ctypes.c_int64(sms * 8192 + 1), ctypes.c_int(4), ctypes.c_void_p(M.data_ptr()),
                              ctypes.c_int64(4), ctypes.c_int(1), None, None)
    assert st == 1
    assert b"8192" in lib.frpca_last_error(None)
