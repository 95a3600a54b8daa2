"""The allocation-free small-output GEMM, cvsadc_zgemm_small_noalloc.

For callers that must not let the library allocate device memory (their
memory is owned by another allocator, or cudaMalloc's synchronisation is
not acceptable).  Through the C ABI it must give what the allocating entry
point cvsadc_zgemm (FP64) gives, and what a complex128 product on the CPU
gives, within the FP64 tolerance of the other GEMM tests (1e-13 of
|A||B|), on two calls in a row with different inputs -- the second call
would expose state left in the shared scratch array.  The long-K shape
takes the small-output kernel with as many K slices as the fixed array
holds.
This file is collected last so that a failure here leaves every other test
already run; it also passes alone in a fresh process.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

SHAPES = [(6, 300, 20000), (40, 100, 5000), (17, 13, 70001), (64, 64, 300),
          (64, 64, 300000)]


def _call(lib, stream, A, B, C):
    M, K = A.shape
    N = B.shape[1]
    return lib.cvsadc_zgemm_small_noalloc(
        ctypes.c_void_p(stream), M, N, K, ctypes.c_void_p(A.data_ptr()), K,
        ctypes.c_void_p(B.data_ptr()), N, ctypes.c_void_p(C.data_ptr()), N)


@pytest.mark.parametrize("shape", SHAPES)
def test_noalloc_matches_allocating_entry_point(shape):
    import torch

    import paper_2604_27451_gb300 as pkg
    from paper_2604_27451_gb300 import _lib

    lib = _lib.load()
    M, N, K = shape
    stream = torch.cuda.current_stream().cuda_stream
    ctx = pkg.Context(0)
    g = torch.Generator(device="cuda").manual_seed(M + N + K)
    for call in range(2):
        A = torch.randn(M, K, dtype=torch.complex128, device="cuda", generator=g)
        B = torch.randn(K, N, dtype=torch.complex128, device="cuda", generator=g)
        C = torch.full((M, N), complex(np.nan, np.nan), dtype=torch.complex128,
                       device="cuda")
        assert _call(lib, stream, A, B, C) == 0
        ref = ctx.zgemm(A, B, "fp64")
        cpu = A.cpu().numpy() @ B.cpu().numpy()
        bound = (A.abs() @ B.abs()).cpu().numpy()
        Cn = C.cpu().numpy()
        for want in (ref.cpu().numpy(), cpu):
            err = np.abs(Cn - want) / bound
            assert np.isfinite(err).all()
            assert err.max() < 1e-13, (call, err.max())
    ctx.close()


def test_noalloc_rejects_sizes_beyond_the_limit():
    import torch

    from paper_2604_27451_gb300 import _lib

    lib = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    A = torch.zeros(65, 8, dtype=torch.complex128, device="cuda")
    B = torch.zeros(8, 64, dtype=torch.complex128, device="cuda")
    C = torch.zeros(65, 64, dtype=torch.complex128, device="cuda")
    assert _call(lib, stream, A, B, C) == -1  # 65 * 64 > 4096
    A2 = torch.zeros(2, 8, dtype=torch.complex128, device="cuda")
    B2 = torch.zeros(8, 383, dtype=torch.complex128, device="cuda")
    C2 = torch.zeros(2, 383, dtype=torch.complex128, device="cuda")
    assert _call(lib, stream, A2, B2, C2) == -1  # M + N > 384
    assert lib.cvsadc_zgemm_small_noalloc(None, 2, 2, 2, None, 2, None, 2, None, 2) == -1
