"""The code paths the bench takes, element by element.

* K-chunked slice GEMM: once the packed operands of a product exceed the
  packing budget (3 GB), the exact-slice GEMM runs over K in chunks and
  every chunk after the first accumulates with beta = 1.  A product with
  five chunks is compared with the FP64 engine at the slice bounds of
  tests/test_gpu_tc.py (SLICE4 1e-6, FP64_SLICE7 1e-13 of |A||B|).
* The medium workload (6/60/300/1500) sigma on an 8-vector block: its S and
  G products chunk over K, and the packed slices of the static B^P operand
  come from the context's cache on the second call.  Both calls must agree
  bit for bit, and the doubles part of sigma for sampled valence spinors j
  -- (M21 x1)[:, j] + M22 x2, which the oracle builds one spinor at a time
  from explicit <ab||cj> -- must match the oracle (FP64 1e-11, SLICE4 1e-7
  of the largest entry).
* The medium workload's FP64-class eigenpairs (FP64_SLICE7, 8 roots): on
  the sampled spinors the doubles rows of M x - w x, built by the oracle,
  stay below the converged residual.
* Row slabs: a tall product whose packed A would force K into chunks of a
  few blocks runs as slabs of rows with K whole; compared with the FP64
  engine and cuBLAS at the slice bounds.
* M12 against M21 (Eq. 8: M12 = M21^H): for v = (x1, 0) the sigma gives
  (M11 x1, M21 x1); for w = (0, M21 x1) its singles part is M12 M21 x1, so
  x1^H (M12 M21 x1) = ||M21 x1||^2 exactly.  This pins the singles part of
  sigma (the S and sigma1^T products) at any size; at the medium and the
  large workload (the bench's 4-vector block, SLICE4) with the doubles
  rows of M21 x1 sampled against the oracle and M11 x1 against the
  prepared M11.
"""

import numpy as np
import pytest

from oracle import adc2
from synth import WORKLOADS, make_instance

pytestmark = pytest.mark.gpu

J_SAMPLE = (0, 29, 59)


@pytest.fixture(scope="module")
def medium():
    w = WORKLOADS["medium"]
    inst = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=0)
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    N1 = nc * nv
    sig = adc2.Sigma(inst.eps, inst.B, nc, nw, nv, M11=np.zeros((N1, N1), complex),
                     cache_blocks=True)
    return inst, sig


def _oracle_s2_rows(inst, sig, x, j):
    """(M x)[doubles of valence spinor j] as [ncore][pair] from the oracle
    ((M21 x1)[:, j] from the oracle's coupling block, plus M22 x2)."""
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    N1 = nc * nv
    X = x[:N1].reshape(nc, nv)
    pl = adc2.pair_list(nv)
    npair = len(pl)
    x2 = x[N1:].reshape(nc, nw, npair)
    # the doubles of spinor j unpacked; the block reads only that slice
    Yj = np.zeros((nc, nv, nv), dtype=np.complex128)
    Yj[:, pl[:, 0], pl[:, 1]] = x2[:, j]
    Yj[:, pl[:, 1], pl[:, 0]] = -x2[:, j]
    Y = np.lib.stride_tricks.as_strided(
        Yj, shape=(nc, nw, nv, nv), strides=(Yj.strides[0], 0) + Yj.strides[1:])
    s2j, _ = sig.coupling_block(X, Y, j)
    d22 = sig.d22.reshape(nc, nw, npair)
    return s2j[:, pl[:, 0], pl[:, 1]] + d22[:, j] * x2[:, j]


def _gpu_s2_rows(inst, s, j):
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    N1 = nc * nv
    npair = nv * (nv - 1) // 2
    return s[N1:].reshape(nc, nw, npair)[:, j]


@pytest.mark.parametrize("prec,tol", [("slice4", 1e-6), ("fp64_slice7", 1e-13)])
def test_k_chunked_slice_gemm(prec, tol):
    import torch

    import paper_2604_27451_gb300 as pkg

    M, N, K = 8192, 4096, 20000  # packed slices ~13 GB (4) / ~37 GB (7): chunked over K
    ctx = pkg.Context(0)
    g = torch.Generator(device="cuda").manual_seed(17)
    A = torch.complex(torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g))
    B = torch.complex(torch.randn(K, N, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(K, N, dtype=torch.float64, device="cuda", generator=g))
    C = ctx.zgemm(A, B, prec)
    R = ctx.zgemm(A, B, "fp64")
    bound = A.abs() @ B.abs()
    err = ((C - R).abs() / bound).max().item()
    assert err < tol, err
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("slice4", 1e-7)])
def test_medium_sigma_cached_and_sampled_rows(medium, prec, tol):
    import torch

    import paper_2604_27451_gb300 as pkg

    inst, sig = medium
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    ctx = pkg.Context(0)
    ctx.prepare(torch.tensor(inst.eps, device="cuda"), torch.tensor(inst.B, device="cuda"),
                None, nc, nw, nv, precision=prec)
    N = ctx.shape["N"]
    nvec = 8 if prec != "fp64" else 2
    g = torch.Generator(device="cuda").manual_seed(23)
    X = torch.complex(torch.randn(nvec, N, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(nvec, N, dtype=torch.float64, device="cuda", generator=g))
    S1 = ctx.sigma(X, prec).cpu().numpy()
    S2 = ctx.sigma(X, prec).cpu().numpy()  # packed B^P slices from the cache
    assert np.array_equal(S1, S2)
    Xh = X.cpu().numpy()
    for q in (0, nvec - 1):
        for j in J_SAMPLE:
            ref = _oracle_s2_rows(inst, sig, Xh[q], j)
            got = _gpu_s2_rows(inst, S1[q], j)
            assert np.abs(got - ref).max() < tol * np.abs(ref).max(), (q, j)
    ctx.close()


def test_medium_eigenpairs_sampled_residual(medium):
    import paper_2604_27451_gb300 as pkg

    inst, sig = medium
    w = WORKLOADS["medium"]
    nc, nw, nv, k = inst.ncore, inst.nval, inst.nvirt, w["nroots"]
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, None, nc, nw, nv, k, precision="fp64_slice7",
                    conv=1e-6, return_x=True)
    assert out["status"] == 0
    assert out["info"]["max_residual"] <= 1e-6
    X = out["X"]
    for q in range(k):
        assert abs(np.linalg.norm(X[q]) - 1.0) < 1e-10
        for j in J_SAMPLE:
            r = _oracle_s2_rows(inst, sig, X[q], j) - out["omega"][q] * _gpu_s2_rows(inst, X[q], j)
            assert np.linalg.norm(r) <= 1.5e-6, (q, j, np.linalg.norm(r))
    ctx.close()


@pytest.mark.parametrize("prec,tol", [("slice4", 1e-6), ("fp64_slice7", 1e-13)])
def test_row_slab_slice_gemm(prec, tol):
    import torch

    import paper_2604_27451_gb300 as pkg

    M, N, K = 400000, 4, 1000  # K would run in chunks of <= 448: slabs of rows instead
    ctx = pkg.Context(0)
    g = torch.Generator(device="cuda").manual_seed(29)
    A = torch.complex(torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(M, K, dtype=torch.float64, device="cuda", generator=g))
    B = torch.complex(torch.randn(K, N, dtype=torch.float64, device="cuda", generator=g),
                      torch.randn(K, N, dtype=torch.float64, device="cuda", generator=g))
    C = ctx.zgemm(A, B, prec)
    R = A @ B  # cuBLAS ZGEMM
    bound = A.abs() @ B.abs()
    assert ((C - R).abs() / bound).max().item() < tol
    # the FP64 engine's few-column path (a warp per row of A)
    C64 = ctx.zgemm(A, B, "fp64")
    assert ((C64 - R).abs() / bound).max().item() < 1e-13
    ctx.close()


def _adjoint_check(ctx, prec, N1, X1, tol):
    """x1^H (M12 M21 x1) = ||M21 x1||^2 for each row of X1; returns the
    sigma of (x1, 0)."""
    import torch

    nvec = X1.shape[0]
    N = ctx.shape["N"]
    V = torch.zeros(nvec, N, dtype=torch.complex128, device="cuda")
    V[:, :N1] = X1
    SV = ctx.sigma(V, prec)
    W = torch.zeros_like(V)
    W[:, N1:] = SV[:, N1:]
    SW = ctx.sigma(W, prec)
    lhs = (X1.conj() * SW[:, :N1]).sum(dim=1)
    rhs = (SV[:, N1:].abs() ** 2).sum(dim=1)
    err = ((lhs - rhs).abs() / rhs).max().item()
    assert err < tol, err
    return SV


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-12), ("slice4", 1e-6)])
def test_medium_sigma_singles_part_is_adjoint(medium, prec, tol):
    import torch

    import paper_2604_27451_gb300 as pkg

    inst, _ = medium
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    N1 = nc * nv
    ctx = pkg.Context(0)
    ctx.prepare(torch.tensor(inst.eps, device="cuda"), torch.tensor(inst.B, device="cuda"),
                None, nc, nw, nv, precision=prec)
    g = torch.Generator(device="cuda").manual_seed(31)
    X1 = torch.complex(torch.randn(4, N1, dtype=torch.float64, device="cuda", generator=g),
                       torch.randn(4, N1, dtype=torch.float64, device="cuda", generator=g))
    SV = _adjoint_check(ctx, prec, N1, X1, tol)
    M11 = torch.tensor(ctx.get_m11(), device="cuda")
    ref = X1 @ M11.T
    assert (SV[:, :N1] - ref).abs().max().item() < 1e-12 * ref.abs().max().item()
    ctx.close()


def test_large_sigma_block_sampled_rows_and_adjoint():
    """The bench's workload and launch configuration: SLICE4 sigma of a
    4-vector block on the large workload (12/120/600/3000)."""
    import torch

    import paper_2604_27451_gb300 as pkg

    w = WORKLOADS["large"]
    inst = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=0)
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    N1 = nc * nv
    npair = nv * (nv - 1) // 2
    sig = adc2.Sigma(inst.eps, inst.B, nc, nw, nv, M11=np.zeros((N1, N1), complex),
                     cache_blocks=False)
    ctx = pkg.Context(0)
    ctx.prepare(torch.tensor(inst.eps, device="cuda"), torch.tensor(inst.B, device="cuda"),
                None, nc, nw, nv, precision="slice4")
    g = torch.Generator(device="cuda").manual_seed(37)
    X1 = torch.complex(torch.randn(4, N1, dtype=torch.float64, device="cuda", generator=g),
                       torch.randn(4, N1, dtype=torch.float64, device="cuda", generator=g))
    SV = _adjoint_check(ctx, "slice4", N1, X1, 1e-6)
    M11 = torch.tensor(ctx.get_m11(), device="cuda")
    ref = X1 @ M11.T
    assert (SV[:, :N1] - ref).abs().max().item() < 1e-12 * ref.abs().max().item()
    # doubles rows a in {0, 1} of (M21 x1)[:, j] from the oracle (x2 = 0)
    zero = np.zeros(1, dtype=np.complex128)
    Y0 = np.lib.stride_tricks.as_strided(zero, shape=(nc, nw, nv, nv), strides=(0, 0, 0, 0))
    Xh = X1.cpu().numpy()
    S2 = SV[:, N1:].reshape(4, nc, nw, npair)
    for q in (0, 3):
        for j in (0, nw - 1):
            s2j, _ = sig.coupling_block(Xh[q].reshape(nc, nv), Y0, j, slice(0, 2))
            got = S2[q, :, j, :2 * nv - 3].cpu().numpy()
            ref = np.concatenate([s2j[:, 0, 1:], s2j[:, 1, 2:]], axis=1)
            assert np.abs(got - ref).max() < 1e-7 * np.abs(ref).max(), (q, j)
    ctx.close()
