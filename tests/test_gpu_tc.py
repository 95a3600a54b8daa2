"""The tcgen05 tensor-core GEMMs and the mixed-precision path.

BF16X3: x = x_h + x_l + r with |r| <= 2^-18 |x|; a real product keeps
x_h y_h + x_h y_l + x_l y_h, off by ~2^-16 |x||y|; the tensor-memory FP32
accumulation adds an error that grows with K.  Element-wise,
|C - C_ref| <= 6e-5 (|A| |B|) covers both for the sizes here.

SLICE4 / FP64_SLICE7: values are scaled by a power of two per row of A and
per column of B and cut into s 7-bit integer slices, so the truncation is
<= 2^-7s of the scale and every tensor-core run sums exactly; the error per
element is bounded by (s + 1) 2^-7s K (row max)(column max) plus the
float-float accumulation (~2^-48).  The tests use 1e-6 and 1e-13 of
|A| |B| (Gaussian data: K (row max)(col max) <~ 10 (|A| |B|)).
The FP64 engine is checked at 1e-13.
"""

import numpy as np
import pytest

from oracle import adc2
from synth import make_instance

pytestmark = pytest.mark.gpu

SHAPES = [(64, 32, 64), (130, 70, 200), (257, 300, 1000), (1000, 513, 3000),
          (129, 257, 65)]


@pytest.fixture(scope="module")
def ctx():
    import paper_2604_27451_gb300 as pkg

    c = pkg.Context(0)
    yield c
    c.close()


def _rand(rng, *shape):
    return np.ascontiguousarray(rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


@pytest.mark.parametrize("shape", SHAPES)
def test_zgemm_tc_against_numpy(ctx, shape):
    M, N, K = shape
    rng = np.random.default_rng(M * 7 + N)
    A, B = _rand(rng, M, K), _rand(rng, K, N)
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    C = ctx.zgemm(A, B, "bf16x3")
    err = np.abs(C - ref) / bound
    assert err.max() < 6e-5, err.max()
    # the split keeps far more than bf16 alone: typical error ~1e-6
    assert np.median(err) < 5e-6
    C64 = ctx.zgemm(A, B, "fp64")
    assert (np.abs(C64 - ref) / bound).max() < 1e-13


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec,tol", [("slice4", 1e-6), ("fp64_slice7", 1e-13)])
def test_zgemm_slices_against_numpy(ctx, shape, prec, tol):
    M, N, K = shape
    rng = np.random.default_rng(M * 5 + N + K)
    A, B = _rand(rng, M, K), _rand(rng, K, N)
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    C = ctx.zgemm(A, B, prec)
    err = np.abs(C - ref) / bound
    assert err.max() < tol, err.max()


@pytest.mark.parametrize("shape", [(1300, 1, 2000), (2000, 3, 5000), (5000, 8, 700)])
def test_fp64_few_columns_against_numpy(ctx, shape):
    # N <= 8 with A's rows contiguous: the FP64 engine's warp-per-row path
    M, N, K = shape
    rng = np.random.default_rng(M + N + K)
    A, B = _rand(rng, M, K), _rand(rng, K, N)
    ref = A @ B
    bound = np.abs(A) @ np.abs(B)
    assert (np.abs(ctx.zgemm(A, B, "fp64") - ref) / bound).max() < 1e-13


def test_slice_accumulation_does_not_grow_with_k(ctx):
    # positive data: every partial sum has the sign of the total, so any
    # rounding in the accumulation shows up in full
    rng = np.random.default_rng(2)
    for K in (512, 8192):
        A = np.ascontiguousarray(rng.random((256, K)) + 0j)
        B = np.ascontiguousarray(rng.random((K, 256)) + 0j)
        ref = A @ B
        e4 = (np.abs(ctx.zgemm(A, B, "slice4") - ref) / np.abs(ref)).max()
        e7 = (np.abs(ctx.zgemm(A, B, "fp64_slice7") - ref) / np.abs(ref)).max()
        assert e4 < 2e-8, (K, e4)
        # 49 bits of slices plus the FP32 low word of the float-float sum
        # (~n_runs 2^-48, a few hundred runs here)
        assert e7 < 5e-12, (K, e7)


def test_zgemm_tc_repeatable(ctx):
    rng = np.random.default_rng(3)
    A, B = _rand(rng, 300, 200), _rand(rng, 200, 260)
    for prec in ("bf16x3", "slice4"):
        C1 = ctx.zgemm(A, B, prec)
        C2 = ctx.zgemm(A, B, prec)
        assert np.array_equal(C1, C2)


MIX = dict(ncore=4, nval=10, nvirt=50, naux=150, seed=4)


@pytest.fixture(scope="module")
def mixed_problem():
    import paper_2604_27451_gb300 as pkg

    c = MIX
    inst = make_instance(c["ncore"], c["nval"], c["nvirt"], c["naux"], seed=c["seed"])
    ctx64 = pkg.Context(0)
    ctx64.prepare(inst.eps, inst.B, inst.dip, inst.ncore, inst.nval, inst.nvirt)
    yield inst, ctx64
    ctx64.close()


def test_sigma_mixed_close_to_fp64(mixed_problem):
    inst, ctx = mixed_problem
    N = ctx.shape["N"]
    rng = np.random.default_rng(9)
    x = _rand(rng, 2, N)
    s64 = ctx.sigma(x, "fp64")
    s16 = ctx.sigma(x, "bf16x3")
    rel = np.abs(s16 - s64).max() / np.abs(s64).max()
    assert rel < 2e-4, rel
    sig = adc2.Sigma(inst.eps, inst.B, inst.ncore, inst.nval, inst.nvirt)
    r1, r2 = sig(x[0, :ctx.shape["N1"]], x[0, ctx.shape["N1"]:])
    ref = np.concatenate([r1, r2])
    assert np.abs(s64[0] - ref).max() / np.abs(ref).max() < 1e-11


def test_mixed_prepare_m11_close(mixed_problem):
    import paper_2604_27451_gb300 as pkg

    inst, ctx64 = mixed_problem
    m64 = ctx64.get_m11()
    c = pkg.Context(0)
    c.prepare(inst.eps, inst.B, inst.dip, inst.ncore, inst.nval, inst.nvirt,
              precision="bf16x3")
    m16 = c.get_m11()
    assert np.abs(m16 - m64).max() / np.abs(m64).max() < 2e-4
    t64, e64 = ctx64.get_t2()
    t16, e16 = c.get_t2()
    assert abs(e16 - e64) < 1e-4 * abs(e64)
    c.close()


def test_slice_sigma_and_prepare(mixed_problem):
    import paper_2604_27451_gb300 as pkg

    inst, ctx64 = mixed_problem
    N = ctx64.shape["N"]
    rng = np.random.default_rng(19)
    x = _rand(rng, 2, N)
    s64 = ctx64.sigma(x, "fp64")
    for prec, tol in (("slice4", 1e-7), ("fp64_slice7", 1e-13)):
        s = ctx64.sigma(x, prec)
        assert np.abs(s - s64).max() / np.abs(s64).max() < tol, prec
        c = pkg.Context(0)
        c.prepare(inst.eps, inst.B, inst.dip, inst.ncore, inst.nval, inst.nvirt,
                  precision=prec)
        m = c.get_m11()
        m64 = ctx64.get_m11()
        assert np.abs(m - m64).max() / np.abs(m64).max() < tol, prec
        c.close()


@pytest.mark.parametrize("prec,tol", [("slice4", 1e-5), ("fp64_slice7", 1e-9)])
def test_slice_solve_matches_oracle(prec, tol):
    import paper_2604_27451_gb300 as pkg

    c = MIX
    inst = make_instance(c["ncore"], c["nval"], c["nvirt"], c["naux"], seed=c["seed"])
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    M11 = adc2.m11(inst.eps, inst.B, nc, nw, nv)
    M21 = adc2.m21(inst.eps, inst.B, nc, nw, nv)
    d22 = adc2.m22(inst.eps, nc, nw, nv)
    w_ref, _ = adc2.eig_partitioned(M11, M21, d22, 3)
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, 3, precision=prec,
                    conv=1e-7)
    assert np.abs(out["omega"] - w_ref).max() < tol
    ctx.close()


def test_mixed_solve_refined_matches_oracle():
    import paper_2604_27451_gb300 as pkg

    c = MIX
    inst = make_instance(c["ncore"], c["nval"], c["nvirt"], c["naux"], seed=c["seed"])
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    M11 = adc2.m11(inst.eps, inst.B, nc, nw, nv)
    M21 = adc2.m21(inst.eps, inst.B, nc, nw, nv)
    d22 = adc2.m22(inst.eps, nc, nw, nv)
    w_ref, X_ref = adc2.eig_partitioned(M11, M21, d22, 3)
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, 3, precision="bf16x3",
                    conv=1e-7, refine_sweeps=6)
    # BF16X3 carries ~1e-5 relative GEMM error (accumulation-limited) in the
    # Davidson sigma only: the problem is built with the FP64-class product,
    # so the FP64-class correction sweeps converge to the right matrix's
    # roots
    assert np.abs(out["omega"] - w_ref).max() < 1e-5
    ctx.close()
