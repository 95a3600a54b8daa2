"""The Davidson solver's inner products (cvsadc_block_dot) against the CPU.

The FP64-class precisions use plain FP64 FMAs; the mixed precisions use
double-float on the FP32 pipes (float hi/lo pairs, 16-term tiles summed in
FP64).  Each input is split once into hi + lo with |x - hi - lo| <=
2^-48 |x|, and a product keeps the exact rounding error of hi*hi plus the
two cross terms, so one product is off by <= ~2^-46 |a||b|; the tile sums
and the sum over tiles run in FP64 exactly as in the FP64 arithmetic.
Element-wise both are checked to 1e-13 of sum |a||b| on a block of 2^26
complex elements (the size of a Davidson vector of the medium workload x4),
against numpy's complex128 vdot.

The float exponent range bounds the double-float path: products below
~1e-38 flush to zero.  A block scaled by 1e-15 (products ~1e-30) keeps its
accuracy; FP64 keeps it at 1e-30 (products ~1e-60), which the double-float
path cannot represent -- that path only sees the mixed phases' normalised
vectors and their corrections.
"""

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _block(g, m, n, torch):
    re = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)
    im = torch.randn(m, n, dtype=torch.float64, device="cuda", generator=g)
    return torch.complex(re, im).contiguous()


def _check(ctx, A, B, prec, tol):
    got = ctx.block_dot(A, B, prec)
    An, Bn = A.cpu().numpy(), B.cpu().numpy()
    ref = np.array([[np.vdot(a, b) for b in Bn] for a in An])
    bound = np.abs(An) @ np.abs(Bn).T
    err = np.abs(got - ref) / bound
    assert np.isfinite(err).all()
    assert err.max() < tol, (prec, err.max())


@pytest.mark.parametrize("prec", ["fp64", "fp64_slice7", "slice4"])
def test_block_dot_large_block(prec):
    import torch

    import paper_2604_27451_gb300 as pkg

    ctx = pkg.Context(0)
    g = torch.Generator(device="cuda").manual_seed(5)
    N = 1 << 26
    A = _block(g, 3, N, torch)
    B = _block(g, 2, N, torch)
    _check(ctx, A, B, prec, 1e-13)
    _check(ctx, A, A, prec, 1e-13)
    ctx.close()


@pytest.mark.parametrize("prec,scale", [("fp64", 1e-30), ("slice4", 1e-15)])
def test_block_dot_small_magnitudes(prec, scale):
    import torch

    import paper_2604_27451_gb300 as pkg

    ctx = pkg.Context(0)
    g = torch.Generator(device="cuda").manual_seed(6)
    N = 100003
    A = _block(g, 4, N, torch) * scale
    B = _block(g, 3, N, torch) * scale
    _check(ctx, A, B, prec, 1e-13)
    ctx.close()
