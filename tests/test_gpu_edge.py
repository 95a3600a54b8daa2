"""GPU edge cases: the smallest partitions the method allows, every root
of a problem, an empty batch and a root count beyond the space — each
against the oracle's exact answer or the documented error — and the error
path of the bounded device waits."""

import numpy as np
import pytest

from oracle import solve as osolve
from synth import make_instance

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(1, 1, 2, 1), (1, 2, 3, 2), (2, 2, 3, 4)])
def test_all_roots_of_tiny_problems(shape):
    """N = ncore nvirt + ncore nval nvirt (nvirt - 1) / 2 roots: the whole
    spectrum (nvirt = 2 leaves one virtual pair)."""
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L = shape
    N = nc * nv + nc * nw * nv * (nv - 1) // 2
    inst = make_instance(nc, nw, nv, L, seed=4, scale=0.2)
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, N, conv=1e-9)
    ref = osolve.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, N, method="dense",
                       want_vectors=False)
    assert out["status"] == 0
    assert np.abs(out["omega"] - ref["omega"]).max() < 1e-9
    assert np.abs(out["osc"] - ref["osc"]).max() < 1e-8
    ctx.close()


def test_root_count_beyond_the_space_is_rejected():
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L = 1, 1, 2, 1
    N = nc * nv + nc * nw * nv * (nv - 1) // 2
    inst = make_instance(nc, nw, nv, L, seed=4, scale=0.2)
    ctx = pkg.Context(0)
    with pytest.raises(pkg.CvsadcError) as e:
        ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, N + 1)
    assert e.value.code == -1  # CVSADC_EINVAL
    ctx.close()


def test_empty_batch():
    import paper_2604_27451_gb300 as pkg

    ctx = pkg.Context(0)
    assert ctx.solve_batched([], 4) == []
    ctx.close()


def test_more_roots_than_singles_with_the_preconditioner():
    """ncore nvirt = 3 singles but 5 roots: the guesses cannot all come from
    the folded singles block, yet every root must match the oracle."""
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L = 1, 4, 3, 12
    inst = make_instance(nc, nw, nv, L, seed=6)
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, 5, conv=1e-9)
    ref = osolve.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, 5, method="dense",
                       want_vectors=False)
    assert np.abs(out["omega"] - ref["omega"]).max() < 1e-9
    ctx.close()


def test_bounded_wait_expires_with_etimeout():
    """A bounded device wait that nothing satisfies gives up after its limit
    and surfaces as CVSADC_ETIMEOUT; the kernel returns, so the context
    (and its error flag) is usable for the next call."""
    import time

    import paper_2604_27451_gb300 as pkg
    from paper_2604_27451_gb300._lib import CVSADC_ETIMEOUT

    ctx = pkg.Context(0)
    t0 = time.perf_counter()
    with pytest.raises(pkg.CvsadcError) as ei:
        ctx.wait_probe(200_000_000)
    assert ei.value.code == CVSADC_ETIMEOUT
    assert time.perf_counter() - t0 >= 0.2
    rng = np.random.default_rng(8)
    A = rng.standard_normal((300, 400)) + 1j * rng.standard_normal((300, 400))
    B = rng.standard_normal((400, 200)) + 1j * rng.standard_normal((400, 200))
    C = ctx.zgemm(A, B, "slice4")
    assert (np.abs(C - A @ B) / (np.abs(A) @ np.abs(B))).max() < 1e-6
    ctx.close()
