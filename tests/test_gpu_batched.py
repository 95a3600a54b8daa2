"""GPU: many ragged problems through cvsadc_solve_batched.

Each instance of a batch must give what the unbatched call gives on the
same inputs (the lanes run the same kernels on the same data, so FP64
results are bit-identical, whatever the lane count or completion order),
and the smallest instances are checked against the oracle's exact roots.
The shapes follow the batched workload's recipe (ncore 6, even nval,
naux = 5 nvirt, seed 1000 + i) at sizes the oracle finishes in seconds.
"""

import numpy as np
import pytest

from oracle import solve as osolve
from synth import make_instance

pytestmark = pytest.mark.gpu


def _batch(count=7, seed=5):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nval = int(rng.integers(1, 5)) * 2
        nvirt = int(rng.integers(6, 25))
        inst = make_instance(6, nval, nvirt, 5 * nvirt, seed=1000 + i, scale=0.2)
        out.append(dict(eps=inst.eps, B=inst.B, dip=inst.dip, ncore=6, nval=nval,
                        nvirt=nvirt))
    return out


@pytest.mark.parametrize("precision", ["fp64", "slice4"])
def test_batched_equals_unbatched(precision):
    import paper_2604_27451_gb300 as pkg

    batch = _batch()
    ctx = pkg.Context(0)
    k = 4
    res3 = ctx.solve_batched(batch, k, precision=precision, conv=1e-8, lanes=3,
                             return_x=True)
    res1 = ctx.solve_batched(batch, k, precision=precision, conv=1e-8, lanes=1)
    for b, r3, r1 in zip(batch, res3, res1):
        one = ctx.solve(b["eps"], b["B"], b["dip"], b["ncore"], b["nval"], b["nvirt"], k,
                        precision=precision, conv=1e-8, return_x=True)
        assert r3["status"] == 0 and r1["status"] == 0
        # same kernels on the same data: identical bits
        np.testing.assert_array_equal(r3["omega"], one["omega"])
        np.testing.assert_array_equal(r1["omega"], one["omega"])
        # eigenvectors too: lanes running beside each other change the order
        # in which blocks of a kernel run, which must not change any result
        np.testing.assert_array_equal(r3["X"], one["X"])
        np.testing.assert_array_equal(r3["osc"], one["osc"])
        np.testing.assert_array_equal(r1["osc"], one["osc"])
        assert r3["info"]["converged"] == k
    # the two smallest against the oracle's exact roots
    order = np.argsort([b["nvirt"] * b["nval"] for b in batch])
    for i in order[:2]:
        b = batch[i]
        ref = osolve.solve(b["eps"], b["B"], b["dip"], 6, b["nval"], b["nvirt"], k,
                           want_vectors=False)
        tol = 1e-9 if precision == "fp64" else 1e-5
        assert np.abs(res3[i]["omega"] - ref["omega"]).max() < tol
    ctx.close()


def test_batched_reports_per_instance_errors():
    import paper_2604_27451_gb300 as pkg

    batch = _batch(3)
    bad = dict(batch[1])
    B = bad["B"].copy()
    B[0, 0, 1] += 0.5  # no longer Hermitian
    bad["B"] = B
    batch[1] = bad
    ctx = pkg.Context(0)
    with pytest.raises(pkg.CvsadcError) as e:
        ctx.solve_batched(batch, 2, conv=1e-8, lanes=2)
    assert e.value.code == -2  # CVSADC_ENONHERM, from instance 1
    assert "instance 1" in str(e.value)
    ctx.close()


def test_estimate_bounds_device_bytes():
    """The admission estimate is an upper bound of what a solve holds."""
    import paper_2604_27451_gb300 as pkg

    ctx = pkg.Context(0)
    for (nc, nw, nv, L), prec in [((6, 8, 40, 200), "fp64"), ((6, 20, 100, 500), "slice4")]:
        inst = make_instance(nc, nw, nv, L, seed=3, scale=0.2)
        ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, 4, precision=prec, conv=1e-6,
                  max_iter=60)
        held = ctx.device_bytes()
        est = pkg.estimate_bytes(nc, nw, nv, L, nroots=4, precision=prec)
        assert held <= est <= 3 * held + (256 << 20), (held, est)
    ctx.close()
