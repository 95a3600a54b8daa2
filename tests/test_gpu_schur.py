"""GPU: the Schur-complement preconditioner of the Davidson solver.

S(theta) = M11 + M12 (theta - M22)^-1 M21 from the library (built from
<ab||cj> and <Kb||Ij> contractions) against the oracle's explicit blocks,
element by element; then solves with the preconditioner against solves
without it and against the oracle's exact roots.  The preconditioner only
steers the iteration, so the roots agree to the solver tolerance.
"""

import json
import os

import numpy as np
import pytest

from bounds import osc_tolerance
from oracle import adc2
from oracle import solve as osolve
from synth import WORKLOADS, make_instance

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.mark.parametrize("shape,seed", [((3, 7, 37, 70), 2), ((2, 4, 9, 14), 5)])
def test_schur_matrix_against_oracle(shape, seed):
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L = shape
    inst = make_instance(nc, nw, nv, L, seed=seed)
    ctx = pkg.Context(0)
    ctx.prepare(inst.eps, inst.B, None, nc, nw, nv)
    M11 = adc2.m11(inst.eps, inst.B, nc, nw, nv)
    M21 = adc2.m21(inst.eps, inst.B, nc, nw, nv)
    D = adc2.m22(inst.eps, nc, nw, nv).reshape(-1)
    for theta in (D.min() - 3.0, D.min() - 0.25, D.min() - 40.0):
        ref = M11 + (M21.conj().T / (theta - D)) @ M21
        S = ctx.get_schur(theta)
        assert np.abs(S - ref).max() < 1e-11 * np.abs(ref).max(), theta
    ctx.close()


@pytest.mark.parametrize("precision", ["fp64", "slice4"])
def test_schur_preconditioned_roots(precision):
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L, k = 3, 6, 20, 60, 4
    inst = make_instance(nc, nw, nv, L, seed=8)
    ctx = pkg.Context(0)
    a = ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, k, precision=precision,
                  conv=1e-8)
    b = ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, k, precision=precision,
                  conv=1e-8, precond="diag")
    ref = osolve.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, k + 1, want_vectors=False)
    ref = {"omega": ref["omega"][:k], "osc": ref["osc"][:k], "next": ref["omega"][k]}
    assert a["info"]["schur_theta"] != 0.0
    assert b["info"]["schur_theta"] == 0.0
    tol = 1e-9 if precision == "fp64" else 1e-5
    assert np.abs(a["omega"] - ref["omega"]).max() < tol
    assert np.abs(a["omega"] - b["omega"]).max() < tol
    assert (np.abs(a["osc"] - ref["osc"]) <= osc_tolerance(ref["omega"], ref["next"], 1e-8,
                                                          ref["osc"])).all()
    # theta0 sits at or above the lowest root (Newton from above)
    assert a["info"]["schur_theta"] >= ref["omega"][0] - 1e-6
    ctx.close()


def test_schur_small_workload_golden_and_work():
    """The small workload: roots against the oracle's stored exact values,
    and the preconditioned solve does less than half the sigma work."""
    import paper_2604_27451_gb300 as pkg

    w = WORKLOADS["small"]
    with open(os.path.join(GOLDEN, "small_fp64.json")) as f:
        gold = json.load(f)
    inst = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=0)
    ctx = pkg.Context(0)
    args = (inst.eps, inst.B, inst.dip, w["ncore"], w["nval"], w["nvirt"], w["nroots"])
    a = ctx.solve(*args, conv=1e-7)
    b = ctx.solve(*args, conv=1e-7, precond="diag")
    assert np.abs(a["omega"] - np.array(gold["omega"])).max() < 1e-9
    work_a = a["info"]["sigma_vectors"] + 0.5 * a["info"]["coupling_vectors"]
    work_b = b["info"]["sigma_vectors"]
    print("sigma work with / without the Schur preconditioner:", work_a, work_b,
          "iterations", a["info"]["iterations"], b["info"]["iterations"],
          "theta0", a["info"]["schur_theta"], "builds", a["info"]["schur_builds"])
    assert work_a < 0.5 * work_b
    ctx.close()
