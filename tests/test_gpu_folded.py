"""The doubles-folded solver (CVSADC_FLAG_FOLDED) against the oracle.

M22 is diagonal, so the eigenvalues of M below the lowest M22 entry are the
fixed points of the singles-space pseudo-eigenvalue problem S(w) x1 = w x1,
S(w) = M11 + M12 (w - M22)^-1 M21 (Eqs. 11-12).  The folded solver never
stores a doubles vector; its Rayleigh-Ritz step is nevertheless the one of
M in the full space, so FP64 roots must match the oracle's exact
eigenvalues to 1e-9 Eh (the FP64 path's bar) and the mixed precision
(SLICE4 with the FP64-class continuation) to 1e-5 Eh (the mixed bar: its
problem, t2 and M11, is built with 4-slice products, ~1e-8 Eh here),
oscillator strengths within the residual / gap bound of tests/bounds.py,
and the rebuilt full eigenvectors must be eigenvectors of the oracle's
explicit matrix.
"""

import json
import os

import numpy as np
import pytest

from bounds import osc_tolerance
from oracle import adc2
from oracle import solve as osolve
from synth import make_instance

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
TOL = {"fp64": 1e-9, "slice4": 1e-5}


@pytest.mark.parametrize("prec,precond", [("fp64", "schur"), ("slice4", "schur"),
                                          ("fp64", "diag")])
def test_folded_roots_and_osc_match_oracle(prec, precond):
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L, k = 3, 7, 37, 70, 4
    inst = make_instance(nc, nw, nv, L, seed=2)
    ref = osolve.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, k + 1, method="partitioned")
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, nc, nw, nv, k, precision=prec, conv=1e-8,
                    precond=precond, solver="folded", return_x=True, max_iter=400)
    assert out["status"] == 0, out["info"]
    assert out["info"]["sigma_vectors"] == 0  # no full-space sigma was built
    assert np.abs(out["omega"] - ref["omega"][:k]).max() < TOL[prec]
    tol = osc_tolerance(ref["omega"][:k], ref["omega"][k], 1e-8, ref["osc"][:k])
    assert (np.abs(out["osc"] - ref["osc"][:k]) <= tol).all()
    # the rebuilt full vectors: normalised eigenvectors of the explicit M
    M11 = adc2.m11(inst.eps, inst.B, nc, nw, nv)
    sig = adc2.Sigma(inst.eps, inst.B, nc, nw, nv, M11=M11)
    X = out["X"]
    N1 = nc * nv
    for q in range(k):
        x = X[q]
        s1, s2 = sig(x[:N1], x[N1:])
        r = np.concatenate([s1, s2]) - out["omega"][q] * x
        assert abs(np.linalg.norm(x) - 1.0) < 1e-10
        assert np.linalg.norm(r) < (1e-7 if prec == "fp64" else 1e-5)
    ctx.close()


def test_folded_small_workload_golden():
    """The small workload (6/14/40/240, 4 roots) against the stored exact
    roots and oscillator strengths (tests/golden/small_fp64.json, written by
    the oracle)."""
    import paper_2604_27451_gb300 as pkg

    g = json.load(open(os.path.join(GOLDEN, "small_fp64.json")))
    sh = g["shape"]
    inst = make_instance(sh["ncore"], sh["nval"], sh["nvirt"], sh["naux"], seed=g["seed"])
    ctx = pkg.Context(0)
    for prec in ("fp64", "slice4"):
        out = ctx.solve(inst.eps, inst.B, inst.dip, sh["ncore"], sh["nval"], sh["nvirt"],
                        sh["nroots"], precision=prec, conv=1e-8, solver="folded")
        assert out["status"] == 0, (prec, out["info"])
        assert np.abs(out["omega"] - np.array(g["omega"])).max() < TOL[prec], prec
        tol = osc_tolerance(g["omega"], g["omega_next"], 1e-8, g["osc"])
        assert (np.abs(out["osc"] - np.array(g["osc"])) <= tol).all(), prec
    ctx.close()


def test_folded_agrees_with_full_space_solver():
    """Same roots from the two solvers on a problem with more roots (8)."""
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L, k = 4, 10, 50, 150, 8
    inst = make_instance(nc, nw, nv, L, seed=9)
    ctx = pkg.Context(0)
    a = ctx.solve(inst.eps, inst.B, None, nc, nw, nv, k, precision="fp64", conv=1e-8)
    b = ctx.solve(inst.eps, inst.B, None, nc, nw, nv, k, precision="fp64", conv=1e-8,
                  solver="folded")
    assert a["status"] == 0 and b["status"] == 0
    assert np.abs(a["omega"] - b["omega"]).max() < 1e-9
    ctx.close()


def test_folded_large_singles_space():
    """N1 = 12 x 360 = 4320 exceeds the dense Schur decomposition's range:
    the preconditioner is then the lowest eigenpairs of S(theta0) from a
    block Davidson, built with BF16X3 products and an approximate cross
    term.  It only steers the iteration, so the roots must still be exact
    eigenvalues: the rebuilt eigenvectors satisfy ||M x - w x|| <= 1e-6
    under the oracle's matrix-free sigma, and the roots agree to 1e-9 Eh
    with the same solver preconditioned by the diagonal."""
    import paper_2604_27451_gb300 as pkg

    nc, nw, nv, L, k = 12, 2, 360, 40, 3
    inst = make_instance(nc, nw, nv, L, seed=13)
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, None, nc, nw, nv, k, precision="fp64", conv=1e-8,
                    solver="folded", return_x=True, max_iter=400)
    assert out["status"] == 0, out["info"]
    assert out["info"]["schur_theta"] != 0.0  # the large-space preconditioner ran
    ref = ctx.solve(inst.eps, inst.B, None, nc, nw, nv, k, precision="fp64", conv=1e-8,
                    solver="folded", precond="diag", max_iter=2000)
    assert ref["status"] == 0, ref["info"]
    assert np.abs(out["omega"] - ref["omega"]).max() < 1e-9
    sig = adc2.Sigma(inst.eps, inst.B, nc, nw, nv)
    N1 = nc * nv
    for q in range(k):
        x = out["X"][q]
        s1, s2 = sig(x[:N1], x[N1:])
        r = np.concatenate([s1, s2]) - out["omega"][q] * x
        assert np.linalg.norm(r) < 1e-6, (q, np.linalg.norm(r))
    ctx.close()


def test_spectrum_matches_oracle():
    """The broadened spectrum of the small workload's roots and oscillator
    strengths (FWHM 0.3 eV, a -4.1 eV shift) against the oracle's sum of
    Lorentzians, to 1e-12 of its maximum."""
    import paper_2604_27451_gb300 as pkg
    from oracle import spectrum

    g = json.load(open(os.path.join(GOLDEN, "small_fp64.json")))
    om, f = np.array(g["omega"]), np.array(g["osc"])
    ctx = pkg.Context(0)
    e0, de, n = 400.0, 0.01, 6001
    got = ctx.spectrum(om, f, e0, de, n, 0.3, -4.1)
    ref = spectrum.lorentzian_spectrum(om, f, e0 + de * np.arange(n), 0.3, -4.1)
    assert np.abs(got - ref).max() < 1e-12 * ref.max()
    assert np.abs(ctx.spectrum([], [], e0, de, 3) ).max() == 0.0
    ctx.close()
