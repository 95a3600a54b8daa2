"""GPU parity: the CUDA path through the C ABI against the CPU oracle.

Sizes span several 64x64x8 GEMM tiles with ragged tails in every
dimension.  FP64 tolerances follow from the arithmetic: every quantity is
a sum of O(K) products in FP64 with a different summation order than the
oracle, so the element-wise error bound is ~K * 2^-53 * sum|a||b|; the
tests use 1e-11 relative to the largest entry (K <= 10^4 here), and 1e-9
Eh absolute on eigenvalues (the accuracy required of the FP64 path).
"""

import json
import os

import numpy as np
import pytest

from bounds import osc_tolerance
from oracle import adc2, fns, mp2
from oracle import solve as osolve
from synth import make_instance

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")

# ragged against the 64x64x8 tiles: o = 10, v = 37, naux = 70
RAGGED = dict(ncore=3, nval=7, nvirt=37, naux=70, seed=2)


@pytest.fixture(scope="module")
def pkg():
    import paper_2604_27451_gb300 as p

    return p


@pytest.fixture(scope="module")
def ragged(pkg):
    c = RAGGED
    inst = make_instance(c["ncore"], c["nval"], c["nvirt"], c["naux"], seed=c["seed"])
    ctx = pkg.Context(0)
    ctx.prepare(inst.eps, inst.B, inst.dip, inst.ncore, inst.nval, inst.nvirt)
    yield inst, ctx
    ctx.close()


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def test_t2_and_mp2_energy(ragged):
    inst, ctx = ragged
    t2, e = ctx.get_t2()
    ref = mp2.t2_amplitudes(inst.eps, inst.B, inst.ncore, inst.nval, inst.nvirt)
    eref = mp2.mp2_energy(inst.eps, inst.B, inst.ncore, inst.nval, inst.nvirt).real
    assert _rel(t2, ref) < 1e-12
    assert abs(e - eref) < 1e-12 * abs(eref)


def test_m11(ragged):
    inst, ctx = ragged
    m = ctx.get_m11()
    ref = adc2.m11(inst.eps, inst.B, inst.ncore, inst.nval, inst.nvirt)
    assert _rel(m, ref) < 1e-11


def test_transition_moments(ragged):
    inst, ctx = ragged
    F = ctx.get_moments()
    ref = adc2.transition_moments(inst.eps, inst.B, inst.dip, inst.ncore,
                                  inst.nval, inst.nvirt)
    assert _rel(F, ref) < 1e-11


def test_sigma_fp64(ragged):
    inst, ctx = ragged
    N1, _, N2 = adc2.sizes(inst.ncore, inst.nval, inst.nvirt)
    rng = np.random.default_rng(5)
    x = rng.standard_normal((2, N1 + N2)) + 1j * rng.standard_normal((2, N1 + N2))
    s = ctx.sigma(np.ascontiguousarray(x), "fp64")
    sig = adc2.Sigma(inst.eps, inst.B, inst.ncore, inst.nval, inst.nvirt)
    for q in range(2):
        r1, r2 = sig(x[q, :N1], x[q, N1:])
        ref = np.concatenate([r1, r2])
        assert _rel(s[q], ref) < 1e-11


def test_sigma_device_pointers_match_host(ragged, pkg):
    import torch

    inst, ctx = ragged
    N = ctx.shape["N"]
    rng = np.random.default_rng(6)
    x = rng.standard_normal((1, N)) + 1j * rng.standard_normal((1, N))
    host = ctx.sigma(np.ascontiguousarray(x), "fp64")
    xd = torch.from_numpy(x).to("cuda:0")
    dev = ctx.sigma(xd, "fp64").cpu().numpy()
    assert np.array_equal(host, dev)


def test_davidson_tiny_dense():
    import paper_2604_27451_gb300 as pkg

    inst = make_instance(2, 4, 12, 20, seed=12)
    nroots = 5
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, 2, 4, 12, nroots, conv=1e-9,
                    return_x=True)
    ref = osolve.solve(inst.eps, inst.B, inst.dip, 2, 4, 12, nroots + 1, method="dense")
    assert out["status"] == 0
    assert np.abs(out["omega"] - ref["omega"][:nroots]).max() < 1e-9
    tol = osc_tolerance(ref["omega"][:nroots], ref["omega"][nroots], 1e-9, ref["osc"][:nroots])
    assert (np.abs(out["osc"] - ref["osc"][:nroots]) <= tol).all()
    # eigenvectors: unit norm, residual small against the oracle matrix
    M = adc2.adc_matrix(inst.eps, inst.B, 2, 4, 12)
    for k in range(nroots):
        x = out["X"][k]
        assert abs(np.linalg.norm(x) - 1) < 1e-10
        assert np.linalg.norm(M @ x - out["omega"][k] * x) < 1e-8
        j = np.argmax(np.abs(x))
        assert abs(x[j].imag) < 1e-14 and x[j].real > 0
    ctx.close()


def test_small_workload_roots_against_golden():
    """The small workload (6/14/40/240, 4 roots) against the oracle's exact
    partitioned eigenvalues stored by tests/golden/make_golden.py."""
    import paper_2604_27451_gb300 as pkg

    g = json.load(open(os.path.join(GOLDEN, "small_fp64.json")))
    w = g["shape"]
    inst = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=g["seed"])
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, w["ncore"], w["nval"], w["nvirt"],
                    w["nroots"], conv=1e-7)
    assert out["status"] == 0
    assert np.abs(out["omega"] - np.array(g["omega"])).max() < 1e-9
    assert abs(out["info"]["emp2"] - g["emp2"]) < 1e-12 * abs(g["emp2"])
    tol = osc_tolerance(g["omega"], g["omega_next"], 1e-7, g["osc"])
    assert (np.abs(out["osc"] - np.array(g["osc"])) <= tol).all()
    ctx.close()


def test_fns_truncation_roots():
    import paper_2604_27451_gb300 as pkg

    inst = make_instance(2, 4, 14, 20, seed=33, scale=0.1)
    D = mp2.density_vv(inst.eps, inst.B, 2, 4, 14)
    occ = np.sort(np.linalg.eigvalsh(D))[::-1]
    tau = 0.5 * (occ[8] + occ[9])
    ctx = pkg.Context(0)
    out = ctx.solve(inst.eps, inst.B, inst.dip, 2, 4, 14, 3, tau=tau, conv=1e-9)
    assert ctx.shape["nvirt"] == 9
    ref = osolve.solve(inst.eps, inst.B, inst.dip, 2, 4, 14, 3, tau=tau, method="dense")
    assert np.abs(out["omega"] - ref["omega"]).max() < 1e-9
    occ_gpu, U = ctx.get_fns()
    assert np.abs(occ_gpu - occ).max() < 1e-13 * occ.max()
    assert np.abs(U.conj().T @ U - np.eye(9)).max() < 1e-12
    n_o, U_o, et = fns.natural_spinors(inst.eps, inst.B, 2, 4, 14, tau)
    # U is defined up to a phase per column: compare |U^H U_o|
    ov = np.abs(U.conj().T @ U_o)
    assert np.abs(ov - np.eye(9)).max() < 1e-9
    ctx.close()


def test_nonhermitian_input_rejected():
    import paper_2604_27451_gb300 as pkg

    inst = make_instance(2, 2, 4, 5, seed=1)
    B = inst.B.copy()
    B[1, 0, 3] += 1e-6
    ctx = pkg.Context(0)
    with pytest.raises(pkg.CvsadcError) as e:
        ctx.solve(inst.eps, B, inst.dip, 2, 2, 4, 1)
    assert e.value.code == -2
    with pytest.raises(pkg.CvsadcError) as e:
        ctx.solve(inst.eps, inst.B, inst.dip, 0, 2, 4, 1)
    assert e.value.code == -1
    ctx.close()
