"""Write the stored oracle values used by the GPU parity tests.

Calls only ``oracle/`` and ``synth/``.  Run from the repository root:
    python tests/golden/make_golden.py
"""

import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

from oracle import adc2, mp2  # noqa: E402
from synth import WORKLOADS, make_instance  # noqa: E402


def small():
    w = WORKLOADS["small"]
    inst = make_instance(w["ncore"], w["nval"], w["nvirt"], w["naux"], seed=0)
    nc, nw, nv = inst.ncore, inst.nval, inst.nvirt
    t2 = mp2.t2_amplitudes(inst.eps, inst.B, nc, nw, nv)
    e2 = mp2.mp2_energy(inst.eps, inst.B, nc, nw, nv, t2=t2).real
    M11 = adc2.m11(inst.eps, inst.B, nc, nw, nv, t2=t2)
    M21 = adc2.m21(inst.eps, inst.B, nc, nw, nv)
    d22 = adc2.m22(inst.eps, nc, nw, nv)
    w_, X = adc2.eig_partitioned(M11, M21, d22, w["nroots"] + 1)
    omega_next = float(w_[-1])  # root k + 1: the gap of root k (eigenvector bounds)
    w_, X = w_[:-1], X[:-1]
    F = adc2.transition_moments(inst.eps, inst.B, inst.dip, nc, nw, nv, t2=t2)
    f = adc2.oscillator_strengths(w_, X, F)
    out = dict(
        source="oracle: exact Lowdin-partitioned eigenvalues of the explicit "
               "CVS-ADC(2) matrix (oracle/adc2.py), seeded synthetic inputs",
        shape=w, seed=0, emp2=float(e2), omega=[float(x) for x in w_],
        omega_next=omega_next,
        osc=[float(x) for x in f],
        singles_weight=[float(np.sum(np.abs(X[k, :M11.shape[0]]) ** 2)) for k in range(len(w_))],
    )
    with open(os.path.join(HERE, "small_fp64.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(json.dumps(out, indent=1))


if __name__ == "__main__":
    small()
