"""Top-level oracle solve: spinor energies, Cholesky vectors and dipoles in;
excitation energies, eigenvectors and oscillator strengths out.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Follows the paper's pipeline (section "Implementation and Computational
Details"): MP2 amplitudes and energy from the Cholesky vectors; optional
frozen-natural-spinor truncation and rotation of B^P; the CVS-ADC(2)
matrix in the (truncated) basis; its lowest eigenpairs (Eq. 11); the
transition moments and oscillator strengths (section "Properties in ISR
formulation").
"""

from __future__ import annotations

import numpy as np

from . import adc2, fns, mp2


def solve(eps, B, dip, ncore, nval, nvirt, nroots, tau=0.0, method="auto",
          want_vectors=True):
    out = {}
    if tau > 0:
        n, U, et = fns.natural_spinors(eps, B, ncore, nval, nvirt, tau)
        eps, B = fns.rotate(eps, B, ncore, nval, nvirt, U, et)
        if dip is not None:
            o = ncore + nval
            d2 = np.empty((dip.shape[0],) + B.shape[1:], dtype=np.complex128)
            d2[:, :o, :o] = dip[:, :o, :o]
            d2[:, :o, o:] = dip[:, :o, o:] @ U
            d2[:, o:, :o] = U.conj().T @ dip[:, o:, :o]
            d2[:, o:, o:] = U.conj().T @ dip[:, o:, o:] @ U
            dip = d2
        out["occupations"] = n
        nvirt = U.shape[1]
        out["nvirt_kept"] = nvirt
    t2 = mp2.t2_amplitudes(eps, B, ncore, nval, nvirt)
    out["emp2"] = float(np.real(mp2.mp2_energy(eps, B, ncore, nval, nvirt, t2=t2)))
    N1, npair, N2 = adc2.sizes(ncore, nval, nvirt)
    M11 = adc2.m11(eps, B, ncore, nval, nvirt, t2=t2)
    d22 = adc2.m22(eps, ncore, nval, nvirt)
    if method == "auto":
        method = "dense" if N1 + N2 <= 4000 else "partitioned"
    M21 = adc2.m21(eps, B, ncore, nval, nvirt)
    if method == "dense":
        M = np.block([[M11, M21.conj().T], [M21, np.diag(d22).astype(complex)]])
        w, X = adc2.eig_dense(M, nroots)
    elif method == "partitioned":
        w, X = adc2.eig_partitioned(M11, M21, d22, nroots)
    elif method == "lanczos":
        w, X = adc2.eig_lanczos(M11, M21, d22, nroots)
    else:
        raise ValueError(method)
    out["omega"] = w
    if want_vectors:
        out["X"] = X
    if dip is not None:
        F = adc2.transition_moments(eps, B, dip, ncore, nval, nvirt, t2=t2)
        out["osc"] = adc2.oscillator_strengths(w, X, F)
    return out
