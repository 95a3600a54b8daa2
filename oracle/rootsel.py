"""Root-specific CVS-ADC(2) roots in the frozen-natural-spinor basis.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section "Implementation and Computational Details" builds its initial
guesses for CVS-ADC(2) in the truncated FNS basis from the canonical CIS
eigenvectors, transformed into that basis. It then follows each root with a
root-specific Davidson (root homing), so that each FNS root corresponds to
its canonical counterpart. Written out on an explicit matrix:

* The FNS virtuals are phi'_a' = sum_a phi_a U_{a a'} (``oracle.fns``), so a
  singles vector with coefficients b_{Ia} on phi_a has coefficients
  b'_{Ia'} = sum_a conj(U_{a a'}) b_{Ia} on phi'_a' (U^H b per core row).
  With every virtual kept, U is unitary and this maps CIS eigenvectors of
  the canonical problem onto CIS eigenvectors of the rotated one.
* Root following picks, for each guess g_k in turn, the eigenpair (w, x) of
  the FNS-basis CVS-ADC(2) matrix M whose singles part has the largest
  |g_k^H x_1|^2 among the eigenpairs not yet taken. That is the eigenvector
  a root-homing Davidson converges to from g_k when the overlaps are
  distinct.
"""

from __future__ import annotations

import numpy as np

from . import adc2, cisd, fns


def cis_guesses_in_fns(eps, B, ncore, nval, nvirt, nroots, U):
    """The lowest nroots canonical CIS eigenvectors [nroots, ncore*nvirt]
    expressed in the FNS virtual basis of U [nvirt, nvirt']."""
    _, _, b = cisd.cisd_energies(eps, B, ncore, nval, nvirt, nroots)
    bb = b.reshape(nroots, ncore, nvirt)
    return np.einsum("aA,kIa->kIA", np.conj(U), bb).reshape(nroots, -1)


def follow_roots(M, N1, guesses):
    """(omega [k], X [k, N]) of M, one eigenpair per guess [k, N1] by
    largest singles overlap, each eigenpair taken once."""
    w, V = np.linalg.eigh(M)
    ov = np.abs(np.conj(guesses) @ V[:N1, :]) ** 2  # [k, all]
    taken, out_w, out_x = set(), [], []
    for k in range(guesses.shape[0]):
        order = np.argsort(-ov[k], kind="stable")
        j = next(int(j) for j in order if int(j) not in taken)
        taken.add(j)
        out_w.append(w[j])
        out_x.append(V[:, j])
    return np.array(out_w), adc2.fix_phase(np.array(out_x))


def root_specific_fns(eps, B, ncore, nval, nvirt, nroots, tau):
    """CVS-ADC(2) roots in the FNS basis at threshold tau that follow the
    lowest nroots canonical CIS states: (omega, X, guesses)."""
    _, U, et = fns.natural_spinors(eps, B, ncore, nval, nvirt, tau)
    e2, B2 = fns.rotate(eps, B, ncore, nval, nvirt, U, et)
    nv2 = U.shape[1]
    g = cis_guesses_in_fns(eps, B, ncore, nval, nvirt, nroots, U)
    M = adc2.adc_matrix(e2, B2, ncore, nval, nv2)
    w, X = follow_roots(M, ncore * nv2, g)
    return w, X, g
