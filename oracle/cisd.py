"""CIS(D) excitation energies and the frozen-natural-spinor correction of
Eqs. 21-22.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section "State-Average Frozen Natural Spinors" corrects each CVS-ADC(2)
root computed in the truncated FNS basis. The correction is the change of
the CIS(D) energy of the same state between the canonical and the FNS basis:

    dE(k)          = E_CIS(D)^canonical(k) - E_CIS(D)^FNS(k)      (Eq. 21)
    E_corrected(k) = E_ADC(2)^FNS(k) + dE(k)                       (Eq. 22)

The paper does not print CIS(D). It is the perturbative doubles correction
to CIS (Head-Gordon, Rico, Oumi and Lee, 1994), and it equals the first-order
estimate of the ADC(2) eigenvalue from the CIS eigenvector. Here it is
restricted to the CVS spaces: core singles, and core-valence doubles with
M22 diagonal (Eqs. 11-12).

    omega_CIS(D) = omega_CIS + E_v + E_u
    E_v = b^H M11^(2) b
    E_u = sum_d |(M21 b)_d|^2 / (omega_CIS - M22_d)
        = - sum_{I j a<b} |u^{ab}_{Ij}|^2 / (e_a + e_b - e_I - e_j - omega_CIS)
    u^{ab}_{Ij} = sum_c <ab||cj> b_Ic - sum_K (<Kb||Ij> b_Ka - <Ka||Ij> b_Kb)

Here (omega_CIS, b) is an eigenpair of the CIS block M11^(0+1)
= d_IJ d_ab (e_a - e_I) - <aJ||bI>, and M11^(2) is the second-order part of
M11 (``oracle.adc2``). States are matched by energy order in the two bases.

Pins (tests/test_oracle_pins.py):

- E_v + E_u is the lambda^2 coefficient of the lowest eigenvalues of the
  coupling-scaled matrix [[M_CIS + lambda^2 M11^(2), lambda M12],
  [lambda M21, M22]], whose eigenvalue at lambda = 0 is omega_CIS.
- E_u from the explicit u above (integrals, not M21) equals the folded form.
- Keeping every virtual in the FNS step leaves dE = 0 to rounding.
"""

from __future__ import annotations

import numpy as np

from . import adc2, fns
from .integrals import antisym
from .mp2 import t2_amplitudes


def cis_block(eps, B, ncore, nval, nvirt):
    """M11^(0+1) of the CVS singles, [N1, N1]."""
    return adc2.m11(eps, B, ncore, nval, nvirt, second_order=False)


def cisd_energies(eps, B, ncore, nval, nvirt, nroots, t2=None):
    """(omega_CIS, omega_CIS(D), b [nroots, N1]) for the lowest nroots CIS
    states (module docstring)."""
    if t2 is None:
        t2 = t2_amplitudes(eps, B, ncore, nval, nvirt)
    A = cis_block(eps, B, ncore, nval, nvirt)
    w, U = np.linalg.eigh(A)
    w, b = w[:nroots], U[:, :nroots].T
    M2 = adc2.m11(eps, B, ncore, nval, nvirt, t2=t2) - A
    M21 = adc2.m21(eps, B, ncore, nval, nvirt)
    d22 = adc2.m22(eps, ncore, nval, nvirt)
    ev = np.einsum("ki,ij,kj->k", np.conj(b), M2, b).real
    z = b @ M21.T  # (M21 b_k) as rows
    eu = np.sum(np.abs(z) ** 2 / (w[:, None] - d22[None, :]), axis=1)
    return w, w + ev + eu, b


def doubles_term_explicit(eps, B, ncore, nval, nvirt, omega, b):
    """E_u of one CIS state from the explicit u^{ab}_{Ij} (module docstring),
    summed over the CVS doubles (I core, j valence, a < b)."""
    C = np.arange(ncore)
    W = np.arange(ncore, ncore + nval)
    V = np.arange(ncore + nval, ncore + nval + nvirt)
    bI = b.reshape(ncore, nvirt)  # b_Ic
    vvvw = antisym(B, V, V, V, W)  # <ab||cj> as [a, b, c, j]
    cvcw = antisym(B, C, V, C, W)  # <Kb||Ij> as [K, b, I, j]
    u = (np.einsum("abcj,Ic->Ijab", vvvw, bI)
         - np.einsum("KbIj,Ka->Ijab", cvcw, bI)
         + np.einsum("KaIj,Kb->Ijab", cvcw, bI))
    den = (eps[V][None, None, :, None] + eps[V][None, None, None, :]
           - eps[C][:, None, None, None] - eps[W][None, :, None, None] - omega)
    iu = np.triu_indices(nvirt, 1)
    return -np.sum(np.abs(u[:, :, iu[0], iu[1]]) ** 2 / den[:, :, iu[0], iu[1]])


def fns_correction(eps, B, ncore, nval, nvirt, nroots, tau):
    """Eqs. 21-22: (dE, E_ADC(2)^FNS, E_corrected) for the lowest nroots
    states, with the FNS truncation of ``oracle.fns`` at threshold tau."""
    _, cisd_can, _ = cisd_energies(eps, B, ncore, nval, nvirt, nroots)
    _, U, et = fns.natural_spinors(eps, B, ncore, nval, nvirt, tau)
    e2, B2 = fns.rotate(eps, B, ncore, nval, nvirt, U, et)
    nv2 = U.shape[1]
    _, cisd_fns, _ = cisd_energies(e2, B2, ncore, nval, nv2, nroots)
    M = adc2.adc_matrix(e2, B2, ncore, nval, nv2)
    w_adc = np.linalg.eigvalsh(M)[:nroots]
    dE = cisd_can - cisd_fns
    return dE, w_adc, w_adc + dE
