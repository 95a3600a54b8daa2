"""MP2 amplitudes, MP2 energy and the MP2 virtual-virtual density.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Spinors are ordered [core | valence | virtual]; occupied indices i, j run
over core and valence (all correlated occupied spinors: the frozen core lies
below the metal 2p levels and is not part of the input).

* t^{ab}_{ij} = <ab||ij> / (e_i + e_j - e_a - e_b): the first-order doubles
  amplitudes whose ratios appear in Eq. 15 (section "State-Average Frozen
  Natural Spinors"); they are built on the fly from the Cholesky vectors
  (section "Implementation and Computational Details").
* E_MP2 = 1/4 sum_{ijab} <ij||ab> t^{ab}_{ij}.
* D_ab = 1/2 sum_{cij} <ac||ij><ij||bc> / (e^{ac}_{ij} e^{bc}_{ij}), Eq. 15.

Pins (tests/test_oracle_pins.py): E_MP2 equals the Rayleigh-Schrodinger
second-order energy of the determinant-space Hamiltonian; t2 is
antisymmetric in both index pairs; D is Hermitian, positive semidefinite
with trace 1/2 sum |t|^2.
"""

from __future__ import annotations

import numpy as np

from .integrals import antisym


def _ranges(ncore, nval, nvirt):
    o = ncore + nval
    return np.arange(o), np.arange(o, o + nvirt)


def denominators(eps, ncore, nval, nvirt):
    """e_i + e_j - e_a - e_b as [i, j, a, b]."""
    O, V = _ranges(ncore, nval, nvirt)
    eo, ev = eps[O], eps[V]
    return (eo[:, None, None, None] + eo[None, :, None, None]
            - ev[None, None, :, None] - ev[None, None, None, :])


def t2_amplitudes(eps, B, ncore, nval, nvirt):
    """t[i, j, a, b] = <ab||ij> / (e_i + e_j - e_a - e_b)."""
    O, V = _ranges(ncore, nval, nvirt)
    vvoo = antisym(B, V, V, O, O)  # [a, b, i, j]
    return vvoo.transpose(2, 3, 0, 1) / denominators(eps, ncore, nval, nvirt)


def mp2_energy(eps, B, ncore, nval, nvirt, t2=None):
    """E_MP2 = 1/4 sum <ij||ab> t^{ab}_{ij} (real for Hermitian B^P)."""
    O, V = _ranges(ncore, nval, nvirt)
    if t2 is None:
        t2 = t2_amplitudes(eps, B, ncore, nval, nvirt)
    oovv = antisym(B, O, O, V, V)
    return 0.25 * np.sum(oovv * t2)


def density_vv(eps, B, ncore, nval, nvirt):
    """Eq. 15: D_ab = 1/2 sum_{cij} <ac||ij> <ij||bc> / (e^{ac}_{ij} e^{bc}_{ij})."""
    O, V = _ranges(ncore, nval, nvirt)
    den = denominators(eps, ncore, nval, nvirt)  # [i, j, a, c]
    vvoo = antisym(B, V, V, O, O)  # <ac||ij> as [a, c, i, j]
    oovv = antisym(B, O, O, V, V)  # <ij||bc> as [i, j, b, c]
    left = vvoo / den.transpose(2, 3, 0, 1)  # <ac||ij>/e^{ac}_{ij}
    right = oovv / den  # <ij||bc>/e^{bc}_{ij}
    return 0.5 * np.einsum("acij,ijbc->ab", left, right, optimize=True)
