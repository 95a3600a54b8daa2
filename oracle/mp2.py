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

* Second-order ground-state amplitudes (Rayleigh-Schrodinger with the
  Moller-Plesset partitioning H0 = sum_p e_p a_p^+ a_p of section
  "Relativistic Algebraic Diagrammatic Construction Method", intermediate
  normalisation, Phi_kl^cd = a_c^+ a_d^+ a_l a_k Phi_0), the ground-state
  pieces of the second-order transition moments:
    (e_k - e_c) s_kc = 1/2 sum_{lde} <cl||de> t^{de}_{kl}
                       - 1/2 sum_{lmd} <lm||kd> t^{cd}_{lm}
    (e_k + e_l - e_c - e_d) u^{cd}_{kl} = 1/2 sum_{ef} <cd||ef> t^{ef}_{kl}
                       + 1/2 sum_{mn} <mn||kl> t^{cd}_{mn}
                       + P(kl) P(cd) sum_{me} <mc||ek> t^{ed}_{ml}
  with P(kl) X = X - X(k <-> l).

Pins (tests/test_oracle_pins.py): E_MP2 equals the Rayleigh-Schrodinger
second-order energy of the determinant-space Hamiltonian; t2 is
antisymmetric in both index pairs; D is Hermitian, positive semidefinite
with trace 1/2 sum |t|^2, and its orientation is that of the exact
ground-state 1-RDM at lambda^2; t2, s and u are the lambda^1 and lambda^2
coefficients of the exact ground state's determinant amplitudes.
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


def second_order_singles(eps, B, ncore, nval, nvirt, t2=None):
    """s[k, c] = <Phi_k^c|Psi^(2)> for all occupied k, virtual c (module
    docstring)."""
    O, V = _ranges(ncore, nval, nvirt)
    if t2 is None:
        t2 = t2_amplitudes(eps, B, ncore, nval, nvirt)
    vovv = antisym(B, V, O, V, V)  # <cl||de> as [c, l, d, e]
    ooov = antisym(B, O, O, O, V)  # <lm||kd> as [l, m, k, d]
    rhs = (0.5 * np.einsum("clde,klde->kc", vovv, t2, optimize=True)
           - 0.5 * np.einsum("lmkd,lmcd->kc", ooov, t2, optimize=True))
    return rhs / (eps[O][:, None] - eps[V][None, :])


def second_order_doubles(eps, B, ncore, nval, nvirt, t2=None, rows=None):
    """u[k, l, c, d] = <Phi_kl^cd|Psi^(2)> (module docstring) for k in
    ``rows`` (a slice of the occupied spinors, default all) and all l."""
    O, V = _ranges(ncore, nval, nvirt)
    rows = slice(None) if rows is None else rows
    if t2 is None:
        t2 = t2_amplitudes(eps, B, ncore, nval, nvirt)
    Ok = O[rows]
    vvvv = antisym(B, V, V, V, V)  # <cd||ef>
    oooo = antisym(B, O, O, Ok, O)  # <mn||kl> as [m, n, k, l]
    ovvo = antisym(B, O, V, V, O)  # <mc||ek> as [m, c, e, k]
    pp = 0.5 * np.einsum("cdef,klef->klcd", vvvv, t2[rows], optimize=True)
    hh = 0.5 * np.einsum("mnkl,mncd->klcd", oooo, t2, optimize=True)
    # R^{cd}_{kl} = sum_me <mc||ek> t^{ed}_{ml}, with k in rows (R1) and with
    # l in rows (R2, for the k <-> l exchange)
    r1 = np.einsum("mcek,mled->klcd", ovvo[:, :, :, rows], t2, optimize=True)
    r2 = np.einsum("mcel,mked->klcd", ovvo, t2[:, rows], optimize=True)
    ring = r1 - r2 - r1.transpose(0, 1, 3, 2) + r2.transpose(0, 1, 3, 2)
    den = denominators(eps, ncore, nval, nvirt)[rows]
    return (pp + hh + ring) / den
